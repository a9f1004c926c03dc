"""Pins of the oracle's touched-lattice-point marks (the exact count behind the algorithmic bytes
of a step): the density grid's points read by every sample outside the known free space, the colour
/ feature grid's points read by every kept sample -- the 8 corners of each such sample's cell."""
import math

import numpy as np

import oracle
import synth


def test_axis_aligned_ray_closed_form():
    """4^3 lattice on [-1, 1]^3 (spacing 2/3), one ray along +x at y = 0.1, z = -0.2, delta = 0.1:
    u_y = 1.65 and u_z = 1.2 put every sample in row j0 = 1, k0 = 1; the 20 samples sit at
    u_x = 0.075 + 0.15 k, k = 0..19, in cells i0 = 0, 1, 2 -> density marks i = 0..3, j, k in {1, 2}.
    Raw density 5 for i <= 1 and -20 for i >= 2 with tau_f = 1e-3: samples in cell 0 are kept, in
    cell 1 those with 5 - 25 f above softplus^-1(0.01) (f <= 0.38), none in cell 2 -> colour marks
    i = 0..2."""
    dens = np.full((4, 4, 4), 5.0)
    dens[2:] = -20.0
    P = oracle.Params(grid_shape=(4, 4, 4), delta=0.1, tau_f=1e-3, mode=0, feat_dim=3)
    r = oracle.render(P, dens, np.zeros((4, 4, 4, 3)), [[-3.0, 0.1, -0.2]], [[1.0, 0.0, 0.0]], touched=True)
    assert r.n_samples[0] == 20
    exp_d = np.zeros((4, 4, 4), bool)
    exp_d[0:4, 1:3, 1:3] = True
    exp_c = np.zeros((4, 4, 4), bool)
    exp_c[0:3, 1:3, 1:3] = True
    assert np.array_equal(r.touched["density"], exp_d)
    assert np.array_equal(r.touched["cgrid"], exp_c)
    # the threshold on f used above: softplus(5 - 25 f) * 0.1 >= 1e-3
    f_max = (5.0 - math.log(math.expm1(0.01))) / 25.0
    assert 0.375 < f_max < 0.39


def test_marks_equal_the_corner_sets_of_the_samples():
    """Random rays, nothing skipped: both marks are the union of the 8 corners of every sample's
    cell, re-derived here from the samples' positions with numpy floor / clip."""
    case = synth.coarse_case(seed=3, n_rays=60, res=9)
    P = oracle.Params(grid_shape=(9, 9, 9), delta=0.07, mode=0, feat_dim=3, tau_f=0.0)
    jit = np.random.default_rng(4).uniform(size=60)
    r = oracle.render(P, case["density"], case["rgb"], case["rays_o"], case["rays_d"], jitter=jit, touched=True)
    exp = np.zeros((9, 9, 9), bool)
    for i in range(60):
        _, t0, t1, dn, n = oracle.ray_bounds(P, case["rays_o"][i], case["rays_d"][i], jit[i])
        for k in range(n):
            x = case["rays_o"][i] + (t0 + (k + jit[i]) * 0.07) * dn
            c0 = np.clip(np.floor((x + 1.0) / 2.0 * 8), 0, 7).astype(int)
            exp[c0[0]:c0[0] + 2, c0[1]:c0[1] + 2, c0[2]:c0[2] + 2] = True
    assert exp.sum() > 100
    assert np.array_equal(r.touched["density"], exp)
    assert np.array_equal(r.touched["cgrid"], exp)


def test_known_free_samples_mark_no_fine_point():
    """Fine stage with a coarse grid that is free everywhere: no sample queries the fine grids."""
    res = 6
    P = oracle.Params(grid_shape=(res,) * 3, mode=1, feat_dim=12, delta=0.1)
    fs = oracle.FreeSpace(density=np.full((4, 4, 4), -30.0), shift_b=0.0, delta=0.1, tau=1e-3)
    mlp = synth.mlp_weights(39, 128, 3, seed=1)
    o, d = synth.sphere_rays(20, seed=2)
    r = oracle.render(P, np.zeros((res,) * 3), np.zeros((res,) * 3 + (12,)), o, d, mlp=mlp, freespace=fs,
                      touched=True)
    assert r.n_samples.sum() > 0
    assert not r.touched["density"].any() and not r.touched["cgrid"].any()
