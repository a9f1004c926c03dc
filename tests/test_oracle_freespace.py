"""Pins of the oracle's known-free-space test and fine-box allocation (Sec. 4.2): the skip rule is
checked against the same render on an explicit list of the samples that survive it, and the box
against planted cases and an enclosure property on random points."""
import numpy as np

import oracle
import synth


def _coarse(res=12, seed=70, r_in=0.35, r_out=0.6, v_in=8.0):
    """Coarse raw density: known free (-20) except a ball of high density and a shell of values
    that straddle the threshold."""
    g = np.linspace(-1.0, 1.0, res)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    r = np.sqrt((X - 0.2) ** 2 + (Y + 0.1) ** 2 + (Z - 0.05) ** 2)
    v = np.where(r < r_in, v_in, -20.0)
    shell = (r >= r_in) & (r < r_out)
    v[shell] = synth.normal_grid((res,) * 3, 1, 3.0, seed)[shell] - 6.0
    return v


def _fine_case(res=20, R=64, seed=71):
    dens = synth.normal_grid((res,) * 3, 1, 1.0, seed) + 0.5
    feat = synth.normal_grid((res,) * 3, 12, 0.5, seed + 1)
    mlp = synth.mlp_weights(39, 16, 3, seed + 2)
    o, d = synth.sphere_rays(R, seed + 3, jitter_sd=0.05)
    jit = synth.jitter(R, seed + 4)
    P = oracle.Params(grid_shape=(res,) * 3, shift_b=-2.0, delta=2.0 / res / 2, bg=(0.2, 0.5, 0.8), mode=1,
                      feat_dim=12, n_freq=4, hidden=16)
    return P, dens, feat, mlp, o, d, jit


def _fs(tau=1e-3):
    res_c = 12
    b_c = oracle.shift_from_alpha_init(1e-6, 2.0 / res_c)
    return oracle.FreeSpace(density=_coarse(res_c), shift_b=b_c, delta=2.0 / res_c / 2, tau=tau)


def test_tau_c_zero_changes_nothing():
    P, dens, feat, mlp, o, d, jit = _fine_case()
    gC = np.random.default_rng(5).normal(size=(o.shape[0], 3))
    a = oracle.render(P, dens, feat, o, d, jitter=jit, mlp=mlp, grad_rgb=gC)
    b = oracle.render(P, dens, feat, o, d, jitter=jit, mlp=mlp, grad_rgb=gC, freespace=_fs(tau=0.0))
    np.testing.assert_array_equal(a.rgb, b.rgb)
    for k in a.grads:   # grid gradients are atomic sums across threads: equal up to their order
        np.testing.assert_allclose(a.grads[k], b.grads[k], rtol=0, atol=1e-12 * np.abs(a.grads[k]).max())


def test_skipped_points_equal_a_render_without_them():
    """Colours, transmittance and every gradient of the free-space render equal, ray by ray, those of
    a render on the explicit list of the uniform samples whose coarse alpha is >= tau_c (a skipped
    point contributes alpha 0, so removing it leaves the quadrature unchanged)."""
    P, dens, feat, mlp, o, d, jit = _fine_case()
    fs = _fs()
    R = o.shape[0]
    gC = np.random.default_rng(6).normal(size=(R, 3))
    full = oracle.render(P, dens, feat, o, d, jitter=jit, mlp=mlp, grad_rgb=gC, freespace=fs)
    skipped_total = kept_total = 0
    acc = {k: np.zeros_like(v) for k, v in full.grads.items()}
    for r in range(R):
        _, t0, t1, dn, n = oracle.ray_bounds(P, o[r], d[r], float(jit[r]))
        t = t0 + (np.arange(n) + jit[r]) * P.delta
        keep = np.array([oracle.coarse_alpha(fs, o[r] + tk * dn) >= fs.tau for tk in t], bool)
        skipped_total += int((~keep).sum())
        kept_total += int(keep.sum())
        if keep.sum() == 0:
            np.testing.assert_allclose(full.rgb[r], P.bg, rtol=0, atol=1e-15)
            continue
        one = oracle.render(P, dens, feat, o[r:r + 1], d[r:r + 1], mlp=mlp, grad_rgb=gC[r:r + 1],
                            explicit_t=t[keep][None], explicit_dt=np.full((1, int(keep.sum())), P.delta))
        np.testing.assert_allclose(full.rgb[r], one.rgb[0], rtol=0, atol=1e-12)
        np.testing.assert_allclose(full.tfinal[r], one.tfinal[0], rtol=0, atol=1e-12)
        for k in acc:
            acc[k] += one.grads[k]
    assert skipped_total > 100 and kept_total > 60            # both branches exercised
    for k in acc:
        scale = max(np.abs(acc[k]).max(), 1e-30)
        np.testing.assert_allclose(full.grads[k], acc[k], rtol=0, atol=1e-11 * scale, err_msg=k)


def test_unknown_bbox_planted_point_and_clamping():
    res = 9
    v = np.full((res,) * 3, -30.0)
    fs = oracle.FreeSpace(density=v, shift_b=0.0, delta=0.1, tau=1e-3)
    assert oracle.unknown_bbox(fs)[0] == 0                     # everything known free
    v[4, 2, 7] = 10.0
    n, lo, hi = oracle.unknown_bbox(oracle.FreeSpace(density=v, shift_b=0.0, delta=0.1, tau=1e-3))
    assert n == 1 and lo == (3, 1, 6) and hi == (5, 3, 8)
    v[0, 8, 8] = 10.0                                          # on the faces: clamped
    n, lo, hi = oracle.unknown_bbox(oracle.FreeSpace(density=v, shift_b=0.0, delta=0.1, tau=1e-3))
    assert n == 2 and lo == (0, 1, 6) and hi == (5, 8, 8)


def test_unknown_bbox_encloses_the_unknown_space():
    """Every point whose coarse alpha is >= tau_c lies inside the box; every unclamped face of the
    box is one cell beyond an unknown lattice point (tight at lattice resolution)."""
    fs = _fs()
    n, lo, hi = oracle.unknown_bbox(fs)
    res = fs.density.shape[0]
    assert n > 0 and all(0 < lo[a] < hi[a] < res - 1 for a in range(3))
    h = 2.0 / (res - 1)
    bmin = np.array([-1.0 + lo[a] * h for a in range(3)])
    bmax = np.array([-1.0 + hi[a] * h for a in range(3)])
    x = np.random.default_rng(9).uniform(-1.0, 1.0, size=(20000, 3))
    inside = 0
    for p in x:
        if oracle.coarse_alpha(fs, p) >= fs.tau:
            assert np.all(p >= bmin - 1e-12) and np.all(p <= bmax + 1e-12)
            inside += 1
    assert inside > 100
    alpha_lat = -np.expm1(-np.logaddexp(0.0, fs.density + fs.shift_b) * fs.delta)
    unknown = alpha_lat >= fs.tau
    for a in range(3):
        idx = np.nonzero(unknown.any(axis=tuple(b for b in range(3) if b != a)))[0]
        assert idx.min() - 1 == lo[a] and idx.max() + 1 == hi[a]
