"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: a value the paper prints, a
closed form, an invariant, a library routine, a brute-force count or a finite difference.
"""
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _coarse_params(res=4, **kw):
    kw.setdefault("delta", 0.1)
    return oracle.Params(grid_shape=(res, res, res), mode=0, feat_dim=3, **kw)


# ------------------------------------------------------------------------------------------
# Low-density initialisation (Sec. 4.1 Eq. low_density_init, Supp. F)
# ------------------------------------------------------------------------------------------

def test_shift_b_closed_form_values():
    # Supp. F: with all raw densities 0, passing a distance s decays transmittance by 1 - alpha_init.
    for a_init, s in [(1e-6, 0.0625), (1e-2, 2 / 160), (0.3, 0.5)]:
        b = oracle.shift_from_alpha_init(a_init, s)
        sigma = math.log1p(math.exp(b))
        assert math.exp(-sigma * s) == pytest.approx(1 - a_init, rel=1e-12)
    # 32^3 coarse grid of the coarse-stage workload: b = -11.0429 (to 4 decimals).
    assert oracle.shift_from_alpha_init(1e-6, 0.0625) == pytest.approx(-11.0429, abs=5e-5)


def test_zero_grid_transmittance_over_box_is_alpha_init_power():
    # Axis-aligned ray through [-1,1]^3: 2 / delta samples, total distance 2 = 32 voxel sizes.
    s = 0.0625
    a_init = 0.3
    b = oracle.shift_from_alpha_init(a_init, s)
    P = _coarse_params(res=32, shift_b=b, delta=s / 2, bg=(0.0, 0.0, 0.0))
    dens = np.zeros((32, 32, 32))
    rgb = np.zeros((32, 32, 32, 3))
    res = oracle.render(P, dens, rgb, [[-4.0, 0.1, 0.2]], [[1.0, 0.0, 0.0]])
    assert res.n_samples[0] == 64
    assert res.tfinal[0] == pytest.approx((1 - a_init) ** (2 / s), rel=1e-10)


# ------------------------------------------------------------------------------------------
# Sampling (Eq. coarse_sample, Sec. 4.2 fine-stage sampling, Supp. A jitter)
# ------------------------------------------------------------------------------------------

def test_sample_count_matches_brute_force():
    o, d = synth.sphere_rays(300, seed=5, jitter_sd=0.4)
    P = _coarse_params(res=8, delta=0.0731)
    p = synth.jitter(300, 9)
    for i in range(300):
        rc, t0, t1, dn, n = oracle.ray_bounds(P, o[i], d[i], float(p[i]))
        assert rc == 0
        assert np.linalg.norm(dn) == pytest.approx(1.0, abs=1e-15)
        # brute force: every k with t0 + (k + p) delta < t1
        cnt = 0
        if t1 > t0:
            while t0 + (cnt + float(p[i])) * P.delta < t1:
                cnt += 1
        assert n == cnt
        if t1 > t0:
            # the clip points lie on the box surface
            for t in (t0, t1):
                x = o[i].astype(np.float64) + t * dn
                assert np.max(np.abs(x)) == pytest.approx(1.0, abs=1e-12)
            inside = o[i].astype(np.float64) + 0.5 * (t0 + t1) * dn
            assert np.all(np.abs(inside) < 1.0)


def test_ray_missing_box_and_zero_direction():
    P = _coarse_params(res=8)
    rc, t0, t1, dn, n = oracle.ray_bounds(P, [0.0, 3.0, 0.0], [1.0, 0.0, 0.0])
    assert rc == 0 and n == 0
    rc, *_ = oracle.ray_bounds(P, [0.0, 0.0, 0.0], [0.0, 0.0, 0.0])
    assert rc == -1
    # origin inside the box: t_enter is t_near (Sec. 4.2)
    rc, t0, t1, dn, n = oracle.ray_bounds(P, [0.2, 0.1, 0.0], [0.0, 0.0, 2.0])
    assert t0 == 0.0 and t1 == pytest.approx(1.0)


# ------------------------------------------------------------------------------------------
# Trilinear interpolation (Sec. 3 Eq. interp)
# ------------------------------------------------------------------------------------------

def _lattice(res, lo=-1.0, hi=1.0):
    ax = np.linspace(lo, hi, res)
    return np.meshgrid(ax, ax, ax, indexing="ij")


def test_trilinear_reproduces_multilinear_fields_per_channel():
    res = 7
    X, Y, Z = _lattice(res)
    # three channels with distinct multilinear fields: a transposed axis or channel fails
    grid = np.stack([1.5 * X - 0.25 * Y + 3.0 * Z + 0.5,
                     X * Y * Z - 2.0 * X * Z + 0.3,
                     -0.7 * Y + 0.2 * X * Y + 4.0], axis=-1)
    P = oracle.Params(grid_shape=(res, res, res))
    g = np.random.default_rng(0)
    for _ in range(200):
        x = g.uniform(-1, 1, size=3)
        cell = np.floor((x + 1) / 2 * (res - 1))
        # multilinear terms are reproduced only within one cell; use the cell's local field
        lo = -1 + cell * 2 / (res - 1)
        hi = lo + 2 / (res - 1)
        f = (x - lo) / (hi - lo)
        # exact trilinear value from the eight corner values, computed independently
        exp = np.zeros(3)
        for c in range(8):
            bx, by, bz = (c >> 2) & 1, (c >> 1) & 1, c & 1
            idx = tuple(int(v) for v in cell + np.array([bx, by, bz]))
            w = (f[0] if bx else 1 - f[0]) * (f[1] if by else 1 - f[1]) * (f[2] if bz else 1 - f[2])
            exp += w * grid[idx]
        out = oracle.interp(P, grid, x)
        np.testing.assert_allclose(out, exp, rtol=1e-13, atol=1e-13)
        # affine channel: exact everywhere
        assert out[0] == pytest.approx(1.5 * x[0] - 0.25 * x[1] + 3.0 * x[2] + 0.5, abs=1e-12)


def test_trilinear_hits_lattice_values():
    res = 5
    grid = np.random.default_rng(1).normal(size=(res, res, res))
    P = oracle.Params(grid_shape=(res, res, res))
    ax = np.linspace(-1, 1, res)
    for i, j, k in [(0, 0, 0), (4, 4, 4), (1, 3, 2), (4, 0, 2)]:
        assert oracle.interp(P, grid, [ax[i], ax[j], ax[k]])[0] == pytest.approx(grid[i, j, k], abs=1e-13)


# ------------------------------------------------------------------------------------------
# Post-activation worked examples (Supp. G)
# ------------------------------------------------------------------------------------------

EPS, DELTA_RENDER = 1e-4, 0.5


def _a_upper(c, Dl, eps=EPS, delta=DELTA_RENDER):
    # Supp. G.1, Eq. 1d_a_upper_bound, branch delta < 1
    return (math.log(2 ** (1 / delta) - 1) * (c + Dl) / Dl
            - math.log(1 / eps ** (1 / delta) - 1) * c / Dl)


def _b_of_a(a, c, delta=DELTA_RENDER):
    # Supp. G.1, Eq. 1d_b_linear_to_a
    return a * (c - 1) / c + math.log(2 ** (1 / delta) - 1) / c


def _golden_rows(kind):
    rows = []
    with open(os.path.join(GOLDEN, "post_activation_examples.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].split()
            if line and line[0] == kind:
                rows.append([float(v) for v in line[1:]])
    return rows


def test_1d_examples_printed_values_and_oracle_alpha():
    rows = _golden_rows("1d")
    assert len(rows) == 6
    P = oracle.Params(grid_shape=(2, 2, 2), xyz_min=(0, 0, 0), xyz_max=(1, 1, 1), shift_b=0.0)
    for c, Dl, a_pr, b_pr in rows:
        a = _a_upper(c, Dl)
        b = _b_of_a(a, c)
        assert abs(a - a_pr) <= 0.05 + 1e-9 and abs(b - b_pr) <= 0.05 + 1e-9
        V = np.zeros((2, 2, 2))
        V[0], V[1] = a, b
        S = lambda x: oracle.alpha_at(P, V, [x, 0.37, 0.81], DELTA_RENDER)
        assert S(c) == pytest.approx(0.5, abs=1e-9)
        # the upper bound makes the first constraint (Eq. 1d_proof_c1) tight, the second hold
        assert 1 - S(c + Dl) == pytest.approx(EPS, rel=1e-6)
        assert S(c - Dl) <= EPS * (1 + 1e-9)
        # monotone step: far to the left is free, far to the right is occupied
        if 0 < c < 1:
            assert S(0.0) < EPS and 1 - S(1.0) < EPS


def test_2d_examples_bilinear_boundary():
    rows = _golden_rows("2d")
    assert len(rows) == 4
    P = oracle.Params(grid_shape=(2, 2, 2), xyz_min=(0, 0, 0), xyz_max=(1, 1, 1), shift_b=0.0)
    for c0, c1, Dl, tl, tr, bl, br in rows:
        a0, a1 = _a_upper(c0, Dl), _a_upper(c1, Dl)
        b0, b1 = _b_of_a(a0, c0), _b_of_a(a1, c1)
        for mine, printed in [(a0, tl), (b0, tr), (a1, bl), (b1, br)]:
            assert abs(mine - printed) <= 0.05 + 1e-9
        # grid axis 0 = x (left/right), axis 1 = t (top/bottom), axis 2 duplicated
        V = np.zeros((2, 2, 2))
        V[0, 0, :], V[1, 0, :], V[0, 1, :], V[1, 1, :] = a0, b0, a1, b1
        for t in np.linspace(0, 1, 9):
            c = c0 + (c1 - c0) * t
            S = lambda x: oracle.alpha_at(P, V, [x, t, 0.4], DELTA_RENDER)
            assert S(c) == pytest.approx(0.5, abs=1e-9)
            assert 1 - S(c + Dl) == pytest.approx(EPS, rel=1e-6)
            assert S(c - Dl) <= EPS * (1 + 1e-9)


# ------------------------------------------------------------------------------------------
# Volume-rendering quadrature (Sec. 2 Eq. volume_rendering)
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("x0,b", [(0.3, 0.0), (-2.0, 1.5), (4.0, -3.0)])
def test_constant_grid_closed_form(x0, b):
    res = 6
    delta = 0.0917
    c = np.array([0.2, 0.55, 0.9])
    bg = np.array([0.1, 0.7, 0.3])
    P = _coarse_params(res=res, shift_b=b, delta=delta, bg=tuple(bg))
    dens = np.full((res,) * 3, x0)
    rgb = np.broadcast_to(c, (res, res, res, 3)).copy()
    o, d = synth.sphere_rays(64, seed=3, jitter_sd=0.3)
    p = synth.jitter(64, 4)
    r = oracle.render(P, dens, rgb, o, d, jitter=p)
    alpha = 1 - (1 + math.exp(x0 + b)) ** (-delta)   # Supp. G, Eq. supp_post_activation
    for i in range(64):
        K = r.n_samples[i]
        T = (1 - alpha) ** K
        np.testing.assert_allclose(r.rgb[i], c * (1 - T) + bg * T, rtol=1e-12, atol=1e-14)
        assert r.tfinal[i] == pytest.approx(T, rel=1e-12, abs=1e-300)


def test_weights_plus_final_transmittance_is_one():
    res = 9
    P = _coarse_params(res=res, shift_b=0.5, delta=0.05, bg=(1.0, 1.0, 1.0))
    dens = synth.normal_grid((res,) * 3, 1, 2.0, 11).astype(np.float64)
    ones = np.ones((res, res, res, 3))
    o, d = synth.sphere_rays(50, seed=12, jitter_sd=0.2)
    r = oracle.render(P, dens, ones, o, d)
    np.testing.assert_allclose(r.rgb, 1.0, atol=1e-14)            # sum w + T_K = 1
    P0 = _coarse_params(res=res, shift_b=0.5, delta=0.05, bg=(0.0, 0.0, 0.0))
    r0 = oracle.render(P0, dens, ones, o, d)
    np.testing.assert_allclose(r0.rgb[:, 0], 1.0 - r0.tfinal, atol=1e-14)


def test_empty_space_gives_background():
    res = 5
    P = _coarse_params(res=res, shift_b=0.0, delta=0.05, bg=(0.25, 0.5, 0.75))
    dens = np.full((res,) * 3, -60.0)
    rgb = np.random.default_rng(2).uniform(size=(res, res, res, 3))
    o, d = synth.sphere_rays(20, seed=13)
    r = oracle.render(P, dens, rgb, o, d)
    np.testing.assert_allclose(r.rgb, np.broadcast_to([0.25, 0.5, 0.75], (20, 3)), atol=1e-20)


def test_compositing_is_associative_over_a_split():
    """Render [t_enter, t_mid) and [t_mid, t_exit) separately and fold them with the 'over'
    operator: C = C1 + T1 C2, T = T1 T2 (Eq. volume_rendering is a product / prefix sum)."""
    res = 8
    delta = 0.04
    bg = np.array([0.3, 0.6, 0.9])
    dens = synth.normal_grid((res,) * 3, 1, 1.5, 21).astype(np.float64)
    rgb = np.random.default_rng(22).uniform(size=(res, res, res, 3))
    o = np.array([[-3.0, 0.13, -0.21]])
    d = np.array([[1.0, 0.05, 0.02]])
    p = 0.37
    Pfull = _coarse_params(res=res, shift_b=0.2, delta=delta, bg=tuple(bg))
    full = oracle.render(Pfull, dens, rgb, o, d, jitter=[p])
    t0 = full.t_enter[0]
    m = 17
    t_mid = t0 + m * delta
    P1 = _coarse_params(res=res, shift_b=0.2, delta=delta, bg=(0, 0, 0), t_far=t_mid)
    P2 = _coarse_params(res=res, shift_b=0.2, delta=delta, bg=tuple(bg), t_near=t_mid)
    r1 = oracle.render(P1, dens, rgb, o, d, jitter=[p])
    r2 = oracle.render(P2, dens, rgb, o, d, jitter=[p])
    assert r1.n_samples[0] == m and r1.n_samples[0] + r2.n_samples[0] == full.n_samples[0]
    np.testing.assert_allclose(r1.rgb[0] + r1.tfinal[0] * r2.rgb[0], full.rgb[0], rtol=1e-12)
    assert r1.tfinal[0] * r2.tfinal[0] == pytest.approx(full.tfinal[0], rel=1e-12)


def test_loss_is_mean_over_rays_of_channel_sum():
    res = 5
    P = _coarse_params(res=res, shift_b=0.0, delta=0.1)
    dens = synth.normal_grid((res,) * 3, 1, 1.0, 31).astype(np.float64)
    rgb = synth.normal_grid((res,) * 3, 3, 1.0, 32).astype(np.float64)
    o, d = synth.sphere_rays(10, seed=33)
    tgt = synth.targets(10, 34)
    r = oracle.render(P, dens, rgb, o, d, target=tgt)
    assert r.loss == pytest.approx(np.sum((r.rgb - tgt) ** 2) / 10, rel=1e-13)


# ------------------------------------------------------------------------------------------
# Colour model (Sec. 4.2 Eq. fine_queries, Supp. A)
# ------------------------------------------------------------------------------------------

def _np_mlp(mlp, e):
    relu = lambda v: np.maximum(v, 0)
    h1 = relu(e @ mlp["w1"] + mlp["b1"])
    h2 = relu(h1 @ mlp["w2"] + mlp["b2"])
    return 1 / (1 + np.exp(-(h2 @ mlp["w3"] + mlp["b3"])))


def test_mlp_matches_matmul_chain():
    mlp = {k: v.astype(np.float64) for k, v in synth.mlp_weights(39, 128, 3, seed=40).items()}
    mlp["b3"] = np.random.default_rng(41).normal(size=3)
    e = np.random.default_rng(42).normal(size=(37, 39))
    P = oracle.Params(grid_shape=(2, 2, 2), mode=1, feat_dim=12, n_freq=4, hidden=128)
    np.testing.assert_allclose(oracle.mlp_forward(P, mlp, e), _np_mlp(mlp, e), rtol=1e-12)


@pytest.mark.parametrize("col", [0, 11, 12, 14, 15, 15 + 4 * 1 + 2, 15 + 12, 15 + 12 + 4 * 2 + 3])
def test_fine_mlp_input_layout(col):
    """Route one input column straight to the red output and compare with its closed form.
    Columns: features 0..11, d 12..14, sin(2^k d_c) at 15 + 4c + k, cos(2^k d_c) at 27 + 4c + k."""
    C, F, H = 12, 4, 8
    I = C + 3 + 6 * F
    res = 4
    g = np.random.default_rng(50 + col)
    feat_val = g.uniform(-1, 1, size=C)
    feat = np.broadcast_to(feat_val, (res, res, res, C)).copy()
    x0, b, delta = 0.7, -0.2, 0.08
    dens = np.full((res,) * 3, x0)
    w1 = np.zeros((I, H)); w1[col, 0], w1[col, 1] = 1.0, -1.0
    w2 = np.zeros((H, H)); w2[0, 0] = w2[1, 1] = 1.0
    w3 = np.zeros((H, 3)); w3[0, 0], w3[1, 0] = 1.0, -1.0
    mlp = dict(w1=w1, b1=np.zeros(H), w2=w2, b2=np.zeros(H), w3=w3, b3=np.zeros(3))
    P = oracle.Params(grid_shape=(res,) * 3, mode=1, feat_dim=C, n_freq=F, hidden=H, shift_b=b,
                      delta=delta, bg=(0.0, 0.0, 0.0))
    dvec = np.array([0.3, -0.5, 0.8])
    dn = dvec / np.linalg.norm(dvec)
    o = -3.5 * dn + np.array([0.05, 0.02, -0.04])
    r = oracle.render(P, dens, feat, [o], [dvec], mlp=mlp)
    if col < C:
        v = feat_val[col]
    elif col < C + 3:
        v = dn[col - C]
    elif col < C + 3 + 3 * F:
        c, k = divmod(col - C - 3, F)
        v = math.sin(2 ** k * dn[c])
    else:
        c, k = divmod(col - C - 3 - 3 * F, F)
        v = math.cos(2 ** k * dn[c])
    T = r.tfinal[0]
    assert r.n_samples[0] > 10
    sig = lambda z: 1 / (1 + math.exp(-z))
    np.testing.assert_allclose(r.rgb[0], (1 - T) * np.array([sig(v), 0.5, 0.5]), rtol=1e-12)


# ------------------------------------------------------------------------------------------
# Gradients: central finite differences on tiny problems
# ------------------------------------------------------------------------------------------

def _tiny_problem(mode, rgb_act=0, seed=60):
    res, C, F, H = 4, (2 if mode == 1 else 3), 2, 8
    g = np.random.default_rng(seed)
    P = oracle.Params(grid_shape=(res,) * 3, mode=mode, rgb_act=rgb_act, feat_dim=C, n_freq=F,
                      hidden=H, shift_b=0.4, delta=0.21, bg=(0.2, 0.4, 0.6))
    dens = g.normal(scale=1.5, size=(res,) * 3)
    cg = g.normal(scale=0.8, size=(res, res, res, C))
    o, d = synth.sphere_rays(3, seed=seed + 1, radius=3.0, jitter_sd=0.05)
    o = o.astype(np.float64); d = d.astype(np.float64)
    p = g.uniform(size=3)
    mlp = None
    if mode == 1:
        mlp = {k: v.astype(np.float64) for k, v in synth.mlp_weights(C + 3 + 6 * F, H, 3, seed + 2).items()}
        mlp["b3"] = g.normal(scale=0.3, size=3)
    gC = g.normal(size=(3, 3))
    gT = g.normal(size=3)
    return P, dens, cg, o, d, p, mlp, gC, gT


def _objective(P, dens, cg, o, d, p, mlp, gC, gT):
    r = oracle.render(P, dens, cg, o, d, jitter=p, mlp=mlp)
    return float(np.sum(gC * r.rgb) + np.sum(gT * r.tfinal))


@pytest.mark.parametrize("mode,rgb_act", [(0, 0), (0, 1), (1, 0)])
def test_gradients_match_central_differences(mode, rgb_act):
    P, dens, cg, o, d, p, mlp, gC, gT = _tiny_problem(mode, rgb_act)
    r = oracle.render(P, dens, cg, o, d, jitter=p, mlp=mlp, grad_rgb=gC, grad_tfinal=gT)
    assert r.n_samples.min() > 5
    params = {"density": dens, "cgrid": cg}
    if mlp:
        params.update(mlp)
    h = 1e-6
    for name, arr in params.items():
        ana = r.grads[name]
        num = np.zeros_like(arr)
        flat = arr.reshape(-1)
        for i in range(flat.size):
            old = flat[i]
            flat[i] = old + h
            fp = _objective(P, dens, cg, o, d, p, mlp, gC, gT)
            flat[i] = old - h
            fm = _objective(P, dens, cg, o, d, p, mlp, gC, gT)
            flat[i] = old
            num.reshape(-1)[i] = (fp - fm) / (2 * h)
        scale = max(np.abs(num).max(), 1e-3)
        np.testing.assert_allclose(ana, num, rtol=0, atol=2e-7 * scale, err_msg=name)
        assert np.abs(ana).max() > 0, name


def test_skipped_samples_get_no_gradient():
    # tau_f above every alpha: nothing is kept, colour is the background, gradients vanish.
    P, dens, cg, o, d, p, mlp, gC, gT = _tiny_problem(0)
    P.tau_f = 2.0
    r = oracle.render(P, dens, cg, o, d, jitter=p, grad_rgb=gC, grad_tfinal=gT)
    np.testing.assert_allclose(r.rgb, np.broadcast_to(P.bg, (3, 3)))
    assert np.all(r.grads["density"] == 0) and np.all(r.grads["cgrid"] == 0)


# ------------------------------------------------------------------------------------------
# Adam (Kingma & Ba) and the decay of Supp. A
# ------------------------------------------------------------------------------------------

def test_adam_constant_gradient_closed_form():
    # With a constant gradient the bias-corrected moments are exactly g and g^2 at every step,
    # so each step moves every parameter by -lr * g / (|g| + eps).
    g = np.random.default_rng(70).normal(size=1000)
    p = np.random.default_rng(71).normal(size=1000)
    p0 = p.copy()
    m = np.zeros(1000); v = np.zeros(1000)
    lr, eps = 0.1, 1e-8
    for t in range(1, 6):
        grad = g.copy()
        oracle.adam(p, grad, m, v, lr, t, eps=eps)
        assert np.all(grad == 0)                                  # zero_grad
        np.testing.assert_allclose(p, p0 - t * lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-14)


def test_lr_decay_reaches_one_tenth_at_20k():
    assert oracle.lr_decay(0.1, 0) == pytest.approx(0.1)
    assert oracle.lr_decay(0.1, 20000) == pytest.approx(0.01, rel=1e-14)
    assert oracle.lr_decay(1e-3, 10000) == pytest.approx(1e-3 / math.sqrt(10), rel=1e-14)


def test_adam_lr_scale_prior2():
    # Sec. 4.1 Prior 2: a per-voxel scale n_j / n_max on the learning rate; scale 0 freezes.
    n = 64
    g = np.random.default_rng(72).normal(size=n)
    scale = np.linspace(0, 1, n)
    p = np.zeros(n); m = np.zeros(n); v = np.zeros(n)
    oracle.adam(p, g.copy(), m, v, 0.1, 1, lr_scale=scale)
    np.testing.assert_allclose(p, -0.1 * scale * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)
