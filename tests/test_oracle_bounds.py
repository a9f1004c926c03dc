"""Pins of the oracle's running error bound (og_bound in oracle/dvgo_oracle.c, test
infrastructure): the per-element tolerance the GPU gradient tests use for the BF16 tensor-core
path and for the FP32 colour-error model.

What fixes the bound is first-order error analysis, independent of the oracle's code:

* the worst case, over relative perturbations |eps_r| <= u of every rounded operand, of a
  computed quantity y is u * sum_r |dy/deps_r| to first order; that sum is evaluated here with
  torch float64 autograd on a separately written MLP chain with a perturbation factor (1 + eps_r)
  at every rounding point (X, H1, H2 forward; dL/do, dZ2, dZ1 backward).  The bound must never
  be below it (validity: a dropped term fails it); where every path of the chain has the same sign
  the triangle inequality it applies layer by layer is an equality, and the bound must equal that
  worst case (a doubled or misrouted term fails it);
* a ReLU whose input lies inside its rounding band may flip: the bound must cover the flip;
* with u = 0 the bound is exactly 0;
* on a whole render, perturbing the feature grid by a relative u' moves every gradient by no more
  than the bound computed for input errors of that size.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

U_BF16 = 2.0 ** -8


def _mlp(I, H, seed, scale=1.0):
    g = np.random.default_rng(seed)
    return {"w1": g.normal(scale=scale / np.sqrt(I), size=(I, H)), "b1": g.normal(scale=0.1, size=H),
            "w2": g.normal(scale=scale / np.sqrt(H), size=(H, H)), "b2": g.normal(scale=0.1, size=H),
            "w3": g.normal(scale=1.0 / np.sqrt(H), size=(H, 3)), "b3": g.normal(scale=0.3, size=3)}


def _first_order_worst(mlp, e, dc, u):
    """u * sum_r |dy/deps_r| for every output y of one sample, with the masks of the unperturbed
    chain (first order), by autograd through a chain written here with (1 + eps) factors."""
    t = {k: torch.as_tensor(v, dtype=torch.float64) for k, v in mlp.items()}
    x0 = torch.as_tensor(e, dtype=torch.float64)
    dct = torch.as_tensor(dc, dtype=torch.float64)
    I, H = mlp["w1"].shape
    z1 = x0 @ t["w1"] + t["b1"]
    z2 = torch.relu(z1) @ t["w2"] + t["b2"]
    m1, m2 = (z1 > 0).double(), (z2 > 0).double()
    sizes = [I, H, H, 3, H, H]

    def chain(eps):
        ex, eh1, eh2, edo, edz2, edz1 = torch.split(eps, sizes)
        x = x0 * (1 + ex)
        h1 = (x @ t["w1"] + t["b1"]) * m1 * (1 + eh1)
        h2 = (h1 @ t["w2"] + t["b2"]) * m2 * (1 + eh2)
        c = torch.sigmoid(h2 @ t["w3"] + t["b3"])
        dout0 = dct * c * (1 - c)
        dout = dout0 * (1 + edo)               # the operand; db3 sums dL/do unrounded
        dz2 = (dout @ t["w3"].T) * m2 * (1 + edz2)
        dz1 = (dz2 @ t["w2"].T) * m1 * (1 + edz1)
        de = dz1 @ t["w1"].T
        return torch.cat([c, de, torch.outer(x, dz1).reshape(-1), dz1, torch.outer(h1, dz2).reshape(-1), dz2,
                          torch.outer(h2, dout).reshape(-1), dout0])

    J = torch.autograd.functional.jacobian(chain, torch.zeros(sum(sizes), dtype=torch.float64))
    worst = (u * J.abs().sum(1)).numpy()
    y0 = chain(torch.zeros(sum(sizes), dtype=torch.float64)).detach().numpy()
    return worst, y0, (z1.numpy(), z2.numpy())


def _split(v, I, H):
    out, o = {}, 0
    for k, n in (("c", 3), ("de", I), ("w1", I * H), ("b1", H), ("w2", H * H), ("b2", H), ("w3", H * 3), ("b3", 3)):
        out[k] = v[o:o + n]
        o += n
    return out


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_sample_bound_is_the_first_order_worst_case_up_to_the_triangle_inequality(seed):
    C_, F, H = 4, 2, 16
    P = oracle.Params(grid_shape=(2, 2, 2), mode=1, feat_dim=C_, n_freq=F, hidden=H)
    I = P.in_dim
    mlp = _mlp(I, H, seed)
    g = np.random.default_rng(100 + seed)
    e = g.normal(size=I)
    dc = g.normal(size=3)
    c, ec, de, ede, gw, eb = oracle.mlp_sample_bound(P, mlp, e, np.zeros(I), dc, 0.0, U_BF16, 0.0)
    worst, y0, (z1, z2) = _first_order_worst(mlp, e, dc, U_BF16)
    W, Y = _split(worst, I, H), _split(y0, I, H)
    # the oracle's sample values are the chain's
    np.testing.assert_allclose(c, Y["c"], rtol=1e-13)
    np.testing.assert_allclose(de, Y["de"], rtol=1e-11, atol=1e-14)
    for k in ("w1", "b1", "w2", "b2", "w3", "b3"):
        np.testing.assert_allclose(gw[k].reshape(-1), Y[k], rtol=1e-11, atol=1e-14)
    got = {"c": ec, "de": ede} | {k: eb[k].reshape(-1) for k in ("w1", "b1", "w2", "b2", "w3", "b3")}
    ratios = []
    for k, b in got.items():
        w = W[k]
        assert np.all(b >= w * (1 - 1e-9) - 1e-300), (k, np.min(b - w))       # validity
        nz = w > 1e-12 * np.abs(w).max()
        ratios.append(b[nz] / w[nz])
    r = np.concatenate(ratios)
    assert np.median(r) < 20.0, np.median(r)         # only the triangle inequality's slack


def test_sample_bound_equals_the_first_order_worst_case_without_cancellation():
    """Positive weights, inputs and upstream gradient, and an output logit below 0 (so that
    1 - 2c > 0): every path of the chain has the same sign, the triangle inequality is an equality,
    and the bound must equal u * sum_r |dy/deps_r| for every output -- a dropped, doubled or
    misrouted term breaks the equality."""
    C_, F, H = 3, 1, 8
    P = oracle.Params(grid_shape=(2, 2, 2), mode=1, feat_dim=C_, n_freq=F, hidden=H)
    I = P.in_dim
    g = np.random.default_rng(21)
    mlp = {k: np.abs(v) for k, v in _mlp(I, H, 20).items()}
    mlp["b3"] = -np.array([30.0, 32.0, 35.0])
    e = g.uniform(0.2, 1.0, size=I)
    dc = g.uniform(0.3, 1.0, size=3)
    c, ec, de, ede, gw, eb = oracle.mlp_sample_bound(P, mlp, e, np.zeros(I), dc, 0.0, U_BF16, 0.0)
    assert np.all(c < 0.5)
    worst, _, (z1, z2) = _first_order_worst(mlp, e, dc, U_BF16)
    assert np.all(z1 > 0) and np.all(z2 > 0)
    W = _split(worst, I, H)
    got = {"c": ec, "de": ede} | {k: eb[k].reshape(-1) for k in ("w1", "b1", "w2", "b2", "w3", "b3")}
    for k, b in got.items():
        np.testing.assert_allclose(b, W[k], rtol=1e-10, err_msg=k)


def test_sample_bound_covers_a_relu_inside_its_rounding_band():
    C_, F, H = 4, 1, 8
    P = oracle.Params(grid_shape=(2, 2, 2), mode=1, feat_dim=C_, n_freq=F, hidden=H)
    I = P.in_dim
    mlp = _mlp(I, H, 7)
    e = np.random.default_rng(8).normal(size=I)
    dc = np.array([0.7, -0.4, 0.9])
    # put hidden unit 0 of layer 1 just above its kink: z1_0 = 1e-12
    mlp["b1"][0] = 1e-12 - float(e @ mlp["w1"][:, 0])
    _, _, de, ede, gw, eb = oracle.mlp_sample_bound(P, mlp, e, np.zeros(I), dc, 0.0, U_BF16, 0.0)
    # the flipped branch: unit 0 masked off changes dL/de by W1[:, 0] dh1_0 and dW1[:, 0] by e dh1_0
    _, y0, (z1, z2) = _first_order_worst(mlp, e, dc, U_BF16)
    Y = _split(y0, I, H)
    dh1_0 = Y["b1"][0]          # dz1_0 = dh1_0 while the unit is active
    assert abs(dh1_0) > 0
    assert np.all(ede >= np.abs(mlp["w1"][:, 0] * dh1_0))
    assert np.all(eb["w1"][:, 0] >= np.abs(e * dh1_0))
    assert eb["b1"][0] >= abs(dh1_0)


def _render_case(res=6, R=40, seed=3):
    C_, F, H = 12, 4, 16
    c, r = synth.random_spheres(3, seed, rmin=0.2, rmax=0.4)
    dens = synth.sphere_density(res, c, r, 8.0) + synth.normal_grid((res,) * 3, 1, 0.5, seed + 1)
    feat = synth.normal_grid((res,) * 3, C_, 1.0, seed + 2)
    P = oracle.Params(grid_shape=(res,) * 3, mode=1, feat_dim=C_, n_freq=F, hidden=H, delta=2.0 / res * 0.5,
                      shift_b=0.5, bg=(1.0, 1.0, 1.0))
    mlp = _mlp(P.in_dim, H, seed + 3)
    o, d, jit, _ = synth.fine_batch(R, seed + 4)
    gC = np.random.default_rng(seed + 5).normal(size=(R, 3))
    return P, dens, feat, mlp, o, d, jit, gC


def test_render_bound_is_zero_without_rounding_and_positive_with_it():
    P, dens, feat, mlp, o, d, jit, gC = _render_case()
    r0 = oracle.render(P, dens, feat, o, d, jitter=jit, mlp=mlp, grad_rgb=gC, error_bound=(0.0, 0.0))
    assert set(r0.bounds) == set(r0.grads)
    for k, v in r0.bounds.items():
        assert np.all(v == 0.0), k
    r1 = oracle.render(P, dens, feat, o, d, jitter=jit, mlp=mlp, grad_rgb=gC, error_bound=(U_BF16, 2.0 ** -24))
    for k, v in r1.bounds.items():
        touched = r1.grads[k] != 0
        assert np.all(v[touched] > 0), k
        assert np.all(v >= 0), k
    # the gradients themselves do not depend on the bound (up to the order of the OpenMP atomics)
    for k in r0.grads:
        np.testing.assert_allclose(r0.grads[k], r1.grads[k], rtol=1e-12, atol=1e-14 * np.abs(r0.grads[k]).max())


def test_render_bound_covers_a_perturbed_feature_grid():
    """Relative perturbations of at most u' on every feature value move each MLP input feature by
    at most u' sum_c w_c |V_c|, which the bound's input-error model (12 u_acc sum_c w_c |V_c| with
    u_acc = u') covers; every gradient element must then move by no more than its bound."""
    P, dens, feat, mlp, o, d, jit, gC = _render_case()
    up = 1e-7
    base = oracle.render(P, dens, feat, o, d, jitter=jit, mlp=mlp, grad_rgb=gC, error_bound=(0.0, up))
    g = np.random.default_rng(11)
    for trial in range(3):
        pert = feat * (1 + up * g.uniform(-1, 1, size=feat.shape))
        r = oracle.render(P, dens, pert, o, d, jitter=jit, mlp=mlp, grad_rgb=gC)
        for k in base.grads:
            diff = np.abs(r.grads[k] - base.grads[k])
            assert np.all(diff <= base.bounds[k] * (1 + 1e-6) + 1e-15), (k, trial, float((diff - base.bounds[k]).max()))


# ---------------------------------------------------------------------------------------------
# BF16-operand arithmetic (og_params.mlp_operands = 1: the chosen form's MLP, operands rounded to
# BF16, products accumulated exactly) and its bound against an FP32 evaluation
# ---------------------------------------------------------------------------------------------

def test_bf16_rounding_is_round_to_nearest_even():
    g = np.random.default_rng(40)
    v = np.concatenate([g.normal(size=4000) * 10.0 ** g.integers(-20, 20, size=4000),
                        g.uniform(-3, 3, size=4000)]).astype(np.float32).astype(np.float64)
    ref = torch.as_tensor(v, dtype=torch.float32).to(torch.bfloat16).double().numpy()
    np.testing.assert_array_equal(oracle.bf16(v), ref)
    ties = np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, -(1 + 2.0 ** -8), 0.0, 2.0 ** -130 * 0 + 1.5])
    np.testing.assert_array_equal(oracle.bf16(ties), [1.0, 1 + 2.0 ** -6, -1.0, 0.0, 1.5])


def _torch_chain(mlp, e, dc, dtype, rnd):
    """The sample's forward and backward written separately: operands passed through rnd at the
    contraction inputs, arithmetic in dtype."""
    t = {k: torch.as_tensor(v, dtype=dtype) for k, v in mlp.items()}
    x = rnd(torch.as_tensor(e, dtype=dtype))
    z1 = x @ t["w1"] + t["b1"]
    h1 = rnd(torch.relu(z1))
    z2 = h1 @ t["w2"] + t["b2"]
    h2 = rnd(torch.relu(z2))
    c = torch.sigmoid(h2 @ t["w3"] + t["b3"])
    dout = torch.as_tensor(dc, dtype=dtype) * c * (1 - c)
    do = rnd(dout)
    dz2 = rnd((do @ t["w3"].T) * (z2 > 0))
    dz1 = rnd((dz2 @ t["w2"].T) * (z1 > 0))
    de = dz1 @ t["w1"].T
    grads = {"w1": torch.outer(x, dz1), "b1": dz1, "w2": torch.outer(h1, dz2), "b2": dz2,
             "w3": torch.outer(h2, do), "b3": dout}
    ops = torch.cat([h1, h2, do, dz2, dz1]).double().numpy()
    return c, de, grads, ops


def _bf(x):
    return x.to(torch.bfloat16).to(x.dtype)


def test_bf16_operand_sample_matches_a_separate_chain_and_needs_no_bound_without_fp32_error():
    C_, F, H = 4, 2, 16
    P = oracle.Params(grid_shape=(2, 2, 2), mode=1, feat_dim=C_, n_freq=F, hidden=H, mlp_operands=1)
    I = P.in_dim
    mlp = {k: oracle.bf16(v) if k in ("w1", "b1", "w2", "w3") else v for k, v in _mlp(I, H, 30).items()}
    g = np.random.default_rng(31)
    e, dc = g.normal(size=I), g.normal(size=3)
    c, ec, de, ede, gw, eb = oracle.mlp_sample_bound(P, mlp, e, np.zeros(I), dc, 0.0, 0.0, 0.0)
    tc, tde, tg, _ = _torch_chain(mlp, e, dc, torch.float64, _bf)
    np.testing.assert_allclose(c, tc.numpy(), rtol=1e-14)
    np.testing.assert_allclose(de, tde.numpy(), rtol=1e-12, atol=1e-15)
    for k in tg:
        np.testing.assert_allclose(gw[k], tg[k].numpy(), rtol=1e-12, atol=1e-15, err_msg=k)
    # exact arithmetic on both sides: the operands agree, so the bound is 0
    assert np.all(ec == 0) and np.all(ede == 0) and all(np.all(v == 0) for v in eb.values())


@pytest.mark.parametrize("seed", [50, 51])
def test_bf16_operand_bound_covers_an_fp32_evaluation_brute_force(seed):
    """Many samples through a float32 evaluation of the same BF16-operand chain (torch CPU, its own
    summation order): wherever FP32 moves a value across a BF16 rounding midpoint the two operands
    differ by a BF16 step, and the bound must cover that, as it must cover the FP32 accumulation
    everywhere else."""
    C_, F, H = 12, 4, 128
    P = oracle.Params(grid_shape=(2, 2, 2), mode=1, feat_dim=C_, n_freq=F, hidden=H, mlp_operands=1)
    I = P.in_dim
    mlp = {k: oracle.bf16(v) if k in ("w1", "b1", "w2", "w3") else v for k, v in _mlp(I, H, seed).items()}
    mlp32 = {k: v.astype(np.float32).astype(np.float64) for k, v in mlp.items()}
    g = np.random.default_rng(seed + 1)
    u = 2.0 ** -24
    flips = 0
    worst = 0.0
    for n in range(1500):
        e = g.normal(size=I).astype(np.float32).astype(np.float64)
        dc = g.normal(size=3).astype(np.float32).astype(np.float64)
        c, ec, de, ede, gw, eb = oracle.mlp_sample_bound(P, mlp32, e, np.zeros(I), dc, 0.0, 0.0, u)
        c32, de32, g32, ops32 = _torch_chain(mlp32, e, dc, torch.float32, _bf)
        # operands that the FP32 and the exact evaluation round to different BF16 numbers
        _, _, _, ops64 = _torch_chain(mlp32, e, dc, torch.float64, _bf)
        flips += int(np.count_nonzero(ops32 != ops64))
        pairs = [(c32, c, ec), (de32, de, ede)] + [(g32[k], gw[k], eb[k]) for k in g32]
        for got, ref, b in pairs:
            d = np.abs(got.double().numpy() - ref)
            assert np.all(d <= b * (1 + 1e-9) + 1e-300), (n, float((d - b).max()))
            worst = max(worst, float((d / np.maximum(b, 1e-300)).max()))
    print(f"BF16 operands rounded differently by the FP32 evaluation: {flips}")
    assert flips >= 1, flips   # not vacuous: rounding flips occurred and were covered
