"""Degenerate fine-stage batches through both colour paths (FP32 SIMT and the chosen form's BF16
tensor-core kernels), against the FP64 oracle.

* No sample reaches the MLP: every ray misses the box, or every sample's alpha lies below tau_f
  (Sec. 4.2 free-space skipping).  The persistent colour kernels then run with zero tiles; the
  render is the background with T_final = 1 and every gradient is exactly zero.
* Exact and ragged tile counts with explicit per-ray samples (the proposal path), all kept
  (tau_f = 0, every ray hits the box), so that the kept count is R K exactly: one sample (one
  tile with 127 empty rows), exactly one 128-row tile, exactly two tiles for every one of the
  GPU's CTAs (the producers' deferred scatter then runs only after the loop), and a ragged tail.
  The BF16 kernels are compared with the oracle in BF16-operand arithmetic within its bound.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import BOUND_BF16_OPERANDS, BOUND_FP32, RTOL_COLOUR, assert_close, mlp_flat, oracle_params
from test_gpu_bf16_tiles import _bf16, _check
from test_gpu_parity import _fine_inputs, _run_fine
from test_gpu_pe_x import _bf16_operands

pytestmark = pytest.mark.gpu

dvgo = pytest.importorskip("paper_2111_11215_gb300")

RES = 24
PRECS = [dvgo.DVGO_MLP_FP32, dvgo.DVGO_MLP_BF16]
PREC_IDS = ["fp32", "bf16"]


def _params(prec, **kw):
    return dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=2.0 / RES * 0.5, bg=(0.25, 0.5, 0.75), mlp_prec=prec,
                       shift_b=dvgo.dvgo_shift_from_alpha_init(1e-2, 2.0 / RES), **kw)


def _missing_rays(R, seed):
    """Rays that never enter the [-1, 1]^3 box: half start beyond x = 1 and point away from it, half
    run parallel to the x axis outside the box's y range."""
    g = np.random.default_rng(seed)
    h = R // 2
    o1 = np.stack([g.uniform(1.5, 3.0, h), g.uniform(-0.9, 0.9, h), g.uniform(-0.9, 0.9, h)], 1)
    d1 = np.stack([np.ones(h), g.uniform(-0.2, 0.2, h), g.uniform(-0.2, 0.2, h)], 1)
    o2 = np.stack([np.full(R - h, -3.0), g.choice([-1.0, 1.0], R - h) * g.uniform(1.2, 2.0, R - h),
                   g.uniform(-0.9, 0.9, R - h)], 1)
    d2 = np.tile([1.0, 0.0, 0.0], (R - h, 1))
    o = np.concatenate([o1, o2]).astype(np.float32)
    d = np.concatenate([d1, d2])
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    return o, d, g.uniform(size=R).astype(np.float32)


def _assert_empty_render(got, p, R):
    bg = np.tile(np.float32(p.bg), (R, 1))
    np.testing.assert_array_equal(got["rgb"], bg)
    np.testing.assert_array_equal(got["tfinal"], np.ones(R, np.float32))
    for k in ("g_d", "g_f", "g_m"):
        assert not np.any(got[k]), k


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
def test_fine_every_ray_misses_the_box(prec):
    R = 300
    dens, feat, mlp, _, _, _, _ = _fine_inputs(RES, R, seed=800)
    o, d, jit = _missing_rays(R, 801)
    p = _params(prec)
    g = np.random.default_rng(802)
    gC, gT = g.normal(size=(R, 3)), g.normal(size=R)
    got = _run_fine(p, RES, dens, _bf16(feat), mlp, o, d, jit, gC, gT, torch.bfloat16)
    ref = oracle.render(oracle_params(p, (RES,) * 3, 12), dens, _bf16(feat), o, d, jitter=jit, mlp=mlp)
    assert not np.any(ref.n_samples)
    np.testing.assert_array_equal(got["counts"], ref.n_samples)
    assert got["total"] == 0
    _assert_empty_render(got, p, R)


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
def test_fine_every_sample_below_tau_f(prec):
    """Rays cross the box, but the raw density is -30 everywhere, so every alpha (~1e-14) is below
    tau_f = 1e-4: every sample is skipped before the colour MLP (alpha 0, no gradient)."""
    R = 300
    _, feat, mlp, o, d, jit, _ = _fine_inputs(RES, R, seed=810)
    dens = np.full((RES,) * 3, -30.0, np.float32)
    p = _params(prec, tau_f=1e-4)
    g = np.random.default_rng(811)
    gC, gT = g.normal(size=(R, 3)), g.normal(size=R)
    got = _run_fine(p, RES, dens, _bf16(feat), mlp, o, d, jit, gC, gT, torch.bfloat16)
    P = oracle_params(p, (RES,) * 3, 12)
    ref = oracle.render(P, dens, _bf16(feat), o, d, jitter=jit, mlp=mlp, grad_rgb=gC, grad_tfinal=gT,
                        error_bound=BOUND_FP32)
    assert ref.n_samples.sum() > 10 * 128                      # the rays do cross the box
    np.testing.assert_array_equal(got["counts"], ref.n_samples)
    np.testing.assert_array_equal(ref.rgb, np.tile(np.float64(np.float32(p.bg)), (R, 1)))
    assert not np.any(ref.grads["density"]) and not np.any(ref.grads["cgrid"])
    _assert_empty_render(got, p, R)


def _hitting_rays(R, seed):
    """R seeded rays of the synthetic rig that cross the box, with their clip interval."""
    o, d, _, _ = synth.fine_batch(4 * R + 64, seed)
    P = oracle_params(_params(dvgo.DVGO_MLP_BF16), (RES,) * 3, 12)
    t0, t1 = np.empty(len(o)), np.empty(len(o))
    for r in range(len(o)):
        _, t0[r], t1[r], _, _ = oracle.ray_bounds(P, o[r], d[r], 0.5)
    hit = np.nonzero(t1 - t0 > 0.05)[0][:R]
    assert len(hit) == R
    return o[hit], d[hit], t0[hit], t1[hit]


def _explicit_samples(t0, t1, K, seed):
    """K stratified samples per ray strictly inside (t_enter, t_exit), one in each of K equal strata
    and at least 0.2 of a stratum apart, so that every dt = distance to the next sample (last: 1 / K
    of the interval) is positive."""
    g = np.random.default_rng(seed)
    L = (t1 - t0)[:, None]
    u = 0.01 + 0.98 * (np.arange(K)[None, :] + g.uniform(0.1, 0.9, size=(len(t0), K))) / K
    ts = (t0[:, None] + u * L).astype(np.float32)
    dts = np.diff(np.concatenate([ts, ts[:, -1:] + (L / K).astype(np.float32)], axis=1), axis=1)
    return ts, np.maximum(dts, 0.0).astype(np.float32)


@pytest.mark.parametrize("R,K", [(1, 1), (2, 64), (608, 64), (37, 48)],
                         ids=["one_sample", "one_full_tile", "two_tiles_per_cta", "ragged"])
def test_bf16_explicit_samples_exact_and_ragged_tiles(R, K, capsys):
    dens, feat, mlp, _, _, _, _ = _fine_inputs(RES, 8, seed=820)
    feat = _bf16(feat)
    o, d, t0, t1 = _hitting_rays(R, 821)
    ts, dts = _explicit_samples(t0, t1, K, 822)
    p = _params(dvgo.DVGO_MLP_BF16)
    g = np.random.default_rng(823)
    gC = g.normal(scale=1e-2, size=(R, 3))
    dd, cd = dvgo.GridDesc((RES,) * 3, 1), dvgo.GridDesc((RES,) * 3, 12, dtype=dvgo.DVGO_DTYPE_BF16)
    r = dvgo.Renderer(p, dd, cd, R, samples_per_ray=K)
    flat = torch.as_tensor(mlp_flat(mlp), dtype=torch.float32, device="cuda")
    views = dvgo.render.mlp_views(flat)
    cu = lambda a, dt=torch.float32: torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)  # noqa: E731
    D, F = cu(dens), cu(feat, torch.bfloat16)
    samples = (cu(ts), cu(dts))
    rgb, tf, _ = r.forward(D, F, views, cu(o), cu(d), None, samples)
    g_d, g_f, g_m = torch.zeros_like(D), torch.zeros(F.shape, device="cuda"), torch.zeros_like(flat)
    r.backward(D, F, views, cu(o), cu(d), None, samples, cu(gC), None, g_d, g_f, g_m)
    torch.cuda.synchronize()
    kept = int(r.workspace[8:12].view(torch.int32).item())
    assert kept == R * K, kept
    assert dvgo.dvgo_workspace_status(r.workspace) == 0
    ref = oracle.render(oracle_params(p, (RES,) * 3, 12, bf16_operands=True), dens, feat, o, d,
                        mlp=_bf16_operands(mlp), explicit_t=ts, explicit_dt=dts, grad_rgb=gC,
                        error_bound=BOUND_BF16_OPERANDS)
    assert_close(tf.cpu().numpy(), ref.tfinal, RTOL_COLOUR, "tfinal")
    got = {"rgb": rgb.cpu().numpy(), "g_d": g_d.cpu().numpy(), "g_f": g_f.cpu().numpy(), "g_m": g_m.cpu().numpy()}
    _check(got, ref, capsys, f"explicit {R} x {K} = {kept} samples ({kept / 128:.3g} tiles)")
