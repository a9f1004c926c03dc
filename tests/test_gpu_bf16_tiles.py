"""The chosen form's BF16 tensor-core colour backward against the FP64 oracle at production tile
counts: enough samples that every persistent CTA of the colour kernels runs many 128-sample
tiles, so that the paths a one-tile-per-CTA case never reaches are compared element by element --
the second X panel (tile i uses buffer i & 1), the producers' deferred feature-gradient scatter of
the tile two back, and the weight gradients accumulated in TMEM across a CTA's tiles and flushed
once (Sec. 4.2 Eq. fine_queries_rgb, backward by the chain rule).

Inputs: a 64^3 scene (5 balls, raw density 20, noise), BF16 feature storage, the 39-128-128-3 MLP;
(1) 4096 rays with uniform 0.5-voxel steps (~274 k samples, ~14 tiles per CTA) and (2) 6144 rays
with 48 explicit samples each, clustered around a random depth per ray the way proposal samples
gather at surfaces (~230 k samples, ~12 tiles per CTA).

Oracle: the chosen form's arithmetic -- the MLP's contraction operands (X, H1, H2, dL/do, dZ2, dZ1)
rounded to BF16, products accumulated exactly -- on the operands the kernel multiplies (the
BF16-rounded W1 | b1, W2, W3 and features).  Both sides then round the same values to BF16, so an
operand differs only where the kernel's FP32 accumulation moves a value across a BF16 rounding
midpoint, and the oracle's running error bound flags exactly those operands.

Tolerance per element: 1e-4 max(|o|, 1e-2 max|o|) plus that bound.  Reading of the faults the
test must catch: a tile whose feature gradients were never scattered removes the full
contributions of its 128 samples from the voxels they touch (the bound is ~20 % of a typical
feature-gradient element here), and weight-gradient sums that lost a CTA's earlier tiles are off by
most of their value (the bound is 10-25 % of a typical W2, b2 or W3 element).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import BOUND_BF16_OPERANDS, assert_within_bound, mlp_flat, oracle_params
from test_gpu_parity import _fine_inputs, _run_fine
from test_gpu_pe_x import _bf16_operands

pytestmark = pytest.mark.gpu

dvgo = pytest.importorskip("paper_2111_11215_gb300")

N_SM = 152
TILE = 128


def _bf16(a):
    return torch.as_tensor(np.asarray(a, np.float32)).to(torch.bfloat16).float().numpy()


def _params(res):
    return dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=2.0 / res * 0.5, bg=(1.0, 1.0, 1.0),
                       mlp_prec=dvgo.DVGO_MLP_BF16, shift_b=dvgo.dvgo_shift_from_alpha_init(1e-2, 2.0 / res))


def _check(got, ref, capsys, label):
    worst = {}
    worst["density"], rd = assert_within_bound(got["g_d"], ref.grads["density"], ref.bounds["density"],
                                               f"{label} grad_density")
    worst["feat"], rf = assert_within_bound(got["g_f"], ref.grads["cgrid"], ref.bounds["cgrid"], f"{label} grad_feat")
    off, rel = 0, {"density": rd, "feat": rf}
    for k in ("w1", "b1", "w2", "b2", "w3", "b3"):
        n = ref.grads[k].size
        worst[k], rel[k] = assert_within_bound(got["g_m"][off:off + n], ref.grads[k], ref.bounds[k], f"{label} grad_{k}")
        off += n
    col = float(np.abs(got["rgb"] - ref.rgb).max())
    with capsys.disabled():
        print(f"\n{label}: colours max abs {col:.3g}; worst error / tolerance "
              + ", ".join(f"{k} {v:.2f}" for k, v in worst.items())
              + "; relative L2 " + ", ".join(f"{k} {v:.3g}" for k, v in rel.items()))
    assert col < 1e-2


def test_bf16_backward_uniform_steps_many_tiles_per_cta(capsys):
    res, R = 64, 4096
    dens, feat, mlp, o, d, jit, _ = _fine_inputs(res, R, seed=500)
    feat = _bf16(feat)
    p = _params(res)
    g = np.random.default_rng(501)
    gC = g.normal(scale=1e-2, size=(R, 3))
    gT = g.normal(scale=1e-2, size=R)
    got = _run_fine(p, res, dens, feat, mlp, o, d, jit, gC, gT, torch.bfloat16)
    assert got["total"] / TILE / N_SM >= 8, got["total"]           # every CTA runs many tiles
    ref = oracle.render(oracle_params(p, (res,) * 3, 12, bf16_operands=True), dens, feat, o, d, jitter=jit,
                        mlp=_bf16_operands(mlp), grad_rgb=gC, grad_tfinal=gT, error_bound=BOUND_BF16_OPERANDS)
    np.testing.assert_array_equal(got["counts"], ref.n_samples)
    _check(got, ref, capsys, f"uniform, {got['total']} samples")


def _clustered_samples(t0, t1, K, seed):
    """K sorted samples per ray inside [t_enter, t_exit]: 3/4 drawn around a random depth (sd 4 %
    of the interval), 1/4 uniform; dt = distance to the next sample (last: 1/K of the interval)."""
    g = np.random.default_rng(seed)
    R = t0.shape[0]
    L = np.maximum(t1 - t0, 0.0)[:, None]
    centre = g.uniform(0.2, 0.8, size=(R, 1))
    n_c = 3 * K // 4
    u = np.concatenate([np.clip(centre + 0.04 * g.normal(size=(R, n_c)), 0.0, 0.999),
                        g.uniform(size=(R, K - n_c))], axis=1)
    u = np.sort(u, axis=1)
    ts = np.where(L > 0, t0[:, None] + u * L, 0.0).astype(np.float32)
    dts = np.diff(np.concatenate([ts, ts[:, -1:] + (L / K).astype(np.float32)], axis=1), axis=1).astype(np.float32)
    return ts, np.maximum(dts, 0.0).astype(np.float32)


def test_bf16_backward_explicit_samples_many_tiles_per_cta(capsys):
    res, R, K = 64, 6144, 48
    dens, feat, mlp, o, d, _, _ = _fine_inputs(res, R, seed=510)
    feat = _bf16(feat)
    p = _params(res)
    P = oracle_params(p, (res,) * 3, 12)
    base = oracle.render(P, dens, feat, o, d, mlp=mlp)
    ts, dts = _clustered_samples(base.t_enter, base.t_exit, K, 511)
    g = np.random.default_rng(512)
    gC = g.normal(scale=1e-2, size=(R, 3))
    dd, cd = dvgo.GridDesc((res,) * 3, 1), dvgo.GridDesc((res,) * 3, 12, dtype=dvgo.DVGO_DTYPE_BF16)
    r = dvgo.Renderer(p, dd, cd, R, samples_per_ray=K)
    flat = torch.as_tensor(mlp_flat(mlp), dtype=torch.float32, device="cuda")
    views = dvgo.render.mlp_views(flat)
    cu = lambda a, dt=torch.float32: torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)  # noqa: E731
    D, F = cu(dens), cu(feat, torch.bfloat16)
    samples = (cu(ts), cu(dts))
    rgb, _, _ = r.forward(D, F, views, cu(o), cu(d), None, samples)
    g_d, g_f, g_m = torch.zeros_like(D), torch.zeros(F.shape, device="cuda"), torch.zeros_like(flat)
    r.backward(D, F, views, cu(o), cu(d), None, samples, cu(gC), None, g_d, g_f, g_m)
    torch.cuda.synchronize()
    hit = int((base.t_exit > base.t_enter).sum())
    assert hit * K / TILE / N_SM >= 8, hit
    ref = oracle.render(oracle_params(p, (res,) * 3, 12, bf16_operands=True), dens, feat, o, d,
                        mlp=_bf16_operands(mlp), explicit_t=ts, explicit_dt=dts, grad_rgb=gC,
                        error_bound=BOUND_BF16_OPERANDS)
    got = {"rgb": rgb.cpu().numpy(), "g_d": g_d.cpu().numpy(), "g_f": g_f.cpu().numpy(), "g_m": g_m.cpu().numpy()}
    _check(got, ref, capsys, f"explicit, {hit * K} samples")


def _pack(a, desc, dtype):
    return dvgo.dvgo_pack_grid(desc, a.reshape(-1).contiguous(),
                               desc.with_(layout=dvgo.DVGO_LAYOUT_PACKED, dtype=dtype))


def _unpack(a, desc):
    return dvgo.dvgo_pack_grid(desc.with_(layout=dvgo.DVGO_LAYOUT_PACKED), a, desc).reshape(
        tuple(desc.shape) + ((desc.channels,) if desc.channels > 1 else ()))


@pytest.mark.parametrize("pex", [False, True], ids=["39in", "72in"])
@pytest.mark.parametrize("feat_bf16", [True, False], ids=["bf16feat", "f32feat"])
@pytest.mark.parametrize("packed", [False, True], ids=["canonical", "packed"])
def test_bf16_backward_every_kernel_variant_many_tiles_per_cta(pex, feat_bf16, packed, capsys):
    """Every compiled variant of the tensor-core colour kernels (feature storage FP32 / BF16, 39 or
    72 inputs -- PE(x, 5) with its tail panel --, canonical or packed grid layout) at >= 8 tiles per
    CTA, against the BF16-operand oracle within its rounding bound."""
    res, R = 64, 3000
    seed = 520 + 4 * pex + 2 * feat_bf16 + packed
    dens, feat, mlp, o, d, jit, _ = _fine_inputs(res, R, seed=seed)
    if pex:
        mlp = synth.mlp_weights(72, 128, 3, seed + 3)
        mlp["b3"] = np.random.default_rng(seed + 4).normal(scale=0.3, size=3).astype(np.float32)
    if feat_bf16:
        feat = _bf16(feat)
    p = _params(res).with_(n_freq_pos=5 if pex else 0)
    fdt = dvgo.DVGO_DTYPE_BF16 if feat_bf16 else dvgo.DVGO_DTYPE_F32
    lay = dvgo.DVGO_LAYOUT_PACKED if packed else dvgo.DVGO_LAYOUT_CANONICAL
    dd0, cd0 = dvgo.GridDesc((res,) * 3, 1), dvgo.GridDesc((res,) * 3, 12)
    dd, cd = dd0.with_(layout=lay), cd0.with_(layout=lay, dtype=fdt)
    cu = lambda a, dt=torch.float32: torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)  # noqa: E731
    if packed:
        D = _pack(cu(dens), dd0, dvgo.DVGO_DTYPE_F32)
        F = _pack(cu(feat), cd0, fdt)
    else:
        D, F = cu(dens), cu(feat, torch.bfloat16 if feat_bf16 else torch.float32)
    flat = cu(mlp_flat(mlp))
    views = dvgo.render.mlp_views(flat, 72 if pex else 39)
    r = dvgo.Renderer(p, dd, cd, R)
    g = np.random.default_rng(seed + 9)
    gC = g.normal(scale=1e-2, size=(R, 3))
    rgb, _, _ = r.forward(D, F, views, cu(o), cu(d), cu(jit))
    g_d, g_f, g_m = torch.zeros_like(D), torch.zeros(F.shape, device="cuda"), torch.zeros_like(flat)
    r.backward(D, F, views, cu(o), cu(d), cu(jit), None, cu(gC), None, g_d, g_f, g_m)
    torch.cuda.synchronize()
    kept = int(r.workspace[8:12].view(torch.int32).item())
    assert kept / TILE / N_SM >= 8, kept
    if packed:
        g_d, g_f = _unpack(g_d, dd0), _unpack(g_f, cd0)
    ref = oracle.render(oracle_params(p, (res,) * 3, 12, bf16_operands=True), dens, feat, o, d, jitter=jit,
                        mlp=_bf16_operands(mlp), grad_rgb=gC, error_bound=BOUND_BF16_OPERANDS)
    got = {"rgb": rgb.cpu().numpy(), "g_d": g_d.cpu().numpy(), "g_f": g_f.cpu().numpy(), "g_m": g_m.cpu().numpy()}
    _check(got, ref, capsys, f"{'72' if pex else '39'} inputs, {'BF16' if feat_bf16 else 'FP32'} features, "
                             f"{'packed' if packed else 'canonical'}, {kept} samples")
