"""GPU parity of the 72-input colour MLP (Sec. 4.2 Eq. fine_queries_rgb with PE(x, 5), Supp. A
k_x = 5) and of the trilinear grid resize of progressive scaling (Sec. 4.2) against the FP64 oracle.

FP32 (SIMT) path: colours 1e-5 and gradients 1e-4 relative per element (floored), as for the
39-input MLP; the positional encoding of x is formed in FP32 from the fixed-point sample position
(one sincosf per axis and the double-angle identities), whose ~1e-6 absolute error on sin(16 x)
stays far below those bounds.  BF16 tensor-core path: the reference is the FP64 oracle run with
the weight operands the kernel multiplies (W1, b1, W2, W3 rounded to BF16; b2, b3 stay FP32), so
what remains is the rounding of activations and backward operands; the bounds of the 39-input BF16
tests apply, and the same relative-L2 bound to each block of W1 rows -- features + PE(d) (0-38),
PE(x) entries in the X panel (39-62) and in the tail panel (63-71, accumulated by the MMA whose
MN-major operand starts inside the swizzled rows).  (Against the unrounded weights the gradients of
the explicit-sample case move by 0.16 relative L2 in the oracle itself: ReLU masks flip.)

Resize: FP32 output of an FP64 interpolation, so 1 ulp of FP32 (relative 2^-24) against the FP64
oracle on the same FP32 input, in both layouts and with a destination box that pokes outside the
source box."""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import BOUND_BF16_OPERANDS, BOUND_FP32, RTOL_COLOUR, assert_close, assert_within_bound, oracle_params
from test_gpu_parity import _counts, _mlp_flat, cuda

pytestmark = pytest.mark.gpu

dvgo = pytest.importorskip("paper_2111_11215_gb300")

IN72 = 72
COLOUR_ABS_BOUND = 1e-2
GRAD_REL_L2_BOUND = 5e-2
MLP_KEYS = ("w1", "b1", "w2", "b2", "w3", "b3")


def _inputs(res, R, seed):
    c, rad = synth.random_spheres(5, seed, rmin=0.2, rmax=0.45)
    dens = (synth.sphere_density(res, c, rad, 20.0) + synth.normal_grid((res,) * 3, 1, 0.5, seed + 1)).astype(np.float32)
    feat = synth.smooth_features(res, 12, seed + 2)
    mlp = synth.mlp_weights(IN72, 128, 3, seed + 3)
    mlp["b3"] = np.random.default_rng(seed + 4).normal(scale=0.3, size=3).astype(np.float32)
    o, d, jit, _ = synth.fine_batch(R, seed + 5)
    return dens, feat, mlp, o, d, jit


def _run(p, res, dens, feat, mlp, o, d, jit, gC, gT, feat_dtype=torch.float32, samples=None):
    R = o.shape[0]
    fdt = dvgo.DVGO_DTYPE_BF16 if feat_dtype == torch.bfloat16 else dvgo.DVGO_DTYPE_F32
    dd, cd = dvgo.GridDesc((res,) * 3, 1), dvgo.GridDesc((res,) * 3, 12, dtype=fdt)
    r = dvgo.Renderer(p, dd, cd, R, samples_per_ray=None if samples is None else samples[0].shape[1])
    flat = cuda(_mlp_flat(mlp))
    views = dvgo.render.mlp_views(flat, IN72)
    D, F = cuda(dens), cuda(feat, feat_dtype)
    ro, rd, jt = cuda(o), cuda(d), (None if jit is None else cuda(jit))
    sm = None if samples is None else (cuda(samples[0]), cuda(samples[1]))
    rgb, tf, _ = r.forward(D, F, views, ro, rd, jt, sm)
    counts, total = _counts(r, R)
    g_d, g_f, g_m = torch.zeros_like(D), torch.zeros(F.shape, device="cuda"), torch.zeros_like(flat)
    r.backward(D, F, views, ro, rd, jt, sm, cuda(gC), None if gT is None else cuda(gT), g_d, g_f, g_m)
    torch.cuda.synchronize()
    return dict(rgb=rgb.cpu().numpy(), tfinal=tf.cpu().numpy(), counts=counts, total=total, g_d=g_d.cpu().numpy(),
                g_f=g_f.cpu().numpy(), g_m=g_m.cpu().numpy())


def _params(res, prec):
    return dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=2.0 / res * 0.5, bg=(1.0, 1.0, 1.0), mlp_prec=prec,
                       shift_b=dvgo.dvgo_shift_from_alpha_init(1e-2, 2.0 / res), n_freq_pos=5)


def _ref_flat(ref):
    return np.concatenate([ref.grads[k].reshape(-1) for k in MLP_KEYS])


@pytest.mark.parametrize("feat_dtype", [torch.float32, torch.bfloat16])
def test_pe_x_fp32_mlp_parity(feat_dtype):
    res, R = 24, 300
    dens, feat, mlp, o, d, jit = _inputs(res, R, seed=110)
    if feat_dtype == torch.bfloat16:
        feat = torch.as_tensor(feat).to(torch.bfloat16).float().numpy()
    p = _params(res, dvgo.DVGO_MLP_FP32)
    assert p.mlp_in_dim() == IN72
    g = np.random.default_rng(111)
    gC, gT = g.normal(scale=1e-2, size=(R, 3)), g.normal(scale=1e-2, size=R)
    got = _run(p, res, dens, feat, mlp, o, d, jit, gC, gT, feat_dtype)
    P = oracle_params(p, (res,) * 3, 12)
    assert P.in_dim == IN72
    ref = oracle.render(P, dens, feat, o, d, jitter=jit, mlp=mlp, grad_rgb=gC, grad_tfinal=gT, error_bound=BOUND_FP32)
    np.testing.assert_array_equal(got["counts"], ref.n_samples)
    assert got["total"] % 64 != 0 and got["total"] > 64 * 10
    assert_close(got["rgb"], ref.rgb, RTOL_COLOUR, "rgb")
    assert_within_bound(got["g_d"], ref.grads["density"], ref.bounds["density"], "grad_density")
    assert_within_bound(got["g_f"], ref.grads["cgrid"], ref.bounds["cgrid"], "grad_feat")
    off = 0
    for k in MLP_KEYS:
        n = mlp[k].size
        assert_within_bound(got["g_m"][off:off + n], ref.grads[k], ref.bounds[k], f"grad_{k}")
        off += n


def _rel_l2(got, ref):
    return float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-30))


def _bf16_operands(mlp):
    """The weights as the tensor-core kernel multiplies them: W1, b1 (the bias column of X), W2, W3
    rounded to BF16; b2, b3 are added in FP32 in the epilogues."""
    bf = lambda a: torch.as_tensor(np.asarray(a, np.float32)).to(torch.bfloat16).double().numpy()   # noqa: E731
    return {k: (bf(v) if k in ("w1", "b1", "w2", "w3") else np.asarray(v, np.float64)) for k, v in mlp.items()}


@pytest.mark.parametrize("feat_dtype", [torch.float32, torch.bfloat16])
def test_pe_x_bf16_tensor_core_mlp(feat_dtype, capsys):
    res, R = 24, 400
    dens, feat, mlp, o, d, jit = _inputs(res, R, seed=120)
    if feat_dtype == torch.bfloat16:
        feat = torch.as_tensor(feat).to(torch.bfloat16).float().numpy()
    p = _params(res, dvgo.DVGO_MLP_BF16)
    g = np.random.default_rng(121)
    gC, gT = g.normal(scale=1e-2, size=(R, 3)), g.normal(scale=1e-2, size=R)
    got = _run(p, res, dens, feat, mlp, o, d, jit, gC, gT, feat_dtype)
    ref = oracle.render(oracle_params(p, (res,) * 3, 12), dens, feat, o, d, jitter=jit, mlp=_bf16_operands(mlp),
                        grad_rgb=gC, grad_tfinal=gT)
    H = 128
    gw1 = got["g_m"][:IN72 * H].reshape(IN72, H)
    rw1 = ref.grads["w1"]
    errs = {"rgb_max_abs": float(np.abs(got["rgb"] - ref.rgb).max()),
            "grad_density_rel_l2": _rel_l2(got["g_d"], ref.grads["density"]),
            "grad_feat_rel_l2": _rel_l2(got["g_f"], ref.grads["cgrid"]),
            "w1_rows_0_38_rel_l2": _rel_l2(gw1[:39], rw1[:39]),
            "w1_rows_39_62_rel_l2": _rel_l2(gw1[39:63], rw1[39:63]),
            "w1_rows_63_71_rel_l2": _rel_l2(gw1[63:], rw1[63:])}
    ref_m, off = _ref_flat(ref), 0
    for k in MLP_KEYS:
        n = mlp[k].size
        errs[f"grad_{k}_rel_l2"] = _rel_l2(got["g_m"][off:off + n], ref_m[off:off + n])
        off += n
    with capsys.disabled():
        print(f"\nBF16 72-input MLP ({feat_dtype}) vs FP64 oracle:", {k: f"{v:.3g}" for k, v in errs.items()})
    assert errs["rgb_max_abs"] < COLOUR_ABS_BOUND
    for k, v in errs.items():
        if k.endswith("rel_l2"):
            assert v < GRAD_REL_L2_BOUND, (k, v)


@pytest.mark.parametrize("prec", [dvgo.DVGO_MLP_FP32, dvgo.DVGO_MLP_BF16])
def test_pe_x_explicit_samples(prec):
    """The proposal path (explicit t, dt): the PE(x) of every explicit sample position."""
    res, R, K = 20, 96, 48
    dens, feat, mlp, o, d, _ = _inputs(res, R, seed=130)
    p = _params(res, prec)
    P = oracle_params(p, (res,) * 3, 12)
    base = oracle.render(P, dens, feat, o, d, mlp=mlp)
    g = np.random.default_rng(131)
    u = np.sort(g.uniform(size=(R, K)), axis=1)
    t0, t1 = base.t_enter[:, None], base.t_exit[:, None]
    ts = np.where(t1 > t0, t0 + u * (t1 - t0), 0.0).astype(np.float32)
    dts = np.diff(np.concatenate([ts, ts[:, -1:] + 0.01], axis=1), axis=1).astype(np.float32)
    gC = g.normal(scale=1e-2, size=(R, 3))
    got = _run(p, res, dens, feat, mlp, o, d, None, gC, None, samples=(ts, dts))
    bf = prec == dvgo.DVGO_MLP_BF16
    ref = oracle.render(oracle_params(p, (res,) * 3, 12, bf16_operands=bf), dens, feat, o, d,
                        mlp=_bf16_operands(mlp) if bf else mlp, explicit_t=ts, explicit_dt=dts, grad_rgb=gC,
                        error_bound=BOUND_BF16_OPERANDS if bf else BOUND_FP32)
    assert_within_bound(got["g_f"], ref.grads["cgrid"], ref.bounds["cgrid"], "grad_feat")
    assert_within_bound(got["g_m"][:IN72 * 128], ref.grads["w1"], ref.bounds["w1"], "grad_w1")
    if not bf:
        assert_close(got["rgb"], ref.rgb, RTOL_COLOUR, "rgb")
    else:
        errs = {"rgb_max_abs": float(np.abs(got["rgb"] - ref.rgb).max()),
                "grad_feat_rel_l2": _rel_l2(got["g_f"], ref.grads["cgrid"]),
                "w1_rel_l2": _rel_l2(got["g_m"][:IN72 * 128], ref.grads["w1"].reshape(-1))}
        print("BF16 72-input MLP, explicit samples:", {k: f"{v:.3g}" for k, v in errs.items()})
        assert errs["rgb_max_abs"] < COLOUR_ABS_BOUND
        assert errs["grad_feat_rel_l2"] < GRAD_REL_L2_BOUND and errs["w1_rel_l2"] < GRAD_REL_L2_BOUND


def test_pe_x_unsupported_frequency_count_is_rejected():
    res = 8
    p = dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=0.1, n_freq_pos=3)
    dd, cd = dvgo.GridDesc((res,) * 3, 1), dvgo.GridDesc((res,) * 3, 12)
    ws = torch.empty(dvgo.dvgo_workspace_size(p, dd, 4), dtype=torch.uint8, device="cuda")
    flat = torch.zeros(dvgo.render.mlp_flat_size(12 + 3 + 24 + 3 + 18), device="cuda")
    ro = torch.zeros((4, 3), device="cuda")
    out = torch.empty((4, 3), device="cuda")
    with pytest.raises(dvgo.DVGOError) as ei:
        dvgo.dvgo_render_fwd(p, dd, torch.zeros(res ** 3, device="cuda"), cd, torch.zeros(res ** 3 * 12, device="cuda"),
                             dvgo.render.mlp_views(flat, 12 + 3 + 24 + 3 + 18), ro, ro + 1.0, None, None, None, out,
                             None, None, None, ws)
    assert ei.value.status == -3


# ------------------------------------------------------------------------------------------
# Trilinear resize (progressive scaling)
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("C,src,dst,layouts", [
    (1, (23, 17, 30), (46, 34, 60), (0, 0)),
    (12, (20, 20, 20), (25, 25, 25), (0, 1)),
    (12, (25, 21, 18), (19, 30, 22), (1, 0)),
    (3, (9, 9, 9), (9, 9, 9), (1, 1)),
])
def test_resize_matches_oracle(C, src, dst, layouts):
    g = np.random.default_rng(140 + C)
    a = g.normal(size=tuple(src) + ((C,) if C > 1 else ())).astype(np.float32)
    sbox = ((-1.0, -0.75, -1.25), (1.0, 0.5, 1.0))
    dbox = ((-1.1, -0.5, -1.25), (0.9, 0.6, 0.75))      # reaches past the source box on two axes
    sd = dvgo.GridDesc(src, C, sbox[0], sbox[1])
    dd = dvgo.GridDesc(dst, C, dbox[0], dbox[1])
    x = cuda(a).reshape(-1)
    if layouts[0]:
        x = dvgo.dvgo_pack_grid(sd, x, sd.with_(layout=1))
    out = dvgo.dvgo_resize_grid(sd.with_(layout=layouts[0]), x, dd.with_(layout=layouts[1]))
    if layouts[1]:
        out = dvgo.dvgo_pack_grid(dd.with_(layout=1), out, dd)
    got = out.reshape(tuple(dst) + ((C,) if C > 1 else ())).cpu().numpy()
    f32 = lambda box: tuple(tuple(float(np.float32(v)) for v in b) for b in box)   # noqa: E731
    ref = oracle.resize_grid(a, dst, f32(sbox), f32(dbox))
    # FP32 rounding of the result; atol covers values that cancel to ~0 (FMA contraction on the GPU)
    np.testing.assert_allclose(got, ref, rtol=2 ** -23, atol=1e-12)


def test_resize_rejects_mismatched_channels_and_aliasing():
    sd, dd = dvgo.GridDesc((8, 8, 8), 3), dvgo.GridDesc((12, 12, 12), 1)
    x = torch.zeros(8 ** 3 * 3, device="cuda")
    with pytest.raises(dvgo.DVGOError):
        dvgo.dvgo_resize_grid(sd, x, dd)
    with pytest.raises(dvgo.DVGOError):
        dvgo.dvgo_resize_grid(sd, x, sd, out=x)
