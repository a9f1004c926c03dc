"""Free-space skipping by the fine grid's own alpha (Sec. 4.2: a query point whose alpha is below
tau_f is skipped -- alpha 0, no colour query, no gradient) against the FP64 oracle, colours and
gradients, at tau_f = 1e-4 (Supp. A) and 1e-3; and the forward-only frame renderer, which skips
the same way at test time, against the oracle.

The skip decision compares alpha with tau_f in FP32 on the GPU and in FP64 in the oracle, so rays
with a sample whose alpha lies within 1e-3 (relative) of tau_f are left out of the comparison
(counted, and they must be few); every other ray must match: the FP32 path at the FP32 tolerances
(colours 1e-5, gradients 1e-4 with the 1 % floor plus the oracle's running error bound), the BF16
tensor-core path against the oracle in BF16-operand arithmetic within its bound.
"""
import numpy as np
import pytest
import torch

import oracle
from helpers import (BOUND_BF16_OPERANDS, BOUND_FP32, RTOL_COLOUR, assert_close, assert_within_bound, mlp_flat,
                     oracle_params)
from test_gpu_parity import _fine_inputs, _mlp_flat, _run_fine, cuda
from test_gpu_pe_x import _bf16_operands

pytestmark = pytest.mark.gpu

dvgo = pytest.importorskip("paper_2111_11215_gb300")


def _robust_rays(P, dens, o, d, jit, tau, band=1e-3):
    """Rays none of whose uniform samples has an alpha within `band` (relative) of tau, and the
    numbers of samples below / at or above tau on them."""
    keep, below, above = [], 0, 0
    for r in range(o.shape[0]):
        _, t0, t1, dn, n = oracle.ray_bounds(P, o[r], d[r], float(jit[r]))
        t = t0 + (np.arange(n) + float(jit[r])) * P.delta
        a = np.array([oracle.alpha_at(P, dens, o[r].astype(np.float64) + tk * dn, P.delta) for tk in t])
        if n and np.any(np.abs(a - tau) < band * tau):
            continue
        keep.append(r)
        below += int((a < tau).sum())
        above += int((a >= tau).sum())
    return np.array(keep), below, above


def _case(res, R, seed, tau):
    dens, feat, mlp, o, d, jit, _ = _fine_inputs(res, R, seed=seed)
    return dens, feat, mlp, o, d, jit


@pytest.mark.parametrize("tau", [1e-4, 1e-3])
@pytest.mark.parametrize("prec", [dvgo.DVGO_MLP_FP32, dvgo.DVGO_MLP_BF16])
def test_tau_f_skipping_colours_and_gradients(tau, prec, capsys):
    res, R = 24, 500
    dens, feat, mlp, o, d, jit = _case(res, R, 600, tau)
    bf = prec == dvgo.DVGO_MLP_BF16
    if bf:
        feat = torch.as_tensor(feat).to(torch.bfloat16).float().numpy()
    # alpha_init 1e-6: empty space falls below tau, the balls' surroundings cross it
    p = dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=2.0 / res * 0.5, bg=(1.0, 1.0, 1.0), tau_f=tau, mlp_prec=prec,
                    shift_b=dvgo.dvgo_shift_from_alpha_init(1e-6, 2.0 / res))
    P = oracle_params(p, (res,) * 3, 12, bf16_operands=bf)
    idx, below, above = _robust_rays(P, dens, o, d, jit, float(np.float32(tau)))
    assert len(idx) >= 0.9 * R and below > 5000 and above > 1000, (len(idx), below, above)
    o, d, jit = o[idx], d[idx], jit[idx]
    n = len(idx)
    g = np.random.default_rng(601)
    gC, gT = g.normal(scale=1e-2, size=(n, 3)), g.normal(scale=1e-2, size=n)
    got = _run_fine(p, res, dens, feat, mlp, o, d, jit, gC, gT, torch.bfloat16 if bf else torch.float32)
    ref = oracle.render(P, dens, feat, o, d, jitter=jit, mlp=_bf16_operands(mlp) if bf else mlp, grad_rgb=gC,
                        grad_tfinal=gT, error_bound=BOUND_BF16_OPERANDS if bf else BOUND_FP32)
    np.testing.assert_array_equal(got["counts"], ref.n_samples)
    if not bf:
        assert_close(got["rgb"], ref.rgb, RTOL_COLOUR, "rgb")
    else:
        assert np.abs(got["rgb"] - ref.rgb).max() < 1e-3
    assert_close(got["tfinal"], ref.tfinal, RTOL_COLOUR, "tfinal")
    assert_within_bound(got["g_d"], ref.grads["density"], ref.bounds["density"], "grad_density")
    assert_within_bound(got["g_f"], ref.grads["cgrid"], ref.bounds["cgrid"], "grad_feat")
    assert_within_bound(got["g_m"], mlp_flat(ref.grads), mlp_flat(ref.bounds), "grad_mlp")
    # not vacuous: skipping changes the render
    no_skip = oracle.render(oracle_params(p.with_(tau_f=0.0), (res,) * 3, 12, bf16_operands=bf), dens, feat, o, d,
                            jitter=jit, mlp=_bf16_operands(mlp) if bf else mlp)
    assert np.abs(no_skip.rgb - ref.rgb).max() > 1e-6
    with capsys.disabled():
        print(f"\ntau_f {tau} ({'BF16' if bf else 'FP32'} MLP): {R - n} of {R} rays set aside; "
              f"{below} samples skipped, {above} kept")


def test_frame_renderer_with_tau_f_matches_the_oracle():
    """Forward-only test-time rendering in chunks (tau_f = 1e-4, FP32 MLP) against the oracle."""
    res, R, tau = 24, 1000, 1e-4
    dens, feat, mlp, o, d, _ = _case(res, R, 610, tau)
    p = dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=2.0 / res * 0.5, bg=(1.0, 1.0, 1.0), tau_f=tau,
                    shift_b=dvgo.dvgo_shift_from_alpha_init(1e-6, 2.0 / res))
    P = oracle_params(p, (res,) * 3, 12)
    half = np.full(R, 0.5)
    idx, below, above = _robust_rays(P, dens, o, d, half, float(np.float32(tau)))
    assert len(idx) >= 0.9 * R and below > 1000 and above > 1000
    o, d = o[idx], d[idx]
    dd, cd = dvgo.GridDesc((res,) * 3, 1), dvgo.GridDesc((res,) * 3, 12)
    views = dvgo.render.mlp_views(cuda(_mlp_flat(mlp)))
    rgb, tf = dvgo.FrameRenderer(p, dd, cd, chunk=384).render(cuda(dens), cuda(feat), views, cuda(o), cuda(d))
    torch.cuda.synchronize()
    ref = oracle.render(P, dens, feat, o, d, mlp=mlp)
    assert_close(rgb.cpu().numpy(), ref.rgb, RTOL_COLOUR, "rgb")
    assert_close(tf.cpu().numpy(), ref.tfinal, RTOL_COLOUR, "tfinal")
