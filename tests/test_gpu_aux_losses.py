"""GPU parity of the auxiliary losses (Supp. A: per-point rgb, background entropy) against the FP64
oracle: the forward's total loss, and the backward seeded with the forward's photometric
dL/dC_hat only (the library adds the auxiliary gradients from the targets the forward kept)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import BOUND_FP32, RTOL_GRAD, assert_close, assert_within_bound, mlp_flat, oracle_params
from test_gpu_parity import _fine_inputs, _mlp_flat, cuda

pytestmark = pytest.mark.gpu

dvgo = pytest.importorskip("paper_2111_11215_gb300")


@pytest.mark.parametrize("w_pt,w_bg", [(0.1, 0.01), (0.0, 0.3), (0.5, 0.0)])
def test_coarse_aux_losses(w_pt, w_bg):
    case = synth.coarse_case(seed=0)
    R, res = case["rays_o"].shape[0], case["density"].shape[0]
    p = dvgo.Params(mode=dvgo.DVGO_MODE_COARSE, step=0.03125, shift_b=0.0, bg=(1.0, 1.0, 1.0), rgb_act=1,
                    w_pt_rgb=w_pt, w_bg=w_bg)
    dd, cd = dvgo.GridDesc((res,) * 3, 1), dvgo.GridDesc((res,) * 3, 3)
    r = dvgo.Renderer(p, dd, cd, R)
    dens, rgbg = cuda(case["density"]), cuda(case["rgb"])
    ro, rd, tgt = cuda(case["rays_o"]), cuda(case["rays_d"]), cuda(case["target"])
    dloss = torch.empty((R, 3), device="cuda")
    _, _, loss = r.forward(dens, rgbg, None, ro, rd, None, None, tgt, dloss=dloss)
    g_d, g_c = torch.zeros_like(dens), torch.zeros_like(rgbg)
    r.backward(dens, rgbg, None, ro, rd, None, None, dloss, None, g_d, g_c, None)
    torch.cuda.synchronize()
    P = oracle_params(p, (res,) * 3, 3)
    ref = oracle.render(P, case["density"], case["rgb"], case["rays_o"], case["rays_d"], target=case["target"])
    gC = 2.0 * (ref.rgb - case["target"]) / R
    refb = oracle.render(P, case["density"], case["rgb"], case["rays_o"], case["rays_d"], target=case["target"],
                         grad_rgb=gC)
    base = oracle.render(oracle_params(dvgo.Params(mode=dvgo.DVGO_MODE_COARSE, step=0.03125, rgb_act=1), (res,) * 3, 3),
                         case["density"], case["rgb"], case["rays_o"], case["rays_d"], target=case["target"])
    assert abs(ref.loss - base.loss) > 1e-3 * base.loss            # the auxiliary terms are not negligible
    assert float(loss.item()) == pytest.approx(ref.loss, rel=1e-5)
    assert_close(g_d.cpu().numpy(), refb.grads["density"], RTOL_GRAD, "grad_density")
    assert_close(g_c.cpu().numpy(), refb.grads["cgrid"], RTOL_GRAD, "grad_rgb")


def test_fine_aux_losses_fp32():
    res, R = 24, 300
    dens, feat, mlp, o, d, jit, tgt = _fine_inputs(res, R, seed=50)
    p = dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=2.0 / res * 0.5, bg=(1.0, 1.0, 1.0),
                    shift_b=dvgo.dvgo_shift_from_alpha_init(1e-2, 2.0 / res), w_pt_rgb=0.5, w_bg=0.2)
    dd, cd = dvgo.GridDesc((res,) * 3, 1), dvgo.GridDesc((res,) * 3, 12)
    r = dvgo.Renderer(p, dd, cd, R)
    flat = cuda(_mlp_flat(mlp))
    views = dvgo.render.mlp_views(flat)
    D, F = cuda(dens), cuda(feat)
    ro, rd, jt, tg = cuda(o), cuda(d), cuda(jit), cuda(tgt)
    dloss = torch.empty((R, 3), device="cuda")
    _, _, loss = r.forward(D, F, views, ro, rd, jt, None, tg, dloss=dloss)
    g_d, g_f, g_m = torch.zeros_like(D), torch.zeros_like(F), torch.zeros_like(flat)
    r.backward(D, F, views, ro, rd, jt, None, dloss, None, g_d, g_f, g_m)
    torch.cuda.synchronize()
    P = oracle_params(p, (res,) * 3, 12)
    ref = oracle.render(P, dens, feat, o, d, jitter=jit, mlp=mlp, target=tgt)
    gC = 2.0 * (ref.rgb - tgt) / R
    refb = oracle.render(P, dens, feat, o, d, jitter=jit, mlp=mlp, target=tgt, grad_rgb=gC, error_bound=BOUND_FP32)
    assert float(loss.item()) == pytest.approx(ref.loss, rel=1e-5)
    assert_within_bound(g_d.cpu().numpy(), refb.grads["density"], refb.bounds["density"], "grad_density")
    assert_within_bound(g_f.cpu().numpy(), refb.grads["cgrid"], refb.bounds["cgrid"], "grad_feat")
    assert_within_bound(g_m.cpu().numpy(), mlp_flat(refb.grads), mlp_flat(refb.bounds), "grad_mlp")
    # a forward without a target leaves no auxiliary gradient behind
    r.forward(D, F, views, ro, rd, jt)
    g2 = torch.zeros_like(D)
    r.backward(D, F, views, ro, rd, jt, None, dloss, None, g2, torch.zeros_like(F), torch.zeros_like(flat))
    plain = oracle.render(P, dens, feat, o, d, jitter=jit, mlp=mlp, grad_rgb=gC, error_bound=BOUND_FP32)
    assert_within_bound(g2.cpu().numpy(), plain.grads["density"], plain.bounds["density"], "grad_density_no_target")


def test_allocation_free_forward_rejects_aux_weights():
    p = dvgo.Params(mode=dvgo.DVGO_MODE_COARSE, step=0.1, w_bg=0.01)
    dd, cd = dvgo.GridDesc((8,) * 3, 1), dvgo.GridDesc((8,) * 3, 3)
    dens, rgbg = torch.zeros(8, 8, 8, device="cuda"), torch.zeros(8, 8, 8, 3, device="cuda")
    o = torch.zeros((4, 3), device="cuda")
    with pytest.raises(dvgo.DVGOError):
        dvgo.dvgo_render_fwd_noalloc(p, dd, dens, cd, rgbg, o, o + 1.0, None, None, torch.empty((4, 3), device="cuda"),
                                     None, None, None)
