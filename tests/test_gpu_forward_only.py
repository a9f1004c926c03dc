"""dvgo_params.forward_only (the BF16 tensor-core path keeps its input panels for the backward
unless no backward follows).  With the flag the workspace is smaller by 16 KiB per 128 samples and
the forward renders the same colours; a backward after such a forward gathers its inputs again and
gives the gradients of the cached path -- also when the backward is called without the flag on a
workspace that has room for the panels (the forward records that it did not store them).
Gradients are compared up to the run-to-run order of the FP32 atomics."""
import numpy as np
import pytest
import torch

from test_gpu_parity import _fine_inputs, _mlp_flat, cuda

pytestmark = pytest.mark.gpu

dvgo = pytest.importorskip("paper_2111_11215_gb300")
B = dvgo.binding


def _close(a, b, name):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    np.testing.assert_allclose(a, b, rtol=1e-4, atol=1e-5 * np.abs(b).max(), err_msg=name)


def test_forward_only_skips_the_panels_and_the_backward_gathers():
    res, R = 32, 1500
    dens, feat, mlp, o, d, jit, _ = _fine_inputs(res, R, seed=180)
    p = dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=2.0 / res * 0.5, bg=(1.0, 1.0, 1.0), mlp_prec=dvgo.DVGO_MLP_BF16,
                    shift_b=dvgo.dvgo_shift_from_alpha_init(1e-2, 2.0 / res))
    dd = dvgo.GridDesc((res,) * 3, 1)
    cd = dvgo.GridDesc((res,) * 3, 12, dtype=dvgo.DVGO_DTYPE_BF16)
    D, F = cuda(dens), cuda(feat).to(torch.bfloat16)
    views = dvgo.render.mlp_views(cuda(_mlp_flat(mlp)))
    ro, rd, jt = cuda(o), cuda(d), cuda(jit)
    gC = cuda(np.random.default_rng(181).normal(scale=1e-2, size=(R, 3)))
    p_fo = p.with_(forward_only=1)
    n_full, n_fo = B.dvgo_workspace_size(p, dd, R), B.dvgo_workspace_size(p_fo, dd, R)
    assert n_full - n_fo >= 16384 * (R // 128)          # at least one 16 KiB panel per 128 rays

    def run(rend, p_fwd, p_bwd):
        g = [torch.zeros_like(D), torch.zeros(F.shape, device="cuda"), torch.zeros(views_numel(), device="cuda")]
        rgb, tf = torch.empty((R, 3), device="cuda"), torch.empty(R, device="cuda")
        B.dvgo_render_fwd(p_fwd, dd, D, cd, F, views, ro, rd, jt, None, None, rgb, tf, None, None, rend.workspace)
        B.dvgo_render_bwd(p_bwd, dd, D, cd, F, views, ro, rd, jt, None, gC, None, g[0], g[1], g[2], rend.workspace)
        torch.cuda.synchronize()
        return rgb, g

    def views_numel():
        return _mlp_flat(mlp).size

    full, small = dvgo.Renderer(p, dd, cd, R), dvgo.Renderer(p_fo, dd, cd, R)
    assert small.workspace.numel() == n_fo and full.workspace.numel() == n_full
    rgb_c, g_c = run(full, p, p)                 # panels stored and reloaded
    rgb_g, g_g = run(small, p_fo, p_fo)          # no panels: the backward gathers
    rgb_m, g_m = run(full, p_fo, p)              # forward without panels, backward allowed to use them
    np.testing.assert_array_equal(rgb_g.cpu().numpy(), rgb_c.cpu().numpy())
    np.testing.assert_array_equal(rgb_m.cpu().numpy(), rgb_c.cpu().numpy())
    for name, a, b in (("density", g_g[0], g_c[0]), ("feat", g_g[1], g_c[1]), ("mlp", g_g[2], g_c[2])):
        _close(a, b, "gather vs cached: " + name)
    for name, a, b in (("density", g_m[0], g_c[0]), ("feat", g_m[1], g_c[1]), ("mlp", g_m[2], g_c[2])):
        _close(a, b, "mixed flags vs cached: " + name)
