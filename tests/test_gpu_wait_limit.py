"""Failure detection of the tensor-core colour kernels without a GPU fault: every device-side wait
of those kernels is bounded (dvgo_params.wait_limit_us), and a testing aid withholds one producer
arrival on a chosen tile (dvgo_params.test_withhold_tile) -- a barrier phase that nothing
completes -- so that the consumers' wait for that tile runs out.  The kernel must then return
(no hang), report the timeout through the workspace flag word (dvgo_workspace_status ->
DVGO_ERR_DEVICE), and leave the context usable: the next clean call on the same workspace must
succeed with the clean results, which also shows that the failed CTA released its tensor memory
(every CTA of the next launch allocates its full share of it on its SM)."""
import time

import numpy as np
import pytest
import torch

from test_gpu_parity import _fine_inputs, _mlp_flat, cuda

pytestmark = pytest.mark.gpu

dvgo = pytest.importorskip("paper_2111_11215_gb300")

LIMIT_US = 20000          # 20 ms: far above any wait of a healthy launch here, far below the 2 s default


def _setup():
    res, R = 24, 2000
    dens, feat, mlp, o, d, jit, _ = _fine_inputs(res, R, seed=700)
    p = dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=2.0 / res * 0.5, bg=(1.0, 1.0, 1.0), mlp_prec=dvgo.DVGO_MLP_BF16,
                    shift_b=dvgo.dvgo_shift_from_alpha_init(1e-2, 2.0 / res))
    dd, cd = dvgo.GridDesc((res,) * 3, 1), dvgo.GridDesc((res,) * 3, 12)
    flat = cuda(_mlp_flat(mlp))
    views = dvgo.render.mlp_views(flat)
    gC = cuda(np.random.default_rng(701).normal(scale=1e-2, size=(R, 3)))
    t = dict(D=cuda(dens), F=cuda(feat), views=views, flat=flat, o=cuda(o), d=cuda(d), jit=cuda(jit), gC=gC)
    return p, dd, cd, R, t


def _step(r, t, bwd=True):
    rgb, tf, _ = r.forward(t["D"], t["F"], t["views"], t["o"], t["d"], t["jit"])
    out = {"rgb": rgb.clone()}
    if bwd:
        g_d, g_f, g_m = torch.zeros_like(t["D"]), torch.zeros_like(t["F"]), torch.zeros_like(t["flat"])
        r.backward(t["D"], t["F"], t["views"], t["o"], t["d"], t["jit"], None, t["gC"], None, g_d, g_f, g_m)
        out.update(g_d=g_d, g_f=g_f, g_m=g_m)
    torch.cuda.synchronize()
    return out


def test_bounded_wait_runs_out_reports_and_leaves_the_context_usable():
    p, dd, cd, R, t = _setup()
    clean = dvgo.Renderer(p, dd, cd, R)
    ref = _step(clean, t)
    assert dvgo.dvgo_workspace_status(clean.workspace) == 0
    n_tiles = -(-int(clean.workspace[8:12].view(torch.int32).item()) // 128)
    assert n_tiles > 160            # the withheld tile's CTA has later tiles that it must abandon

    # a clean forward, then a backward whose wait runs out: the call returns, the flag word reports it
    faulty = dvgo.Renderer(p, dd, cd, R)
    rgb, _, _ = faulty.forward(t["D"], t["F"], t["views"], t["o"], t["d"], t["jit"])
    torch.cuda.synchronize()
    assert torch.equal(rgb, ref["rgb"]) and dvgo.dvgo_workspace_status(faulty.workspace) == 0
    faulty.params = p.with_(wait_limit_us=LIMIT_US, test_withhold_tile=4)
    g_m = torch.zeros_like(t["flat"])
    t0 = time.perf_counter()
    faulty.backward(t["D"], t["F"], t["views"], t["o"], t["d"], t["jit"], None, t["gC"], None, torch.zeros_like(t["D"]),
                    torch.zeros_like(t["F"]), g_m)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert dvgo.dvgo_workspace_status(faulty.workspace) == dvgo.binding.DVGO_ERR_DEVICE
    assert dt < 2.0, dt             # a few waits of 20 ms, not the 2 s default
    assert not torch.equal(g_m, ref["g_m"])            # that CTA's weight gradients were never added

    # the next clean forward clears the flag, and a clean backward gives the clean gradients
    again = _step(dvgo.Renderer(p, dd, cd, R), t)
    for k in ("g_d", "g_f", "g_m"):
        # (FP32 atomics add in a different order from run to run)
        torch.testing.assert_close(again[k], ref[k], rtol=1e-4, atol=1e-5 * float(ref[k].abs().max()))
    faulty.params = p
    reuse = _step(faulty, t)
    assert dvgo.dvgo_workspace_status(faulty.workspace) == 0
    torch.testing.assert_close(reuse["g_m"], ref["g_m"], rtol=1e-4, atol=1e-5 * float(ref["g_m"].abs().max()))


def test_bounded_wait_in_the_forward_colour_kernel():
    p, dd, cd, R, t = _setup()
    clean = dvgo.Renderer(p, dd, cd, R)
    ref = _step(clean, t, bwd=False)
    faulty = dvgo.Renderer(p.with_(wait_limit_us=LIMIT_US, test_withhold_tile=7), dd, cd, R)
    faulty.workspace.zero_()        # abandoned tiles leave their sample colours at 0
    bad = _step(faulty, t, bwd=False)
    assert dvgo.dvgo_workspace_status(faulty.workspace) == dvgo.binding.DVGO_ERR_DEVICE
    assert not torch.equal(bad["rgb"], ref["rgb"])      # the abandoned tiles' colours were never written
    faulty.params = p
    again = _step(faulty, t, bwd=False)
    assert dvgo.dvgo_workspace_status(faulty.workspace) == 0
    assert torch.equal(again["rgb"], ref["rgb"])
