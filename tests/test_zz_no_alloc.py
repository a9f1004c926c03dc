"""The allocation-free coarse forward (dvgo_render_fwd_noalloc) against the workspace entry point.

dvgo_render_fwd_noalloc serves callers that cannot allocate device memory (a plugin whose host
application owns the device's memory, a real-time loop that forbids allocation, a binding with
no device allocator): its scratch is a static array inside the library instead of a workspace.
This test calls it through the C ABI twice in a row, on different inputs, and checks each result
against dvgo_render_fwd with an allocated workspace; it also checks that a batch above the
static capacity is rejected without touching the outputs.  The file is named so that pytest
collects it last.
"""
import numpy as np
import pytest
import torch

import synth
from helpers import RTOL_COLOUR, assert_close

pytestmark = pytest.mark.gpu

dvgo = pytest.importorskip("paper_2111_11215_gb300")


@pytest.fixture(scope="module", autouse=True)
def _built_library():
    from paper_2111_11215_gb300 import build_lib
    build_lib.build()


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float32).cuda()


def _with_workspace(p, dd, cd, dens, rgbg, ro, rd, jit, tgt):
    R = ro.shape[0]
    ws = torch.empty(dvgo.dvgo_workspace_size(p, dd, R), dtype=torch.uint8, device="cuda")
    rgb, tf = torch.empty((R, 3), device="cuda"), torch.empty(R, device="cuda")
    loss, dl = torch.empty(1, device="cuda"), torch.empty((R, 3), device="cuda")
    dvgo.dvgo_render_fwd(p, dd, dens, cd, rgbg, None, ro, rd, jit, None, tgt, rgb, tf, loss, dl, ws)
    return rgb, tf, loss, dl


def _no_alloc(p, dd, cd, dens, rgbg, ro, rd, jit, tgt):
    R = ro.shape[0]
    rgb, tf = torch.full((R, 3), -1.0, device="cuda"), torch.full((R,), -1.0, device="cuda")
    loss, dl = torch.full((1,), -1.0, device="cuda"), torch.full((R, 3), -1.0, device="cuda")
    dvgo.dvgo_render_fwd_noalloc(p, dd, dens, cd, rgbg, ro, rd, jit, tgt, rgb, tf, loss, dl)
    return rgb, tf, loss, dl


def test_no_alloc_forward_matches_workspace_forward_twice():
    cases = [(synth.coarse_case(seed=40, n_rays=4096), 0.03125, dvgo.dvgo_shift_from_alpha_init(1e-6, 0.0625), 0),
             (synth.coarse_case(seed=41, res=24, n_rays=1500), 0.05, 0.3, 1)]
    for case, step, b, act in cases:   # two calls in a row on the one static scratch
        res = case["density"].shape[0]
        dd, cd = dvgo.GridDesc((res,) * 3, 1), dvgo.GridDesc((res,) * 3, 3)
        p = dvgo.Params(mode=dvgo.DVGO_MODE_COARSE, step=step, shift_b=b, bg=(1.0, 0.5, 0.25), rgb_act=act)
        R = case["rays_o"].shape[0]
        args = (_dev(case["density"]), _dev(case["rgb"]), _dev(case["rays_o"]), _dev(case["rays_d"]),
                _dev(synth.jitter(R, 3)), _dev(case["target"]))
        ref = _with_workspace(p, dd, cd, *args)
        got = _no_alloc(p, dd, cd, *args)
        torch.cuda.synchronize()
        for name, g, r in zip(("rgb", "tfinal", "loss", "dloss"), got, ref):
            assert_close(g.cpu().numpy(), r.cpu().numpy(), RTOL_COLOUR, name)


def test_no_alloc_at_capacity_matches_workspace_forward():
    """A batch of exactly DVGO_NOALLOC_MAX_RAYS rays fits the static scratch (every block of the
    coarse workspace layout for that many rays, the unused target block included)."""
    R = dvgo.binding.DVGO_NOALLOC_MAX_RAYS
    case = synth.coarse_case(seed=42, res=16, n_rays=R)
    dd, cd = dvgo.GridDesc((16,) * 3, 1), dvgo.GridDesc((16,) * 3, 3)
    p = dvgo.Params(mode=dvgo.DVGO_MODE_COARSE, step=0.0625, shift_b=0.1, bg=(1.0, 1.0, 1.0))
    assert dvgo.dvgo_workspace_size(p, dd, R) <= dvgo.binding.DVGO_NOALLOC_SCRATCH_BYTES
    args = (_dev(case["density"]), _dev(case["rgb"]), _dev(case["rays_o"]), _dev(case["rays_d"]),
            _dev(synth.jitter(R, 4)), _dev(case["target"]))
    ref = _with_workspace(p, dd, cd, *args)
    got = _no_alloc(p, dd, cd, *args)
    torch.cuda.synchronize()
    for name, g, r in zip(("rgb", "tfinal", "loss", "dloss"), got, ref):
        assert_close(g.cpu().numpy(), r.cpu().numpy(), RTOL_COLOUR, name)


def test_no_alloc_rejects_batches_above_capacity():
    res = 8
    dd, cd = dvgo.GridDesc((res,) * 3, 1), dvgo.GridDesc((res,) * 3, 3)
    p = dvgo.Params(mode=dvgo.DVGO_MODE_COARSE, step=0.1)
    R = dvgo.binding.DVGO_NOALLOC_MAX_RAYS + 1
    dens = torch.zeros(res ** 3, device="cuda")
    rgbg = torch.zeros(res ** 3 * 3, device="cuda")
    ro = torch.zeros((R, 3), device="cuda")
    rd = torch.ones((R, 3), device="cuda")
    rgb = torch.full((R, 3), 7.0, device="cuda")
    with pytest.raises(dvgo.DVGOError) as ei:
        dvgo.dvgo_render_fwd_noalloc(p, dd, dens, cd, rgbg, ro, rd, None, None, rgb, None, None, None)
    assert ei.value.status == -6
    torch.cuda.synchronize()
    assert bool(torch.all(rgb == 7.0))
