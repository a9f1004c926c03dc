"""dvgo_params.cgrid_ready and density_ready: the render calls make their stream wait on the caller's event right
before their first kernel that reads the colour / feature grid.  A side stream sleeps (a bounded
spin of ~25 ms), then overwrites the feature grid and records the event; a forward given that event
on the main stream must render the new grid as a forward issued after a full synchronisation
does (same kernels, same inputs: equal to 1e-6), for the FP32 SIMT and the BF16 tensor-core
colour kernels."""
import numpy as np
import pytest
import torch

from test_gpu_parity import _fine_inputs, _mlp_flat, cuda

pytestmark = pytest.mark.gpu

dvgo = pytest.importorskip("paper_2111_11215_gb300")


@pytest.mark.parametrize("prec", [dvgo.DVGO_MLP_FP32, dvgo.DVGO_MLP_BF16])
def test_forward_waits_for_cgrid_event(prec):
    res, R = 24, 512
    dens, feat, mlp, o, d, jit, _ = _fine_inputs(res, R, seed=170)
    feat_new = np.random.default_rng(171).normal(scale=0.5, size=feat.shape).astype(np.float32)
    bf = prec == dvgo.DVGO_MLP_BF16
    dt = torch.bfloat16 if bf else torch.float32
    p = dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=2.0 / res * 0.5, bg=(1.0, 1.0, 1.0), mlp_prec=prec,
                    shift_b=dvgo.dvgo_shift_from_alpha_init(1e-2, 2.0 / res))
    dd = dvgo.GridDesc((res,) * 3, 1)
    cd = dvgo.GridDesc((res,) * 3, 12, dtype=dvgo.DVGO_DTYPE_BF16 if bf else dvgo.DVGO_DTYPE_F32)
    rend = dvgo.Renderer(p, dd, cd, R)
    D, views = cuda(dens), dvgo.render.mlp_views(cuda(_mlp_flat(mlp)))
    ro, rd, jt = cuda(o), cuda(d), cuda(jit)
    new = cuda(feat_new).to(dt)
    # references: the new and the old grid, everything synchronised
    ref = rend.forward(D, new, views, ro, rd, jt)[0].clone()
    cgrid = cuda(feat).to(dt)
    old = rend.forward(D, cgrid, views, ro, rd, jt)[0].clone()
    torch.cuda.synchronize()
    assert float((ref - old).abs().max()) > 1e-2          # the two grids render differently
    main, side = torch.cuda.current_stream(), torch.cuda.Stream()
    ev = torch.cuda.Event()
    side.wait_stream(main)
    with torch.cuda.stream(side):
        torch.cuda._sleep(50_000_000)
        cgrid.copy_(new)
        ev.record(side)
    got = rend.forward(D, cgrid, views, ro, rd, jt, cgrid_ready=ev)[0]
    main.wait_stream(side)
    torch.cuda.synchronize()
    np.testing.assert_allclose(got.cpu().numpy(), ref.cpu().numpy(), rtol=0, atol=1e-6)


@pytest.mark.parametrize("prec", [dvgo.DVGO_MLP_FP32, dvgo.DVGO_MLP_BF16])
def test_forward_waits_for_density_event(prec):
    """dvgo_params.density_ready: the same for the density grid -- the stream waits on the event
    right before the density pass (the ray set-up and the sample scan do not)."""
    res, R = 24, 512
    dens, feat, mlp, o, d, jit, _ = _fine_inputs(res, R, seed=172)
    dens_new = np.random.default_rng(173).normal(scale=3.0, size=dens.shape).astype(np.float32)
    bf = prec == dvgo.DVGO_MLP_BF16
    dt = torch.bfloat16 if bf else torch.float32
    p = dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=2.0 / res * 0.5, bg=(1.0, 1.0, 1.0), mlp_prec=prec,
                    shift_b=dvgo.dvgo_shift_from_alpha_init(1e-2, 2.0 / res))
    dd = dvgo.GridDesc((res,) * 3, 1)
    cd = dvgo.GridDesc((res,) * 3, 12, dtype=dvgo.DVGO_DTYPE_BF16 if bf else dvgo.DVGO_DTYPE_F32)
    rend = dvgo.Renderer(p, dd, cd, R)
    F, views = cuda(feat).to(dt), dvgo.render.mlp_views(cuda(_mlp_flat(mlp)))
    ro, rd, jt = cuda(o), cuda(d), cuda(jit)
    new = cuda(dens_new)
    ref = rend.forward(new, F, views, ro, rd, jt)[0].clone()
    D = cuda(dens)
    old = rend.forward(D, F, views, ro, rd, jt)[0].clone()
    torch.cuda.synchronize()
    assert float((ref - old).abs().max()) > 1e-2          # the two density grids render differently
    main, side = torch.cuda.current_stream(), torch.cuda.Stream()
    ev = torch.cuda.Event()
    side.wait_stream(main)
    with torch.cuda.stream(side):
        torch.cuda._sleep(50_000_000)
        D.copy_(new)
        ev.record(side)
    got = rend.forward(D, F, views, ro, rd, jt, density_ready=ev)[0]
    main.wait_stream(side)
    torch.cuda.synchronize()
    np.testing.assert_allclose(got.cpu().numpy(), ref.cpu().numpy(), rtol=0, atol=1e-6)
