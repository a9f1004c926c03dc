"""Early ray termination in the fine density pass: a sample whose transmittance, formed exactly as
the compositing pass forms it, is 0 in FP32 has weight 0 and no gradient, so it is left out of the
colour kernels.  On a ball of raw density 120 and radius 0.7 (optical depth ~3.3 per step, and
each ray crosses at least ~40 steps of it) most samples lie behind that point; the render and its gradients still match the FP64 oracle (which never
terminates: its transmittance does not underflow), with both colour paths, uniform and explicit
samples.

Tolerances: colours, feature and MLP gradients at the FP32 bounds of the other parity tests.  The
density gradient of rays probing a dense ball is built from differences of FP32 MLP colours and
is checked like the others against 1e-4 max(|ref|, 1 % of the largest) plus the oracle's running
error bound of the FP32 path, which carries the FP32 colour error through those differences
(errors are the same with termination switched off: relative L2 1.38e-5, worst element 2.2e-4
relative at 6 % of the largest), and its relative L2 error must stay below 2e-5."""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import BOUND_FP32, RTOL_COLOUR, assert_close, assert_within_bound, mlp_flat, oracle_params
from test_gpu_parity import _counts, _mlp_flat, cuda

pytestmark = pytest.mark.gpu

dvgo = pytest.importorskip("paper_2111_11215_gb300")


def _kept(workspace):
    """Samples the last forward kept (the third int of the workspace header)."""
    return int(workspace[8:12].view(torch.int32).item())


@pytest.mark.parametrize("prec", [dvgo.DVGO_MLP_FP32, dvgo.DVGO_MLP_BF16])
@pytest.mark.parametrize("explicit", [False, True])
def test_terminated_rays_match_the_oracle(prec, explicit):
    res, R = 32, 256
    dens = synth.sphere_density(res, [(0.0, 0.05, -0.05)], [0.7], 120.0).astype(np.float32)
    # random features: with a smooth field the colour hardly changes along a ray inside the ball and
    # the density gradient, built from colour differences, is ill-conditioned for FP32 colours
    feat = synth.normal_grid((res,) * 3, 12, 0.5, 260)
    mlp = synth.mlp_weights(39, 128, 3, 261)
    o, d = synth.blob_rays(R, seed=262, blob_radius=0.3)
    jit = synth.jitter(R, 263)
    p = dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=2.0 / res * 0.5, bg=(1.0, 1.0, 1.0), mlp_prec=prec,
                    shift_b=dvgo.dvgo_shift_from_alpha_init(1e-6, 2.0 / res))
    P = oracle_params(p, (res,) * 3, 12)
    samples = None
    if explicit:
        base = oracle.render(P, dens, feat, o, d, mlp=mlp)
        g = np.random.default_rng(264)
        u = np.sort(g.uniform(size=(R, 96)), axis=1)
        t0, t1 = base.t_enter[:, None], base.t_exit[:, None]
        ts = np.where(t1 > t0, t0 + u * (t1 - t0), 0.0).astype(np.float32)
        dts = np.diff(np.concatenate([ts, ts[:, -1:] + 0.01], axis=1), axis=1).astype(np.float32)
        samples = (ts, dts)
    dd, cd = dvgo.GridDesc((res,) * 3, 1), dvgo.GridDesc((res,) * 3, 12)
    r = dvgo.Renderer(p, dd, cd, R, samples_per_ray=None if samples is None else 96)
    flat = cuda(_mlp_flat(mlp))
    views = dvgo.render.mlp_views(flat)
    D, F = cuda(dens), cuda(feat)
    sm = None if samples is None else (cuda(samples[0]), cuda(samples[1]))
    rgb, tf, _ = r.forward(D, F, views, cuda(o), cuda(d), cuda(jit), sm)
    kept = _kept(r.workspace)
    counts, total = _counts(r, R)
    gC = np.random.default_rng(265).normal(scale=1e-2, size=(R, 3))
    g_d, g_f, g_m = torch.zeros_like(D), torch.zeros_like(F), torch.zeros_like(flat)
    r.backward(D, F, views, cuda(o), cuda(d), cuda(jit), sm, cuda(gC), None, g_d, g_f, g_m)
    torch.cuda.synchronize()
    kw = dict(explicit_t=samples[0], explicit_dt=samples[1]) if explicit else dict(jitter=jit)
    ref = oracle.render(P, dens, feat, o, d, mlp=mlp, grad_rgb=gC, error_bound=BOUND_FP32, **kw)
    assert kept < 0.8 * total, (kept, total)             # a good part of the samples lies behind the termination point
    assert np.all(tf.cpu().numpy() == 0.0)                # every ray ends inside the ball
    if prec == dvgo.DVGO_MLP_FP32:
        assert_close(rgb.cpu().numpy(), ref.rgb, RTOL_COLOUR, "rgb")
        gd, rd = g_d.cpu().numpy(), ref.grads["density"]
        assert np.linalg.norm(gd - rd) <= 2e-5 * np.linalg.norm(rd)
        assert_within_bound(gd, rd, ref.bounds["density"], "grad_density")
        assert_within_bound(g_f.cpu().numpy(), ref.grads["cgrid"], ref.bounds["cgrid"], "grad_feat")
        assert_within_bound(g_m.cpu().numpy(), mlp_flat(ref.grads), mlp_flat(ref.bounds), "grad_mlp")
    else:
        assert np.abs(rgb.cpu().numpy() - ref.rgb).max() < 1e-2
        rd = g_d.cpu().numpy() - ref.grads["density"]
        assert np.linalg.norm(rd) <= 5e-2 * np.linalg.norm(ref.grads["density"])
