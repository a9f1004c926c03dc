"""GPU parity of the touched-lattice-point count (dvgo_touched_points) against the FP64 oracle's
marks: bit for bit, after a uniform forward with tau_f skipping, after a forward with the known
free space of a coarse grid, and after an explicit-sample forward.  (Integer results: exact; the
GPU's cells come from the fixed-point coordinate, the oracle's from FP64, which differ only within
~3e-10 lattice units of a lattice plane.)"""
import numpy as np
import pytest
import torch

import oracle
from helpers import oracle_params
from test_gpu_freespace import _freespace, _robust_rays
from test_gpu_parity import _fine_inputs, _mlp_flat, cuda

pytestmark = pytest.mark.gpu

dvgo = pytest.importorskip("paper_2111_11215_gb300")


def _bits(bm, shape):
    n = int(np.prod(shape))
    b = np.unpackbits(bm.cpu().numpy().view(np.uint8), bitorder="little")
    return b[:n].reshape(shape).astype(bool)


def _gpu_marks(p, res, dens, feat, mlp, o, d, jit, samples=None):
    dd, cd = dvgo.GridDesc((res,) * 3, 1), dvgo.GridDesc((res,) * 3, 12)
    R = o.shape[0]
    r = dvgo.Renderer(p, dd, cd, R, samples_per_ray=None if samples is None else samples[0].shape[1])
    sm = None if samples is None else (cuda(samples[0]), cuda(samples[1]))
    r.forward(cuda(dens), cuda(feat), dvgo.render.mlp_views(cuda(_mlp_flat(mlp))), cuda(o), cuda(d),
              None if jit is None else cuda(jit), sm)
    bm, counts = dvgo.dvgo_touched_points(p, dd, R, sm, r.workspace)
    torch.cuda.synchronize()
    return _bits(bm[0], (res,) * 3), _bits(bm[1], (res,) * 3), counts.cpu().numpy()


def _check(got, ref):
    dm, fm, counts = got
    assert counts[0] == dm.sum() and counts[1] == fm.sum()
    assert np.array_equal(dm, ref.touched["density"]), (dm.sum(), ref.touched["density"].sum(),
                                                        (dm != ref.touched["density"]).sum())
    assert np.array_equal(fm, ref.touched["cgrid"]), (fm.sum(), ref.touched["cgrid"].sum(),
                                                      (fm != ref.touched["cgrid"]).sum())
    assert not np.any(fm & ~dm)         # a kept sample's corners are density corners too
    return dm, fm


def test_touched_after_a_uniform_forward_with_tau_f():
    res, R = 28, 400
    dens, feat, mlp, o, d, jit, _ = _fine_inputs(res, R, seed=200)
    p = dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=2.0 / res * 0.5, bg=(1.0, 1.0, 1.0), tau_f=1e-3,
                    shift_b=dvgo.dvgo_shift_from_alpha_init(1e-4, 2.0 / res))
    ref = oracle.render(oracle_params(p, (res,) * 3, 12), dens, feat, o, d, jitter=jit, mlp=mlp, touched=True)
    dm, fm = _check(_gpu_marks(p, res, dens, feat, mlp, o, d, jit), ref)
    assert fm.sum() < dm.sum()          # tau_f removed samples


def test_touched_with_the_known_free_space():
    fs_gpu, fs_ora = _freespace()
    res, R = 24, 300
    dens, feat, mlp, o, d, jit, _ = _fine_inputs(res, R, seed=210)
    p = dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=2.0 / res * 0.5, bg=(1.0, 1.0, 1.0), tau_f=1e-4,
                    shift_b=dvgo.dvgo_shift_from_alpha_init(1e-2, 2.0 / res), freespace=fs_gpu)
    P = oracle_params(p, (res,) * 3, 12)
    keep, skipped, _ = _robust_rays(P, fs_ora, o, d, jit)
    assert skipped > 100
    o, d, jit = o[keep], d[keep], jit[keep]
    ref = oracle.render(P, dens, feat, o, d, jitter=jit, mlp=mlp, freespace=fs_ora, touched=True)
    _check(_gpu_marks(p, res, dens, feat, mlp, o, d, jit), ref)


def test_touched_after_an_explicit_sample_forward():
    res, R, K = 20, 96, 48
    dens, feat, mlp, o, d, _, _ = _fine_inputs(res, R, seed=220)
    p = dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=0.05, shift_b=-1.0, bg=(0.3, 0.3, 0.3), tau_f=1e-3)
    P = oracle_params(p, (res,) * 3, 12)
    base = oracle.render(P, dens, feat, o, d, mlp=mlp)
    g = np.random.default_rng(221)
    u = np.sort(g.uniform(size=(R, K)), axis=1)
    t0, t1 = base.t_enter[:, None], base.t_exit[:, None]
    ts = np.where(t1 > t0, t0 + u * (t1 - t0), 0.0).astype(np.float32)
    dts = np.diff(np.concatenate([ts, ts[:, -1:] + 0.01], axis=1), axis=1).astype(np.float32)
    ref = oracle.render(P, dens, feat, o, d, mlp=mlp, explicit_t=ts, explicit_dt=dts, touched=True)
    _check(_gpu_marks(p, res, dens, feat, mlp, o, d, None, (ts, dts)), ref)
