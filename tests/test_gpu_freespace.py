"""GPU parity of the known-free-space test and the fine-box allocation (Sec. 4.2) against the FP64
oracle.  The skip decision compares the coarse alpha with tau_c in FP32 on the GPU and in FP64 in
the oracle, so rays with a sample whose coarse alpha lies within 1e-3 (relative) of tau_c are
left out of the comparison (they are counted, and must be few); every other ray must match at the
FP32 tolerances, colours and gradients."""
import numpy as np
import pytest
import torch

import oracle
from helpers import BOUND_FP32, RTOL_COLOUR, assert_close, assert_within_bound, mlp_flat, oracle_params
from test_gpu_parity import _fine_inputs, _mlp_flat, _run_fine, cuda
from test_oracle_freespace import _coarse

pytestmark = pytest.mark.gpu

dvgo = pytest.importorskip("paper_2111_11215_gb300")

TAU_C = 1e-3


def _freespace(res_c=12, box=((-1.0,) * 3, (1.0,) * 3)):
    v = _coarse(res_c, r_in=0.55, r_out=0.8, v_in=20.0).astype(np.float32)
    b_c = float(np.float32(dvgo.dvgo_shift_from_alpha_init(1e-6, 2.0 / res_c)))
    step_c = float(np.float32(2.0 / res_c / 2))
    fs_gpu = dvgo.FreeSpace(density=cuda(v), desc=dvgo.GridDesc((res_c,) * 3, 1, box[0], box[1]), shift_b=b_c,
                            step=step_c, tau=TAU_C)
    fs_ora = oracle.FreeSpace(density=v.astype(np.float64), xyz_min=box[0], xyz_max=box[1], shift_b=b_c,
                              delta=step_c, tau=float(np.float32(TAU_C)))
    return fs_gpu, fs_ora


def _robust_rays(P, fs_ora, o, d, jit, band=1e-3):
    """Rays none of whose uniform samples has a coarse alpha within `band` (relative) of tau_c."""
    keep, skipped, kept = [], 0, 0
    for r in range(o.shape[0]):
        _, t0, t1, dn, n = oracle.ray_bounds(P, o[r], d[r], float(jit[r]))
        t = t0 + (np.arange(n) + float(jit[r])) * P.delta
        a = np.array([oracle.coarse_alpha(fs_ora, o[r].astype(np.float64) + tk * dn) for tk in t])
        if n and np.any(np.abs(a - fs_ora.tau) < band * fs_ora.tau):
            continue
        keep.append(r)
        skipped += int((a < fs_ora.tau).sum())
        kept += int((a >= fs_ora.tau).sum())
    return np.array(keep), skipped, kept


@pytest.mark.parametrize("feat_dtype", [torch.float32, torch.bfloat16])
def test_fine_freespace_parity(feat_dtype):
    res, R = 24, 400
    dens, feat, mlp, o, d, jit, _ = _fine_inputs(res, R, seed=30)
    if feat_dtype == torch.bfloat16:
        feat = torch.as_tensor(feat).to(torch.bfloat16).float().numpy()
    fs_gpu, fs_ora = _freespace()
    p = dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=2.0 / res * 0.5, bg=(1.0, 1.0, 1.0), mlp_prec=dvgo.DVGO_MLP_FP32,
                    shift_b=dvgo.dvgo_shift_from_alpha_init(1e-2, 2.0 / res), freespace=fs_gpu)
    P = oracle_params(p, (res,) * 3, 12)
    idx, skipped, kept = _robust_rays(P, fs_ora, o, d, jit)
    assert len(idx) >= 0.95 * R and skipped > 2000 and kept > 400    # both branches, few rays left out
    o, d, jit = o[idx], d[idx], jit[idx]
    g = np.random.default_rng(31)
    gC = g.normal(scale=1e-2, size=(len(idx), 3))
    got = _run_fine(p, res, dens, feat, mlp, o, d, jit, gC, np.zeros(len(idx)), feat_dtype)
    ref = oracle.render(P, dens, feat, o, d, jitter=jit, mlp=mlp, grad_rgb=gC, freespace=fs_ora,
                        error_bound=BOUND_FP32)
    np.testing.assert_array_equal(got["counts"], ref.n_samples)     # skipping keeps the sample grid
    assert_close(got["rgb"], ref.rgb, RTOL_COLOUR, "rgb")
    assert_close(got["tfinal"], ref.tfinal, RTOL_COLOUR, "tfinal")
    assert_within_bound(got["g_d"], ref.grads["density"], ref.bounds["density"], "grad_density")
    assert_within_bound(got["g_f"], ref.grads["cgrid"], ref.bounds["cgrid"], "grad_feat")
    assert_within_bound(got["g_m"], mlp_flat(ref.grads), mlp_flat(ref.bounds), "grad_mlp")
    # the test is not vacuous: skipping changes the render
    no_fs = oracle.render(P, dens, feat, o, d, jitter=jit, mlp=mlp, grad_rgb=gC)
    assert np.abs(no_fs.rgb - ref.rgb).max() > 1e-3


def test_fine_freespace_bf16_mlp_and_offset_boxes():
    """BF16 tensor-core colour kernels read the same compact list; the coarse grid on a box that
    differs from the fine one exercises the fixed-point map between the lattices."""
    res, R = 20, 256
    dens, feat, mlp, o, d, jit, _ = _fine_inputs(res, R, seed=32)
    box_c = ((-1.1, -0.9, -1.2), (0.95, 1.2, 1.05))
    fs_gpu, fs_ora = _freespace(res_c=13, box=box_c)
    for prec, tol in ((dvgo.DVGO_MLP_FP32, None), (dvgo.DVGO_MLP_BF16, 1e-2)):
        p = dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=2.0 / res * 0.5, bg=(1.0, 1.0, 1.0), mlp_prec=prec,
                        shift_b=dvgo.dvgo_shift_from_alpha_init(1e-2, 2.0 / res), freespace=fs_gpu)
        P = oracle_params(p, (res,) * 3, 12)
        idx, skipped, kept = _robust_rays(P, fs_ora, o, d, jit)
        assert len(idx) >= 0.95 * R and skipped > 2000 and kept > 300
        got = _run_fine(p, res, dens, feat, mlp, o[idx], d[idx], jit[idx], None, None, bwd=False)
        ref = oracle.render(P, dens, feat, o[idx], d[idx], jitter=jit[idx], mlp=mlp, freespace=fs_ora)
        if tol is None:
            assert_close(got["rgb"], ref.rgb, RTOL_COLOUR, "rgb_fp32")
        else:
            assert np.abs(got["rgb"] - ref.rgb).max() < tol


def test_unknown_bbox_matches_oracle():
    for res_c, seed in ((12, 70), (17, 71), (33, 72)):
        v = _coarse(res_c, seed).astype(np.float32)
        b = float(np.float32(-3.0))
        a_lat = -np.expm1(-np.logaddexp(0.0, v.astype(np.float64) + b) * 0.05)
        assert np.abs(a_lat / TAU_C - 1.0).min() > 1e-4                 # no lattice value on the threshold
        fs = dvgo.FreeSpace(density=cuda(v), desc=dvgo.GridDesc((res_c,) * 3, 1), shift_b=b, step=0.05, tau=TAU_C)
        out = dvgo.dvgo_unknown_bbox(fs).cpu().numpy()
        n, lo, hi = oracle.unknown_bbox(oracle.FreeSpace(density=v.astype(np.float64), shift_b=b, delta=0.05,
                                                         tau=float(np.float32(TAU_C))))
        assert n > 0 and out[0] == n and tuple(out[1:4]) == lo and tuple(out[4:7]) == hi
    # all known free
    v = np.full((9, 9, 9), -40.0, np.float32)
    fs = dvgo.FreeSpace(density=cuda(v), desc=dvgo.GridDesc((9, 9, 9), 1), shift_b=0.0, step=0.05, tau=TAU_C)
    assert int(dvgo.dvgo_unknown_bbox(fs)[0].item()) == 0
