"""GPU parity of the lazy Adam variant (dvgo_adam_step with skip_zero_grad) against the oracle:
all-zero 4-element vectors (skipped without touching p, m, v), vectors with some zero elements,
a ragged scalar tail, the BF16 copy, and a FineModel that trains with it (only the touched grid
points move)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import assert_close
from test_gpu_parity import _mlp_flat, cuda

pytestmark = pytest.mark.gpu

dvgo = pytest.importorskip("paper_2111_11215_gb300")


def test_lazy_adam_matches_oracle():
    g = np.random.default_rng(240)
    n = 4099                                            # a ragged tail of 3 elements
    p0 = g.normal(size=n).astype(np.float32)
    P, M, V = cuda(p0), torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    pb = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    Gd = torch.zeros(n, device="cuda")
    po, mo, vo = p0.astype(np.float64), np.zeros(n), np.zeros(n)
    for t in range(1, 5):
        grad = g.normal(size=n).astype(np.float32)
        grad[np.repeat(g.uniform(size=(n + 3) // 4) < 0.5, 4)[:n]] = 0.0   # whole zero vectors
        grad[g.uniform(size=n) < 0.2] = 0.0                                # and single zeros
        Gd.copy_(cuda(grad))
        lr = dvgo.dvgo_lr_at(0.1, t - 1)
        dvgo.dvgo_adam_step(P, Gd, M, V, lr, t, param_bf16_out=pb, skip_zero_grad=True)
        oracle.adam(po, grad.astype(np.float64), mo, vo, float(np.float32(lr)), t, beta1=float(np.float32(0.9)),
                    beta2=float(np.float32(0.999)), eps=float(np.float32(1e-8)), skip_zero_grad=True)
    torch.cuda.synchronize()
    assert_close(P.cpu().numpy(), po, 1e-5, "param")
    assert_close(M.cpu().numpy(), mo, 1e-5, "m")
    assert_close(V.cpu().numpy(), vo, 1e-5, "v")
    # elements never touched kept their start value exactly; the BF16 copy matches where written
    never = mo == 0.0                                  # no nonzero gradient in four steps
    assert never.sum() > 100
    np.testing.assert_array_equal(P.cpu().numpy()[never], p0[never])


def test_model_with_lazy_grid_adam_moves_only_touched_points():
    res, R = 24, 64
    dens = synth.normal_grid((res,) * 3, 1, 0.5, 241).astype(np.float32)
    feat = synth.smooth_features(res, 12, 242)
    mlp = synth.mlp_weights(39, 128, 3, 243)
    p = dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=1.0 / res, bg=(1.0, 1.0, 1.0),
                    shift_b=dvgo.dvgo_shift_from_alpha_init(1e-2, 2.0 / res))
    m = dvgo.FineModel(cuda(dens), cuda(feat), cuda(_mlp_flat(mlp)), p, R, lazy_grid_adam=True)
    o, d, jit, tgt = (cuda(a) for a in synth.fine_batch(R, 244))
    m.forward(o, d, jit)
    bm, counts = dvgo.dvgo_touched_points(m.params, m.dd, R, None, m.renderer.workspace)
    m.train_step(o, d, jit, tgt)
    torch.cuda.synchronize()
    bits = np.unpackbits(bm[0].cpu().numpy().view(np.uint8), bitorder="little")[:res ** 3].reshape((res,) * 3)
    moved = m.density.cpu().numpy() != dens
    assert moved.sum() > 0 and not np.any(moved & ~bits.astype(bool))
    assert 0 < int(counts[0]) < res ** 3
