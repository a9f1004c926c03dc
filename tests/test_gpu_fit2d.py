"""GPU parity of the image-fitting toy (Sec. 3, Fig. exdv_poc) against the FP64 oracle: the
predicted image, the MSE and its gradient for the three activation orders, on images with ragged
32-pixel tiles, with the shared-memory gradient patch (grid coarser than the image) and without it
(grid finer than the image); and five Adam steps of the fit against the oracle's Adam.

Tolerances: image 1e-6 absolute (FP32 activations of values in [0, 1]), loss 1e-5 relative,
gradient 1e-4 relative per element (floored at 1e-2 of the largest), the FP32 bounds of the
renderer's parity tests."""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import RTOL_GRAD, assert_close
from test_gpu_parity import cuda

pytestmark = pytest.mark.gpu

dvgo = pytest.importorskip("paper_2111_11215_gb300")


def _run(V, T, order, b, delta):
    img = torch.empty(T.shape, device="cuda")
    grad = torch.zeros(V.shape, device="cuda")
    loss = torch.empty(1, device="cuda")
    dvgo.dvgo_fit2d(cuda(V), cuda(T), order, b, delta, image_out=img, grad_out=grad, loss_out=loss)
    torch.cuda.synchronize()
    return img.cpu().numpy(), float(loss.item()), grad.cpu().numpy()


@pytest.mark.parametrize("order", [dvgo.DVGO_ACT_POST, dvgo.DVGO_ACT_PRE, dvgo.DVGO_ACT_IN])
@pytest.mark.parametrize("H,W,gh,gw", [(100, 170, 21, 35), (50, 40, 80, 63), (64, 64, 2, 2)])
def test_fit2d_matches_oracle(order, H, W, gh, gw):
    g = np.random.default_rng(190 + order + gh)
    V = g.normal(scale=2.0, size=(gh, gw)).astype(np.float32)
    T = synth.binary_image(H, W, seed=gh)
    b, delta = 0.3, 1.0
    img, loss, grad = _run(V, T, order, b, delta)
    rimg, rloss, rgrad = oracle.fit2d(V, T, order, b, delta, grad=True)
    np.testing.assert_allclose(img, rimg, rtol=0, atol=1e-6)
    assert loss == pytest.approx(rloss, rel=1e-5)
    assert_close(grad, rgrad, RTOL_GRAD, "grad")


def test_fit2d_adam_steps_match_oracle():
    H, W, gh, gw = 96, 80, 20, 17
    T = synth.binary_image(H, W, seed=3)
    V = np.zeros((gh, gw), np.float32)
    Vg = cuda(V)
    m, v = torch.zeros_like(Vg), torch.zeros_like(Vg)
    grad = torch.zeros_like(Vg)
    Vo, mo, vo = V.astype(np.float64), np.zeros((gh, gw)), np.zeros((gh, gw))
    Tg = cuda(T)
    for t in range(1, 6):
        dvgo.dvgo_fit2d(Vg, Tg, dvgo.DVGO_ACT_POST, 0.0, 1.0, grad_out=grad)
        dvgo.dvgo_adam_step(Vg, grad, m, v, 0.1, t)
        _, _, go = oracle.fit2d(Vo, T, 0, 0.0, 1.0, grad=True)
        oracle.adam(Vo, go, mo, vo, 0.1, t)
    torch.cuda.synchronize()
    # Adam's first steps move each value by ~lr sign(g); a gradient within rounding of 0 can flip
    # one step's sign, so compare all but a handful of elements tightly
    diff = np.abs(Vg.cpu().numpy() - Vo)
    assert np.mean(diff < 1e-4) > 0.99 and np.abs(Vo).max() > 0.3


def test_fit2d_rejects_bad_descriptors():
    V = torch.zeros((1, 5), device="cuda")
    with pytest.raises(dvgo.DVGOError):
        dvgo.dvgo_fit2d(V, torch.zeros((8, 8), device="cuda"))
    with pytest.raises(ValueError):
        dvgo.dvgo_fit2d(torch.zeros((4, 4), device="cuda"), torch.zeros((8, 8), device="cuda"),
                        image_out=torch.zeros(10, device="cuda"))
