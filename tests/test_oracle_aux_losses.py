"""Pins of the oracle's auxiliary losses (Supp. A: per-point rgb loss, background entropy loss):
closed forms on constant grids, zero weights, and central finite differences of the total loss
(photometric + weighted auxiliary terms) -- the per-point loss holds the compositing weights
constant, so its gradient reaches the colour parameters and not the density."""
import math

import numpy as np
import pytest

import oracle
from test_oracle_pins import _tiny_problem


def _H(a):
    a = min(max(a, 1e-6), 1 - 1e-6)
    return -a * math.log(a) - (1 - a) * math.log(1 - a)


def test_closed_forms_on_constant_grids():
    """Constant raw density x and constant colour c (coarse, identity activation): every sample has
    the same alpha, T_K = (1 - alpha)^K, sum_k w_k = 1 - T_K, so L_pt = (1 - T_K) ||c - C||^2 and
    L_bg = H(1 - T_K)."""
    res = 5
    P = oracle.Params(grid_shape=(res,) * 3, mode=0, feat_dim=3, shift_b=-1.0, delta=0.07, bg=(0.1, 0.2, 0.3))
    dens = np.full((res,) * 3, 0.4)
    c = np.array([0.3, 0.6, 0.9])
    cg = np.broadcast_to(c, (res,) * 3 + (3,)).copy()
    o, d = np.array([[0.0, 0.0, -3.0]]), np.array([[0.05, -0.02, 1.0]])
    tgt = np.array([[0.5, 0.1, 0.7]])
    base = oracle.render(P, dens, cg, o, d, target=tgt)
    for w_pt, w_bg in ((0.1, 0.0), (0.0, 0.01), (0.3, 0.2)):
        P2 = oracle.Params(**{**P.__dict__, "w_pt": w_pt, "w_bg": w_bg})
        r = oracle.render(P2, dens, cg, o, d, target=tgt)
        TK = float(r.tfinal[0])
        _, _, _, _, K = oracle.ray_bounds(P, o[0], d[0])
        alpha = -math.expm1(-math.log1p(math.exp(0.4 - 1.0)) * 0.07)
        assert TK == pytest.approx((1 - alpha) ** K, rel=1e-12)
        photo = float(np.sum((r.rgb - tgt) ** 2))
        assert base.loss == pytest.approx(photo, rel=1e-12)
        expect = photo + w_pt * (1 - TK) * float(np.sum((c - tgt[0]) ** 2)) + w_bg * _H(1 - TK)
        assert r.loss == pytest.approx(expect, rel=1e-12)


def _total(P, dens, cg, o, d, p, mlp, tgt):
    return oracle.render(P, dens, cg, o, d, jitter=p, mlp=mlp, target=tgt).loss


def _grad(P, dens, cg, o, d, p, mlp, tgt):
    r = oracle.render(P, dens, cg, o, d, jitter=p, mlp=mlp, target=tgt)
    gC = 2.0 * (r.rgb - tgt) / o.shape[0]
    return oracle.render(P, dens, cg, o, d, jitter=p, mlp=mlp, target=tgt, grad_rgb=gC).grads


def _fd(fn, arr, h=1e-6):
    num = np.zeros_like(arr)
    flat = arr.reshape(-1)
    for i in range(flat.size):
        old = flat[i]
        flat[i] = old + h
        fp = fn()
        flat[i] = old - h
        fm = fn()
        flat[i] = old
        num.reshape(-1)[i] = (fp - fm) / (2 * h)
    return num


@pytest.mark.parametrize("mode,rgb_act", [(0, 0), (0, 1), (1, 0)])
def test_background_entropy_gradient_matches_central_differences(mode, rgb_act):
    P, dens, cg, o, d, p, mlp, _, _ = _tiny_problem(mode, rgb_act, seed=80)
    P = oracle.Params(**{**P.__dict__, "w_bg": 0.7})
    tgt = np.random.default_rng(81).uniform(size=(3, 3))
    ana = _grad(P, dens, cg, o, d, p, mlp, tgt)
    params = {"density": dens, "cgrid": cg}
    if mlp:
        params.update(mlp)
    for name, arr in params.items():
        num = _fd(lambda: _total(P, dens, cg, o, d, p, mlp, tgt), arr)
        scale = max(np.abs(num).max(), 1e-3)
        np.testing.assert_allclose(ana[name], num, rtol=0, atol=2e-7 * scale, err_msg=name)
    # the entropy term moves the density gradient
    P0 = oracle.Params(**{**P.__dict__, "w_bg": 0.0})
    assert np.abs(_grad(P0, dens, cg, o, d, p, mlp, tgt)["density"] - ana["density"]).max() > 1e-6


@pytest.mark.parametrize("mode,rgb_act", [(0, 0), (0, 1), (1, 0)])
def test_per_point_rgb_gradient(mode, rgb_act):
    """Colour-side parameters: the per-point loss depends on them only through c_k, so central
    differences of the total loss give their gradient.  Density: the loss holds w_k constant, so
    its density gradient equals that of the photometric loss alone."""
    P, dens, cg, o, d, p, mlp, _, _ = _tiny_problem(mode, rgb_act, seed=82)
    P = oracle.Params(**{**P.__dict__, "w_pt": 0.5})
    tgt = np.random.default_rng(83).uniform(size=(3, 3))
    ana = _grad(P, dens, cg, o, d, p, mlp, tgt)
    params = {"cgrid": cg}
    if mlp:
        params.update(mlp)
    for name, arr in params.items():
        num = _fd(lambda: _total(P, dens, cg, o, d, p, mlp, tgt), arr)
        scale = max(np.abs(num).max(), 1e-3)
        np.testing.assert_allclose(ana[name], num, rtol=0, atol=2e-7 * scale, err_msg=name)
    P0 = oracle.Params(**{**P.__dict__, "w_pt": 0.0})
    ana0 = _grad(P0, dens, cg, o, d, p, mlp, tgt)
    np.testing.assert_allclose(ana["density"], ana0["density"], rtol=0, atol=1e-14)
    assert np.abs(ana["cgrid"] - ana0["cgrid"]).max() > 1e-6


def test_zero_weights_change_nothing():
    P, dens, cg, o, d, p, mlp, gC, gT = _tiny_problem(1, 0, seed=84)
    tgt = np.random.default_rng(85).uniform(size=(3, 3))
    a = oracle.render(P, dens, cg, o, d, jitter=p, mlp=mlp, grad_rgb=gC, grad_tfinal=gT)
    b = oracle.render(P, dens, cg, o, d, jitter=p, mlp=mlp, grad_rgb=gC, grad_tfinal=gT, target=tgt)
    for k in a.grads:
        np.testing.assert_allclose(a.grads[k], b.grads[k], rtol=0, atol=1e-14 * max(np.abs(a.grads[k]).max(), 1))
    assert b.loss == pytest.approx(float(np.sum((b.rgb - tgt) ** 2)) / 3, rel=1e-12)
