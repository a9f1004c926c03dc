"""Pins of the oracle's interpolation / activation orders (Sec. 3 Eq. pre_in_post): the three
orders agree on constant grids, differ in between lattice points exactly as their definitions
order the operations (checked at a cell centre), and their gradients match central finite
differences."""
import math

import numpy as np
import pytest

import oracle
from test_oracle_pins import _objective, _tiny_problem


def test_orders_agree_on_constant_grids_and_differ_at_a_cell_centre():
    res = 4
    for val in (-3.0, 0.0, 2.5):
        out = []
        for order in (0, 1, 2):
            P = oracle.Params(grid_shape=(res,) * 3, mode=0, feat_dim=3, shift_b=0.3, delta=0.2, act_order=order)
            r = oracle.render(P, np.full((res,) * 3, val), np.full((res,) * 3 + (3,), 0.5),
                              np.array([[0.1, -0.05, -3.0]]), np.array([[0.0, 0.0, 1.0]]))
            out.append(r.tfinal[0])
        assert out[0] == pytest.approx(out[1], rel=1e-13) and out[0] == pytest.approx(out[2], rel=1e-13)
    # one ray along the cell's centre line through a 2^3 grid whose corners differ: the three
    # orders give different transmittances, each matching its definition evaluated by hand at
    # the samples (bilinear weights in x, y are 1/4 each; z varies along the ray)
    v = np.array([[[-4.0, 3.0], [1.0, -2.0]], [[2.0, -1.0], [0.5, 4.0]]])
    delta, b = 0.1, 0.3
    sp = lambda z: math.log1p(math.exp(z))
    T = {}
    for order in (0, 1, 2):
        P = oracle.Params(grid_shape=(2, 2, 2), xyz_min=(0, 0, 0), xyz_max=(1, 1, 1), shift_b=b, delta=delta,
                          mode=0, feat_dim=3, act_order=order)
        r = oracle.render(P, v, np.full((2, 2, 2, 3), 0.5), np.array([[0.5, 0.5, -1.0]]), np.array([[0.0, 0.0, 1.0]]))
        T[order] = r.tfinal[0]
        t_hand = 1.0
        for k in range(int(r.n_samples[0])):
            z = (k + 0.5) * delta                       # lattice coordinate along z (box entry at t = 1)
            w = [(1 - z) / 4, z / 4]                     # weights of the z = 0 / z = 1 corners
            raw = sum(w[kz] * v[ix, iy, kz] for ix in (0, 1) for iy in (0, 1) for kz in (0, 1))
            if order == 0:
                a = -math.expm1(-sp(raw + b) * delta)
            elif order == 1:
                a = sum(w[kz] * -math.expm1(-sp(v[ix, iy, kz] + b) * delta) for ix in (0, 1) for iy in (0, 1)
                        for kz in (0, 1))
            else:
                a = -math.expm1(-sum(w[kz] * sp(v[ix, iy, kz] + b) for ix in (0, 1) for iy in (0, 1)
                                     for kz in (0, 1)) * delta)
            t_hand *= 1 - a
        assert T[order] == pytest.approx(t_hand, rel=1e-12)
    assert abs(T[0] - T[1]) > 1e-3 and abs(T[0] - T[2]) > 1e-3 and abs(T[1] - T[2]) > 1e-4


@pytest.mark.parametrize("mode,order", [(0, 1), (0, 2), (1, 1), (1, 2)])
def test_gradients_match_central_differences(mode, order):
    P, dens, cg, o, d, p, mlp, gC, gT = _tiny_problem(mode, 0, seed=90 + order)
    P = oracle.Params(**{**P.__dict__, "act_order": order})
    r = oracle.render(P, dens, cg, o, d, jitter=p, mlp=mlp, grad_rgb=gC, grad_tfinal=gT)
    params = {"density": dens, "cgrid": cg}
    h = 1e-6
    for name, arr in params.items():
        num = np.zeros_like(arr)
        flat = arr.reshape(-1)
        for i in range(flat.size):
            old = flat[i]
            flat[i] = old + h
            fp = _objective(P, dens, cg, o, d, p, mlp, gC, gT)
            flat[i] = old - h
            fm = _objective(P, dens, cg, o, d, p, mlp, gC, gT)
            flat[i] = old
            num.reshape(-1)[i] = (fp - fm) / (2 * h)
        scale = max(np.abs(num).max(), 1e-3)
        np.testing.assert_allclose(r.grads[name], num, rtol=0, atol=2e-7 * scale, err_msg=name)
        assert np.abs(r.grads[name]).max() > 0
