"""Pins of the oracle's positional encoding of the query point (Sec. 4.2 Eq. fine_queries_rgb,
Supp. A k_x = 5) and of its trilinear grid resize (Sec. 4.2 progressive scaling).

PE(x): one explicit sample per ray at a chosen world point routes a single MLP input column to the
red output; the column's value is compared with the unit-circle values at that point.  With the
PE(x) rows of W1 zero the render equals that of the 39-input model.  Central differences of the
render objective cover the gradients through the longer input row.

Resize: trilinear interpolation reproduces every multilinear field exactly (affine fields and
products of per-axis linear functions), so resizing such a field onto any lattice must give the
field's values there; a separable product of arbitrary per-axis profiles must equal three 1D linear
interpolations (numpy.interp, which also clamps outside the source box like the resize); the
same lattice is the identity."""
import math

import numpy as np
import pytest

import oracle
from test_oracle_pins import _objective, _tiny_problem

SIG = lambda z: 1.0 / (1.0 + math.exp(-z))      # noqa: E731


def _route_column(col, I, H=8):
    w1 = np.zeros((I, H)); w1[col, 0], w1[col, 1] = 1.0, -1.0
    w2 = np.zeros((H, H)); w2[0, 0] = w2[1, 1] = 1.0
    w3 = np.zeros((H, 3)); w3[0, 0], w3[1, 0] = 1.0, -1.0
    return dict(w1=w1, b1=np.zeros(H), w2=w2, b2=np.zeros(H), w3=w3, b3=np.zeros(3))


# x = (pi/32, -pi/16, pi/64): 2^k x_c runs through pi/4 and pi/2 for k <= 4
XPT = np.array([math.pi / 32, -math.pi / 16, math.pi / 64])


def _pe_x_expected(j):
    """Value of entry j of PE(x, 5) at XPT from the unit circle: sin / cos of multiples of pi/64."""
    if j < 3:
        return XPT[j]
    c, k = divmod((j - 3) % 15, 5)
    m = [2, -4, 1][c] * 2 ** k          # 2^k x_c = m pi / 64
    table_sin = {1: math.sin(math.pi / 64), 2: math.sin(math.pi / 32), 4: math.sin(math.pi / 16),
                 8: math.sin(math.pi / 8), 16: math.sqrt(0.5), 32: 1.0, 64: 0.0}
    table_cos = {1: math.cos(math.pi / 64), 2: math.cos(math.pi / 32), 4: math.cos(math.pi / 16),
                 8: math.cos(math.pi / 8), 16: math.sqrt(0.5), 32: 0.0, 64: -1.0}
    if j < 18:
        return math.copysign(table_sin[abs(m)], m) if table_sin[abs(m)] != 0.0 else 0.0
    return table_cos[abs(m)]


@pytest.mark.parametrize("j", [0, 1, 2, 3, 6, 7, 9, 12, 13, 17, 18, 21, 22, 24, 27, 28, 32])
def test_pe_x_columns_at_a_unit_circle_point(j):
    """Column 39 + j of the 72-wide input row (feat 12, PE(d, 4) 27, PE(x, 5) 33) at XPT."""
    C, F, FX, H, res = 12, 4, 5, 8, 4
    I = C + 3 + 6 * F + 3 + 6 * FX
    assert I == 72
    x0, b, dt = 0.9, -0.1, 0.05
    dens = np.full((res,) * 3, x0)
    feat = np.full((res, res, res, C), 0.25)
    P = oracle.Params(grid_shape=(res,) * 3, mode=1, feat_dim=C, n_freq=F, hidden=H, shift_b=b, delta=dt,
                      bg=(0.0, 0.0, 0.0), n_freq_pos=FX)
    dvec = np.array([0.2, 0.4, -0.9])
    dn = dvec / np.linalg.norm(dvec)
    t = 3.0
    o = XPT - t * dn
    r = oracle.render(P, dens, feat, [o], [dvec], mlp=_route_column(C + 27 + j, I),
                      explicit_t=[[t]], explicit_dt=[[dt]])
    alpha = -math.expm1(-math.log1p(math.exp(x0 + b)) * dt)
    v = _pe_x_expected(j)
    np.testing.assert_allclose(r.rgb[0], alpha * np.array([SIG(v), 0.5, 0.5]), rtol=1e-12, atol=1e-15)


def test_pe_d_columns_keep_their_place_with_pe_x():
    """The direction encoding stays at columns 12..38 when PE(x) is appended."""
    C, F, FX, H, res = 12, 4, 5, 8, 4
    I = C + 3 + 6 * F + 3 + 6 * FX
    dvec = np.array([0.2, 0.4, -0.9])
    dn = dvec / np.linalg.norm(dvec)
    P = oracle.Params(grid_shape=(res,) * 3, mode=1, feat_dim=C, n_freq=F, hidden=H, shift_b=0.0, delta=0.05,
                      bg=(0.0, 0.0, 0.0), n_freq_pos=FX)
    for col, v in ((12, dn[0]), (C + 3 + 1 * F + 2, math.sin(4 * dn[1])), (C + 3 + 3 * F + 2 * F + 3,
                                                                           math.cos(8 * dn[2]))):
        r = oracle.render(P, np.full((res,) * 3, 0.9), np.zeros((res, res, res, C)),
                          [XPT - 3.0 * dn], [dvec], mlp=_route_column(col, I), explicit_t=[[3.0]],
                          explicit_dt=[[0.05]])
        alpha = -math.expm1(-math.log1p(math.exp(0.9)) * 0.05)
        np.testing.assert_allclose(r.rgb[0, 0], alpha * SIG(v), rtol=1e-12)


def test_zero_pe_x_rows_reduce_to_the_39_input_model():
    P0, dens, cg, o, d, p, mlp0, gC, gT = _tiny_problem(1, 0, seed=90)
    I0 = P0.in_dim
    P1 = oracle.Params(**{**P0.__dict__, "n_freq_pos": 3})
    mlp1 = dict(mlp0)
    mlp1["w1"] = np.concatenate([mlp0["w1"], np.zeros((P1.in_dim - I0, mlp0["w1"].shape[1]))])
    a = oracle.render(P0, dens, cg, o, d, jitter=p, mlp=mlp0, grad_rgb=gC, grad_tfinal=gT)
    b = oracle.render(P1, dens, cg, o, d, jitter=p, mlp=mlp1, grad_rgb=gC, grad_tfinal=gT)
    np.testing.assert_allclose(b.rgb, a.rgb, rtol=1e-14)
    for k in ("density", "cgrid", "b1", "w2", "w3"):
        np.testing.assert_allclose(b.grads[k], a.grads[k], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(b.grads["w1"][:I0], a.grads["w1"], rtol=1e-12, atol=1e-15)
    assert np.abs(b.grads["w1"][I0:]).max() > 1e-6      # the PE(x) rows still receive gradient


def test_gradients_with_pe_x_match_central_differences():
    P0, dens, cg, o, d, p, _, gC, gT = _tiny_problem(1, 0, seed=91)
    P = oracle.Params(**{**P0.__dict__, "n_freq_pos": 2})
    import synth
    mlp = {k: v.astype(np.float64) for k, v in synth.mlp_weights(P.in_dim, P.hidden, 3, 93).items()}
    mlp["b3"] = np.random.default_rng(94).normal(scale=0.3, size=3)
    r = oracle.render(P, dens, cg, o, d, jitter=p, mlp=mlp, grad_rgb=gC, grad_tfinal=gT)
    h = 1e-6
    for name, arr in [("density", dens), ("cgrid", cg)] + list(mlp.items()):
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


# ------------------------------------------------------------------------------------------
# Trilinear resize (progressive scaling)
# ------------------------------------------------------------------------------------------

def _lattice(n, lo, hi):
    return [np.linspace(lo[a], hi[a], n[a]) for a in range(3)]


@pytest.mark.parametrize("src,dst", [((5, 4, 6), (9, 7, 11)), ((8, 8, 8), (5, 5, 5)), ((3, 7, 4), (3, 7, 4))])
def test_resize_reproduces_multilinear_fields(src, dst):
    lo, hi = (-1.0, -0.5, -2.0), (1.0, 1.5, 0.0)
    g = np.random.default_rng(7)
    cf = g.normal(size=(8, 2))                  # 2 channels of a0 + a1 x + a2 y + a3 z + a4 xy + ... + a7 xyz

    def field(X, Y, Z):
        terms = [np.ones_like(X), X, Y, Z, X * Y, Y * Z, X * Z, X * Y * Z]
        return np.stack([sum(cf[i, c] * terms[i] for i in range(8)) for c in range(2)], axis=-1)
    Xs = np.meshgrid(*_lattice(src, lo, hi), indexing="ij")
    Xd = np.meshgrid(*_lattice(dst, lo, hi), indexing="ij")
    out = oracle.resize_grid(field(*Xs), dst, (lo, hi))
    np.testing.assert_allclose(out, field(*Xd), rtol=0, atol=1e-12)


def test_resize_sub_box_and_clamp_match_per_axis_linear_interpolation():
    """f(x) g(y) h(z) with arbitrary per-axis profiles: trilinear resize = product of three 1D
    linear interpolations; the destination box reaches outside the source box on two axes, where
    both clamp to the edge value."""
    src, dst = (6, 9, 5), (13, 4, 10)
    slo, shi = (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0)
    dlo, dhi = (-0.6, -1.3, -0.2), (0.9, 0.7, 1.25)
    g = np.random.default_rng(8)
    prof = [g.normal(size=n) for n in src]
    grid = prof[0][:, None, None] * prof[1][None, :, None] * prof[2][None, None, :]
    out = oracle.resize_grid(grid, dst, (slo, shi), (dlo, dhi))
    ax_s, ax_d = _lattice(src, slo, shi), _lattice(dst, dlo, dhi)
    per = [np.interp(ax_d[a], ax_s[a], prof[a]) for a in range(3)]
    expect = per[0][:, None, None] * per[1][None, :, None] * per[2][None, None, :]
    np.testing.assert_allclose(out, expect, rtol=0, atol=1e-12)


def test_resize_to_the_same_lattice_is_the_identity():
    g = np.random.default_rng(9).normal(size=(7, 5, 6, 12))
    np.testing.assert_allclose(oracle.resize_grid(g, (7, 5, 6)), g, rtol=0, atol=1e-14)   # up to rounding of u
