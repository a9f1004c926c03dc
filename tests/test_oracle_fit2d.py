"""Pins of the oracle's image-fitting toy (Sec. 3, Fig. exdv_poc: a binary image regressed by a
low-resolution 2D grid under the pre-, in- and post-activation orders of Eq. pre_in_post).

* Against the 3D renderer of the same oracle, an independent code path: the 2D grid extruded into
  a 3D grid of two identical z-slices, with a colour grid of ones and a black background, rendered
  with one explicit sample per pixel (a ray along +z through the pixel's position) gives C = alpha
  of that order; the renderer's density gradient summed over the two slices is the toy's gradient.
* Constant grids: every order gives alpha = 1 - exp(-softplus(v + b) delta).
* Central differences of the loss for the gradient of each order.
"""
import math

import numpy as np
import pytest

import oracle


def _pixels(H, W):
    i, j = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    return (i + 0.5) / H, (j + 0.5) / W


@pytest.mark.parametrize("order", [0, 1, 2])
def test_fit2d_matches_the_3d_renderer_on_an_extruded_grid(order):
    H, W, gh, gw = 11, 9, 5, 4
    g = np.random.default_rng(170 + order)
    V = g.normal(scale=1.5, size=(gh, gw))
    T = (g.uniform(size=(H, W)) > 0.5).astype(np.float64)
    b, delta = -0.3, 0.8
    img, loss, grad = oracle.fit2d(V, T, order, b, delta, grad=True)
    # the renderer: box [0, 1]^3, density lattice (gh, gw, 2), colour 1, background 0
    P = oracle.Params(grid_shape=(gh, gw, 2), xyz_min=(0.0, 0.0, 0.0), xyz_max=(1.0, 1.0, 1.0), shift_b=b,
                      delta=delta, bg=(0.0, 0.0, 0.0), mode=0, feat_dim=3, act_order=order)
    dens = np.repeat(V[:, :, None], 2, axis=2)
    col = np.ones((gh, gw, 2, 3))
    x, y = _pixels(H, W)
    o = np.stack([x.ravel(), y.ravel(), np.full(H * W, -1.0)], axis=1)
    d = np.tile([0.0, 0.0, 1.0], (H * W, 1))
    ts, dts = np.full((H * W, 1), 1.5), np.full((H * W, 1), delta)     # the sample at z = 0.5
    gC = np.zeros((H * W, 3))
    gC[:, 0] = 2.0 * (img.ravel() - T.ravel()) / (H * W)
    r = oracle.render(P, dens, col, o, d, explicit_t=ts, explicit_dt=dts, grad_rgb=gC)
    np.testing.assert_allclose(r.rgb[:, 0], img.ravel(), rtol=1e-13, atol=1e-15)
    assert loss == pytest.approx(float(np.mean((r.rgb[:, 0] - T.ravel()) ** 2)), rel=1e-12)
    np.testing.assert_allclose(r.grads["density"].sum(axis=2), grad, rtol=1e-11, atol=1e-16)


@pytest.mark.parametrize("order", [0, 1, 2])
def test_constant_grid_closed_form(order):
    v, b, delta = 0.7, -1.2, 0.6
    img, _, _ = oracle.fit2d(np.full((3, 6), v), np.zeros((8, 7)), order, b, delta)
    np.testing.assert_allclose(img, 1.0 - math.exp(-math.log1p(math.exp(v + b)) * delta), rtol=1e-14)


@pytest.mark.parametrize("order", [0, 1, 2])
def test_fit2d_gradient_matches_central_differences(order):
    H, W, gh, gw = 7, 8, 4, 3
    g = np.random.default_rng(180 + order)
    V = g.normal(scale=1.2, size=(gh, gw))
    T = (g.uniform(size=(H, W)) > 0.4).astype(np.float64)
    _, _, grad = oracle.fit2d(V, T, order, 0.2, 1.3, grad=True)
    num = np.zeros_like(V)
    h = 1e-6
    for k in range(V.size):
        Vp, Vm = V.copy(), V.copy()
        Vp.flat[k] += h
        Vm.flat[k] -= h
        num.flat[k] = (oracle.fit2d(Vp, T, order, 0.2, 1.3)[1] - oracle.fit2d(Vm, T, order, 0.2, 1.3)[1]) / (2 * h)
    np.testing.assert_allclose(grad, num, rtol=0, atol=1e-7 * np.abs(num).max())
    assert np.abs(grad).max() > 0


def test_post_activation_is_sharper_than_pre_on_one_cell():
    """Sec. 3 Fig. pre_in_post_patch: on one cell with corner values of opposite sign and a large
    magnitude, post-activation switches from ~0 to ~1 across a line, pre-activation blends linearly."""
    V = np.array([[-300.0, 300.0], [-300.0, 300.0]])
    img_post = oracle.fit2d(V, np.zeros((1, 64)), 0, 0.0, 1.0)[0][0]
    img_pre = oracle.fit2d(V, np.zeros((1, 64)), 1, 0.0, 1.0)[0][0]
    x = (np.arange(64) + 0.5) / 64
    np.testing.assert_allclose(img_pre, x, atol=1e-12)          # corner alphas 0 and 1, blended linearly
    assert np.all(img_post[x < 0.45] < 1e-12) and np.all(img_post[x > 0.55] > 1 - 1e-12)
