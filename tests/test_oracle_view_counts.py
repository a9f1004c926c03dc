"""Pins of the oracle's view counts (Sec. 4.1 Prior 2: n_j, the number of training views that see
grid point j, and the learning-rate scale n_j / n_max).

* Unprojection: a point built from a pixel position (u, v) and a depth along the camera's viewing
  axis, x = c + R (depth ((u - cx) / fx, -(v - cy) / fy, -1)), is seen by that camera exactly when
  (u, v) lies in the image and the depth exceeds the near distance.  The construction runs the
  camera model the other way (camera to world), so a transposed rotation, a flipped image axis or
  a swapped focal length fails it; the principal point is off centre so that a sign error on either
  image axis does too.
* A lattice under one camera looking straight down: each z layer sees a rectangle of the lattice
  whose sides follow from the layer's depth; counted with exact rational arithmetic per axis.  The
  lattice is not a cube, so a swapped axis or index order fails it.
* Several views: the counts add up over the views; the scale is n_j / n_max with maximum 1, and 1
  everywhere when no point is seen.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth


def _rotation(seed):
    q, r = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def _unproject(R, c, u, v, depth, fx, fy, cx, cy):
    dc = np.stack([(u - cx) / fx, -(v - cy) / fy, -np.ones_like(u)], axis=-1) * depth[:, None]
    return c + dc @ R.T


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_points_built_from_pixels_and_depths(seed):
    g = np.random.default_rng(seed)
    H, W, fx, fy, cx, cy, near = 60, 90, 75.0, 52.0, 31.0, 17.5, 0.4
    R, c = _rotation(seed + 10), g.normal(size=3)
    c2w = np.concatenate([R, c[:, None]], axis=1)[None]
    n = 400
    u_in, v_in = g.uniform(0.01, W - 0.01, n), g.uniform(0.01, H - 0.01, n)
    d_in = g.uniform(near + 0.01, 8.0, n)
    pts, labels = [_unproject(R, c, u_in, v_in, d_in, fx, fy, cx, cy)], [np.ones(n)]
    # just outside each side of the image, at a valid depth
    for u, v in ((g.uniform(-0.3, -0.01, n), v_in), (g.uniform(W + 0.01, W + 0.3, n), v_in),
                 (u_in, g.uniform(-0.3, -0.01, n)), (u_in, g.uniform(H + 0.01, H + 0.3, n))):
        pts.append(_unproject(R, c, u, v, d_in, fx, fy, cx, cy))
        labels.append(np.zeros(n))
    # inside the image but nearer than the near distance, or behind the camera
    for d in (g.uniform(0.01, near - 0.01, n), -g.uniform(0.01, 5.0, n)):
        pts.append(_unproject(R, c, u_in, v_in, d, fx, fy, cx, cy))
        labels.append(np.zeros(n))
    got = oracle.view_counts_points(np.concatenate(pts), c2w, H, W, fx, fy, cx, cy, near)
    np.testing.assert_array_equal(got, np.concatenate(labels).astype(np.uint32))


def _interval_count(lo, hi, m, n):
    """Lattice positions lo_box + i (hi_box - lo_box) / (n - 1), box [-1, 1], inside [lo, hi] (exact)."""
    return sum(1 for i in range(n) if lo <= Fraction(-1) + Fraction(2 * i, n - 1) <= hi)


def test_lattice_under_a_camera_looking_down():
    shape, D = (5, 7, 4), Fraction(7, 2)
    H, W, fx, fy, cx, cy = 40, 50, Fraction(61), Fraction(47), Fraction(23), Fraction(27)
    c2w = np.array([[[1.0, 0, 0, 0], [0, 1.0, 0, 0], [0, 0, 1.0, float(D)]]])
    counts, scale, n_max = oracle.view_counts(shape, c2w, H, W, float(fx), float(fy), float(cx), float(cy))
    expect = np.zeros(shape, dtype=np.uint32)
    for k in range(shape[2]):
        dep = D - (Fraction(-1) + Fraction(2 * k, shape[2] - 1))
        # 0 <= cx + fx x / dep <= W  and  0 <= cy - fy y / dep <= H
        xs = [i for i in range(shape[0])
              if -cx * dep / fx <= Fraction(-1) + Fraction(2 * i, shape[0] - 1) <= (W - cx) * dep / fx]
        ys = [j for j in range(shape[1])
              if -(H - cy) * dep / fy <= Fraction(-1) + Fraction(2 * j, shape[1] - 1) <= cy * dep / fy]
        for i in xs:
            expect[i, ys, k] = 1
    assert 0 < expect.sum() < expect.size          # the frustum cuts the lattice
    assert len({int(expect[:, :, k].sum()) for k in range(shape[2])}) > 1
    np.testing.assert_array_equal(counts, expect)
    assert n_max == 1
    np.testing.assert_array_equal(scale, expect.astype(np.float64))


def test_counts_add_over_views_and_scale_is_relative_to_the_maximum():
    rig = synth.hemisphere_rig(7, seed=5, radius=2.2, height=64, width=48, focal=40.0)
    shape, box = (9, 6, 8), ((-1.0, -0.8, -0.5), (1.2, 0.9, 1.0))
    counts, scale, n_max = oracle.view_counts(shape, rig.c2w, rig.height, rig.width, rig.focal, near=0.1, box=box)
    single = sum(oracle.view_counts(shape, rig.c2w[v:v + 1], rig.height, rig.width, rig.focal, near=0.1,
                                    box=box)[0].astype(np.int64) for v in range(7))
    np.testing.assert_array_equal(counts, single)
    assert n_max == counts.max() and 0 < counts.min() < n_max <= 7
    np.testing.assert_allclose(scale, counts / n_max, rtol=1e-16)
    assert scale.max() == 1.0


def test_no_point_seen_gives_unit_scale():
    c2w = np.array([[[1.0, 0, 0, 0], [0, 1.0, 0, 0], [0, 0, 1.0, -5.0]]])     # looks away from the box
    counts, scale, n_max = oracle.view_counts((3, 4, 5), c2w, 10, 10, 10.0)
    assert n_max == 0 and not counts.any()
    np.testing.assert_array_equal(scale, np.ones((3, 4, 5)))
