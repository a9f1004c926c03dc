"""The guard band of the view-count kernel's FP32 fast test, checked on the CPU.

The kernel decides a (point, view) pair in FP32 from five forms affine in the lattice indices
(u >= 0, u <= W, v >= 0, v <= H, depth > near, each multiplied through by the depth), scaled by the
power of two that brings the guard 2^-15 * 3M (M the magnitude sum of a form's terms over the box)
into (1/2, 1]; the minimum over the forms decides (> 1 seen, < -1 not seen) and the pairs in between
go to the FP64 definition.  The argument is that FP32 rounding moves a form by far less than its
guard.  Here the coefficients and the forms are evaluated in FP32 (numpy, one rounding per
operation, the kernel's order) on rigs chosen to stress the bound -- cameras inside the box with a
near plane, off-centre principal points, long and short focal lengths, large images, boxes away from
the origin -- and every pair the FP32 test decides must agree with the FP64 oracle.  The fraction of
pairs left to the FP64 path is reported and must stay small.
"""
import numpy as np
import pytest

import oracle

f32 = np.float32


def _coefficients(c2w, box, n, H, W, fx, fy, cx, cy, near):
    mn, mx = np.asarray(box[0], f32), np.asarray(box[1], f32)
    step = ((mx - mn) / f32(np.asarray(n) - 1)).astype(f32)
    bmax = np.maximum(np.abs(mn), np.abs(mx))
    terms_cx, terms_wcx, terms_cy, terms_hcy = f32(cx), f32(W - cx), f32(cy), f32(H - cy)
    out = []
    for P in c2w:
        R, c = P[:, :3].astype(f32), P[:, 3].astype(f32)
        amp = bmax + np.abs(c)
        rows = []
        for m in range(5):
            al, mag, b = np.zeros(3, f32), f32(near if m == 4 else 0.0), f32(-near if m == 4 else 0.0)
            for a in range(3):
                t0, t1 = [(f32(fx) * R[a, 0], -terms_cx * R[a, 2]), (-f32(fx) * R[a, 0], -terms_wcx * R[a, 2]),
                          (-f32(fy) * R[a, 1], -terms_cy * R[a, 2]), (f32(fy) * R[a, 1], -terms_hcy * R[a, 2]),
                          (f32(0.0), -R[a, 2])][m]
                al[a] = t0 + t1
                mag = f32(mag + (abs(t0) + abs(t1)) * amp[a])
                b = f32(al[a] * (mn[a] - c[a]) + b)
            _, e = np.frexp(f32(2.0 ** -15) * f32(3.0) * mag)
            sc = f32(2.0 ** -int(e))
            rows.append((b * sc, al[0] * step[0] * sc, al[1] * step[1] * sc, al[2] * step[2] * sc))
        out.append(np.asarray(rows, f32))
    return out


def _rig(n_views, seed, box, inside):
    g = np.random.default_rng(seed)
    lo, hi = np.asarray(box[0]), np.asarray(box[1])
    c2w = np.zeros((n_views, 3, 4))
    for v in range(n_views):
        q, r = np.linalg.qr(g.normal(size=(3, 3)))
        q = q * np.sign(np.diag(r))
        if np.linalg.det(q) < 0:
            q[:, 0] = -q[:, 0]
        if inside:
            c = g.uniform(lo, hi)
        else:   # outside, looking roughly at the box centre
            centre = 0.5 * (lo + hi)
            d = g.normal(size=3)
            c = centre + 0.9 * np.linalg.norm(hi - lo) * d / np.linalg.norm(d)   # frusta cut the box
            z = (c - centre) / np.linalg.norm(c - centre)         # backward axis
            x = np.cross(g.normal(size=3), z)
            x /= np.linalg.norm(x)
            q = np.stack([x, np.cross(z, x), z], axis=1)
        c2w[v, :, :3], c2w[v, :, 3] = q, c
    return c2w


CASES = [
    # box, lattice, views inside?, H, W, fx, fy, cx, cy, near
    (((-1.0, -1.0, -1.0), (1.0, 1.0, 1.0)), (40, 36, 44), False, 800, 800, 1111.0, 1111.0, 400.0, 400.0, 0.0),
    (((-0.7, -1.1, 0.2), (0.9, 0.4, 1.3)), (31, 23, 29), True, 90, 130, 70.0, 55.5, 41.25, 60.75, 0.15),
    (((3.0, -2.0, 7.5), (5.5, 1.0, 9.0)), (33, 41, 25), False, 3000, 4000, 5200.0, 5100.0, 1900.5, 1523.25, 0.5),
    (((-50.0, -50.0, -10.0), (50.0, 50.0, 10.0)), (45, 45, 21), True, 64, 48, 20.0, 20.0, 30.0, 25.0, 1.0),
]


def _check(c2w, box, n, H, W, fx, fy, cx, cy, near):
    """Every pair the FP32 test decides agrees with the oracle; returns (decided, band) pairs."""
    F = _coefficients(c2w, box, n, H, W, fx, fy, cx, cy, near)
    I, J, K = (a.ravel().astype(f32) for a in np.meshgrid(*[np.arange(k) for k in n], indexing="ij"))
    lo, hi = np.asarray(box[0], np.float64), np.asarray(box[1], np.float64)
    # lattice points exactly as the oracle places them (FP32 box corners taken exactly)
    lo32, hi32 = lo.astype(f32).astype(np.float64), hi.astype(f32).astype(np.float64)
    idx = np.stack([I, J, K], axis=1).astype(np.float64)
    pts = lo32 + idx * (hi32 - lo32) / (np.asarray(n) - 1)
    decided = band = 0
    for v, Fv in enumerate(F):
        forms = np.stack([((Fv[m, 0] + I * Fv[m, 1]) + J * Fv[m, 2]) + K * Fv[m, 3] for m in range(5)])
        mn = forms.min(axis=0)
        ref = oracle.view_counts_points(pts, c2w[v:v + 1], H, W, fx, fy, cx, cy, near).astype(bool)
        assert not np.any((mn > 1) & ~ref), f"view {v}: FP32 says seen, FP64 says not"
        assert not np.any((mn < -1) & ref), f"view {v}: FP32 says not seen, FP64 says seen"
        decided += int(np.sum(np.abs(mn) > 1))
        band += int(np.sum(np.abs(mn) <= 1))
    counts = oracle.view_counts(n, c2w, H, W, fx, fy, cx, cy, near, box=(tuple(lo32), tuple(hi32)))[0]
    assert counts.min() < counts.max()          # the frusta cut the lattice: boundaries are crossed
    return decided, band


@pytest.mark.parametrize("case", range(len(CASES)))
def test_fp32_fast_test_agrees_with_the_fp64_definition(case):
    box, n, inside, H, W, fx, fy, cx, cy, near = CASES[case]
    decided, band = _check(_rig(12, 600 + case, box, inside), box, n, H, W, fx, fy, cx, cy, near)
    assert band < 0.01 * (band + decided)


def test_ties_in_the_reals_go_to_the_fp64_path():
    """Lattice points whose projection lies exactly on an image edge in exact arithmetic, with
    coordinates (1/3, 10/3) that neither FP32 nor FP64 represents: both round to either side of the
    edge, so only the guard band keeps the FP32 test from contradicting the FP64 decision.  A camera
    at (0, 0, 10/3) looking down -z with fx = fy = 9 on a 2 x 2 image puts x = +-1/3 (and y) at
    depth 3 (z = 1/3) exactly on the edges."""
    box, n = ((-1.0, -1.0, -1.0), (1.0, 1.0, 1.0)), (4, 4, 4)
    c2w = np.array([[[1.0, 0, 0, 0], [0, 1.0, 0, 0], [0, 0, 1.0, 10.0 / 3.0]]])
    decided, band = _check(c2w, box, n, 2, 2, 9.0, 9.0, 1.0, 1.0, 0.0)
    assert band >= 4                            # the edge points were left to the FP64 path
