"""GPU parity of the view counts of Prior 2 (Sec. 4.1; dvgo_view_counts) against the FP64 oracle:
counts bit for bit (an integer decision per point and view, which the kernel takes in FP32 only
outside a guard band around each boundary and in FP64 with the oracle's operations inside it), the
learning-rate scale n_j / n_max bit for bit after FP32 rounding, and n_max exactly.

Cases: the coarse lattice of the per-scene optimisation (100^3 points, 100 inward views of
800x800 pixels); a ragged lattice over a sub-box with off-centre principal point, unequal focal
lengths, a near distance and cameras inside the box, with more views than one shared-memory chunk
holds; the packed storage layout; a lattice whose points fall exactly on the image edges (every
decision there goes through the FP64 path); no views; invalid rigs."""
import numpy as np
import pytest
import torch

import oracle
import synth
from test_gpu_parity import cuda

pytestmark = pytest.mark.gpu

dvgo = pytest.importorskip("paper_2111_11215_gb300")


def _rig_inside(n_views, seed, box):
    """Cameras at random points of a slightly enlarged box, looking in random directions."""
    g = np.random.default_rng(seed)
    lo, hi = np.array(box[0]), np.array(box[1])
    c2w = np.zeros((n_views, 3, 4))
    for v in range(n_views):
        q, r = np.linalg.qr(g.normal(size=(3, 3)))
        q = q * np.sign(np.diag(r))
        if np.linalg.det(q) < 0:
            q[:, 0] = -q[:, 0]
        c2w[v, :, :3] = q
        c2w[v, :, 3] = g.uniform(lo - 0.3, hi + 0.3)
    return c2w


def _gpu(desc, c2w, H, W, fx, fy=None, cx=None, cy=None, near=0.0):
    counts, scale, n_max = dvgo.dvgo_view_counts(desc, cuda(c2w, torch.float64), H, W, fx, fy, cx, cy, near)
    torch.cuda.synchronize()
    return counts, scale, int(n_max.item())


def _check(desc, c2w, H, W, fx, fy=None, cx=None, cy=None, near=0.0):
    counts, scale, n_max = _gpu(desc, c2w, H, W, fx, fy, cx, cy, near)
    box = (desc.xyz_min, desc.xyz_max)
    ref_c, ref_s, ref_max = oracle.view_counts(desc.shape, c2w, H, W, fx, fy, cx, cy, near, box=box)
    np.testing.assert_array_equal(counts.cpu().numpy().reshape(desc.shape), ref_c.astype(np.int32))
    assert n_max == ref_max
    np.testing.assert_array_equal(scale.cpu().numpy().reshape(desc.shape), ref_s.astype(np.float32))
    return ref_c


def test_coarse_lattice_100cube_100_views():
    rig = synth.hemisphere_rig(100, seed=2024)
    ref = _check(dvgo.GridDesc((100,) * 3, 1), rig.c2w, rig.height, rig.width, rig.focal)
    assert ref.min() < ref.max() == 100          # corners leave some views' frusta


def test_ragged_sub_box_many_views_near_plane():
    box = ((-0.7, -1.1, 0.2), (0.9, 0.4, 1.3))
    desc = dvgo.GridDesc((37, 23, 41), 1, box[0], box[1])
    c2w = _rig_inside(700, 7, box)               # > 512 views: several shared-memory chunks
    ref = _check(desc, c2w, 90, 130, 70.0, 55.5, 41.25, 60.75, near=0.15)
    assert ref.min() < ref.max()


def test_packed_layout():
    rig = synth.hemisphere_rig(24, seed=3, radius=2.5, height=120, width=160, focal=150.0)
    desc = dvgo.GridDesc((21, 18, 26), 1, layout=dvgo.DVGO_LAYOUT_PACKED)
    counts, scale, n_max = _gpu(desc, rig.c2w, rig.height, rig.width, rig.focal, near=0.05)
    canon = desc.with_(layout=dvgo.DVGO_LAYOUT_CANONICAL)
    c = dvgo.dvgo_pack_grid(desc, counts.view(torch.float32), canon).view(torch.int32)
    s = dvgo.dvgo_pack_grid(desc, scale, canon)
    torch.cuda.synchronize()
    ref_c, ref_s, ref_max = oracle.view_counts(desc.shape, rig.c2w, rig.height, rig.width, rig.focal, near=0.05)
    np.testing.assert_array_equal(c.cpu().numpy().reshape(desc.shape), ref_c.astype(np.int32))
    np.testing.assert_array_equal(s.cpu().numpy().reshape(desc.shape), ref_s.astype(np.float32))
    assert n_max == ref_max


def test_points_exactly_on_the_image_edges():
    """Cameras 2.5 units from the centre looking straight down, up, and along -x: with fx = fy = 2
    and a 2x2 image, u = 1 + 2 x / depth lands exactly on 0 or 2 (the closed edges) at the lattice
    points of depth 2, and outside the image at depth 1.5."""
    c2w = np.array([[[1.0, 0, 0, 0], [0, 1.0, 0, 0], [0, 0, 1.0, 2.5]],          # above, looking -z
                    [[1.0, 0, 0, 0], [0, -1.0, 0, 0], [0, 0, -1.0, -2.5]],        # below, looking +z
                    [[0, 0, 1.0, 2.5], [1.0, 0, 0, 0], [0, 1.0, 0, 0]]])          # at +x, looking -x
    ref = _check(dvgo.GridDesc((5, 5, 5), 1), c2w, 2, 2, 2.0)
    assert 0 < ref.sum() < 3 * 125
    assert ref[0, 2, 3] == 3          # x = -1, z = 0.5: on the left edge of the first view (u = 0)
    assert ref[0, 2, 4] == 2          # x = -1, z = 1: outside the first view (u = -1/3)


def test_no_views():
    desc = dvgo.GridDesc((6, 5, 4), 1)
    counts, scale, n_max = _gpu(desc, np.zeros((0, 3, 4)), 10, 10, 5.0)
    assert n_max == 0 and not counts.any()
    assert torch.equal(scale, torch.ones_like(scale))


@pytest.mark.parametrize("bad", [dict(fx=0.0), dict(fx=-1.0), dict(near=-0.1), dict(H=0), dict(fy=float("nan"))])
def test_invalid_rig_is_rejected(bad):
    a = dict(H=10, W=10, fx=5.0, fy=None, near=0.0)
    a.update(bad)
    with pytest.raises(dvgo.DVGOError):
        dvgo.dvgo_view_counts(dvgo.GridDesc((4, 4, 4), 1), cuda(np.zeros((2, 3, 4)), torch.float64), a["H"], a["W"],
                              a["fx"], a["fy"], near=a["near"])


def test_coarse_model_applies_the_view_count_scale():
    """A coarse step with the Prior 2 scale: points no view sees keep their density, and the
    density update equals the oracle's Adam with lr_scale = n_j / n_max."""
    res = 24
    rig = synth.hemisphere_rig(6, seed=11, radius=2.6, height=80, width=80, focal=150.0)   # corners unseen
    g = np.random.default_rng(12)
    dens = g.normal(size=(res,) * 3).astype(np.float32)
    rgb = g.uniform(size=(res,) * 3 + (3,)).astype(np.float32)
    p = dvgo.Params(mode=dvgo.DVGO_MODE_COARSE, step=0.5 * 2.0 / res, bg=(1.0, 1.0, 1.0), shift_b=-2.0)
    m = dvgo.CoarseModel(cuda(dens), cuda(rgb), p, 1024)
    n_max = m.set_view_counts(cuda(rig.c2w, torch.float64), rig.height, rig.width, rig.focal)
    ref_c, ref_s, ref_max = oracle.view_counts((res,) * 3, rig.c2w, rig.height, rig.width, rig.focal)
    assert n_max == ref_max and (ref_c == 0).any()
    o, d, _ = synth.random_pixel_rays(rig, 1024, seed=13)
    o, d = cuda(o), cuda(d)
    jit, tgt = cuda(g.uniform(size=1024)), cuda(g.uniform(size=(1024, 3)))
    m.train_step(o, d, jit, tgt)
    torch.cuda.synchronize()
    g_dens = np.zeros_like(dens, dtype=np.float64)
    # gradient of this step from a second model without the scale (same inputs, same kernels)
    m2 = dvgo.CoarseModel(cuda(dens), cuda(rgb), p, 1024)
    m2.renderer.forward(m2.density, m2.rgb_grid, None, o, d, jit, None, tgt, m2.rgb, m2.tfinal, m2.loss, m2.dloss)
    m2.renderer.backward(m2.density, m2.rgb_grid, None, o, d, jit, None, m2.dloss, None, m2.g_density, m2.g_rgb, None)
    torch.cuda.synchronize()
    g_dens[...] = m2.g_density.cpu().numpy()
    pr = dens.astype(np.float64)
    oracle.adam(pr, g_dens.copy(), np.zeros_like(pr), np.zeros_like(pr), float(np.float32(m.lr_grid)), 1,
                beta1=float(np.float32(0.9)), beta2=float(np.float32(0.999)), eps=float(np.float32(1e-8)),
                lr_scale=ref_s.astype(np.float32).astype(np.float64))
    got = m.density.cpu().numpy()
    np.testing.assert_array_equal(got[ref_c == 0], dens[ref_c == 0])
    np.testing.assert_allclose(got, pr, rtol=0, atol=1e-5)
    assert np.abs(got - dens).max() > 0.05           # the seen points moved
