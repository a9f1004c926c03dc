"""The packed grid layout (4x4x4 bricks, Morton order inside a brick): the copy between layouts
against the layout's definition, and renders on packed grids against the FP64 oracle on the
canonical data (coarse; fine with the FP32 SIMT and the BF16 tensor-core colour kernels, forward
and backward; the known-free-space test on a packed coarse grid)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import BOUND_FP32, RTOL_COLOUR, RTOL_GRAD, assert_close, assert_within_bound, oracle_params
from test_gpu_parity import _fine_inputs, _mlp_flat, cuda

pytestmark = pytest.mark.gpu

dvgo = pytest.importorskip("paper_2111_11215_gb300")
PACKED = dvgo.DVGO_LAYOUT_PACKED


def _packed_positions(nx, ny, nz):
    """Packed point index of every lattice point (i, j, k), from the layout's definition in dvgo.h:
    row-major 4^3 bricks, Morton bits (i0 j0 k0) low, (i1 j1 k1) above inside a brick."""
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    nby, nbz = -(-ny // 4), -(-nz // 4)
    brick = ((i >> 2) * nby + (j >> 2)) * nbz + (k >> 2)
    m = ((i & 1) << 2) | ((j & 1) << 1) | (k & 1) | (((i >> 1) & 1) << 5) | (((j >> 1) & 1) << 4) | (((k >> 1) & 1) << 3)
    return brick * 64 + m


def _pack(a, desc, dtype=dvgo.DVGO_DTYPE_F32):
    return dvgo.dvgo_pack_grid(desc, a.reshape(-1).contiguous(), desc.with_(layout=PACKED, dtype=dtype))


def _unpack(a, desc):
    return dvgo.dvgo_pack_grid(desc.with_(layout=PACKED), a, desc).reshape(tuple(desc.shape) + (
        (desc.channels,) if desc.channels > 1 else ()))


@pytest.mark.parametrize("shape,C", [((13, 6, 9), 1), ((8, 8, 8), 12), ((5, 17, 4), 3)])
def test_pack_matches_the_layout_definition(shape, C):
    g = dvgo.GridDesc(shape, C)
    a = torch.randn(tuple(shape) + ((C,) if C > 1 else ()), device="cuda")
    p = _pack(a, g)
    pos = _packed_positions(*shape).reshape(-1)
    exp = np.zeros(dvgo.dvgo_grid_elements(g.with_(layout=PACKED)), np.float32).reshape(-1, C)
    exp[pos] = a.reshape(-1, C).cpu().numpy()
    np.testing.assert_array_equal(p.cpu().numpy().reshape(-1, C), exp)     # padding points are 0
    back = _unpack(p, g)
    assert torch.equal(back, a)
    pb = _pack(a, g, dvgo.DVGO_DTYPE_BF16)                                 # FP32 -> packed BF16
    assert torch.equal(_unpack(pb.float(), g), a.to(torch.bfloat16).float())


def test_coarse_render_on_packed_grids():
    case = synth.coarse_case(seed=4, n_rays=2000)
    res, R = 32, 2000
    p = dvgo.Params(mode=dvgo.DVGO_MODE_COARSE, step=0.03125, shift_b=0.2, bg=(0.3, 0.6, 0.9), rgb_act=1)
    dd, cd = dvgo.GridDesc((res,) * 3, 1, layout=PACKED), dvgo.GridDesc((res,) * 3, 3, layout=PACKED)
    D = _pack(cuda(case["density"]), dd.with_(layout=0))
    Cg = _pack(cuda(case["rgb"]), cd.with_(layout=0))
    r = dvgo.Renderer(p, dd, cd, R)
    gC = np.random.default_rng(5).normal(scale=1e-2, size=(R, 3))
    rgb, tf, _ = r.forward(D, Cg, None, cuda(case["rays_o"]), cuda(case["rays_d"]))
    g_d, g_c = torch.zeros_like(D), torch.zeros_like(Cg)
    r.backward(D, Cg, None, cuda(case["rays_o"]), cuda(case["rays_d"]), None, None, cuda(gC), None, g_d, g_c, None)
    torch.cuda.synchronize()
    P = oracle_params(p, (res,) * 3, 3)
    ref = oracle.render(P, case["density"], case["rgb"], case["rays_o"], case["rays_d"], grad_rgb=gC)
    assert_close(rgb.cpu().numpy(), ref.rgb, RTOL_COLOUR, "rgb")
    assert_close(_unpack(g_d, dd.with_(layout=0)).cpu().numpy(), ref.grads["density"], RTOL_GRAD, "grad_density")
    assert_close(_unpack(g_c, cd.with_(layout=0)).cpu().numpy(), ref.grads["cgrid"], RTOL_GRAD, "grad_rgb")
    # the padding points of the packed gradients receive nothing
    pad = np.ones(g_d.numel(), bool)
    pad[_packed_positions(res, res, res).reshape(-1)] = False
    assert not np.any(g_d.cpu().numpy()[pad])


@pytest.mark.parametrize("prec", [dvgo.DVGO_MLP_FP32, dvgo.DVGO_MLP_BF16])
def test_fine_render_on_packed_grids(prec):
    res, R = 22, 300                                             # 22 = 5 bricks + 2 points: ragged bricks
    dens, feat, mlp, o, d, jit, _ = _fine_inputs(res, R, seed=70)
    bf = prec == dvgo.DVGO_MLP_BF16
    if bf:
        feat = torch.as_tensor(feat).to(torch.bfloat16).float().numpy()
    p = dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=2.0 / res * 0.5, bg=(1.0, 1.0, 1.0), mlp_prec=prec,
                    shift_b=dvgo.dvgo_shift_from_alpha_init(1e-2, 2.0 / res))
    dd = dvgo.GridDesc((res,) * 3, 1, layout=PACKED)
    cd = dvgo.GridDesc((res,) * 3, 12, layout=PACKED, dtype=dvgo.DVGO_DTYPE_BF16 if bf else dvgo.DVGO_DTYPE_F32)
    D = _pack(cuda(dens), dd.with_(layout=0))
    F = _pack(cuda(feat), cd.with_(layout=0, dtype=dvgo.DVGO_DTYPE_F32), cd.dtype)
    flat = cuda(_mlp_flat(mlp))
    views = dvgo.render.mlp_views(flat)
    r = dvgo.Renderer(p, dd, cd, R)
    gC = np.random.default_rng(71).normal(scale=1e-2, size=(R, 3))
    rgb, tf, _ = r.forward(D, F, views, cuda(o), cuda(d), cuda(jit))
    g_d = torch.zeros_like(D)
    g_f = torch.zeros(F.numel(), device="cuda")
    g_m = torch.zeros_like(flat)
    r.backward(D, F, views, cuda(o), cuda(d), cuda(jit), None, cuda(gC), None, g_d, g_f, g_m)
    torch.cuda.synchronize()
    P = oracle_params(p, (res,) * 3, 12)
    ref = oracle.render(P, dens, feat, o, d, jitter=jit, mlp=mlp, grad_rgb=gC, error_bound=BOUND_FP32)
    gd = _unpack(g_d, dd.with_(layout=0)).cpu().numpy()
    gf = _unpack(g_f, cd.with_(layout=0, dtype=dvgo.DVGO_DTYPE_F32)).cpu().numpy()
    if not bf:
        assert_close(rgb.cpu().numpy(), ref.rgb, RTOL_COLOUR, "rgb")
        assert_within_bound(gd, ref.grads["density"], ref.bounds["density"], "grad_density")
        assert_within_bound(gf, ref.grads["cgrid"], ref.bounds["cgrid"], "grad_feat")
    else:
        # BF16 MLP: the canonical-layout BF16 render is the reference (same arithmetic, other layout)
        dd0, cd0 = dd.with_(layout=0), cd.with_(layout=0)
        r0 = dvgo.Renderer(p, dd0, cd0, R)
        F0 = cuda(feat).to(torch.bfloat16)
        rgb0, _, _ = r0.forward(cuda(dens), F0, views, cuda(o), cuda(d), cuda(jit))
        g_d0, g_f0 = torch.zeros_like(cuda(dens)), torch.zeros(F0.shape, device="cuda")
        r0.backward(cuda(dens), F0, views, cuda(o), cuda(d), cuda(jit), None, cuda(gC), None, g_d0, g_f0,
                    torch.zeros_like(flat))
        torch.cuda.synchronize()
        assert torch.equal(rgb, rgb0)                                      # gathers read the same values
        assert_close(gd, g_d0.cpu().numpy(), 1e-5, "grad_density_vs_canonical")
        assert_close(gf, g_f0.cpu().numpy(), 1e-5, "grad_feat_vs_canonical")
        assert np.abs(rgb.cpu().numpy() - ref.rgb).max() < 1e-2


def test_freespace_and_bbox_on_a_packed_coarse_grid():
    from test_gpu_freespace import _freespace, TAU_C
    fs_gpu, fs_ora = _freespace()
    res_c = fs_gpu.desc.shape[0]
    packed = dvgo.FreeSpace(density=_pack(fs_gpu.density, fs_gpu.desc), desc=fs_gpu.desc.with_(layout=PACKED),
                            shift_b=fs_gpu.shift_b, step=fs_gpu.step, tau=TAU_C)
    assert torch.equal(dvgo.dvgo_unknown_bbox(packed), dvgo.dvgo_unknown_bbox(fs_gpu))
    res, R = 24, 300
    dens, feat, mlp, o, d, jit, _ = _fine_inputs(res, R, seed=30)
    outs = []
    for fs in (fs_gpu, packed):
        p = dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=2.0 / res * 0.5, bg=(1.0, 1.0, 1.0), freespace=fs,
                        shift_b=dvgo.dvgo_shift_from_alpha_init(1e-2, 2.0 / res))
        r = dvgo.Renderer(p, dvgo.GridDesc((res,) * 3, 1), dvgo.GridDesc((res,) * 3, 12), R)
        rgb, _, _ = r.forward(cuda(dens), cuda(feat), dvgo.render.mlp_views(cuda(_mlp_flat(mlp))), cuda(o), cuda(d),
                              cuda(jit))
        outs.append(rgb.clone())
    assert res_c == 12 and torch.equal(outs[0], outs[1])
