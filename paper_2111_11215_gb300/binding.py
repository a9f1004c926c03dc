"""ctypes binding of libdvgo (include/dvgo.h): argument marshalling only.

Each ``dvgo_*`` function here has the name and argument order of the C entry point; tensors are
passed as device pointers, structs as ctypes mirrors.  A non-zero status raises ``DVGOError``.
"""
from __future__ import annotations

import ctypes as C
import os
import dataclasses
from dataclasses import dataclass

import torch

DVGO_OK = 0
DVGO_ERR_INVALID_ARG, DVGO_ERR_WORKSPACE, DVGO_ERR_UNSUPPORTED = -1, -2, -3
DVGO_ERR_CUDA, DVGO_ERR_DEVICE, DVGO_ERR_CAPACITY = -4, -5, -6
DVGO_DTYPE_F32, DVGO_DTYPE_BF16 = 0, 1
DVGO_MODE_COARSE, DVGO_MODE_FINE = 0, 1
DVGO_MLP_FP32, DVGO_MLP_BF16 = 0, 1

EXPORTED_SYMBOLS = (
    "dvgo_workspace_size", "dvgo_render_fwd", "dvgo_render_bwd", "dvgo_adam_step", "dvgo_adam_step_multi",
    "dvgo_lr_at",
    "dvgo_workspace_status", "dvgo_sample_counts", "dvgo_shift_from_alpha_init", "dvgo_status_string",
    "dvgo_abi_version", "dvgo_profile_enable", "dvgo_profile_read", "dvgo_profile_trace", "dvgo_launch_counter",
    "dvgo_render_fwd_noalloc", "dvgo_weight_bins", "dvgo_proposal_fwd", "dvgo_proposal_bwd", "dvgo_sample_pdf",
    "dvgo_unknown_bbox", "dvgo_grid_elements", "dvgo_pack_grid", "dvgo_resize_grid", "dvgo_fit2d",
    "dvgo_touched_points", "dvgo_view_counts",
)
DVGO_NOALLOC_MAX_RAYS = 16384
DVGO_NOALLOC_SCRATCH_BYTES = 2621696
DVGO_ACT_POST, DVGO_ACT_PRE, DVGO_ACT_IN = 0, 1, 2   # Sec. 3 interpolation / activation orders
DVGO_LAYOUT_CANONICAL, DVGO_LAYOUT_PACKED = 0, 1     # grid storage layouts

KERNEL_KINDS = ("ray_setup", "scan", "coarse_fwd", "coarse_bwd", "fine_density", "fine_colour_fwd",
                "fine_composite", "fine_comp_bwd", "fine_colour_bwd", "adam", "aux", "weight_bins", "proposal_fwd",
                "proposal_bwd", "sample_pdf", "view_counts")

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None


def library_path() -> str:
    return os.path.join(_HERE, "libdvgo.so")


class DVGOError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {lib().dvgo_status_string(status).decode()} (status {status})")
        self.status = status


class _GridDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("channels", C.c_int),
                ("xyz_min", C.c_float * 3), ("xyz_max", C.c_float * 3), ("dtype", C.c_int), ("layout", C.c_int)]


class _FreeSpace(C.Structure):
    _fields_ = [("desc", _GridDesc), ("density", C.c_void_p), ("shift_b", C.c_float), ("step", C.c_float),
                ("tau", C.c_float)]


class _Params(C.Structure):
    _fields_ = [("mode", C.c_int), ("rgb_act", C.c_int), ("mlp_prec", C.c_int), ("n_freq_dir", C.c_int),
                ("hidden", C.c_int), ("step", C.c_float), ("shift_b", C.c_float), ("tau_f", C.c_float),
                ("t_near", C.c_float), ("t_far", C.c_float), ("bg", C.c_float * 3),
                ("freespace", C.POINTER(_FreeSpace)), ("w_pt_rgb", C.c_float), ("w_bg", C.c_float),
                ("act_order", C.c_int), ("n_freq_pos", C.c_int), ("wait_limit_us", C.c_int),
                ("test_withhold_tile", C.c_int), ("cgrid_ready", C.c_void_p), ("forward_only", C.c_int),
                ("density_ready", C.c_void_p)]


class _Fit2d(C.Structure):
    _fields_ = [("height", C.c_int), ("width", C.c_int), ("grid_h", C.c_int), ("grid_w", C.c_int),
                ("act_order", C.c_int), ("shift_b", C.c_float), ("delta", C.c_float)]


class _Mlp(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("w1", "b1", "w2", "b2", "w3", "b3")]


class _Samples(C.Structure):
    _fields_ = [("t", C.c_void_p), ("dt", C.c_void_p), ("n_per_ray", C.c_int)]


class _ViewRig(C.Structure):
    _fields_ = [("n_views", C.c_int), ("height", C.c_int), ("width", C.c_int), ("fx", C.c_double),
                ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double), ("near", C.c_double)]


class _AdamH(C.Structure):
    _fields_ = [("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("step", C.c_int), ("skip_zero_grad", C.c_int)]


class _AdamTensor(C.Structure):
    _fields_ = [("param", C.c_void_p), ("grad", C.c_void_p), ("m", C.c_void_p), ("v", C.c_void_p),
                ("n", C.c_size_t), ("h", _AdamH), ("lr_scale", C.c_void_p), ("param_bf16_out", C.c_void_p),
                ("zero_grad", C.c_int)]


DVGO_ADAM_MAX_TENSORS = 4


def lib():
    """Load libdvgo.so; raise if it has not been built (there is no fallback path)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                               "or python paper_2111_11215_gb300/build_lib.py")
        L = C.CDLL(path)
        vp, i, sz, f = C.c_void_p, C.c_int, C.c_size_t, C.c_float
        L.dvgo_workspace_size.restype = sz
        L.dvgo_workspace_size.argtypes = [vp, vp, i, vp]
        L.dvgo_render_fwd.restype = i
        L.dvgo_render_fwd.argtypes = [vp, vp, vp, vp, vp, vp, i, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]
        L.dvgo_render_bwd.restype = i
        L.dvgo_render_bwd.argtypes = [vp, vp, vp, vp, vp, vp, i, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]
        L.dvgo_adam_step.restype = i
        L.dvgo_adam_step.argtypes = [vp, vp, vp, vp, sz, vp, vp, vp, i, vp]
        L.dvgo_adam_step_multi.restype = i
        L.dvgo_adam_step_multi.argtypes = [vp, i, vp]
        L.dvgo_lr_at.restype = f
        L.dvgo_lr_at.argtypes = [f, i, f]
        L.dvgo_workspace_status.restype = i
        L.dvgo_workspace_status.argtypes = [vp, vp]
        L.dvgo_sample_counts.restype = i
        L.dvgo_sample_counts.argtypes = [vp, i, vp, vp, vp]
        L.dvgo_weight_bins.restype = i
        L.dvgo_weight_bins.argtypes = [vp, vp, i, i, vp, sz, vp, vp]
        L.dvgo_proposal_fwd.restype = i
        L.dvgo_proposal_fwd.argtypes = [vp, vp, vp, vp, i, vp, vp, vp, vp, vp, vp]
        L.dvgo_proposal_bwd.restype = i
        L.dvgo_proposal_bwd.argtypes = [vp, vp, vp, vp, i, vp, vp, vp, vp, vp]
        L.dvgo_sample_pdf.restype = i
        L.dvgo_sample_pdf.argtypes = [vp, vp, i, vp, vp, vp, i, i, vp, f, vp, vp, vp]
        L.dvgo_unknown_bbox.restype = i
        L.dvgo_unknown_bbox.argtypes = [vp, vp, vp]
        L.dvgo_grid_elements.restype = sz
        L.dvgo_grid_elements.argtypes = [vp]
        L.dvgo_pack_grid.restype = i
        L.dvgo_pack_grid.argtypes = [vp, vp, vp, vp, vp]
        L.dvgo_resize_grid.restype = i
        L.dvgo_resize_grid.argtypes = [vp, vp, vp, vp, vp]
        L.dvgo_fit2d.restype = i
        L.dvgo_fit2d.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.dvgo_touched_points.restype = i
        L.dvgo_touched_points.argtypes = [vp, vp, i, vp, vp, sz, vp, vp, vp]
        L.dvgo_view_counts.restype = i
        L.dvgo_view_counts.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.dvgo_render_fwd_noalloc.restype = i
        L.dvgo_render_fwd_noalloc.argtypes = [vp, vp, vp, vp, vp, i, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.dvgo_profile_enable.restype = i
        L.dvgo_profile_enable.argtypes = [i]
        L.dvgo_profile_read.restype = i
        L.dvgo_profile_read.argtypes = [i, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]
        L.dvgo_profile_trace.restype = i
        L.dvgo_profile_trace.argtypes = [i, C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                         C.POINTER(C.c_int)]
        L.dvgo_launch_counter.restype = C.c_longlong
        L.dvgo_launch_counter.argtypes = []
        L.dvgo_shift_from_alpha_init.restype = f
        L.dvgo_shift_from_alpha_init.argtypes = [f, f]
        L.dvgo_status_string.restype = C.c_char_p
        L.dvgo_status_string.argtypes = [i]
        L.dvgo_abi_version.restype = i
        _lib = L
    return _lib


# ----------------------------------------------------------------------------------------------
# Python-side descriptors
# ----------------------------------------------------------------------------------------------

@dataclass
class GridDesc:
    shape: tuple                     # lattice points (nx, ny, nz)
    channels: int
    xyz_min: tuple = (-1.0, -1.0, -1.0)
    xyz_max: tuple = (1.0, 1.0, 1.0)
    dtype: int = DVGO_DTYPE_F32
    layout: int = DVGO_LAYOUT_CANONICAL

    def c(self) -> _GridDesc:
        g = _GridDesc()
        g.nx, g.ny, g.nz = (int(v) for v in self.shape)
        g.channels = int(self.channels)
        g.xyz_min[:] = [float(v) for v in self.xyz_min]
        g.xyz_max[:] = [float(v) for v in self.xyz_max]
        g.dtype = int(self.dtype)
        g.layout = int(self.layout)
        return g

    def with_(self, **kw) -> "GridDesc":
        return dataclasses.replace(self, **kw)


@dataclass
class FreeSpace:
    """Known free space of the fine stage (Sec. 4.2): the optimised coarse density grid (CUDA
    FP32 tensor [nx, ny, nz]) on its lattice `desc`, with the coarse stage's shift and step, and
    the threshold tau_c."""
    density: torch.Tensor
    desc: "GridDesc"
    shift_b: float
    step: float
    tau: float = 1e-3

    def c(self) -> _FreeSpace:
        f = _FreeSpace()
        f.desc = self.desc.c()
        f.density = _dev(self.density, "freespace.density", torch.float32)
        f.shift_b, f.step, f.tau = float(self.shift_b), float(self.step), float(self.tau)
        return f


@dataclass
class Params:
    mode: int = DVGO_MODE_COARSE
    step: float = 0.03125
    shift_b: float = 0.0
    tau_f: float = 0.0
    t_near: float = 0.0
    t_far: float = 1e30
    bg: tuple = (1.0, 1.0, 1.0)
    rgb_act: int = 0
    mlp_prec: int = DVGO_MLP_FP32
    n_freq_dir: int = 4
    hidden: int = 128
    freespace: FreeSpace | None = None
    w_pt_rgb: float = 0.0        # per-point rgb loss weight (Supp. A)
    w_bg: float = 0.0            # background entropy loss weight (Supp. A)
    act_order: int = 0           # Sec. 3 interpolation / activation order: 0 post, 1 pre, 2 in
    n_freq_pos: int = 0          # PE frequencies on the query point x (Supp. A: 5); 0: x not an MLP input
    wait_limit_us: int = 0       # tensor-core kernels: bound on every device wait (0: 2 s)
    test_withhold_tile: int = 0  # testing aid: k > 0 withholds one producer arrival on tile k - 1
    cgrid_ready: int = 0         # cudaEvent_t handle (torch.cuda.Event.cuda_event) the render calls
                                 # wait on before their first kernel that reads the colour grid; 0: none
    forward_only: int = 0        # no backward follows the forward: keep nothing for one
    density_ready: int = 0       # cudaEvent_t handle the render calls wait on before their first kernel
                                 # that reads the density grid; 0: none

    def mlp_in_dim(self, channels: int = 12) -> int:
        """Width of the fine MLP's input row (Sec. 4.2 Eq. fine_queries_rgb): 39, or 72 with PE(x)."""
        return channels + 3 + 6 * self.n_freq_dir + (3 + 6 * self.n_freq_pos if self.n_freq_pos > 0 else 0)

    def with_(self, **kw) -> "Params":
        return dataclasses.replace(self, **kw)

    def c(self) -> _Params:
        p = _Params()
        p.mode, p.rgb_act, p.mlp_prec = int(self.mode), int(self.rgb_act), int(self.mlp_prec)
        p.n_freq_dir, p.hidden = int(self.n_freq_dir), int(self.hidden)
        p.step, p.shift_b, p.tau_f = float(self.step), float(self.shift_b), float(self.tau_f)
        p.t_near, p.t_far = float(self.t_near), float(self.t_far)
        p.bg[:] = [float(v) for v in self.bg]
        p.w_pt_rgb, p.w_bg = float(self.w_pt_rgb), float(self.w_bg)
        p.act_order = int(self.act_order)
        p.n_freq_pos = int(self.n_freq_pos)
        p.wait_limit_us = int(self.wait_limit_us)
        p.test_withhold_tile = int(self.test_withhold_tile)
        p.cgrid_ready = int(self.cgrid_ready) or None
        p.forward_only = int(self.forward_only)
        p.density_ready = int(self.density_ready) or None
        if self.freespace is not None:
            p._fs = self.freespace.c()          # kept alive with the struct that points to it
            p.freespace = C.pointer(p._fs)
        return p


def _dev(t, name, dtype=None, allow_none=False):
    if t is None:
        if allow_none:
            return None
        raise ValueError(f"{name} is required")
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype not in (dtype if isinstance(dtype, tuple) else (dtype,)):
        raise ValueError(f"{name} must have dtype {dtype}, got {t.dtype}")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _mlp_struct(mlp):
    if mlp is None:
        return None
    m = _Mlp()
    for k in ("w1", "b1", "w2", "b2", "w3", "b3"):
        setattr(m, k, _dev(mlp[k], f"mlp.{k}", torch.float32))
    return m


def _samples_struct(samples):
    if samples is None:
        return None
    t, dt = samples
    s = _Samples()
    s.t = _dev(t, "samples.t", torch.float32)
    s.dt = _dev(dt, "samples.dt", torch.float32)
    s.n_per_ray = int(t.shape[-1])
    return s


def _ref(x):
    return None if x is None else C.byref(x)


def _check(status, where):
    if status != DVGO_OK:
        raise DVGOError(status, where)


# ----------------------------------------------------------------------------------------------
# Entry points (same names and argument order as include/dvgo.h)
# ----------------------------------------------------------------------------------------------

def dvgo_abi_version() -> int:
    return int(lib().dvgo_abi_version())


def dvgo_status_string(status: int) -> str:
    return lib().dvgo_status_string(int(status)).decode()


def dvgo_shift_from_alpha_init(alpha_init: float, voxel_size: float) -> float:
    return float(lib().dvgo_shift_from_alpha_init(alpha_init, voxel_size))


def dvgo_lr_at(lr0: float, step: int, decay_steps: float = 20000.0) -> float:
    return float(lib().dvgo_lr_at(lr0, step, decay_steps))


def dvgo_touched_points(params: Params, density_desc: GridDesc, n_rays: int, samples, workspace, stream=None):
    """Lattice points the last fine forward on `workspace` read: returns (bitmaps [2, W] int32 view of
    the uint32 words -- density, then features -- and counts [2] int64, both on the device)."""
    n = int(density_desc.shape[0]) * int(density_desc.shape[1]) * int(density_desc.shape[2])
    words = (n + 31) // 32
    bm = torch.empty((2, words), dtype=torch.int32, device=workspace.device)
    counts = torch.empty(2, dtype=torch.int64, device=workspace.device)
    p, g = params.c(), density_desc.c()
    s = _samples_struct(samples)
    _check(lib().dvgo_touched_points(C.byref(p), C.byref(g), int(n_rays), _ref(s),
                                     _dev(workspace, "workspace", torch.uint8), workspace.numel(),
                                     C.c_void_p(bm.data_ptr()), C.c_void_p(counts.data_ptr()), _stream(stream)),
           "dvgo_touched_points")
    return bm, counts


def dvgo_view_counts(desc: GridDesc, c2w, height: int, width: int, fx: float, fy=None, cx=None, cy=None,
                     near: float = 0.0, with_scale: bool = True, stream=None):
    """Sec. 4.1 Prior 2 on the lattice of `desc`: per point the number of views (camera-to-world CUDA
    float64 [V, 3, 4], OpenGL axes) that see it, and the learning-rate scale n_j / n_max.  Returns
    (counts int32 view of the uint32 grid in desc's storage layout, scale float32 or None, n_max
    int32 [1]), all on the device; fy defaults to fx, (cx, cy) to the image centre."""
    c2w = c2w.reshape(-1, 3, 4)
    r = _ViewRig()
    r.n_views, r.height, r.width = int(c2w.shape[0]), int(height), int(width)
    r.fx = float(fx)
    r.fy = float(fx if fy is None else fy)
    r.cx = float(0.5 * width if cx is None else cx)
    r.cy = float(0.5 * height if cy is None else cy)
    r.near = float(near)
    g = desc.c()
    n = int(dvgo_grid_elements(desc))
    counts = torch.empty(n, dtype=torch.int32, device=c2w.device)
    scale = torch.empty(n, dtype=torch.float32, device=c2w.device) if with_scale else None
    n_max = torch.empty(1, dtype=torch.int32, device=c2w.device)
    _check(lib().dvgo_view_counts(C.byref(g), C.byref(r), _dev(c2w, "c2w", torch.float64),
                                  C.c_void_p(counts.data_ptr()), _dev(scale, "lr_scale", torch.float32, True),
                                  C.c_void_p(n_max.data_ptr()), _stream(stream)), "dvgo_view_counts")
    return counts, scale, n_max


def dvgo_workspace_size(params: Params, density_desc: GridDesc, n_rays: int, samples=None) -> int:
    p, g = params.c(), density_desc.c()
    s = _samples_struct(samples) if samples is not None else None
    return int(lib().dvgo_workspace_size(C.byref(p), C.byref(g), int(n_rays), _ref(s)))


def dvgo_render_fwd(params: Params, density_desc: GridDesc, density, cgrid_desc: GridDesc, cgrid, mlp,
                    rays_o, rays_d, jitter, samples, target, rgb_out, tfinal_out, loss_out, dloss_drgb_out,
                    workspace, stream=None):
    p, dd, cd = params.c(), density_desc.c(), cgrid_desc.c()
    m, s = _mlp_struct(mlp), _samples_struct(samples)
    R = int(rays_o.shape[0])
    st = lib().dvgo_render_fwd(
        C.byref(p), C.byref(dd), _dev(density, "density", torch.float32), C.byref(cd),
        _dev(cgrid, "cgrid", (torch.float32, torch.bfloat16)), _ref(m), R,
        _dev(rays_o, "rays_o", torch.float32), _dev(rays_d, "rays_d", torch.float32),
        _dev(jitter, "jitter", torch.float32, True), _ref(s), _dev(target, "target", torch.float32, True),
        _dev(rgb_out, "rgb_out", torch.float32), _dev(tfinal_out, "tfinal_out", torch.float32, True),
        _dev(loss_out, "loss_out", torch.float32, True), _dev(dloss_drgb_out, "dloss_drgb_out", torch.float32, True),
        _dev(workspace, "workspace", torch.uint8), workspace.numel(), _stream(stream))
    _check(st, "dvgo_render_fwd")


def dvgo_render_bwd(params: Params, density_desc: GridDesc, density, cgrid_desc: GridDesc, cgrid, mlp,
                    rays_o, rays_d, jitter, samples, grad_rgb, grad_tfinal, grad_density, grad_cgrid, grad_mlp,
                    workspace, stream=None):
    p, dd, cd = params.c(), density_desc.c(), cgrid_desc.c()
    m, s = _mlp_struct(mlp), _samples_struct(samples)
    R = int(rays_o.shape[0])
    st = lib().dvgo_render_bwd(
        C.byref(p), C.byref(dd), _dev(density, "density", torch.float32), C.byref(cd),
        _dev(cgrid, "cgrid", (torch.float32, torch.bfloat16)), _ref(m), R,
        _dev(rays_o, "rays_o", torch.float32), _dev(rays_d, "rays_d", torch.float32),
        _dev(jitter, "jitter", torch.float32, True), _ref(s), _dev(grad_rgb, "grad_rgb", torch.float32),
        _dev(grad_tfinal, "grad_tfinal", torch.float32, True), _dev(grad_density, "grad_density", torch.float32),
        _dev(grad_cgrid, "grad_cgrid", torch.float32), _dev(grad_mlp, "grad_mlp", torch.float32, True),
        _dev(workspace, "workspace", torch.uint8), workspace.numel(), _stream(stream))
    _check(st, "dvgo_render_bwd")


def dvgo_adam_step(param, grad, m, v, lr: float, step: int, beta1=0.9, beta2=0.999, eps=1e-8,
                   lr_scale=None, param_bf16_out=None, zero_grad=True, stream=None, skip_zero_grad=False):
    h = _AdamH()
    h.lr, h.beta1, h.beta2, h.eps, h.step = float(lr), float(beta1), float(beta2), float(eps), int(step)
    h.skip_zero_grad = int(bool(skip_zero_grad))
    st = lib().dvgo_adam_step(
        _dev(param, "param", torch.float32), _dev(grad, "grad", torch.float32), _dev(m, "m", torch.float32),
        _dev(v, "v", torch.float32), param.numel(), C.byref(h), _dev(lr_scale, "lr_scale", torch.float32, True),
        _dev(param_bf16_out, "param_bf16_out", torch.bfloat16, True), int(bool(zero_grad)), _stream(stream))
    _check(st, "dvgo_adam_step")


def dvgo_adam_step_multi(tensors, stream=None):
    """dvgo_adam_step on several tensors in one launch.  tensors: sequence of dicts with the keys
    of dvgo_adam_step (param, grad, m, v, lr, step; optional beta1, beta2, eps, lr_scale,
    param_bf16_out, zero_grad, skip_zero_grad)."""
    arr = (_AdamTensor * max(len(tensors), 1))()
    keep = []
    for j, t in enumerate(tensors):
        x = arr[j]
        x.param, x.grad = _dev(t["param"], "param", torch.float32), _dev(t["grad"], "grad", torch.float32)
        x.m, x.v = _dev(t["m"], "m", torch.float32), _dev(t["v"], "v", torch.float32)
        x.n = t["param"].numel()
        x.h.lr, x.h.beta1, x.h.beta2 = float(t["lr"]), float(t.get("beta1", 0.9)), float(t.get("beta2", 0.999))
        x.h.eps, x.h.step = float(t.get("eps", 1e-8)), int(t["step"])
        x.h.skip_zero_grad = int(bool(t.get("skip_zero_grad", False)))
        x.lr_scale = _dev(t.get("lr_scale"), "lr_scale", torch.float32, True)
        x.param_bf16_out = _dev(t.get("param_bf16_out"), "param_bf16_out", torch.bfloat16, True)
        x.zero_grad = int(bool(t.get("zero_grad", True)))
        keep.append(t)
    _check(lib().dvgo_adam_step_multi(arr, len(tensors), _stream(stream)), "dvgo_adam_step_multi")


def dvgo_workspace_status(workspace, stream=None) -> int:
    return int(lib().dvgo_workspace_status(_dev(workspace, "workspace", torch.uint8), _stream(stream)))


def dvgo_sample_counts(workspace, n_rays: int, counts_out, total_out=None, stream=None):
    st = lib().dvgo_sample_counts(_dev(workspace, "workspace", torch.uint8), int(n_rays),
                                  _dev(counts_out, "counts_out", torch.int32), _dev(total_out, "total_out", torch.int32, True),
                                  _stream(stream))
    _check(st, "dvgo_sample_counts")


def dvgo_profile_enable(on: bool):
    _check(lib().dvgo_profile_enable(int(bool(on))), "dvgo_profile_enable")


def dvgo_profile_read(kind) -> tuple:
    """(total device ms, launches) of one kernel kind since the last read; kind is an index or a
    name from KERNEL_KINDS."""
    k = KERNEL_KINDS.index(kind) if isinstance(kind, str) else int(kind)
    ms, n = C.c_double(0.0), C.c_longlong(0)
    _check(lib().dvgo_profile_read(k, C.byref(ms), C.byref(n)), "dvgo_profile_read")
    return ms.value, n.value


def dvgo_profile_trace(max_records: int = 65536) -> list:
    """The launches recorded while profiling was enabled, in launch order: (kind name, start ms,
    end ms) relative to the first one's start; forgets every record."""
    n = int(max_records)
    kinds, a, b = (C.c_int * max(n, 1))(), (C.c_double * max(n, 1))(), (C.c_double * max(n, 1))()
    got = C.c_int(0)
    _check(lib().dvgo_profile_trace(n, kinds, a, b, C.byref(got)), "dvgo_profile_trace")
    return [(KERNEL_KINDS[kinds[i]], a[i], b[i]) for i in range(got.value)]


def dvgo_launch_counter() -> int:
    return int(lib().dvgo_launch_counter())


def dvgo_render_fwd_noalloc(params: Params, density_desc: GridDesc, density, cgrid_desc: GridDesc, cgrid, rays_o,
                            rays_d, jitter, target, rgb_out, tfinal_out, loss_out, dloss_drgb_out, stream=None):
    """Coarse forward with the library's static scratch instead of a workspace (for callers that
    cannot allocate device memory); at most DVGO_NOALLOC_MAX_RAYS rays per call."""
    p, dd, cd = params.c(), density_desc.c(), cgrid_desc.c()
    st = lib().dvgo_render_fwd_noalloc(
        C.byref(p), C.byref(dd), _dev(density, "density", torch.float32), C.byref(cd),
        _dev(cgrid, "cgrid", torch.float32), int(rays_o.shape[0]), _dev(rays_o, "rays_o", torch.float32),
        _dev(rays_d, "rays_d", torch.float32), _dev(jitter, "jitter", torch.float32, True),
        _dev(target, "target", torch.float32, True), _dev(rgb_out, "rgb_out", torch.float32),
        _dev(tfinal_out, "tfinal_out", torch.float32, True), _dev(loss_out, "loss_out", torch.float32, True),
        _dev(dloss_drgb_out, "dloss_drgb_out", torch.float32, True), _stream(stream))
    _check(st, "dvgo_render_fwd_noalloc")


# ----------------------------------------------------------------------------------------------
# Learned sample proposal
# ----------------------------------------------------------------------------------------------

PROP_KEYS = ("w0", "b0", "w1", "b1", "w2", "b2", "w3", "b3")


class _PropDesc(C.Structure):
    _fields_ = [("n_bins", C.c_int), ("n_freq", C.c_int), ("width", C.c_int), ("precision", C.c_int)]


class _PropMlp(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in PROP_KEYS]


def _prop(n_bins, n_freq, width, mlp, precision=DVGO_MLP_FP32):
    d = _PropDesc()
    d.n_bins, d.n_freq, d.width, d.precision = int(n_bins), int(n_freq), int(width), int(precision)
    m = _PropMlp()
    for k in PROP_KEYS:
        setattr(m, k, _dev(mlp[k], f"proposal.{k}", torch.float32))
    return d, m


def dvgo_weight_bins(params: Params, density_desc: GridDesc, n_rays: int, n_bins: int, workspace, labels_out,
                     stream=None):
    p, g = params.c(), density_desc.c()
    st = lib().dvgo_weight_bins(C.byref(p), C.byref(g), int(n_rays), int(n_bins),
                                _dev(workspace, "workspace", torch.uint8), workspace.numel(),
                                _dev(labels_out, "labels_out", torch.float32), _stream(stream))
    _check(st, "dvgo_weight_bins")


def dvgo_proposal_fwd(params: Params, density_desc: GridDesc, n_bins: int, n_freq: int, width: int, mlp, rays_o,
                      rays_d, labels, probs_out, loss_out, stream=None, precision=DVGO_MLP_FP32):
    p, g = params.c(), density_desc.c()
    d, m = _prop(n_bins, n_freq, width, mlp, precision)
    st = lib().dvgo_proposal_fwd(C.byref(p), C.byref(g), C.byref(d), C.byref(m), int(rays_o.shape[0]),
                                 _dev(rays_o, "rays_o", torch.float32), _dev(rays_d, "rays_d", torch.float32),
                                 _dev(labels, "labels", torch.float32, True), _dev(probs_out, "probs_out", torch.float32),
                                 _dev(loss_out, "loss_out", torch.float32, True), _stream(stream))
    _check(st, "dvgo_proposal_fwd")


def dvgo_proposal_bwd(params: Params, density_desc: GridDesc, n_bins: int, n_freq: int, width: int, mlp, rays_o,
                      rays_d, labels, grad_mlp, stream=None, precision=DVGO_MLP_FP32):
    p, g = params.c(), density_desc.c()
    d, m = _prop(n_bins, n_freq, width, mlp, precision)
    st = lib().dvgo_proposal_bwd(C.byref(p), C.byref(g), C.byref(d), C.byref(m), int(rays_o.shape[0]),
                                 _dev(rays_o, "rays_o", torch.float32), _dev(rays_d, "rays_d", torch.float32),
                                 _dev(labels, "labels", torch.float32), _dev(grad_mlp, "grad_mlp", torch.float32),
                                 _stream(stream))
    _check(st, "dvgo_proposal_bwd")


def dvgo_sample_pdf(params: Params, density_desc: GridDesc, rays_o, rays_d, probs, n_samples: int, jitter, eta,
                    t_out, dt_out, stream=None):
    p, g = params.c(), density_desc.c()
    st = lib().dvgo_sample_pdf(C.byref(p), C.byref(g), int(rays_o.shape[0]), _dev(rays_o, "rays_o", torch.float32),
                               _dev(rays_d, "rays_d", torch.float32), _dev(probs, "probs", torch.float32),
                               int(probs.shape[-1]), int(n_samples), _dev(jitter, "jitter", torch.float32, True),
                               float(eta), _dev(t_out, "t_out", torch.float32), _dev(dt_out, "dt_out", torch.float32),
                               _stream(stream))
    _check(st, "dvgo_sample_pdf")


def dvgo_unknown_bbox(fs: FreeSpace, out=None, stream=None):
    """Sec. 4.2 fine voxels allocation on the coarse grid: int32 device tensor [count, lo(3), hi(3)]."""
    out = torch.empty(7, dtype=torch.int32, device=fs.density.device) if out is None else out
    f = fs.c()
    _check(lib().dvgo_unknown_bbox(C.byref(f), _dev(out, "out", torch.int32), _stream(stream)), "dvgo_unknown_bbox")
    return out


def dvgo_grid_elements(desc: GridDesc) -> int:
    """Scalar elements of a grid's storage in its layout (padding points of the packed layout
    included)."""
    g = desc.c()
    return int(lib().dvgo_grid_elements(C.byref(g)))


def dvgo_fit2d(grid, target=None, act_order: int = DVGO_ACT_POST, shift_b: float = 0.0, delta: float = 1.0,
               image_out=None, grad_out=None, loss_out=None, stream=None, image_shape=None):
    """Image-fitting toy of Sec. 3: grid [gh, gw] and target [H, W] (CUDA FP32).  Writes the
    predicted image (image_out), the MSE (loss_out[0]) and accumulates dL/dgrid (grad_out), each
    optional.  Without a target, image_shape (H, W) gives the image size."""
    H, W = (target.shape if target is not None else image_shape)
    for t, n, name in ((target, H * W, "target"), (image_out, H * W, "image_out"),
                       (grad_out, grid.numel(), "grad_out")):
        if t is not None and t.numel() != n:
            raise ValueError(f"dvgo_fit2d: {name} has {t.numel()} elements, expected {n}")
    if grid.dim() != 2 or (loss_out is not None and loss_out.numel() < 1):
        raise ValueError("dvgo_fit2d: grid must be [grid_h, grid_w] and loss_out hold one element")
    d = _Fit2d()
    d.height, d.width, d.grid_h, d.grid_w = int(H), int(W), int(grid.shape[0]), int(grid.shape[1])
    d.act_order, d.shift_b, d.delta = int(act_order), float(shift_b), float(delta)
    _check(lib().dvgo_fit2d(C.byref(d), _dev(grid, "grid", torch.float32),
                            _dev(target, "target", torch.float32, allow_none=True),
                            _dev(image_out, "image_out", torch.float32, allow_none=True),
                            _dev(grad_out, "grad_out", torch.float32, allow_none=True),
                            _dev(loss_out, "loss_out", torch.float32, allow_none=True), _stream(stream)), "dvgo_fit2d")


def dvgo_resize_grid(src_desc: GridDesc, src, dst_desc: GridDesc, out=None, stream=None):
    """Progressive scaling (Sec. 4.2): trilinear resize of an FP32 grid onto the lattice of
    dst_desc; returns the (flat) output tensor."""
    if out is None:
        out = torch.empty(dvgo_grid_elements(dst_desc), dtype=torch.float32, device=src.device)
    if out.numel() != dvgo_grid_elements(dst_desc) or src.numel() != dvgo_grid_elements(src_desc):
        raise ValueError("dvgo_resize_grid: tensor sizes do not match the descriptors")
    a, b = src_desc.c(), dst_desc.c()
    _check(lib().dvgo_resize_grid(C.byref(a), _dev(src, "src", torch.float32), C.byref(b),
                                  _dev(out, "out", torch.float32), _stream(stream)), "dvgo_resize_grid")
    return out


def dvgo_pack_grid(src_desc: GridDesc, src, dst_desc: GridDesc, out=None, stream=None):
    """Copy a grid into another layout / element type on the same lattice; returns the (flat)
    output tensor."""
    dt = torch.bfloat16 if dst_desc.dtype == DVGO_DTYPE_BF16 else torch.float32
    st = torch.bfloat16 if src_desc.dtype == DVGO_DTYPE_BF16 else torch.float32
    if out is None:
        out = torch.empty(dvgo_grid_elements(dst_desc), dtype=dt, device=src.device)
    if out.numel() != dvgo_grid_elements(dst_desc) or src.numel() != dvgo_grid_elements(src_desc):
        raise ValueError("dvgo_pack_grid: tensor sizes do not match the descriptors")
    a, b = src_desc.c(), dst_desc.c()
    _check(lib().dvgo_pack_grid(C.byref(a), _dev(src, "src", st), C.byref(b), _dev(out, "out", dt), _stream(stream)),
           "dvgo_pack_grid")
    return out
