"""FP64 CPU oracle for the DVGO render step (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs
of ``bench.py`` may import this package.  The product (the CUDA library and its Python binding)
never imports it and shares no code with it.

The arithmetic lives in ``dvgo_oracle.c`` (plain C, double precision, one loop per ray); this
module only compiles it with gcc and marshals numpy arrays through ctypes.  Every function cites
the passage of the paper (Sun, Sun & Chen, "Direct Voxel Grid Optimization", arXiv 2111.11215)
that it restates; the C file lists the readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dvgo_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libdvgo_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available, no FP contraction)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", _SRC, "-o", _LIB_PATH + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)  # single-threaded fallback
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.oracle_shift_from_alpha_init.restype = C.c_double
        _lib.oracle_shift_from_alpha_init.argtypes = [C.c_double, C.c_double]
        _lib.oracle_lr_decay.restype = C.c_double
        _lib.oracle_lr_decay.argtypes = [C.c_double, C.c_int, C.c_double]
        _lib.oracle_alpha_at.restype = C.c_double
        _lib.oracle_num_threads.restype = C.c_int
    return _lib


def num_threads() -> int:
    return int(lib().oracle_num_threads())


# ----------------------------------------------------------------------------------------------
# ctypes mirrors of the C structs
# ----------------------------------------------------------------------------------------------

_dp = C.POINTER(C.c_double)


class _Params(C.Structure):
    _fields_ = [("mode", C.c_int), ("rgb_act", C.c_int), ("feat_dim", C.c_int), ("n_freq", C.c_int),
                ("hidden", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("xyz_min", C.c_double * 3), ("xyz_max", C.c_double * 3), ("shift_b", C.c_double),
                ("delta", C.c_double), ("tau_f", C.c_double), ("t_near", C.c_double),
                ("t_far", C.c_double), ("bg", C.c_double * 3), ("w_pt", C.c_double), ("w_bg", C.c_double),
                ("act_order", C.c_int), ("n_freq_pos", C.c_int), ("mlp_operands", C.c_int)]


class _FreeSpace(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("xyz_min", C.c_double * 3),
                ("xyz_max", C.c_double * 3), ("shift_b", C.c_double), ("delta", C.c_double), ("tau", C.c_double),
                ("density", _dp)]


class _Model(C.Structure):
    _fields_ = [(n, _dp) for n in ("density", "cgrid", "w1", "b1", "w2", "b2", "w3", "b3")] + \
        [("fs", C.POINTER(_FreeSpace)), ("mark_density", C.POINTER(C.c_ubyte)), ("mark_cgrid", C.POINTER(C.c_ubyte))]


class _Grads(C.Structure):
    _fields_ = [(n, _dp) for n in ("density", "cgrid", "w1", "b1", "w2", "b2", "w3", "b3")]


class _Bound(C.Structure):
    _fields_ = [("u_op", C.c_double), ("u_acc", C.c_double), ("E", _Grads)]


class _Prop(C.Structure):
    _fields_ = [("n_bins", C.c_int), ("n_freq", C.c_int), ("width", C.c_int),
                ("w", _dp * 4), ("b", _dp * 4)]


class _PropGrads(C.Structure):
    _fields_ = [("w", _dp * 4), ("b", _dp * 4)]


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_dp)


@dataclass
class Params:
    """Render parameters (Eq. volume_rendering, Eq. density_activation, Sec. 4.2 sampling)."""
    grid_shape: tuple            # lattice points (nx, ny, nz)
    xyz_min: tuple = (-1.0, -1.0, -1.0)
    xyz_max: tuple = (1.0, 1.0, 1.0)
    shift_b: float = 0.0
    delta: float = 0.03125
    tau_f: float = 0.0
    t_near: float = 0.0
    t_far: float = 1e30
    bg: tuple = (1.0, 1.0, 1.0)
    mode: int = 0                # 0 coarse (colour grid), 1 fine (feature grid + MLP)
    rgb_act: int = 0
    feat_dim: int = 3
    n_freq: int = 4
    hidden: int = 128
    w_pt: float = 0.0            # per-point rgb loss weight (Supp. A w_pt_rgb)
    w_bg: float = 0.0            # background entropy loss weight (Supp. A w_bg)
    act_order: int = 0           # Sec. 3: 0 post- (the paper's), 1 pre-, 2 in-activation
    n_freq_pos: int = 0          # PE frequencies on the query point x (Supp. A k_x = 5); 0: x not input
    mlp_operands: int = 0        # colour-MLP contractions: 0 exact; 1 BF16 operands (the chosen form's arithmetic)

    @property
    def in_dim(self) -> int:
        """Width of the fine MLP input row (Eq. fine_queries_rgb)."""
        return self.feat_dim + 3 + 6 * self.n_freq + (3 + 6 * self.n_freq_pos if self.n_freq_pos > 0 else 0)

    def _c(self) -> _Params:
        p = _Params()
        p.mode, p.rgb_act, p.feat_dim, p.n_freq, p.hidden = self.mode, self.rgb_act, self.feat_dim, self.n_freq, self.hidden
        p.nx, p.ny, p.nz = (int(v) for v in self.grid_shape)
        p.xyz_min[:] = [float(v) for v in self.xyz_min]
        p.xyz_max[:] = [float(v) for v in self.xyz_max]
        p.shift_b, p.delta, p.tau_f = float(self.shift_b), float(self.delta), float(self.tau_f)
        p.t_near, p.t_far = float(self.t_near), float(self.t_far)
        p.bg[:] = [float(v) for v in self.bg]
        p.w_pt, p.w_bg = float(self.w_pt), float(self.w_bg)
        p.act_order = int(self.act_order)
        p.n_freq_pos = int(self.n_freq_pos)
        p.mlp_operands = int(self.mlp_operands)
        return p


@dataclass
class RenderResult:
    rgb: np.ndarray
    tfinal: np.ndarray
    n_samples: np.ndarray
    t_enter: np.ndarray
    t_exit: np.ndarray
    loss: float | None = None
    grads: dict = field(default_factory=dict)
    wbins: np.ndarray | None = None
    touched: dict | None = None
    bounds: dict = field(default_factory=dict)


MLP_KEYS = ("w1", "b1", "w2", "b2", "w3", "b3")


def shift_from_alpha_init(alpha_init: float, voxel_size: float) -> float:
    """Sec. 4.1 Eq. low_density_init."""
    return float(lib().oracle_shift_from_alpha_init(alpha_init, voxel_size))


def lr_decay(lr0: float, step: int, decay_steps: float = 20000.0) -> float:
    """Supp. A: learning rates are scaled by 0.1 at 20k iterations, exponentially."""
    return float(lib().oracle_lr_decay(lr0, step, decay_steps))


@dataclass
class FreeSpace:
    """Known free space of Sec. 4.2: the optimised coarse density grid with its lattice, shift b_c,
    step delta_c and threshold tau_c."""
    density: np.ndarray
    xyz_min: tuple = (-1.0, -1.0, -1.0)
    xyz_max: tuple = (1.0, 1.0, 1.0)
    shift_b: float = 0.0
    delta: float = 0.03125
    tau: float = 1e-3

    def _c(self):
        F = _FreeSpace()
        d = _f64(self.density)
        F.nx, F.ny, F.nz = (int(v) for v in d.shape[:3])
        F.xyz_min[:] = [float(v) for v in self.xyz_min]
        F.xyz_max[:] = [float(v) for v in self.xyz_max]
        F.shift_b, F.delta, F.tau = float(self.shift_b), float(self.delta), float(self.tau)
        F.density = _ptr(d)
        return F, d


def coarse_alpha(fs: FreeSpace, x) -> float:
    """Post-activated alpha of the coarse grid at one point (the known-free-space test)."""
    F, keep = fs._c()
    lib().oracle_coarse_alpha.restype = C.c_double
    lib().oracle_coarse_alpha.argtypes = [C.POINTER(_FreeSpace), _dp]
    return float(lib().oracle_coarse_alpha(C.byref(F), _ptr(_f64(x))))


def unknown_bbox(fs: FreeSpace):
    """Sec. 4.2 fine voxels allocation: (count, lo, hi) lattice-index box of the cells that can hold
    unknown space (alpha_c >= tau_c); lo = hi = None when everything is known free."""
    F, keep = fs._c()
    lo = (C.c_int * 3)()
    hi = (C.c_int * 3)()
    lib().oracle_unknown_bbox.restype = C.c_long
    n = int(lib().oracle_unknown_bbox(C.byref(F), lo, hi))
    if n == 0:
        return 0, None, None
    return n, tuple(lo), tuple(hi)


def render(params: Params, density, cgrid, rays_o, rays_d, jitter=None, mlp: dict | None = None,
           target=None, grad_rgb=None, grad_tfinal=None, explicit_t=None, explicit_dt=None,
           n_bins: int = 0, freespace: FreeSpace | None = None, touched: bool = False,
           error_bound: tuple | None = None) -> RenderResult:
    """Render a ray batch forward and, if ``grad_rgb`` is given, backward (Sec. 2-4).

    density: [nx, ny, nz]; cgrid: [nx, ny, nz, C] (coarse colour or fine features);
    rays_o, rays_d: [R, 3]; jitter: [R] in [0, 1) or None (0.5); mlp: dict of w1..b3 (fine);
    grad_rgb: [R, 3] upstream dL/dC_hat; grad_tfinal: [R] or None; freespace: the known-free-space
    test of Sec. 4.2 (skips points where the coarse grid's alpha is below tau_c); touched: also
    return the lattice points the render reads (boolean [nx, ny, nz] per grid, in ``touched``).
    error_bound: (u_op, u_acc) -- fine stage with grad_rgb: also return in ``bounds`` (keys as
    ``grads``) a first-order bound on |finite-precision gradient - this gradient| per element for MLP
    operands rounded to relative u_op (BF16: 2^-8) and accumulation with unit roundoff u_acc (FP32:
    2^-24); test infrastructure, defined in dvgo_oracle.c (og_bound).
    Returns colours, final transmittances, sample counts, clip bounds, loss and gradients.
    """
    P = params._c()
    density = _f64(density)
    cgrid = _f64(cgrid)
    rays_o = _f64(rays_o).reshape(-1, 3)
    rays_d = _f64(rays_d).reshape(-1, 3)
    R = rays_o.shape[0]
    jit = None if jitter is None else _f64(jitter).reshape(R)
    M = _Model()
    M.density, M.cgrid = _ptr(density), _ptr(cgrid)
    if freespace is not None:
        fs_c, fs_keep = freespace._c()
        M.fs = C.pointer(fs_c)
    marks = None
    if touched:
        marks = {k: np.zeros(tuple(params.grid_shape), dtype=np.uint8) for k in ("density", "cgrid")}
        M.mark_density = marks["density"].ctypes.data_as(C.POINTER(C.c_ubyte))
        M.mark_cgrid = marks["cgrid"].ctypes.data_as(C.POINTER(C.c_ubyte))
    mlp_arrs = {}
    if params.mode == 1:
        for k in MLP_KEYS:
            mlp_arrs[k] = _f64(mlp[k])
            setattr(M, k, _ptr(mlp_arrs[k]))
    tgt = None if target is None else _f64(target).reshape(R, 3)
    rgb = np.zeros((R, 3)); tf = np.zeros(R); ns = np.zeros(R, dtype=np.int32)
    t0 = np.zeros(R); t1 = np.zeros(R); loss = C.c_double(0.0)
    gC = None if grad_rgb is None else _f64(grad_rgb).reshape(R, 3)
    gT = None if grad_tfinal is None else _f64(grad_tfinal).reshape(R)
    G = _Grads()
    grads = {}
    if gC is not None:
        grads["density"] = np.zeros_like(density)
        grads["cgrid"] = np.zeros_like(cgrid)
        G.density, G.cgrid = _ptr(grads["density"]), _ptr(grads["cgrid"])
        if params.mode == 1:
            for k in MLP_KEYS:
                grads[k] = np.zeros_like(mlp_arrs[k])
                setattr(G, k, _ptr(grads[k]))
    n_expl = 0
    ts = dts = None
    if explicit_t is not None:
        ts = _f64(explicit_t).reshape(R, -1)
        dts = _f64(explicit_dt).reshape(R, -1)
        n_expl = ts.shape[1]
    wb = np.zeros((R, n_bins)) if n_bins > 0 else None
    Bd, bounds = None, {}
    if error_bound is not None and gC is not None and params.mode == 1:
        Bd = _Bound()
        Bd.u_op, Bd.u_acc = float(error_bound[0]), float(error_bound[1])
        for k, v in grads.items():
            bounds[k] = np.zeros_like(v)
            setattr(Bd.E, k, _ptr(bounds[k]))
    lib().oracle_render(C.byref(P), C.byref(M), C.c_int(R), _ptr(rays_o), _ptr(rays_d), _ptr(jit),
                        C.c_int(n_expl), _ptr(ts), _ptr(dts), _ptr(tgt), _ptr(rgb), _ptr(tf),
                        ns.ctypes.data_as(C.POINTER(C.c_int)), _ptr(t0), _ptr(t1), C.byref(loss),
                        _ptr(gC), _ptr(gT), C.byref(G) if gC is not None else None, _ptr(wb),
                        C.c_int(n_bins), C.byref(Bd) if Bd is not None else None)
    res = RenderResult(rgb=rgb, tfinal=tf, n_samples=ns, t_enter=t0, t_exit=t1,
                       loss=float(loss.value) if tgt is not None else None, grads=grads, wbins=wb, bounds=bounds)
    if marks is not None:
        res.touched = {k: v.astype(bool) for k, v in marks.items()}
    return res


def bf16(v) -> np.ndarray:
    """Values rounded to BF16 (8 significant bits, to nearest, ties to even), as FP64."""
    v = _f64(v)
    f = lib().oracle_bf16
    f.restype = C.c_double
    f.argtypes = [C.c_double]
    return np.array([f(float(x)) for x in v.reshape(-1)]).reshape(v.shape)


def mlp_sample_bound(params: Params, mlp: dict, e_in, e_err, dc, rho_dc: float, u_op: float, u_acc: float):
    """One fine-MLP sample with its running error bound (og_bound in dvgo_oracle.c; test
    infrastructure): input row e_in [I] with absolute errors e_err [I], upstream dL/dc [3] with
    relative error rho_dc.  Returns (c, bound of c, dL/de, its bound, per-sample weight gradients,
    their bounds), the last two as dicts w1..b3."""
    P = params._c()
    M = _Model()
    arrs = {k: _f64(mlp[k]) for k in MLP_KEYS}
    for k in MLP_KEYS:
        setattr(M, k, _ptr(arrs[k]))
    e_in, e_err, dc = _f64(e_in), _f64(e_err), _f64(dc)
    I = params.in_dim
    c, ec, de, ede = np.zeros(3), np.zeros(3), np.zeros(I), np.zeros(I)
    g = {k: np.zeros_like(v) for k, v in arrs.items()}
    eb = {k: np.zeros_like(v) for k, v in arrs.items()}
    G, Eb = _Grads(), _Grads()
    for k in MLP_KEYS:
        setattr(G, k, _ptr(g[k]))
        setattr(Eb, k, _ptr(eb[k]))
    lib().oracle_mlp_sample_bound(C.byref(P), C.byref(M), _ptr(e_in), _ptr(e_err), _ptr(dc), C.c_double(rho_dc),
                                  C.c_double(u_op), C.c_double(u_acc), _ptr(c), _ptr(ec), _ptr(de), _ptr(ede),
                                  C.byref(G), C.byref(Eb))
    return c, ec, de, ede, g, eb


def ray_bounds(params: Params, o, d, p: float = 0.5):
    """Slab clip and sample count of one ray (Eq. coarse_sample, Sec. 4.2)."""
    P = params._c()
    o = _f64(o); d = _f64(d)
    t0 = C.c_double(); t1 = C.c_double(); n = C.c_int(); dn = np.zeros(3)
    rc = lib().oracle_ray_bounds(C.byref(P), _ptr(o), _ptr(d), C.c_double(p), C.byref(t0), C.byref(t1),
                                 _ptr(dn), C.byref(n))
    return rc, t0.value, t1.value, dn, n.value


def interp(params: Params, grid, x):
    """Sec. 3 Eq. interp: trilinear interpolation of a channel-last grid at one point."""
    P = params._c()
    grid = _f64(grid)
    Cc = 1 if grid.ndim == 3 else grid.shape[-1]
    out = np.zeros(Cc)
    lib().oracle_interp(C.byref(P), _ptr(grid), C.c_int(Cc), _ptr(_f64(x)), _ptr(out))
    return out


def resize_grid(grid, dst_shape, src_box=((-1.0,) * 3, (1.0,) * 3), dst_box=None):
    """Progressive scaling (Sec. 4.2): trilinear resize of a channel-last grid onto the
    align-corners lattice of ``dst_shape`` points over ``dst_box`` (default: the source box)."""
    grid = _f64(grid)
    n = np.array(grid.shape[:3], dtype=np.int32)
    Cc = 1 if grid.ndim == 3 else grid.shape[-1]
    n2 = np.array([int(v) for v in dst_shape], dtype=np.int32)
    dst_box = src_box if dst_box is None else dst_box
    out = np.zeros(tuple(n2) + ((Cc,) if grid.ndim == 4 else ()))
    ip = C.POINTER(C.c_int)
    lib().oracle_resize_grid(n.ctypes.data_as(ip), _ptr(_f64(src_box[0])), _ptr(_f64(src_box[1])), C.c_int(Cc),
                             _ptr(grid), n2.ctypes.data_as(ip), _ptr(_f64(dst_box[0])), _ptr(_f64(dst_box[1])),
                             _ptr(out))
    return out


def fit2d(grid, target, order: int = 0, shift_b: float = 0.0, delta: float = 1.0, grad: bool = False):
    """Image-fitting toy of Sec. 3 (Fig. exdv_poc): the grid's predicted image (bilinear
    interpolation under the pre- / in- / post-activation order, order 1 / 2 / 0), the mean squared
    error to the target and, with grad, dL/dgrid.  Returns (image, loss, grad or None)."""
    V = _f64(grid)
    T = _f64(target)
    (gh, gw), (H, W) = V.shape, T.shape
    img = np.zeros((H, W))
    g = np.zeros_like(V) if grad else None
    f = lib().oracle_fit2d
    f.restype = C.c_double
    loss = f(C.c_int(H), C.c_int(W), C.c_int(gh), C.c_int(gw), C.c_int(order), C.c_double(shift_b),
             C.c_double(delta), _ptr(V), _ptr(T), _ptr(img), _ptr(g))
    return img, float(loss), g


def alpha_at(params: Params, density, x, delta: float) -> float:
    """Eq. post_activation: alpha(softplus(interp(x, V) + b), delta) at one point."""
    P = params._c()
    lib().oracle_alpha_at.argtypes = [C.POINTER(_Params), _dp, _dp, C.c_double]
    return float(lib().oracle_alpha_at(C.byref(P), _ptr(_f64(density)), _ptr(_f64(x)), C.c_double(delta)))


def mlp_forward(params: Params, mlp: dict, e):
    """Shallow colour MLP of Sec. 4.2 / Supp. A on a batch of input rows."""
    P = params._c()
    e = _f64(e)
    M = _Model()
    arrs = {k: _f64(mlp[k]) for k in MLP_KEYS}
    for k in MLP_KEYS:
        setattr(M, k, _ptr(arrs[k]))
    out = np.zeros((e.shape[0], 3))
    lib().oracle_mlp_forward(C.byref(P), C.byref(M), C.c_int(e.shape[0]), _ptr(e), _ptr(out))
    return out


def adam(param, grad, m, v, lr, t, beta1=0.9, beta2=0.999, eps=1e-8, lr_scale=None, zero_grad=True,
         skip_zero_grad=False):
    """One Adam step (Kingma & Ba), in place on float64 arrays; lr already decayed.  skip_zero_grad:
    the lazy variant, elements with an exactly zero gradient keep parameter and moments."""
    for a in (param, grad, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().oracle_adam(C.c_long(param.size), _ptr(param), _ptr(grad), _ptr(m), _ptr(v), C.c_double(lr),
                      C.c_double(beta1), C.c_double(beta2), C.c_double(eps), C.c_int(t),
                      _ptr(None if lr_scale is None else _f64(lr_scale)), C.c_int(int(zero_grad)),
                      C.c_int(int(skip_zero_grad)))


PROP_KEYS = ("w0", "b0", "w1", "b1", "w2", "b2", "w3", "b3")


def proposal(params: Params, prop: dict, n_bins: int, n_freq: int, rays_o, rays_d, labels=None,
             want_grads: bool = False):
    """Sample-proposal network: per-ray softmax PDF over n_bins equal bins of [t_enter, t_exit];
    with labels, the mean cross-entropy loss and (optionally) its gradient."""
    P = params._c()
    rays_o = _f64(rays_o).reshape(-1, 3); rays_d = _f64(rays_d).reshape(-1, 3)
    R = rays_o.shape[0]
    arrs = {k: _f64(prop[k]) for k in PROP_KEYS}
    Q = _Prop()
    Q.n_bins, Q.n_freq, Q.width = n_bins, n_freq, arrs["w1"].shape[0]
    for i in range(4):
        Q.w[i] = _ptr(arrs[f"w{i}"]); Q.b[i] = _ptr(arrs[f"b{i}"])
    probs = np.zeros((R, n_bins))
    loss = C.c_double(0.0)
    lab = None if labels is None else _f64(labels).reshape(R, n_bins)
    grads = None
    G = None
    if want_grads:
        grads = {k: np.zeros_like(arrs[k]) for k in PROP_KEYS}
        G = _PropGrads()
        for i in range(4):
            G.w[i] = _ptr(grads[f"w{i}"]); G.b[i] = _ptr(grads[f"b{i}"])
    lib().oracle_proposal(C.byref(P), C.byref(Q), C.c_int(R), _ptr(rays_o), _ptr(rays_d), _ptr(lab),
                          _ptr(probs), C.byref(loss), C.byref(G) if G is not None else None)
    return probs, (float(loss.value) if lab is not None else None), grads


def sample_pdf(probs, t0: float, t1: float, n_samples: int, jit: float = 0.5, eta: float = 1e-3):
    """Inverse-CDF sampling of sorted samples from a piecewise-constant PDF over equal bins."""
    probs = _f64(probs)
    t = np.zeros(n_samples); dt = np.zeros(n_samples)
    lib().oracle_sample_pdf(C.c_int(probs.size), _ptr(probs), C.c_double(t0), C.c_double(t1),
                            C.c_int(n_samples), C.c_double(jit), C.c_double(eta), _ptr(t), _ptr(dt))
    return t, dt


def _rig_args(c2w, height, width, fx, fy=None, cx=None, cy=None, near=0.0):
    c2w = np.ascontiguousarray(_f64(c2w).reshape(-1, 3, 4))
    fy = fx if fy is None else fy
    cx = 0.5 * width if cx is None else cx
    cy = 0.5 * height if cy is None else cy
    return c2w, (C.c_int(c2w.shape[0]), _ptr(c2w), C.c_int(height), C.c_int(width), C.c_double(fx), C.c_double(fy),
                 C.c_double(cx), C.c_double(cy), C.c_double(near))


def view_counts_points(points, c2w, height: int, width: int, fx: float, fy=None, cx=None, cy=None, near=0.0):
    """Sec. 4.1 Prior 2: the number of pinhole views (camera-to-world [V, 3, 4], OpenGL axes) whose
    image rectangle a world point projects into, in front of the camera beyond ``near``."""
    pts = np.ascontiguousarray(_f64(points).reshape(-1, 3))
    out = np.zeros(pts.shape[0], dtype=np.uint32)
    keep, a = _rig_args(c2w, height, width, fx, fy, cx, cy, near)
    lib().oracle_view_counts_points(C.c_long(pts.shape[0]), _ptr(pts), *a, out.ctypes.data_as(C.POINTER(C.c_uint)))
    return out


def view_counts(shape, c2w, height: int, width: int, fx: float, fy=None, cx=None, cy=None, near=0.0,
                box=((-1.0,) * 3, (1.0,) * 3)):
    """Sec. 4.1 Prior 2 on the align-corners lattice of ``shape`` over ``box``: (counts n_j as a
    uint32 grid, learning-rate scale n_j / n_max, n_max)."""
    n = np.array([int(s) for s in shape], dtype=np.int32)
    counts = np.zeros(tuple(n), dtype=np.uint32)
    scale = np.zeros(tuple(n))
    keep, a = _rig_args(c2w, height, width, fx, fy, cx, cy, near)
    f = lib().oracle_view_counts
    f.restype = C.c_uint
    n_max = f(n.ctypes.data_as(C.POINTER(C.c_int)), _ptr(_f64(box[0])), _ptr(_f64(box[1])), *a,
              counts.ctypes.data_as(C.POINTER(C.c_uint)), _ptr(scale))
    return counts, scale, int(n_max)
