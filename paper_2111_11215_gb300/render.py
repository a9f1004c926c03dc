"""Torch-facing helpers over the C ABI: a renderer that owns the workspace, an autograd
Function, the fine-stage model container and its Adam state.  Every step runs in libdvgo."""
from __future__ import annotations

import torch

from . import binding as B

MLP_KEYS = ("w1", "b1", "w2", "b2", "w3", "b3")


def mlp_shapes(in_dim: int, hidden: int):
    return {"w1": (in_dim, hidden), "b1": (hidden,), "w2": (hidden, hidden), "b2": (hidden,),
            "w3": (hidden, 3), "b3": (3,)}


def mlp_flat_size(in_dim: int = 39, hidden: int = 128) -> int:
    return sum(int(torch.tensor(s).prod()) for s in mlp_shapes(in_dim, hidden).values())


def mlp_views(flat: torch.Tensor, in_dim: int = 39, hidden: int = 128) -> dict:
    """Views w1..b3 into one flat buffer laid out w1 | b1 | w2 | b2 | w3 | b3 (the ABI's order)."""
    out, off = {}, 0
    for k, shp in mlp_shapes(in_dim, hidden).items():
        n = int(torch.tensor(shp).prod())
        out[k] = flat[off:off + n].view(shp)
        off += n
    return out


class Renderer:
    """Owns the descriptors and the workspace of one ray-batch size."""

    def __init__(self, params: B.Params, density_desc: B.GridDesc, cgrid_desc: B.GridDesc, n_rays: int,
                 samples_per_ray: int | None = None, device="cuda"):
        self.params, self.dd, self.cd = params, density_desc, cgrid_desc
        self.n_rays = n_rays
        dummy = None
        if samples_per_ray is not None:
            z = torch.empty((max(n_rays, 1), samples_per_ray), device=device)
            dummy = (z, z)
        self.ws_bytes = B.dvgo_workspace_size(params, density_desc, n_rays, dummy)
        self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=device)

    def forward(self, density, cgrid, mlp, rays_o, rays_d, jitter=None, samples=None, target=None,
                rgb=None, tfinal=None, loss=None, dloss=None, stream=None, cgrid_ready=None, density_ready=None):
        """cgrid_ready: an event (torch.cuda.Event) whose completion the colour kernels wait for;
        the kernels before them (ray set-up, sample scan, density pass) do not.  density_ready: the
        same for the density pass (the ray set-up and the sample scan do not wait)."""
        R = rays_o.shape[0]
        dev = rays_o.device
        rgb = torch.empty((R, 3), device=dev) if rgb is None else rgb
        tfinal = torch.empty(R, device=dev) if tfinal is None else tfinal
        if target is not None:
            loss = torch.empty(1, device=dev) if loss is None else loss
        params = self.params
        if cgrid_ready is not None:
            params = params.with_(cgrid_ready=cgrid_ready.cuda_event)
        if density_ready is not None:
            params = params.with_(density_ready=density_ready.cuda_event)
        B.dvgo_render_fwd(params, self.dd, density, self.cd, cgrid, mlp, rays_o, rays_d, jitter, samples,
                          target, rgb, tfinal, loss, dloss, self.workspace, stream)
        return rgb, tfinal, loss

    def backward(self, density, cgrid, mlp, rays_o, rays_d, jitter, samples, grad_rgb, grad_tfinal,
                 grad_density, grad_cgrid, grad_mlp, stream=None):
        B.dvgo_render_bwd(self.params, self.dd, density, self.cd, cgrid, mlp, rays_o, rays_d, jitter, samples,
                          grad_rgb, grad_tfinal, grad_density, grad_cgrid, grad_mlp, self.workspace, stream)


class FrameRenderer:
    """Forward-only rendering of any number of rays (e.g. full frames at test time) in fixed-size
    chunks through one workspace; free-space skipping (tau_f, params.freespace) applies as in
    training (Sec. 4.2: "in both training and testing")."""

    def __init__(self, params: B.Params, density_desc: B.GridDesc, cgrid_desc: B.GridDesc, chunk: int = 65536,
                 device="cuda"):
        self.chunk = int(chunk)
        self.renderer = Renderer(params.with_(forward_only=1), density_desc, cgrid_desc, self.chunk, device=device)

    def render(self, density, cgrid, mlp, rays_o, rays_d, rgb=None, tfinal=None, stream=None):
        R, dev = rays_o.shape[0], rays_o.device
        rgb = torch.empty((R, 3), device=dev) if rgb is None else rgb
        tfinal = torch.empty(R, device=dev) if tfinal is None else tfinal
        for s in range(0, R, self.chunk):
            e = min(R, s + self.chunk)
            self.renderer.forward(density, cgrid, mlp, rays_o[s:e], rays_d[s:e], None, None, None, rgb[s:e],
                                  tfinal[s:e], stream=stream)
        return rgb, tfinal


class RenderFunction(torch.autograd.Function):
    """(density, cgrid, mlp_flat) -> (rgb, T_final) with the library's backward.

    The forward leaves per-sample state in the renderer's workspace; the backward of a call
    must run before the next forward on the same renderer (checked by a generation count)."""

    @staticmethod
    def forward(ctx, renderer: Renderer, density, cgrid, mlp_flat, rays_o, rays_d, jitter, samples_t, samples_dt):
        samples = None if samples_t is None else (samples_t, samples_dt)
        mlp = None
        if renderer.params.mode == B.DVGO_MODE_FINE:
            mlp = mlp_views(mlp_flat, renderer.params.mlp_in_dim(renderer.cd.channels), renderer.params.hidden)
        rgb, tfinal, _ = renderer.forward(density, cgrid, mlp, rays_o, rays_d, jitter, samples)
        renderer._gen = getattr(renderer, "_gen", 0) + 1
        ctx.gen = renderer._gen
        ctx.renderer = renderer
        ctx.mlp = mlp
        ctx.samples = samples
        ctx.cgrid_dtype = cgrid.dtype
        ctx.save_for_backward(density, cgrid, mlp_flat, rays_o, rays_d, jitter)
        return rgb, tfinal

    @staticmethod
    def backward(ctx, grad_rgb, grad_tfinal):
        density, cgrid, mlp_flat, rays_o, rays_d, jitter = ctx.saved_tensors
        r = ctx.renderer
        if r._gen != ctx.gen:
            raise RuntimeError("the renderer's workspace was reused by another forward before this backward")
        g_d = torch.zeros_like(density)
        g_c = torch.zeros(cgrid.shape, dtype=torch.float32, device=cgrid.device)
        g_m = torch.zeros_like(mlp_flat) if mlp_flat is not None else None
        grad_rgb = torch.zeros((rays_o.shape[0], 3), device=rays_o.device) if grad_rgb is None else grad_rgb.contiguous()
        gT = None if grad_tfinal is None else grad_tfinal.contiguous()
        r.backward(density, cgrid, ctx.mlp, rays_o, rays_d, jitter, ctx.samples, grad_rgb, gT, g_d, g_c, g_m)
        return None, g_d, g_c, g_m, None, None, None, None, None


class AdamState:
    """First and second moments of one FP32 parameter tensor."""

    def __init__(self, param: torch.Tensor):
        self.m = torch.zeros_like(param)
        self.v = torch.zeros_like(param)


# Checkpoint / resume.  A state_dict() holds device tensors cloned on the caller's stream (so that
# the snapshot is ordered after every step queued before it) and plain Python scalars; torch.save
# writes it as it is and torch.load(..., map_location=...) reads it back.  The library draws no
# random numbers (jitter and batches come from the caller), so the caller's own RNG state is the
# only other thing a resumed run needs.
STATE_VERSION = 1


def _clone_on(t, stream):
    if t is None:
        return None
    if stream is None:
        return t.detach().clone()
    with torch.cuda.stream(stream):
        return t.detach().clone()


def _copy_on(dst, src, stream):
    if tuple(dst.shape) != tuple(src.shape) or dst.dtype != src.dtype:
        raise ValueError(f"load_state_dict: tensor {tuple(src.shape)} {src.dtype} does not fit "
                         f"{tuple(dst.shape)} {dst.dtype}")
    if stream is None:
        dst.copy_(src)
    else:
        with torch.cuda.stream(stream):
            dst.copy_(src)


def _zero_on(t, stream):
    if stream is None:
        t.zero_()
    else:
        with torch.cuda.stream(stream):
            t.zero_()


def _check_version(sd, what):
    if not isinstance(sd, dict) or sd.get("version") != STATE_VERSION or sd.get("kind") != what:
        raise ValueError(f"load_state_dict: not a {what} state of version {STATE_VERSION}")


class FineModel:
    """Fine-stage parameters (Sec. 4.2): density grid, feature grid (FP32 master, optional BF16
    storage copy written by the Adam step), colour MLP in one flat buffer; their gradients and
    Adam state; and one training step (forward, backward, Adam) on a ray batch.

    overlap_adam: the feature-grid Adam step (HBM-bound, the largest of the three) is deferred to a
    side stream: it is launched by launch_feat_adam (after the backward and after whatever the
    caller queued meanwhile, e.g. the next step's proposal forward, so that it overlaps the work
    queued next that does not read the features), or at the latest by the next read of the
    features through this object (wait_params)."""

    def __init__(self, density: torch.Tensor, feat: torch.Tensor, mlp_flat: torch.Tensor, params: B.Params,
                 n_rays: int, bf16_feat: bool = False, box=((-1.0,) * 3, (1.0,) * 3),
                 lr_grid: float = 0.1, lr_mlp: float = 1e-3, decay_steps: float = 20000.0,
                 overlap_adam: bool = False, layout: int = B.DVGO_LAYOUT_CANONICAL, lazy_grid_adam: bool = False):
        self.params = params
        res = tuple(density.shape)
        C = feat.shape[-1]
        self.layout = layout
        if layout == B.DVGO_LAYOUT_PACKED:
            # the grids (and with them their gradients and Adam state) live in the packed layout
            density = B.dvgo_pack_grid(B.GridDesc(res, 1, box[0], box[1]), density.contiguous(),
                                       B.GridDesc(res, 1, box[0], box[1], layout=layout))
            feat = B.dvgo_pack_grid(B.GridDesc(res, C, box[0], box[1]), feat.contiguous(),
                                    B.GridDesc(res, C, box[0], box[1], layout=layout))
        self.density = density.contiguous()
        self._feat = feat.contiguous()
        self.mlp_flat = mlp_flat.contiguous()
        self.mlp = mlp_views(self.mlp_flat, params.mlp_in_dim(C), params.hidden)
        self.bf16_feat = bf16_feat
        self._feat_bf16 = self._feat.to(torch.bfloat16) if bf16_feat else None
        self.dd = B.GridDesc(res, 1, box[0], box[1], layout=layout)
        self.cd = B.GridDesc(res, C, box[0], box[1], B.DVGO_DTYPE_BF16 if bf16_feat else B.DVGO_DTYPE_F32, layout=layout)
        self.renderer = Renderer(params, self.dd, self.cd, n_rays, device=density.device)
        self.g_density = torch.zeros_like(self.density)
        self.g_feat = torch.zeros_like(self._feat)
        self.g_mlp = torch.zeros_like(self.mlp_flat)
        self.adam = {k: AdamState(t) for k, t in (("density", self.density), ("feat", self._feat), ("mlp", self.mlp_flat))}
        self.lr_grid, self.lr_mlp, self.decay_steps = lr_grid, lr_mlp, decay_steps
        self.lazy_grid_adam = lazy_grid_adam   # grids' Adam skips elements with a zero gradient
        dev = density.device
        self.rgb = torch.empty((n_rays, 3), device=dev)
        self.tfinal = torch.empty(n_rays, device=dev)
        self.loss = torch.zeros(1, device=dev)
        self.dloss = torch.empty((n_rays, 3), device=dev)
        self.step_count = 0
        self.grid_t0 = 0               # step count at the last rescale: the grids' Adam restarts there
        self._side = torch.cuda.Stream(device=dev) if overlap_adam else None
        self._ev_bwd = torch.cuda.Event() if overlap_adam else None
        self._ev_after = torch.cuda.Event() if overlap_adam else None
        self._ev_feat = torch.cuda.Event() if overlap_adam else None
        self._feat_pending = False     # an Adam step was launched on the side stream
        self._feat_deferred = None     # (lr, t) of an Adam step not launched yet

    @property
    def feat(self):
        """FP32 feature grid (master copy), ordered after any pending Adam step on the current stream."""
        self.wait_params()
        return self._feat

    @property
    def feat_bf16(self):
        """BF16 storage copy of the feature grid (None without bf16_feat), ordered like feat."""
        self.wait_params()
        return self._feat_bf16

    @property
    def cgrid(self):
        """The feature grid the renderer reads (BF16 copy or FP32), ordered like feat."""
        self.wait_params()
        return self._feat_bf16 if self.bf16_feat else self._feat

    def _cur(self, stream):
        return stream if stream is not None else torch.cuda.current_stream(self.density.device)

    def launch_feat_adam(self, stream=None):
        """Launch a deferred feature-grid Adam step on the side stream, ordered after the backward
        and after everything queued on `stream` so far."""
        if self._feat_deferred is None:
            return
        lr_g, t = self._feat_deferred
        self._feat_deferred = None
        self._ev_after.record(self._cur(stream))
        self._side.wait_event(self._ev_bwd)
        self._side.wait_event(self._ev_after)
        B.dvgo_adam_step(self._feat, self.g_feat, self.adam["feat"].m, self.adam["feat"].v, lr_g, t,
                         param_bf16_out=self._feat_bf16, stream=self._side, skip_zero_grad=self.lazy_grid_adam)
        self._ev_feat.record(self._side)
        self._feat_pending = True

    def wait_params(self, stream=None):
        """Order `stream` (default: the current stream) after the feature-grid Adam step (launching
        it first if it is still deferred)."""
        self.launch_feat_adam(stream)
        if self._feat_pending:
            self._cur(stream).wait_event(self._ev_feat)

    @property
    def shape(self):
        return tuple(self.dd.shape)

    def rescale(self, shape, step: float, stream=None, adam: str = "reset"):
        """Progressive scaling (Sec. 4.2): resize the density and feature grids to `shape` lattice
        points on the same box by trilinear interpolation (dvgo_resize_grid) and render with the
        sampling step `step` from now on (the step follows the voxel size).  The shift b stays, so
        the activated density field is unchanged.  The grids' Adam state: adam="reset" restarts the
        moments from zero with their bias-correction count; adam="resize" resizes both moments with
        the grids (trilinear, so the second moment stays >= 0) and keeps the count.  The
        learning-rate decay and the MLP's Adam state continue either way."""
        if adam not in ("reset", "resize"):
            raise ValueError("rescale: adam must be 'reset' or 'resize'")
        self.wait_params(stream)
        shape = tuple(int(v) for v in shape)
        C = self.cd.channels
        dd = self.dd.with_(shape=shape)
        cd32 = self.cd.with_(shape=shape, dtype=B.DVGO_DTYPE_F32)
        cd32_old = self.cd.with_(dtype=B.DVGO_DTYPE_F32)

        def grid_shape(t, channels):
            if self.layout != B.DVGO_LAYOUT_CANONICAL:
                return t
            return t.view(shape + ((channels,) if channels > 1 else ()))
        moments = None
        if adam == "resize":
            moments = {"density": [grid_shape(B.dvgo_resize_grid(self.dd, x.reshape(-1), dd, stream=stream), 1)
                                   for x in (self.adam["density"].m, self.adam["density"].v)],
                       "feat": [grid_shape(B.dvgo_resize_grid(cd32_old, x.reshape(-1), cd32, stream=stream), C)
                                for x in (self.adam["feat"].m, self.adam["feat"].v)]}
        self.density = grid_shape(B.dvgo_resize_grid(self.dd, self.density.reshape(-1), dd, stream=stream), 1)
        self._feat = grid_shape(B.dvgo_resize_grid(cd32_old, self._feat.reshape(-1), cd32, stream=stream), C)
        if self.bf16_feat:
            self._feat_bf16 = B.dvgo_pack_grid(cd32, self._feat.reshape(-1), cd32.with_(dtype=B.DVGO_DTYPE_BF16),
                                               stream=stream).view(self._feat.shape)
        self.dd, self.cd = dd, self.cd.with_(shape=shape)
        self.params = self.params.with_(step=float(step))
        self.renderer = Renderer(self.params, self.dd, self.cd, self.renderer.n_rays, device=self.density.device)
        self._expl = None
        self.g_density = torch.zeros_like(self.density)
        self.g_feat = torch.zeros_like(self._feat)
        self.adam["density"], self.adam["feat"] = AdamState(self.density), AdamState(self._feat)
        if moments is None:
            self.grid_t0 = self.step_count
        else:
            for k, (m, v) in moments.items():
                self.adam[k].m, self.adam[k].v = m, v

    def state_dict(self, stream=None) -> dict:
        """Snapshot for checkpoint / resume: the density grid, the feature grid (FP32 master and the
        BF16 copy), the MLP, the Adam moments of all three, the step counts and the lattice (shape
        and sampling step, which progressive scaling changes).  Taken on `stream` (default:
        current) after any pending feature-grid Adam step.  Gradients are not part of it: every
        Adam step leaves them zero."""
        self.wait_params(stream)
        c = lambda t: _clone_on(t, stream)  # noqa: E731
        return {"kind": "FineModel", "version": STATE_VERSION, "shape": self.shape, "channels": self.cd.channels,
                "layout": self.layout, "bf16_feat": self.bf16_feat, "step": float(self.params.step),
                "density": c(self.density), "feat": c(self._feat), "feat_bf16": c(self._feat_bf16),
                "mlp": c(self.mlp_flat), "adam": {k: {"m": c(a.m), "v": c(a.v)} for k, a in self.adam.items()},
                "step_count": self.step_count, "grid_t0": self.grid_t0}

    def load_state_dict(self, sd: dict, stream=None):
        """Restore a state_dict() snapshot (tensors on any device) on `stream` (default: current).
        The model must have the snapshot's grid layout, channel count, MLP size and BF16 setting; a
        snapshot on another lattice (taken after progressive scaling) replaces the grids and the
        renderer with ones of its shape and sampling step.  Gradients are cleared."""
        _check_version(sd, "FineModel")
        if (sd["layout"] != self.layout or sd["channels"] != self.cd.channels
                or bool(sd["bf16_feat"]) != self.bf16_feat or sd["mlp"].numel() != self.mlp_flat.numel()):
            raise ValueError("load_state_dict: the snapshot's layout, channels, MLP size or BF16 setting differ")
        self.wait_params(stream)
        self._feat_deferred = None
        dev = self.density.device
        shape = tuple(int(v) for v in sd["shape"])
        if shape != self.shape or tuple(sd["density"].shape) != tuple(self.density.shape):
            self.dd, self.cd = self.dd.with_(shape=shape), self.cd.with_(shape=shape)
            self.density = torch.empty(sd["density"].shape, device=dev)
            self._feat = torch.empty(sd["feat"].shape, device=dev)
            if self.bf16_feat:
                self._feat_bf16 = torch.empty(sd["feat_bf16"].shape, dtype=torch.bfloat16, device=dev)
            self.g_density = torch.zeros_like(self.density)
            self.g_feat = torch.zeros_like(self._feat)
            self.adam["density"], self.adam["feat"] = AdamState(self.density), AdamState(self._feat)
        if shape != tuple(self.renderer.dd.shape) or float(sd["step"]) != float(self.params.step):
            self.params = self.params.with_(step=float(sd["step"]))
            self.renderer = Renderer(self.params, self.dd, self.cd, self.renderer.n_rays, device=dev)
            self._expl = None
        _copy_on(self.density, sd["density"], stream)
        _copy_on(self._feat, sd["feat"], stream)
        if self.bf16_feat:
            _copy_on(self._feat_bf16, sd["feat_bf16"], stream)
        _copy_on(self.mlp_flat, sd["mlp"], stream)
        for k, a in self.adam.items():
            _copy_on(a.m, sd["adam"][k]["m"], stream)
            _copy_on(a.v, sd["adam"][k]["v"], stream)
        for g in (self.g_density, self.g_feat, self.g_mlp):
            _zero_on(g, stream)
        self.step_count, self.grid_t0 = int(sd["step_count"]), int(sd["grid_t0"])

    def forward(self, rays_o, rays_d, jitter=None, target=None, stream=None):
        self.wait_params(stream)
        return self.renderer.forward(self.density, self.cgrid, self.mlp, rays_o, rays_d, jitter, None, target,
                                     self.rgb, self.tfinal, self.loss if target is not None else None,
                                     self.dloss if target is not None else None, stream)

    def explicit_renderer(self, n_per_ray: int) -> Renderer:
        """Renderer (and workspace) for explicit samples of n_per_ray per ray."""
        r = getattr(self, "_expl", None)
        if r is None or r[0] != n_per_ray:
            rend = Renderer(self.params, self.dd, self.cd, self.renderer.n_rays, samples_per_ray=n_per_ray,
                            device=self.density.device)
            self._expl = (n_per_ray, rend)
        return self._expl[1]

    def train_step(self, rays_o, rays_d, jitter, target, stream=None, samples=None, after_forward=None):
        """One optimisation step: render + MSE (Eq. photo_loss), backward, Adam on every parameter.
        `samples` = (t, dt) [R, n] renders with explicit samples (e.g. from a Proposal) instead of
        uniform steps.  `after_forward(renderer)` (optional) is called between the forward and the
        backward, while the renderer's workspace holds this batch's forward samples."""
        rend = self.renderer if samples is None else self.explicit_renderer(samples[0].shape[1])
        # a pending feature-grid Adam step holds back only the colour kernels of the forward (the
        # stream waits on its event inside the call); the backward follows on the same stream
        self.launch_feat_adam(stream)
        ready = self._ev_feat if self._feat_pending else None
        rend.forward(self.density, self._feat_bf16 if self.bf16_feat else self._feat, self.mlp, rays_o, rays_d,
                     jitter, samples, target, self.rgb, self.tfinal, self.loss, self.dloss, stream,
                     cgrid_ready=ready)
        if after_forward is not None:
            after_forward(rend)
        rend.backward(self.density, self._feat_bf16 if self.bf16_feat else self._feat, self.mlp, rays_o, rays_d,
                      jitter, samples, self.dloss, None, self.g_density, self.g_feat, self.g_mlp, stream)
        self.step_count += 1
        t = self.step_count
        tg = t - self.grid_t0          # the grids' Adam count (restarted by rescale)
        lr_g = B.dvgo_lr_at(self.lr_grid, t - 1, self.decay_steps)
        lr_m = B.dvgo_lr_at(self.lr_mlp, t - 1, self.decay_steps)
        if self._side is not None:
            self._ev_bwd.record(self._cur(stream))
            self._feat_deferred = (lr_g, tg)
        else:
            B.dvgo_adam_step(self._feat, self.g_feat, self.adam["feat"].m, self.adam["feat"].v, lr_g, tg,
                             param_bf16_out=self._feat_bf16, stream=stream, skip_zero_grad=self.lazy_grid_adam)
        B.dvgo_adam_step(self.density, self.g_density, self.adam["density"].m, self.adam["density"].v, lr_g, tg,
                         stream=stream, skip_zero_grad=self.lazy_grid_adam)
        B.dvgo_adam_step(self.mlp_flat, self.g_mlp, self.adam["mlp"].m, self.adam["mlp"].v, lr_m, t, stream=stream)
        return self.loss


class CoarseModel:
    """Coarse-stage parameters (Sec. 4.1): density grid and view-invariant colour grid, their
    gradients and Adam state, and one training step (forward, backward, Adam) on a ray batch."""

    def __init__(self, density: torch.Tensor, rgb: torch.Tensor, params: B.Params, n_rays: int,
                 box=((-1.0,) * 3, (1.0,) * 3), lr_grid: float = 0.1, decay_steps: float = 20000.0):
        self.params = params
        res = tuple(density.shape)
        self.density, self.rgb_grid = density.contiguous(), rgb.contiguous()
        self.dd = B.GridDesc(res, 1, box[0], box[1])
        self.cd = B.GridDesc(res, 3, box[0], box[1])
        self.renderer = Renderer(params, self.dd, self.cd, n_rays, device=density.device)
        self.g_density = torch.zeros_like(self.density)
        self.g_rgb = torch.zeros_like(self.rgb_grid)
        self.adam = {"density": AdamState(self.density), "rgb": AdamState(self.rgb_grid)}
        self.lr_grid, self.decay_steps = lr_grid, decay_steps
        dev = density.device
        self.rgb = torch.empty((n_rays, 3), device=dev)
        self.tfinal = torch.empty(n_rays, device=dev)
        self.loss = torch.zeros(1, device=dev)
        self.dloss = torch.empty((n_rays, 3), device=dev)
        self.step_count = 0
        self.view_counts = None     # Prior 2: per-point view counts n_j (int32 view of the uint32 grid)
        self.lr_scale = None        # Prior 2: per-point density learning-rate scale n_j / n_max

    def set_view_counts(self, c2w: torch.Tensor, height: int, width: int, fx: float, fy=None, cx=None, cy=None,
                        near: float = 0.0, stream=None) -> int:
        """Sec. 4.1 Prior 2: scale each density point's learning rate by n_j / n_max, n_j the number
        of training views (camera-to-world CUDA float64 [V, 3, 4]) that see it.  Returns n_max."""
        counts, scale, n_max = B.dvgo_view_counts(self.dd, c2w, height, width, fx, fy, cx, cy, near, stream=stream)
        self.view_counts, self.lr_scale = counts.view(self.density.shape), scale.view(self.density.shape)
        return int(n_max.item())

    def state_dict(self, stream=None) -> dict:
        """Snapshot for checkpoint / resume: both grids, their Adam moments, the step count and the
        Prior-2 view counts and learning-rate scale when set; taken on `stream` (default: current).
        Gradients are not part of it: every Adam step leaves them zero."""
        c = lambda t: _clone_on(t, stream)  # noqa: E731
        return {"kind": "CoarseModel", "version": STATE_VERSION, "shape": tuple(self.dd.shape),
                "density": c(self.density), "rgb": c(self.rgb_grid),
                "adam": {k: {"m": c(a.m), "v": c(a.v)} for k, a in self.adam.items()},
                "step_count": self.step_count, "view_counts": c(self.view_counts), "lr_scale": c(self.lr_scale)}

    def load_state_dict(self, sd: dict, stream=None):
        """Restore a state_dict() snapshot of a model of the same grid shape on `stream` (default:
        current); gradients are cleared."""
        _check_version(sd, "CoarseModel")
        if tuple(sd["shape"]) != tuple(self.dd.shape):
            raise ValueError("load_state_dict: the snapshot's grid shape differs")
        _copy_on(self.density, sd["density"], stream)
        _copy_on(self.rgb_grid, sd["rgb"], stream)
        for k, a in self.adam.items():
            _copy_on(a.m, sd["adam"][k]["m"], stream)
            _copy_on(a.v, sd["adam"][k]["v"], stream)
        for g in (self.g_density, self.g_rgb):
            _zero_on(g, stream)
        dev = self.density.device
        self.view_counts = None if sd["view_counts"] is None else _clone_on(sd["view_counts"].to(dev), stream)
        self.lr_scale = None if sd["lr_scale"] is None else _clone_on(sd["lr_scale"].to(dev), stream)
        self.step_count = int(sd["step_count"])

    def forward(self, rays_o, rays_d, jitter=None, stream=None):
        return self.renderer.forward(self.density, self.rgb_grid, None, rays_o, rays_d, jitter, None, None,
                                     self.rgb, self.tfinal, None, None, stream)

    def train_step(self, rays_o, rays_d, jitter, target, stream=None):
        self.renderer.forward(self.density, self.rgb_grid, None, rays_o, rays_d, jitter, None, target, self.rgb,
                              self.tfinal, self.loss, self.dloss, stream)
        self.renderer.backward(self.density, self.rgb_grid, None, rays_o, rays_d, jitter, None, self.dloss, None,
                               self.g_density, self.g_rgb, None, stream)
        self.step_count += 1
        t = self.step_count
        lr = B.dvgo_lr_at(self.lr_grid, t - 1, self.decay_steps)
        B.dvgo_adam_step(self.density, self.g_density, self.adam["density"].m, self.adam["density"].v, lr, t,
                         lr_scale=self.lr_scale, stream=stream)
        B.dvgo_adam_step(self.rgb_grid, self.g_rgb, self.adam["rgb"].m, self.adam["rgb"].v, lr, t, stream=stream)
        return self.loss


class Proposal:
    """Learned sample proposal (the library's addition; the paper samples uniformly): an MLP on
    the encoded bin centres gives a 64-bin PDF per ray, trained with cross-entropy against the
    binned compositing weights of a uniform render and sampled by inverse CDF."""

    N_BINS, N_FREQ, WIDTH = 64, 6, 64

    def __init__(self, weights: dict, params: B.Params, density_desc: B.GridDesc, n_rays: int, lr: float = 5e-3,
                 device="cuda", sample_precision: int = B.DVGO_MLP_FP32, decay_steps: float = 5000.0,
                 train_precision: int = B.DVGO_MLP_FP32):
        self.params, self.dd = params, density_desc
        self.sample_precision, self.train_precision = sample_precision, train_precision
        shapes = {"w0": (3 + 6 * self.N_FREQ, self.WIDTH), "b0": (self.WIDTH,), "w1": (self.WIDTH, self.WIDTH),
                  "b1": (self.WIDTH,), "w2": (self.WIDTH, self.WIDTH), "b2": (self.WIDTH,), "w3": (self.WIDTH, 1),
                  "b3": (1,)}
        n = sum(int(torch.tensor(v).prod()) for v in shapes.values())
        self.flat = torch.empty(n, dtype=torch.float32, device=device)
        self.w, off = {}, 0
        for k, shp in shapes.items():
            m = int(torch.tensor(shp).prod())
            self.w[k] = self.flat[off:off + m].view(shp)
            self.w[k].copy_(torch.as_tensor(weights[k]).reshape(shp))
            off += m
        self.grad = torch.zeros_like(self.flat)
        self.adam = AdamState(self.flat)
        self.lr, self.decay_steps, self.step_count = lr, decay_steps, 0
        self.labels = torch.empty((n_rays, self.N_BINS), device=device)
        self.probs = torch.empty((n_rays, self.N_BINS), device=device)
        self.loss = torch.zeros(1, device=device)

    def train_step(self, uniform_workspace, rays_o, rays_d, stream=None, n_train=None, with_loss=True):
        """Labels from the workspace of a uniform fine forward on these rays, then one Adam step
        on the cross-entropy loss of the first n_train rays (all by default), at the rate lr decayed
        by 0.1 over decay_steps proposal steps; returns the loss (device tensor, before the step)
        when with_loss."""
        R = rays_o.shape[0]
        n = R if n_train is None else min(int(n_train), R)
        B.dvgo_weight_bins(self.params, self.dd, R, self.N_BINS, uniform_workspace, self.labels[:R], stream)
        if with_loss:
            B.dvgo_proposal_fwd(self.params, self.dd, self.N_BINS, self.N_FREQ, self.WIDTH, self.w, rays_o[:n],
                                rays_d[:n], self.labels[:n], self.probs[:n], self.loss, stream)
        B.dvgo_proposal_bwd(self.params, self.dd, self.N_BINS, self.N_FREQ, self.WIDTH, self.w, rays_o[:n],
                            rays_d[:n], self.labels[:n], self.grad, stream, precision=self.train_precision)
        self.step_count += 1
        lr = B.dvgo_lr_at(self.lr, self.step_count - 1, self.decay_steps)
        B.dvgo_adam_step(self.flat, self.grad, self.adam.m, self.adam.v, lr, self.step_count, stream=stream)
        return self.loss

    def state_dict(self, stream=None) -> dict:
        """Snapshot for checkpoint / resume: the network's weights, their Adam moments, the step count
        and the learning-rate schedule; taken on `stream` (default: current)."""
        c = lambda t: _clone_on(t, stream)  # noqa: E731
        return {"kind": "Proposal", "version": STATE_VERSION, "flat": c(self.flat), "m": c(self.adam.m),
                "v": c(self.adam.v), "step_count": self.step_count, "lr": self.lr, "decay_steps": self.decay_steps}

    def load_state_dict(self, sd: dict, stream=None):
        """Restore a state_dict() snapshot on `stream` (default: current); the gradient is cleared."""
        _check_version(sd, "Proposal")
        _copy_on(self.flat, sd["flat"], stream)
        _copy_on(self.adam.m, sd["m"], stream)
        _copy_on(self.adam.v, sd["v"], stream)
        _zero_on(self.grad, stream)
        self.step_count, self.lr, self.decay_steps = int(sd["step_count"]), float(sd["lr"]), float(sd["decay_steps"])

    def sample(self, rays_o, rays_d, jitter=None, n_samples: int = 48, eta: float = 0.05, t_out=None, dt_out=None,
               stream=None, after_forward=None):
        """Explicit samples (t, dt) [R, n_samples] drawn from the predicted PDFs mixed with the
        uniform PDF at weight eta (0.05 keeps ~2 of 48 samples spread along the whole ray).
        after_forward() (optional) is called between the proposal forward and the sampling."""
        R = rays_o.shape[0]
        t_out = torch.empty((R, n_samples), device=rays_o.device) if t_out is None else t_out
        dt_out = torch.empty((R, n_samples), device=rays_o.device) if dt_out is None else dt_out
        B.dvgo_proposal_fwd(self.params, self.dd, self.N_BINS, self.N_FREQ, self.WIDTH, self.w, rays_o, rays_d,
                            None, self.probs[:R], None, stream, precision=self.sample_precision)
        if after_forward is not None:
            after_forward()
        B.dvgo_sample_pdf(self.params, self.dd, rays_o, rays_d, self.probs[:R], n_samples, jitter, eta, t_out, dt_out,
                          stream)
        return t_out, dt_out


class ProposalTrainer:
    """Fine-stage training with the learned proposal (the library's chosen form).  Most steps
    render and back-propagate only the proposal's n_samples importance samples per ray.  The
    first `warmup` steps and then every `uniform_every`-th step are full uniform steps (Sec. 4.2
    sampling): their forward also labels the proposal's training rays, and their backward gives
    every voxel along the batch's rays a gradient, including small structures the proposal's
    smooth field cannot resolve, so they are not left untouched."""

    def __init__(self, model: FineModel, proposal: "Proposal", n_samples: int = 48, uniform_every: int = 4,
                 warmup: int = 0, train_rays: int = 1024, eta: float = 0.05):
        if uniform_every < 1 or n_samples < 1:
            raise ValueError("uniform_every and n_samples must be >= 1")
        self.model, self.proposal = model, proposal
        self.n_samples, self.uniform_every, self.warmup = int(n_samples), int(uniform_every), int(warmup)
        self.train_rays, self.eta = int(train_rays), float(eta)
        R, dev = model.renderer.n_rays, model.density.device
        self.t_buf = torch.empty((R, self.n_samples), device=dev)
        self.dt_buf = torch.empty((R, self.n_samples), device=dev)
        self.i = 0
        self.n_uniform = self.n_proposal = 0
        # with the model's overlapped Adam, the proposal's training step of a uniform step runs on a
        # stream of its own beside the backward (it reads only the forward's samples)
        overlap = getattr(model, "_side", None) is not None
        self._side = torch.cuda.Stream(device=dev) if overlap else None
        self._ev_fwd = torch.cuda.Event() if overlap else None
        self._ev_prop = torch.cuda.Event() if overlap else None

    def rescale(self, shape, step: float, stream=None, adam: str = "reset"):
        """Progressive scaling of the model (FineModel.rescale); the proposal renders and labels on
        the new lattice and step from then on."""
        self.model.rescale(shape, step, stream, adam)
        self.proposal.params, self.proposal.dd = self.model.params, self.model.dd

    def state_dict(self, stream=None) -> dict:
        """Snapshot for checkpoint / resume: the model's and the proposal's states and the schedule's
        position (which step comes next, uniform or proposal); taken on `stream` (default: current),
        which the proposal's own training stream has already been joined to."""
        return {"kind": "ProposalTrainer", "version": STATE_VERSION, "model": self.model.state_dict(stream),
                "proposal": self.proposal.state_dict(stream), "i": self.i, "n_uniform": self.n_uniform,
                "n_proposal": self.n_proposal}

    def load_state_dict(self, sd: dict, stream=None):
        """Restore a state_dict() snapshot into this trainer's model and proposal on `stream`."""
        _check_version(sd, "ProposalTrainer")
        self.model.load_state_dict(sd["model"], stream)
        self.proposal.load_state_dict(sd["proposal"], stream)
        self.proposal.params, self.proposal.dd = self.model.params, self.model.dd
        self.i, self.n_uniform, self.n_proposal = int(sd["i"]), int(sd["n_uniform"]), int(sd["n_proposal"])

    def is_uniform(self, i: int) -> bool:
        return i < self.warmup or i % self.uniform_every == 0

    def step(self, rays_o, rays_d, jitter, target, stream=None):
        """One step; returns the model's loss (device tensor)."""
        if self.is_uniform(self.i):
            cur = stream if stream is not None else torch.cuda.current_stream(rays_o.device)

            def label(rend):
                if self._side is None:
                    self.proposal.train_step(rend.workspace, rays_o, rays_d, stream=stream, n_train=self.train_rays,
                                             with_loss=False)
                    return
                self._ev_fwd.record(cur)
                self._side.wait_event(self._ev_fwd)
                self.proposal.train_step(rend.workspace, rays_o, rays_d, stream=self._side, n_train=self.train_rays,
                                         with_loss=False)
                self._ev_prop.record(self._side)
            loss = self.model.train_step(rays_o, rays_d, jitter, target, stream, after_forward=label)
            if self._side is not None:
                # the backward was queued before this wait, so it overlaps the proposal's step; all
                # later work on the stream (the next sampling, the batch's buffers) is ordered after it
                cur.wait_event(self._ev_prop)
            self.n_uniform += 1
        else:
            R = rays_o.shape[0]
            # the previous step's feature-grid Adam (when deferred) overlaps the sampling
            ts, dts = self.proposal.sample(rays_o, rays_d, jitter, self.n_samples, eta=self.eta,
                                           t_out=self.t_buf[:R], dt_out=self.dt_buf[:R], stream=stream,
                                           after_forward=lambda: self.model.launch_feat_adam(stream))
            loss = self.model.train_step(rays_o, rays_d, jitter, target, stream, samples=(ts, dts))
            self.n_proposal += 1
        self.i += 1
        return loss


class BatchStager:
    """Double-buffered host-to-device staging of training batches: the next batch's copy from pinned
    host tensors runs on a copy stream of its own while the current step computes.

        st = BatchStager(example_device_batch)
        st.stage(host_batch_0)
        for k in range(n):
            batch = st.take()                 # device tensors of batch k (the stream waits for its copy)
            if k + 1 < n:
                st.stage(host_batch_k_plus_1)  # copies into the other buffer set
            loss = trainer.step(*batch)
            st.done()                         # batch k's buffers are free once the step's work is done

    A buffer set is refilled only after the stream has passed the done() of the step that used it;
    staging into a set whose batch was taken but not marked done() raises, as does staging a third
    batch before one is taken.  The copy reads the host tensors asynchronously: a host batch must
    not be written again until its batch has been taken and the taking stream has passed that
    point (e.g. at the next done() that is synchronised on)."""

    def __init__(self, like, device=None):
        dev = like[0].device if device is None else device
        self.bufs = [tuple(torch.empty_like(x) for x in like) for _ in range(2)]
        self.copy_stream = torch.cuda.Stream(device=dev)
        self.ev_copied = [torch.cuda.Event(), torch.cuda.Event()]
        self.ev_used = [torch.cuda.Event(), torch.cuda.Event()]
        # batches j < n_staged were staged into set j % 2, j < n_taken taken, j < n_done done
        self.n_staged = self.n_taken = self.n_done = 0

    def stage(self, host_batch):
        """Queue the copy of host_batch (pinned CPU tensors shaped like the example batch)."""
        k = self.n_staged % 2
        if self.n_staged - self.n_taken >= 2:
            raise RuntimeError("BatchStager: both buffer sets hold batches not taken yet")
        if self.n_staged >= 2:
            # set k last held batch n_staged - 2: its step must have been marked done
            if self.n_done < self.n_staged - 1:
                raise RuntimeError("BatchStager: the batch in this buffer set was taken but not marked done()")
            self.copy_stream.wait_event(self.ev_used[k])
        with torch.cuda.stream(self.copy_stream):
            for dst, src in zip(self.bufs[k], host_batch):
                dst.copy_(src, non_blocking=True)
        self.ev_copied[k].record(self.copy_stream)
        self.n_staged += 1

    def take(self, stream=None):
        """The device tensors of the oldest staged batch; `stream` (default: current) waits for its copy."""
        if self.n_taken >= self.n_staged:
            raise RuntimeError("BatchStager: no staged batch to take")
        k = self.n_taken % 2
        cur = stream if stream is not None else torch.cuda.current_stream(self.bufs[k][0].device)
        cur.wait_event(self.ev_copied[k])
        self.n_taken += 1
        return self.bufs[k]

    def done(self, stream=None):
        """The step that used the oldest taken batch not yet marked done has been queued on `stream`
        (default: current)."""
        if self.n_done >= self.n_taken:
            raise RuntimeError("BatchStager: no taken batch to mark done")
        k = self.n_done % 2
        cur = stream if stream is not None else torch.cuda.current_stream(self.bufs[k][0].device)
        self.ev_used[k].record(cur)
        self.n_done += 1
