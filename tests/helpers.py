"""Shared test helpers: parameter conversion between the ABI and the oracle, tolerance checks."""
from __future__ import annotations

import numpy as np

import oracle

# Tolerances of the plain FP32 path against the FP64 oracle (per element, with a floor at 1% of
# the largest magnitude because atomically accumulated FP32 sums lose relative accuracy on
# near-zero elements).
RTOL_COLOUR = 1e-5
RTOL_GRAD = 1e-4
FLOOR = 1e-2
# Fine-stage grid gradients with the FP32 MLP: the per-sample colours carry ~1e-6 absolute FP32
# error (eps_c), and dC/dtau_k = sum_{j>=k} T_{j+1}(c_j - c_{j+1}) inherits |delta D_k| <= 2 eps_c
# T_{k+1}; on elements far below the maximum (behind surfaces, in empty space) that term
# dominates.  The per-element check is |g - o| <= 1e-4 max(|o|, FLOOR_FINE_GRAD max|o|), i.e. an
# absolute floor of 5e-6 of the largest magnitude (measured worst cases: 1.5e-6 at 160^3, 2.3e-6
# at 256^3); the norm-relative error must stay below NORM_RTOL_GRAD.
FLOOR_FINE_GRAD = 5e-2
NORM_RTOL_GRAD = 1e-5


def f32(x):
    return float(np.float32(x))


def oracle_params(p, grid_shape, feat_dim, box=((-1.0,) * 3, (1.0,) * 3)):
    """The oracle's parameters for an ABI Params, every value rounded through FP32 exactly as the
    library receives it."""
    return oracle.Params(
        grid_shape=tuple(grid_shape), xyz_min=tuple(f32(v) for v in box[0]), xyz_max=tuple(f32(v) for v in box[1]),
        shift_b=f32(p.shift_b), delta=f32(p.step), tau_f=f32(p.tau_f), t_near=f32(p.t_near), t_far=f32(p.t_far),
        bg=tuple(f32(v) for v in p.bg), mode=p.mode, rgb_act=p.rgb_act, feat_dim=feat_dim, n_freq=p.n_freq_dir,
        hidden=p.hidden, w_pt=f32(p.w_pt_rgb), w_bg=f32(p.w_bg), act_order=p.act_order,
        n_freq_pos=p.n_freq_pos)


def floor_err(got, ref, rtol, floor=FLOOR):
    """max over elements of |got - ref| / (rtol * max(|ref|, floor * max|ref|)); <= 1 passes."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = max(np.abs(ref).max(initial=0.0), 1e-30)
    den = rtol * np.maximum(np.abs(ref), floor * scale)
    return float(np.max(np.abs(got - ref) / den, initial=0.0))


def assert_close(got, ref, rtol, name, floor=FLOOR):
    e = floor_err(got, ref, rtol, floor)
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    rel2 = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-30)
    if e > 1.0:
        g, r = got.reshape(-1), ref.reshape(-1)
        scale = np.abs(r).max()
        den = rtol * np.maximum(np.abs(r), floor * scale)
        i = int(np.argmax(np.abs(g - r) / den))
        raise AssertionError(f"{name}: normalised error {e:.3g} (> 1), relative L2 {rel2:.3g}; worst element "
                             f"{np.unravel_index(i, ref.shape)}: got {g[i]:.9g} ref {r[i]:.9g} "
                             f"(|ref| / max|ref| = {abs(r[i]) / scale:.3g})")
    return e, rel2
