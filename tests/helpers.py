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
NORM_RTOL_GRAD = 1e-5

# Fine-stage gradients: besides the relative tolerance above, each element gets the oracle's running
# error bound (og_bound in oracle/dvgo_oracle.c) for the arithmetic of the path under test -- how far
# finite precision can move it from the exact value: (u_op, u_acc) = relative rounding of the MLP
# operands and unit roundoff of the accumulation.  It carries, among the rest, the FP32 error of the
# MLP colours into the density gradient dC/dtau_k = T_{k+1} c_k - S_k, whose colour differences
# cancel on elements behind surfaces and in empty space.
U_FP32 = 2.0 ** -24
U_BF16 = 2.0 ** -8
BOUND_FP32 = (0.0, U_FP32)             # FP32 SIMT MLP: operands as they are, FP32 arithmetic
# BF16 tensor-core MLP against the exact oracle: BF16 operands on the kernel's side only (a worst
# case summed over samples: valid but loose at large sample counts)
BOUND_BF16 = (U_BF16, 2.0 * U_FP32)
# BF16 tensor-core MLP against the oracle in BF16-operand arithmetic (oracle_params(...,
# bf16_operands=True)): both sides round the same operands, so they differ by the FP32 accumulation
# (taken at 2^-23 for the tensor cores' accumulation) and where that moves a value across a BF16
# rounding midpoint
BOUND_BF16_OPERANDS = (0.0, 2.0 * U_FP32)
MLP_KEYS = ("w1", "b1", "w2", "b2", "w3", "b3")


def mlp_flat(d):
    """w1 | b1 | w2 | b2 | w3 | b3 of a dict of per-block arrays, flattened (the ABI's order)."""
    return np.concatenate([np.asarray(d[k]).reshape(-1) for k in MLP_KEYS])


def f32(x):
    return float(np.float32(x))


def oracle_params(p, grid_shape, feat_dim, box=((-1.0,) * 3, (1.0,) * 3), bf16_operands=False):
    """The oracle's parameters for an ABI Params, every value rounded through FP32 exactly as the
    library receives it; bf16_operands: the MLP contractions in BF16-operand arithmetic."""
    return oracle.Params(
        grid_shape=tuple(grid_shape), xyz_min=tuple(f32(v) for v in box[0]), xyz_max=tuple(f32(v) for v in box[1]),
        shift_b=f32(p.shift_b), delta=f32(p.step), tau_f=f32(p.tau_f), t_near=f32(p.t_near), t_far=f32(p.t_far),
        bg=tuple(f32(v) for v in p.bg), mode=p.mode, rgb_act=p.rgb_act, feat_dim=feat_dim, n_freq=p.n_freq_dir,
        hidden=p.hidden, w_pt=f32(p.w_pt_rgb), w_bg=f32(p.w_bg), act_order=p.act_order,
        n_freq_pos=p.n_freq_pos, mlp_operands=1 if bf16_operands else 0)


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


def assert_within_bound(got, ref, bound, name, rtol=RTOL_GRAD, floor=FLOOR):
    """Per element |got - ref| <= rtol * max(|ref|, floor * max|ref|) + bound, where bound is the
    oracle's running error bound of the element; returns (worst normalised error, relative L2)."""
    got = np.asarray(got, dtype=np.float64).reshape(-1)
    ref = np.asarray(ref, dtype=np.float64).reshape(-1)
    bound = np.asarray(bound, dtype=np.float64).reshape(-1)
    scale = max(np.abs(ref).max(initial=0.0), 1e-30)
    tol = rtol * np.maximum(np.abs(ref), floor * scale) + bound
    err = np.abs(got - ref) / np.maximum(tol, 1e-300)
    worst = float(err.max(initial=0.0))
    rel2 = float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-30))
    if worst > 1.0:
        i = int(np.argmax(err))
        raise AssertionError(f"{name}: normalised error {worst:.3g} (> 1), relative L2 {rel2:.3g}; worst element {i}: "
                             f"got {got[i]:.9g} ref {ref[i]:.9g} (|ref| / max|ref| = {abs(ref[i]) / scale:.3g}), "
                             f"bound {bound[i]:.3g}, relative part {rtol * max(abs(ref[i]), floor * scale):.3g}")
    return worst, rel2
