"""Grid sizing and the progressive-scaling schedule of the fine stage (host logic).

Sec. 4.1: for an expected number of voxels M in a box of side lengths L_x, L_y, L_z the voxel size
is s = (L_x L_y L_z / M)^(1/3) and the grid has floor(L_a / s) voxels along axis a.  Sec. 4.2
(progressive scaling): with checkpoint steps pg_ckpt the fine stage starts from
floor(M / 2^|pg_ckpt|) voxels and doubles the voxel count at every checkpoint, reaching M after the
last one; the grids are resized by trilinear interpolation (dvgo_resize_grid) and the voxel size,
hence the sampling step delta = ratio * s, follows.
"""
from __future__ import annotations

import math

# floor(L / s) is taken with this relative slack so that an exact integer ratio (e.g. 2 / (2 / 160))
# is not lost to the rounding of the cube root.
_FLOOR_SLACK = 1e-9


def voxel_grid(n_voxels: float, lengths) -> tuple[tuple[int, int, int], float]:
    """(grid dimensions, voxel size s) for n_voxels voxels in a box with the given side lengths."""
    L = [float(v) for v in lengths]
    if n_voxels < 1 or min(L) <= 0:
        raise ValueError("voxel_grid: need n_voxels >= 1 and positive lengths")
    s = (L[0] * L[1] * L[2] / float(n_voxels)) ** (1.0 / 3.0)
    dims = tuple(max(2, int(math.floor(v / s * (1.0 + _FLOOR_SLACK)))) for v in L)
    return dims, s


def pg_schedule(n_voxels: float, lengths, pg_ckpt) -> list[tuple[int, tuple[int, int, int], float]]:
    """[(first step, grid dimensions, voxel size)] of the fine stage: the initial grid at step 0 and
    one entry per checkpoint (sorted), the voxel count doubling at each."""
    ck = sorted(int(c) for c in pg_ckpt)
    if any(c <= 0 for c in ck) or len(set(ck)) != len(ck):
        raise ValueError("pg_schedule: checkpoints must be distinct positive steps")
    n = len(ck)
    out = []
    for j, start in enumerate([0] + ck):
        dims, s = voxel_grid(math.floor(n_voxels / 2 ** (n - j)), lengths)
        out.append((start, dims, s))
    return out
