"""Host logic of progressive scaling (Sec. 4.2) and of grid sizing (Sec. 4.1): the schedule of voxel
counts and grid dimensions.  Expected values are worked by hand from the two formulas: M voxels in
a box of sides L give s = (L_x L_y L_z / M)^(1/3) and floor(L_a / s) voxels per axis; the fine stage
starts from floor(M / 2^|pg_ckpt|) voxels and doubles at each checkpoint."""
import math

import pytest

from paper_2111_11215_gb300.progressive import pg_schedule, voxel_grid


def test_fine_stage_schedule_of_the_paper():
    """M = 160^3 on a 2-unit cube with pg_ckpt = {1000, 2000, 3000} (Supp. A):
    512000 voxels -> s = 1/40 -> 80; 1024000 -> s = 128000^(-1/3) = 0.019843 -> 2/s = 100.79 -> 100;
    2048000 -> s = 256000^(-1/3) = 0.015749 -> 126.99 -> 126; 4096000 -> s = 1/80 -> 160."""
    sched = pg_schedule(160 ** 3, (2.0, 2.0, 2.0), [3000, 1000, 2000])
    assert [a for a, _, _ in sched] == [0, 1000, 2000, 3000]
    assert [g for _, g, _ in sched] == [(80,) * 3, (100,) * 3, (126,) * 3, (160,) * 3]
    assert sched[0][2] == pytest.approx(0.025, rel=1e-12)
    assert sched[1][2] == pytest.approx(128000 ** (-1 / 3), rel=1e-12)
    assert sched[3][2] == pytest.approx(0.0125, rel=1e-12)


def test_voxel_grid_of_a_box():
    """M = 100^3 in a 2 x 1 x 0.5 box: s = (1 / 10^6)^(1/3) = 0.01 -> 200 x 100 x 50 voxels."""
    dims, s = voxel_grid(100 ** 3, (2.0, 1.0, 0.5))
    assert dims == (200, 100, 50) and s == pytest.approx(0.01, rel=1e-12)
    # a box that does not divide evenly: M = 10^6 in 1.3 x 0.7 x 1.1: s = 1.001^(1/3) / 100
    dims, s = voxel_grid(10 ** 6, (1.3, 0.7, 1.1))
    assert s == pytest.approx((1.3 * 0.7 * 1.1 / 1e6) ** (1 / 3), rel=1e-12)
    assert dims == tuple(math.floor(L / s) for L in (1.3, 0.7, 1.1)) == (129, 69, 109)
    assert dims[0] * dims[1] * dims[2] <= 10 ** 6


def test_schedule_without_checkpoints_and_bad_input():
    assert pg_schedule(64 ** 3, (2.0, 2.0, 2.0), []) == [(0, (64,) * 3, pytest.approx(2 / 64))]
    with pytest.raises(ValueError):
        pg_schedule(64 ** 3, (2.0, 2.0, 2.0), [100, 100])
    with pytest.raises(ValueError):
        voxel_grid(0, (1.0, 1.0, 1.0))
