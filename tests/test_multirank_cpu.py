"""Multi-rank paths on the CPU: two processes on the gloo backend (127.0.0.1).

* bench.py's aggregation for N > 1 independent replicas: the timed region's maximum over ranks
  and the whole-job rate (units of all ranks / the slowest rank's time).
* The exchange step a spatial split of the grid across ranks would need (each rank composites the
  segment of every ray that crosses its slab; one exchange of per-ray (C, T) tuples folded with
  C = C_front + T_front C_back, T = T_front T_back, the background added once at the end): checked
  on the FP64 oracle against the undivided render.  This run builds replicas only, so the fold is
  exercised here on the host and nowhere in the product path.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, fn_name, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, globals()[fn_name](rank, world)))
    except Exception as e:  # reported to the parent, which fails the test
        q.put((rank, repr(e)))
    finally:
        dist.destroy_process_group()


def _run(fn_name, world=2, timeout=120):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, fn_name, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    try:
        for _ in range(world):
            rank, val = q.get(timeout=timeout)
            out[rank] = val
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
    for p in procs:
        assert p.exitcode == 0, f"rank process exited with {p.exitcode}"
    return out


# ------------------------------------------------------------------------------------------------

def _bench_aggregation(rank, world):
    import bench
    ms = [10.0, 12.5][rank]
    ms_max = bench.max_over_ranks(ms, world, torch.device("cpu"))
    return {"ms_max": ms_max, "rate": bench.whole_job_rate(8192 * 5, world, ms_max)}


def test_bench_max_over_ranks_and_whole_job_rate():
    out = _run("_bench_aggregation")
    for rank in (0, 1):
        assert isinstance(out[rank], dict), out[rank]
        assert out[rank]["ms_max"] == 12.5                       # the slowest rank sets the time
        assert out[rank]["rate"] == pytest.approx(8192 * 5 * 2 / 0.0125)
    import bench
    assert bench.max_over_ranks(3.0, 1, None) == 3.0                # one rank: no collective


# ------------------------------------------------------------------------------------------------

N_S = 40


def _slab_inputs():
    import oracle
    import synth
    res, R = 12, 24
    dens = synth.normal_grid((res,) * 3, 1, 1.0, seed=900) + 1.0
    feat = synth.normal_grid((res,) * 3, 12, 0.5, seed=901)
    mlp = synth.mlp_weights(39, 16, 3, seed=902)
    o, d = synth.sphere_rays(R, seed=903)
    P = oracle.Params(grid_shape=(res,) * 3, shift_b=-1.0, delta=2.0 / res / 2, bg=(0.3, 0.6, 0.9), mode=1,
                      feat_dim=12, n_freq=4, hidden=16)
    t = np.zeros((R, N_S))
    dt = np.zeros((R, N_S))
    for r in range(R):
        _, t0, t1, _, _ = oracle.ray_bounds(P, o[r], d[r])
        assert t1 > t0
        w = (t1 - t0) / N_S
        t[r] = t0 + (np.arange(N_S) + 0.5) * w
        dt[r] = w
    return P, dens, feat, mlp, o, d, t, dt


def _slab_fold(rank, world):
    import dataclasses
    import oracle
    P, dens, feat, mlp, o, d, t, dt = _slab_inputs()
    half = N_S // world
    seg = slice(rank * half, (rank + 1) * half)
    # each rank composites its own segment of every ray, starting from T = 1 with no background
    P0 = dataclasses.replace(P, bg=(0.0, 0.0, 0.0))
    out = oracle.render(P0, dens, feat, o, d, mlp=mlp, explicit_t=t[:, seg], explicit_dt=dt[:, seg])
    mine = torch.from_numpy(np.concatenate([out.rgb, out.tfinal[:, None]], axis=1))
    parts = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(parts, mine)                                  # the one exchange of per-ray tuples
    C = np.zeros_like(out.rgb)
    T = np.ones(out.tfinal.shape)
    for p in parts:                                               # front to back
        C = C + T[:, None] * p[:, :3].numpy()
        T = T * p[:, 3].numpy()
    C = C + T[:, None] * np.asarray(P.bg)[None, :]
    full = oracle.render(P, dens, feat, o, d, mlp=mlp, explicit_t=t, explicit_dt=dt)
    return {"err_c": float(np.abs(C - full.rgb).max()), "err_t": float(np.abs(T - full.tfinal).max()),
            "scale": float(np.abs(full.rgb).max())}


def test_slab_split_exchange_folds_to_the_full_render():
    out = _run("_slab_fold")
    for rank in (0, 1):
        assert isinstance(out[rank], dict), out[rank]
        assert out[rank]["err_c"] <= 1e-12 * max(out[rank]["scale"], 1.0)
        assert out[rank]["err_t"] <= 1e-12
