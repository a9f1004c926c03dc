#!/usr/bin/env python
"""Fine-stage DVGO training-step benchmark (one JSON line on rank 0).

Workload (fine stage at the paper's default resolution, Sec. 5.2 / Supp. A): 160^3 density grid
(8 seeded balls of raw density 50, 0 outside) and a 12-channel feature grid (smooth seeded albedo),
colour MLP 39 -> 128 -> 128 -> 3, step 0.5 voxel, shift b for alpha_init = 1e-6, batches of 8192
rays drawn from 100 inward-facing 800x800 views (radius 4, focal 1111).  One step = forward render
+ MSE + backward + Adam on every parameter (density, features, MLP).

Forms: --form plain  = FP32 feature grid, FP32 SIMT MLP;
       --form chosen = BF16 feature storage (FP32 master updated by Adam), BF16 tensor-core MLP.

--impl reference times the FP64 CPU oracle on the same workload (bounded ray sample per step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fine-stage train rays/s (fwd+bwd) and secs to PSNR target, plain vs chosen"
RES, FEAT, HID, NRAYS = 160, 12, 128, 8192
N_BATCHES = 8
MLP_FWD_FLOP = 2 * (39 * 128 + 128 * 128 + 128 * 3)                              # 43,520
MLP_BWD_FLOP = 2 * (128 * 3 + 128 * 3 + 128 * 128 + 128 * 128 + 39 * 128 + 12 * 128)   # 80,128


def workload(seed=0):
    import synth
    dens, feat = synth.fine_scene(seed=seed, res=RES, feat_dim=FEAT)
    mlp = synth.mlp_weights(39, HID, 3, seed=3)
    batches = [synth.fine_batch(NRAYS, seed=100 + i) for i in range(N_BATCHES)]
    return dens, feat, mlp, batches


def mlp_flat(mlp):
    return np.concatenate([mlp[k].reshape(-1) for k in ("w1", "b1", "w2", "b2", "w3", "b3")]).astype(np.float32)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(dens, feat, mlp, batch, n_rays_sample, with_adam=True):
    """The FP64 oracle on n rays of one batch (fwd + bwd), plus one oracle Adam sweep over all
    parameters; projected to a full 8192-ray step."""
    import oracle
    o, d, jit, tgt = batch
    step = 2.0 / RES * 0.5
    P = oracle.Params(grid_shape=(RES,) * 3, shift_b=float(np.float32(oracle.shift_from_alpha_init(1e-6, 2.0 / RES))),
                      delta=float(np.float32(step)), bg=(1.0, 1.0, 1.0), mode=1, feat_dim=FEAT, n_freq=4, hidden=HID)
    n = n_rays_sample
    dens64, feat64 = dens.astype(np.float64), feat.astype(np.float64)
    mlp64 = {k: v.astype(np.float64) for k, v in mlp.items()}
    t0 = time.perf_counter()
    fwd = oracle.render(P, dens64, feat64, o[:n], d[:n], jitter=jit[:n], mlp=mlp64, target=tgt[:n])
    gC = 2.0 * (fwd.rgb - tgt[:n]) / n
    oracle.render(P, dens64, feat64, o[:n], d[:n], jitter=jit[:n], mlp=mlp64, grad_rgb=gC)
    t_render = time.perf_counter() - t0
    t_adam = 0.0
    if with_adam:
        nparam = dens.size + feat.size + sum(v.size for v in mlp.values())
        p = np.zeros(nparam); g = np.ones(nparam); m = np.zeros(nparam); v = np.zeros(nparam)
        t1 = time.perf_counter()
        oracle.adam(p, g, m, v, 0.1, 1)
        t_adam = time.perf_counter() - t1
    step_s = t_render * NRAYS / n + t_adam
    return {"value": NRAYS / step_s, "unit": "rays/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{n} of 8192 rays of one batch, fwd+bwd ({t_render:.2f} s), plus one Adam sweep over "
                      f"all {dens.size + feat.size + 22019} parameters ({t_adam:.2f} s), projected to a full step"}


def run_reference(args, rank, world):
    """--impl reference: the FP64 oracle on the host cores, rank 0 only."""
    if rank != 0:
        return
    dens, feat, mlp, batches = workload()
    n = args.ref_rays
    vals = []
    for i in range(args.warmup + args.steps):
        r = cpu_baseline(dens, feat, mlp, batches[i % N_BATCHES], n, with_adam=True)
        if i >= args.warmup:
            vals.append(r)
    value = statistics.median(v["value"] for v in vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": NRAYS / value * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args),
            "cpu_baseline": {"value": value, "unit": "rays/s", "cores": vals[0]["cores"], "kind": "oracle",
                             "sample": vals[0]["sample"]},
            "e2e": {"value": value, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(args):
    return {"workload": "DVGO fine stage, 160^3 density + 12-ch feature grid, MLP 39-128-128-3, 8192 rays/batch, "
                        "step 0.5 voxel, 8 balls (raw density 50) + smooth albedo, 100 views 800x800",
            "form": args.form, "global_batch": NRAYS * args.gpus, "grid": RES, "feat_dim": FEAT, "hidden": HID,
            "parallelism": f"replicas x{args.gpus} (independent problems)",
            "l2": "inputs larger than L2: Adam sweeps ~1.7 GB of parameters and moments every step"}


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2111_11215_gb300 as dvgo
    from paper_2111_11215_gb300 import build_lib

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dens, feat, mlp, batches = workload(seed=0)
    chosen = args.form == "chosen"
    step = 2.0 / RES * 0.5
    p = dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=step, shift_b=dvgo.dvgo_shift_from_alpha_init(1e-6, 2.0 / RES),
                    bg=(1.0, 1.0, 1.0), mlp_prec=dvgo.DVGO_MLP_BF16 if chosen else dvgo.DVGO_MLP_FP32)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).to(dev)
    model = dvgo.FineModel(t(dens), t(feat), t(mlp_flat(mlp)), p, NRAYS, bf16_feat=chosen)
    dbatches = [tuple(t(x) for x in b) for b in batches]
    # per-batch sample totals (units of the colour kernels)
    totals = []
    cnt = torch.empty(NRAYS, dtype=torch.int32, device=dev)
    tot = torch.empty(1, dtype=torch.int32, device=dev)
    for b in dbatches:
        model.forward(b[0], b[1], b[2])
        dvgo.dvgo_sample_counts(model.renderer.workspace, NRAYS, cnt, tot)
        totals.append(int(tot.item()))
    mean_samples = float(np.mean(totals))
    # training-quality sanity: loss is finite
    for i in range(args.warmup):
        model.train_step(*dbatches[i % N_BATCHES])
    torch.cuda.synchronize()
    assert np.isfinite(model.loss.item())

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    dvgo.dvgo_profile_enable(True)
    for k in dvgo.KERNEL_KINDS:
        dvgo.dvgo_profile_read(k)
    launches0 = dvgo.dvgo_launch_counter()
    clocks = ClockSampler(local_rank)
    clocks.start()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for i in range(args.steps):
        model.train_step(*dbatches[i % N_BATCHES])
    e1.record(s)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = dvgo.dvgo_launch_counter() - launches0
    dvgo.dvgo_profile_enable(False)
    per_kind = {k: dvgo.dvgo_profile_read(k) for k in dvgo.KERNEL_KINDS}
    ms = e0.elapsed_time(e1)
    if world > 1:
        tt = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        ms = float(tt.item())
    value = NRAYS * world * args.steps / (ms / 1e3)

    # end to end through the public API with host buffers: H2D of each step's rays / jitter /
    # targets from pinned memory, the step, and a D2H read of its loss
    host = [tuple(torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).pin_memory() for x in b) for b in batches]
    bufs = tuple(torch.empty_like(x) for x in dbatches[0])
    loss_host = torch.empty(args.steps, dtype=torch.float32).pin_memory()
    h2d = sum(x.numel() * 4 for x in host[0])
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_host0 = time.perf_counter()
    e2.record(s)
    for i in range(args.steps):
        hb = host[i % N_BATCHES]
        for dst, src in zip(bufs, hb):
            dst.copy_(src, non_blocking=True)
        loss = model.train_step(*bufs)
        loss_host[i:i + 1].copy_(loss, non_blocking=True)
    e3.record(s)
    torch.cuda.synchronize()
    e2e_ms = max(e2.elapsed_time(e3), (time.perf_counter() - t_host0) * 1e3)
    if world > 1:
        tt = torch.tensor([e2e_ms], device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        e2e_ms = float(tt.item())
    e2e_value = NRAYS * world * args.steps / (e2e_ms / 1e3)
    assert np.all(np.isfinite(loss_host.numpy()))

    if rank != 0:
        return
    import json as _json
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = _json.load(open(pk_path))
    # dominant kernel and its roofline
    dom = max(per_kind.items(), key=lambda kv: kv[1][0])
    dom_name, (dom_ms, dom_n) = dom
    avg_ms = dom_ms / max(dom_n, 1)
    roof = roofline(dom_name, avg_ms, mean_samples, chosen, peaks)
    line = {
        "metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16" if chosen else "f32", "data": "synthetic",
        "config": workload_config(args) | {"mean_samples_per_batch": mean_samples},
        "roofline": roof,
        "kernels_ms_per_step": {k: round(v[0] / max(args.steps, 1), 4) for k, v in per_kind.items() if v[1]},
        "e2e": {"value": e2e_value, "unit": "rays/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 4},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(dens, feat, mlp, batches[0], args.cpu_rays)
    print(json.dumps(line), flush=True)


def roofline(kind, avg_ms, samples, chosen, peaks):
    hbm = peaks.get("hbm_gbs")
    if kind in ("fine_colour_bwd", "fine_colour_fwd"):
        flop = samples * (MLP_FWD_FLOP + (MLP_BWD_FLOP if kind == "fine_colour_bwd" else 0))
        achieved = flop / (avg_ms * 1e-3) / 1e12
        if chosen:
            peak = peaks.get("bf16_tflops_sustained", 1700.0)
            return {"bound": "tensor", "kernel": kind, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": None, "peak_source": "measured bf16 sustained"}
        # FP32 SIMT: 152 SMs x 128 FP32 lanes x 2 FLOP/FMA x 2.07 GHz
        peak = 152 * 128 * 2 * 2.07e9 / 1e12
        return {"bound": "alu", "kernel": kind, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "peak_source": "derived: 152 SM x 128 FP32 FMA/clk x 2.07 GHz"}
    if kind == "adam":
        nparam = RES ** 3 * (1 + FEAT) + 22019
        byts = nparam * (32 + (2 if chosen else 0)) / 3.0   # average over the three launches per step
        achieved = byts / (avg_ms * 1e-3) / 1e9
        peak = hbm or 6800.0
        return {"bound": "hbm", "kernel": kind, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None, "peak_source": "measured" if hbm else "fallback"}
    return {"bound": "hbm", "kernel": kind, "achieved": None, "peak": hbm, "unit": "GB/s", "frac": None,
            "traffic": None}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--form", choices=["plain", "chosen"], default="plain")
    ap.add_argument("--cpu-rays", type=int, default=512)
    ap.add_argument("--ref-rays", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    from paper_2111_11215_gb300 import build_lib
    if not build_lib.up_to_date():
        raise SystemExit("libdvgo.so is missing or stale: run __graft_entry__.build() first")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
