#!/usr/bin/env python
"""Fine-stage DVGO training-step benchmark (one JSON line on rank 0).

Workload (fine stage at the paper's default resolution, Sec. 5.2 / Supp. A): 160^3 density grid
(8 seeded balls of raw density 50, 0 outside) and a 12-channel feature grid (smooth seeded albedo),
colour MLP 39 -> 128 -> 128 -> 3, step 0.5 voxel, shift b for alpha_init = 1e-6, batches of 8192
rays drawn from 100 inward-facing 800x800 views (radius 4, focal 1111).  One step = forward render
+ MSE + backward + Adam on every parameter (density, features, MLP).

Forms (both are timed by default; `value` is the chosen form):
  plain  = uniform 0.5-voxel steps, FP32 feature grid, FP32 SIMT MLP;
  chosen = learned proposal (64-bin PDF from a BF16 tensor-core proposal MLP trained by its BF16
           tensor-core backward; 48 inverse-CDF samples per ray from the PDF mixed 0.05 with the
           uniform one; every 4th step is a full uniform step whose forward also labels 1024 rays
           for one proposal Adam step), BF16 feature storage with an FP32 master copy, BF16
           tensor-core MLP.
The line also carries the sample-proposal evaluation on this scene (`proposal_eval`) and, at one
GPU, the FP64 CPU oracle's rate on a bounded sample (`cpu_baseline`).

--impl reference times the FP64 CPU oracle on the same workload (bounded ray sample per step).
"""
from __future__ import annotations

import argparse
import gc
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
N_PROP_SAMPLES = 48
PROPOSAL_EVERY = 4
PROPOSAL_TRAIN_RAYS = 1024
PROPOSAL_ETA = 0.05
# Colour-MLP input width: 39 (features + PE(d), the benchmark's model) or 72 (+ PE(x, 5), --pe-x)
MLP_IN = 39


def mlp_fwd_flop():
    return 2 * (MLP_IN * 128 + 128 * 128 + 128 * 3)                                      # 43,520 at 39


def mlp_bwd_flop():
    return 2 * (128 * 3 + 128 * 3 + 128 * 128 + 128 * 128 + MLP_IN * 128 + 12 * 128)     # 80,128 at 39


def n_params():
    return RES ** 3 * (1 + FEAT) + (MLP_IN + 1) * 128 + 129 * 128 + 129 * 3              # 22,019 MLP at 39


def n_freq_pos():
    return 5 if MLP_IN == 72 else 0
ACT_ORDERS = {"post": 0, "pre": 1, "in": 2}   # Sec. 3 interpolation / activation orders
LAYOUTS = {"canonical": 0, "packed": 1}          # grid storage layouts (dvgo.h)


def max_over_ranks(x: float, world: int, device) -> float:
    """The maximum of x over all ranks (identity on one rank); device is where the process group's
    backend keeps its tensors (CUDA for NCCL, CPU for gloo)."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job throughput of independent replicas: the units all ranks processed divided by the
    slowest rank's time (weak scaling: every rank processes the same units)."""
    return units_per_rank * world / (ms_max / 1e3)


def workload(seed=0):
    import synth
    dens, feat = synth.fine_scene(seed=seed, res=RES, feat_dim=FEAT)
    mlp = synth.mlp_weights(MLP_IN, HID, 3, seed=3)
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

    def wait_ready(self, timeout_s=5.0):
        """Block until the first sample has arrived: nvidia-smi's start-up (NVML initialisation,
        ~0.1-0.2 s of driver work) then lies before the timed region, not inside it."""
        t0 = time.perf_counter()
        while self.proc is not None and not self.lines and time.perf_counter() - t0 < timeout_s:
            time.sleep(0.01)

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


# ------------------------------------------------------------------------------------------------
# CPU legs (the FP64 oracle)
# ------------------------------------------------------------------------------------------------

class OracleStep:
    """The FP64 oracle on n rays of a batch (fwd + bwd) plus one oracle Adam sweep over all
    parameters, projected to a full batch of `batch_rays` rays.  Defaults: the 160^3 training step (160^3
    on [-1, 1]^3, b for alpha_init 1e-6, step 0.5 voxel)."""

    def __init__(self, dens, feat, mlp, shape=None, box=((-1.0,) * 3, (1.0,) * 3), shift_b=None, step=None,
                 pe_pos=None, batch_rays=NRAYS, params=None, adam_sample=None, **_):
        import oracle
        self.oracle = oracle
        shape = tuple(dens.shape[:3]) if shape is None else tuple(shape)
        step = 2.0 / RES * 0.5 if step is None else step
        shift_b = oracle.shift_from_alpha_init(1e-6, 2.0 / RES) if shift_b is None else shift_b
        pe_pos = n_freq_pos() if pe_pos is None else pe_pos
        self.P = params if params is not None else oracle.Params(
            grid_shape=shape, xyz_min=tuple(float(np.float32(v)) for v in box[0]),
            xyz_max=tuple(float(np.float32(v)) for v in box[1]), shift_b=float(np.float32(shift_b)),
            delta=float(np.float32(step)), bg=(1.0, 1.0, 1.0), mode=1, feat_dim=FEAT, n_freq=4, hidden=HID,
            n_freq_pos=pe_pos)
        self.dens64, self.feat64 = dens.astype(np.float64), feat.astype(np.float64)
        self.mlp64 = {k: np.asarray(v).astype(np.float64) for k, v in mlp.items()}
        n_par = int(np.prod(shape)) * (1 + FEAT) + sum(v.size for v in self.mlp64.values())
        self.n_par = n_par
        # the Adam sweep is timed on adam_sample parameters (all by default) and scaled to n_par
        # (its cost is linear in the parameter count)
        self.n_adam = n_par if adam_sample is None else min(int(adam_sample), n_par)
        self.adam_arrays = [np.zeros(self.n_adam), np.ones(self.n_adam), np.zeros(self.n_adam), np.zeros(self.n_adam)]
        self.batch_rays = batch_rays
        self.freespace = None      # oracle.FreeSpace of the known-free-space test, when the recipe has one
        self.t = 0

    def run(self, batch, n):
        o, d, jit, tgt = (np.asarray(x) for x in batch)
        t0 = time.perf_counter()
        fwd = self.oracle.render(self.P, self.dens64, self.feat64, o[:n], d[:n], jitter=jit[:n], mlp=self.mlp64,
                                 target=tgt[:n], freespace=self.freespace)
        gC = 2.0 * (fwd.rgb - tgt[:n]) / n
        self.oracle.render(self.P, self.dens64, self.feat64, o[:n], d[:n], jitter=jit[:n], mlp=self.mlp64,
                           grad_rgb=gC, freespace=self.freespace)
        t_render = time.perf_counter() - t0
        self.t += 1
        p, g, m, v = self.adam_arrays
        t1 = time.perf_counter()
        self.oracle.adam(p, g, m, v, 0.1, self.t, zero_grad=False)
        t_adam = (time.perf_counter() - t1) * self.n_par / self.n_adam
        step_s = t_render * self.batch_rays / n + t_adam
        whole = n == self.batch_rays and self.n_adam == self.n_par
        return {"value": self.batch_rays / step_s, "unit": "rays/s", "cores": self.oracle.num_threads(),
                "kind": "oracle", "step_s": step_s,
                "sample": f"{n} of {self.batch_rays} rays of one batch, fwd+bwd ({t_render:.2f} s), plus one Adam "
                          f"sweep over {self.n_adam} of the {self.n_par} parameters ({t_adam:.2f} s)"
                          + ("" if whole else ", projected to a full step")}


def run_reference(args, rank, world):
    """--impl reference: the FP64 oracle on the host cores, rank 0 only.  Each step is the whole
    step of the plain form: forward + backward of all args.ref_rays (default: all 8192) rays of a
    batch and one Adam sweep over every parameter, so ms_per_step is the measured time of a step."""
    if rank != 0:
        return
    dens, feat, mlp, batches = workload()
    ostep = OracleStep(dens, feat, mlp, batch_rays=args.ref_rays)
    vals = []
    for i in range(args.warmup + args.steps):
        r = ostep.run(batches[i % N_BATCHES], args.ref_rays)
        if i >= args.warmup:
            vals.append(r)
    step_s = statistics.median(v["step_s"] for v in vals)
    total_s = sum(v["step_s"] for v in vals)
    value = args.ref_rays * len(vals) / total_s
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_s / len(vals) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, "plain") | {"global_batch": args.ref_rays},
            "cpu_baseline": {"value": value, "unit": "rays/s", "cores": vals[0]["cores"], "kind": "oracle",
                             "sample": f"every step whole: {args.ref_rays} rays fwd + bwd and one Adam sweep over all "
                                       f"{ostep.n_par} parameters (median step {step_s:.2f} s)"},
            "e2e": {"value": value, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(args, form):
    return {"workload": f"DVGO fine stage, 160^3 density + 12-ch feature grid, MLP {MLP_IN}-128-128-3, 8192 rays/batch, "
                        "step 0.5 voxel, 8 balls (raw density 50) + smooth albedo, 100 views 800x800",
            "form": form, "global_batch": NRAYS * args.gpus, "grid": RES, "feat_dim": FEAT, "hidden": HID,
            "layout": getattr(args, "layout", "canonical"),
            "grid_adam": "lazy (skips zero gradients)" if (form == "chosen" and getattr(args, "lazy_adam", False))
            else "dense",
            "parallelism": f"replicas x{args.gpus} (independent problems)",
            "l2": "inputs larger than L2: Adam sweeps ~1.7 GB of parameters and moments every step"}


# ------------------------------------------------------------------------------------------------
# GPU legs
# ------------------------------------------------------------------------------------------------

class Form:
    """One training form on the benchmark scene: its model, its step, and what it processes."""

    def __init__(self, name, dev, dens, feat, mlp, dvgo, torch, args_layout="canonical", lazy_adam=False):
        import synth
        self.name, self.dvgo, self.torch = name, dvgo, torch
        chosen = name == "chosen"
        step = 2.0 / RES * 0.5
        self.p = dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=step,
                             shift_b=dvgo.dvgo_shift_from_alpha_init(1e-6, 2.0 / RES), bg=(1.0, 1.0, 1.0),
                             mlp_prec=dvgo.DVGO_MLP_BF16 if chosen else dvgo.DVGO_MLP_FP32, n_freq_pos=n_freq_pos())
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).to(dev)
        self.model = dvgo.FineModel(t(dens), t(feat), t(mlp_flat(mlp)), self.p, NRAYS, bf16_feat=chosen,
                                    overlap_adam=chosen, layout=LAYOUTS[args_layout],
                                    lazy_grid_adam=chosen and lazy_adam)
        self.trainer = None
        if chosen:
            prop = dvgo.Proposal(synth.proposal_weights(39, 64, seed=5), self.p, self.model.dd, NRAYS,
                                 sample_precision=dvgo.DVGO_MLP_BF16, train_precision=dvgo.DVGO_MLP_BF16)
            self.trainer = dvgo.ProposalTrainer(self.model, prop, N_PROP_SAMPLES, PROPOSAL_EVERY, 0,
                                                PROPOSAL_TRAIN_RAYS, PROPOSAL_ETA)

    def step(self, batch):
        o, d, jit, tgt = batch
        if self.trainer is None:
            return self.model.train_step(o, d, jit, tgt)
        return self.trainer.step(o, d, jit, tgt)

    def finish(self):
        """Queue any deferred work of the last step (its feature-grid Adam) before the end event."""
        self.model.wait_params()


def measure_form(name, args, dev, dens, feat, mlp, batches, dvgo, torch, world, local_rank, peaks):
    form = Form(name, dev, dens, feat, mlp, dvgo, torch, args.layout, args.lazy_adam)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).to(dev)
    dbatches = [tuple(t(x) for x in b) for b in batches]
    # samples per batch of the uniform forward (units of the colour kernels)
    cnt = torch.empty(NRAYS, dtype=torch.int32, device=dev)
    tot = torch.empty(1, dtype=torch.int32, device=dev)
    totals, hits = [], []
    for b in dbatches:
        form.model.forward(b[0], b[1], b[2])
        dvgo.dvgo_sample_counts(form.model.renderer.workspace, NRAYS, cnt, tot)
        totals.append(int(tot.item()))
        hits.append(int((cnt > 0).sum().item()))
    dense_samples = float(np.mean(totals))
    hit_rays = float(np.mean(hits))
    # the clock sampler runs from before the warm-up through the timed region
    clocks = ClockSampler(local_rank)
    clocks.start()
    clocks.wait_ready()
    for i in range(args.warmup):
        form.step(dbatches[i % N_BATCHES])
    form.finish()                      # the timed region starts with no deferred work pending
    torch.cuda.synchronize()
    assert np.isfinite(form.model.loss.item())

    # the timed region: per-kernel profiling off
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = dvgo.dvgo_launch_counter()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    gc.collect()
    gc.disable()                       # no collector pause while the host issues the timed steps
    e0.record(s)
    for i in range(args.steps):
        form.step(dbatches[i % N_BATCHES])
    form.finish()
    e1.record(s)
    torch.cuda.synchronize()
    gc.enable()
    clk = clocks.stop()
    launches = dvgo.dvgo_launch_counter() - launches0
    ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    value = whole_job_rate(NRAYS * args.steps, world, ms)

    # a separate pass of the same number of steps with per-kernel CUDA-event timing switched on
    # (each launch bracketed by events on its own stream): where the step's time goes
    prof_steps = max(args.steps, 20)
    torch.cuda.synchronize()
    dvgo.dvgo_profile_enable(True)
    for i in range(PROPOSAL_EVERY):    # one recorded, uncounted cycle fills the library's event pool
        form.step(dbatches[i % N_BATCHES])
    form.finish()
    torch.cuda.synchronize()
    for k in dvgo.KERNEL_KINDS:
        dvgo.dvgo_profile_read(k)
    t_first = form.trainer.i if form.trainer is not None else 0
    n_prop_train0 = form.trainer.n_uniform if form.trainer is not None else 0
    for i in range(prof_steps):
        form.step(dbatches[i % N_BATCHES])
    form.finish()
    torch.cuda.synchronize()
    dvgo.dvgo_profile_enable(False)
    per_kind = {k: dvgo.dvgo_profile_read(k) for k in dvgo.KERNEL_KINDS}
    n_prop_train = (form.trainer.n_uniform - n_prop_train0) if form.trainer is not None else 0
    # chosen form: the same number of steps again, each waiting for the previous step's feature-grid
    # Adam before it starts, so that nothing runs beside any kernel: each kernel's own time (the
    # sampling, ray set-up, scan and density pass otherwise share the GPU with that Adam)
    per_kind_alone = None
    if form.trainer is not None:
        dvgo.dvgo_profile_enable(True)
        for i in range(prof_steps):
            form.step(dbatches[i % N_BATCHES])
            form.finish()
        torch.cuda.synchronize()
        dvgo.dvgo_profile_enable(False)
        per_kind_alone = {k: dvgo.dvgo_profile_read(k) for k in dvgo.KERNEL_KINDS}

    # end to end through the public API with host buffers: H2D of each step's rays / jitter /
    # targets from pinned memory, the step, and a D2H read of its loss
    host = [tuple(torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).pin_memory() for x in b) for b in batches]
    stager = dvgo.BatchStager(dbatches[0])   # double-buffered: the next batch copies while a step computes
    loss_host = torch.empty(args.steps, dtype=torch.float32).pin_memory()
    h2d = sum(x.numel() * 4 for x in host[0])
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_host0 = time.perf_counter()
    e2.record(s)
    stager.copy_stream.wait_event(e2)        # the first batch's copy starts inside the timed region
    stager.stage(host[0])
    for i in range(args.steps):
        batch = stager.take(s)
        if i + 1 < args.steps:
            stager.stage(host[(i + 1) % N_BATCHES])
        loss = form.step(batch)
        stager.done(s)
        loss_host[i:i + 1].copy_(loss, non_blocking=True)
    form.finish()
    e3.record(s)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(max(e2.elapsed_time(e3), (time.perf_counter() - t_host0) * 1e3), world, dev)
    assert np.all(np.isfinite(loss_host.numpy()))

    # units processed per launch of the colour kernels (uniform and proposal steps of the profiled pass)
    if name == "plain":
        fwd_units = bwd_units = dense_samples
    else:
        expl = hit_rays * N_PROP_SAMPLES
        n_dense = sum(form.trainer.is_uniform(i) for i in range(t_first, t_first + prof_steps))
        fwd_units = bwd_units = ((prof_steps - n_dense) * expl + n_dense * dense_samples) / prof_steps
    # algorithmic bytes of every Adam launch of the profiled pass: per step the density, feature and
    # MLP sweeps (adam_step_bytes with the touched points' gradients to clear), plus one proposal
    # Adam per proposal training step (chosen form; its gradients are all nonzero: 32 B per parameter)
    prop_params = int(form.trainer.proposal.flat.numel()) if form.trainer is not None else 0
    step_roof = step_hbm_minimum(form, dbatches[0], ms / args.steps, dvgo, torch, peaks)
    nz = step_roof["grad_nonzero_per_step"]
    adam_bytes = prof_steps * adam_step_bytes(name == "chosen", nz) + n_prop_train * 32 * prop_params
    dom_name, (dom_ms, dom_n) = max(per_kind.items(), key=lambda kv: kv[1][0])
    roof = roofline(dom_name, dom_ms, dom_n, fwd_units, bwd_units, name == "chosen", peaks, adam_bytes,
                    (prof_steps, adam_step_bytes(name == "chosen", nz)))
    return {"value": value, "ms_per_step": ms / args.steps, "dtype": "bf16" if name == "chosen" else "f32",
            "config": workload_config(args, name) | {"dense_samples_per_batch": dense_samples,
                                                     "hit_rays_per_batch": hit_rays,
                                                     "samples_per_hit_ray": N_PROP_SAMPLES if name == "chosen" else None},
            "roofline": roof, "step_roofline": step_roof,
            "kernels_ms_per_step": {k: round(v[0] / prof_steps, 4) for k, v in per_kind.items() if v[1]},
            "kernels_timing": f"a separate pass of {prof_steps} steps with per-launch CUDA events; the timed region "
                              f"runs without them",
            "kernels_alone_ms_per_step": (None if per_kind_alone is None else
                                          {k: round(v[0] / prof_steps, 4) for k, v in per_kind_alone.items() if v[1]}),
            "kernels_alone_timing": (None if per_kind_alone is None else
                                     f"a third pass of {prof_steps} steps, each waiting for the previous step's "
                                     f"feature-grid Adam: no kernel has another running beside it"),
            "e2e": {"value": whole_job_rate(NRAYS * args.steps, world, e2e_ms), "unit": "rays/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 4,
                    "staging": "pinned host batches copied by BatchStager on a copy stream, double-buffered, "
                               "every copy inside the timed region"},
            "gpu_launches": launches, "clocks": clk}


def step_hbm_minimum(form, batch, ms_per_step, dvgo, torch, peaks):
    """The whole step against the HBM roofline: the minimum DRAM bytes of one step -- every touched
    lattice point's density (4 B) and features (48 B FP32 / 24 B BF16) read once and its FP32
    gradients read and written once, the dense Adam sweep (adam_step_bytes: 28 B per parameter, the
    clearing of the touched points' gradients, the 2-byte BF16 feature copy), 48 B of ray input per
    ray -- with the touched points counted exactly (dvgo_touched_points) on one batch; the chosen
    form weights a uniform step and a proposal step by how often each runs."""
    m = form.model
    o, d, jit, _ = batch
    counts = {}
    m.forward(o, d, jit)
    counts["uniform"] = dvgo.dvgo_touched_points(m.params, m.dd, NRAYS, None, m.renderer.workspace)[1]
    mix = {"uniform": 1.0}
    if form.trainer is not None:
        tr = form.trainer
        ts, dts = tr.proposal.sample(o, d, jit, tr.n_samples, eta=tr.eta)
        rend = m.explicit_renderer(tr.n_samples)
        rend.forward(m.density, m.cgrid, m.mlp, o, d, jit, (ts, dts))
        counts["proposal"] = dvgo.dvgo_touched_points(m.params, m.dd, NRAYS, (ts, dts), rend.workspace)[1]
        mix = {"uniform": 1.0 / tr.uniform_every, "proposal": 1.0 - 1.0 / tr.uniform_every}
    torch.cuda.synchronize()
    counts = {k: [int(x) for x in v.cpu()] for k, v in counts.items()}
    feat_b = 24 if m.bf16_feat else 48
    render = sum(w * (counts[k][0] * 4 * 3 + counts[k][1] * (feat_b + 2 * 48)) for k, w in mix.items())
    # gradient elements the backward leaves nonzero: the touched points' density and features, the MLP
    mlp_params = n_params() - RES ** 3 * (1 + FEAT)
    nz = sum(w * (counts[k][0] + counts[k][1] * FEAT) for k, w in mix.items()) + mlp_params
    adam = adam_step_bytes(m.bf16_feat, nz)
    byts = render + adam + 48 * NRAYS
    hbm = peaks.get("hbm_gbs") or 6800.0
    achieved = byts / (ms_per_step * 1e-3) / 1e9
    return {"bound": "hbm", "hbm_min_bytes_per_step": int(byts), "render_bytes": int(render), "adam_bytes": int(adam),
            "touched_points": counts, "grad_nonzero_per_step": int(nz), "achieved": achieved, "unit": "GB/s",
            "peak": hbm, "frac": achieved / hbm,
            "peak_source": "measured" if peaks.get("hbm_gbs") else "fallback"}


def adam_step_bytes(chosen, grad_nonzero=None):
    """Algorithmic bytes of one step's Adam sweeps: 28 B per parameter (read p, g, m, v; write p, m,
    v), 4 B per gradient element the backward left nonzero (cleared for the next step; the kernel
    does not rewrite an element that is already zero; every element when grad_nonzero is None) and,
    in the chosen form, the 2-byte BF16 copy of each feature."""
    nz = n_params() if grad_nonzero is None else grad_nonzero
    return n_params() * 28 + 4 * nz + (RES ** 3 * FEAT * 2 if chosen else 0)


def roofline(kind, total_ms, launches, fwd_units, bwd_units, chosen, peaks, adam_bytes=None,
             adam_step_launch_bytes=None):
    """The dominant kernel against its roofline: achieved = algorithmic work per launch / average
    launch time (CUDA events), i.e. the work of all its launches over their summed time."""
    hbm = peaks.get("hbm_gbs")
    launches = max(int(launches), 1)
    avg_ms = total_ms / launches
    if kind in ("fine_colour_bwd", "fine_colour_fwd"):
        units = bwd_units if kind == "fine_colour_bwd" else fwd_units
        flop = units * (mlp_fwd_flop() + (mlp_bwd_flop() if kind == "fine_colour_bwd" else 0))
        achieved = flop / (avg_ms * 1e-3) / 1e12
        if chosen:
            peak = peaks.get("bf16_tflops_sustained", 1700.0)
            return {"bound": "tensor", "kernel": kind, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": traffic_from_profiles(kind, chosen), "units_per_launch": units,
                    "flop_per_launch": flop, "ms_per_launch": avg_ms, "launches": launches,
                    "peak_source": "measured bf16 sustained" if "bf16_tflops_sustained" in peaks else "fallback"}
        peak = 152 * 128 * 2 * 2.07e9 / 1e12
        return {"bound": "alu", "kernel": kind, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic_from_profiles(kind, chosen), "units_per_launch": units,
                "flop_per_launch": flop, "ms_per_launch": avg_ms, "launches": launches,
                "peak_source": "derived: 152 SM x 128 FP32 FMA/clk x 2 FLOP x 2.07 GHz"}
    if kind == "adam":
        byts = adam_bytes / launches
        achieved = byts / (avg_ms * 1e-3) / 1e9
        peak = hbm or 6800.0
        # the ncu summary gives the DRAM bytes per launch averaged over one step's three grid / MLP
        # launches; the proposal's small launches (chosen form) are counted at their algorithmic bytes
        tr = traffic_from_profiles(kind, chosen)
        if tr is not None and adam_step_launch_bytes is not None:
            n_step, step_b = adam_step_launch_bytes
            tr = (tr * 3 * n_step + (adam_bytes - n_step * step_b)) / launches
        return {"bound": "hbm", "kernel": kind, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": tr,
                "algorithmic_bytes_per_launch": byts, "ms_per_launch": avg_ms, "launches": launches,
                "note": "launches of the density, feature-grid and MLP sweeps of every step (and of the "
                        "proposal's, chosen form) averaged: their bytes over their summed time",
                "peak_source": "measured" if hbm else "fallback"}
    return {"bound": "hbm", "kernel": kind, "achieved": None, "peak": hbm, "unit": "GB/s", "frac": None,
            "traffic": None}


def traffic_from_profiles(kind, chosen):
    """DRAM bytes per launch from the committed ncu summary of this kernel, if it was taken on the
    current source (the summary records the source file's hash)."""
    import hashlib
    import re
    prof, src = {("fine_colour_bwd", False): ("fine_colour_bwd_fp32_160cube_8192rays.md", "fine_simt.cu"),
                 ("fine_colour_bwd", True): ("fine_kernels_bf16_chosen_160cube_8192rays.md", "fine_tc.cu"),
                 ("adam", False): ("adam_fine_step_160cube.md", "adam.cu"),
                 ("adam", True): ("adam_fine_step_160cube.md", "adam.cu")}.get((kind, chosen), (None, None))
    if prof is None or not os.path.exists(os.path.join(ROOT, "profiles", prof)):
        return None
    text = open(os.path.join(ROOT, "profiles", prof)).read()
    m = re.search(r"traffic_bytes_per_launch: (\d+) \(\S+ sha256 prefix: (\w+)\)", text)
    if not m:
        return None
    sha = hashlib.sha256(open(os.path.join(ROOT, "paper_2111_11215_gb300", "csrc", src), "rb").read()).hexdigest()
    return int(m.group(1)) if sha.startswith(m.group(2)) else None


def proposal_eval(dev, dens, feat, mlp, dvgo, torch, n_train=400):
    """Sample proposal on the benchmark scene (fixed grids and MLP): train the proposal (BF16
    tensor-core forward and backward) on labels from uniform FP32 renders, then compare 48 proposal samples and 48 uniform samples per ray
    against the uniform 0.5-voxel FP32 render (which matches the FP64 oracle to 1e-5)."""
    import synth
    step = 2.0 / RES * 0.5
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).to(dev)
    mk = lambda prec: dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=step, bg=(1.0, 1.0, 1.0), mlp_prec=prec,
                                  shift_b=dvgo.dvgo_shift_from_alpha_init(1e-6, 2.0 / RES), n_freq_pos=n_freq_pos())
    p32 = mk(dvgo.DVGO_MLP_FP32)
    m32 = dvgo.FineModel(t(dens), t(feat), t(mlp_flat(mlp)), p32, NRAYS)
    prop = dvgo.Proposal(synth.proposal_weights(39, 64, seed=5), p32, m32.dd, NRAYS,
                         sample_precision=dvgo.DVGO_MLP_BF16, train_precision=dvgo.DVGO_MLP_BF16)
    losses = []
    for i in range(n_train):
        o, d, _, _ = (t(x) for x in synth.fine_batch(NRAYS, seed=5000 + i))
        m32.forward(o, d, None)
        losses.append(prop.train_step(m32.renderer.workspace, o, d).clone())
    losses = [float(x.item()) for x in losses[::50]] + [float(losses[-1].item())]
    o, d, _, _ = (t(x) for x in synth.fine_batch(NRAYS, seed=9999))
    ref = m32.forward(o, d, None)[0].clone()
    ts, dts = prop.sample(o, d, None, N_PROP_SAMPLES)
    rend = m32.explicit_renderer(N_PROP_SAMPLES)
    c_prop = rend.forward(m32.density, m32.cgrid, m32.mlp, o, d, None, (ts, dts))[0].clone()
    uni = torch.full((NRAYS, 64), 1.0 / 64, device=dev)
    tu, dtu = torch.empty_like(ts), torch.empty_like(dts)
    dvgo.dvgo_sample_pdf(p32, m32.dd, o, d, uni, N_PROP_SAMPLES, None, 1e-3, tu, dtu)
    c_uni = rend.forward(m32.density, m32.cgrid, m32.mlp, o, d, None, (tu, dtu))[0].clone()
    # the chosen form's arithmetic: BF16 feature storage and BF16 tensor-core MLP on the proposal samples
    pbf = mk(dvgo.DVGO_MLP_BF16)
    mbf = dvgo.FineModel(t(dens), t(feat), t(mlp_flat(mlp)), pbf, NRAYS, bf16_feat=True)
    c_chosen = mbf.explicit_renderer(N_PROP_SAMPLES).forward(mbf.density, mbf.cgrid, mbf.mlp, o, d, None,
                                                             (ts, dts))[0].clone()
    torch.cuda.synchronize()

    def stats(c):
        err = (c - ref).abs()
        mse = float(((c - ref) ** 2).mean().item())
        return {"psnr_vs_uniform_dense": -10 * np.log10(max(mse, 1e-20)), "max_abs": float(err.max().item()),
                "mean_abs": float(err.mean().item())}
    return {"train_steps": n_train, "loss_every_50": losses, "samples_per_ray": N_PROP_SAMPLES,
            "reference": "uniform 0.5-voxel FP32 render (matches the FP64 oracle to 1e-5, tests/test_gpu_parity.py)",
            "proposal_fp32_mlp": stats(c_prop), "uniform48_fp32_mlp": stats(c_uni),
            "proposal_chosen_bf16": stats(c_chosen)}


def run_time_to_psnr(args):
    print(json.dumps(time_to_psnr(args)), flush=True)


def time_to_psnr(args):
    """Full per-scene optimisation on the analytic 20-primitive scene: ground truth for 100 training and
    20 held-out 800x800 views, coarse stage (100^3 density + RGB, 5k steps), fine stage (160^3 density
    + 12-channel features + MLP, 20k steps, Adam 0.1 / 1e-3 with the decay of Supp. A, 8192 rays per
    step) for the plain and the chosen form from the same coarse result.  Held-out PSNR is measured
    with the uniform FP32 renderer every `eval_every` steps on 2 held-out views; the fine-stage time
    excludes evaluation.  The PSNR target is the plain form's final PSNR minus 0.5 dB unless given."""
    import torch
    import synth
    import paper_2111_11215_gb300 as dvgo
    from paper_2111_11215_gb300 import progressive

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    t_start = time.perf_counter()
    scene = synth.analytic_scene(seed=0)
    rig_tr, rig_te = synth.hemisphere_rig(100, seed=2024), synth.hemisphere_rig(20, seed=2025)

    def gt(rig):
        o, d = synth.rig_rays_torch(rig, dev)
        img = torch.empty_like(o)
        for s in range(0, o.shape[0], 1 << 22):
            img[s:s + (1 << 22)] = synth.render_analytic(scene, o[s:s + (1 << 22)], d[s:s + (1 << 22)])
        return o, d, img
    o_tr, d_tr, c_tr = gt(rig_tr)
    o_te, d_te, c_te = gt(rig_te)
    n_eval = 2 * 800 * 800
    torch.cuda.synchronize()
    t_gt = time.perf_counter() - t_start
    gen = torch.Generator(device=dev)

    def batch(step, seed):
        gen.manual_seed(seed * 1000003 + step)
        idx = torch.randint(0, o_tr.shape[0], (NRAYS,), device=dev, generator=gen)
        jit = torch.rand(NRAYS, device=dev, generator=gen)
        return o_tr[idx].contiguous(), d_tr[idx].contiguous(), jit, c_tr[idx].contiguous()

    def timed_loop(fn, n, finish=None):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(n):
            fn()
        if finish is not None:
            finish()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    # ---------------- coarse stage ----------------
    rc = 100
    # Supp. A auxiliary loss weights (per-point rgb, background entropy): 1e-1 / 1e-2 coarse, 1e-2 / 1e-3 fine
    aux_c, aux_f = ((0.1, 0.01), (1e-2, 1e-3)) if args.aux_losses else ((0.0, 0.0), (0.0, 0.0))
    pc = dvgo.Params(mode=dvgo.DVGO_MODE_COARSE, step=0.5 * 2.0 / rc, bg=(1.0, 1.0, 1.0),
                     shift_b=dvgo.dvgo_shift_from_alpha_init(1e-6, 2.0 / rc), w_pt_rgb=aux_c[0], w_bg=aux_c[1],
                     act_order=ACT_ORDERS[args.act_order])
    coarse = dvgo.CoarseModel(torch.zeros((rc,) * 3, device=dev), torch.zeros((rc,) * 3 + (3,), device=dev), pc, NRAYS)
    prior2 = None
    if args.prior2:
        # Sec. 4.1 Prior 2: the coarse density's learning rate scaled by n_j / n_max (view counts of
        # the training rig); the setup call is timed once cold and then over repeats (the kernel's
        # roofline: 27 FP32 flops per (point, view) pair against the FP32 FMA peak)
        c2w = torch.as_tensor(rig_tr.c2w, dtype=torch.float64).to(dev).contiguous()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        n_max = coarse.set_view_counts(c2w, rig_tr.height, rig_tr.width, rig_tr.focal)
        e1.record()
        torch.cuda.synchronize()
        t_first = e0.elapsed_time(e1)
        for _ in range(3):
            dvgo.dvgo_view_counts(coarse.dd, c2w, rig_tr.height, rig_tr.width, rig_tr.focal, with_scale=False)
        reps = 20
        e0.record()
        for _ in range(reps):
            dvgo.dvgo_view_counts(coarse.dd, c2w, rig_tr.height, rig_tr.width, rig_tr.focal, with_scale=False)
        e1.record()
        torch.cuda.synchronize()
        t_ms = e0.elapsed_time(e1) / reps
        pairs = rc ** 3 * rig_tr.c2w.shape[0]
        achieved = 27.0 * pairs / (t_ms * 1e-3) / 1e12
        peak = 152 * 128 * 2 * 2.07e9 / 1e12
        cnt = coarse.view_counts
        prior2 = {"n_max": n_max, "min_count": int(cnt.min().item()),
                  "points_below_half": int((cnt * 2 < n_max).sum().item()), "setup_ms_first_call": round(t_first, 4),
                  "roofline": {"bound": "alu", "kernel": "view_count_kernel", "ms_per_launch": round(t_ms, 4),
                               "pairs": pairs, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                               "frac": achieved / peak,
                               "peak_source": "derived: 152 SM x 128 FP32 FMA/clk x 2 FLOP x 2.07 GHz"}}
    it = [0]

    def coarse_step():
        coarse.train_step(*batch(it[0], 1))
        it[0] += 1
    t_coarse = timed_loop(coarse_step, args.coarse_steps)

    # ---------------- fine-stage initial state (shared by both forms) ----------------
    box = ((-1.0,) * 3, (1.0,) * 3)
    fshape, s_f = (RES,) * 3, 2.0 / RES
    freespace, tau_f, recipe = None, 0.0, {"name": "full-box", "grid": list(fshape), "box": box}
    pe_pos = 5 if args.pe_x else 0
    in_dim = 39 + (3 + 6 * pe_pos if pe_pos else 0)
    pg = sorted(int(c) for c in args.pg_ckpt.split(",") if c.strip())
    if args.fine_recipe == "paper":
        # Sec. 4.2: known free space of the coarse grid (tau_c = 1e-3), the fine grid allocated on the
        # box of the unknown space with M_f = 160^3 voxels, and tau_f = 1e-4 (Supp. A)
        freespace = dvgo.FreeSpace(density=coarse.density, desc=dvgo.GridDesc((rc,) * 3, 1), shift_b=pc.shift_b,
                                   step=pc.step, tau=1e-3)
        bb = dvgo.dvgo_unknown_bbox(freespace).cpu().numpy()
        h = 2.0 / (rc - 1)
        bmin, bmax = -1.0 + bb[1:4] * h, -1.0 + bb[4:7] * h
        fshape, s_f = progressive.voxel_grid(RES ** 3, bmax - bmin)
        box = (tuple(float(v) for v in bmin), tuple(float(v) for v in bmax))
        tau_f = 1e-4
        recipe = {"name": "paper (coarse known free space tau_c=1e-3, fine box from the coarse grid, tau_f=1e-4)",
                  "grid": list(fshape), "box": box, "unknown_coarse_points": int(bb[0])}
    # progressive scaling (Sec. 4.2): M_f / 2^|pg| voxels first, doubled at every checkpoint; b_f from
    # alpha_init^(f) and the final voxel size
    sched = progressive.pg_schedule(int(np.prod(fshape)), np.subtract(box[1], box[0]), pg) if pg else \
        [(0, tuple(fshape), s_f)]
    fshape0, s0 = sched[0][1], sched[0][2]
    b_f = dvgo.dvgo_shift_from_alpha_init(1e-2, s_f)
    fine_init = args.fine_init if args.fine_init != "auto" else ("zero" if args.fine_recipe == "paper" else "coarse")
    if fine_init == "zero":
        # Sec. 4.2 / Supp. A: the fine density grid starts low-density, raw 0 with b_f for
        # alpha_init^(f) = 1e-2; the known free space of the coarse grid keeps queries off empty space
        dens0 = torch.zeros(fshape0, device=dev)
    else:
        # full box without free-space skipping: the same activated density as the coarse result on the
        # finer lattice, raw_f = resize(raw_c) + b_c - b_f (trilinear; the coarse box is [-1, 1]^3)
        dens0 = dvgo.dvgo_resize_grid(coarse.dd, coarse.density.reshape(-1), dvgo.GridDesc(fshape0, 1, box[0], box[1]))
        dens0 = (dens0.view(fshape0) + (pc.shift_b - b_f)).contiguous()
    feat0 = torch.as_tensor(synth.normal_grid(fshape0, FEAT, 1e-2, seed=11), device=dev)
    mlp0 = torch.as_tensor(mlp_flat(synth.mlp_weights(in_dim, HID, 3, seed=12)), device=dev)
    p_eval = dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=0.5 * s0, shift_b=b_f, bg=(1.0, 1.0, 1.0), tau_f=tau_f,
                         freespace=freespace, act_order=ACT_ORDERS[args.act_order], n_freq_pos=pe_pos)
    eval_cache = {}
    oracle_proj = None
    if not args.no_cpu_baseline:
        # the FP64 oracle's rate on 256 rays of a fine-stage batch (fwd + bwd + Adam, the first
        # grid of the schedule, the recipe's skipping), projected to the fine stage's steps
        import oracle
        Po = oracle.Params(grid_shape=fshape0, xyz_min=tuple(float(np.float32(v)) for v in box[0]),
                           xyz_max=tuple(float(np.float32(v)) for v in box[1]), shift_b=float(np.float32(b_f)),
                           delta=float(np.float32(0.5 * s0)), tau_f=float(np.float32(tau_f)), bg=(1.0, 1.0, 1.0),
                           mode=1, feat_dim=FEAT, n_freq=4, hidden=HID, n_freq_pos=pe_pos,
                           w_pt=float(np.float32(aux_f[0])), w_bg=float(np.float32(aux_f[1])))
        mv = {k: v.cpu().numpy() for k, v in dvgo.mlp_views(mlp0, in_dim, HID).items()}
        ost = OracleStep(dens0.cpu().numpy(), feat0.cpu().numpy(), mv, params=Po)
        if freespace is not None:
            ost.freespace = oracle.FreeSpace(density=coarse.density.cpu().numpy().astype(np.float64),
                                             shift_b=float(np.float32(pc.shift_b)), delta=float(np.float32(pc.step)),
                                             tau=float(np.float32(1e-3)))
        r0 = ost.run(tuple(x.cpu().numpy() for x in batch(0, 2)), 256)
        oracle_proj = {"rays_per_s": r0["value"], "cores": r0["cores"], "step_s": r0["step_s"],
                       "projected_fine_stage_s": r0["step_s"] * args.fine_steps, "sample": r0["sample"]}

    def psnr(model, n_rays):
        # the uniform FP32 renderer on the model's current lattice and step
        if model.shape not in eval_cache:
            eval_cache[model.shape] = dvgo.Renderer(p_eval.with_(step=model.params.step), model.dd,
                                                    model.cd.with_(dtype=dvgo.DVGO_DTYPE_F32), NRAYS)
        eval_r = eval_cache[model.shape]
        se = torch.zeros((), device=dev, dtype=torch.float64)
        views = model.mlp
        for s in range(0, n_rays, NRAYS):
            o, d, c = o_te[s:s + NRAYS], d_te[s:s + NRAYS], c_te[s:s + NRAYS]
            if o.shape[0] < NRAYS:
                break
            rgb = eval_r.forward(model.density, model.feat, views, o.contiguous(), d.contiguous())[0]
            se += ((rgb - c) ** 2).sum().double()
        mse = float(se.item()) / (3 * (n_rays // NRAYS) * NRAYS)
        return -10 * np.log10(max(mse, 1e-20))

    # form name -> (BF16 MLP + BF16 feature storage, learned proposal)
    form_defs = {"plain": (False, False), "chosen": (True, True), "bf16-uniform": (True, False),
                 "fp32-proposal": (False, True)}
    forms = [f for f in args.ttp_forms.split(",") if f]
    n_ps, every, eta = args.prop_samples, args.prop_every, args.prop_eta
    results = {}
    for form in forms:
        bf16, use_prop = form_defs[form]
        p = dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=0.5 * s0, shift_b=b_f, bg=(1.0, 1.0, 1.0),
                        mlp_prec=dvgo.DVGO_MLP_BF16 if bf16 else dvgo.DVGO_MLP_FP32, tau_f=tau_f, freespace=freespace,
                        w_pt_rgb=aux_f[0], w_bg=aux_f[1], act_order=ACT_ORDERS[args.act_order], n_freq_pos=pe_pos)
        model = dvgo.FineModel(dens0.clone(), feat0.clone(), mlp0.clone(), p, NRAYS, bf16_feat=bf16,
                               overlap_adam=use_prop, box=box, lazy_grid_adam=use_prop and args.lazy_adam)
        prop = trainer = None
        if use_prop:
            prop = dvgo.Proposal(synth.proposal_weights(39, 64, seed=5), p, model.dd, NRAYS,
                                 sample_precision=dvgo.DVGO_MLP_BF16, train_precision=dvgo.DVGO_MLP_BF16)
            trainer = dvgo.ProposalTrainer(model, prop, n_ps, every, args.prop_warmup, PROPOSAL_TRAIN_RAYS, eta)
            tb, dtb = torch.empty((NRAYS, n_ps), device=dev), torch.empty((NRAYS, n_ps), device=dev)
        st = [0]
        rescale_at = {start: (dims, s) for start, dims, s in sched[1:]}

        def fine_step():
            if st[0] in rescale_at:
                dims, s = rescale_at[st[0]]
                (trainer or model).rescale(dims, 0.5 * s, adam=args.pg_adam)
            o, d, jit, tgt = batch(st[0], 2)
            if trainer is None:
                model.train_step(o, d, jit, tgt)
            else:
                trainer.step(o, d, jit, tgt)
            st[0] += 1
        curve, t_train = [], 0.0
        while st[0] < args.fine_steps:
            n = min(args.eval_every, args.fine_steps - st[0])
            t_train += timed_loop(fine_step, n, model.wait_params)
            curve.append({"step": st[0], "train_s": round(t_train, 3), "psnr": round(psnr(model, n_eval), 3)})
        results[form] = {"curve": curve, "fine_train_s": t_train, "final_psnr_2views": curve[-1]["psnr"],
                         "final_psnr_20views": psnr(model, o_te.shape[0]),
                         "ms_per_step": 1e3 * t_train / args.fine_steps}
        if prop is not None:
            # the form's own inference: proposal samples + its MLP precision
            se, nb = 0.0, 0
            for s in range(0, n_eval, NRAYS):
                o, d, c = o_te[s:s + NRAYS].contiguous(), d_te[s:s + NRAYS].contiguous(), c_te[s:s + NRAYS]
                ts, dts = prop.sample(o, d, None, n_ps, eta=eta, t_out=tb, dt_out=dtb)
                rgb = model.explicit_renderer(n_ps).forward(model.density, model.cgrid, model.mlp, o, d,
                                                            None, (ts, dts))[0]
                se += float(((rgb - c) ** 2).sum().item())
                nb += 1
            results[form]["own_inference_psnr_2views"] = -10 * np.log10(se / (3 * nb * NRAYS))
    if args.psnr_target is None and "plain" not in results:
        raise SystemExit("time-to-psnr: give --psnr-target when the plain form is not run")
    target = args.psnr_target if args.psnr_target is not None else results["plain"]["final_psnr_2views"] - 0.5
    for form, r in results.items():
        hit = [c for c in r["curve"] if c["psnr"] >= target]
        r["secs_to_target"] = hit[0]["train_s"] if hit else None
        r["steps_to_target"] = hit[0]["step"] if hit else None
    line = {"metric": METRIC, "workload": "time-to-psnr", "unit": "s", "higher_is_better": False,
            "value": results["chosen"]["secs_to_target"] if "chosen" in results else None, "psnr_target": target,
            "psnr_target_rule": "given" if args.psnr_target is not None else "plain final PSNR (2 held-out views) - 0.5 dB",
            "coarse_steps": args.coarse_steps, "coarse_s": t_coarse, "fine_steps": args.fine_steps,
            "eval_every": args.eval_every, "ground_truth_render_s": t_gt, "data": "synthetic (analytic 20-primitive "
            "scene, 100 train + 20 held-out 800x800 views, radius 4, focal 1111)",
            "fine_recipe": recipe, "aux_losses": {"coarse": aux_c, "fine": aux_f}, "act_order": args.act_order,
            "fine_density_init": fine_init, "lazy_grid_adam_chosen": args.lazy_adam, "mlp_inputs": in_dim,
            "prior2_view_count_lr": prior2,
            "cpu_baseline": oracle_proj,
            "progressive": {"pg_ckpt": pg, "grids": [list(g) for _, g, _ in sched],
                                                  "adam": args.pg_adam},
            "proposal": {"samples_per_ray": n_ps, "uniform_every": every, "uniform_warmup": args.prop_warmup,
                         "train_rays": PROPOSAL_TRAIN_RAYS, "eta": eta},
            "forms": results}
    if "chosen" in results and "plain" in results:
        line["chosen_minus_plain_final_psnr_db"] = (results["chosen"]["final_psnr_20views"]
                                                    - results["plain"]["final_psnr_20views"])
    return line


# the recipe of the time-to-PSNR entry of the default line: the paper's whole fine stage (Sec. 4.2,
# Supp. A) -- fine density from raw 0 at alpha_init^(f) = 1e-2, known free space of the coarse grid
# (tau_c = 1e-3) and the fine box from it, tau_f = 1e-4, the auxiliary losses, the 72-input MLP with
# PE(x, 5), progressive scaling at 1k / 2k / 3k steps
PAPER_RECIPE = {"fine_recipe": "paper", "aux_losses": True, "pe_x": True, "pg_ckpt": "1000,2000,3000",
                "fine_init": "auto", "act_order": "post", "prior2": False, "lazy_adam": False, "pg_adam": "reset",
                "ttp_forms": "plain,chosen", "no_cpu_baseline": True}


def time_to_psnr_summary(args):
    """Both forms' wall time to the frozen PSNR target on the analytic scene with the paper's recipe
    (the second half of the benchmark's metric), for the default line."""
    ns = argparse.Namespace(**(vars(args) | PAPER_RECIPE))
    t0 = time.perf_counter()
    r = time_to_psnr(ns)
    wall = time.perf_counter() - t0
    f = r["forms"]
    return {"unit": "s", "higher_is_better": False, "target_psnr_db": r["psnr_target"],
            "plain_s": f["plain"]["secs_to_target"], "chosen_s": f["chosen"]["secs_to_target"],
            "plain_steps_to_target": f["plain"]["steps_to_target"],
            "chosen_steps_to_target": f["chosen"]["steps_to_target"],
            "final_psnr_20views_db": {"plain": f["plain"]["final_psnr_20views"],
                                      "chosen": f["chosen"]["final_psnr_20views"]},
            "chosen_minus_plain_db": r["chosen_minus_plain_final_psnr_db"],
            "ms_per_step": {"plain": f["plain"]["ms_per_step"], "chosen": f["chosen"]["ms_per_step"]},
            "fine_steps": r["fine_steps"], "coarse_steps": r["coarse_steps"], "coarse_s": r["coarse_s"],
            "ground_truth_render_s": r["ground_truth_render_s"], "wall_s": wall,
            "timing": "fine-stage training time (CUDA events); evaluation (held-out PSNR on 2 views every "
                      f"{r['eval_every']} steps with the uniform FP32 renderer) excluded",
            "recipe": "paper: " + r["fine_recipe"]["name"] + ", auxiliary losses, 72-input MLP with PE(x, 5), "
                      "progressive scaling at " + ",".join(str(c) for c in r["progressive"]["pg_ckpt"]),
            "fine_grids": r["progressive"]["grids"], "data": r["data"],
            "curves": {k: [(c["step"], c["train_s"], c["psnr"]) for c in v["curve"]] for k, v in f.items()}}


def run_stress(args):
    """Large-grid stress: 256^3 density (one ball of raw density 200, radius 0.3, at the
    origin) + 12-channel BF16 feature grid, BF16 tensor-core MLP, 65,536 rays per batch from the
    radius-4 sphere all aimed into the ball (maximal gradient-scatter contention), uniform 0.5-voxel
    steps, fused backward with recomputation, Adam on all ~218 M parameters."""
    import torch
    import synth
    import paper_2111_11215_gb300 as dvgo

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    rs, nr = 256, args.stress_rays
    dens = synth.sphere_density(rs, [(0.0, 0.0, 0.0)], [0.3], 200.0)
    feat = synth.smooth_features(rs, FEAT, seed=21)
    mlp = synth.mlp_weights(39, HID, 3, seed=22)
    p = dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=0.5 * 2.0 / rs, bg=(1.0, 1.0, 1.0), mlp_prec=dvgo.DVGO_MLP_BF16,
                    shift_b=dvgo.dvgo_shift_from_alpha_init(1e-6, 2.0 / rs))
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).to(dev)
    model = dvgo.FineModel(t(dens), t(feat), t(mlp_flat(mlp)), p, nr, bf16_feat=True, layout=LAYOUTS[args.layout])
    batches = []
    for i in range(4):
        o, d = synth.blob_rays(nr, seed=300 + i)
        batches.append((t(o), t(d), t(synth.jitter(nr, 400 + i)), t(synth.targets(nr, 500 + i))))
    cnt = torch.empty(nr, dtype=torch.int32, device=dev)
    tot = torch.empty(1, dtype=torch.int32, device=dev)
    model.forward(*batches[0][:3])
    dvgo.dvgo_sample_counts(model.renderer.workspace, nr, cnt, tot)
    samples = int(tot.item())
    clocks = ClockSampler(0)
    clocks.start()
    clocks.wait_ready()
    for i in range(args.warmup):
        model.train_step(*batches[i % 4])
    torch.cuda.synchronize()
    dvgo.dvgo_profile_enable(True)
    for k in dvgo.KERNEL_KINDS:
        dvgo.dvgo_profile_read(k)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(args.steps):
        model.train_step(*batches[i % 4])
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    dvgo.dvgo_profile_enable(False)
    per_kind = {k: dvgo.dvgo_profile_read(k) for k in dvgo.KERNEL_KINDS}
    ms = e0.elapsed_time(e1) / args.steps
    cpu = None
    if not args.no_cpu_baseline:
        # the FP64 oracle on 256 of the batch's rays (fwd + bwd, the FP32-feature model), projected
        hb = tuple(x.cpu().numpy() for x in batches[0])
        cpu = OracleStep(dens, feat, mlp, step=0.5 * 2.0 / rs, shift_b=dvgo.dvgo_shift_from_alpha_init(1e-6, 2.0 / rs),
                         pe_pos=0, batch_rays=nr).run(hb, 256)
    n_params = rs ** 3 * (1 + FEAT) + 22019
    adam_ms = per_kind["adam"][0] / args.steps
    kernels = {k: round(v[0] / args.steps, 4) for k, v in per_kind.items() if v[1]}
    print(json.dumps({"metric": METRIC, "workload": "stress-256cube-blob", "value": nr / (ms / 1e3), "unit": "rays/s",
                      "higher_is_better": True, "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup,
                      "dtype": "bf16", "data": "synthetic", "samples_per_step": samples,
                      "config": {"grid": rs, "feat_dim": FEAT, "rays": nr, "feat_storage": "bf16", "mlp": "bf16 tensor cores",
                                 "layout": args.layout,
                                 "scene": "one ball r=0.3 raw density 200 at the origin; rays aimed into it"},
                      "kernels_ms_per_step": kernels,
                      "adam_gbs": n_params * (32 + 0) / 1e9 / (adam_ms / 1e3) + rs ** 3 * FEAT * 2 / 1e9 / (adam_ms / 1e3),
                      "colour_bwd_samples_per_s": samples / (kernels.get("fine_colour_bwd", 1e9) / 1e3),
                      "clocks": clk, "cpu_baseline": cpu}), flush=True)


def run_trace(args):
    """Per-launch timeline of the chosen training step on the config-2 scene: both streams, one
    cycle of PROPOSAL_EVERY steps (a uniform step, then proposal steps) after 3 warm-up cycles,
    every launch of the library with its kernel kind, start and end in ms from the cycle's first
    launch (dvgo_profile_trace: CUDA events around every launch, comparable across streams)."""
    import torch
    import paper_2111_11215_gb300 as dvgo
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    dens, feat, mlp, batches = workload(seed=0)
    form = Form("chosen", dev, dens, feat, mlp, dvgo, torch, args.layout, args.lazy_adam)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).to(dev)  # noqa: E731
    dbatches = [tuple(t(x) for x in b) for b in batches]
    for i in range(3 * PROPOSAL_EVERY):
        if i == 2 * PROPOSAL_EVERY:
            dvgo.dvgo_profile_enable(True)     # one recorded warm-up cycle fills the event pool
        form.step(dbatches[i % N_BATCHES])
    torch.cuda.synchronize()               # the last warm-up step's feature-grid Adam stays deferred:
    dvgo.dvgo_profile_trace()              # the traced cycle starts in the steady state; drop earlier records
    for i in range(PROPOSAL_EVERY):
        form.step(dbatches[i % N_BATCHES])
    form.finish()
    torch.cuda.synchronize()
    dvgo.dvgo_profile_enable(False)
    tr = dvgo.dvgo_profile_trace()
    line = {"metric": "per-launch timeline of the chosen training step", "workload": "trace", "unit": "ms",
            "steps": PROPOSAL_EVERY, "cycle_ms": round(tr[-1][2], 4) if tr else None,
            "data": "synthetic", "config": workload_config(args, "chosen"),
            "launches": [[k, round(a, 4), round(b, 4)] for k, a, b in tr],
            "note": "the feature-grid Adam (kind adam, ~0.25 ms) runs on a side stream beside the next step's "
                    "sampling, ray set-up, scan and density pass; every other launch is on the main stream"}
    print(json.dumps(line), flush=True)


def run_render(args):
    """Test-time rendering (forward only) of full 800x800 frames of the 160^3 eight-ball scene (160^3 density
    of 8 balls, 12-channel features, MLP 39-128-128-3, 0.5-voxel steps) in 65,536-ray chunks, FP32 and
    BF16 MLP, without skipping and with the paper's test-time skipping of samples below
    tau_f = 1e-4 (Sec. 4.2).  The paper's figure for context: 0.64 s per 800x800 frame on an
    RTX 2080 Ti (Sec. 5, trained Synthetic-NeRF scenes)."""
    import torch
    import synth
    import paper_2111_11215_gb300 as dvgo

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    dens, feat, mlp, _ = workload()
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).to(dev)
    D, Fe, flat = t(dens), t(feat), t(mlp_flat(mlp))
    Fb = Fe.to(torch.bfloat16)
    views = dvgo.mlp_views(flat)
    rig = synth.hemisphere_rig(args.frames, seed=4242)
    o, d = synth.rig_rays_torch(rig, dev)
    n_px = rig.height * rig.width
    dd = dvgo.GridDesc((RES,) * 3, 1)
    out = {}
    for name, prec, tau_f in (("fp32", dvgo.DVGO_MLP_FP32, 0.0), ("fp32_skip", dvgo.DVGO_MLP_FP32, 1e-4),
                              ("bf16", dvgo.DVGO_MLP_BF16, 0.0), ("bf16_skip", dvgo.DVGO_MLP_BF16, 1e-4)):
        p = dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=0.5 * 2.0 / RES, bg=(1.0, 1.0, 1.0), mlp_prec=prec, tau_f=tau_f,
                        shift_b=dvgo.dvgo_shift_from_alpha_init(1e-6, 2.0 / RES))
        bf = prec == dvgo.DVGO_MLP_BF16
        cd = dvgo.GridDesc((RES,) * 3, FEAT, dtype=dvgo.DVGO_DTYPE_BF16 if bf else dvgo.DVGO_DTYPE_F32)
        fr = dvgo.FrameRenderer(p, dd, cd, chunk=65536)
        grid = Fb if bf else Fe
        fr.render(D, grid, views, o[:n_px], d[:n_px])          # warm-up frame
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        rgb, _ = fr.render(D, grid, views, o, d)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[name] = {"s_per_frame": ms / 1e3 / args.frames, "rays_per_s": o.shape[0] / (ms / 1e3),
                     "mean_rgb": float(rgb.mean().item())}
    print(json.dumps({"metric": "test-time render, 800x800 frames", "workload": "render", "unit": "s/frame",
                      "higher_is_better": False, "value": out["bf16_skip"]["s_per_frame"], "frames": args.frames,
                      "chunk_rays": 65536, "data": "synthetic (160^3 scene: 8 balls of raw density 50, smooth albedo)",
                      "forms": out, "paper_context": "0.64 s/frame on an RTX 2080 Ti (trained Synthetic-NeRF scenes)"}),
          flush=True)


def run_toy2d(args):
    """Image-fitting toy of Sec. 3 (Fig. exdv_poc): a binary image regressed by a 2D grid of stride s
    (grid (H/s) x (W/s)) under the post-, pre- and in-activation orders; full-image Adam steps (lr
    0.1 decayed by 0.1 over the run, the paper's grid rate) from a zero grid (b = 0, delta = 1).
    Reports the final PSNR per order and stride, and the stride at which post-activation matches
    pre-activation's PSNR at stride 2 (log-linear interpolation between measured strides)."""
    import torch
    import synth
    import paper_2111_11215_gb300 as dvgo

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    H = W = args.toy_res
    T = torch.as_tensor(synth.binary_image(H, W, seed=0), device=dev)
    strides = [float(v) for v in args.toy_strides.split(",")]
    orders = {"post": dvgo.DVGO_ACT_POST, "pre": dvgo.DVGO_ACT_PRE, "in": dvgo.DVGO_ACT_IN}
    loss = torch.empty(1, device=dev)
    res, ms = {}, {}
    for name, order in orders.items():
        res[name] = {}
        for st in strides:
            gh, gw = max(2, int(H / st)), max(2, int(W / st))
            V = torch.zeros((gh, gw), device=dev)
            g, m, v = torch.zeros_like(V), torch.zeros_like(V), torch.zeros_like(V)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for t in range(1, args.toy_steps + 1):
                dvgo.dvgo_fit2d(V, T, order, 0.0, 1.0, grad_out=g)
                dvgo.dvgo_adam_step(V, g, m, v, dvgo.dvgo_lr_at(0.1, t - 1, args.toy_steps), t)
            e1.record()
            dvgo.dvgo_fit2d(V, T, order, 0.0, 1.0, loss_out=loss)
            torch.cuda.synchronize()
            res[name][st] = -10.0 * np.log10(max(float(loss.item()), 1e-20))
            ms.setdefault(name, []).append(e0.elapsed_time(e1) / args.toy_steps)
    match = None
    if 2.0 in res["pre"]:
        ref = res["pre"][2.0]
        pts = sorted(res["post"].items())
        for (s0, p0), (s1, p1) in zip(pts, pts[1:]):
            if p0 >= ref >= p1 and p0 != p1:
                a = (p0 - ref) / (p0 - p1)
                match = float(np.exp(np.log(s0) + a * (np.log(s1) - np.log(s0))))
                break
    # the kernel alone on an image larger than L2 (the 512^2 target tiled to 8192^2, 268 MB; stride 8):
    # algorithmic bytes = the 4-byte target per pixel (grid reads and gradient atomics stay in L2)
    big = args.toy_big
    Tb = T.repeat(big // H, big // W).contiguous()
    Vb = torch.zeros((big // 8, big // 8), device=dev)
    gb = torch.zeros_like(Vb)
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    for _ in range(3):
        dvgo.dvgo_fit2d(Vb, Tb, dvgo.DVGO_ACT_POST, 0.0, 1.0, grad_out=gb, loss_out=loss)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_launch = 20
    e0.record()
    for _ in range(n_launch):
        dvgo.dvgo_fit2d(Vb, Tb, dvgo.DVGO_ACT_POST, 0.0, 1.0, grad_out=gb, loss_out=loss)
    e1.record()
    torch.cuda.synchronize()
    t_ms = e0.elapsed_time(e1) / n_launch
    achieved = 4.0 * Tb.numel() / (t_ms * 1e-3) / 1e9
    hbm = peaks.get("hbm_gbs")
    roof = {"bound": "hbm", "kernel": "fit2d (post, loss + gradient)", "image": [int(Tb.shape[0]), int(Tb.shape[1])],
            "grid": list(Vb.shape), "ms_per_launch": round(t_ms, 4), "achieved": achieved, "unit": "GB/s",
            "peak": hbm or 6800.0, "frac": achieved / (hbm or 6800.0),
            "peak_source": "measured" if hbm else "fallback", "algorithmic_bytes_per_launch": 4 * Tb.numel()}
    line = {"metric": "image-fitting toy: final PSNR per activation order and grid stride", "workload": "toy2d",
            "unit": "dB", "higher_is_better": True, "image": [H, W], "steps": args.toy_steps,
            "data": "synthetic binary image (discs, rotated rectangles, strokes), seed 0",
            "psnr_db": {k: {str(s_): round(p, 3) for s_, p in r.items()} for k, r in res.items()},
            "post_stride_matching_pre_at_2": match,
            "ms_per_step": {k: round(float(np.mean(v)), 4) for k, v in ms.items()}, "roofline": roof}
    print(json.dumps(line), flush=True)


def run_view_counts(args):
    """Prior 2 of Sec. 4.1 on its own: the view counts n_j and the scale n_j / n_max of a lattice of
    vc_res^3 points over [-1, 1]^3 under vc_views inward 800x800 views (radius 4, focal 1111; the
    default 100^3 x 100 is the coarse stage of the per-scene optimisation).  The kernel is timed with
    CUDA events over repeated launches; the roofline counts 27 FP32 flops per (point, view) pair (the
    projection of the definition: 3 sub, 9 mul + 6 add, 4 image bounds as mul + add, 1 sub) against
    the FP32 FMA peak.  The FP64 oracle runs the same problem on the host cores (cpu_baseline) and
    its counts are compared with the GPU's."""
    import torch
    import synth
    import paper_2111_11215_gb300 as dvgo

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    res, nv = args.vc_res, args.vc_views
    rig = synth.hemisphere_rig(nv, seed=2024)
    c2w = torch.as_tensor(rig.c2w, dtype=torch.float64).to(dev).contiguous()
    desc = dvgo.GridDesc((res,) * 3, 1)

    def call():
        return dvgo.dvgo_view_counts(desc, c2w, rig.height, rig.width, rig.focal)
    for _ in range(max(args.warmup, 3)):
        counts, scale, n_max = call()
    torch.cuda.synchronize()
    reps = args.vc_reps
    launches0 = dvgo.dvgo_launch_counter()
    clk = ClockSampler(0)
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        counts, scale, n_max = call()
    e1.record()
    torch.cuda.synchronize()
    clocks = clk.stop()
    launches = dvgo.dvgo_launch_counter() - launches0
    t_ms = e0.elapsed_time(e1) / reps
    # the count kernel alone (no scale pass), for the roofline
    e0.record()
    for _ in range(reps):
        dvgo.dvgo_view_counts(desc, c2w, rig.height, rig.width, rig.focal, with_scale=False)
    e1.record()
    torch.cuda.synchronize()
    k_ms = e0.elapsed_time(e1) / reps
    pairs = res ** 3 * nv
    peak = 152 * 128 * 2 * 2.07e9 / 1e12
    line = {"metric": "Prior 2 view counts: (point, view) visibility decisions per second", "workload": "view-counts",
            "value": pairs / (t_ms * 1e-3), "unit": "pairs/s", "higher_is_better": True, "n_gpus": 1,
            "steps": reps, "warmup": max(args.warmup, 3), "ms_per_call": round(t_ms, 5), "dtype": "f32 (+f64 at ties)",
            "data": "synthetic (seeded hemisphere rig)",
            "config": {"workload": f"view counts + lr scale, {res}^3 lattice over [-1,1]^3, {nv} inward 800x800 views "
                                   "(radius 4, focal 1111)", "output_bytes": int(8 * res ** 3),
                       "l2": "output 8 B/point; repeated calls on the same buffers (the camera data stays in L2)"},
            "n_max": int(n_max.item()), "gpu_launches": int(launches), "clocks": clocks}
    achieved = 27.0 * pairs / (k_ms * 1e-3) / 1e12
    line["roofline"] = {"bound": "alu", "kernel": "view_count_kernel", "ms_per_launch": round(k_ms, 5),
                        "achieved": achieved,
                        "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                        "algorithmic_flops_per_pair": 27, "pairs_per_call": pairs,
                        "peak_source": "derived: 152 SM x 128 FP32 FMA/clk x 2 FLOP x 2.07 GHz"}
    if not args.no_cpu_baseline:
        import oracle
        t0 = time.perf_counter()
        ref_c, _, ref_max = oracle.view_counts((res,) * 3, rig.c2w, rig.height, rig.width, rig.focal)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": pairs / dt, "unit": "pairs/s", "cores": oracle.num_threads(), "kind": "oracle",
                                "sample": f"the whole problem ({pairs} pairs), FP64"}
        line["matches_oracle"] = bool(np.array_equal(counts.cpu().numpy().reshape((res,) * 3), ref_c.astype(np.int32))
                                      and ref_max == int(n_max.item()))
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2111_11215_gb300 as dvgo

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dens, feat, mlp, batches = workload(seed=0)
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    forms = ["plain", "chosen"] if args.form == "both" else [args.form]
    res = {name: measure_form(name, args, dev, dens, feat, mlp, batches, dvgo, torch, world, local_rank, peaks)
           for name in forms}
    if rank != 0:
        return
    head = res["chosen" if "chosen" in res else forms[0]]
    line = {"metric": METRIC, "value": head["value"], "unit": "rays/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": head["dtype"], "data": "synthetic", "config": head["config"]}
    if "plain" in res and head is not res["plain"]:
        pl = res["plain"]
        line["plain"] = {"value": pl["value"], "unit": "rays/s", "ms_per_step": pl["ms_per_step"], "dtype": pl["dtype"],
                         "e2e": pl["e2e"]["value"], "roofline_frac": pl["roofline"]["frac"],
                         "roofline_kernel": pl["roofline"]["kernel"]}
    if not args.no_time_to_psnr and world == 1:
        line["time_to_psnr"] = None        # filled in below; placed early so that a cut tail keeps it
    line.update({
            "roofline": head["roofline"], "step_roofline": head["step_roofline"],
            "kernels_ms_per_step": head["kernels_ms_per_step"],
            "kernels_alone_ms_per_step": head.get("kernels_alone_ms_per_step"), "e2e": head["e2e"],
            "gpu_launches": head["gpu_launches"], "clocks": head["clocks"],
            "forms": res})
    if not args.no_time_to_psnr and world == 1:
        line["time_to_psnr"] = time_to_psnr_summary(args)
    if not args.no_proposal_eval and world == 1:
        line["proposal_eval"] = proposal_eval(dev, dens, feat, mlp, dvgo, torch)
    if not args.no_cpu_baseline and world == 1:
        # a bounded sample: the whole first batch through the oracle args.cpu_reps times (~10-20 s of
        # CPU work on the GPU machine's host cores), the median step reported
        ostep = OracleStep(dens, feat, mlp)
        runs = [ostep.run(batches[0], args.cpu_rays) for _ in range(args.cpu_reps)]
        best = sorted(runs, key=lambda r: r["value"])[len(runs) // 2]
        line["cpu_baseline"] = best | {"sample": best["sample"] + f"; median of {len(runs)} repetitions"}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 1000 for the training step -- long enough for several clock "
                         "samples -- 50 for the stress workload, 5 for the oracle reference arm)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--form", choices=["both", "plain", "chosen"], default="both")
    ap.add_argument("--cpu-rays", type=int, default=8192, help="rays of the oracle's CPU baseline sample")
    ap.add_argument("--cpu-reps", type=int, default=3, help="repetitions of the oracle's CPU baseline sample")
    ap.add_argument("--ref-rays", type=int, default=NRAYS, help="--impl reference: rays per oracle step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-proposal-eval", action="store_true")
    ap.add_argument("--no-time-to-psnr", action="store_true",
                    help="step workload: leave out the time-to-PSNR run of both forms (paper recipe) from the line")
    ap.add_argument("--workload", choices=["step", "time-to-psnr", "stress", "render", "toy2d", "view-counts", "trace"],
                    default="step")
    ap.add_argument("--vc-res", type=int, default=100, help="view-counts: lattice points per axis")
    ap.add_argument("--vc-views", type=int, default=100, help="view-counts: number of views")
    ap.add_argument("--vc-reps", type=int, default=2000, help="view-counts: timed calls")
    ap.add_argument("--toy-res", type=int, default=512, help="toy2d: image side in pixels")
    ap.add_argument("--toy-steps", type=int, default=2000, help="toy2d: Adam steps per fit")
    ap.add_argument("--toy-strides", default="2,3,4,5,6,8,10,12,16", help="toy2d: grid strides")
    ap.add_argument("--toy-big", type=int, default=8192, help="toy2d: image side of the bandwidth measurement")
    ap.add_argument("--frames", type=int, default=8, help="render workload: 800x800 frames timed")
    ap.add_argument("--coarse-steps", type=int, default=5000)
    ap.add_argument("--fine-steps", type=int, default=20000)
    ap.add_argument("--eval-every", type=int, default=1000)
    ap.add_argument("--ttp-forms", default="plain,chosen",
                    help="time-to-psnr forms, comma separated: plain, chosen, bf16-uniform, fp32-proposal")
    ap.add_argument("--prop-samples", type=int, default=N_PROP_SAMPLES)
    ap.add_argument("--prop-every", type=int, default=PROPOSAL_EVERY)
    ap.add_argument("--prop-eta", type=float, default=PROPOSAL_ETA)
    ap.add_argument("--prop-warmup", type=int, default=0)
    ap.add_argument("--stress-rays", type=int, default=65536, help="rays per batch of the 256^3 stress workload")
    ap.add_argument("--layout", choices=list(LAYOUTS), default="canonical",
                    help="grid storage layout of the training-step and stress workloads")
    ap.add_argument("--act-order", choices=list(ACT_ORDERS), default="post",
                    help="time-to-psnr: interpolation / activation order of the density in both stages (Sec. 3)")
    ap.add_argument("--prior2", action="store_true",
                    help="time-to-psnr: Sec. 4.1 Prior 2, the coarse density's learning rate scaled by n_j / n_max "
                         "(per-point view counts of the training views)")
    ap.add_argument("--aux-losses", action="store_true",
                    help="time-to-psnr: add the per-point rgb and background entropy losses with the Supp. A weights")
    ap.add_argument("--pe-x", action="store_true",
                    help="time-to-psnr and step: the paper's 72-input MLP, PE(x, 5) of the query point appended "
                         "(Supp. A); the step workload's default is the 39-input model")
    ap.add_argument("--pg-ckpt", default="",
                    help="time-to-psnr: progressive-scaling checkpoints of the fine stage, e.g. 1000,2000,3000 "
                         "(Supp. A); empty = the final grid from the start")
    ap.add_argument("--lazy-adam", action="store_true",
                    help="step and time-to-psnr: the chosen form's grid Adam skips elements with a zero gradient "
                         "(lazy variant, this library's option; the paper's Adam is dense)")
    ap.add_argument("--pg-adam", choices=["reset", "resize"], default="reset",
                    help="time-to-psnr: the grids' Adam moments at a progressive-scaling checkpoint")
    ap.add_argument("--fine-init", choices=["auto", "zero", "coarse"], default="auto",
                    help="time-to-psnr: fine density from raw 0 at alpha_init 1e-2 (the paper's, default of the paper "
                         "recipe) or the coarse result resized onto the fine lattice (default of the full-box recipe)")
    ap.add_argument("--fine-recipe", choices=["full-box", "paper"], default="full-box",
                    help="time-to-psnr fine stage: 160^3 on the full box, or the paper's Sec. 4.2 recipe "
                         "(fine box from the coarse grid's unknown space, known-free-space and tau_f skipping)")
    # frozen from the first full plain run: its final held-out PSNR (2 views) 29.391 dB - 0.5 dB
    ap.add_argument("--psnr-target", type=float, default=28.891)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    global MLP_IN
    if args.pe_x and args.workload == "step":
        MLP_IN = 72
    if args.steps is None:
        args.steps = 5 if args.impl == "reference" else (50 if args.workload == "stress" else 1000)
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
    if args.workload == "time-to-psnr":
        if rank == 0:
            run_time_to_psnr(args)
        return
    if args.workload == "stress":
        if rank == 0:
            run_stress(args)
        return
    if args.workload == "trace":
        if rank == 0:
            run_trace(args)
        return
    if args.workload == "render":
        if rank == 0:
            run_render(args)
        return
    if args.workload == "toy2d":
        if rank == 0:
            run_toy2d(args)
        return
    if args.workload == "view-counts":
        if rank == 0:
            run_view_counts(args)
        return
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
