#!/usr/bin/env python
"""Benchmark of the MPS (QTT) wave step on the 1024x1024 Marmousi-shaped
section (n = 10, chi_max = 128, eps = 1e-6): MPS steps per second.

One step = the whole hot path of Eq. 17: zip-up of the Laplacian MPO,
zip-up of diag(c^2), the MPS sum with the rank-1 source, and the QR + SVD
round.  The run starts from the mid-run state of the 4000-step workload
(the dense Eq. 2 field at step 2000, computed on the GPU by the library's
FDTD kernel and compressed to an MPS by the library), where the bond ranks
are saturated at chi_max; per-step cost depends only on the ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs its own replica of the workload (the
stepper does not shard): value = N * steps / max-rank time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "MPS steps/s at 2^20 grid, chi=128, rel-L2<=1e-3: chosen form vs plain FP64 (1 B300)"
UNIT = "steps/s"
WORKLOAD_IDX = 2
MID_RUN = 2000
FP64_PEAK_TFLOPS = 1.25   # nominal B300 FP64 (148 SMs x 2032 MHz x ~4.2 FLOP/clk/SM)
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12  # FP32 FMA pipes at the maximum SM clock


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"qtt_bench_clocks_rank{index}_{os.getpid()}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self) -> dict:
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        try:
            rows = [ln.split(",") for ln in open(self.path) if ln.strip()]
        except OSError:
            return out
        mhz, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                mhz.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if mhz:
            out["sm_mhz"] = statistics.median(mhz)
            out["sm_max_mhz"] = max(mx)
        out["reasons"] = sorted(reasons)
        out["samples"] = len(mhz)
        return out


def _setup_gpu_state(q, wl, ctx, c, amps, stream):
    """Velocity MPS, Laplacian MPO, and the mid-run state (dense FDTD on the
    GPU to MID_RUN, then TT-SVD + round in the library)."""
    import torch
    N = wl.N
    with torch.cuda.stream(stream):
        c_dev = torch.as_tensor(c, device="cuda")
        C = q.qtt_velocity_mps(ctx, c_dev)
        L = q.qtt_laplacian_mpo(ctx)
        c2 = c_dev * c_dev
        up = torch.zeros((N, N), dtype=torch.float64, device="cuda")
        uc, un = up.clone(), up.clone()
        lam2 = wl.lambda2(c)
        for k in range(MID_RUN):
            q.qtt_fdtd_step(ctx, c2, lam2, up, uc, un, wl.sources[0], float(amps[k]))
            up, uc, un = uc, un, up
        prev = q.qtt_mps_from_dense(ctx, up)
        cur = q.qtt_mps_from_dense(ctx, uc)
    stream.synchronize()
    return C, L, prev, cur


def job_rate(t_total_ms: float, steps: int, world: int, device: str = "cuda") -> tuple[float, float]:
    """Whole-job rate of a timed region: the maximum of the ranks' times
    (all_reduce MAX over the process group when world > 1, then a barrier)
    and world * steps / that time.  Returns (max time in ms, steps/s)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        tt = torch.tensor([t_total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_total_ms = float(tt.item())
        dist.barrier()
    return t_total_ms, world * steps / (t_total_ms / 1e3)


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2609_01904_b300 import qtt as q

    torch.cuda.set_device(local_rank)
    wl = W.config(WORKLOAD_IDX)
    c = wl.velocity()
    lam2 = wl.lambda2(c)
    total = MID_RUN + max(args.warmup + args.steps + args.e2e_steps, args.err_steps) + 2
    amps = wl.source_amplitudes(c, total)
    stream = torch.cuda.Stream()
    ctx = q.qtt_ctx_create(n=wl.n, order=wl.order, bc=wl.bc, chi_max=wl.chi, eps=wl.eps, chi_c=wl.chi_c,
                           eps_c=wl.eps_c, prec=args.form, stream=stream)
    t0 = time.time()
    C, L, prev, cur = _setup_gpu_state(q, wl, ctx, c, amps, stream)
    setup_s = time.time() - t0
    src = wl.sources[0]
    step = q.qtt_step_graph if args.graph else q.qtt_step
    k = MID_RUN
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step(L, C, lam2, prev, cur, src, float(amps[k]))
            k += 1
    q.qtt_ctx_sync(ctx)
    ranks0 = q.qtt_mps_ranks(cur)

    # L2 flush between timed steps (outside the events): a 256 MiB write
    flush = torch.empty(32 * 1024 * 1024, dtype=torch.float64, device="cuda")
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    # per-class kernel timing needs events around every launch, which graph
    # replays do not have: with --graph the classes are timed on two plain
    # steps after the timed region (same kernels, same results)
    q.qtt_profile_start(ctx, timing=not args.graph, log_svd=not args.graph)
    with ClockSampler(local_rank) as clk:
        with torch.cuda.stream(stream):
            for i in range(args.steps):
                flush.fill_(float(i))
                evs[i][0].record(stream)
                step(L, C, lam2, prev, cur, src, float(amps[k]))
                evs[i][1].record(stream)
                k += 1
        torch.cuda.synchronize()
    prof = q.qtt_profile_read(ctx)
    launches_timed = dict(prof["launches"])
    prof_steps = args.steps
    if args.graph:
        q.qtt_profile_start(ctx, timing=True, log_svd=True)
        with torch.cuda.stream(stream):
            for _ in range(2):
                q.qtt_step(L, C, lam2, prev, cur, src, float(amps[k]))
                k += 1
        prof = q.qtt_profile_read(ctx)
        prof_steps = 2
        q.qtt_profile_start(ctx, timing=False, log_svd=False)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms_per_step = float(np.mean(step_ms))
    t_total = float(np.sum(step_ms))
    t_total, value = job_rate(t_total, args.steps, world)

    # end to end through the public API: the step's input (the source sample)
    # from pinned host memory, the receiver trace read back to pinned host
    rx = torch.as_tensor(np.array([r[0] for r in wl.receivers]), device="cuda")
    rz = torch.as_tensor(np.array([r[1] for r in wl.receivers]), device="cuda")
    amp_host = torch.as_tensor(np.asarray(amps, dtype=np.float64)).pin_memory()
    amp_dev = torch.empty(1, dtype=torch.float64, device="cuda")
    trace_dev = torch.empty(len(wl.receivers), dtype=torch.float64, device="cuda")
    trace_host = torch.empty(len(wl.receivers), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for _ in range(args.e2e_steps):
            amp_dev.copy_(amp_host[k:k + 1], non_blocking=True)
            step(L, C, lam2, prev, cur, src, float(amp_host[k]))
            q.qtt_sample(cur, rx, rz, trace_dev)
            trace_host.copy_(trace_dev, non_blocking=True)
            stream.synchronize()
            k += 1
    e2e_s = time.perf_counter() - t0
    ranks1 = q.qtt_mps_ranks(cur)

    # roofline of the dominant kernel class, from the live event timing
    ms = prof["ms"]
    dom = max(ms, key=lambda kk: ms[kk])
    launches = prof["launches"]
    svd_flops = prof["svd_flops"]
    roof = {"bound": "alu", "traffic": None, "launches": launches.get(dom, 0),
            "avg_launch_ms": ms[dom] / max(launches.get(dom, 1), 1),
            "avg_sweeps": prof["svd_sweeps"] / max(prof["svd_logged"], 1),
            "work": "6 m n^2 + 20 n^3 per SVD of the reduced n x m factor (Golub-Van Loan), sizes logged per launch"}
    if dom == "jacobi" and args.form == "fp64":
        achieved = svd_flops / (ms["jacobi"] / 1e3) / 1e12
        roof.update({"kernel": "jacobi_kernel (one-sided Jacobi SVD, FP64, cooperative)", "achieved": achieved,
                     "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                     "peak_source": "nominal FP64 of the recipe (1.25 TFLOP/s); FP64 FMA probe measured 0.95"})
    elif dom == "jacobi":
        achieved = svd_flops / (ms["jacobi"] / 1e3) / 1e12
        # DRAM bytes of one 256-vector launch from the ncu capture of the
        # current kernel (profiles/jacobi32_block_qtt1024_marmousi.md)
        roof["traffic"] = 592.9e3
        roof["traffic_note"] = "dram read+write of one 256-vector launch (ncu); the input, read once"
        roof.update({"kernel": "jacobi32_block_kernel (one-sided Jacobi SVD, FP32, one cluster)",
                     "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP32_PEAK_TFLOPS,
                     "peak_source": "FP32 FMA: 148 SMs x 128 FMA/clk x 2 x 2.032 GHz; probe measured 63"})
    else:
        roof.update({"kernel": dom, "achieved": None, "peak": None, "unit": None, "frac": None})
    roof["share_of_step"] = ms[dom] / max(sum(ms.values()), 1e-9)
    roof["class_ms_per_step"] = {kk: round(v / prof_steps, 3) for kk, v in ms.items() if v > 0}

    n_launch = int(sum(launches_timed.values()))

    # context: the dense Eq. 2 update on the same GPU (library FDTD kernel),
    # HBM-bound: reads u^{k-1}, u^k, c^2 and writes u^{k+1} (4 x 8 N^2 bytes)
    dense = None
    if world == 1:
        N = wl.N
        c2d = torch.as_tensor(c * c, device="cuda")
        fd = [torch.zeros((N, N), dtype=torch.float64, device="cuda") for _ in range(3)]
        nfd = 400
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            for i in range(20):
                q.qtt_fdtd_step(ctx, c2d, lam2, fd[0], fd[1], fd[2], src, 0.0)
                fd = [fd[1], fd[2], fd[0]]
            e0.record(stream)
            for i in range(nfd):
                q.qtt_fdtd_step(ctx, c2d, lam2, fd[0], fd[1], fd[2], src, 0.0)
                fd = [fd[1], fd[2], fd[0]]
            e1.record(stream)
        q.qtt_ctx_sync(ctx)
        t_fd = e0.elapsed_time(e1) / 1e3 / nfd
        gbs = 4 * 8 * N * N / t_fd / 1e9
        peak = _peaks().get("hbm_gbs")
        dense = {"steps_per_s": 1.0 / t_fd, "grid_point_updates_per_s": N * N / t_fd, "achieved_gbs": gbs,
                 "peak_gbs": peak, "frac": (gbs / peak) if peak else None,
                 "note": "fdtd_kernel, 4 x 8 N^2 bytes per step (3 reads, 1 write), inputs resident, no L2 flush "
                         "(the 33.6 MB working set fits the 126 MB L2: an upper bound, context only)"}
    result = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if args.form == "fp64" else "f32+f64",
        "data": "synthetic (seeded Marmousi-shaped velocity section; Ricker source)",
        "config": {"workload": wl.name, "n": wl.n, "grid": f"{wl.N}x{wl.N}", "chi_max": wl.chi, "eps": wl.eps,
                   "chi_c": wl.chi_c, "eps_c": wl.eps_c, "order": wl.order, "bc": wl.bc, "form": args.form,
                   "state": f"mid-run (step {MID_RUN} of {wl.steps})", "ranks_start": ranks0,
                   "graph": bool(args.graph),
                   "ranks_end": ranks1, "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": f"replicas x{world}", "grid_point_updates_per_s": value * wl.N * wl.N,
                   "setup_s": round(setup_s, 2)},
        "gpu_launches": n_launch,
        "e2e": {"value": args.e2e_steps / e2e_s * world if args.e2e_steps else None, "unit": UNIT,
                "h2d_bytes_per_step": 8, "d2h_bytes_per_step": 8 * len(wl.receivers)},
        "roofline": roof,
        "dense_fdtd_context": dense,
        "clocks": clk.summary(),
        "step_ms": [round(x, 3) for x in step_ms],
    }
    if args.compare and world == 1:
        result["plain_fp64"], result["error"] = compare_forms(q, wl, c, amps, args)
        if result["plain_fp64"]:
            result["speedup_vs_plain_fp64"] = result["plain_fp64"]["ms_per_step"] / ms_per_step
    return result, (C, L, prev, cur, ctx)


SHOTS_IDX = 3
SHOTS_MID_RUN = 1000


def run_shots(args):
    """The 64-shot workload (512x512 layered section, per-shot bond caps
    drawn from {32, 64, 128, 256}, FP32 form): MPS shot-steps per second of
    the batched step, and the same shots stepped one after another on one
    stream for comparison.  Each shot starts from its own mid-run state (its
    dense Eq. 2 field at step 1000, compressed by the library)."""
    import torch
    from paper_2609_01904_b300 import qtt as q

    wl = W.config(SHOTS_IDX)
    c = wl.velocity()
    lam2 = wl.lambda2(c)
    chis = [int(x) for x in W.chi_per_shot(wl.seed, len(wl.sources))]
    ns = len(chis)
    total = SHOTS_MID_RUN + args.warmup + args.steps + 4
    amps = wl.source_amplitudes(c, total)
    stream = torch.cuda.Stream()
    t0 = time.time()
    batch = q.qtt_batch_create(wl.n, ns, chis, order=wl.order, bc=wl.bc, chi_max=max(chis), eps=wl.eps,
                               chi_c=wl.chi_c, eps_c=wl.eps_c, prec=args.form, stream=stream)
    q.qtt_batch_set_graphs(batch, bool(args.graph))
    N = wl.N
    with torch.cuda.stream(stream):
        c_dev = torch.as_tensor(c, device="cuda")
        C = q.qtt_velocity_mps(batch.ctxs[0], c_dev)
        L = q.qtt_laplacian_mpo(batch.ctxs[0])
        c2 = c_dev * c_dev
        prev, cur = [], []
        for s in range(ns):
            up = torch.zeros((N, N), dtype=torch.float64, device="cuda")
            uc, un = up.clone(), up.clone()
            for k in range(SHOTS_MID_RUN):
                q.qtt_fdtd_step(batch.ctxs[s], c2, lam2, up, uc, un, wl.sources[s], float(amps[k]))
                up, uc, un = uc, un, up
            prev.append(q.qtt_mps_from_dense(batch.ctxs[s], up))
            cur.append(q.qtt_mps_from_dense(batch.ctxs[s], uc))
    stream.synchronize()
    setup_s = time.time() - t0
    k = SHOTS_MID_RUN
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            q.qtt_step_batched(batch, L, C, lam2, prev, cur, wl.sources, [float(amps[k])] * ns)
            k += 1
    stream.synchronize()
    ranks0 = [max(q.qtt_mps_ranks(x)) for x in cur]
    flush = torch.empty(32 * 1024 * 1024, dtype=torch.float64, device="cuda")
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for x in batch.ctxs:
        q.qtt_profile_start(x, timing=False, log_svd=False)
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        with torch.cuda.stream(stream):
            for i in range(args.steps):
                flush.fill_(float(i))
                evs[i][0].record(stream)
                q.qtt_step_batched(batch, L, C, lam2, prev, cur, wl.sources, [float(amps[k])] * ns)
                evs[i][1].record(stream)
                k += 1
        torch.cuda.synchronize()
    launches = sum(sum(q.qtt_profile_read(x)["launches"].values()) for x in batch.ctxs)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms_per_step = float(np.mean(step_ms))
    value = ns * args.steps / (float(np.sum(step_ms)) / 1e3)
    # the same shots, one after another on the batch's stream
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        flush.fill_(-1.0)
        e0.record(stream)
        for s in range(ns):
            (q.qtt_step_graph if args.graph else q.qtt_step)(L, C, lam2, prev[s], cur[s], wl.sources[s],
                                                             float(amps[k]))
        e1.record(stream)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1)
    return {
        "metric": "MPS shot-steps/s, 64 shots on a 2^18 grid, per-shot chi in {32,64,128,256} (1 B300)",
        "value": value, "unit": "shot-steps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.form == "fp64" else "f32+f64", "data": "synthetic (seeded layered section)",
        "config": {"workload": wl.name, "n": wl.n, "shots": ns, "chi_per_shot": chis, "eps": wl.eps,
                   "graph": bool(args.graph),
                   "form": args.form, "state": f"mid-run (step {SHOTS_MID_RUN})", "max_rank_start": ranks0,
                   "l2": "flushed between timed steps (256 MiB write)", "setup_s": round(setup_s, 1)},
        "gpu_launches": int(launches),
        "sequential": {"ms_per_batch_step": seq_ms, "value": ns / (seq_ms / 1e3),
                       "note": "the same 64 shot-steps issued one after another on one stream"},
        "speedup_vs_sequential": seq_ms / ms_per_step,
        "clocks": clk.summary(),
        "step_ms": [round(x, 3) for x in step_ms],
    }


def compare_forms(q, wl, c, amps, args):
    """The plain FP64 form timed on the same mid-run state, and the error of
    both forms after args.err_steps steps: against each other, and against
    the dense Eq. 2 update continued from the same dense field."""
    import torch
    N = wl.N
    lam2 = wl.lambda2(c)
    src = wl.sources[0]
    rx = torch.as_tensor(np.array([r[0] for r in wl.receivers]), device="cuda")
    rz = torch.as_tensor(np.array([r[1] for r in wl.receivers]), device="cuda")
    out = {}
    fields, traces = {}, {}
    for form in ("fp64", args.form):
        if form in fields:
            continue
        stream = torch.cuda.Stream()
        ctx = q.qtt_ctx_create(n=wl.n, order=wl.order, bc=wl.bc, chi_max=wl.chi, eps=wl.eps, chi_c=wl.chi_c,
                               eps_c=wl.eps_c, prec=form, stream=stream)
        C, L, prev, cur = _setup_gpu_state(q, wl, ctx, c, amps, stream)
        tr = torch.zeros((args.err_steps, len(wl.receivers)), dtype=torch.float64, device="cuda")
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.err_steps + 1)]
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            for kk in range(args.err_steps):
                q.qtt_step(L, C, lam2, prev, cur, src, float(amps[MID_RUN + kk]))
                ev[kk + 1].record(stream)
                q.qtt_sample(cur, rx, rz, tr[kk])
        q.qtt_ctx_sync(ctx)
        if form == "fp64":
            t = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.err_steps)]
            out = {"ms_per_step": float(np.mean(t)), "value": 1000.0 / float(np.mean(t)), "unit": UNIT,
                   "steps": args.err_steps, "note": "same state and steps as the error check, no L2 flush"}
        dense = torch.zeros((N, N), dtype=torch.float64, device="cuda")
        q.qtt_to_dense(cur, dense)
        q.qtt_ctx_sync(ctx)
        fields[form] = dense.cpu().numpy()
        traces[form] = tr.cpu().numpy()
        del prev, cur, C, L, ctx
    # dense FDTD from the same dense state, same source samples
    ctx = q.qtt_ctx_create(n=wl.n, order=wl.order, bc=wl.bc, chi_max=wl.chi, eps=wl.eps, prec="fp64")
    c_dev = torch.as_tensor(c, device="cuda")
    c2 = c_dev * c_dev
    up = torch.zeros((N, N), dtype=torch.float64, device="cuda")
    uc, un = up.clone(), up.clone()
    for kk in range(MID_RUN + args.err_steps):
        q.qtt_fdtd_step(ctx, c2, lam2, up, uc, un, src, float(amps[kk]))
        up, uc, un = uc, un, up
    q.qtt_ctx_sync(ctx)
    fd = uc.cpu().numpy()
    rel = lambda a, b: float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    err = {"steps_from_mid_run": args.err_steps,
           "field_rel_l2_vs_fp64_mps": rel(fields[args.form], fields["fp64"]),
           "trace_rel_l2_vs_fp64_mps": rel(traces[args.form], traces["fp64"]),
           "field_rel_l2_vs_dense_fdtd": {f: rel(fields[f], fd) for f in fields},
           "threshold": 1e-3}
    err["eligible"] = err["field_rel_l2_vs_fp64_mps"] <= 1e-3 and err["trace_rel_l2_vs_fp64_mps"] <= 1e-3
    return out, err


def oracle_baseline(seconds: float, mid_run: int = 600):
    """The FP64 oracle on the host cores: a bounded sample of the same
    workload (its own FDTD to a state with saturated ranks, then timed MPS
    steps until ~`seconds` of stepping)."""
    from oracle import qtt_oracle as O
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:  # pragma: no cover
        cores = os.cpu_count() or 1
    wl = W.config(WORKLOAD_IDX)
    n = wl.n
    c = wl.velocity()
    c2 = c * c
    lam2 = wl.lambda2(c)
    amps = wl.source_amplitudes(c, mid_run + 64)
    up = np.zeros((wl.N, wl.N))
    uc = np.zeros((wl.N, wl.N))
    for k in range(mid_run):
        up, uc = uc, O.fdtd_step(up, uc, c2, lam2, wl.bc, wl.sources[0], float(amps[k]))
    Co = O.velocity_mps(c, n, wl.order, wl.eps_c, wl.chi_c)
    Lo = O.laplacian_mpo(n, wl.order, wl.bc)
    prev = O.state_from_dense(up, n, wl.order, wl.eps, wl.chi)
    cur = O.state_from_dense(uc, n, wl.order, wl.eps, wl.chi)
    t0 = time.perf_counter()
    steps = 0
    k = mid_run
    while True:
        prev, cur = cur, O.mps_step(Lo, Co, lam2, prev, cur, wl.eps, wl.chi, wl.sources[0], float(amps[k]), n,
                                    wl.order)
        steps += 1
        k += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": steps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{steps} oracle steps of {wl.name} from its own FDTD state at step {mid_run} "
                      f"(ranks {max(O.mps_ranks(cur))} max), {dt:.1f} s"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    from oracle import qtt_oracle as O
    wl = W.config(WORKLOAD_IDX)
    n = wl.n
    c = wl.velocity()
    lam2 = wl.lambda2(c)
    mid = 600
    amps = wl.source_amplitudes(c, mid + args.warmup + args.steps + 2)
    up = np.zeros((wl.N, wl.N))
    uc = np.zeros((wl.N, wl.N))
    for k in range(mid):
        up, uc = uc, O.fdtd_step(up, uc, c * c, lam2, wl.bc, wl.sources[0], float(amps[k]))
    Co = O.velocity_mps(c, n, wl.order, wl.eps_c, wl.chi_c)
    Lo = O.laplacian_mpo(n, wl.order, wl.bc)
    prev = O.state_from_dense(up, n, wl.order, wl.eps, wl.chi)
    cur = O.state_from_dense(uc, n, wl.order, wl.eps, wl.chi)
    k = mid
    for _ in range(args.warmup):
        prev, cur = cur, O.mps_step(Lo, Co, lam2, prev, cur, wl.eps, wl.chi, wl.sources[0], float(amps[k]), n,
                                    wl.order)
        k += 1
    t0 = time.perf_counter()
    for _ in range(args.steps):
        prev, cur = cur, O.mps_step(Lo, Co, lam2, prev, cur, wl.eps, wl.chi, wl.sources[0], float(amps[k]), n,
                                    wl.order)
        k += 1
    dt = time.perf_counter() - t0
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:  # pragma: no cover
        cores = os.cpu_count() or 1
    v = args.steps / dt
    return {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "n": n, "chi_max": wl.chi, "eps": wl.eps, "form": "fp64 oracle (numpy)",
                   "state": f"oracle FDTD at step {mid}"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} timed oracle steps after {args.warmup} warm-up, {dt:.1f} s"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="fp32", choices=["fp64", "fp32"],
                    help="fp32: the chosen form (FP32 contractions/QR, FP64-accurate SVDs); fp64: the plain form")
    ap.add_argument("--compare", type=int, default=1, help="also time the plain FP64 form and measure errors")
    ap.add_argument("--err-steps", type=int, default=20)
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--graph", type=int, default=1, help="1: replay each step from a CUDA graph (qtt_step_graph); 0: launch the kernels")
    ap.add_argument("--workload", default="qtt1024_marmousi", choices=["qtt1024_marmousi", "qtt512_64shots"],
                    help="qtt512_64shots: the batched multi-shot step instead of the headline workload")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res), flush=True)
        return
    if args.workload == "qtt512_64shots":
        if rank == 0:
            print(json.dumps(run_shots(args)), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    res, _keep = run_ours(args, rank, world, local_rank)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            res["cpu_baseline"] = oracle_baseline(args.cpu_seconds)
        else:
            res["cpu_baseline"] = None
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
