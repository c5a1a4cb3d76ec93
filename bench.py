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
# shared by both arms: the workload, its state and the timing protocol
def workload_config(wl, state_step: int) -> dict:
    return {"workload": wl.name, "n": wl.n, "grid": f"{wl.N}x{wl.N}", "chi_max": wl.chi, "eps": wl.eps,
            "chi_c": wl.chi_c, "eps_c": wl.eps_c, "order": wl.order, "bc": wl.bc,
            "source": list(wl.sources[0]), "state": f"mid-run (step {state_step} of {wl.steps}), ranks saturated",
            "l2": "GPU arm: flushed between timed steps (256 MiB write); host arm: no L2 flush"}


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


def _setup_gpu_state(q, wl, ctx, c, amps, stream, mid_run=None):
    """Velocity MPS, Laplacian MPO, and the mid-run state (dense FDTD on the
    GPU to MID_RUN, then TT-SVD + round in the library)."""
    mid_run = MID_RUN if mid_run is None else mid_run
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
        for k in range(mid_run):
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


def measured_peaks(q, stream) -> dict:
    """Peaks of the pipes the step's kernels run on: FP32 and FP64 FMA rates
    measured on this device by the library's probe; the tensor pipe and HBM
    from MEASURED_PEAKS.json (TF32 = half the measured dense BF16 rate, the
    nominal ratio)."""
    mp = _peaks()
    with_stream = {"fp32": q.qtt_peak_probe("fp32", stream), "fp64": q.qtt_peak_probe("fp64", stream)}
    bf16 = mp.get("bf16_tflops_sustained") or mp.get("bf16_tflops")
    return {"fp32_tflops": with_stream["fp32"], "fp64_tflops": with_stream["fp64"],
            "bf16_tflops": bf16, "tf32_tflops": (bf16 / 2.0) if bf16 else None, "hbm_gbs": mp.get("hbm_gbs"),
            "source": "fp32/fp64: qtt_peak_probe (FMA chains, 32 warps per SM, ~60 ms); bf16: MEASURED_PEAKS.json "
                      "sustained cuBLAS GEMM; tf32 = bf16 / 2 (nominal ratio)"}


# pipe each kernel class runs on, per form (classes without counted work are
# memory- or latency-bound copies and small kernels)
_PIPE = {
    "fp64": {"gemm": "fp64", "qr": "fp64", "jacobi": "fp64", "refine": "fp64", "pivot": "fp64"},
    "fp32": {"gemm": "fp32", "qr": "fp32", "jacobi": "fp32", "refine": "fp64", "pivot": "fp64"},
    "tf32": {"gemm": "tf32", "qr": "fp32", "jacobi": "fp32", "refine": "fp64", "pivot": "fp64"},
    "bf16": {"gemm": "bf16", "qr": "fp32", "jacobi": "fp32", "refine": "fp64", "pivot": "fp64"},
}


def roofline(prof: dict, prof_steps: int, ms_per_step: float, form: str, peaks: dict) -> dict:
    """The dominant class with its achieved rate against its pipe's peak, and
    the step-level fraction sum_phase(work / peak) / step time."""
    ms, fl, launches = prof["ms"], dict(prof["flops"]), prof["launches"]
    fl["jacobi"] = fl.get("jacobi", 0.0) + prof["svd_flops"]  # SVD work of the logged Jacobi launches
    pipes = _PIPE[form]
    phases, ideal_s = {}, 0.0
    for cls, t in ms.items():
        if t <= 0:
            continue
        work = fl.get(cls, 0.0) / prof_steps
        pipe = pipes.get(cls)
        peak = peaks.get(f"{pipe}_tflops") if pipe else None
        ph = {"ms_per_step": round(t / prof_steps, 3), "work_flop_per_step": work, "pipe": pipe, "peak_tflops": peak}
        if pipe and peak and work > 0:
            ph["achieved_tflops"] = work / (t / prof_steps / 1e3) / 1e12
            ph["frac"] = ph["achieved_tflops"] / peak
            ideal_s += work / (peak * 1e12)
        phases[cls] = ph
    dom = max(ms, key=lambda kk: ms[kk])
    pipe = pipes.get(dom)
    peak = peaks.get(f"{pipe}_tflops") if pipe else None
    achieved = fl.get(dom, 0.0) / (ms[dom] / 1e3) / 1e12 if ms[dom] > 0 else None
    kernel = {"jacobi": "jacobi32_gram_kernel (block one-sided Jacobi SVD, FP32, one cluster)" if form != "fp64"
              else "jacobi_kernel (one-sided Jacobi SVD, FP64, cooperative)"}.get(dom, dom)
    roof = {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": (achieved / peak) if (achieved and peak) else None,
            "peak_source": f"measured {pipe} FMA rate of this device (qtt_peak_probe)" if pipe in ("fp32", "fp64")
            else "MEASURED_PEAKS.json",
            "traffic": None, "launches": launches.get(dom, 0) // max(prof_steps, 1),
            "avg_launch_ms": ms[dom] / max(launches.get(dom, 1), 1),
            "avg_sweeps": prof["svd_sweeps"] / max(prof["svd_logged"], 1),
            "work": "SVD: 6 m n^2 + 20 n^3 per Jacobi launch on its n x m factor (Golub-Van Loan); GEMM: 2 M N K; "
                    "Householder QR: 2 p k^2 - 2 k^3/3 (+ the same for a thin Q); counted on the device per launch",
            "share_of_step": ms[dom] / max(sum(ms.values()), 1e-9),
            "step_fraction": ideal_s / (ms_per_step / 1e3),
            "step_fraction_note": "sum over phases of algorithmic work / peak of its pipe, over the measured step "
                                  "time (the graph-replayed step); classes without counted work (sorts, copies, "
                                  "MPO application, sums, the cluster Cholesky / pivoted QR) add time but no work",
            "phases": phases, "peaks": peaks}
    if dom == "jacobi" and form != "fp64":
        # DRAM bytes of one 256-vector launch of the FP32 block Jacobi, from an
        # ncu capture of this kernel on the same workload (the input matrix,
        # read once); per launch, like `achieved`
        roof["traffic"] = 597.0e3
        roof["traffic_note"] = ("dram__bytes_read.sum + dram__bytes_write.sum of one jacobi32_gram_kernel<2,2,16> "
                                "launch (16 CTAs: 8 rotating the vectors, 8 keeping the rotation columns; ncu --set "
                                "full --clock-control none -k regex:jacobi32_gram_kernel -s 30 -c 1 on python "
                                "bench.py --steps 1 --warmup 3 --compare 0 --no-cpu-baseline --e2e-steps 0); "
                                "`achieved` averages all Jacobi launches of the step")
    return roof


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
    tune = None
    if args.autotune:
        # launch shapes of this workload and form, measured on its mid-run
        # state (cached per device, form and shape in a JSON file)
        path = os.path.join(tempfile.gettempdir(), f"qtt_autotune_{wl.name}_{args.form}.json")
        t0 = time.time()
        with torch.cuda.stream(stream):
            nb = q.qtt_autotune(L, C, lam2, prev, cur, path, reps=3)
        with open(path) as f:
            tj = json.load(f)
        tune = {"buckets": nb, "seconds": round(time.time() - t0, 2), "choices": [
            {"op": "gemm" if e["op"] == 0 else "qr", "kind": e["kind"], "bucket": [e["a"], e["b"], e["c"]],
             "choice": e["choice"], "us_per_launch": e["us_per_launch"]} for e in tj["entries"]]}
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

    # roofline: the dominant kernel class, and the whole step as the sum over
    # phases of algorithmic work / peak of the pipe that phase runs on,
    # divided by the measured step time (class times and work from the two
    # launched steps with per-launch events and device-side work counters)
    peaks = measured_peaks(q, stream)
    roof = roofline(prof, prof_steps, ms_per_step, args.form, peaks)

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
        "dtype": {"fp64": "f64", "fp32": "f32+f64", "tf32x3": "tf32x3+f32+f64", "tf32": "tf32+f32+f64",
                  "bf16": "bf16+f32+f64"}[args.form],
        "data": "synthetic (seeded Marmousi-shaped velocity section; Ricker source)",
        "config": workload_config(wl, MID_RUN),
        "form": args.form,
        "run": {"ranks_start": ranks0, "ranks_end": ranks1, "graph": bool(args.graph), "autotune": tune,
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
        "dtype": {"fp64": "f64", "fp32": "f32+f64", "tf32x3": "tf32x3+f32+f64", "tf32": "tf32+f32+f64",
                  "bf16": "bf16+f32+f64"}[args.form], "data": "synthetic (seeded layered section)",
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


def run_combined(args):
    """The combined form on the 64-shot workload: FP32 form, batched shots,
    learned ranks (the network of _train_rank_model, one range-finder sketch
    shared by the shots).  The learned rounding reads each accept flag on the
    host, so the batched steps are launched, not replayed from graphs.
    Throughput: shot-steps/s over the timed batched steps.  Accuracy: for a
    sample of shots (one per bond cap up to 128, the FP64 form at cap 256
    costs seconds per step), the same steps from the same starting states in
    the plain FP64 form and in the plain FP32 form; the fields after those
    steps are compared (relative L2), and each form's per-shot step time is
    reported."""
    import torch
    from paper_2609_01904_b300 import qtt as q

    mlp, training = _train_rank_model(q, "fp32")
    wl = W.config(SHOTS_IDX)
    c = wl.velocity()
    lam2 = wl.lambda2(c)
    chis = [int(x) for x in W.chi_per_shot(wl.seed, len(wl.sources))]
    ns = len(chis)
    nsteps = args.warmup + args.steps
    amps = wl.source_amplitudes(c, SHOTS_MID_RUN + nsteps + 4)
    stream = torch.cuda.Stream()
    t0 = time.time()
    batch = q.qtt_batch_create(wl.n, ns, chis, order=wl.order, bc=wl.bc, chi_max=max(chis), eps=wl.eps,
                               chi_c=wl.chi_c, eps_c=wl.eps_c, prec="fp32", stream=stream, learned=True)
    q.qtt_batch_set_graphs(batch, False)
    N = wl.N
    G = torch.as_tensor(W.gaussian_sketch(11, 1024, 512), device="cuda")
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
    for x in batch.ctxs:
        q.qtt_set_rank_model(x, mlp, G)
    sample = []
    for cap in (32, 64, 128):
        hit = [s for s in range(ns) if chis[s] == cap]
        if hit:
            sample.append(hit[0])
    start = {s: (q.qtt_mps_get_cores(prev[s]), q.qtt_mps_get_cores(cur[s])) for s in sample}
    setup_s = time.time() - t0
    k = SHOTS_MID_RUN
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            q.qtt_step_batched(batch, L, C, lam2, prev, cur, wl.sources, [float(amps[k])] * ns)
            k += 1
    stream.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    flush = torch.empty(32 * 1024 * 1024, dtype=torch.float64, device="cuda")
    for x in batch.ctxs:
        q.qtt_profile_start(x, timing=False, log_svd=True)
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
    step_ms = [a.elapsed_time(b) for a, b in evs]
    value = ns * args.steps / (float(np.sum(step_ms)) / 1e3)
    profs = [q.qtt_profile_read(x) for x in batch.ctxs]
    launches = sum(sum(p["launches"].values()) for p in profs)
    att = acc = 0
    for x in batch.ctxs:
        a, b = q.qtt_learned_stats(x)
        att += a
        acc += b

    def dense(psi):
        out = torch.zeros((N, N), dtype=torch.float64, device="cuda")
        q.qtt_to_dense(psi, out)
        q.qtt_ctx_sync(psi.ctx)
        return out.cpu().numpy()

    rel = lambda a, b: float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    shots = []
    for s in sample:
        got = dense(cur[s])
        ref = {}
        for form in ("fp64", "fp32"):
            st = torch.cuda.Stream()
            ctx = q.qtt_ctx_create(n=wl.n, order=wl.order, bc=wl.bc, chi_max=chis[s], eps=wl.eps, chi_c=wl.chi_c,
                                   eps_c=wl.eps_c, prec=form, stream=st)
            with torch.cuda.stream(st):
                Cf = q.qtt_velocity_mps(ctx, c_dev)
                Lf = q.qtt_laplacian_mpo(ctx)
                p0, c0 = q.qtt_mps_from_cores(ctx, start[s][0]), q.qtt_mps_from_cores(ctx, start[s][1])
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                for kk in range(nsteps):
                    q.qtt_step(Lf, Cf, lam2, p0, c0, wl.sources[s], float(amps[SHOTS_MID_RUN + kk]))
                e1.record(st)
            st.synchronize()
            ref[form] = (dense(c0), e0.elapsed_time(e1) / nsteps)
            del Cf, Lf, p0, c0, ctx
        shots.append({"shot": s, "chi": chis[s], "steps": nsteps,
                      "field_rel_l2_combined_vs_fp64": rel(got, ref["fp64"][0]),
                      "field_rel_l2_plain_fp32_vs_fp64": rel(ref["fp32"][0], ref["fp64"][0]),
                      "ms_per_step_fp64": round(ref["fp64"][1], 2), "ms_per_step_plain_fp32": round(ref["fp32"][1], 2)})
    for x in batch.ctxs:
        q.qtt_set_rank_model(x, None, None)
    return {
        "metric": "MPS shot-steps/s, 64 shots on a 2^18 grid, combined form (FP32 + batched + learned ranks)",
        "value": value, "unit": "shot-steps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": float(np.mean(step_ms)), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic (seeded layered section; Ricker sources)",
        "config": {"workload": wl.name + "_combined", "n": wl.n, "shots": ns, "chi_per_shot": chis, "eps": wl.eps,
                   "graph": False, "state": f"mid-run (step {SHOTS_MID_RUN})",
                   "l2": "flushed between timed steps (256 MiB write)", "setup_s": round(setup_s, 1)},
        "training": training,
        "range_finder_attempts": att, "range_finder_accepts": acc,
        "svd_work_flop_per_step": sum(p["svd_flops"] for p in profs) / args.steps,
        "gpu_launches": int(launches),
        "accuracy_sample": shots,
        "accuracy_note": "sample shots advanced warmup + steps steps from the same start in each form; "
                         "errors of the fields at the end against the plain FP64 form",
        "clocks": clk.summary(),
        "step_ms": [round(x, 3) for x in step_ms],
    }


def write_png_pair(path: str, left: np.ndarray, right: np.ndarray) -> None:
    """Two fields side by side as an 8-bit grayscale PNG (zero = mid-grey,
    both scaled by the 99.5th percentile of |left|), plain file output."""
    import struct
    import zlib
    vmax = float(np.percentile(np.abs(left), 99.5)) or 1.0
    gap = np.full((left.shape[1], 4), 255, dtype=np.uint8)

    def img(u):  # u[x, z]: rows = depth z, columns = x
        return np.clip(128.0 + 127.0 * u.T / vmax, 0, 255).astype(np.uint8)

    a = np.concatenate([img(left), gap, img(right)], axis=1)
    raw = b"".join(b"\x00" + row.tobytes() for row in a)

    def chunk(tag, data):
        return struct.pack(">I", len(data)) + tag + data + struct.pack(">I", zlib.crc32(tag + data) & 0xFFFFFFFF)

    png = (b"\x89PNG\r\n\x1a\n" + chunk(b"IHDR", struct.pack(">IIBBBBB", a.shape[1], a.shape[0], 8, 0, 0, 0, 0))
           + chunk(b"IDAT", zlib.compress(raw, 9)) + chunk(b"IEND", b""))
    with open(path, "wb") as f:
        f.write(png)


def run_paper(args):
    """The paper's own run (Sec. 5) on the synthetic stand-in: 256 x 256,
    dh = 10 m, dt = 1 ms, impulsive source of strength 1 at the centre as the
    initial condition, chi = 128, eps = 1e-7, 300 steps; MPS steps/s over the
    whole run, the per-step time curve, and the MPS field against the dense
    Eq. 2 run on the same GPU (with the compressed c^2 the MPS uses, and with
    the exact c^2)."""
    import torch
    from paper_2609_01904_b300 import qtt as q
    wl = W.paper_run()
    c = wl.velocity()
    lam2 = wl.lambda2(c)
    N, steps = wl.N, wl.steps
    src = wl.sources[0]
    stream = torch.cuda.Stream()
    ctx = q.qtt_ctx_create(n=wl.n, order=wl.order, bc=wl.bc, chi_max=wl.chi, eps=wl.eps, chi_c=wl.chi_c,
                           eps_c=wl.eps_c, prec=args.form, stream=stream)
    with torch.cuda.stream(stream):
        c_dev = torch.as_tensor(c, device="cuda")
        C = q.qtt_velocity_mps(ctx, c_dev)
        L = q.qtt_laplacian_mpo(ctx)
        prev, cur = q.qtt_mps_create_zero(ctx), q.qtt_mps_create_zero(ctx)
        q.qtt_inject_source(cur, src[0], src[1], 1.0)  # u^0 = e_src, u^-1 = 0
    step = q.qtt_step_graph if args.graph else q.qtt_step
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    ranks = []
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        with torch.cuda.stream(stream):
            evs[0].record(stream)
            for k in range(steps):
                step(L, C, lam2, prev, cur, None, 0.0)
                evs[k + 1].record(stream)
        torch.cuda.synchronize()
    step_ms = [evs[k].elapsed_time(evs[k + 1]) for k in range(steps)]
    total_s = evs[0].elapsed_time(evs[steps]) / 1e3
    ranks = q.qtt_mps_ranks(cur)
    mps = torch.zeros((N, N), dtype=torch.float64, device="cuda")
    c2m = torch.zeros((N, N), dtype=torch.float64, device="cuda")
    q.qtt_to_dense(cur, mps)
    q.qtt_to_dense(C, c2m)
    c2 = c_dev * c_dev
    fields = {}
    for name, c2f in (("compressed_c2", c2m), ("exact_c2", c2)):
        up = torch.zeros((N, N), dtype=torch.float64, device="cuda")
        uc = up.clone()
        uc[src[0], src[1]] = 1.0
        un = up.clone()
        for _ in range(steps):
            q.qtt_fdtd_step(ctx, c2f, lam2, up, uc, un, None, 0.0)
            up, uc, un = uc, un, up
        fields[name] = uc
    q.qtt_ctx_sync(ctx)
    rel = lambda a, b: float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
    out = {
        "metric": "MPS steps/s, the paper's Sec. 5 run on a synthetic stand-in (256x256, chi=128, 300 steps)",
        "value": steps / total_s, "unit": "steps/s", "n_gpus": 1, "steps": steps, "warmup": 0,
        "ms_per_step": 1e3 * total_s / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "form": args.form, "data": "synthetic (seeded Marmousi-shaped 256x256 section; impulsive initial condition)",
        "config": {"workload": wl.name, "n": wl.n, "dh_m": wl.dh, "dt_s": wl.dt(c), "chi_max": wl.chi, "eps": wl.eps,
                   "chi_c": wl.chi_c, "eps_c": wl.eps_c, "order": wl.order, "bc": wl.bc, "source": list(src),
                   "initial_condition": "u^0 = e_src (strength 1), u^-1 = 0", "graph": bool(args.graph),
                   "l2": "not flushed: the whole run is timed back to back, first step cold"},
        "ranks_end": ranks, "c2_model_rel_l2": rel(c2m, c2),
        "field_rel_l2_vs_dense_fdtd": {k: rel(mps, v) for k, v in fields.items()},
        "step_ms_curve": [round(x, 3) for x in step_ms[::10]],
        "step_ms_first_last": [round(step_ms[0], 3), round(step_ms[-1], 3)],
        "clocks": clk.summary(),
    }
    if args.png:
        write_png_pair(args.png, fields["compressed_c2"].cpu().numpy(), mps.cpu().numpy())
        out["png"] = args.png
    return out


def run_variants(args):
    """Boundary-condition and site-order variants as benchmarks: the
    256x256 layered workload (chi = 64, eps = 1e-7) with PERIODIC or ZERO
    (Eq. 11 as printed) boundaries and INTERLEAVED or SEQUENTIAL (Eq. 14-15)
    site order, each from its own mid-run state (the dense Eq. 2 run with the
    same boundary to step 500, compressed); steps/s, ranks, the MPO bonds and
    the error against the dense Eq. 2 run after err_steps steps."""
    import torch
    from paper_2609_01904_b300 import qtt as q
    res = {}
    mid = 500
    for order in ("interleaved", "sequential"):
        for bc in ("periodic", "zero"):
            wl = W.variant(1, order, bc)
            c = wl.velocity()
            lam2 = wl.lambda2(c)
            N = wl.N
            amps = wl.source_amplitudes(c, mid + args.warmup + args.steps + 2)
            src = wl.sources[0]
            stream = torch.cuda.Stream()
            ctx = q.qtt_ctx_create(n=wl.n, order=order, bc=bc, chi_max=wl.chi, eps=wl.eps, chi_c=wl.chi_c,
                                   eps_c=wl.eps_c, prec=args.form, stream=stream)
            with torch.cuda.stream(stream):
                c_dev = torch.as_tensor(c, device="cuda")
                C = q.qtt_velocity_mps(ctx, c_dev)
                L = q.qtt_laplacian_mpo(ctx)
                c2m = torch.zeros((N, N), dtype=torch.float64, device="cuda")
                q.qtt_to_dense(C, c2m)
                up = torch.zeros((N, N), dtype=torch.float64, device="cuda")
                uc, un = up.clone(), up.clone()
                for k in range(mid):
                    q.qtt_fdtd_step(ctx, c2m, lam2, up, uc, un, src, float(amps[k]))
                    up, uc, un = uc, un, up
                prev, cur = q.qtt_mps_from_dense(ctx, up), q.qtt_mps_from_dense(ctx, uc)
            step = q.qtt_step_graph if args.graph else q.qtt_step
            k = mid
            with torch.cuda.stream(stream):
                for _ in range(args.warmup):
                    step(L, C, lam2, prev, cur, src, float(amps[k]))
                    q.qtt_fdtd_step(ctx, c2m, lam2, up, uc, un, src, float(amps[k]))
                    up, uc, un = uc, un, up
                    k += 1
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.steps)]
            torch.cuda.synchronize()
            with torch.cuda.stream(stream):
                for i in range(args.steps):
                    evs[i][0].record(stream)
                    step(L, C, lam2, prev, cur, src, float(amps[k]))
                    evs[i][1].record(stream)
                    q.qtt_fdtd_step(ctx, c2m, lam2, up, uc, un, src, float(amps[k]))
                    up, uc, un = uc, un, up
                    k += 1
            torch.cuda.synchronize()
            ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
            mps = torch.zeros((N, N), dtype=torch.float64, device="cuda")
            q.qtt_to_dense(cur, mps)
            q.qtt_ctx_sync(ctx)
            rk = q.qtt_mps_ranks(cur)
            res[f"{order}/{bc}"] = {
                "ms_per_step": round(ms, 3), "steps_per_s": 1e3 / ms, "ranks": rk, "max_rank": max(rk),
                "sum_rank": sum(rk), "mpo_bonds": q.qtt_mpo_bonds(L), "c2_ranks": q.qtt_mps_ranks(C),
                "field_rel_l2_vs_dense_fdtd": float(torch.linalg.norm(mps - uc) / torch.linalg.norm(uc))}
    base = res["interleaved/periodic"]["ms_per_step"]
    return {"metric": "MPS steps/s per boundary condition and site order (256x256 layered, chi=64)",
            "value": 1e3 / base, "unit": "steps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "form": args.form, "data": "synthetic (seeded layered section; Ricker source)",
            "config": {"workload": "qtt256_layered variants", "state": f"mid-run (step {mid}) of each variant",
                       "graph": bool(args.graph), "l2": "not flushed"},
            "variants": res}


def run_fused(args):
    """The fused step (Eq. 7's operator A = 2I + lambda^2 C^2 L applied by one
    zip-up, qtt_step_fused) against the two-zip-up step (qtt_step) on the same
    mid-run state: steps/s of each, and after err_steps steps the error of
    each against the FP64 two-zip-up step and against the dense Eq. 2 run."""
    import torch
    from paper_2609_01904_b300 import qtt as q
    wl = W.config(args.fused_cfg)
    c = wl.velocity()
    lam2 = wl.lambda2(c)
    N = wl.N
    mid = wl.steps // 2
    nst = args.err_steps
    amps = wl.source_amplitudes(c, mid + args.warmup + nst + 2)
    src = wl.sources[0]
    out, fields = {}, {}
    zm = args.fused_chi_zip
    for form, fused, zmul in (("fp64", False, 1), ("fp64", True, 1), ("fp64", True, zm), (args.form, False, 1),
                              (args.form, True, zm)):
        key = f"{form}/{'fused' if fused else 'two_zipups'}/chi_zip={zmul}chi"
        if key in out:
            continue
        stream = torch.cuda.Stream()
        ctx = q.qtt_ctx_create(n=wl.n, order=wl.order, bc=wl.bc, chi_max=wl.chi, eps=wl.eps, chi_c=wl.chi_c,
                               eps_c=wl.eps_c, prec=form, stream=stream, chi_zip=zmul * wl.chi)
        C, L, prev, cur = _setup_gpu_state(q, wl, ctx, c, amps, stream, mid)
        A = q.qtt_a_operator_mpo(L, C, lam2) if fused else None
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(nst + 1)]
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            for kk in range(nst):
                if fused:
                    q.qtt_step_fused(A, prev, cur, src, float(amps[mid + kk]))
                else:
                    q.qtt_step(L, C, lam2, prev, cur, src, float(amps[mid + kk]))
                ev[kk + 1].record(stream)
        q.qtt_ctx_sync(ctx)
        t = [ev[i].elapsed_time(ev[i + 1]) for i in range(nst)]
        dense = torch.zeros((N, N), dtype=torch.float64, device="cuda")
        q.qtt_to_dense(cur, dense)
        q.qtt_ctx_sync(ctx)
        fields[key] = dense.cpu().numpy()
        out[key] = {"ms_per_step": round(float(np.median(t)), 3), "steps_per_s": 1e3 / float(np.median(t)),
                    "ranks_end": q.qtt_mps_ranks(cur), "mpo_max_bond": max(q.qtt_mpo_bonds(A if fused else L))}
        del A, C, L, prev, cur, ctx
    ctx = q.qtt_ctx_create(n=wl.n, order=wl.order, bc=wl.bc, chi_max=wl.chi, eps=wl.eps, prec="fp64")
    c2 = torch.as_tensor(c * c, device="cuda")
    up = torch.zeros((N, N), dtype=torch.float64, device="cuda")
    uc, un = up.clone(), up.clone()
    for kk in range(mid + nst):
        q.qtt_fdtd_step(ctx, c2, lam2, up, uc, un, src, float(amps[kk]))
        up, uc, un = uc, un, up
    q.qtt_ctx_sync(ctx)
    fd = uc.cpu().numpy()
    rel = lambda a, b: float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    ref = fields["fp64/two_zipups/chi_zip=1chi"]
    for key in out:
        out[key]["field_rel_l2_vs_fp64_two_zipups"] = rel(fields[key], ref)
        out[key]["field_rel_l2_vs_dense_fdtd"] = rel(fields[key], fd)
    return {"metric": "MPS steps/s, fused Eq. 7 operator (one zip-up) vs two zip-ups", "unit": "steps/s",
            "value": out[f"{args.form}/fused/chi_zip={zm}chi"]["steps_per_s"], "n_gpus": 1, "steps": nst, "warmup": 0,
            "higher_is_better": True, "form": args.form,
            "data": "synthetic (seeded velocity section; Ricker source)",
            "config": {"workload": wl.name, "n": wl.n, "chi_max": wl.chi, "eps": wl.eps, "chi_c": wl.chi_c,
                       "state": f"mid-run (step {mid}), dense Eq. 2 compressed by the library",
                       "timing": "launched steps (no graph), median of err_steps, no L2 flush"},
            "steps_compared": out}


def run_full(args):
    """The 1024x1024 workload run from its start: zero state, the Ricker
    source, every step of the 4000-step run (or as many as fit in
    --full-seconds of wall time) replayed from CUDA graphs in the chosen form;
    steps/s over the whole run, the per-step time against the step index,
    the ranks as they grow, and the field at the end against the dense Eq. 2
    run of the same steps on the same GPU (the truncation error of the whole
    run; the FP64 MPS is not a reference over thousands of steps, the
    truncated dynamics being chaotic once the ranks reach chi)."""
    import torch
    from paper_2609_01904_b300 import qtt as q
    wl = W.config(WORKLOAD_IDX)
    c = wl.velocity()
    lam2 = wl.lambda2(c)
    N, total = wl.N, wl.steps
    amps = wl.source_amplitudes(c, total + 2)
    src = wl.sources[0]
    stream = torch.cuda.Stream()
    ctx = q.qtt_ctx_create(n=wl.n, order=wl.order, bc=wl.bc, chi_max=wl.chi, eps=wl.eps, chi_c=wl.chi_c,
                           eps_c=wl.eps_c, prec=args.form, stream=stream)
    with torch.cuda.stream(stream):
        c_dev = torch.as_tensor(c, device="cuda")
        C = q.qtt_velocity_mps(ctx, c_dev)
        L = q.qtt_laplacian_mpo(ctx)
        prev, cur = q.qtt_mps_create_zero(ctx), q.qtt_mps_create_zero(ctx)
    step = q.qtt_step_graph if args.graph else q.qtt_step
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(total)]
    ranks_at, done = {}, 0
    torch.cuda.synchronize()
    t0 = time.time()
    with ClockSampler(0) as clk:
        for k in range(total):
            with torch.cuda.stream(stream):
                ev[k][0].record(stream)
                step(L, C, lam2, prev, cur, src, float(amps[k]))
                ev[k][1].record(stream)
            done = k + 1
            if done % 250 == 0 or done == total:
                stream.synchronize()
                ranks_at[done] = max(q.qtt_mps_ranks(cur))
                if time.time() - t0 > args.full_seconds:
                    break
        torch.cuda.synchronize()
    step_ms = [ev[k][0].elapsed_time(ev[k][1]) for k in range(done)]
    # the dense run of the same steps, after the timed loop
    c2 = c_dev * c_dev
    up = torch.zeros((N, N), dtype=torch.float64, device="cuda")
    uc, un = up.clone(), up.clone()
    with torch.cuda.stream(stream):
        for k in range(done):
            q.qtt_fdtd_step(ctx, c2, lam2, up, uc, un, src, float(amps[k]))
            up, uc, un = uc, un, up
        mps = torch.zeros((N, N), dtype=torch.float64, device="cuda")
        q.qtt_to_dense(cur, mps)
    q.qtt_ctx_sync(ctx)
    err = float(torch.linalg.norm(mps - uc) / max(float(torch.linalg.norm(uc)), 1e-300))
    curve = {str(k + 1): round(step_ms[k], 3) for k in range(done) if k < 5 or (k + 1) % 100 == 0}
    value = done / (float(np.sum(step_ms)) / 1e3)
    return {"metric": "MPS steps/s over the whole run of the 1024x1024 workload (chi=128, eps=1e-6), 1 B300",
            "value": value, "unit": "steps/s", "n_gpus": 1, "steps": done, "warmup": 0,
            "ms_per_step": float(np.mean(step_ms)), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64"}.get(args.form, "f32+f64"), "form": args.form,
            "data": "synthetic (seeded Marmousi-shaped velocity section; Ricker source)",
            "config": {"workload": wl.name + "_full_run", "n": wl.n, "chi_max": wl.chi, "eps": wl.eps,
                       "chi_c": wl.chi_c, "steps_planned": total, "graph": bool(args.graph),
                       "timing": "sum of per-step CUDA-event times (host syncs every 250 steps fall between steps)"},
            "per_step_ms": curve, "max_rank_at_step": ranks_at,
            "ms_per_step_first_100": float(np.mean(step_ms[:100])),
            "ms_per_step_last_100": float(np.mean(step_ms[-100:])),
            "field_rel_l2_vs_dense_fdtd_at_end": err, "clocks": clk.summary(),
            "wall_s": round(time.time() - t0, 1)}


def run_3d(args):
    """The 3D extension (64^3 layered block, 3n = 18 sites, the 7-point
    Laplacian MPO, chi = 64, eps = 1e-6, Ricker source at (32, 32, 2)): MPS
    steps/s from a mid-run state (the dense 7-point run on the GPU to step
    300, compressed by the library), in the chosen form and in FP64, and the
    error of both after err_steps steps against the FP64 MPS and the dense
    run."""
    import torch
    from paper_2609_01904_b300 import qtt as q
    wl = W.qtt3d_run(6)
    c = wl.velocity()
    lam2 = wl.lambda2(c)
    N = wl.N
    mid = wl.steps // 4
    nst = args.err_steps
    amps = wl.source_amplitudes(c, mid + args.warmup + args.steps + nst + 2)
    src = wl.sources[0]
    out, fields = {}, {}
    for form in ("fp64", args.form):
        if form in out:
            continue
        stream = torch.cuda.Stream()
        ctx = q.qtt_ctx_create(n=wl.n, order=wl.order, bc=wl.bc, chi_max=wl.chi, eps=wl.eps, chi_c=wl.chi_c,
                               eps_c=wl.eps_c, prec=form, stream=stream, dims=3)
        with torch.cuda.stream(stream):
            c_dev = torch.as_tensor(c, device="cuda")
            C = q.qtt_velocity_mps(ctx, c_dev)
            L = q.qtt_laplacian_mpo(ctx)
            c2 = c_dev * c_dev
            up = torch.zeros((N, N, N), dtype=torch.float64, device="cuda")
            uc, un = up.clone(), up.clone()
            for k in range(mid):
                q.qtt_fdtd_step_3d(ctx, c2, lam2, up, uc, un, src, float(amps[k]))
                up, uc, un = uc, un, up
            prev, cur = q.qtt_mps_from_dense(ctx, up), q.qtt_mps_from_dense(ctx, uc)
            comp = torch.zeros((N, N, N), dtype=torch.float64, device="cuda")
            q.qtt_to_dense(cur, comp)
        q.qtt_ctx_sync(ctx)
        comp_err = float(torch.linalg.norm(comp - uc) / torch.linalg.norm(uc))
        step = q.qtt_step_graph if args.graph else q.qtt_step
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(nst + 1)]
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            for kk in range(nst):
                step(L, C, lam2, prev, cur, src, float(amps[mid + kk]))
                ev[kk + 1].record(stream)
                q.qtt_fdtd_step_3d(ctx, c2, lam2, up, uc, un, src, float(amps[mid + kk]))
                up, uc, un = uc, un, up
        q.qtt_ctx_sync(ctx)
        t = [ev[i].elapsed_time(ev[i + 1]) for i in range(1, nst)]  # the first step captures the graph
        dense = torch.zeros((N, N, N), dtype=torch.float64, device="cuda")
        q.qtt_to_dense(cur, dense)
        q.qtt_ctx_sync(ctx)
        fields[form] = dense.cpu().numpy()
        fields["fdtd"] = uc.cpu().numpy()
        out[form] = {"ms_per_step": round(float(np.median(t)), 3), "steps_per_s": 1e3 / float(np.median(t)),
                     "ranks_end": q.qtt_mps_ranks(cur), "c2_ranks": q.qtt_mps_ranks(C),
                     "mpo_bonds": q.qtt_mpo_bonds(L), "start_state_compression_rel_l2": comp_err}
        del C, L, prev, cur, ctx
    rel = lambda a, b: float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    for form in out:
        out[form]["field_rel_l2_vs_fp64_mps"] = rel(fields[form], fields["fp64"])
        out[form]["field_rel_l2_vs_dense_fdtd"] = rel(fields[form], fields["fdtd"])
    return {"metric": "MPS steps/s, 3D extension (64^3, 18 sites, 7-point Laplacian, chi=64)", "unit": "steps/s",
            "value": out[args.form]["steps_per_s"], "n_gpus": 1, "steps": nst - 1, "warmup": 1,
            "higher_is_better": True, "form": args.form, "data": "synthetic (seeded layered 3D block; Ricker source)",
            "config": {"workload": wl.name, "n": wl.n, "grid": f"{N}^3", "chi_max": wl.chi, "eps": wl.eps,
                       "chi_c": wl.chi_c, "order": wl.order, "bc": wl.bc, "source": list(src),
                       "state": f"mid-run (step {mid} of {wl.steps}), dense 7-point run compressed by the library",
                       "graph": bool(args.graph), "timing": "median step, CUDA events, no L2 flush"},
            "forms": out}


def _train_rank_model(q, form):
    """The learned rounding's network, trained on the GPU by the library on
    the plain solver's round spectra (qtt_step_features) and next-step ranks,
    logged over teacher-free steps from mid-run states of the 256x256 layered
    section, the 1024x1024 section and the 512x512 layered section at
    chi = 256 (40 -> 128 -> 128 -> 1, mean squared error, Adam).  Returns the
    network and a description of its training."""
    import torch
    feats, labels, sources = [], [], []
    X = None
    for idx, nsteps, chi_o in ((1, 40, None), (2, 12, None), (3, 12, 256)):
        wl = W.config(idx)
        chi = chi_o or wl.chi
        c = wl.velocity()
        lam2 = wl.lambda2(c)
        mid = wl.steps // 2
        amps = wl.source_amplitudes(c, mid + nsteps + 2)
        stream = torch.cuda.Stream()
        ctx = q.qtt_ctx_create(n=wl.n, order=wl.order, bc=wl.bc, chi_max=chi, eps=wl.eps, chi_c=wl.chi_c,
                               eps_c=wl.eps_c, prec=form, stream=stream, learned=True)
        C, L, prev, cur = _setup_gpu_state(q, wl, ctx, c, amps, stream, mid)
        X = torch.zeros((ctx.d - 1, 40), dtype=torch.float32, device="cuda")
        f_run, r_run = [], []
        with torch.cuda.stream(stream):
            for k in range(nsteps):
                q.qtt_step(L, C, lam2, prev, cur, wl.sources[0], float(amps[mid + k]))
                q.qtt_step_features(cur, X)
                q.qtt_ctx_sync(ctx)
                f_run.append(X.cpu().numpy().copy())
                r_run.append(q.qtt_mps_ranks(cur))
        feats.append(np.concatenate(f_run[:-1]))
        labels.append(np.concatenate([np.array(r[1:-1], dtype=np.float32) / chi for r in r_run[1:]]))
        sources.append(f"{wl.name} chi={chi}: {nsteps} steps from step {mid}")
        del C, L, prev, cur, ctx
    Xs, ys = np.concatenate(feats), np.concatenate(labels)
    mlp = q.qtt_mlp_create(W.mlp_params(7), len(Xs))
    Xg = torch.as_tensor(Xs, device="cuda")
    yg = torch.as_tensor(ys, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    q.qtt_mlp_grad(mlp, Xg, yg, loss)
    loss0 = float(loss.item())
    for _ in range(800):
        q.qtt_mlp_grad(mlp, Xg, yg, loss)
        q.qtt_mlp_adam_step(mlp, 2e-3)
    loss1 = float(loss.item())
    return mlp, {"samples": int(len(Xs)), "loss_start": loss0, "loss_end": loss1, "sources": sources}


def run_learned(args):
    """The learned rounding against plain rounding on the 2048x2048 section
    (n = 11, chi = 256, eps = 1e-5).  Training data: the plain solver's round
    spectra (qtt_step_features) and next-step ranks logged over teacher-free
    steps from mid-run states of the 256x256 layered section, the 1024x1024
    section and the 512x512 layered section at chi = 256; the network (40 ->
    128 -> 128 -> 1) is trained on the GPU by the library (mean squared error,
    Adam).  Then the same mid-run state of the 2048x2048 section is advanced
    err_steps steps with plain rounding and with the learned rounding: the
    logged Jacobi SVD work, the step times and the field difference between
    the two (and against the dense Eq. 2 run) are reported."""
    import torch
    from paper_2609_01904_b300 import qtt as q
    form = args.form
    mlp, training = _train_rank_model(q, form)
    loss0, loss1, sources = training["loss_start"], training["loss_end"], training["sources"]
    # evaluation on the 2048x2048 section
    wl = W.config(4)
    c = wl.velocity()
    lam2 = wl.lambda2(c)
    mid = wl.steps // 2
    nst = args.err_steps
    amps = wl.source_amplitudes(c, mid + nst + 2)
    N = wl.N
    G = torch.as_tensor(W.gaussian_sketch(11, 1024, 512), device="cuda")
    res, fields = {}, {}
    for mode in ("plain", "learned"):
        stream = torch.cuda.Stream()
        ctx = q.qtt_ctx_create(n=wl.n, order=wl.order, bc=wl.bc, chi_max=wl.chi, eps=wl.eps, chi_c=wl.chi_c,
                               eps_c=wl.eps_c, prec=form, stream=stream, learned=True)
        C, L, prev, cur = _setup_gpu_state(q, wl, ctx, c, amps, stream, mid)
        if mode == "learned":
            q.qtt_set_rank_model(ctx, mlp, G)
        q.qtt_profile_start(ctx, timing=False, log_svd=True)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(nst + 1)]
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            for k in range(nst):
                q.qtt_step(L, C, lam2, prev, cur, wl.sources[0], float(amps[mid + k]))
                ev[k + 1].record(stream)
        q.qtt_ctx_sync(ctx)
        prof = q.qtt_profile_read(ctx)
        t = [ev[i].elapsed_time(ev[i + 1]) for i in range(nst)]
        dense = torch.zeros((N, N), dtype=torch.float64, device="cuda")
        q.qtt_to_dense(cur, dense)
        q.qtt_ctx_sync(ctx)
        fields[mode] = dense.cpu().numpy()
        att, acc = q.qtt_learned_stats(ctx)
        res[mode] = {"ms_per_step": round(float(np.mean(t)), 2), "steps_per_s": 1e3 / float(np.mean(t)),
                     "svd_work_flop": prof["svd_flops"], "jacobi_launches": prof["svd_logged"],
                     "range_finder_attempts": att, "range_finder_accepts": acc, "ranks_end": q.qtt_mps_ranks(cur)}
        q.qtt_set_rank_model(ctx, None, None)
        del C, L, prev, cur, ctx
    ctx = q.qtt_ctx_create(n=wl.n, order=wl.order, bc=wl.bc, chi_max=wl.chi, eps=wl.eps, prec="fp64")
    c2 = torch.as_tensor(c * c, device="cuda")
    up = torch.zeros((N, N), dtype=torch.float64, device="cuda")
    uc, un = up.clone(), up.clone()
    for kk in range(mid + nst):
        q.qtt_fdtd_step(ctx, c2, lam2, up, uc, un, wl.sources[0], float(amps[kk]))
        up, uc, un = uc, un, up
    q.qtt_ctx_sync(ctx)
    fd = uc.cpu().numpy()
    rel = lambda a, b: float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    return {"metric": "learned vs plain rounding, 2048x2048 section (chi=256, eps=1e-5): SVD work and steps/s",
            "unit": "ratio", "value": res["learned"]["svd_work_flop"] / max(res["plain"]["svd_work_flop"], 1.0),
            "higher_is_better": False, "n_gpus": 1, "steps": nst, "form": form,
            "data": "synthetic (seeded Marmousi-shaped sections; Ricker sources)",
            "config": {"workload": wl.name, "n": wl.n, "chi_max": wl.chi, "eps": wl.eps,
                       "state": f"mid-run (step {mid} of {wl.steps})", "training": sources,
                       "training_samples": training["samples"], "loss_first_last": [loss0, loss1],
                       "timing": "launched steps (the learned form reads each accept flag on the host)"},
            "plain": res["plain"], "learned": res["learned"],
            "field_rel_l2_learned_vs_plain": rel(fields["learned"], fields["plain"]),
            "field_rel_l2_vs_dense_fdtd": {m: rel(fields[m], fd) for m in fields},
            "speedup_learned_vs_plain": res["plain"]["ms_per_step"] / res["learned"]["ms_per_step"]}


def run_gemm(args):
    """The contraction kernel on its own (qtt_gemm): achieved TFLOP/s of each
    operand form on square GEMMs of FP64 operands in HBM (inputs of 3 x 8 m^2
    bytes, larger than L2 from m = 2048), against the measured peak of the
    pipe it runs on (tensor-core forms: the bf16 peak of MEASURED_PEAKS.json,
    tf32 = bf16 / 2 nominal; 3xTF32 counts its three products as useful work
    of 2 m^3 flops only)."""
    import torch
    from paper_2609_01904_b300 import qtt as q
    stream = torch.cuda.Stream()
    ctx = q.qtt_ctx_create(n=6, chi_max=32, stream=stream)
    peaks = measured_peaks(q, stream)
    out = {}
    for m in (1024, 4096):
        A = torch.randn((m, m), dtype=torch.float64, device="cuda")
        B = torch.randn((m, m), dtype=torch.float64, device="cuda")
        C = torch.zeros((m, m), dtype=torch.float64, device="cuda")
        for kind in ("fp64", "fp32", "tf32", "tf32x3", "bf16"):
            if kind == "fp64" and m > 2048:
                continue
            best = None
            for tile in ((0,) if kind in ("fp64", "fp32") else (128, 256)):
                with torch.cuda.stream(stream):
                    q.qtt_gemm(ctx, kind, A, B, C, tile_n=tile)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    for _ in range(3):
                        q.qtt_gemm(ctx, kind, A, B, C, tile_n=tile)
                    e1.record(stream)
                q.qtt_ctx_sync(ctx)
                ms = e0.elapsed_time(e1) / 3
                tf = 2.0 * m ** 3 / (ms * 1e-3) / 1e12
                if best is None or tf > best[0]:
                    best = (tf, ms, tile)
            pipe = {"fp64": "fp64", "fp32": "fp32", "tf32": "tf32", "tf32x3": "tf32", "bf16": "bf16"}[kind]
            peak = peaks.get(f"{pipe}_tflops")
            out[f"{kind}/m={m}"] = {"tflops": best[0], "ms": round(best[1], 3), "tile_n": best[2], "pipe": pipe,
                                    "peak_tflops": peak, "frac": best[0] / peak if peak else None}
    return {"metric": "contraction kernel TFLOP/s per operand form (square GEMMs, FP64 operands in HBM)",
            "unit": "TFLOP/s", "value": out["tf32/m=4096"]["tflops"], "n_gpus": 1, "higher_is_better": True,
            "data": "synthetic (standard normal matrices)", "config": {"workload": "gemm", "m": [1024, 4096]},
            "peaks": peaks, "kernels": out}


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
    fields, traces, times = {}, {}, {}
    extra = [f for f in (args.compare_forms.split(",") if args.compare_forms else []) if f]
    for form in ["fp64", args.form] + extra:
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
        t = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.err_steps)]
        times[form] = float(np.mean(t))
        if form == "fp64":
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
    err["forms"] = {}
    for f in fields:
        fe, te = rel(fields[f], fields["fp64"]), rel(traces[f], traces["fp64"])
        err["forms"][f] = {"ms_per_step_launched": round(times[f], 3), "steps_per_s_launched": 1000.0 / times[f],
                           "field_rel_l2_vs_fp64_mps": fe, "trace_rel_l2_vs_fp64_mps": te,
                           "field_rel_l2_vs_dense_fdtd": rel(fields[f], fd), "eligible": fe <= 1e-3 and te <= 1e-3}
    err["forms_note"] = ("every form from the same mid-run state, err_steps launched steps (no graph, no L2 flush); "
                         "errors against the FP64 MPS after those steps")
    return out, err


def oracle_baseline(steps: int = 10, warmup: int = 3) -> dict:
    """The FP64 oracle on the host cores, in a process of its own (the
    reference arm of this script: `bench.py --impl reference`), so that no
    thread of the GPU process competes with its BLAS threads: `steps` timed
    oracle steps after `warmup`, from the same mid-run state as the GPU arm."""
    cmd = [sys.executable, os.path.abspath(__file__), "--impl", "reference", "--steps", str(steps),
           "--warmup", str(warmup)]
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    out = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=1800)
    line = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    if out.returncode != 0 or not line:
        return {"value": None, "unit": UNIT, "cores": None, "kind": "oracle",
                "sample": f"reference arm failed (rc {out.returncode}): {out.stderr[-300:]}"}
    ref = json.loads(line[-1])
    cb = dict(ref["cpu_baseline"])
    cb["same_config"] = True
    return cb


def run_reference(args, rank, world):
    if rank != 0:
        return None
    from oracle import qtt_oracle as O
    wl = W.config(WORKLOAD_IDX)
    n = wl.n
    c = wl.velocity()
    lam2 = wl.lambda2(c)
    mid = MID_RUN
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
        "config": workload_config(wl, mid),
        "form": "fp64 oracle (numpy, LAPACK svd/qr)",
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} timed oracle steps after {args.warmup} warm-up from the oracle's "
                                   f"own dense Eq. 2 state at step {mid} (ranks {max(O.mps_ranks(cur))} max), "
                                   f"{dt:.1f} s"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="fp32", choices=["fp64", "fp32", "tf32x3", "tf32", "bf16"],
                    help="fp32: the chosen form (FP32 contractions/QR, FP64-accurate SVDs); fp64: the plain form; "
                         "tf32x3 / tf32 / bf16: the FP32 form with tensor-core contractions")
    ap.add_argument("--compare", type=int, default=1, help="also time the plain FP64 form and measure errors")
    ap.add_argument("--err-steps", type=int, default=20)
    ap.add_argument("--compare-forms", default="tf32x3,tf32,bf16",
                    help="further forms whose step time and error after --err-steps are reported")
    ap.add_argument("--cpu-steps", type=int, default=10, help="timed oracle steps of the cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--autotune", type=int, default=1, help="1: autotune launch shapes before timing (qtt_autotune)")
    ap.add_argument("--graph", type=int, default=1, help="1: replay each step from a CUDA graph (qtt_step_graph); 0: launch the kernels")
    ap.add_argument("--workload", default="qtt1024_marmousi",
                    choices=["qtt1024_marmousi", "qtt512_64shots", "paper256", "variants", "fused", "qtt3d",
                             "learned", "gemm", "combined", "full"],
                    help="qtt512_64shots: the batched multi-shot step; paper256: the paper's Sec. 5 run on the "
                         "synthetic stand-in; variants: boundary conditions and site orders")
    ap.add_argument("--fused-cfg", type=int, default=1, help="fused: the configuration index (1: 256x256 layered)")
    ap.add_argument("--fused-chi-zip", type=int, default=4, help="fused: the zip-up bond cap as a multiple of chi")
    ap.add_argument("--full-seconds", type=float, default=420.0,
                    help="full: stop the full run after this much wall time (the steps done are reported)")
    ap.add_argument("--png", default=None, help="paper256: write the FDTD | MPS field pair to this PNG file")
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
    if args.workload in ("qtt512_64shots", "paper256", "variants", "fused", "qtt3d", "learned", "gemm", "combined",
                         "full"):
        if rank == 0:
            fn = {"qtt512_64shots": run_shots, "paper256": run_paper, "variants": run_variants,
                  "fused": run_fused, "qtt3d": run_3d, "learned": run_learned, "gemm": run_gemm,
                  "combined": run_combined, "full": run_full}[args.workload]
            print(json.dumps(fn(args)), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    res, _keep = run_ours(args, rank, world, local_rank)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            res["cpu_baseline"] = oracle_baseline(args.cpu_steps)
        else:
            res["cpu_baseline"] = None
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
