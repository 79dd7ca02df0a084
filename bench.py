#!/usr/bin/env python
"""Throughput benchmark of the FP64 cyclic-reduction solver on GB300.

One step = crsolve_factor + crsolve_solve of one synthetic Hermitian positive
definite block-tridiagonal system: N = 2^20 blocks, m = 8, k = 4, complex128,
generated by synthetic.gen_system (seed 1000).  The metric is block-rows/s =
N / (factor + solve time), inputs resident in HBM (A alone is 1 GiB, far
larger than the 126 MB L2, so no L2 flush is needed between steps).

Prints one JSON line (rank 0).  Extra keys:
  roofline      the dominant kernel (k_factor_odd, all levels) against the FP64
                pipe: algorithmic flops / CUDA-event time of its launches
  e2e           the same metric through crsolve_solve_host (pinned host
                buffers, H2D + factor + solve + D2H inside the timed region)
  cpu_baseline  the CPU oracle on the host cores on a bounded sample
  clocks        nvidia-smi samples taken during the timed region

  extra         (one GPU, rank 0; --no-extras skips it) the other forms on the
                same GPU in the same run, each with its speedup and its error
                against the CPU oracle: batched (4096 uneven systems in one
                persistent launch vs the plain path called per system), mixed
                (FP32 levels + FP64 refinement vs the FP64 path at kappa
                1e2/1e4/1e6) and adjoint (factor + solve + crsolve_backward)

--workload selects another form as the main line: batched, adjoint, mixed or
alg1 (the paper's Algorithm 1 on the plain workload's system, with classic
reduction timed beside it).  --impl reference times the CPU oracle alone on
the plain workload's full system (the reference arm).
Under torchrun (N > 1) every rank solves its own independent system (weak
scaling; the only collectives are the timing barrier and max).
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

import synthetic  # noqa: E402

N_BLOCKS, M, K_RHS = 1 << 20, 8, 4
SEED = 1000
WORKLOAD = f"plain CR, one HPD block-tridiagonal system: N=2^20 blocks, m={M}, k={K_RHS}, complex128"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# GB300: 2 FP64 FMA per clock per SM (measured by a DFMA throughput probe at
# ~1.9 DFMA/clk/SM), 152 SMs, 2070 MHz maximum SM clock
FP64_FMA_PER_CLK_SM, N_SM, SM_MAX_MHZ = 2, 152, 2070.0
FP64_PEAK_GFLOPS = FP64_FMA_PER_CLK_SM * 2 * N_SM * SM_MAX_MHZ / 1e3
# DRAM traffic of the dominant kernel from one ncu capture (dram__bytes_read.sum
# + dram__bytes_write.sum of k_factor_odd<8, double>, level 0 of N = 2^18, 2^17
# odd blocks: 537,975,296 + 624,427,776 bytes), valid only while the sources
# of the kernel's device code are the ones captured (their SHA-256 below).
# Otherwise the line reports null.
TRAFFIC_CAPTURE = {"bytes_per_odd_block": (537975296 + 624427776) / (1 << 17),
                   "sources": ("paper_1807_00370_gb300/csrc/cr_core.cuh", "paper_1807_00370_gb300/csrc/cr_device.cuh"),
                   "sha256": "0bd90a121a9eef595ab08f3a2c51afd23043dea0d0daca35ce1979fa79ddd871"}


def captured_traffic_per_odd_block():
    """The captured bytes per odd block if the kernel sources still hash to the
    captured ones, else None."""
    import hashlib
    if not TRAFFIC_CAPTURE["sha256"]:
        return None
    h = hashlib.sha256()
    for rel in TRAFFIC_CAPTURE["sources"]:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return TRAFFIC_CAPTURE["bytes_per_odd_block"] if h.hexdigest() == TRAFFIC_CAPTURE["sha256"] else None


def host_link(dev, pinned):
    """Bandwidth of the host link for the e2e number: a pinned host tensor
    copied to the device and back (CUDA events), and the CPUs the process
    may run on against the GPU's local CPUs (a far NUMA node slows pinned
    copies)."""
    import torch
    out = {}
    d = torch.empty(pinned.shape, dtype=pinned.dtype, device=dev)
    for name, src, dst in (("h2d_gbs", pinned, d), ("d2h_gbs", d, pinned)):
        dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            dst.copy_(src, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        out[name] = 3 * pinned.numel() * pinned.element_size() / (e0.elapsed_time(e1) * 1e-3) / 1e9
    del d
    try:
        out["process_cpus"] = len(os.sched_getaffinity(0))
    except Exception:  # noqa: BLE001
        pass
    return out


def fp64_probe():
    """Measured FP64 FMA rate of this GPU (crsolve_peak_probe): TFLOP/s, FMA
    lanes per SM per clock, and the SM clock the probe ran at."""
    import paper_1807_00370_gb300 as crs
    try:
        r = crs.crsolve_peak_probe("fp64")
    except Exception as e:  # noqa: BLE001 - reported, not fatal
        return {"failed": str(e)}
    return {"tflops": r["gflops"] / 1e3, "fma_per_clk_sm": r["fma_per_clk_sm"], "sm_mhz": r["sm_mhz"],
            "tflops_at_max_clock": 2.0 * r["fma_per_clk_sm"] * N_SM * SM_MAX_MHZ / 1e6}


def flops_factor_per_odd_block(m: int) -> float:
    """Algorithmic flops of one odd block in the factor sweep (complex, 8 real
    flops per multiply-add): Cholesky m^3/6, L^{-1}[B|B^H] m^3, lower triangle
    of the 2m x 2m product Z^H Z 2m^3 (leading order)."""
    return 8.0 * (m ** 3 / 6.0 + m ** 3 + 2.0 * m ** 3)


def flops_solve_per_odd_block(m: int, k: int) -> float:
    """Forward solve m^2 k/2, Z^H r 2 m^2 k, Z x 2 m^2 k, backward solve m^2 k/2."""
    return 8.0 * 5.0 * m * m * k


def flops_per_block_row(m: int, k: int) -> float:
    # every block row is an odd block at exactly one level
    return flops_factor_per_odd_block(m) + flops_solve_per_odd_block(m, k)


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.rows, self.proc, self.t0, self.t1 = index, [], None, None, None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), line.strip()))

    def mark(self, begin: bool):
        if begin:
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait(timeout=5)
        self.thread.join(timeout=2)
        sms, maxs, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, line in self.rows:
            if self.t0 is not None and not (self.t0 - 0.2 <= ts <= (self.t1 or ts) + 0.2):
                continue
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                maxs.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sms) if sms else None,
                "sm_max_mhz": max(maxs) if maxs else None,
                "reasons": sorted(reasons), "samples": len(sms)}


def kernel_breakdown(crs, plan, step, steps: int, stream):
    """Per-kernel CUDA-event times over `steps` more steps, with an event pair
    around every launch of the plan.  The pairs cost about 2 us per launch
    (0.6 ms of a 21 ms adjoint step), so the step time itself comes from a
    run without them; this run gives the kernels' shares and durations.
    Returns the records [(kind, level, units, ms)] and this run's step time."""
    import torch
    crs.crsolve_timing_enable(plan, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    recs = crs.crsolve_timing_read(plan)
    crs.crsolve_timing_enable(plan, False)
    return recs, e0.elapsed_time(e1) / steps


def reduce_over_ranks(ms: float, units: int, device="cpu"):
    """Max of the timed region and sum of the units over all ranks (the job's
    clock is the slowest rank; the job's work is everyone's).  Works with any
    torch.distributed backend (nccl on GPUs, gloo in the CPU tests)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms, units
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), int(u.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return ws, int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0"))


def cpu_oracle_sample(seconds: float = 12.0, n_sample: int = 1 << 17):
    """The CPU oracle as it stands on the host cores, on a bounded sample of
    the workload (the same recipe with fewer blocks).  Returns (value, cores,
    sample description, (A, B, y, x_oracle))."""
    import oracle
    A, B, y = synthetic.gen_system(n_sample, M, K_RHS, seed=SEED)
    cores = oracle.max_threads()
    x, info = oracle.cr_solve(A, B, y)       # warm-up, also the reference x of the sample
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.cr_solve(A, B, y)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    value = n_sample * reps / el
    desc = f"{reps} oracle solves (factor+solve) of an N=2^{n_sample.bit_length() - 1} system, m={M}, k={K_RHS}, {el:.1f} s"
    return value, cores, desc, (A, B, y, x)


def cpu_oracle_single_thread(seconds: float = 5.0, n_sample: int = 1 << 14):
    """The same oracle on one host core (OpenMP set to one thread), on a
    smaller sample of the same workload."""
    import oracle
    A, B, y = synthetic.gen_system(n_sample, M, K_RHS, seed=SEED)
    cores = oracle.max_threads()
    oracle.set_threads(1)
    try:
        oracle.cr_solve(A, B, y)
        reps, t0 = 0, time.perf_counter()
        while True:
            oracle.cr_solve(A, B, y)
            reps += 1
            el = time.perf_counter() - t0
            if el >= seconds:
                break
    finally:
        oracle.set_threads(cores)
    return {"value": n_sample * reps / el, "unit": "block-rows/s", "cores": 1, "kind": "oracle",
            "sample": f"{reps} single-thread oracle solves of an N=2^{n_sample.bit_length() - 1} system, "
                      f"m={M}, k={K_RHS}, {el:.1f} s"}


def oracle_rate(systems, seconds: float = 10.0, backward: bool = False):
    """The CPU oracle as it stands, on the host cores, over a list of
    (A, B, y[, c]) systems, repeated for about `seconds`; block-rows/s."""
    import oracle
    rows = sum(s[0].shape[0] for s in systems)
    reps, t0 = 0, time.perf_counter()
    while True:
        for sysm in systems:
            x, _ = oracle.cr_solve(*sysm[:3])
            if backward:
                oracle.cr_backward(sysm[0], sysm[1], x, sysm[3])
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return rows * reps / el, oracle.max_threads(), reps, el


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    n = 1 << args.log2n
    A, B, y = synthetic.gen_system(n, M, K_RHS, seed=SEED)
    for _ in range(args.warmup):
        oracle.cr_solve(A, B, y)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.cr_solve(A, B, y)
    el = time.perf_counter() - t0
    value = n * args.steps / el
    cores = oracle.max_threads()
    workload = WORKLOAD.replace("N=2^20", f"N=2^{args.log2n}")
    line = {"impl": "reference", "metric": "block-rows/s", "value": value, "unit": "block-rows/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c128 (f64)", "data": "synthetic",
            "config": {"workload": workload, "N": n, "m": M, "k": K_RHS, "seed": SEED},
            "cpu_baseline": {"value": value, "unit": "block-rows/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} oracle solves (factor+solve) of the whole N=2^{args.log2n}, "
                                       f"m={M}, k={K_RHS} system, {el:.1f} s"},
            "e2e": {"value": value, "unit": "block-rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# steps of the batched / mixed / adjoint measurements inside the default run
# (the adjoint step is short and takes four times as many)
EXTRA_STEPS, EXTRA_WARMUP = 3, 1

BATCH_SEED = 3003
BATCH_WORKLOAD = ("batched CR: 4096 independent HPD block-tridiagonal systems in one persistent launch, "
                  "N ~ U[16, 4096], m in {4, 8, 16, 32}, k ~ U[1, 16], complex128")


def batched_residual_eta(b, A, B, y, x) -> float:
    """Worst max-norm backward error over every system of a batch (torch ops
    on the measurement side)."""
    import torch
    worst = 0.0
    with torch.no_grad():
        for i in range(len(b.Ns)):
            a, bb, xi = b.system_view(i, A, B, x)
            yi = b.system_view(i, A, B, y)[2]
            Ah = torch.tril(a, -1)
            Ah = Ah + Ah.conj().transpose(1, 2) + torch.diag_embed(torch.diagonal(a, dim1=1, dim2=2).real.to(a.dtype))
            r = yi - torch.bmm(Ah, xi)
            if len(bb):
                r[1:] -= torch.bmm(bb, xi[:-1])
                r[:-1] -= torch.bmm(bb.conj().transpose(1, 2), xi[1:])
            nA = (Ah.abs().sum(2).max() + 2 * (bb.abs().sum(2).max() if len(bb) else 0)).item()
            worst = max(worst, (r.abs().amax() / (nA * xi.abs().amax())).item())
    return worst


def measure_batched(steps: int, warmup: int, nsys: int = 4096, with_oracle: bool = True,
                    cpu_seconds: float = 10.0) -> dict:
    """4096 uneven systems (seed 3003): one persistent launch replayed as a CUDA
    graph with autotuned tiles, against the plain single-system path called
    per system on the same GPU; sampled systems against the oracle and every
    system by its residual."""
    import torch
    import paper_1807_00370_gb300 as crs
    Ns, ms, ks = synthetic.gen_batch_shapes(4096, seed=BATCH_SEED)
    Ns, ms, ks = Ns[:nsys], ms[:nsys], ks[:nsys]
    A, B, y = synthetic.gen_batch_device(Ns, ms, ks, seed=BATCH_SEED)
    x = torch.empty_like(y)
    t_tune = time.perf_counter()
    b = crs.Batch(Ns, ms, ks, tiles="auto")
    t_tune = time.perf_counter() - t_tune
    rows = int(Ns.sum())
    flops = float((Ns * (25.33 * ms.astype(float) ** 3 + 40.0 * ms.astype(float) ** 2 * ks)).sum())
    stream = torch.cuda.current_stream()
    for _ in range(max(warmup, 1)):
        crs.crsolve_batch_graph_launch(b, A, B, y, x)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        crs.crsolve_batch_graph_launch(b, A, B, y, x)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_step = e0.elapsed_time(e1) / steps
    infos = crs.crsolve_batch_info(b)
    # the plain path: one plan per system, all on the same stream
    xp = torch.empty_like(y)
    e0.record(stream)
    for i in range(len(Ns)):
        p = crs.Plan(int(Ns[i]), int(ms[i]), int(ks[i]))
        a, bb, yy = b.system_view(i, A, B, y)
        crs.crsolve_factor(p, a, bb if Ns[i] > 1 else None)
        crs.crsolve_solve(p, yy, b.system_view(i, A, B, xp)[2])
    e1.record(stream)
    torch.cuda.synchronize()
    ms_plain = e0.elapsed_time(e1)
    same = bool(torch.equal(x, xp))
    peak_tf = FP64_PEAK_GFLOPS / 1e3
    out = {
        "metric": "block-rows/s", "value": rows / (ms_step * 1e-3), "unit": "block-rows/s",
        "ms_per_step": ms_step, "steps": steps, "warmup": max(warmup, 1),
        "config": {"workload": BATCH_WORKLOAD, "systems": len(Ns), "block_rows": rows, "seed": BATCH_SEED,
                   "slots": b.nslots, "l2": "inputs larger than L2, no flush",
                   "tiles": {str(k): v for k, v in b.tiles.items()}, "autotune_s": t_tune},
        "roofline": {"bound": "alu", "kernel": "k_batch (whole step)", "achieved": flops / (ms_step * 1e-3) / 1e12,
                     "peak": peak_tf, "unit": "TFLOP/s", "frac": flops / (ms_step * 1e-3) / 1e12 / peak_tf,
                     "traffic": None},
        "speedup_vs_plain": {"plain_ms": ms_plain, "batched_ms": ms_step, "speedup": ms_plain / ms_step,
                             "bitwise_equal": same},
        "breakdown_count": sum(1 for r in infos if r["status"]),
        "gpu_launches": steps,
    }
    err = {"residual_eta_worst": batched_residual_eta(b, A, B, y, x), "bound": 1e-10}
    if with_oracle:
        import oracle
        rng = np.random.default_rng(0)
        pick = []
        for cls in (4, 8, 16, 32):
            idx = np.flatnonzero(ms == cls)
            if len(idx):
                pick += [int(i) for i in rng.choice(idx, min(2, len(idx)), replace=False)]
        worst, flags = 0.0, True
        for i in pick:
            a, bb, yy = (t.cpu().numpy() for t in b.system_view(i, A, B, y))
            xo, io = oracle.cr_solve(a, bb, yy)
            xi = b.system_view(i, A, B, x)[2].cpu().numpy()
            worst = max(worst, float(np.linalg.norm(xi - xo) / np.linalg.norm(xo)))
            flags = flags and infos[i] == io
        err.update({"rel_err_vs_oracle_max": worst, "flags_equal": flags,
                    "oracle_systems": [f"#{i} N={Ns[i]} m={ms[i]} k={ks[i]}" for i in pick]})
        sample = [tuple(t.cpu().numpy() for t in b.system_view(int(i), A, B, y))
                  for i in rng.choice(len(Ns), 32, replace=False)]
        v, cores, reps, el = oracle_rate(sample, seconds=cpu_seconds)
        out["cpu_baseline"] = {"value": v, "unit": "block-rows/s", "cores": cores, "kind": "oracle",
                               "sample": f"{reps} passes over 32 randomly chosen systems of the batch "
                                         f"({sum(s_[0].shape[0] for s_ in sample)} block rows), {el:.1f} s"}
    out["error"] = err
    b.close()
    del A, B, y, x, xp
    torch.cuda.empty_cache()
    return out


def run_batched(args):
    import torch
    torch.cuda.set_device(0)
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(1.0)
    sampler.mark(True)
    res = measure_batched(args.steps, args.warmup, args.nsys, with_oracle=not args.no_cpu_baseline)
    sampler.mark(False)
    line = {"metric": res["metric"], "value": res["value"], "unit": res["unit"], "n_gpus": 1,
            "steps": res["steps"], "warmup": res["warmup"], "ms_per_step": res["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128 (f64)",
            "data": "synthetic"}
    line.update({k: v for k, v in res.items() if k not in line and k != "metric"})
    line.update({"clocks": sampler.stop(), "e2e": None})
    line.setdefault("cpu_baseline", None)
    print(json.dumps(line), flush=True)


ADJ_N, ADJ_M, ADJ_K, ADJ_SEED = 1 << 16, 16, 8, 2000
ADJ_WORKLOAD = ("differentiation: factor + solve + crsolve_backward (re-solve and gA, gB outer products), "
                "N=2^16, m=16, k=8, complex128, loss Re sum(conj(c) x)")


def adjoint_flops_per_row(m: int, k: int) -> float:
    """gA (lower triangle, two k-term products per entry) + gB (full, two)."""
    return 8.0 * (m * (m + 1) / 2 + m * m) * 2 * k


def adjoint_keep_levels(args, dA, dB, dy, dc, full_bytes, full_ms):
    """Memory held between the forward and the backward pass against the
    time of one forward + backward step, for plans that keep the factors of
    the first `keep` levels only (crsolve_plan_keep_levels): forward = factor +
    solve, then the scratch (coarse levels, solve buffers) is released; the
    backward pass binds a new scratch, which re-factors the coarse levels."""
    import torch
    import paper_1807_00370_gb300 as crs
    N, m, k = dy.shape
    out = [{"keep": "all", "held_bytes": full_bytes, "ms_per_step": full_ms}]
    stream = torch.cuda.current_stream()
    for keep in (2, 1, 0):
        plan = crs.Plan(N, m, k, keep_levels=keep)
        x = torch.empty_like(dy)

        def step():
            crs.crsolve_factor(plan, dA, dB)
            crs.crsolve_solve(plan, dy, x)
            plan.release_scratch()
            return crs.crsolve_backward(plan, x, dc)

        for _ in range(2):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        out.append({"keep": keep, "held_bytes": plan.workspace_bytes, "scratch_bytes": plan.scratch_bytes,
                    "ms_per_step": e0.elapsed_time(e1) / args.steps})
    return out


def measure_adjoint(steps: int, warmup: int, with_oracle: bool = True, keep_levels: bool = True,
                    cpu_seconds: float = 10.0) -> dict:
    """Forward + backward (factor, solve, crsolve_backward) at N = 2^16, m = 16,
    k = 8; gradients against the oracle's adjoint on the whole system."""
    import torch
    import paper_1807_00370_gb300 as crs
    N, m, k = ADJ_N, ADJ_M, ADJ_K
    A, B, y = synthetic.gen_system(N, m, k, seed=ADJ_SEED)
    c = synthetic.gen_cotangent(N, m, k, seed=ADJ_SEED)
    dA, dB, dy, dc = (torch.from_numpy(a).cuda() for a in (A, B, y, c))
    plan = crs.Plan(N, m, k)
    x = torch.empty_like(dy)
    stream = torch.cuda.current_stream()

    def step():
        crs.crsolve_factor(plan, dA, dB)
        crs.crsolve_solve(plan, dy, x)
        return crs.crsolve_backward(plan, x, dc)

    for _ in range(max(warmup, 3)):
        step()
    torch.cuda.synchronize()
    launches0 = crs.crsolve_launch_count(plan)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        grads = step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_step = e0.elapsed_time(e1) / steps
    launches = crs.crsolve_launch_count(plan) - launches0
    recs, ms_step_ev = kernel_breakdown(crs, plan, step, steps, stream)
    adj_ms = sum(r[3] for r in recs if r[0] == "adjoint_outer") / steps
    flops = N * (flops_per_block_row(m, k) + flops_solve_per_odd_block(m, k) + adjoint_flops_per_row(m, k))
    peak_tf = FP64_PEAK_GFLOPS / 1e3
    by = {}
    for kind, _, _, kms in recs:
        by[kind] = by.get(kind, 0.0) + kms / steps
    out = {
        "metric": "block-rows/s", "value": N / (ms_step * 1e-3), "unit": "block-rows/s",
        "ms_per_step": ms_step, "ms_per_step_with_kernel_events": ms_step_ev, "steps": steps,
        "warmup": max(warmup, 3),
        "config": {"workload": ADJ_WORKLOAD, "N": N, "m": m, "k": k, "seed": ADJ_SEED},
        "roofline": {"bound": "alu", "kernel": "whole forward + backward step",
                     "achieved": flops / (ms_step * 1e-3) / 1e12, "peak": peak_tf, "unit": "TFLOP/s",
                     "frac": flops / (ms_step * 1e-3) / 1e12 / peak_tf, "traffic": None,
                     "adjoint_outer_frac": (N * adjoint_flops_per_row(m, k) / (adj_ms * 1e-3) / 1e12 / peak_tf)
                     if adj_ms else None},
        "kernels": {kk: {"ms_per_step": v} for kk, v in by.items()},
        "gpu_launches": launches,
    }
    if with_oracle:
        import oracle
        xo, io = oracle.cr_solve(A, B, y)
        gyo, gAo, gBo, st = oracle.cr_backward(A, B, xo, c)
        gy, gA, gB = (g.cpu().numpy() for g in grads)

        def rel(a, b):
            return float(np.linalg.norm(a - b) / np.linalg.norm(b))
        out["error"] = {"x": rel(x.cpu().numpy(), xo), "gy": rel(gy, gyo), "gA": rel(gA, gAo), "gB": rel(gB, gBo),
                        "flags_equal": crs.crsolve_info_get(plan) == io, "bound": 1e-10,
                        "reference": "oracle solve + adjoint on the whole system"}
        sA, sB, sy = synthetic.gen_system(1 << 12, m, k, seed=ADJ_SEED)
        sc = synthetic.gen_cotangent(1 << 12, m, k, seed=ADJ_SEED)
        v, cores, reps, el = oracle_rate([(sA, sB, sy, sc)], seconds=cpu_seconds, backward=True)
        out["cpu_baseline"] = {"value": v, "unit": "block-rows/s", "cores": cores, "kind": "oracle",
                               "sample": f"{reps} oracle solve + backward of an N=2^12, m={m}, k={k} system, {el:.1f} s"}
    if keep_levels:
        class _A:
            pass
        a = _A()
        a.steps = steps
        out["keep_levels"] = adjoint_keep_levels(a, dA, dB, dy, dc, plan.workspace_bytes, ms_step)
    plan.close()
    del dA, dB, dy, dc, x
    torch.cuda.empty_cache()
    return out


def run_adjoint(args):
    import torch
    torch.cuda.set_device(0)
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(1.0)
    sampler.mark(True)
    res = measure_adjoint(args.steps, args.warmup, with_oracle=not args.no_cpu_baseline)
    sampler.mark(False)
    line = {"metric": res["metric"], "value": res["value"], "unit": res["unit"], "n_gpus": 1,
            "steps": res["steps"], "warmup": res["warmup"], "ms_per_step": res["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128 (f64)",
            "data": "synthetic"}
    line.update({k: v for k, v in res.items() if k not in line and k != "metric"})
    line.update({"clocks": sampler.stop(), "e2e": None})
    line.setdefault("cpu_baseline", None)
    print(json.dumps(line), flush=True)


MIX_N, MIX_M, MIX_K, MIX_SEED = 1 << 14, 64, 32, 4000
MIX_WORKLOAD = ("precision: FP32 fine levels + FP64 coarse levels, FP64 residual and iterative refinement, "
                "N=2^14, m=64, k=32, complex, kappa in {1e2, 1e4, 1e6}")


def residual_eta(dA, dB, dy, dx) -> float:
    """max-norm backward error ||y - A x|| / (||A|| ||x||) of a device solution
    (torch ops on the measurement side, not part of the solver)."""
    import torch
    with torch.no_grad():
        Ah = torch.tril(dA, -1)
        Ah = Ah + Ah.conj().transpose(1, 2) + torch.diag_embed(torch.diagonal(dA, dim1=1, dim2=2).real.to(dA.dtype))
        r = dy - torch.bmm(Ah, dx)
        r[1:] -= torch.bmm(dB, dx[:-1])
        r[:-1] -= torch.bmm(dB.conj().transpose(1, 2), dx[1:])
        normA = (Ah.abs().sum(2).max() + 2 * dB.abs().sum(2).max()).item()
        return (r.abs().amax() / (normA * dx.abs().amax())).item()


def measure_mixed(steps: int, warmup: int, log2n: int = 14, with_oracle: bool = True, cpu_seconds: float = 10.0):
    """For each kappa: the mixed form and the plain FP64 path on the same
    system and GPU; the mixed solution against the oracle on the whole
    system."""
    import torch
    import paper_1807_00370_gb300 as crs
    from paper_1807_00370_gb300 import _native as nat
    N, m, k = 1 << log2n, MIX_M, MIX_K
    name = f"mixed_N2p{log2n}_m64_k32"
    table = json.load(open(os.path.join(ROOT, "tests", "golden", "kappa_shifts.json")))
    shifts = table.get(name, {"shifts": {"1e+02": 1.0, "1e+04": 1.0, "1e+06": 1.0}})
    stream = torch.cuda.current_stream()
    runs = []
    for kap in ("1e+02", "1e+04", "1e+06"):
        A, B, y = synthetic.gen_system(N, m, k, seed=MIX_SEED, shift=shifts["shifts"][kap])
        dA, dB, dy = (torch.from_numpy(a).cuda() for a in (A, B, y))
        res = {}
        for pname, prec in (("mixed", nat.CRSOLVE_MIXED), ("fp64", nat.CRSOLVE_FP64)):
            plan = crs.Plan(N, m, k, precision=prec)
            x = torch.empty_like(dy)
            for _ in range(max(warmup, 1)):
                crs.crsolve_factor(plan, dA, dB)
                crs.crsolve_solve(plan, dy, x)
            torch.cuda.synchronize()
            launches0 = crs.crsolve_launch_count(plan)

            def step():
                crs.crsolve_factor(plan, dA, dB)
                crs.crsolve_solve(plan, dy, x)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                step()
            e1.record(stream)
            torch.cuda.synchronize()
            launches = (crs.crsolve_launch_count(plan) - launches0) // steps
            stats = crs.crsolve_mixed_stats(plan) if prec == nat.CRSOLVE_MIXED else None
            recs, _ = kernel_breakdown(crs, plan, step, steps, stream)
            by = {}
            for kind, _, _, kms in recs:
                by[kind] = round(by.get(kind, 0.0) + kms / steps, 3)
            res[pname] = {"ms": e0.elapsed_time(e1) / steps, "x": x, "kernels_ms": by,
                          "launches": launches, "info": crs.crsolve_info_get(plan), "stats": stats}
            plan.close()
        err = float((torch.linalg.norm(res["mixed"]["x"] - res["fp64"]["x"]) / torch.linalg.norm(res["fp64"]["x"])).item())
        run = {"kappa": float(kap), "shift": shifts["shifts"][kap], "mixed_ms": res["mixed"]["ms"],
               "fp64_ms": res["fp64"]["ms"], "speedup": res["fp64"]["ms"] / res["mixed"]["ms"],
               "rel_err_vs_fp64_path": err, "residual_eta_mixed": residual_eta(dA, dB, dy, res["mixed"]["x"]),
               "refinement": res["mixed"]["stats"], "launches_per_step": res["mixed"]["launches"],
               "mixed_kernels_ms": res["mixed"]["kernels_ms"], "fp64_kernels_ms": res["fp64"]["kernels_ms"]}
        if kap == "1e+02":
            # the refinement's FP64-accurate residual: tensor-core splitting against the FP64 pipe
            rt = {}
            for meth in ("split", "fp64"):
                rr = crs.crsolve_residual(dA, dB, res["mixed"]["x"], dy, method=meth)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(5):
                    crs.crsolve_residual(dA, dB, res["mixed"]["x"], dy, method=meth, r=rr)
                e1.record(stream)
                torch.cuda.synchronize()
                rt[meth] = {"ms": e0.elapsed_time(e1) / 5, "r": rr}
            run["residual_ms"] = {"split": rt["split"]["ms"], "fp64": rt["fp64"]["ms"],
                                  "speedup": rt["fp64"]["ms"] / rt["split"]["ms"],
                                  "max_abs_diff": float((rt["split"]["r"] - rt["fp64"]["r"]).abs().max().item()),
                                  "max_abs_residual": float(rt["fp64"]["r"].abs().max().item())}
            del rt
        if with_oracle:
            import oracle
            xo, io = oracle.cr_solve(A, B, y)
            xm = res["mixed"]["x"].cpu().numpy()
            run["rel_err_vs_oracle"] = float(np.linalg.norm(xm - xo) / np.linalg.norm(xo))
            run["flags_equal_oracle"] = res["mixed"]["info"] == io
            run["bound"] = 1e-10
        runs.append(run)
        del dA, dB, dy, res
        torch.cuda.empty_cache()
    peak_tf = FP64_PEAK_GFLOPS / 1e3
    out = {"metric": "block-rows/s", "value": N / (runs[0]["mixed_ms"] * 1e-3), "unit": "block-rows/s",
           "ms_per_step": runs[0]["mixed_ms"], "steps": steps, "warmup": max(warmup, 1),
           "config": {"workload": MIX_WORKLOAD.replace("N=2^14", f"N=2^{log2n}"), "N": N, "m": m, "k": k,
                      "seed": MIX_SEED, "value_is": "kappa ~ 1e2"},
           "speedup_vs_fp64": {r["kappa"]: r["speedup"] for r in runs},
           "runs": runs,
           "fp64_path_frac_of_peak": N * flops_per_block_row(m, k) / (runs[0]["fp64_ms"] * 1e-3) / 1e12 / peak_tf}
    if with_oracle:
        small = table.get("mixed_N2p10_m64_k32", {"shifts": {"1e+02": 1.0}})["shifts"]["1e+02"]
        v, cores, reps, el = oracle_rate([synthetic.gen_system(1 << 10, m, k, seed=MIX_SEED, shift=small)],
                                         seconds=cpu_seconds)
        out["cpu_baseline"] = {"value": v, "unit": "block-rows/s", "cores": cores, "kind": "oracle",
                               "sample": f"{reps} oracle solves of an N=2^10, m={m}, k={k}, kappa~1e2 system, {el:.1f} s"}
    return out


def run_mixed(args):
    import torch
    torch.cuda.set_device(0)
    log2n = 14 if args.log2n in (14, 20) else args.log2n      # smaller cases are for profiling only
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(1.0)
    sampler.mark(True)
    res = measure_mixed(args.steps, args.warmup, log2n, with_oracle=not args.no_cpu_baseline)
    sampler.mark(False)
    line = {"metric": res["metric"], "value": res["value"], "unit": res["unit"], "n_gpus": 1,
            "steps": res["steps"], "warmup": res["warmup"], "ms_per_step": res["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64 fine levels / c128",
            "data": "synthetic"}
    line.update({k: v for k, v in res.items() if k not in line and k != "metric"})
    line.update({"clocks": sampler.stop(), "e2e": None})
    line.setdefault("cpu_baseline", None)
    print(json.dumps(line), flush=True)


ALG1_WORKLOAD = ("Algorithm 1 (both halves reduced at every level, Sec. 3), one HPD block-tridiagonal system: "
                 "N=2^20 blocks, m=8, k=4, complex128")


def alg1_flops(N: int, m: int, k: int) -> float:
    """Algorithmic flops of one factor + solve by Algorithm 1 with N = 2^L:
    L split levels that each eliminate all N blocks (factor as for an odd
    block of classic reduction; down sweep r = L^{-1} y m^2 k/2 and Z^H r
    2 m^2 k), then N single-block Cholesky solves (m^3/6 + m^2 k)."""
    L = N.bit_length() - 1
    per_level = N * (flops_factor_per_odd_block(m) + 8.0 * 2.5 * m * m * k)
    base = N * 8.0 * (m ** 3 / 6.0 + m * m * k)
    return L * per_level + base


def run_alg1(args):
    """One step = crsolve_factor + crsolve_solve of an Algorithm 1 plan on the
    plain workload's system (same generator and seed)."""
    import torch
    import paper_1807_00370_gb300 as crs
    from paper_1807_00370_gb300 import _native as nat
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    N = 1 << args.log2n
    L = args.log2n
    workload = ALG1_WORKLOAD.replace("N=2^20", f"N=2^{args.log2n}")
    A, B, y = synthetic.gen_system(N, M, K_RHS, seed=SEED + rank)
    dA, dB, dy = (torch.from_numpy(a).to(dev) for a in (A, B, y))
    plan = crs.Plan(N, M, K_RHS, flags=nat.CRSOLVE_PLAN_ALG1 | (0 if args.no_e2e else nat.CRSOLVE_PLAN_HOST_STAGING))
    dx = torch.empty_like(dy)
    stream = torch.cuda.current_stream()

    def step():
        crs.crsolve_factor(plan, dA, dB)
        crs.crsolve_solve(plan, dy, dx)

    for _ in range(max(args.warmup, 3)):
        step()
    info = crs.crsolve_info_get(plan)
    torch.cuda.synchronize()
    sampler = ClockSampler(dev.index)
    sampler.start()
    time.sleep(1.0)
    launches0 = crs.crsolve_launch_count(plan)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler.mark(True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    launches = crs.crsolve_launch_count(plan) - launches0
    recs, _ = kernel_breakdown(crs, plan, step, args.steps, stream)
    sampler.mark(False)
    clocks = sampler.stop()
    ms, total_units = reduce_over_ranks(ms, N * args.steps, dev)
    ms_step = ms / args.steps
    value = total_units / (ms * 1e-3)
    by_kind = {}
    for kind, level, units, kms in recs:
        d = by_kind.setdefault(kind, {"ms": 0.0, "launches": 0})
        d["ms"] += kms
        d["launches"] += 1
    # dominant kernel: k_factor_odd on the split levels (the single-block level
    # is excluded: it only needs the Cholesky factors)
    fac_ms = sum(kms for kind, level, units, kms in recs if kind == "factor_odd" and level < L)
    fac_launches = sum(1 for kind, level, units, kms in recs if kind == "factor_odd" and level < L)
    fac_flops = args.steps * L * N * flops_factor_per_odd_block(M)
    peak_tf = FP64_PEAK_GFLOPS / 1e3
    achieved = fac_flops / (fac_ms * 1e-3) / 1e12 if fac_ms else None
    step_flops = alg1_flops(N, M, K_RHS)

    # classic reduction on the same system and GPU, for the cost of the split
    cplan = crs.Plan(N, M, K_RHS)
    for _ in range(3):
        crs.crsolve_factor(cplan, dA, dB)
        crs.crsolve_solve(cplan, dy, dx)
    torch.cuda.synchronize()
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    for _ in range(args.steps):
        crs.crsolve_factor(cplan, dA, dB)
        crs.crsolve_solve(cplan, dy, dx)
    c1.record(stream)
    torch.cuda.synchronize()
    classic_ms = c0.elapsed_time(c1) / args.steps
    cplan.close()
    step()
    torch.cuda.synchronize()

    eta = residual_eta(dA, dB, dy, dx)

    e2e = None
    if not args.no_e2e:
        tA, tB, ty = (torch.from_numpy(a).pin_memory() for a in (A, B, y))
        tx = torch.empty_like(ty).pin_memory()
        crs.crsolve_solve_host(plan, tA, tB, ty, tx)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            crs.crsolve_solve_host(plan, tA, tB, ty, tx)
        el = time.perf_counter() - t0
        e2e = {"value": N * args.e2e_steps / el * ws, "unit": "block-rows/s",
               "h2d_bytes_per_step": int(tA.numel() + tB.numel() + ty.numel()) * 16,
               "d2h_bytes_per_step": int(tx.numel()) * 16 + 8, "steps": args.e2e_steps}

    cpu, sample_err = None, None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        n_sample = 1 << 14
        sA, sB, sy = synthetic.gen_system(n_sample, M, K_RHS, seed=SEED)
        sx, _ = oracle.alg1_solve(sA, sB, sy)
        reps, t0 = 0, time.perf_counter()
        while True:
            oracle.alg1_solve(sA, sB, sy)
            reps += 1
            el = time.perf_counter() - t0
            if el >= 10.0:
                break
        cpu = {"value": n_sample * reps / el, "unit": "block-rows/s", "cores": oracle.max_threads(),
               "kind": "oracle",
               "sample": f"{reps} Algorithm 1 oracle solves of an N=2^14, m={M}, k={K_RHS} system, {el:.1f} s"}
        xs = crs.solve(*(torch.from_numpy(a).to(dev) for a in (sA, sB, sy)), method="alg1").cpu().numpy()
        sample_err = float(np.linalg.norm(xs - sx) / np.linalg.norm(sx))

    if rank == 0:
        line = {
            "metric": "block-rows/s", "value": value, "unit": "block-rows/s", "n_gpus": ws,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128 (f64)",
            "data": "synthetic",
            "config": {"workload": workload, "N": N, "m": M, "k": K_RHS, "seed": SEED,
                       "l2": "inputs larger than L2 (A alone 1 GiB), no flush",
                       "parallelism": f"{ws} independent system(s), one per GPU"},
            "roofline": {"bound": "alu", "kernel": f"k_factor_odd<{M}>, split levels 0..{L - 1}",
                         "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s",
                         "frac": (achieved / peak_tf) if achieved else None, "traffic": None,
                         "peak_source": "FP64 pipe: 2 DFMA/clk/SM x 152 SMs x 2070 MHz (derived)",
                         "flops_per_unit": flops_factor_per_odd_block(M), "units": L * N,
                         "launches_per_step": fac_launches // args.steps},
            "step_roofline": {"flops_per_step": step_flops, "achieved": step_flops / (ms_step * 1e-3) / 1e12,
                              "frac": step_flops / (ms_step * 1e-3) / 1e12 / peak_tf},
            "vs_classic": {"classic_ms_per_step": classic_ms, "ratio": ms_step / classic_ms,
                           "flop_ratio": step_flops / (N * flops_per_block_row(M, K_RHS))},
            "kernels": {k: {"ms_per_step": v["ms"] / args.steps, "launches_per_step": v["launches"] // args.steps}
                        for k, v in by_kind.items()},
            "error": {"residual_eta": eta, "sample_rel_err_vs_oracle": sample_err, "bound": 1e-10},
            "breakdown": info, "gpu_launches": launches, "clocks": clocks, "e2e": e2e, "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def plain_variant_runs(args, plan, dev):
    """The other two runs of the plain workload at N = 2^20, m = 8, k = 4: the
    diagonal shift that makes kappa ~ 1e6 (tests/golden/kappa_shifts.json),
    and A_{N/2} - 3I (indefinite).  Each: factor + solve time (CUDA events),
    and the check against the CPU oracle on the whole system (relative error
    and the a-priori estimate kappa * eta; the breakdown flag and location)."""
    import torch
    import oracle
    import paper_1807_00370_gb300 as crs
    table = json.load(open(os.path.join(ROOT, "tests", "golden", "kappa_shifts.json")))
    case = table["plain_N2p20_m8_k4"]
    out = []
    stream = torch.cuda.current_stream()
    for name in ("kappa~1e6", "indefinite A_{N/2} - 3I"):
        if name.startswith("kappa"):
            A, B, y = synthetic.gen_system(N_BLOCKS, M, K_RHS, seed=case["seed"], shift=case["shifts"]["1e+06"])
        else:
            A, B, y = synthetic.gen_system(N_BLOCKS, M, K_RHS, seed=SEED)
            A = synthetic.make_indefinite(A)
        dA, dB, dy = (torch.from_numpy(a).to(dev) for a in (A, B, y))
        dx = torch.empty_like(dy)
        for _ in range(2):
            crs.crsolve_factor(plan, dA, dB)
            crs.crsolve_solve(plan, dy, dx)
        torch.cuda.synchronize()
        steps = 10
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            crs.crsolve_factor(plan, dA, dB)
            crs.crsolve_solve(plan, dy, dx)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        info = crs.crsolve_info_get(plan)
        xo, io = oracle.cr_solve(A, B, y)
        run = {"run": name, "ms_per_step": ms, "value": N_BLOCKS / (ms * 1e-3), "breakdown": info,
               "breakdown_equals_oracle": info == io}
        if info["status"] == 0:
            x = dx.cpu().numpy()
            eta = residual_eta(dA, dB, dy, dx)
            run.update({"rel_err_vs_oracle": float(np.linalg.norm(x - xo) / np.linalg.norm(xo)),
                        "residual_eta": eta, "kappa_estimate": 1e6, "a_priori_kappa_eta": 1e6 * eta,
                        "bound": 1e-10})
        else:
            run["x_all_nan"] = bool(torch.isnan(dx).all().item())
        out.append(run)
        del dA, dB, dy, dx
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched, mixed and adjoint measurements of the default run")
    ap.add_argument("--workload", default="plain", choices=["plain", "batched", "adjoint", "mixed", "alg1"])
    ap.add_argument("--nsys", type=int, default=4096, help="systems of the batched workload")
    ap.add_argument("--log2n", type=int, default=20,
                    help="log2 of the block count (smaller cases are for profiling only)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "adjoint":
        return run_adjoint(args)
    if args.workload == "mixed":
        return run_mixed(args)
    if args.workload == "alg1":
        return run_alg1(args)

    import torch
    import paper_1807_00370_gb300 as crs
    global N_BLOCKS, WORKLOAD
    if args.log2n != 20:
        N_BLOCKS = 1 << args.log2n
        WORKLOAD = WORKLOAD.replace("N=2^20", f"N=2^{args.log2n}")
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    A, B, y = synthetic.gen_system(N_BLOCKS, M, K_RHS, seed=SEED + rank)
    dA, dB, dy = (torch.from_numpy(a).to(dev) for a in (A, B, y))
    plan = crs.Plan(N_BLOCKS, M, K_RHS, flags=0 if args.no_e2e else 1)
    dx = torch.empty_like(dy)
    stream = torch.cuda.current_stream()

    def step():
        crs.crsolve_factor(plan, dA, dB)
        crs.crsolve_solve(plan, dy, dx)

    for _ in range(max(args.warmup, 3)):
        step()
    info = crs.crsolve_info_get(plan)
    torch.cuda.synchronize()

    sampler = ClockSampler(dev.index)
    sampler.start()
    time.sleep(1.0)
    launches0 = crs.crsolve_launch_count(plan)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler.mark(True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    launches = crs.crsolve_launch_count(plan) - launches0
    recs, ms_step_ev = kernel_breakdown(crs, plan, step, args.steps, stream)
    sampler.mark(False)
    clocks = sampler.stop()
    ms, total_units = reduce_over_ranks(ms, N_BLOCKS * args.steps, dev)

    # per-kernel breakdown and the dominant kernel's roofline (FP64 pipe)
    by_kind = {}
    for kind, level, units, kms in recs:
        d = by_kind.setdefault(kind, {"ms": 0.0, "launches": 0, "units": 0})
        d["ms"] += kms
        d["launches"] += 1
        d["units"] += units
    fac = by_kind.get("factor_odd", {"ms": 0.0, "units": 0, "launches": 0})
    fac_flops = fac["units"] * flops_factor_per_odd_block(M)
    achieved = fac_flops / (fac["ms"] * 1e-3) / 1e12 if fac["ms"] else None
    peak_tf = FP64_PEAK_GFLOPS / 1e3
    step_flops = N_BLOCKS * flops_per_block_row(M, K_RHS)
    ms_step = ms / args.steps
    value = total_units / (ms * 1e-3)

    # measurement-side residual check (torch ops, not part of the solver)
    eta = residual_eta(dA, dB, dy, dx)
    traffic_blk = captured_traffic_per_odd_block()

    e2e = None
    if not args.no_e2e:
        tA, tB, ty = (torch.from_numpy(a).pin_memory() for a in (A, B, y))
        tx = torch.empty_like(ty).pin_memory()
        crs.crsolve_solve_host(plan, tA, tB, ty, tx)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            crs.crsolve_solve_host(plan, tA, tB, ty, tx)
        el = time.perf_counter() - t0
        e2e = {"value": N_BLOCKS * args.e2e_steps / el * ws, "unit": "block-rows/s",
               "h2d_bytes_per_step": int(tA.numel() + tB.numel() + ty.numel()) * 16,
               "d2h_bytes_per_step": int(tx.numel()) * 16 + 8, "steps": args.e2e_steps,
               "host_link": host_link(dev, tA)}

    cpu = None
    sample_err = None
    variants = None
    probe = fp64_probe()
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and N_BLOCKS == 1 << 20:
        variants = plain_variant_runs(args, plan, dev)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, cores, desc, (sA, sB, sy, sx) = cpu_oracle_sample()
        cpu = {"value": v, "unit": "block-rows/s", "cores": cores, "kind": "oracle", "sample": desc,
               "single_thread": cpu_oracle_single_thread()}
        # the GPU on the same sample, for the error at which the rate is quoted
        xs = crs.solve(*(torch.from_numpy(a).to(dev) for a in (sA, sB, sy))).cpu().numpy()
        sample_err = float(np.linalg.norm(xs - sx) / np.linalg.norm(sx))

    extra = None
    if rank == 0 and ws == 1 and not args.no_extras and N_BLOCKS == 1 << 20:
        # the other forms on the same GPU, after the plain workload's buffers are released
        plan.close()
        del dA, dB, dy, dx
        torch.cuda.empty_cache()
        extra = {}
        xs_ = dict(batched=lambda: measure_batched(EXTRA_STEPS, EXTRA_WARMUP, with_oracle=not args.no_cpu_baseline,
                                                   cpu_seconds=5.0),
                   mixed=lambda: measure_mixed(EXTRA_STEPS, EXTRA_WARMUP, with_oracle=not args.no_cpu_baseline,
                                               cpu_seconds=5.0),
                   adjoint=lambda: measure_adjoint(EXTRA_STEPS * 4, EXTRA_WARMUP, with_oracle=not args.no_cpu_baseline,
                                                   cpu_seconds=5.0))
        sampler2 = ClockSampler(dev.index)
        sampler2.start()
        time.sleep(0.5)
        sampler2.mark(True)
        for name, fn in xs_.items():
            try:
                extra[name] = fn()
            except Exception as e:  # noqa: BLE001 - recorded in the line; the main number stands
                extra[name] = {"failed": f"{type(e).__name__}: {e}"}
        sampler2.mark(False)
        extra["clocks"] = sampler2.stop()

    if rank == 0:
        line = {
            "metric": "block-rows/s", "value": value, "unit": "block-rows/s", "n_gpus": ws,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms_step,
            "ms_per_step_with_kernel_events": ms_step_ev,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128 (f64)",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": N_BLOCKS, "m": M, "k": K_RHS, "seed": SEED,
                       "l2": "inputs larger than L2 (A alone 1 GiB), no flush", "parallelism":
                       f"{ws} independent system(s), one per GPU"},
            "roofline": {"bound": "alu", "kernel": "k_factor_odd<8> (and its coarse-level form "
                                                  "k_factor_odd_wide<8>), all levels; per-launch CUDA events "
                                                  "over a second run of the same steps",
                         "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s",
                         "frac": (achieved / peak_tf) if achieved else None,
                         "traffic": (traffic_blk * (fac["units"] / max(fac["launches"], 1))) if traffic_blk else None,
                         "traffic_note": "dram read+write per launch: the ncu capture of level 0 at N=2^18 scaled "
                                         "by odd blocks; null when the kernel sources differ from the captured ones",
                         "peak_source": "FP64 pipe: 2 DFMA/clk/SM x 152 SMs x 2070 MHz (derived)",
                         "peak_probe": probe,
                         "frac_of_probe": (achieved / probe["tflops"]) if achieved and "tflops" in probe else None,
                         "flops_per_unit": flops_factor_per_odd_block(M), "units": fac["units"] // args.steps,
                         "launches_per_step": fac["launches"] // args.steps},
            "step_roofline": {"flops_per_step": step_flops, "achieved": step_flops / (ms_step * 1e-3) / 1e12,
                              "frac": step_flops / (ms_step * 1e-3) / 1e12 / peak_tf},
            "kernels": {k: {"ms_per_step": v["ms"] / args.steps, "launches_per_step": v["launches"] // args.steps}
                        for k, v in by_kind.items()},
            "error": {"residual_eta": eta, "sample_rel_err_vs_oracle": sample_err, "bound": 1e-10},
            "variants": variants,
            "breakdown": info,
            "gpu_launches": launches,
            "clocks": clocks,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "extra": extra,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
