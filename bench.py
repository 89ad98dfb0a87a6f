"""Benchmark: TR-ALS sweeps/s on one GB300 (one step = one full ALS sweep over all N core updates).

Default workload: the order-5 40^5 tensor (102.4M entries) generated as a TR of ranks
(8,10,12,10,8) with iid N(0,1) cores plus 1e-3 relative Gaussian noise; fit ranks (8,10,12,10,8);
Cholesky normal equations with the structured Gamma-chain coefficient matrix.  The headline
``value`` is the reduced-precision mode (``--mode``, default bf16: X stored once as BF16, RHS
contraction on tensor cores with FP32 accumulation, FP64 Gram chain and solve); the FP64 mode on
the same workload is reported beside it under ``fp64``.  ``--config`` selects another workload.

The roofline object covers the dominant kernel, the RHS contraction (MTTSP, Alg. 2 lines 7-8):
its main kernel is timed alone with CUDA events on the plan's stream after an L2 eviction, once per
mode; ``achieved`` = the bytes of X it must read (the algorithmic traffic) / that time.

``--impl reference`` times the CPU FP64 oracle (regular TR-ALS with the explicit subchain
matrix, Alg. 1) on the same workload instead.
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
METRIC = "TR-ALS sweeps/s at fixed rel. residual, mixed vs FP64; p50/p99 serving latency"
sys.path.insert(0, ROOT)

import trals_inputs as TI  # noqa: E402


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int = 0):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value, device):
    """The largest per-rank value (the job's step time is its slowest rank's), by an all-reduce over the
    default process group; tensors on `device` ("cuda" under NCCL, "cpu" under gloo)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(ms_max, world):
    """Whole-job sweeps/s: every rank runs its own replica of the workload (weak scaling), so the job
    completes `world` sweeps per slowest-rank step."""
    return world * 1000.0 / ms_max


# ----------------------------------------------------------------------------- data
def make_X_device(w, seed, P, torch, dtype):
    """Observed tensor on the device: X_true = TR(true cores) by the library's reconstruction
    kernel, plus the relative noise of the paper's protocol (added with torch)."""
    N = len(w.I)
    if w.kind == "sinusoid":
        f, phi = TI.sinusoid_params(seed, w.terms, N)
        X = TI.sinusoid_tensor(w.I, f, phi) + w.eta * TI.gaussian_noise(seed, w.I)
        return torch.from_numpy(TI.flat_f(X)).to("cuda").to(dtype)
    truth = TI.gaussian_cores(seed, w.I, w.R_true)
    ctx = P.trals_create(0)
    cd = [P.core_to_device(G) for G in truth]
    Xt = torch.empty(w.numel, dtype=torch.float64, device="cuda")
    P.trals_reconstruct(ctx, w.I, w.R_true, cd, Xt)
    noise = torch.from_numpy(TI.flat_f(TI.gaussian_noise(seed, w.I))).to("cuda")
    X = Xt + w.eta * (torch.linalg.vector_norm(Xt) / torch.linalg.vector_norm(noise)) * noise
    ctx.close()
    return X.to(dtype)


def workload_config(w):
    """The workload both arms run (the same dict in both JSON lines)."""
    return {"workload": w.name, "I": list(w.I), "R_fit": list(w.R_fit), "eta": w.eta, "sweeps": w.sweeps,
            "noise": "relative Frobenius" if w.kind == "tr" else "absolute std"}


def mode_xdtype(mode, torch):
    return {"fp64": torch.float64, "fp32": torch.float32, "bf16": torch.float32, "bf16x2": torch.float32,
            "bf16x3": torch.float32}[mode]


# ----------------------------------------------------------------------------- GPU arm
SOLVERS = {"cholesky": 0, "qr": 1}
GRAMS = {"structured": 0, "explicit": 1}


def opts_for(P, mode, args):
    return P.make_opts(mode, solver=SOLVERS[args.solver], gram=GRAMS[args.gram])


def evict_l2(flush_buf, scratch):
    """Evict L2 (129 MB) by reading a 256 MB buffer.  A read leaves clean lines: a flush by writing would
    leave about 100 MB of dirty lines whose write-back the next kernel pays in DRAM bandwidth, a cost no
    sweep has (X itself, 204.8 MB per mode, is larger than L2 and is read, never written)."""
    scratch.copy_(flush_buf.sum())


def time_mode(P, torch, w, X, mode, steps, warmup, seed, flush_buf, X_full, opts):
    stream = torch.cuda.Stream()
    ctx = P.trals_create(0, stream)
    plan = P.Plan(ctx, w.I, w.R_fit, X, opts)
    init = TI.init_cores(seed, w.I, w.R_fit)
    plan.set_cores(init)
    plan.run(warmup, use_graph=True)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    scratch = torch.zeros((), dtype=flush_buf.dtype, device=flush_buf.device)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    torch.cuda.synchronize()
    for k in range(steps):
        with torch.cuda.stream(stream):
            evict_l2(flush_buf, scratch)   # > L2: evicts X between timed sweeps
            ev[k][0].record(stream)
        plan.run(1, use_graph=True)
        with torch.cuda.stream(stream):
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    times = [a.elapsed_time(b) for a, b in ev]
    res = plan.residuals()
    launches = plan.launches_per_sweep()
    # relative residual of the cores after the run, measured against the full-precision X
    r2, x2 = P.trals_residual_explicit(ctx, w.I, w.R_fit, X_full, [plan.core_dev(n) for n in range(len(w.I))])
    res_explicit = float(np.sqrt(max(r2, 0.0) / x2))
    # dominant kernel: the MTTSP of each mode, its main kernel timed alone (events on the plan's
    # stream, recorded by the library around that launch) after an L2 flush
    kern, whole = [], []
    for n in range(len(w.I)):
        per_k, per_t = [], []
        for _ in range(7):
            with torch.cuda.stream(stream):
                evict_l2(flush_buf, scratch)
            k_ms, t_ms = plan.time_mttsp(n)
            per_k.append(k_ms)
            per_t.append(t_ms)
        kern.append(statistics.median(per_k))
        whole.append(statistics.median(per_t))
    paths = [plan.mttsp_path(n) for n in range(len(w.I))]
    plan.close()
    ctx.close()
    return {"ms_per_step": sum(times) / len(times), "times": times, "residual": res_explicit,
            "residual_in_sweep": float(res[-1]) if len(res) else None, "sweeps_run": warmup + steps,
            "launches_per_sweep": launches, "mttsp_kernel_ms": kern, "mttsp_ms": whole, "clocks": clk,
            "mttsp_paths": paths}


def smooth_qr_run(P, torch, seed, peaks, flush):
    """Sub-line: the 256x256x3x256 sinusoid workload (R = 16) in the BF16 mode with the QR-stabilised
    solve (Sec. 3.2), the solver for subproblems whose normal equations are not numerically SPD.
    One warm-up sweep and two timed sweeps (L2 evicted between them), the explicit residual against the
    FP64 X, and the MTTSP of each mode timed alone (the path the plan runs: the two-stage GEMM MTTSP,
    timed from its GEMM through its FP64 reduction)."""
    w = TI.WORKLOADS["sin256x256x3x256_r16"]
    X64 = make_X_device(w, seed, P, torch, torch.float64)
    X32 = X64.to(torch.float32)
    opts = P.make_opts("bf16", solver=SOLVERS["qr"])
    r = time_mode(P, torch, w, X32, "bf16", 2, 1, seed, flush, X64, opts)
    del X64, X32
    nbytes = 2 * w.numel   # the BF16 copy of X, read once per MTTSP
    kern = r["mttsp_kernel_ms"]
    achieved = nbytes / (sum(kern) / len(kern) * 1e-3) / 1e9
    return {"workload": w.name, "mode": "bf16", "solver": "qr", "ms_per_sweep": r["ms_per_step"],
            "sweeps_per_s": 1000.0 / r["ms_per_step"], "residual": r["residual"], "timed_sweeps": len(r["times"]),
            "warmup_sweeps": 1, "mttsp_path_per_mode": [P.MTTSP_PATHS[c] for c in r["mttsp_paths"]],
            "mttsp_ms_per_mode": kern,
            "roofline": {"bound": "hbm", "achieved_gbs": achieved, "hbm_peak_gbs": peaks["hbm_gbs"],
                         "frac_of_hbm": achieved / peaks["hbm_gbs"], "algorithmic_bytes_per_launch": nbytes,
                         "note": "no tensor-core geometry at R = 16 with I_n * r = 65536 (stage-1 table 256 "
                                 "columns wide): the two-stage GEMM MTTSP, one cuBLAS GEMM over the BF16 X, "
                                 "this library's stage-2 kernel and FP64 reduction, timed together; the "
                                 "algorithmic bytes are the BF16 X read once"}}


def mixed_subchain_gram(cores_a, cores_b, n):
    """C = (G_a^{!=n}_[2])^T G_b^{!=n}_[2] (r_a x r_b, columns a + R_n b) from the mixed Gram chain
    Pi = prod over the subchain modes of sum_i A_k(i) (x) B_k(i) (the inner-product structure of the
    paper's by-product proposition), without forming either subchain matrix."""
    N = len(cores_a)
    Pi = None
    for m in [(n + t) % N for t in range(1, N)]:
        A, B = cores_a[m], cores_b[m]
        g = np.einsum("pis,qit->pqst", A, B).reshape(A.shape[0] * B.shape[0], A.shape[2] * B.shape[2])
        Pi = g if Pi is None else Pi @ g
    Ra1, Rb1 = cores_a[n].shape[2], cores_b[n].shape[2]
    Ra0, Rb0 = cores_a[n].shape[0], cores_b[n].shape[0]
    T = Pi.reshape(Ra1, Rb1, Ra0, Rb0).transpose(2, 0, 3, 1)      # (a, b, a', b')
    return T.reshape(Ra0 * Ra1, Rb0 * Rb1, order="F")


def subspace_angle(cores_a, cores_b, n):
    """Largest principal angle (radians) between range(G^{!=n}_[2]) of two TR solutions: with the
    Cholesky factors L_a, L_b of the two Gram matrices, the cosines are the singular values of
    L_a^{-1} C_ab L_b^{-T}.  Gauge invariant; angles below ~1e-8 are not resolved."""
    La = np.linalg.cholesky(mixed_subchain_gram(cores_a, cores_a, n))
    Lb = np.linalg.cholesky(mixed_subchain_gram(cores_b, cores_b, n))
    C = mixed_subchain_gram(cores_a, cores_b, n)
    K = np.linalg.solve(La, np.linalg.solve(Lb, C.T).T)
    s = np.linalg.svd(K, compute_uv=False)
    return float(np.arccos(np.clip(s.min(), -1.0, 1.0)))


def oracle_reference(workload, seed):
    """The FP64 oracle's stored run of a workload (tests/golden/make_oracle_reference.py): per-sweep
    residuals and final cores, or None when no file was written for it."""
    path = os.path.join(ROOT, "tests", "golden", f"oracle_{workload}_seed{seed}.npz")
    if not os.path.exists(path):
        return None
    z = np.load(path)
    N = len(z["I"])
    return {"residuals": z["residuals"], "cores": [z[f"core{n}"] for n in range(N)], "sweeps": int(z["sweeps"])}


def accuracy_run(P, torch, w, X, X_full, mode, opts, seed, ref):
    """The workload's own sweep count from the seeded init in `mode`, then the final relative residual
    (explicit, against the FP64 X) and its gap to the FP64 oracle's, the largest principal angle
    between the subchain ranges of the two solutions over all modes, and the sweeps needed to reach the
    target of the metric's "fixed relative residual": the oracle's final residual + 1e-4.  The
    per-sweep residual is the identity in FP64 and an explicit pass in the reduced modes (which does not
    change the cores)."""
    ctx = P.trals_create(0)
    o2 = P.make_opts(opts.mode, solver=opts.solver, gram=opts.gram, explicit_residual=mode != "fp64")
    plan = P.Plan(ctx, w.I, w.R_fit, X, o2)
    try:
        plan.set_cores(TI.init_cores(seed, w.I, w.R_fit))
        plan.run(ref["sweeps"], use_graph=True)
        torch.cuda.synchronize()
        cores = plan.get_cores()
        hist = plan.residuals()
        r2, x2 = P.trals_residual_explicit(ctx, w.I, w.R_fit, X_full,
                                           [plan.core_dev(n) for n in range(len(w.I))])
    finally:
        plan.close()
        ctx.close()
    res = float(np.sqrt(max(r2, 0.0) / x2))
    angles = [subspace_angle(cores, ref["cores"], n) for n in range(len(w.I))]
    gap = abs(res - float(ref["residuals"][-1]))
    target = float(ref["residuals"][-1]) + 1e-4
    hit = [k + 1 for k, v in enumerate(hist) if np.isfinite(v) and v <= target]
    return {"mode": mode, "sweeps": ref["sweeps"], "residual": res, "oracle_residual": float(ref["residuals"][-1]),
            "gap": gap, "gap_within_1e-4": gap <= 1e-4, "angle_max_rad": max(angles), "angle_per_mode_rad": angles,
            "target_residual": target, "sweeps_to_target": hit[0] if hit else None,
            "oracle_sweeps_to_target": int(np.argmax(ref["residuals"] <= target)) + 1
            if (ref["residuals"] <= target).any() else None}


def e2e_run(P, torch, w, X_dev, opts, seed, sweeps):
    """End to end through trals_decompose with host buffers (pinned X, host cores)."""
    Xh = X_dev.cpu().pin_memory()
    init = TI.init_cores(seed, w.I, w.R_fit)
    ctx = P.trals_create(0)
    cores = [G.copy() for G in init]
    P.trals_decompose(ctx, w.I, w.R_fit, Xh, cores, 1, opts)   # warm (module load, graph)
    cores = [G.copy() for G in init]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = P.trals_decompose(ctx, w.I, w.R_fit, Xh, cores, sweeps, opts)
    dt = time.perf_counter() - t0
    ctx.close()
    core_bytes = sum(G.size * 8 for G in cores)
    return {"value": sweeps / dt, "unit": "sweeps/s", "h2d_bytes_per_step": int((Xh.numel() * Xh.element_size()
                                                                                 + core_bytes) / sweeps),
            "d2h_bytes_per_step": int((core_bytes + 8 * sweeps) / sweeps), "sweeps": sweeps,
            "residual": float(res[-1])}


def serve_run(P, torch, seed, count, budget_bytes, slots, mode="bf16", group_limit=None):
    """The serving workload: `count` TR-ALS requests with Poisson arrivals at 200/s, order uniform in
    3-5, mode sizes uniform in 16-64, ranks uniform in 2-8, FP32 X = TR(N(0,1) cores) + 1e-2 relative
    noise generated on the device from each request's seed, 15 sweeps each, run by the serving loop
    (continuous batching).  X is generated before the clock starts (reported separately); latency is
    arrival -> result back on the host, on the server's clock."""
    reqs = TI.request_stream(seed, count)
    ctx = P.trals_create(0)
    data = []
    t0 = time.perf_counter()
    for q in reqs:
        numel = int(np.prod(q.I))
        cd = [P.core_to_device(G) for G in TI.gaussian_cores(q.seed, q.I, q.R)]
        X = torch.empty(numel, dtype=torch.float32, device="cuda")
        P.trals_reconstruct(ctx, q.I, q.R, cd, X)
        g = torch.Generator(device="cuda")
        g.manual_seed(q.seed)
        noise = torch.randn(numel, generator=g, device="cuda", dtype=torch.float32)
        X.add_(noise * (q.eta * torch.linalg.vector_norm(X) / torch.linalg.vector_norm(noise)))
        del noise
        data.append((X, TI.init_cores(q.seed, q.I, q.R)))
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    ctx.close()
    opts = P.make_opts(mode)
    srv = P.Server(0, hbm_budget_bytes=budget_bytes, max_slots=slots)
    if group_limit is not None:
        srv.set_group_limit(group_limit)
    try:
        tickets = []
        start = time.perf_counter()
        for q, (X, init) in zip(reqs, data):
            delay = start + q.arrival_s - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets.append(srv.submit(q.I, q.R, X, init, q.sweeps, opts))
        out = [srv.wait(t, timeout=900.0) for t in tickets]
        wall = time.perf_counter() - start
        stats = srv.stats()
    finally:
        srv.close()
    bad = [o for o in out if o is None or o[0]["status"] != P.OK]
    lat = np.array([o[0]["done_s"] - o[0]["submit_s"] for o in out if o is not None])
    first = min(o[0]["submit_s"] for o in out)
    last = max(o[0]["done_s"] for o in out)
    fin = np.array([o[2][-1] for o in out if o is not None])
    by_order = {}
    for N in sorted({len(q.I) for q in reqs}):
        lo = np.array([o[0]["done_s"] - o[0]["submit_s"] for q, o in zip(reqs, out) if o is not None and len(q.I) == N])
        by_order[str(N)] = {"requests": int(lo.size), "p50_latency_ms": float(np.percentile(lo, 50) * 1e3),
                            "p99_latency_ms": float(np.percentile(lo, 99) * 1e3)}
    sweeps = sum(q.sweeps for q in reqs)
    return {"requests": count, "failed": len(bad), "p50_latency_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_latency_ms": float(np.percentile(lat, 99) * 1e3), "max_latency_ms": float(lat.max() * 1e3),
            "throughput_req_s": count / (last - first), "sweeps_per_s": sweeps / (last - first),
            "span_s": last - first, "wall_s": wall, "arrival_window_s": reqs[-1].arrival_s,
            "data_generation_s": gen_s, "mode": mode, "slots": slots, "hbm_budget_gb": budget_bytes / 2**30,
            "peak_active": stats["peak_active"], "peak_used_gb": stats["peak_used_bytes"] / 2**30,
            "latency_by_order": by_order,
            "host_start_s_total": stats["host_start_s"], "grouped_requests": stats["grouped_completed"],
            "grouped_steps": stats["grouped_steps"],
            "final_residual_median": float(np.median(fin)),
            "workload": "512 requests, Poisson 200/s, order U{3..5}, sizes U{16..64}, ranks U{2..8}, "
                        "FP32 X = TR + 1e-2 noise, 15 sweeps"}


def cpu_baseline_run(w, seed, budget_s=20.0):
    """The oracle (regular TR-ALS, FP64 NumPy) on host cores: core updates of the same workload,
    as many as fit ~budget_s, scaled to sweeps/s."""
    import oracle as O
    X = TI.make_tensor_host(w, seed, O.tr_full)
    cores = TI.init_cores(seed, w.I, w.R_fit)
    N = len(w.I)
    t0 = time.perf_counter()
    done = 0
    while True:
        n = done % N
        cores[n] = O.als_update(X, cores, n, "chol")
        done += 1
        if time.perf_counter() - t0 > budget_s or done >= 2 * N:
            break
    dt = time.perf_counter() - t0
    return {"value": (done / N) / dt, "unit": "sweeps/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{done} core updates (modes 1..{min(done, N)}) of the same workload, Cholesky NE on the "
                      f"explicit subchain matrix, {dt:.1f} s"}


def _recorded_traffic(config, mode):
    """DRAM bytes per launch of the MTTSP main kernel, per mode, from the committed ncu summary of
    this workload -- or None when the kernel source changed since that capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"mttsp_tc_{config}.md")
    src = os.path.join(ROOT, "paper_2210_11362_gb300", "csrc", "mttsp_tc.cu")
    if mode != "bf16" or not os.path.exists(path):
        return None
    rec = {}
    with open(path) as f:
        for ln in f:
            if ln.startswith("kernel_source_sha256:"):
                rec["sha"] = ln.split(":", 1)[1].strip()
            elif ln.startswith("dram_bytes_per_launch:"):
                rec["bytes"] = [float(v) for v in ln.split(":", 1)[1].split(",")]
    with open(src) as f:
        text = f.read()
    # the kernel and its device helpers precede the host-side planner in the source
    sha = hashlib.sha256(text[:text.index("TcChoice tc_choose(")].encode()).hexdigest()
    if rec.get("sha") != sha or "bytes" not in rec:
        return None
    return rec["bytes"]


def roofline_for(w, mode, kernel_ms, peaks, src, step_ms=None):
    """Roofline of the RHS contraction.  ``frac`` is the main contraction kernel alone (the dominant
    kernel: its CUDA-event time per launch); ``frac_contraction`` is the whole contraction step of a
    core update as ``trals_plan_time_mttsp`` times it (the link of the subchain tables through the
    core updated just before, the kernel, and the FP64 reduction of the per-CTA partials), which is
    the figure the >= 0.60 target of the RHS contraction is compared with."""
    numel = w.numel
    N = len(w.I)
    esize = {"fp64": 8, "fp32": 4, "bf16": 2, "bf16x2": 2, "bf16x3": 4}[mode]
    bytes_per = numel * esize
    flops = [2.0 * numel * w.R_fit[n] * w.R_fit[(n + 1) % N] for n in range(N)]
    t = sum(kernel_ms) * 1e-3          # all N launches
    if mode == "fp64":
        achieved = sum(flops) / t / 1e12
        return {"bound": "alu", "achieved": achieved, "peak": 1.25, "unit": "TFLOP/s",
                "frac": achieved / 1.25, "traffic": None,
                "note": "nominal FP64 1.25 TFLOP/s; the SM's shared FP64 unit issues one warp instruction per "
                        "19 cycles (measured), i.e. 152 x 32/19 x 2 FLOP x 2.07 GHz = 1.06 TFLOP/s"}
    achieved = N * bytes_per / t / 1e9
    peak = peaks["hbm_gbs"]
    tr = _recorded_traffic(w.name, mode)
    out = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
           "traffic": (sum(tr) / len(tr)) if tr else None, "peak_source": f"{src} hbm_gbs (burst copy)",
           "algorithmic_bytes_per_launch": bytes_per, "launch_ms_per_mode": kernel_ms,
           "frac_of": "the main contraction kernel alone (mttsp_tc_kernel), CUDA events on its stream"}
    if step_ms:
        ach_step = N * bytes_per / (sum(step_ms) * 1e-3) / 1e9
        out.update({"achieved_contraction": ach_step, "frac_contraction": ach_step / peak,
                    "contraction_ms_per_mode": step_ms,
                    "frac_contraction_of": "the whole contraction step (last table link + kernel + FP64 "
                                           "partial reduction)"})
    return out


def run_ours(args):
    import torch
    import paper_2210_11362_gb300 as P
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    w = TI.WORKLOADS[args.config]
    peaks, src = _peaks()
    flush = torch.ones(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    out = {}
    X_f64 = make_X_device(w, args.seed, P, torch, torch.float64)
    modes = [args.mode] + ([] if args.mode == "fp64" or args.no_fp64 else ["fp64"])
    if args.mode == "bf16" and not args.no_fp64:
        modes += ["bf16x3", "bf16x2"]   # the compensated split-BF16 variants beside the headline
    # per-config accuracy against the FP64 oracle's stored run, every mode measured below
    ref = oracle_reference(w.name, args.seed)
    for mode in modes:
        X = X_f64 if mode == "fp64" else X_f64.to(mode_xdtype(mode, torch))
        if world > 1:
            torch.distributed.barrier()
        # the FP64 mode beside the headline runs ~90x slower per sweep: a tenth of the steps, except where
        # no oracle run is stored, since its residual is then the reference and must come after as many
        # sweeps as the other modes'
        steps = (args.steps if mode != "fp64" or mode == args.mode or ref is None
                 else max(10, args.steps // 10))
        out[mode] = time_mode(P, torch, w, X, mode, steps, args.warmup, args.seed, flush, X_f64,
                              opts_for(P, mode, args))
        out[mode]["X"] = X
    accuracy = {}
    for mode in out:
        if ref is None:
            accuracy[mode] = {"unavailable": f"no stored oracle run for {w.name} seed {args.seed}"}
            if mode != "fp64" and "fp64" in out and out[mode]["sweeps_run"] == out["fp64"]["sweeps_run"]:
                # too large for the oracle: the gap to the FP64 GPU run of the same solver and sweeps
                accuracy[mode]["gap_vs_fp64_gpu"] = abs(out[mode]["residual"] - out["fp64"]["residual"])
                accuracy[mode]["fp64_gpu_residual"] = out["fp64"]["residual"]
                accuracy[mode]["residual"] = out[mode]["residual"]
                accuracy[mode]["sweeps"] = out[mode]["sweeps_run"]
            continue
        accuracy[mode] = accuracy_run(P, torch, w, out[mode]["X"], X_f64, mode, opts_for(P, mode, args), args.seed,
                                      ref)
        k = accuracy[mode]["sweeps_to_target"]
        # time to the target residual at the timed rate of this mode's sweep
        accuracy[mode]["time_to_target_ms"] = k * out[mode]["ms_per_step"] if k else None
    main = out[args.mode]
    ms = main["ms_per_step"]
    if world > 1:
        ms = max_over_ranks(ms, "cuda")
    if rank != 0:
        return
    e2e = e2e_run(P, torch, w, main["X"], opts_for(P, args.mode, args), args.seed, w.sweeps)
    line = {
        "metric": METRIC,
        "value": job_rate(ms, world), "unit": "sweeps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "bf16": "bf16", "bf16x2": "bf16x2", "bf16x3": "bf16x3"}[args.mode],
        "data": "synthetic",
        "config": workload_config(w),
        "variant": {"mode": args.mode, "solver": args.solver, "gram": args.gram,
                    "parallelism": "replicas" if world > 1 else "single"},
        "l2": "inputs larger than L2 (204.8 MB of X per core update) and L2 evicted between timed sweeps by a "
              "256 MB read", "residual_after_run": main["residual"],
        "roofline": roofline_for(w, args.mode, main["mttsp_kernel_ms"], peaks, src, main["mttsp_ms"]),
        "mttsp_ms_per_mode": main["mttsp_ms"],
        "gpu_launches": main["launches_per_sweep"] * args.steps,
        "clocks": main["clocks"],
        "e2e": e2e,
        "accuracy": {w.name: accuracy},
    }
    if "fp64" in out and args.mode != "fp64":
        f = out["fp64"]
        line["fp64"] = {"value": 1000.0 / f["ms_per_step"], "ms_per_step": f["ms_per_step"], "steps": len(f["times"]),
                        "residual": f["residual"], "mttsp_ms_per_mode": f["mttsp_ms"],
                        "roofline": roofline_for(w, "fp64", f["mttsp_kernel_ms"], peaks, src)}
        line["speedup_vs_fp64"] = f["ms_per_step"] / main["ms_per_step"]
    for v in ("bf16x3", "bf16x2"):
        if v in out and args.mode != v:
            b = out[v]
            line[v] = {"value": 1000.0 / b["ms_per_step"], "ms_per_step": b["ms_per_step"], "steps": len(b["times"]),
                       "residual": b["residual"], "mttsp_ms_per_mode": b["mttsp_ms"],
                       "roofline": roofline_for(w, v, b["mttsp_kernel_ms"], peaks, src, b["mttsp_ms"])}
    if not args.no_smooth and args.config == "tr40x5_r8-12":
        for k in list(out):
            out[k].pop("X", None)
        X = X_f64 = None
        torch.cuda.empty_cache()
        line["smooth_qr"] = smooth_qr_run(P, torch, args.seed, peaks, flush)
    if not args.no_serve:
        for k in list(out):
            out[k].pop("X", None)
        X = X_f64 = flush = None
        torch.cuda.empty_cache()
        line["serving"] = serve_run(P, torch, args.seed, args.serve_requests, int(args.serve_budget_gb * 2**30),
                                    args.serve_slots, group_limit=args.serve_group_limit)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_run(w, args.seed, args.cpu_budget)
    print(json.dumps(line))


STABILITY_SOLVERS = {"ne_cholesky": 0, "qr_stabilised": 1, "qrne": 2, "qr_compressed": 3}


def run_stability(args):
    """The ill-conditioned stability experiments of Sec. 4 (B-II: collinearity-controlled cores; B-III:
    multivariate-t cores with correlation theta^|i-j|, one degree of freedom): 100 x 100 x 100 tensors
    generated as TR with 5 x 100 x 5 cores, relative noise eta, fitted with ranks 5 from a Gaussian init
    for 20 sweeps in FP64 by every solver; the final relative residual (explicit, against the FP64 X) of
    `--trials` seeded trials per point of the grid, summarised by median and spread.  A solver that stops
    (a non-positive Cholesky pivot) counts as a failure."""
    import torch
    import paper_2210_11362_gb300 as P
    I, R = (100, 100, 100), (5, 5, 5)
    etas = [1e-4, 1e-7, 1e-10]
    grids = {"collinear_gamma": [1 - 1e-4, 1 - 1e-7, 1 - 1e-10], "mvt_theta": [1 - 1e-1, 1 - 1e-4, 1 - 1e-7]}
    ctx = P.trals_create(0)
    out = {}
    t_start = time.perf_counter()
    for exp, levels in grids.items():
        for lev in levels:
            for eta in etas:
                key = f"{exp}={lev:.10g},eta={eta:g}"
                per = {k: [] for k in STABILITY_SOLVERS}
                fails = {k: 0 for k in STABILITY_SOLVERS}
                for t in range(args.trials):
                    seed = 1000 + t
                    if exp == "collinear_gamma":
                        truth = TI.collinear_cores(seed, I, R, lev)
                    else:
                        truth = TI.multivariate_t_cores(seed, I, R, lev, dof=1.0)
                    cd = [P.core_to_device(G) for G in truth]
                    Xt = torch.empty(int(np.prod(I)), dtype=torch.float64, device="cuda")
                    P.trals_reconstruct(ctx, I, R, cd, Xt)
                    noise = torch.from_numpy(TI.flat_f(TI.gaussian_noise(seed, I))).to("cuda")
                    X = Xt + eta * (torch.linalg.vector_norm(Xt) / torch.linalg.vector_norm(noise)) * noise
                    init = TI.init_cores(seed, I, R)
                    for name, solver in STABILITY_SOLVERS.items():
                        cores = [G.copy() for G in init]
                        try:
                            P.trals_decompose(ctx, I, R, X, cores, 20, P.make_opts("fp64", solver=solver))
                            r2, x2 = P.trals_residual_explicit(ctx, I, R, X, [P.core_to_device(G) for G in cores])
                            res = float(np.sqrt(max(r2, 0.0) / x2))
                            if np.isfinite(res):
                                per[name].append(res)
                            else:
                                fails[name] += 1
                        except P.TralsError:
                            fails[name] += 1
                out[key] = {name: {"median": float(np.median(v)) if v else None,
                                   "q25": float(np.percentile(v, 25)) if v else None,
                                   "q75": float(np.percentile(v, 75)) if v else None,
                                   "worst": float(max(v)) if v else None, "failed": fails[name], "runs": len(v)}
                            for name, v in per.items()}
    ctx.close()
    print(json.dumps({"experiment": "stability (Sec. 4, Exp. B-II and B-III)", "tensor": list(I), "ranks": list(R),
                      "sweeps": 20, "trials": args.trials, "dtype": "f64", "wall_s": time.perf_counter() - t_start,
                      "results": out}))


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle as O
    w = TI.WORKLOADS[args.config]
    X = TI.make_tensor_host(w, args.seed, O.tr_full)
    cores = TI.init_cores(args.seed, w.I, w.R_fit)
    N = len(w.I)
    for k in range(args.warmup):
        cores[k % N] = O.als_update(X, cores, k % N, "chol")
    t = []
    for k in range(args.steps):
        n = (args.warmup + k) % N
        t0 = time.perf_counter()
        cores[n] = O.als_update(X, cores, n, "chol")
        t.append(time.perf_counter() - t0)
    per_update = sum(t) / len(t)
    value = 1.0 / (N * per_update)
    # one timed step is one core update: ms_per_step x steps is the timed region
    line = {"impl": "reference", "metric": METRIC,
            "value": value, "unit": "sweeps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * per_update, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w),
            "step": "one core update of the CPU oracle per timed step (sweeps/s = 1 / (N x mean update time))",
            "cpu_baseline": {"value": value, "unit": "sweeps/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{args.steps} timed core updates after {args.warmup} warm-up updates"},
            "e2e": {"value": value, "unit": "sweeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="tr40x5_r8-12", choices=sorted(TI.WORKLOADS))
    ap.add_argument("--mode", default="bf16", choices=["fp64", "fp32", "bf16", "bf16x2", "bf16x3"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-smooth", action="store_true",
                    help="skip the 256x256x3x256 QR-solver sub-line of the default workload")
    ap.add_argument("--solver", default="cholesky", choices=sorted(SOLVERS))
    ap.add_argument("--gram", default="structured", choices=sorted(GRAMS))
    ap.add_argument("--serve-requests", type=int, default=512)
    ap.add_argument("--serve-slots", type=int, default=16)
    ap.add_argument("--serve-budget-gb", type=float, default=64.0)
    ap.add_argument("--serve-group-limit", type=int, default=None,
                    help="largest request (entries) served by the grouped step engine (default: the server's)")
    ap.add_argument("--serve-only", action="store_true", help="run only the serving workload and print its line")
    ap.add_argument("--stability", action="store_true",
                    help="run the ill-conditioned stability experiments (Sec. 4, B-II and B-III) instead")
    ap.add_argument("--trials", type=int, default=10)
    args = ap.parse_args()
    if args.stability:
        run_stability(args)
        return
    if args.serve_only:
        import torch
        import paper_2210_11362_gb300 as P
        print(json.dumps({"serving": serve_run(P, torch, args.seed, args.serve_requests,
                                                int(args.serve_budget_gb * 2**30), args.serve_slots,
                                                group_limit=args.serve_group_limit)}))
        return
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
