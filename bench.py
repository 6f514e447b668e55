#!/usr/bin/env python
"""Benchmark of the GB300 LOBPCG hot path.

A step is one LOBPCG iteration (Section 2.2 of the BLOPEX paper: residual,
V-cycle preconditioner, Cholesky orthonormalisation of W and P, stencil SpMV, Gram matrices,
Rayleigh-Ritz, Ritz update) over the whole block.  Default workload: the paper's 10^8-unknown scale,
the 7-point Dirichlet Laplacian on a 464^3 interior grid (99,897,344 unknowns), m = 8 eigenpairs,
8-level V-cycle.  The JSON line's value is the float64 form; the mixed form (float32 / bfloat16
blocks, double-float X, float64 Rayleigh-Ritz and correction sweep) is timed the same way and
reported beside it.  The timed steps run with tol = 0 so that every column stays active (fixed work
per step); the time to reach tol = 1e-8 is measured separately for both forms, with the
per-eigenpair relative errors against the closed-form eigenvalues of the discrete Laplacian.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload c4]

Prints one JSON line (rank 0).  With N > 1 (torchrun, one process per GPU) every rank solves an
independent replica with its own seed ("replicas only": the solver has no data-path collective);
`value` is the total iterations of all ranks / the slowest rank's time.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LOBPCG time-to-tol (s) & iters/s, 7-pt Laplacian, m eigenpairs; HBM % of peak"

WORKLOADS = {
    "c1": dict(dims=(48, 48, 48), m=8, levels=4),
    "c2": dict(dims=(128, 128, 128), m=16, levels=6),
    "c3": dict(dims=(256, 256, 256), m=32, levels=7),
    "c4": dict(dims=(464, 464, 464), m=8, levels=8),
    # the 464^3 workload's block size on a 128^3 grid (the size the per-kernel ncu captures use)
    "s4": dict(dims=(128, 128, 128), m=8, levels=6),
}

# Time to tol: seeded starts, and timed solves per seed after one warm-up solve (medians over
# both); fewer timed solves on the two largest grids.
TTT_SEEDS = (2, 3, 4)
TTT_RUNS = {"c1": 5, "c2": 5, "c3": 3, "c4": 3, "s4": 3}

# The oracle's bounded sample for the CPU figures: one oracle iteration on a grid of the same m and
# V-cycle whose point count the host finishes in seconds; the figure is scaled to the workload by
# the ratio of point counts (every step of an iteration is O(n) at fixed m).
CPU_SAMPLE = {"c1": "c1", "c2": "c2", "c3": "s3", "c4": "s4", "s4": "s4"}
SAMPLES = {"s3": dict(dims=(96, 96, 96), m=32, levels=5), "s4": dict(dims=(128, 128, 128), m=8, levels=6)}

# FP64 peak of GB300 from unit counts and clocks: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12


def _measured_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (copy bandwidth, measured)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


HBM_PEAK_GBS, HBM_PEAK_SOURCE = _measured_hbm()

# DRAM traffic of the Gram phase (k_oz_exponents + k_gram_oz, the Gram matrices of the Rayleigh-Ritz basis) per iteration, from one
# ncu capture on the 128^3 grid (its first-iteration Gram, q = 16 columns: read + write of both
# launches) scaled by the columns (24 / 16) and the points (464^3 / 128^3) to the workload, keyed
# by the SHA-256 of k_gram_oz.cu and oz_digits.cuh; a changed source invalidates it (traffic = null;
# the key was renewed twice, after edits of comments only).
NCU_TRAFFIC = {("c4", "3591edfac0184e1b"): (536.889600e6 + 3.006976e6 + 537.195776e6 + 2.186752e6) * (24 / 16) *
               99897344 / 2097152}

# DRAM traffic of one update launch of k_tsmm_oz (the Ritz update, 3m columns in, 2m out), from one
# ncu capture of the same launches on the 128^3 grid (mean of the X-side and A-side launch: read +
# write; up to ~50 MB of the writes were still in L2 at the end of the small launch) scaled by the
# points to the workload, keyed by the SHA-256 of k_tsmm_oz.cu and oz_digits.cuh (traffic = null
# after an edit of either).
NCU_TRAFFIC_UPDATE = {("c4", "e790013c613854da"): ((402.801920e6 + 402.797824e6) / 2 + (216.686080e6 + 215.953664e6) / 2) *
                      99897344 / 2097152}


def closed_form_eigenvalues(dims, scale, m):
    """The m smallest eigenvalues of the scaled 7-point Dirichlet Laplacian, scale * sum over the
    axes of 4 sin^2(i pi / (2 (n + 1))) (the paper's Section 4.1 formula), ascending."""
    import math
    axes = [[4.0 * math.sin(i * math.pi / (2.0 * (n + 1))) ** 2 for i in range(1, min(n, m) + 1)] for n in dims]
    vals = sorted(scale * (a + b + c) for a in axes[0] for b in axes[1] for c in axes[2])
    return vals[:m]


def rel_errors(lam, dims, m):
    nx, ny, nz = dims
    scale = float(nx + 1) ** 2 if nx == ny == nz else 1.0
    exact = closed_form_eigenvalues(dims, scale, m)
    return [abs(a - b) / abs(b) for a, b in zip(lam, exact)]


def workload_desc(w):
    d = WORKLOADS[w]
    n = d["dims"][0] * d["dims"][1] * d["dims"][2]
    return (f"7-point Dirichlet Laplacian {d['dims'][0]}x{d['dims'][1]}x{d['dims'][2]} ({n:,} unknowns), "
            f"m={d['m']}, {d['levels']}-level GMG V-cycle (2+2 weighted Jacobi, w=2/3); float64 form timed, "
            f"mixed form beside it")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"], samples=0)
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(smax) if smax else None,
                    reasons=sorted(reasons), samples=len(sm))


def gram_flops_per_launch(n, m):
    """Algorithmic flops of the Gram matrices of the Rayleigh-Ritz basis at b = m: upper triangles of gramA and gramB, q = 3m."""
    q = 3 * m
    return 2.0 * n * 2 * (q * (q + 1) // 2)


def gram_bytes_per_launch(n, m):
    """Compulsory bytes of the Gram matrices of the Rayleigh-Ritz basis at b = m: the float64 blocks [X W P] and [AX AW AP]
    (q = 3m columns each) read once, (2m + 4b) * 8 bytes per point."""
    return 2.0 * 3 * m * 8 * n


def source_hash(*names):
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_0705_2626_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def update_bytes_per_launch(n, m):
    """Compulsory bytes of one update launch (the Ritz update, Section 2.2) at b = m: the 3m input
    columns read once, the 2m outputs (X and P, or AX and AP) written once, 8 bytes each."""
    return (3 * m + 2 * m) * 8.0 * n


def kernel_source_hash():
    """Hash of k_gram_oz.cu and oz_digits.cuh (the float64 Gram on the tensor cores, its exponent
    pass and its digit split), the key under which the Gram phase's ncu DRAM traffic is recorded:
    an edit of either file invalidates it."""
    h = hashlib.sha256()
    for name in ("k_gram_oz.cu", "oz_digits.cuh"):
        with open(os.path.join(ROOT, "paper_0705_2626_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def level_points(dims, levels):
    out, d = [], tuple(dims)
    for _ in range(levels):
        out.append(d[0] * d[1] * d[2])
        d = tuple(x // 2 for x in d)
    return out


def vcycle_bytes(dims, levels, b, s0, sc):
    """Compulsory bytes of one V-cycle on b columns as the library runs it: per level above the
    coarsest, 14 passes over level vectors (fused first two pre-sweeps 2, residual 3, restriction
    read 1, prolongation read+write 2, two post-sweeps 6) plus the coarse vector written and
    read once (2 x 1/8); the coarsest level is read and written once.  s0: bytes per value on
    level 0, sc: on coarser levels."""
    pts = level_points(dims, levels)
    total = 0.0
    for l, n_l in enumerate(pts):
        s_l = s0 if l == 0 else sc
        if l == len(pts) - 1:
            total += n_l * b * 2 * s_l
        else:
            total += n_l * b * (14 * s_l + 2 * sc / 8)
    return total


def hbm_frac(nbytes, ms):
    gbs = nbytes / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
    return dict(bytes=nbytes, ms=ms, achieved_gbs=gbs, peak_gbs=HBM_PEAK_GBS, frac=gbs / HBM_PEAK_GBS)


def cpu_baseline_sample(w, iters=1):
    """The oracle (numpy/scipy float64) timed on this host for `iters` iterations of workload (or
    sample grid) w."""
    import numpy as np  # noqa: F401
    from oracle import lobpcg as olob, multigrid, rng
    d = WORKLOADS[w] if w in WORKLOADS else SAMPLES[w]
    A = olob.Laplace7(d["dims"])
    T = multigrid.VCycle(d["dims"], A.scale, d["levels"])
    X0 = rng.uniform_block(2, A.n, d["m"])
    marks = []
    # iters + 1 passes; the spacing of the pass ends excludes the set-up and pass 0
    # (pass 0 has no P block)
    olob.lobpcg(A, X0, 0.0, iters + 1, T=T, on_pass=lambda k: marks.append(time.perf_counter()))
    per = (marks[-1] - marks[0]) / (len(marks) - 1)
    return 1.0 / per, per


def cpu_single_thread_sample(w, iters=1):
    """cpu_baseline_sample with one thread for every library call (BLAS, OpenMP): run in a child
    process whose thread-count variables are set before numpy loads.  Returns (iters/s, s per
    iteration), or None if the child fails."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               BLIS_NUM_THREADS="1", VECLIB_MAXIMUM_THREADS="1", NUMEXPR_NUM_THREADS="1")
    code = ("import json, bench; print(json.dumps(bench.cpu_baseline_sample(%r, %d)))" % (w, iters))
    try:
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                           timeout=1800)
        ips, per = json.loads(r.stdout.strip().splitlines()[-1])
        return float(ips), float(per)
    except (subprocess.SubprocessError, ValueError, IndexError, OSError):
        return None


def max_over_ranks(x, world, device):
    """The largest x over the ranks of the default process group (x itself when world = 1)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(steps, world, t_ms):
    """Iterations per second of the whole job: each of the `world` ranks (an independent replica)
    ran `steps` iterations, and the job took the slowest rank's time t_ms."""
    return world * steps / (t_ms / 1e3)


def time_to_tol_over_seeds(solve, seeds, runs):
    """Time to tol 1e-8 (solve only; setup reported apart) from the seeded starts `seeds`:
    solve(seed) runs one solve and returns the solver's result dict.  One warm-up solve (first
    seed), then per seed the median of `runs` solves; the headline figures are the medians over
    the seeds (the random start moves the iteration count by 10-20 %), the worst residual and
    status over all of them.  Returns (the first timed result, the summary)."""
    per_seed, first = [], None
    solve(seeds[0])
    for sd in seeds:
        rs = [solve(sd) for _ in range(runs)]
        first = first or rs[0]
        per_seed.append(dict(seed=sd, time_to_tol_s=statistics.median(r["solve_ms"] for r in rs) / 1e3,
                             setup_s=statistics.median(r["setup_ms"] for r in rs) / 1e3,
                             iters=rs[0]["iters"], fp64_checks=rs[0]["fp64_sweeps"], status=rs[0]["status_name"],
                             max_rel_resid=max(r["max_rel_resid"] for r in rs)))
    t = statistics.median(p["time_to_tol_s"] for p in per_seed)
    iters = statistics.median(p["iters"] for p in per_seed)
    bad = [p["status"] for p in per_seed if p["status"] != "ok"]
    return first, dict(time_to_tol_s=t, setup_s=statistics.median(p["setup_s"] for p in per_seed),
                       iters=iters, iters_per_s=iters / t, status=bad[0] if bad else "ok",
                       max_rel_resid=max(p["max_rel_resid"] for p in per_seed),
                       fp64_checks=max(p["fp64_checks"] for p in per_seed), tol=1e-8,
                       seeds=[p["seed"] for p in per_seed], runs_per_seed=runs, per_seed=per_seed)


def cpu_sample_desc(w):
    """(sample key, its point count, scale factor to workload w, text)."""
    key = CPU_SAMPLE[w]
    d = WORKLOADS[key] if key in WORKLOADS else SAMPLES[key]
    n_s = d["dims"][0] * d["dims"][1] * d["dims"][2]
    wd = WORKLOADS[w]["dims"]
    n_w = wd[0] * wd[1] * wd[2]
    dims = "x".join(map(str, d["dims"]))
    if n_s == n_w:
        return key, n_s, 1.0, f"oracle LOBPCG iteration on the workload itself ({dims}, m={d['m']})"
    return key, n_s, n_s / n_w, (f"oracle LOBPCG iteration on {dims}, m={d['m']}, {d['levels']} levels (same m), "
                                 f"iters/s scaled to the workload by the point-count ratio {n_s}/{n_w}")


def run_reference(args, rank, world):
    """The oracle on the host cores: W warm-up steps and K timed steps, each step one oracle
    iteration on the bounded sample grid of the workload (scaled to its iters/s)."""
    if rank != 0:
        return
    import numpy as np  # noqa: F401
    from oracle import lobpcg as olob, multigrid, rng
    w = args.workload
    key, n_s, factor, text = cpu_sample_desc(w)
    d = WORKLOADS[key] if key in WORKLOADS else SAMPLES[key]
    A = olob.Laplace7(d["dims"])
    T = multigrid.VCycle(d["dims"], A.scale, d["levels"])
    X0 = rng.uniform_block(2, A.n, d["m"])
    marks = []
    # the set-up and pass 0 (no P block) are not steps; then W + K timed passes
    olob.lobpcg(A, X0, 0.0, args.warmup + args.steps + 1, T=T, on_pass=lambda k: marks.append(time.perf_counter()))
    timed = marks[args.warmup:]
    per = (timed[-1] - timed[0]) / args.steps
    ips = factor / per
    cores = os.cpu_count()
    single = cpu_single_thread_sample(key, iters=1) if w in ("c1", "c2", "c4") else None
    wd = WORKLOADS[w]
    line = dict(impl="reference", metric=METRIC, value=ips, unit="iters/s", n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 / ips, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic",
                config=dict(workload=workload_desc(w), grid=list(wd["dims"]), m=wd["m"], levels=wd["levels"]),
                cpu_baseline=dict(value=ips, unit="iters/s", cores=cores, kind="oracle",
                                  sample=f"each step one {text} (numpy elementwise ops single-threaded, "
                                         "BLAS calls multi-threaded)"),
                e2e=dict(value=ips, unit="iters/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    if single is not None:
        line["cpu_baseline"]["single_thread"] = dict(value=single[0] * factor, unit="iters/s", cores=1,
                                                     sample="1 " + text + ", every library call on one thread")
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import ctypes

    import torch
    import torch.distributed as dist
    from paper_0705_2626_gb300 import capi
    from paper_0705_2626_gb300.solver import Solver

    w = args.workload
    d = WORKLOADS[w]
    dims, m, levels = d["dims"], d["m"], d["levels"]
    n = dims[0] * dims[1] * dims[2]
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    seed = 2 + rank

    def barrier():
        if world > 1:
            dist.barrier()

    def rank_max(x):
        return max_over_ranks(x, world, dev)

    def timed_form(precision, sampler=None):
        """K iterations with every column active (tol = 0), inputs resident in HBM; then the same
        K iterations again with the library's per-phase events for the kernel rooflines."""
        s = Solver(dims, levels=levels, device=local_rank, precision=precision)
        s.begin(m, tol=0.0, seed=seed)
        s.iterate(args.warmup)
        barrier()
        torch.cuda.synchronize(dev)
        if sampler:
            sampler.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        s.iterate(args.steps)
        e1.record(s.stream)
        e1.synchronize()
        torch.cuda.synchronize(dev)
        barrier()
        clocks = sampler.stop() if sampler else None
        launches = int(s.info.kernel_launches)
        t_ms = rank_max(e0.elapsed_time(e1))
        s.set_options(phase_timing=True)
        s.begin(m, tol=0.0, seed=seed)
        s.iterate(args.warmup)
        before = list(s.info.phase_ms)
        s.iterate(args.steps)
        after = list(s.info.phase_ms)
        s.set_options(phase_timing=False)
        phase = {nm: (after[i] - before[i]) / args.steps for i, nm in enumerate(capi.PHASE_NAMES)}
        return s, t_ms, launches, phase, clocks

    def time_to_tol(s):
        return time_to_tol_over_seeds(
            lambda sd: s.solve(m, tol=1e-8, maxit=300, seed=sd, with_vectors=False),
            [x + len(TTT_SEEDS) * rank for x in TTT_SEEDS], TTT_RUNS[w])

    # ---- float64 form: the timed steps of the JSON line
    sampler = ClockSampler(local_rank)
    s64, t64, launches, ph64, clocks = timed_form("fp64", sampler)
    value = replica_throughput(args.steps, world, t64)
    gram_ms = ph64["gram"]
    achieved = gram_bytes_per_launch(n, m) / (gram_ms * 1e-3) / 1e9
    fp64_equiv = gram_flops_per_launch(n, m) / (gram_ms * 1e-3) / 1e12
    traffic = NCU_TRAFFIC.get((w, kernel_source_hash()))
    upd_launch_ms = ph64["update"] / 2                 # the update phase is two launches of k_tsmm_oz
    upd_achieved = update_bytes_per_launch(n, m) / (upd_launch_ms * 1e-3) / 1e9
    upd_traffic = NCU_TRAFFIC_UPDATE.get((w, source_hash("k_tsmm_oz.cu", "oz_digits.cuh")))
    out64, ttt64 = time_to_tol(s64)

    # ---- end to end through the public API with host buffers (float64 form): X0 from pinned
    # host memory in, eigenvalues and eigenvectors back to pinned host memory, K iterations
    X0 = torch.empty((m, n), dtype=torch.float64).pin_memory()
    X0.uniform_(-1.0, 1.0, generator=torch.Generator().manual_seed(seed))
    Xout = torch.empty((m, n), dtype=torch.float64).pin_memory()
    barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    s64.set_initial(X0)
    s64.solve(m, tol=0.0, maxit=args.steps, seed=seed)
    lam = (ctypes.c_double * m)()
    capi.lobpcg_get_eigenpairs(s64.h, lam, ctypes.c_void_p(Xout.data_ptr()), n, 1, None)
    t_e2e = rank_max(time.perf_counter() - t0)
    e2e = dict(value=replica_throughput(args.steps, world, t_e2e * 1e3), unit="iters/s",
               h2d_bytes_per_step=n * m * 8 / args.steps, d2h_bytes_per_step=(n * m * 8 + m * 8) / args.steps,
               note="set_initial(pinned host X0) + solve(tol=0, maxit=K) + get_eigenpairs(to pinned host), wall clock")
    s64.close()
    del X0, Xout
    torch.cuda.empty_cache()

    # ---- mixed form (float32 / bfloat16 blocks, double-float X, float64 sweep)
    smx, tmx, launches_mx, phmx, _ = timed_form("mixed")
    outmx, tttmx = time_to_tol(smx)
    smx.close()
    torch.cuda.empty_cache()
    lam_diff = max(abs(a - b) / abs(b) for a, b in zip(outmx["lam"], out64["lam"]))

    # ---- per-phase HBM fractions from the phase events (all m columns active, b = m)
    q = 3 * m

    def frac(nbytes, ms):
        return round(hbm_frac(nbytes, ms)["frac"], 3)

    kern64 = dict(residual=frac(3 * 8 * n * m, ph64["residual"]), spmv=frac(2 * 8 * n * m, ph64["spmv"]),
                  vcycle=frac(vcycle_bytes(dims, levels, m, 8, 8), ph64["precond"]),
                  gram=frac(2 * q * 8 * n, ph64["gram"]), update=frac((2 * q + 4 * m) * 8 * n, ph64["update"]))
    kernmx = dict(residual=frac(3 * 4 * n * m, phmx["residual"]), spmv=frac(2 * 4 * n * m, phmx["spmv"]),
                  vcycle=frac(vcycle_bytes(dims, levels, m, 4, 2), phmx["precond"]),
                  gram=frac((2 * q + 2 * m) * 4 * n, phmx["gram"]),
                  update=frac((2 * m + 2 * m + 3 * m) * 4 * n, phmx["update"]))

    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        key, _, factor, text = cpu_sample_desc(w)
        ips, per = cpu_baseline_sample(key, iters=1)
        cpu = dict(value=ips * factor, unit="iters/s", cores=os.cpu_count(), kind="oracle",
                   sample="1 " + text + " (numpy elementwise single-threaded, BLAS multi-threaded)")

    def rnd(x, k=4):
        return float(f"{x:.{k}g}")

    def ttt_brief(t, out):
        return dict(time_to_tol_s=rnd(t["time_to_tol_s"]), iters=t["iters"], iters_per_s=rnd(t["iters_per_s"]),
                    status=t["status"], max_rel_resid=rnd(t["max_rel_resid"], 3), fp64_checks=t["fp64_checks"],
                    setup_s=rnd(t["setup_s"]),
                    per_seed=[[p["seed"], rnd(p["time_to_tol_s"]), p["iters"]] for p in t["per_seed"]],
                    rel_err_vs_closed_form=[rnd(e, 2) for e in rel_errors(out["lam"], dims, m)])

    line = dict(
        metric=METRIC, value=value, unit="iters/s", n_gpus=world, steps=args.steps, warmup=args.warmup,
        ms_per_step=t64 / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
        dtype="f64", data="synthetic",
        config=dict(workload=workload_desc(w), grid=list(dims), m=m, levels=levels, tol_timed=0.0,
                    l2=f"no flush: the 6 stored blocks are {6 * n * m * 8 / 1e9:.1f} GB, far above the 129 MB L2",
                    parallelism="replicas" if world > 1 else "single-gpu"),
        time_to_tol=dict(tol=1e-8, seeds=list(TTT_SEEDS), runs_per_seed=TTT_RUNS[w],
                         fp64=ttt_brief(ttt64, out64), mixed=ttt_brief(tttmx, outmx),
                         mixed_speedup=rnd(ttt64["time_to_tol_s"] / tttmx["time_to_tol_s"], 3),
                         max_rel_lambda_diff_mixed_vs_fp64=rnd(lam_diff, 2)),
        roofline=dict(kernel="k_tsmm_oz, one update launch (the Ritz update, Section 2.2: float64 [X W P] C or "
                             "[AX AW AP] C by bfloat16 digit products on the tensor cores; the top kernel of the "
                             "launch list)", bound="hbm",
                      achieved=upd_achieved, peak=HBM_PEAK_GBS, unit="GB/s", frac=upd_achieved / HBM_PEAK_GBS,
                      traffic=upd_traffic, algorithmic_bytes=update_bytes_per_launch(n, m),
                      launch_ms=upd_launch_ms, peak_source=HBM_PEAK_SOURCE),
        roofline_gram=dict(kernel="Gram phase, the Gram matrices of the Rayleigh-Ritz basis: k_oz_exponents + "
                                  "k_gram_oz + k_gram_finalize (float64 Gram by bfloat16 digit products on the "
                                  "tensor cores)", bound="hbm",
                           achieved=achieved, peak=HBM_PEAK_GBS, unit="GB/s", frac=achieved / HBM_PEAK_GBS,
                           traffic=traffic, algorithmic_bytes=gram_bytes_per_launch(n, m),
                           peak_source=HBM_PEAK_SOURCE, fp64_equiv_tflops=fp64_equiv,
                           fp64_pipe_tflops=FP64_PEAK_TFLOPS),
        mixed=dict(value=replica_throughput(args.steps, world, tmx), unit="iters/s", ms_per_step=tmx / args.steps,
                   dtype="f64+f32+bf16", gpu_launches=launches_mx,
                   phase_ms=dict((k, rnd(v)) for k, v in phmx.items()), hbm_frac=kernmx),
        phase_ms=dict((k, rnd(v)) for k, v in ph64.items()), hbm_frac=kern64, hbm_peak_gbs=HBM_PEAK_GBS,
        hbm_peak_source=HBM_PEAK_SOURCE,
        cpu_baseline=cpu, e2e=e2e, gpu_launches=launches, clocks=clocks)
    print(json.dumps(line), flush=True)


def run_inner_pcg_sweep(args):
    """Section 4.2's experiment on this workload: float64 time to tol 1e-8 and outer iterations
    against the number of inner PCG iterations (0 = the V-cycle applied directly); one JSON line."""
    import torch
    from paper_0705_2626_gb300.solver import Solver

    d = WORKLOADS[args.workload]
    dims, m, levels = d["dims"], d["m"], d["levels"]
    torch.cuda.set_device(0)
    s = Solver(dims, levels=levels)
    s.solve(m, tol=1e-8, maxit=300, seed=2, with_vectors=False)        # warm-up
    rows = []
    for k in [int(x) for x in args.inner_pcg_sweep.split(",")]:
        s.set_inner_pcg(k)
        best = None
        for rep in range(3):
            out = s.solve(m, tol=1e-8, maxit=300, seed=2, with_vectors=False)
            t = out["solve_ms"] / 1e3
            best = t if best is None else min(best, t)
        rows.append(dict(inner_iters=k, time_to_tol_s=best, outer_iters=out["iters"], status=out["status_name"],
                         max_rel_resid=out["max_rel_resid"]))
    s.close()
    print(json.dumps(dict(metric="time to tol 1e-8 vs inner PCG iterations (float64)", config=workload_desc(args.workload),
                          rows=rows)))


def run_block_size_sweep(args):
    """Section 4.3's experiment on this grid: seconds per iteration (every column active) and time
    to tol 1e-8 against the block size m, the float64 form up to m = 100 and the mixed form up to
    its limit of 32 columns; one JSON line."""
    import torch
    from paper_0705_2626_gb300.solver import LobpcgError, Solver

    d = WORKLOADS[args.workload]
    dims, levels = d["dims"], d["levels"]
    torch.cuda.set_device(0)
    rows = []
    for m in [int(x) for x in args.m_sweep.split(",")]:
        for precision in ("fp64", "mixed"):
            if precision == "mixed" and m > 32:
                continue
            s = Solver(dims, levels=levels, precision=precision)
            s.begin(m, tol=0.0, seed=2)
            s.iterate(3)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s.stream)
            s.iterate(10)
            e1.record(s.stream)
            e1.synchronize()
            ms_it = e0.elapsed_time(e1) / 10
            row = dict(m=m, precision=precision, ms_per_iter=ms_it, ms_per_iter_per_col=ms_it / m)
            try:
                out = s.solve(m, tol=1e-8, maxit=300, seed=2, with_vectors=False)
                row.update(time_to_tol_s=out["solve_ms"] / 1e3, iters=out["iters"], status=out["status_name"])
            except LobpcgError as e:     # a breakdown of the method (Section 2.2) ends this row only
                row.update(time_to_tol_s=None, iters=None, status=str(e))
            rows.append(row)
            print(json.dumps(row), file=sys.stderr, flush=True)
            s.close()
            torch.cuda.empty_cache()
    print(json.dumps(dict(metric="ms per iteration and time to tol 1e-8 vs block size m",
                          config=workload_desc(args.workload), rows=rows)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c4", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--inner-pcg-sweep", default=None,
                    help="comma-separated inner PCG iteration counts: print that sweep instead of the bench line")
    ap.add_argument("--m-sweep", default=None,
                    help="comma-separated block sizes: print that sweep instead of the bench line")
    args = ap.parse_args()
    if args.m_sweep:
        run_block_size_sweep(args)
        return
    if args.inner_pcg_sweep:
        run_inner_pcg_sweep(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
