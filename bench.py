#!/usr/bin/env python3
"""Throughput of the 2D Walsh -> boundary-wavelet products on GB300.

Metric: (U x + U^* y) pairs per second at N = 4096^2 (Daubechies p = 8 with
vanishing-moments-preserving boundaries, M = 2048^2, q = 1, radial
multilevel sampling of 12% of the Walsh coefficients, seed 4).  One step is
one forward product and one adjoint product (the whole path: IDWT,
upsample-convolve, FWHT, selection, and the transposed chain).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision f32|split_bf16|f64] [--compare split_bf16]
    python bench.py --impl reference      # the CPU oracle on the host cores

The headline precision is FP32 on the CUDA cores (the fastest path within
the 1e-5 accuracy bar on this GPU); the same pair is then timed in split-BF16
on the tensor cores and reported under "comparison".

Under torchrun every rank runs its own replica on its own GPU (the product is
independent per instance: weak scaling, no collective on the data path); the
timed region is bracketed by a barrier and a device synchronisation, and the
slowest rank sets the time.  Prints one JSON line on rank 0.
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

R, Q, P, FRAC, SEED = 11, 1, 8, 0.12, 4
METRIC = "2D U·x+U*·y pairs/s at N=4096²; split-BF16 TC vs FP32; % of HBM roofline"
WORKLOAD = ("2D Daubechies p=8 VMP, M=2048^2 -> N=4096^2 (R=11, q=1), radial multilevel 12% mask "
            "(m=2013266), x level-decaying alpha=1.5, y ~ N(0,1), seed 4")


def aggregate_over_ranks(total_ms, steps, world, dist=None, device="cpu"):
    """Replicas: every rank timed its own `steps` pairs; the job's time is the
    slowest rank's, and the job processed steps * world pairs in it.
    Returns (pairs per second over all ranks, the slowest rank's ms)."""
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return steps * world / (total_ms / 1000.0), total_ms


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return d["hbm_gbs"], "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash(kernel=""):
    """First 16 hex digits of the SHA-256 of the sources that define `kernel`
    and its launch, in name order: for the line operators whose names end in
    _f32 / _tc, their own file (kernels_f32.cu / kernels_tc.cu) and
    line_common.cuh; for any other kernel, every file under csrc/."""
    csrc = os.path.join(ROOT, "paper_2106_00554_gb300", "csrc")
    if kernel.endswith("_f32"):
        files = ["kernels_f32.cu", "line_common.cuh"]
    elif kernel.endswith("_tc"):
        files = ["kernels_tc.cu", "line_common.cuh"]
    else:
        files = os.listdir(csrc)
    h = hashlib.sha256()
    for f in sorted(files):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum)
    of `kernel` from the committed ncu summary profiles/traffic.md, if its
    counters were taken on the current sources of that kernel (the summary
    records kernel_source_hash(name)); None otherwise.  Rows: | name | bytes | hash |."""
    path = os.path.join(ROOT, "profiles", "traffic.md")
    try:
        lines = open(path).read().splitlines()
    except Exception:
        return None
    cur = kernel_source_hash(kernel)
    for ln in lines:
        f = [c.strip().strip("`") for c in ln.strip().strip("|").split("|")]
        if len(f) >= 3 and f[0] == kernel and f[2] == cur:
            try:
                return float(f[1])
            except ValueError:
                return None
    return None


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.dev)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"),
                               f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------
# the CPU oracle (reference arm, cpu_baseline, oracle timings)
#
# Everything here runs in a child process (`bench.py --cpu-oracle ...`) with
# no GPU visible and one BLAS thread per process; the all-core measurements
# spread Algorithm 1's lines over a process pool started with `spawn`.  The
# oracle's own functions do every step; nothing here changes its arithmetic.
# ----------------------------------------------------------------------------
CPU_ENV = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1",
           "CUDA_VISIBLE_DEVICES": ""}


def host_cpu():
    """(cores usable by this process, CPU model name from lscpu)."""
    try:
        cores = len(os.sched_getaffinity(0))
    except Exception:
        cores = os.cpu_count() or 1
    model = "unknown"
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return cores, model


def _alg1_lines(args):
    """Pool worker: the oracle's Algorithm 1 on a block of lines."""
    direction, lines, R_, q, p = args
    from oracle import fast, wavelets as W
    f = fast.alg1_forward if direction == "fwd" else fast.alg1_adjoint
    return f(lines, R_, q, p, W.VMP)


def _vector_pair(args):
    """Pool worker: one 1D forward and adjoint product of the oracle."""
    x, y, R_, q, p, J0, omega = args
    from oracle import fast, wavelets as W
    return fast.forward1d(x, R_, q, p, W.VMP, J0, omega), fast.adjoint1d(y, R_, q, p, W.VMP, J0, omega)


def _map_lines(pool, direction, A, R_, q, p, workers):
    import numpy as np
    if pool is None:
        return _alg1_lines((direction, A, R_, q, p))
    chunks = np.array_split(A, 4 * workers, axis=0)
    return np.concatenate(pool.map(_alg1_lines, [(direction, c, R_, q, p) for c in chunks]), axis=0)


def oracle_pair_2d(pool, workers, x, y, R_, q, p, J0, omega):
    """One forward and one adjoint product of Algorithm 2 (the Mallat IDWT /
    DWT in this process, Algorithm 1 on every line of both passes, in the
    pool when there is one).  Returns (y, x) of the pair."""
    import numpy as np
    from oracle import fast, wavelets as W
    N = 2 ** (R_ + q)
    xi = fast.idwt2d(x, J0, p, W.VMP)
    t = _map_lines(pool, "fwd", xi, R_, q, p, workers)                         # rows: M x N
    a = _map_lines(pool, "fwd", np.ascontiguousarray(t.T), R_, q, p, workers).T  # columns: N x N
    y_out = a.reshape(N * N)[omega]
    A = np.zeros(N * N)
    A[omega] = y
    t = _map_lines(pool, "adj", A.reshape(N, N), R_, q, p, workers)             # rows: N x M
    xi = _map_lines(pool, "adj", np.ascontiguousarray(t.T), R_, q, p, workers).T  # columns: M x M
    return y_out, fast.dwt2d(xi, J0, p, W.VMP)


def _spawn_pool(workers):
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(workers)


def cpu_oracle_reference(steps, warmup, budget_s=300.0):
    """The reference arm: every step one whole pair of Algorithm 2 at the
    benchmark workload on all host cores.  If whole pairs would not fit the
    time budget, each step takes Algorithm 1 on a sample of lines instead and
    says so."""
    import numpy as np
    from oracle import fast, wavelets as W
    from paper_2106_00554_gb300 import inputs
    cores, model = host_cpu()
    rng = np.random.default_rng(SEED)
    N = 2 ** (R + Q)
    omega = inputs.mask_2d(rng, N, FRAC)
    J0 = W.default_J0(P)
    x = inputs.coeffs_2d(rng, R, J0, 1.5)
    y = rng.standard_normal(omega.size)
    fast.alg1_forward(np.zeros((1, 2 ** R)), R, Q, P, W.VMP)          # oracle tables
    pool = _spawn_pool(cores)
    try:
        pool.map(_alg1_lines, [("fwd", np.zeros((1, 2 ** R)), R, Q, P)] * cores)   # workers' tables
        t0 = time.perf_counter()
        oracle_pair_2d(pool, cores, x, y, R, Q, P, J0, omega)
        first = time.perf_counter() - t0
        times, walls = [], []                       # pair time (extrapolated if sampled), step wall time
        if first * (steps + warmup) <= budget_s:
            for s in range(1, steps + warmup):
                t0 = time.perf_counter()
                oracle_pair_2d(pool, cores, x, y, R, Q, P, J0, omega)
                if s >= warmup:
                    times.append(time.perf_counter() - t0)
            if warmup == 0:
                times.insert(0, first)
            walls = list(times)
            how = "whole pairs"
            sample = (f"every step one whole pair of the oracle's Algorithm 2 at N=4096^2 (Mallat IDWT + "
                      f"DWT in one process, Algorithm 1 on all 6144 lines of both passes spread over "
                      f"{cores} processes); CPU {model}")
        else:
            # as many lines per step as fit the step's share of the budget (a
            # multiple of the cores, at least 2 per core), so the pool's
            # per-call overhead is not multiplied up by the extrapolation
            M = 2 ** R
            per_step = budget_s / max(1, steps + warmup)
            L = int((M + N) * per_step / max(first, 1e-9)) // cores * cores
            L = max(2 * cores, min(L, M + N))
            t_ana = 0.0
            t0 = time.perf_counter()
            S = fast.idwt2d(x, J0, P, W.VMP)
            fast.dwt2d(S, J0, P, W.VMP)
            t_ana = time.perf_counter() - t0
            for s in range(steps + warmup):
                xi = rng.standard_normal((L, M))
                al = rng.standard_normal((L, N))
                t0 = time.perf_counter()
                _map_lines(pool, "fwd", xi, R, Q, P, cores)
                _map_lines(pool, "adj", al, R, Q, P, cores)
                t = time.perf_counter() - t0
                if s >= warmup:
                    times.append(t_ana + (M + N) / L * t)
                    walls.append(t)
            how = "sampled"
            sample = (f"whole pairs would exceed {budget_s:.0f} s: the Mallat IDWT + DWT once, then per step "
                      f"Algorithm 1 forward and adjoint on {L} lines over {cores} processes, scaled to the "
                      f"6144 lines of a pair (extrapolated); CPU {model}")
    finally:
        pool.close()
        pool.join()
    return {"pair_s": statistics.median(times), "step_s": times, "step_wall_s": walls, "cores": cores,
            "model": model, "how": how, "sample": sample}


def cpu_oracle_baseline():
    """cpu_baseline (two whole pairs of Algorithm 2 at the benchmark workload
    on all host cores) and the oracle timings: the dense oracle at the 1D
    configuration of 2048 x 1024 (forming U, then the products, one thread),
    and the O(N log N) oracle (Algorithm 1 / 2) on one thread and on all
    cores at that configuration, at the batched 1D configuration and at the
    benchmark workload."""
    import numpy as np
    from oracle import dense, fast, wavelets as W
    from paper_2106_00554_gb300 import inputs
    cores, model = host_cpu()
    out = {"cores": cores, "cpu_model": model}
    # dense, configuration 1: p = 2 VMP, M = 2^10, q = 1, J0 = 3, all 2048 Walsh rows
    rng = np.random.default_rng(0)
    t0 = time.perf_counter()
    U = dense.U1d(10, 1, 2, W.VMP, 3)
    t_form = time.perf_counter() - t0
    x1 = inputs.coeffs_1d(rng, 10, 3, 1.0)
    y1 = inputs.gaussian(rng, 2048)
    reps = 200
    t0 = time.perf_counter()
    for _ in range(reps):
        U @ x1
        U.T @ y1
    t_dense = (time.perf_counter() - t0) / reps
    t0 = time.perf_counter()
    for _ in range(20):
        fast.forward1d(x1, 10, 1, 2, W.VMP, 3)
        fast.adjoint1d(y1, 10, 1, 2, W.VMP, 3)
    t_fast1 = (time.perf_counter() - t0) / 20
    out["config1_dense"] = {"formation_s": t_form, "pair_s": t_dense, "pairs_per_s": 1.0 / t_dense, "threads": 1,
                            "what": "U = H_N T W^{-1} formed from the definitions (2048 x 1024, FP64), then "
                                    "U x and U^T y"}
    out["config1_fast"] = {"pairs_per_s_1thread": 1.0 / t_fast1, "pair_s": t_fast1,
                           "all_cores": "not applicable: one vector of one line"}
    # configuration 2: p = 4, M = 2^16, q = 2, 15% multilevel mask, batch 64 (seed 1)
    rng = np.random.default_rng(1)
    R2, q2, p2 = 16, 2, 4
    om2 = inputs.mask_1d(rng, 2 ** (R2 + q2), 0.15)
    J2 = W.default_J0(p2)
    xs = inputs.coeffs_1d(rng, R2, J2, 1.5, batch=64)
    ys = rng.standard_normal((64, om2.size))
    fast.forward1d(xs[:1], R2, q2, p2, W.VMP, J2, om2)
    t0 = time.perf_counter()
    for b in range(2):
        fast.forward1d(xs[b], R2, q2, p2, W.VMP, J2, om2)
        fast.adjoint1d(ys[b], R2, q2, p2, W.VMP, J2, om2)
    t_c2 = (time.perf_counter() - t0) / 2
    pool = _spawn_pool(cores)
    try:
        pool.map(_vector_pair, [(xs[0], ys[0], R2, q2, p2, J2, om2)] * cores)     # workers' tables
        nv = min(64, cores)
        t0 = time.perf_counter()
        pool.map(_vector_pair, [(xs[b], ys[b], R2, q2, p2, J2, om2) for b in range(nv)])
        t_c2p = time.perf_counter() - t0
        out["config2_fast"] = {"pairs_per_s_1thread": 1.0 / t_c2,
                               "pairs_per_s_all_cores": nv / t_c2p, "cores": cores,
                               "sample": f"1 thread: 2 of the 64 vector pairs; all cores: {nv} vector pairs, one "
                                         f"per process"}
        # configuration 5 / the benchmark workload
        rng = np.random.default_rng(SEED)
        N = 2 ** (R + Q)
        omega = inputs.mask_2d(rng, N, FRAC)
        J0 = W.default_J0(P)
        x = inputs.coeffs_2d(rng, R, J0, 1.5)
        y = rng.standard_normal(omega.size)
        pool.map(_alg1_lines, [("fwd", np.zeros((1, 2 ** R)), R, Q, P)] * cores)
        times = []
        for _ in range(2):
            t0 = time.perf_counter()
            oracle_pair_2d(pool, cores, x, y, R, Q, P, J0, omega)
            times.append(time.perf_counter() - t0)
    finally:
        pool.close()
        pool.join()
    t_all = statistics.median(times)
    # one thread: the Mallat IDWT + DWT once, Algorithm 1 on 64 lines per direction, scaled
    M = 2 ** R
    t0 = time.perf_counter()
    S = fast.idwt2d(x, J0, P, W.VMP)
    fast.dwt2d(S, J0, P, W.VMP)
    t_ana = time.perf_counter() - t0
    L = 64
    xi = rng.standard_normal((L, M))
    al = rng.standard_normal((L, N))
    t0 = time.perf_counter()
    fast.alg1_forward(xi, R, Q, P, W.VMP)
    fast.alg1_adjoint(al, R, Q, P, W.VMP)
    t_l = (time.perf_counter() - t0) / L
    t_one = t_ana + (M + N) * t_l
    out["config5_fast"] = {"pairs_per_s_1thread": 1.0 / t_one, "pairs_per_s_all_cores": 1.0 / t_all,
                           "cores": cores,
                           "sample": "all cores: two whole pairs of Algorithm 2 (median); 1 thread: the Mallat "
                                     "IDWT + DWT once and Algorithm 1 on 64 lines per direction, scaled to "
                                     "the 6144 lines of a pair"}
    baseline = {"value": 1.0 / t_all, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                "sample": (f"two whole pairs of the oracle's Algorithm 2 at N=4096^2 (median of {len(times)}): "
                           f"Mallat IDWT + DWT in one process, Algorithm 1 on all 6144 lines of both passes "
                           f"over {cores} processes; CPU {model}")}
    return {"cpu_baseline": baseline, "oracle_timings": out}


def run_cpu_oracle(what, steps, warmup):
    """Run one CPU oracle measurement in a child process with no GPU visible
    and one BLAS thread per process; returns its JSON result."""
    env = dict(os.environ, **CPU_ENV)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--cpu-oracle", what,
                        "--steps", str(steps), "--warmup", str(warmup)],
                       cwd=ROOT, env=env, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_reference(args):
    """The reference arm: the CPU oracle on the host cores (rank 0 only)."""
    rank, _, world = env_rank()
    if rank != 0:
        return
    t0 = time.perf_counter()
    d = run_cpu_oracle("reference", args.steps, args.warmup)
    wall = time.perf_counter() - t0
    v = 1.0 / d["pair_s"]
    # ms_per_step: the measured time of one timed step (a whole pair, or the
    # sample of lines; the value is then the extrapolated pair rate)
    walls = d.get("step_wall_s") or d["step_s"]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "pairs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * statistics.median(walls),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": "f64 (CPU oracle)", "steps_timed": d["how"],
                       "timed_region_s": round(sum(walls), 2), "wall_s": round(wall, 1)},
            "cpu_baseline": {"value": v, "unit": "pairs/s", "cores": d["cores"], "kind": "oracle",
                             "sample": d["sample"]},
            "e2e": {"value": v, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# the CUDA path
# ----------------------------------------------------------------------------
def _graph_of(fn, stream):
    """fn captured as a CUDA graph (after one eager call on a side stream)."""
    import torch
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        fn()
    stream.wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    torch.cuda.synchronize()
    return g


def _time_replays(g, k, stream, flush):
    """Mean ms of one replay over k replays, each bracketed by CUDA events on
    `stream`, with an L2 flush between replays outside the events."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
    for _ in range(3):
        g.replay()
        flush.fill_(0)
    torch.cuda.synchronize()
    for i, (a, b) in enumerate(ev):
        a.record(stream)
        g.replay()
        b.record(stream)
        flush.fill_(i)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / k


def measure_workload_1d(steps, flush, peak):
    """The batched 1D workload: Daubechies p = 4 VMP, M = 2^16, q = 2
    (N = 2^18), multilevel 15% mask (m = 39322), a batch of 64 level-decaying
    x (alpha = 1.5) and 64 y ~ N(0,1), seed 1.  One step is the forward and
    adjoint product of the whole batch (64 vector pairs), captured as one CUDA
    graph; FP32 (headline) and FP64.  Roofline of the dominant kernel and of
    the batch against the compulsory bytes (x, y and the mask, both ways)."""
    import numpy as np
    import torch
    from paper_2106_00554_gb300 import F32, F64, VMP, Plan, _lib, inputs
    rng = np.random.default_rng(1)
    R1, q1, p1, B = 16, 2, 4, 64
    N1 = 2 ** (R1 + q1)
    om = inputs.mask_1d(rng, N1, 0.15)
    plan = Plan(1, R1, q1, p1, VMP, omega=om, max_batch=B)
    x_np = inputs.coeffs_1d(rng, R1, plan.J0, 1.5, batch=B)
    y_np = rng.standard_normal((B, om.size))
    stream = torch.cuda.current_stream()
    out = {"workload": ("1D Daubechies p=4 VMP, M=2^16 -> N=2^18 (R=16, q=2), multilevel 15% mask (m=39322), "
                        "batch 64, x level-decaying alpha=1.5, y ~ N(0,1), seed 1"),
           "unit": "pairs/s", "batch": B, "launch": "cuda graph of the batch's pair",
           "l2": "flushed between timed steps"}
    for prec, name in ((F32, "f32"), (F64, "f64")):
        dt = torch.float64 if prec == F64 else torch.float32
        esize = 8 if prec == F64 else 4
        x = torch.tensor(x_np, dtype=dt, device="cuda")
        yin = torch.tensor(y_np, dtype=dt, device="cuda")
        y = torch.empty((B, plan.m), dtype=dt, device="cuda")
        xo = torch.empty_like(x)

        def step():
            plan.forward(x, y, precision=prec)
            plan.adjoint(yin, xo, precision=prec)

        g = _graph_of(step, stream)
        k = max(5, min(steps, 100))
        ms = _time_replays(g, k, stream, flush)
        _lib.uw_plan_profile(plan._h, True)
        for i in range(5):
            step()
            flush.fill_(i)
        torch.cuda.synchronize()
        prof = [e for e in _lib.uw_plan_profile_read(plan._h) if e["launches"] > 0]
        _lib.uw_plan_profile(plan._h, False)
        dom = max(prof, key=lambda e: e["total_ms"])
        avg_ms = dom["total_ms"] / dom["launches"]
        words = (N1 + 31) // 32
        comp = 2 * B * (plan.coeffs * esize + plan.m * esize) + 2 * 8 * words
        out[name] = {"value": B * 1000.0 / ms, "ms_per_step": ms, "compulsory_bytes_per_step": comp,
                     "frac_compulsory": comp / (ms / 1000.0) / 1e9 / peak,
                     "dominant_kernel": {"name": dom["name"], "avg_us": 1000.0 * avg_ms,
                                         "achieved_GBps": dom["bytes_per_launch"] / (avg_ms / 1000.0) / 1e9,
                                         "frac": dom["bytes_per_launch"] / (avg_ms / 1000.0) / 1e9 / peak},
                     "kernels": {e["name"]: round(1000.0 * e["total_ms"] / e["launches"], 2) for e in prof}}
    out["value"] = out["f32"]["value"]
    plan.close()
    return out


def measure_fista(plan, flush):
    """The reconstruction of the benchmark workload: 100 FISTA iterations of
    min ||P_Omega U x - y||^2 / 2 + lam ||x||_1 (lam = 1e-3) from
    y = P_Omega U x_true + 1e-3 noise, x_true level-decaying (alpha = 1.5) with
    5% nonzeros (seed 4).  Timed without gradients, and with the gradient of
    1/2 ||x_100 - x_true||^2 with respect to lam and y through checkpointed
    iterations; split-BF16 and FP32 products."""
    import numpy as np
    import torch
    from paper_2106_00554_gb300 import F32, F32_SPLIT_BF16, inputs, solvers
    rng = np.random.default_rng(SEED + 100)
    xt = torch.tensor(inputs.sparse_coeffs_2d(rng, R, plan.J0, 1.5, 0.05), dtype=torch.float32, device="cuda")
    y = plan.forward(xt, precision=F32) + 1e-3 * torch.tensor(rng.standard_normal(plan.m), dtype=torch.float32,
                                                              device="cuda")
    iters = 100
    out = {"iterations": iters, "lam": 1e-3, "unit": "iterations/s",
           "what": "one iteration = U z, U^* of it, and the fused proximal step with momentum"}
    for prec, name in ((F32_SPLIT_BF16, "split_bf16"), (F32, "f32")):
        with torch.no_grad():
            solvers.fista(plan, y, 1e-3, iters=2, precision=prec, checkpoint=False)
            torch.cuda.synchronize()
            flush.fill_(0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            x = solvers.fista(plan, y, 1e-3, iters=iters, precision=prec, checkpoint=False)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
        yv = y.clone().requires_grad_(True)
        lt = torch.tensor(1e-3, dtype=torch.float64, device="cuda", requires_grad=True)
        flush.fill_(1)
        torch.cuda.synchronize()
        e0.record()
        xg = solvers.fista(plan, yv, lt, iters=iters, precision=prec, checkpoint=True)
        loss = solvers.half_sq_dist(xg, xt)
        loss.backward()
        e1.record()
        torch.cuda.synchronize()
        ms_g = e0.elapsed_time(e1)
        rel = float(torch.linalg.norm((x - xt).double()) / torch.linalg.norm(xt.double()))
        out[name] = {"value": iters * 1000.0 / ms, "ms_solve": ms, "ms_solve_and_gradient": ms_g,
                     "gradient_iterations_per_s": iters * 1000.0 / ms_g, "rel_error_to_x_true": rel}
    out["value"] = out["split_bf16"]["value"]
    return out


def run_ours(args):
    import numpy as np
    import torch

    rank, local, world = env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2106_00554_gb300 import F32, F32_SPLIT_BF16, F64, VMP, Plan, _lib, build, inputs
    build.build()
    PREC = {"f32": F32, "split_bf16": F32_SPLIT_BF16, "f64": F64}
    DTYPE = {F32: "f32", F32_SPLIT_BF16: "bf16 split (3 parts per operand), f32 accumulate", F64: "f64"}

    rng = np.random.default_rng(SEED)
    N = 2 ** (R + Q)
    omega = inputs.mask_2d(rng, N, FRAC)
    plan = Plan(2, R, Q, P, VMP, omega=omega)
    x_np = inputs.coeffs_2d(rng, R, plan.J0, 1.5)
    y_np = rng.standard_normal(omega.size)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    def measure(prec, sample_clocks):
        dt = torch.float64 if prec == F64 else torch.float32
        x = torch.tensor(x_np, dtype=dt, device="cuda")
        yin = torch.tensor(y_np, dtype=dt, device="cuda")
        y = torch.empty(plan.m, dtype=dt, device="cuda")
        xo = torch.empty_like(x)

        def step():
            plan.forward(x, y, precision=prec)
            plan.adjoint(yin, xo, precision=prec)

        for _ in range(args.warmup):
            step()
            flush.fill_(1)
        torch.cuda.synchronize()
        # the pair as one CUDA graph (18 launches); eager if the capture is refused
        graph, graph_error = None, None
        if not args.eager:
            try:
                side = torch.cuda.Stream()
                side.wait_stream(stream)
                with torch.cuda.stream(side):
                    step()
                stream.wait_stream(side)
                torch.cuda.synchronize()
                graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(graph):
                    step()
                for _ in range(3):
                    graph.replay()
                torch.cuda.synchronize()
            except Exception as e:  # noqa: BLE001 - reported in the JSON line
                graph = None
                graph_error = f"{type(e).__name__}: {e}"[:200]
        plan.forward(x, y, precision=prec)
        n_fwd = plan.last_launches
        plan.adjoint(yin, xo, precision=prec)
        n_adj = plan.last_launches
        torch.cuda.synchronize()

        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        clk = ClockSampler(local) if sample_clocks else None
        if clk:
            clk.start()
            time.sleep(0.3)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        launches = 0
        for k in range(args.steps):
            starts[k].record(stream)
            if graph is not None:
                graph.replay()
            else:
                step()
            launches += n_fwd + n_adj
            ends[k].record(stream)
            flush.fill_(k)                   # L2 flush between timed steps (not timed)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        clocks = clk.stop() if clk else None
        value, total_ms = aggregate_over_ranks(sum(s.elapsed_time(e) for s, e in zip(starts, ends)), args.steps,
                                               world, dist, "cuda")
        # per-kernel device times: the same pair launched eagerly with the
        # library's event profiler on (events on the launching stream)
        kp = max(3, min(args.steps, 300))
        _lib.uw_plan_profile(plan._h, True)
        for k in range(kp):
            step()
            flush.fill_(k)
        torch.cuda.synchronize()
        prof = [e for e in _lib.uw_plan_profile_read(plan._h) if e["launches"] > 0]
        _lib.uw_plan_profile(plan._h, False)
        launch = ("cuda graph of the pair" if graph is not None else
                  ("eager" if args.eager else f"eager (graph capture failed: {graph_error})"))
        return {"value": value, "ms": total_ms / args.steps, "prof": prof, "kp": kp, "launches": launches,
                "clocks": clocks, "launch": launch}

    prec = PREC[args.precision]
    main_m = measure(prec, True)
    comp_m = None
    if args.compare and args.compare != args.precision:
        comp_m = measure(PREC[args.compare], False)
    esize = 8 if prec == F64 else 4

    # end to end through the host-buffer entry points (copies inside)
    e2e = None
    if not args.no_e2e:
        dt = torch.float64 if prec == F64 else torch.float32
        xh = torch.tensor(x_np, dtype=dt).pin_memory()
        yh = torch.empty(plan.m, dtype=dt).pin_memory()
        yinh = torch.tensor(y_np, dtype=dt).pin_memory()
        xoh = torch.empty_like(xh).pin_memory()
        # two output sets: the pipelined calls of consecutive steps are in flight together
        yh2 = [yh, torch.empty_like(yh).pin_memory()]
        xoh2 = [xoh, torch.empty_like(xoh).pin_memory()]
        # the pipelined calls fill and drain the copy pipeline once per timed
        # run (the first upload and the last download overlap no product):
        # time at least 50 pairs so that this is a small part of the figure
        ke = max(50, min(args.steps, 200))

        def sync_pairs(n):
            for _ in range(n):
                plan.forward_host(xh.data_ptr(), yh.data_ptr(), prec, 1)
                plan.adjoint_host(yinh.data_ptr(), xoh.data_ptr(), prec, 1)

        def pipelined_pairs(n):
            for i in range(n):
                plan.forward_host_async(xh.data_ptr(), yh2[i % 2].data_ptr(), prec, 1)
                plan.adjoint_host_async(yinh.data_ptr(), xoh2[i % 2].data_ptr(), prec, 1)
            plan.host_wait()

        def timed(fn):
            fn(3)
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            t0 = time.perf_counter()
            fn(ke)
            v, _ = aggregate_over_ranks(1000.0 * (time.perf_counter() - t0), ke, world, dist, "cuda")
            return v

        sync_value = timed(sync_pairs)
        e2e_value = timed(pipelined_pairs)
        nbx = plan.coeffs * esize
        nby = plan.m * esize
        e2e = {"value": e2e_value, "unit": "pairs/s", "h2d_bytes_per_step": nbx + nby,
               "d2h_bytes_per_step": nby + nbx, "steps": ke, "sync_value": sync_value,
               "how": "uw_forward_host_async + uw_adjoint_host_async from pinned host buffers, then "
                      "uw_host_wait: every step copies x and y in and y and x out; uploads and downloads "
                      "overlap the neighbouring steps' products (two staging slots); the products run as "
                      "the graphs the library captures at the first call; the first upload and the last "
                      "download of the timed run overlap nothing. sync_value: the blocking "
                      "uw_forward_host + uw_adjoint_host, one call at a time"}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel (event timings of this run)
    peak, peak_kind = peaks()
    prof = main_m["prof"]
    dom = max(prof, key=lambda e: e["total_ms"])
    avg_ms = dom["total_ms"] / max(1, dom["launches"])
    achieved = dom["bytes_per_launch"] / (avg_ms / 1000.0) / 1e9
    traffic = ncu_traffic(dom["name"])
    kernels = {e["name"]: {"launches": e["launches"], "avg_us": 1000.0 * e["total_ms"] / max(1, e["launches"]),
                           "share": e["total_ms"] / sum(z["total_ms"] for z in prof),
                           "GBps": e["bytes_per_launch"] / (e["total_ms"] / max(1, e["launches"]) / 1000) / 1e9}
               for e in prof}
    value = main_m["value"]
    words = N * ((N + 31) // 32)
    comp = 2 * (plan.coeffs * esize + plan.m * esize + 8 * words)      # both directions
    twopass = comp + 2 * 2 * (2 ** R) * N * esize
    line = {
        "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": main_m["ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[prec], "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": args.precision, "batch": 1,
                   "launch": main_m["launch"],
                   "kernel_times": f"library event profiler over {main_m['kp']} further eager pairs",
                   "l2": "flushed between timed steps by a 256 MiB device write outside the event pair",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "kernel": dom["name"], "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "traffic_source": ("profiles/traffic.md: dram__bytes_read.sum + dram__bytes_write.sum of this "
                                        "kernel from a committed ncu capture of the same bench workload, taken on "
                                        "the kernel's current sources (source hash " + kernel_source_hash(dom["name"])
                                        + "); not measured in this run" if traffic is not None else
                                        "no committed ncu capture of this kernel's current sources"),
                     "peak_kind": (f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                                   else "fallback 6.8 TB/s")},
        "pipeline_roofline": {"compulsory_bytes_per_pair": comp, "two_pass_bytes_per_pair": twopass,
                              "frac_compulsory": value * comp / 1e9 / peak,
                              "frac_two_pass": value * twopass / 1e9 / peak},
        "kernels": kernels,
        "gpu_launches": main_m["launches"],
        "clocks": main_m["clocks"],
    }
    if comp_m:
        line["comparison"] = {"precision": args.compare, "dtype": DTYPE[PREC[args.compare]],
                              "value": comp_m["value"], "unit": "pairs/s", "ms_per_step": comp_m["ms"],
                              "launch": comp_m["launch"], "speedup_of_main": value / comp_m["value"]}
    if e2e:
        line["e2e"] = e2e
    if not args.no_extra:
        line["fista"] = measure_fista(plan, flush)
        line["workload_1d"] = measure_workload_1d(args.steps, flush, peak)
    if not args.no_cpu_baseline:
        cb = run_cpu_oracle("baseline", 0, 0)
        line["cpu_baseline"] = cb["cpu_baseline"]
        line["oracle_timings"] = cb["oracle_timings"]
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_uneven(args):
    """The batched uneven workload (instances of R in 6..9, q in 1..2,
    p in {1,2,4,6,8}, either boundary, alpha in [1, 2], 10-40% masks, seed 3):
    one plan per instance in a plan group, tuned, its forward + adjoint pair
    captured as one CUDA graph; pairs/s over all instances, and the same plans
    issued one after another on one stream for comparison.  One JSON line."""
    import numpy as np
    import torch
    from paper_2106_00554_gb300 import F32, F32_SPLIT_BF16, PERIODIC, VMP, Plan, PlanGroup, inputs
    if args.precision not in ("f32", "split_bf16"):
        raise SystemExit("--uneven runs FP32 or split-BF16 (float buffers)")
    prec = F32 if args.precision == "f32" else F32_SPLIT_BF16
    torch.cuda.set_device(0)
    rng = np.random.default_rng(3)
    t0 = time.perf_counter()
    # the library's default coarsest level per p (levels below J0 + 1 have no detail level)
    j0 = {}
    for p in (1, 2, 4, 6, 8):
        probe = Plan(1, 10, 0, p, VMP)
        j0[p] = probe.J0
        probe.close()
    plans, xd, yd = [], [], []
    for _ in range(args.uneven):
        p = int(rng.choice([1, 2, 4, 6, 8]))
        R_ = int(rng.choice([r for r in (6, 7, 8, 9) if r >= j0[p] + 1]))
        q = int(rng.choice([1, 2]))
        bd = int(rng.choice([PERIODIC, VMP]))
        omega = inputs.mask_2d(rng, 2 ** (R_ + q), float(rng.uniform(0.1, 0.4)))
        pl = Plan(2, R_, q, p, bd, omega=omega)
        plans.append(pl)
        xd.append(torch.tensor(inputs.coeffs_2d(rng, R_, pl.J0, float(rng.uniform(1.0, 2.0))),
                               dtype=torch.float32, device="cuda"))
        yd.append(torch.tensor(rng.standard_normal(pl.m), dtype=torch.float32, device="cuda"))
    setup_s = time.perf_counter() - t0
    yo = [torch.empty_like(y) for y in yd]
    xo = [torch.empty_like(x) for x in xd]
    nst = 16
    group = PlanGroup(plans, nstreams=nst)
    t0 = time.perf_counter()
    group.tune([x.clone() for x in xd], [torch.empty_like(y) for y in yd], prec, reps=2)
    tune_s = time.perf_counter() - t0
    prm = group.params()
    s = torch.cuda.Stream()

    def capture():
        with torch.cuda.stream(s):
            group.forward(xd, yo, prec, stream=s)
            group.adjoint(yd, xo, prec, stream=s)
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            group.forward(xd, yo, prec, stream=s)
            group.adjoint(yd, xo, prec, stream=s)
        return g

    def timed(fn, k):
        # everything on stream s: graph replays launch on the current stream,
        # and the events must bracket them on the same stream
        with torch.cuda.stream(s):
            for _ in range(max(3, args.warmup)):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(k):
                fn()
            e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    k = max(3, min(args.steps, 50))
    graph = capture()
    ms_graph = timed(graph.replay, k)
    assert group.device_status() == 0
    in_use = prec == F32 and prm["persistent_in_use"] == 1
    other = None
    if prec == F32 and prm["persistent_available"] == 1:   # the path the tuner did not keep, for comparison
        var = "UW_GROUP_STREAMS" if in_use else "UW_GROUP_PERSISTENT"
        os.environ[var] = "1"
        g2 = capture()
        other = timed(g2.replay, k)
        del os.environ[var]
        assert group.device_status() == 0
    group.close()

    def sequential():
        with torch.cuda.stream(s):
            for pl, x, y, a, b in zip(plans, xd, yd, yo, xo):
                pl.forward(x, a, precision=prec, stream=s)
                pl.adjoint(y, b, precision=prec, stream=s)

    ms_seq = timed(sequential, max(3, k // 5))
    n = len(plans)
    # compulsory bytes of one step: x, the packed y, the mask bits and prefix, both directions
    comp = sum(2 * (4 * pl.coeffs + 4 * pl.m + 8 * pl.N * ((pl.N + 31) // 32)) for pl in plans)
    peak, peak_kind = peaks()
    launch = ("one persistent launch per direction (tasks of (instance, phase, items) drained by one grid), "
              "captured with its counter reset as one CUDA graph" if in_use else
              f"plan group forked over {nst} streams, captured as one CUDA graph")
    line = {
        "metric": f"batched uneven 2D U x + U* y pairs/s ({n} instances)", "value": n * 1000.0 / ms_graph,
        "unit": "pairs/s", "higher_is_better": True, "ms_per_step": ms_graph, "steps": k,
        "dtype": "f32" if prec == F32 else "bf16 split (3 parts per operand), f32 accumulate",
        "data": "synthetic",
        "config": {"workload": f"{n} instances: R in 6..9, q in 1..2, p in {{1,2,4,6,8}}, periodic or VMP, "
                               "alpha in [1,2], 10-40% radial multilevel masks, seed 3",
                   "launch": launch, "tuned": {k2: v for k2, v in prm.items()},
                   "setup_s": round(setup_s, 2), "tune_s": round(tune_s, 2)},
        "roofline": {"bound": "hbm", "achieved": comp / (ms_graph / 1000.0) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": comp / (ms_graph / 1000.0) / 1e9 / peak, "bytes_per_step": comp,
                     "model": "compulsory: x, packed y, mask bits and row prefix of every instance, both directions",
                     "peak_kind": peak_kind},
        "sequential": {"value": n * 1000.0 / ms_seq, "unit": "pairs/s", "ms_per_step": ms_seq,
                       "how": "each plan's forward and adjoint issued in turn on one stream, eager"}}
    if other is not None:
        name = "forked_streams" if in_use else "persistent"
        how = (f"the same group forked over {nst} streams, captured as one CUDA graph" if in_use else
               "the same group as one persistent launch per direction with the tuned parameters, captured")
        line[name] = {"value": n * 1000.0 / other, "unit": "pairs/s", "ms_per_step": other, "how": how}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--eager", action="store_true", help="launch the timed steps without a CUDA graph")
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--compare", default="split_bf16",
                    help="second precision timed the same way (the headline's own name, or '', to skip)")
    ap.add_argument("--precision", default=os.environ.get("UW_BENCH_PRECISION", "f32"),
                    choices=["f32", "split_bf16", "f64"])
    ap.add_argument("--R", type=int, default=R,
                    help="level per dimension (default 11 = the benchmark workload; smaller only for profiling)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the FISTA and 1D workload measurements that ride along the main line")
    ap.add_argument("--workload-1d", action="store_true",
                    help="instead of the benchmark workload: only the batched 1D workload's measurement, one JSON line")
    ap.add_argument("--uneven", type=int, default=0,
                    help="instead of the benchmark workload: the batched uneven workload with this many instances")
    ap.add_argument("--cpu-oracle", default="", choices=["", "reference", "baseline"],
                    help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.cpu_oracle:
        res = (cpu_oracle_reference(args.steps, args.warmup) if args.cpu_oracle == "reference"
               else cpu_oracle_baseline())
        print(json.dumps(res), flush=True)
        return
    if args.uneven:
        run_uneven(args)
        return
    if args.workload_1d:
        import torch
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")
        print(json.dumps(measure_workload_1d(args.steps, flush, peaks()[0])), flush=True)
        return
    globals()["R"] = args.R
    if args.R != 11:
        n = 2 ** (args.R + 1)
        globals()["WORKLOAD"] = (WORKLOAD.replace("M=2048^2 -> N=4096^2 (R=11, q=1)",
                                                  f"M={2 ** args.R}^2 -> N={n}^2 (R={args.R}, q=1)")
                                 .replace("(m=2013266)", f"(m={int(round(FRAC * n * n))})"))
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
