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
# the CPU oracle (reference arm and cpu_baseline)
# ----------------------------------------------------------------------------
def oracle_pair_rate(lines=64):
    """Time the oracle's Algorithm 2 on a bounded sample of the workload and
    scale to one full pair: the Mallat IDWT and DWT on the full 2048^2 array,
    and Algorithm 1 (sum_l D_l H_l plus Prop. 4.4 edges) forward and adjoint
    on `lines` lines of each pass; a full pair applies Algorithm 1 to
    M + N lines in each direction.  Single thread (BLAS pinned to 1)."""
    code = f"""
import time, json, numpy as np
from oracle import fast, wavelets as W
from paper_2106_00554_gb300 import inputs
R, q, p = {R}, {Q}, {P}
M, N = 2 ** R, 2 ** (R + q)
J0 = W.default_J0(p)
rng = np.random.default_rng({SEED})
x = inputs.coeffs_2d(rng, R, J0, 1.5)
fast.alg1_forward(np.zeros((1, M)), R, q, p, W.VMP)       # build the oracle tables first
t0 = time.perf_counter(); S = fast.idwt2d(x, J0, p, W.VMP); t_idwt = time.perf_counter() - t0
t0 = time.perf_counter(); fast.dwt2d(S, J0, p, W.VMP); t_dwt = time.perf_counter() - t0
L = {lines}
xi = rng.standard_normal((L, M)); al = rng.standard_normal((L, N))
t0 = time.perf_counter(); fast.alg1_forward(xi, R, q, p, W.VMP); t_f = (time.perf_counter() - t0) / L
t0 = time.perf_counter(); fast.alg1_adjoint(al, R, q, p, W.VMP); t_a = (time.perf_counter() - t0) / L
pair = t_idwt + t_dwt + (M + N) * (t_f + t_a)
print(json.dumps({{"pair_s": pair, "idwt_s": t_idwt, "dwt_s": t_dwt, "line_fwd_s": t_f, "line_adj_s": t_a}}))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    t0 = time.perf_counter()
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True)
    wall = time.perf_counter() - t0
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": 1.0 / d["pair_s"], "unit": "pairs/s", "cores": 1, "kind": "oracle",
            "sample": (f"oracle Algorithm 2 at N=4096^2: full 2048^2 Mallat IDWT + DWT, Algorithm 1 "
                       f"forward and adjoint timed on {lines} lines each and scaled to the M+N=6144 "
                       f"lines of one pair; single thread; {wall:.1f} s of CPU work"),
            "detail": d}


def run_reference(args):
    """The oracle on the host cores: one-time Mallat IDWT + DWT of the full
    array, then per step Algorithm 1 forward and adjoint on a bounded number
    of lines (sized so the whole run stays within a few minutes), each step
    scaled to one full pair."""
    rank, _, world = env_rank()
    if rank != 0:
        return
    total = args.steps + args.warmup
    code = f"""
import time, json, statistics, numpy as np
from oracle import fast, wavelets as W
from paper_2106_00554_gb300 import inputs
R, q, p = {R}, {Q}, {P}
M, N = 2 ** R, 2 ** (R + q)
J0 = W.default_J0(p)
rng = np.random.default_rng({SEED})
x = inputs.coeffs_2d(rng, R, J0, 1.5)
fast.alg1_forward(np.zeros((1, M)), R, q, p, W.VMP)
t0 = time.perf_counter(); S = fast.idwt2d(x, J0, p, W.VMP); t_idwt = time.perf_counter() - t0
t0 = time.perf_counter(); fast.dwt2d(S, J0, p, W.VMP); t_dwt = time.perf_counter() - t0
budget = 120.0 / {total}
t0 = time.perf_counter(); fast.alg1_forward(rng.standard_normal((1, M)), R, q, p, W.VMP)
fast.alg1_adjoint(rng.standard_normal((1, N)), R, q, p, W.VMP); t1 = time.perf_counter() - t0
L = max(1, min(32, int(budget / max(t1, 1e-6))))
pairs = []
for s in range({total}):
    xi = rng.standard_normal((L, M)); al = rng.standard_normal((L, N))
    t0 = time.perf_counter(); fast.alg1_forward(xi, R, q, p, W.VMP); tf = (time.perf_counter() - t0) / L
    t0 = time.perf_counter(); fast.alg1_adjoint(al, R, q, p, W.VMP); ta = (time.perf_counter() - t0) / L
    if s >= {args.warmup}:
        pairs.append(t_idwt + t_dwt + (M + N) * (tf + ta))
print(json.dumps({{"pair_s": statistics.median(pairs), "lines": L, "steps": len(pairs), "idwt_s": t_idwt,
                  "dwt_s": t_dwt}}))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    t0 = time.perf_counter()
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True)
    wall = time.perf_counter() - t0
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    v = 1.0 / d["pair_s"]
    sample = (f"oracle Algorithm 2 at N=4096^2: the full 2048^2 Mallat IDWT + DWT timed once "
              f"({d['idwt_s'] + d['dwt_s']:.1f} s), then per step Algorithm 1 forward and adjoint on "
              f"{d['lines']} line(s) each, scaled to the M+N=6144 lines of one pair; median over "
              f"{d['steps']} steps; single thread; {wall:.1f} s wall")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "pairs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": "f64 (CPU oracle)"},
            "cpu_baseline": {"value": v, "unit": "pairs/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# the CUDA path
# ----------------------------------------------------------------------------
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
        ke = max(3, min(args.steps, 200))

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
                      "overlap the neighbouring steps' products (two staging slots). sync_value: the "
                      "blocking uw_forward_host + uw_adjoint_host, one call at a time"}

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
    if not args.no_cpu_baseline:
        cb = oracle_pair_rate(lines=384)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
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
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        group.forward(xd, yo, prec, stream=s)
        group.adjoint(yd, xo, prec, stream=s)
    s.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        group.forward(xd, yo, prec, stream=s)
        group.adjoint(yd, xo, prec, stream=s)

    def timed(fn, k):
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
    ms_graph = timed(graph.replay, k)
    group.close()

    def sequential():
        with torch.cuda.stream(s):
            for pl, x, y, a, b in zip(plans, xd, yd, yo, xo):
                pl.forward(x, a, precision=prec, stream=s)
                pl.adjoint(y, b, precision=prec, stream=s)

    ms_seq = timed(sequential, max(3, k // 5))
    n = len(plans)
    print(json.dumps({
        "metric": f"batched uneven 2D U x + U* y pairs/s ({n} instances)", "value": n * 1000.0 / ms_graph,
        "unit": "pairs/s", "higher_is_better": True, "ms_per_step": ms_graph, "steps": k,
        "dtype": "f32" if prec == F32 else "bf16 split (3 parts per operand), f32 accumulate",
        "data": "synthetic",
        "config": {"workload": f"{n} instances: R in 6..9, q in 1..2, p in {{1,2,4,6,8}}, periodic or VMP, "
                               "alpha in [1,2], 10-40% radial multilevel masks, seed 3",
                   "launch": f"plan group over {nst} streams, tuned, pair captured as one CUDA graph",
                   "setup_s": round(setup_s, 2), "tune_s": round(tune_s, 2)},
        "sequential": {"value": n * 1000.0 / ms_seq, "unit": "pairs/s", "ms_per_step": ms_seq,
                       "how": "each plan's forward and adjoint issued in turn on one stream, eager"}}))


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
    ap.add_argument("--uneven", type=int, default=0,
                    help="instead of the benchmark workload: the batched uneven workload with this many instances")
    args = ap.parse_args()
    if args.uneven:
        run_uneven(args)
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
