"""Benchmark of the GE solver on the single large 1D solve:
N = 2^24 interior points, r = 2, 10000 GE steps, zero walls, u0 = eight seeded
sine modes.  One benchmark step = one full solve (reset the state, advance
10000 steps) through the C ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--precision f64|f32|f32c] [--kernel temporal|temporal_df|onestep|canonical]
                    [--depth D] [--no-variants] [--no-cpu]

Prints one JSON line (rank 0).  Under torchrun every rank solves its own
independent problem of the same size (weak scaling, no collective on the
data path); `value` is the updates of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GE grid-point updates/s & HBM-roofline fraction; surrogate speedup at 1e-3 err"
UNIT = "grid-point updates/s"
N_POINTS = 1 << 24
R = 2.0
GE_STEPS = 10000
WORKLOAD = ("single large 1D GE solve: N=2^24 interior points, r=2.0, 10000 steps, Dirichlet zero "
            "walls, u0 = sum of 8 seeded sine modes k in [1,64], amplitudes U(-1,1)")
CPU_SAMPLE_STEPS = 1000    # oracle baseline: 1000 GE steps over the full grid (about 11 s on one core)
REF_SAMPLE_STEPS = 10      # --impl reference: 10 GE steps over the full grid per step
N_SAMPLES = 12             # oracle-checked sample points


def tb_source_digest(kernel_name: str = "tb_kernel") -> str:
    """sha256 over a tiled kernel's sources: ge_tb.cu (or ge_tb_df.cu for the
    double-float kernel) + ge_tb_dev.cuh."""
    import hashlib
    h = hashlib.sha256()
    main = "ge_tb_df.cu" if kernel_name.startswith("tb_df_kernel") else "ge_tb.cu"
    for f in (main, "ge_tb_dev.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1310_3422_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def measured_traffic(kernel_name: str):
    """Per-launch DRAM bytes of `kernel_name` from profiles/traffic.txt, or None
    when absent or when the kernel source (its .cu file and the device helpers
    of ge_tb_dev.cuh) changed since the capture."""
    try:
        digest = tb_source_digest(kernel_name)
        for line in open(os.path.join(ROOT, "profiles", "traffic.txt")):
            if line.startswith("#") or not line.strip():
                continue
            name, sha, nbytes = line.split()[:3]
            if name == kernel_name and digest.startswith(sha):
                return int(nbytes)
    except Exception:
        return None
    return None


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), float(pk.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


# FP64 / FP32 FMA lanes per SM per clock on GB300: FP64 1.25 TFLOP/s nominal
# over 152 SMs at 2.07 GHz is 2 FMA/clk/SM; FP32 is 128 FMA/clk/SM.  The SM
# count is read from the device.
FMA_PER_CLK = {"f64": 2.0, "f32": 128.0, "f32c": 128.0}
# Double-float kernel: FP32-pipe instructions (FADD, FMUL, FFMA alike, one
# issue each) per point and step of its fast path, renormalised every second
# step: 11 + 3/2 (renormalised every second step) when 2r is an FP32 number,
# 21 + 3 otherwise (the exact low-order product sum, renormalised every
# step).  Its peak is 128 such instructions/clk/SM.
DF_OPS_PER_UPDATE = {True: 12.5, False: 24.0}


# The method's own work per point and step (Eqs. (cc)/(dd) as printed): one
# multiply and three multiply-adds, and one FP64 value read and one written.
METHOD_FLOPS_PER_UPDATE = 7
METHOD_BYTES_PER_UPDATE = 16


def fma_probe(B, torch, dev, stream, prec, sms):
    """Measured multiply-add throughput of the register-only probe
    (ge_probe_fma), timed with CUDA events on `stream`: the best rate over
    1, 2 and 4 CTAs of 256 threads per SM and 8, 16 and 32 independent
    chains per thread (each timed twice after a warm-up launch).  Returns
    (multiply-adds per second, CTAs per SM, chains) of the best."""
    best = (0.0, 0, 0)
    fmas_per_launch = 6e9 if prec == B.GE_F64 else 2e11   # about 10 ms each
    sink = torch.empty(4 * sms * B.PROBE_THREADS, dtype=B.dtype_of(prec), device=dev)
    with torch.cuda.stream(stream):
        for cps in (1, 2, 4):
            for chains in (8, 16, 32):
                blocks = cps * sms
                iters = max(1, int(fmas_per_launch / (blocks * B.PROBE_THREADS * chains)))
                B.ge_probe_fma(prec, blocks, chains, iters, sink, stream=stream)
                for _ in range(2):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    fmas = B.ge_probe_fma(prec, blocks, chains, iters, sink, stream=stream)
                    e1.record(stream)
                    e1.synchronize()
                    rate = fmas / (e0.elapsed_time(e1) / 1e3)
                    if rate > best[0]:
                        best = (rate, cps, chains)
    return best


def two_r_is_fp32(r: float) -> bool:
    return float(np.float32(2.0 * r)) == 2.0 * r


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]
        return False

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        # GE_BENCH_DIST_BACKEND=gloo runs the multi-rank code paths with the
        # ranks sharing fewer GPUs than ranks (a check of the host logic; their
        # kernels never wait on one another, halos travel through the host)
        backend = "gloo" if args.impl == "reference" else os.environ.get("GE_BENCH_DIST_BACKEND", "nccl")
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def _oracle_window(task):
    """One worker of the all-core oracle baseline: the oracle, as it stands,
    on one window of the grid; returns its own compute seconds."""
    import oracle
    u, r, bl, br, steps = task
    t0 = time.perf_counter()
    oracle.run(u, r, bl, br, steps)
    return time.perf_counter() - t0


def oracle_all_cores(u0, r, steps):
    """The serial oracle run concurrently on every host core, one window per
    core: core q advances points [a_q - m, b_q + m) with m = steps + 4 (the
    dependency cone of `steps` steps, so the owned range [a_q, b_q) is exact).
    Processes are spawned (the parent holds a CUDA context).  Returns
    (updates/s over the whole grid, cores used, wall seconds)."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    n = u0.size
    m = steps + 4
    m += m % 2
    cuts = [2 * ((n * q) // (2 * cores)) for q in range(cores)] + [n]
    tasks = []
    for q in range(cores):
        lo, hi = max(0, cuts[q] - m), min(n, cuts[q + 1] + m)
        tasks.append((np.ascontiguousarray(u0[lo:hi]), r, 0.0, 0.0, steps))
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        # start-up outside the timing; every wait is bounded (a worker that
        # dies would otherwise leave the pool waiting)
        pool.map_async(_oracle_window, [(np.zeros(8), r, 0.0, 0.0, 1)] * cores).get(timeout=300)
        t0 = time.perf_counter()
        pool.map_async(_oracle_window, tasks, chunksize=1).get(timeout=600)
        wall = time.perf_counter() - t0
    return n * steps / wall, cores, wall


PAPER_CONTEXT = {
    "hardware": "NVIDIA GeForce GT 335M (72 stream processors) against an Intel Core i7-720QM (4 cores, 8 threads)",
    "gpu_vs_cpu_1_thread": 5.0, "gpu_vs_cpu_8_threads": 2.0,
    "note": "ratios stated in the paper's text (Sec. 4); its absolute runtimes are only in figures, so there is "
            "no absolute figure to compare with (context only)"}


def sample_indices(n):
    rng = np.random.default_rng(20240613)
    return sorted(set([0, 1, n // 2, n - 2, n - 1] + [int(i) for i in rng.integers(0, n, N_SAMPLES - 5)]))


def oracle_reference(u0, idx):
    import oracle
    return oracle.sample(u0, R, 0.0, 0.0, GE_STEPS, idx)


def errors(got, want, scale):
    d = np.asarray(got, dtype=np.float64) - want
    return {"max_rel_err": float(np.max(np.abs(d)) / scale),
            "l2_rel_err": float(np.linalg.norm(d) / max(1e-300, np.linalg.norm(want))),
            "samples": int(len(want)), "reference": "CPU FP64 oracle on dependency-cone windows"}


def run_reference(args, world, rank):
    """--impl reference: the oracle as it stands on the host cores."""
    if rank != 0:
        return 0
    import oracle
    from paper_1310_3422_gb300 import inputs
    u0 = inputs.sine_modes_state(N_POINTS)
    oracle.default()
    u = u0.copy()
    for _ in range(args.warmup):
        u = oracle.run(u, R, 0.0, 0.0, REF_SAMPLE_STEPS)
    t0 = time.perf_counter()
    step0 = 0
    for _ in range(args.steps):
        u = oracle.run(u, R, 0.0, 0.0, REF_SAMPLE_STEPS, step0=step0)
        step0 += REF_SAMPLE_STEPS
    dt = time.perf_counter() - t0
    value = N_POINTS * REF_SAMPLE_STEPS * args.steps / dt
    sample = f"{REF_SAMPLE_STEPS} GE steps over the full N=2^24 grid per benchmark step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "n": N_POINTS, "r": R,
                                            "ge_steps_per_sample": REF_SAMPLE_STEPS},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def time_solver(B, torch, ctx, u0_dev, steps, warmup, stream, flush=None):
    """Per-solve CUDA-event timing on the solver's stream; returns ms per solve."""
    def one():
        B.ge_write_state(ctx, u0_dev, 0)
        B.ge_step_n(ctx, GE_STEPS)
    for _ in range(warmup):
        one()
    torch.cuda.synchronize()
    total = 0.0
    for _ in range(steps):
        if flush is not None:
            flush()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        one()
        e1.record(stream)
        e1.synchronize()
        total += e0.elapsed_time(e1)
    return total / steps


def measure_e2e(B, torch, u0, prec, kern, depth, steps, world):
    """The metric through ge_solve with pinned host buffers: every solve
    copies u0 host->device, advances GE_STEPS and copies the result back."""
    pin_in = torch.from_numpy(u0.astype(np.float64 if prec == B.GE_F64 else np.float32)).pin_memory()
    pin_out = torch.empty_like(pin_in).pin_memory()
    hin, hout = pin_in.numpy(), pin_out.numpy()
    B.ge_solve(N_POINTS, R, 0.0, 0.0, prec, kern, depth, GE_STEPS, hin, hout)
    k_e2e = max(1, min(steps, 3))
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        B.ge_solve(N_POINTS, R, 0.0, 0.0, prec, kern, depth, GE_STEPS, hin, hout)
    t_e2e = (time.perf_counter() - t0) / k_e2e
    return {"value": float(N_POINTS) * GE_STEPS * world / t_e2e, "unit": UNIT,
            "h2d_bytes_per_step": int(hin.nbytes), "d2h_bytes_per_step": int(hout.nbytes),
            "ms_per_step": t_e2e * 1e3, "timer": "host wall clock around ge_solve (synchronous)"}


def measure_batch(B, torch, inputs, dev, steps, warmup, only=None, fixed=None):
    """Batched workload: 4096 problems, N log-uniform in [256, 65536], r in
    [0.25, 4], 2000 steps.  One CUDA-graph replay per solve (reset from u0 +
    ge_batch_run); depth and tile geometry autotuned (or `fixed` = (depth,
    rows per tile, CTAs per SM), for profiling one launch shape); sampled
    problems checked against the oracle."""
    import oracle
    bt = inputs.uneven_batch()
    upd = float(bt.n.sum()) * 2000
    out = {"workload": "4096 problems, N log-uniform [256,65536] even, r U[0.25,4], walls U(-1,1), "
                       "u0 = linear + 16-mode Fourier (1/k^2), 2000 steps",
           "updates_per_solve": upd}
    rng = np.random.default_rng(11)
    picks = list(rng.choice(len(bt.n), 6, replace=False)) + [int(np.argmin(bt.n)), int(np.argmax(bt.n))]
    want = {i: oracle.run(bt.u0[bt.offsets[i]:bt.offsets[i] + bt.n[i]], bt.r[i], bt.beta_l[i], bt.beta_r[i], 2000)
            for i in picks}
    for name, prec in (("f32", B.GE_F32), ("f32c", B.GE_F32_COMP), ("f64", B.GE_F64), ("f64_df", B.GE_F64)):
        if only is not None and name != only:
            continue
        s = torch.cuda.Stream(device=dev)
        with torch.cuda.stream(s):
            u0 = torch.from_numpy(bt.u0).to(dev, B.dtype_of(prec))
            u = u0.clone()
            plan = B.ge_batch_create(bt.n, bt.r, bt.beta_l, bt.beta_r, bt.offsets, bt.total, prec, stream=s)
            if name == "f64_df":  # FP64 storage, double-float arithmetic on the FP32 pipes
                B.ge_batch_set_kernel(plan, B.GE_KERNEL_TEMPORAL_DF)
            if fixed is None:
                depth = B.ge_batch_tune(plan, u0, 256)
            else:
                depth = fixed[0]
                B.ge_batch_set_depth(plan, depth)
                B.ge_batch_set_geometry(plan, fixed[1], fixed[2])
                if len(fixed) > 3:
                    B.ge_batch_set_persistent(plan, fixed[3])
            tile_rows, ctas = B.ge_batch_get_geometry(plan)
            persist_flag = B.ge_batch_get_persistent(plan)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                u.copy_(u0)
                B.ge_batch_run(plan, u, 2000)
            for _ in range(warmup):
                g.replay()
            torch.cuda.synchronize()
            # enough replays for the clock sampler to see the region (>= 1 s)
            t0 = time.perf_counter()
            g.replay()
            torch.cuda.synchronize()
            reps = max(steps, int(np.ceil(1.0 / max(1e-4, time.perf_counter() - t0))))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            sampler = ClockSampler(dev.index or 0)
            with sampler:
                e0.record(s)
                for _ in range(reps):
                    g.replay()
                e1.record(s)
                e1.synchronize()
            ms = e0.elapsed_time(e1) / reps
            B.ge_batch_sync(plan)
            got = u.double().cpu().numpy()
            errs = []
            for i in picks:
                o, n = bt.offsets[i], bt.n[i]
                w = want[i]
                errs.append(float(np.max(np.abs(got[o:o + n] - w)) / np.max(np.abs(w))))
            B.ge_batch_destroy(plan)
        persistent = bool(persist_flag)
        out[name] = {"updates_per_s": upd / (ms / 1e3), "ms_per_solve": ms, "depth": depth,
                     "persistent_launch": persistent,
                     "geometry": {"tile_rows": tile_rows, "ctas_per_sm": ctas,
                                  "tuned": fixed is None},
                     "replays_timed": reps, "clocks": sampler.summary(),
                     "launches_per_solve": (1 if persistent else (2000 + depth - 1) // depth)
                     + (2 if name == "f64_df" else 0),
                     "max_rel_err_sampled": max(errs), "problems_checked": len(picks)}
    return out


def shard_problems(n, world: int):
    """Contiguous blocks of problems, one per rank, balanced by points: rank
    q takes problems [cuts[q], cuts[q + 1]) (at least one each)."""
    cum = np.cumsum(np.asarray(n, dtype=np.float64))
    cuts = [0]
    for q in range(1, world):
        c = int(np.searchsorted(cum, cum[-1] * q / world))
        cuts.append(min(max(c, cuts[-1] + 1), len(n) - (world - q)))
    cuts.append(len(n))
    return cuts


def measure_batch_sharded(B, torch, inputs, dev, dist, rank, world, steps, warmup):
    """The batched workload (config 3) sharded by problem over the ranks:
    rank q solves its block of problems (balanced by points) on its own GPU,
    with no collective on the data path.  One CUDA-graph replay per solve
    (reset + ge_batch_run of 2000 steps), depth autotuned per rank; timed
    with a barrier and a device synchronisation on both sides, the max over
    ranks.  updates_per_s counts every problem of the batch."""
    import oracle
    bt = inputs.uneven_batch()
    cuts = shard_problems(bt.n, world)
    i0, i1 = cuts[rank], cuts[rank + 1]
    ns = bt.n[i0:i1]
    offs = np.zeros(len(ns), dtype=np.int64)
    pos = 0
    for k, n in enumerate(ns):
        offs[k] = pos
        pos += ((int(n) + 31) // 32) * 32
    u_host = np.zeros(pos)
    for k in range(len(ns)):
        o = bt.offsets[i0 + k]
        u_host[offs[k]:offs[k] + ns[k]] = bt.u0[o:o + ns[k]]
    upd_all = float(bt.n.sum()) * 2000
    out = {"ranks": world, "problems_per_rank": [cuts[q + 1] - cuts[q] for q in range(world)],
           "points_per_rank": [int(bt.n[cuts[q]:cuts[q + 1]].sum()) for q in range(world)],
           "updates_per_solve": upd_all}
    for name, prec in (("f32", B.GE_F32), ("f64", B.GE_F64)):
        s = torch.cuda.Stream(device=dev)
        with torch.cuda.stream(s):
            u0 = torch.from_numpy(u_host).to(dev, B.dtype_of(prec))
            u = u0.clone()
            plan = B.ge_batch_create(ns, bt.r[i0:i1], bt.beta_l[i0:i1], bt.beta_r[i0:i1], offs, pos, prec,
                                     stream=s)
            depth = B.ge_batch_tune(plan, u0, 256)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                u.copy_(u0)
                B.ge_batch_run(plan, u, 2000)
            for _ in range(warmup):
                g.replay()
            torch.cuda.synchronize()
            dist.barrier()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(steps):
                g.replay()
            e1.record(s)
            e1.synchronize()
            t = torch.tensor([e0.elapsed_time(e1) / steps], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
            B.ge_batch_sync(plan)
            got = u.double().cpu().numpy()
            B.ge_batch_destroy(plan)
        # two of this rank's problems against the oracle
        errs = []
        for k in (0, len(ns) - 1):
            start = u_host[offs[k]:offs[k] + ns[k]]
            if prec == B.GE_F32:
                start = start.astype(np.float32).astype(np.float64)
            w = oracle.run(start, bt.r[i0 + k], bt.beta_l[i0 + k], bt.beta_r[i0 + k], 2000)
            errs.append(float(np.max(np.abs(got[offs[k]:offs[k] + ns[k]] - w)) / np.max(np.abs(w))))
        e = torch.tensor([max(errs)], device=dev)
        dist.all_reduce(e, op=dist.ReduceOp.MAX)
        out[name] = {"updates_per_s": upd_all / (ms / 1e3), "ms_per_solve_max_over_ranks": ms,
                     "depth_rank0": depth if rank == 0 else None,
                     "max_rel_err_sampled": float(e.item()), "problems_checked": 2 * world}
    return out


def measure_split_solve(B, torch, inputs, dev, dist, rank, world, depth=48):
    """Config 2 (N = 2^24, r = 2, 10000 steps) as ONE solve split over the
    ranks: each rank keeps a device-resident GE context over its owned range
    plus depth + 1 halo points per side and exchanges halos with its
    neighbours every `depth` steps (NCCL point-to-point; no collective).
    Strong scaling: the work is fixed, and updates_per_s counts the whole
    grid.  One warm-up solve, one timed solve (barrier + device sync on both
    sides, max over ranks); eight owned points checked against the oracle."""
    import oracle
    from paper_1310_3422_gb300 import decomp
    u0 = inputs.sine_modes_state(N_POINTS)
    p = decomp.partition(N_POINTS, world, rank, depth + 1)
    bl = br = 0.0

    def solve():
        st = decomp.DeviceState(u0[p.lo:p.hi], R, bl, br, 0, depth)
        done = 0
        while done < GE_STEPS:
            L = min(depth, GE_STEPS - done)
            st.step_n(L)
            done += L
            if done < GE_STEPS:
                decomp.exchange_halos(st, p, dist)
        return st

    solve().close()
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = solve()
    torch.cuda.synchronize()
    dt = torch.tensor([time.perf_counter() - t0], device=dev)
    dist.all_reduce(dt, op=dist.ReduceOp.MAX)
    own = st.result(p.a - p.lo, p.b - p.a)
    st.close()
    idx = np.linspace(p.a, p.b - 1, 8).astype(np.int64)
    want = oracle.sample(u0, R, 0.0, 0.0, GE_STEPS, list(idx))
    err = torch.tensor([float(np.max(np.abs(own[idx - p.a] - want)) / np.max(np.abs(u0)))], device=dev)
    dist.all_reduce(err, op=dist.ReduceOp.MAX)
    return {"workload": WORKLOAD + ", one solve split over the ranks", "ranks": world, "depth": depth,
            "halo_points_per_side": p.halo, "owned_points_rank0": p.b - p.a if rank == 0 else None,
            "updates_per_s": float(N_POINTS) * GE_STEPS / float(dt.item()), "seconds_max_over_ranks": float(dt.item()),
            "scaling": "strong", "max_rel_err_sampled": float(err.item()),
            "timer": "host wall clock around the solve, device synchronised, max over ranks"}


SNO_PROBLEMS, SNO_N, SNO_K, SNO_JUMPS, SNO_TOL = 65536, 1024, 256, 8, 1e-3


def measure_surrogate(B, torch, inputs, train_steps):
    """Surrogate workload: the spectral neural operator (4 layers, 16 modes,
    width 64, BF16 weights, FP32 accumulate) trained on the GPU on 100k pairs
    (12,500 GE trajectories x 8 jumps of K = 256 steps, N = 1024, r U[0.5, 4],
    u0 = linear wall profile + 16-mode Fourier (1/k^2) + 2 piecewise-linear
    tents), then 65,536 fresh problems advanced 2048 steps as 8 jumps with the
    GE fallback (1% sample + flagged, tolerance 1e-3 relative L2), against
    plain batched FP32 GE (depth autotuned) on the same problems.  Times are
    wall-clock with a device synchronisation on both sides (the fallback
    pipeline reads its sample results back to the host)."""
    from paper_1310_3422_gb300 import surrogate as SG

    def sync():
        torch.cuda.synchronize()

    def rel_l2(a, b):
        return (torch.linalg.vector_norm(a.double() - b, dim=1) / torch.linalg.vector_norm(b, dim=1)).cpu().numpy()

    def stats(e):
        return {"median": float(np.median(e)), "p99": float(np.percentile(e, 99)), "max": float(np.max(e))}

    t0 = time.perf_counter()
    data = SG.make_training_set(12500, K=SNO_K, jumps=SNO_JUMPS)
    held = SG.make_training_set(256, K=SNO_K, jumps=SNO_JUMPS, seed=inputs.SEED_BASE + 5)
    sync()
    t_data = time.perf_counter() - t0
    sur = SG.Surrogate(max_batch=1024, seed=0)
    ident = rel_l2(held.x, held.y.double())
    t0 = time.perf_counter()
    losses = sur.train(data, steps=train_steps, batch=64, lr=2e-3, warmup=100)
    sync()
    t_train = time.perf_counter() - t0
    one_jump = sur.evaluate(held)
    del data

    pr = inputs.surrogate_problems(SNO_PROBLEMS, SNO_N, seed=inputs.SEED_BASE + 6)
    u0 = torch.tensor(pr.u0, dtype=torch.float32, device="cuda")
    r, bl, br = (torch.tensor(x, dtype=torch.float32, device="cuda") for x in (pr.r, pr.beta_l, pr.beta_r))
    steps = SNO_K * SNO_JUMPS
    # plain batched FP32 GE
    ge = SG.GEBatch(pr.r, pr.beta_l, pr.beta_r, SNO_N, B.GE_F32)
    depth = B.ge_batch_tune(ge.plan, u0, 256)
    x = u0.clone()
    ge.run(x, steps)
    sync()
    ge_ms = []
    for _ in range(3):
        x.copy_(u0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ge.run(x, steps)
        e1.record()
        e1.synchronize()
        ge_ms.append(e0.elapsed_time(e1))
    t_ge = min(ge_ms) / 1e3
    ge.close()
    # surrogate alone, then the pipeline with the fallback
    sur.rollout(u0[:1024], r[:1024], bl[:1024], br[:1024], 1)
    sync()
    t0 = time.perf_counter()
    pred = sur.rollout(u0, r, bl, br, SNO_JUMPS)
    sync()
    t_sur = time.perf_counter() - t0
    # untimed warm-up of the whole pipeline on a slice: the first use of the
    # framework's own reductions (the non-finite row check, nonzero) loads
    # their kernels, which took seconds inside the timed region
    SG.solve_with_fallback(sur, u0[:256], r[:256], bl[:256], br[:256], 1, tol=SNO_TOL, sample_frac=0.01)
    sync()
    t0 = time.perf_counter()
    out, rep = SG.solve_with_fallback(sur, u0, r, bl, br, SNO_JUMPS, tol=SNO_TOL, sample_frac=0.01)
    sync()
    t_pipe = time.perf_counter() - t0
    # accuracy against FP64 GE
    ref = u0.double()
    ge64 = SG.GEBatch(pr.r, pr.beta_l, pr.beta_r, SNO_N, B.GE_F64)
    ge64.run(ref, steps)
    sync()
    ge64.close()
    err_pipe, err_sur, err_ge32 = rel_l2(out, ref), rel_l2(pred, ref), rel_l2(x, ref)
    tc_used = bool(B.ge_sno_get_tensor_cores(sur.model))
    sur.close()
    chunks = -(-SNO_PROBLEMS // 1024)
    return {
        "workload": f"{SNO_PROBLEMS} problems N={SNO_N}, r U[0.5,4], walls U(-1,1), u0 = linear + 16-mode "
                    f"Fourier (1/k^2) + 2 tents; {steps} steps as {SNO_JUMPS} jumps of K={SNO_K}",
        "tolerance_rel_l2": SNO_TOL,
        "speedup_vs_batched_f32_ge": t_ge / t_pipe,
        "pipeline_ms": t_pipe * 1e3, "surrogate_only_ms": t_sur * 1e3, "batched_f32_ge_ms": t_ge * 1e3,
        "ge_depth": depth,
        "fell_back_all": rep.fell_back_all, "sampled": rep.n_sampled, "flagged": rep.n_flagged,
        "sample_over_tol": rep.n_sample_over_tol, "sample_max_err": rep.sample_max_err,
        "err_pipeline_rel_l2": stats(err_pipe), "err_surrogate_only_rel_l2": stats(err_sur),
        "err_batched_f32_ge_rel_l2": stats(err_ge32),
        "one_jump_heldout_rel_l2": stats(one_jump), "identity_one_jump_rel_l2": stats(ident),
        "training": {"pairs": 100000, "steps": train_steps, "batch": 64, "seconds": t_train,
                     "data_seconds": t_data, "loss_first": float(losses[:20].mean()),
                     "loss_last": float(losses[-100:].mean())},
        "surrogate_tflops": 2 * SNO_PROBLEMS * SNO_JUMPS * sno_flops_per_problem() / t_sur / 1e12,
        "gpu_launches_surrogate_only": SNO_JUMPS * chunks * sno_launches_per_forward(),
        "tensor_core_path": tc_used,
    }


SNO_SWEEP_K = (256, 1024, 4096, 16384)


def measure_surrogate_k_sweep(B, torch, inputs, train_steps, Ks=SNO_SWEEP_K, problems=16384, jumps=2):
    """Where the surrogate can pay: for each jump length K, a surrogate trained
    for K (100k pairs from 12,500 FP32 GE trajectories of 8 jumps, same
    network and schedule as the main surrogate run) advances `problems`
    fresh problems (N = 1024, r U[0.5, 4], same u0 distribution) by `jumps`
    jumps, alone and inside the GE fallback pipeline (1 % sample, tolerance
    1e-3 relative L2), against plain batched FP32 GE (depth and geometry
    autotuned) on the same problems.  rows_within_tol: the share of problems
    whose surrogate-only result is within the tolerance of GE's (FP32 GE's
    own error, ~1e-6, is far below it).  Times: best of 3 (GE) or one run
    after a warm-up, device-synchronised wall clock."""
    from paper_1310_3422_gb300 import surrogate as SG

    def sync():
        torch.cuda.synchronize()

    pr = inputs.surrogate_problems(problems, SNO_N, seed=inputs.SEED_BASE + 7)
    u0 = torch.tensor(pr.u0, dtype=torch.float32, device="cuda")
    r, bl, br = (torch.tensor(x, dtype=torch.float32, device="cuda") for x in (pr.r, pr.beta_l, pr.beta_r))
    points = []
    for K in Ks:
        t0 = time.perf_counter()
        data = SG.make_training_set(12500, K=K, jumps=SNO_JUMPS, prec=B.GE_F32)
        sur = SG.Surrogate(K=K, max_batch=1024, seed=0)
        sur.train(data, steps=train_steps, batch=64, lr=2e-3, warmup=100)
        del data
        sync()
        t_train = time.perf_counter() - t0
        steps = jumps * K
        ge = SG.GEBatch(pr.r, pr.beta_l, pr.beta_r, SNO_N, B.GE_F32)
        B.ge_batch_tune(ge.plan, u0, min(256, K))
        x = u0.clone()
        ge.run(x, steps)
        sync()
        t_ge = 1e300
        for _ in range(3):
            x.copy_(u0)
            sync()
            t1 = time.perf_counter()
            ge.run(x, steps)
            sync()
            t_ge = min(t_ge, time.perf_counter() - t1)
        ge.close()
        sur.rollout(u0[:1024], r[:1024], bl[:1024], br[:1024], 1)
        sync()
        t1 = time.perf_counter()
        pred = sur.rollout(u0, r, bl, br, jumps)
        sync()
        t_sur = time.perf_counter() - t1
        SG.solve_with_fallback(sur, u0[:256], r[:256], bl[:256], br[:256], 1, tol=SNO_TOL, sample_frac=0.01)
        sync()
        t1 = time.perf_counter()
        out, rep = SG.solve_with_fallback(sur, u0, r, bl, br, jumps, tol=SNO_TOL, sample_frac=0.01)
        sync()
        t_pipe = time.perf_counter() - t1
        e = (torch.linalg.vector_norm(pred - x, dim=1) / torch.linalg.vector_norm(x, dim=1)).cpu().numpy()
        e_out = (torch.linalg.vector_norm(out - x, dim=1) / torch.linalg.vector_norm(x, dim=1)).cpu().numpy()
        points.append({"K": K, "steps": steps, "speedup_pipeline_vs_batched_f32_ge": t_ge / t_pipe,
                       "speedup_surrogate_only_vs_batched_f32_ge": t_ge / t_sur,
                       "rows_within_tol": float(np.mean(e <= SNO_TOL)), "fell_back_all": rep.fell_back_all,
                       "sample_over_tol": rep.n_sample_over_tol, "surrogate_err_median": float(np.median(e)),
                       "surrogate_err_p99": float(np.percentile(e, 99)),
                       "pipeline_err_max": float(np.max(e_out)),
                       "batched_f32_ge_ms": t_ge * 1e3, "surrogate_only_ms": t_sur * 1e3,
                       "pipeline_ms": t_pipe * 1e3, "train_seconds": t_train,
                       "tensor_core_path": bool(B.ge_sno_get_tensor_cores(sur.model))})
        sur.close()
        del pred, out
    return {"workload": f"{problems} problems N={SNO_N}, r U[0.5,4], walls U(-1,1), u0 = linear + 16-mode Fourier "
                        f"(1/k^2) + 2 tents; {jumps} jumps of K steps; surrogate trained per K ({train_steps} steps)",
            "tolerance_rel_l2": SNO_TOL, "points": points}


def measure_sno_forward(torch, inputs, steps, warmup, problems=4096):
    """Forward passes of the surrogate (untrained, BF16 mode) over `problems`
    problems of N = 1024 in chunks of 1024: time per problem and tensor
    throughput, on the tensor-core (tcgen05) inference path and on the
    mma.sync path.  For profiling the network's kernels alone."""
    from paper_1310_3422_gb300 import binding as B
    from paper_1310_3422_gb300 import surrogate as SG
    pr = inputs.surrogate_problems(problems, SNO_N, seed=inputs.SEED_BASE + 6)
    u0 = torch.tensor(pr.u0, dtype=torch.float32, device="cuda")
    r, bl, br = (torch.tensor(x, dtype=torch.float32, device="cuda") for x in (pr.r, pr.beta_l, pr.beta_r))
    sur = SG.Surrogate(max_batch=1024, seed=0)
    out = torch.empty_like(u0)
    res = {"problems": problems}
    ref = None
    for name, on in (("tcgen05", 1), ("mma_sync", 0)):
        B.ge_sno_set_tensor_cores(sur.model, on)
        tc = B.ge_sno_get_tensor_cores(sur.model) == 1
        for _ in range(warmup):
            sur.predict(u0, r, bl, br, out=out)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            sur.predict(u0, r, bl, br, out=out)
        e1.record()
        e1.synchronize()
        B.ge_sno_sync(sur.model)
        ms = e0.elapsed_time(e1) / steps
        net = (out - u0).double()
        if ref is None:
            ref = net.clone()
            agree = 0.0
        else:
            agree = float((torch.linalg.vector_norm(net - ref, dim=1) / torch.linalg.vector_norm(ref, dim=1)).max())
        res[name] = {"tensor_core_path": tc, "ms_per_forward_pass": ms, "us_per_problem": ms * 1e3 / problems,
                     "tflops": 2 * problems * sno_flops_per_problem() / (ms / 1e3) / 1e12,
                     "launches": -(-problems // 1024) * sno_launches_per_forward(tc=tc),
                     "max_rel_diff_of_network_part_vs_tcgen05": agree}
    B.ge_sno_set_tensor_cores(sur.model, 1)
    sur.close()
    return res


def sno_flops_per_problem(n=SNO_N, C=64, M=16, L=4, H=128):
    """Multiply-adds of one forward pass for one problem (x2 for FLOPs)."""
    per_layer = 2 * (2 * M * n * C) + M * (2 * C) * (2 * C) + n * C * C
    return n * 4 * C + L * per_layer + n * C * H + n * H


def sno_launches_per_forward(L=4, tc=True):
    """Inference launches per chunk.  mma.sync path: weight rounding, lift,
    per layer (spectral weights, DFT, mode mixing, fused layer GEMM), fused
    projection, fixed-order row sum.  tcgen05 path: lift, per layer (DFT,
    mode mixing, fused layer), fused projection; the operands derived from
    the weights (rounding, L + 1 transposes, L spectral-weight assemblies)
    are rebuilt only when the parameters change, so not in a timed loop of
    forward passes."""
    return (1 + 3 * L + 1) if tc else (2 + 4 * L + 2)


def launches_per_solve(kernel, depth):
    """Kernel launches of one solve (the tiled kernels' tile-queue resets are
    memsets, not kernels; the double-float kernel adds its prescale)."""
    if kernel in ("canonical", "subdomain16_onestep"):
        return GE_STEPS
    d = 1 if kernel == "onestep" else depth
    return (GE_STEPS + d - 1) // d + (1 if kernel == "temporal_df" else 0)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="f64", choices=["f64", "f32", "f32c"])
    ap.add_argument("--kernel", default="temporal", choices=["temporal", "temporal_df", "onestep", "canonical"])
    ap.add_argument("--depth", type=int, default=0)
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-probe", action="store_true", help="skip the FMA throughput probe")
    ap.add_argument("--probe-only", action="store_true",
                    help="run only the FMA throughput probe sweep (FP64 and FP32) and print it")
    ap.add_argument("--only-surrogate", action="store_true", help="run only the surrogate workload")
    ap.add_argument("--sno-train-steps", type=int, default=3000)
    ap.add_argument("--no-sno-sweep", action="store_true", help="skip the surrogate's jump-length sweep")
    ap.add_argument("--only-sno-sweep", action="store_true", help="run only the surrogate's jump-length sweep")
    ap.add_argument("--sno-forward-only", action="store_true",
                    help="time only surrogate forward passes (untrained weights; profiling)")
    ap.add_argument("--subdomain", type=int, default=1,
                    help="sub-domain width k of the main solve (k > 1: --kernel temporal runs --depth steps "
                         "per launch, --kernel canonical one launch per step)")
    ap.add_argument("--only-batched", default=None, choices=["f32", "f32c", "f64", "f64_df"],
                    help="run only the batched workload in this precision (profiling)")
    ap.add_argument("--batch-launch", default=None,
                    help="with --only-batched: a fixed launch shape DEPTH,TILE_ROWS,CTAS_PER_SM[,PERSISTENT] "
                         "instead of the autotuner (profiling)")
    args = ap.parse_args()

    world, rank, local, dist = dist_setup(args)
    if args.impl == "reference":
        rc = run_reference(args, world, rank)
        if dist is not None:
            dist.destroy_process_group()
        return rc

    import torch
    from paper_1310_3422_gb300 import binding as B
    from paper_1310_3422_gb300 import inputs

    B.load()
    local = local % max(1, torch.cuda.device_count())
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.only_batched:
        fixed = tuple(int(v) for v in args.batch_launch.split(",")) if args.batch_launch else None
        res = measure_batch(B, torch, inputs, dev, args.steps, args.warmup, only=args.only_batched, fixed=fixed)
        print(json.dumps({"batched": res}), flush=True)
        return 0
    if args.only_surrogate:
        print(json.dumps({"surrogate": measure_surrogate(B, torch, inputs, args.sno_train_steps)}), flush=True)
        return 0
    if args.probe_only:
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        st = torch.cuda.Stream(device=dev)
        res = {}
        for name, pr in (("f64", B.GE_F64), ("f32", B.GE_F32)):
            fma_s, cps, chains = fma_probe(B, torch, dev, st, pr, sms)
            res[name] = {"fma_per_s": fma_s, "fma_per_clk_per_sm_at_max_clock": fma_s / (sms * 2070e6),
                         "best_ctas_per_sm": cps, "best_chains": chains}
        print(json.dumps({"alu_probe": res}), flush=True)
        return 0
    if args.only_sno_sweep:
        print(json.dumps({"surrogate_k_sweep": measure_surrogate_k_sweep(B, torch, inputs, args.sno_train_steps)}),
              flush=True)
        return 0
    if args.sno_forward_only:
        print(json.dumps({"surrogate_forward": measure_sno_forward(torch, inputs, args.steps, args.warmup)}),
              flush=True)
        return 0
    if args.kernel == "temporal_df" and args.precision != "f64":
        ap.error("--kernel temporal_df runs FP64 contexts only")
    prec = {"f64": B.GE_F64, "f32": B.GE_F32, "f32c": B.GE_F32_COMP}[args.precision]
    kern = {"temporal": B.GE_KERNEL_TEMPORAL, "temporal_df": B.GE_KERNEL_TEMPORAL_DF,
            "onestep": B.GE_KERNEL_ONESTEP, "canonical": B.GE_KERNEL_CANONICAL}[args.kernel]
    depth = args.depth or (96 if args.kernel == "temporal_df" else (48 if args.precision == "f64" else 128))
    hbm_gbs, sm_max_mhz, peak_src = load_peaks()
    SMS = torch.cuda.get_device_properties(dev).multi_processor_count

    u0 = inputs.sine_modes_state(N_POINTS, seed=inputs.SEED_BASE + 1 + rank)
    dt = B.dtype_of(prec)
    u0_dev = torch.from_numpy(u0).to(dev, dtype=dt)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        ctx = B.ge_create(N_POINTS, R, 0.0, 0.0, prec, u0_dev, stream=stream)
        B.ge_set_kernel(ctx, kern, depth)
        if args.subdomain > 1:
            B.ge_set_subdomain_width(ctx, args.subdomain)

        # ---- timed region: K full solves --------------------------------
        for _ in range(args.warmup):
            B.ge_write_state(ctx, u0_dev, 0)
            B.ge_step_n(ctx, GE_STEPS)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(local)
        with sampler:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                B.ge_write_state(ctx, u0_dev, 0)
                B.ge_step_n(ctx, GE_STEPS)
            e1.record(stream)
            e1.synchronize()
        torch.cuda.synchronize()
        elapsed_ms = e0.elapsed_time(e1)
        if dist is not None:
            t = torch.tensor([elapsed_ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            elapsed_ms = float(t.item())
            dist.barrier()
        torch.cuda.synchronize()
        out = torch.empty_like(u0_dev)
        B.ge_read_state(ctx, out)
        B.ge_sync(ctx)
    got = out.cpu().numpy()
    clocks = sampler.summary()
    # measured ALU ceiling of the main line's precision, right after the timed region
    probe = None
    if not args.no_probe and args.kernel != "temporal_df":
        p_prec = B.GE_F64 if prec == B.GE_F64 else B.GE_F32
        fma_s, cps, chains = fma_probe(B, torch, dev, stream, p_prec, SMS)
        mhz = clocks.get("sm_mhz") or sm_max_mhz
        probe = {"fma_per_s": fma_s, "flops_per_s": 2.0 * fma_s,
                 "fma_per_clk_per_sm": fma_s / (SMS * mhz * 1e6), "sm_mhz": mhz, "sms": SMS,
                 "best_ctas_per_sm": cps, "best_chains": chains,
                 "how": "ge_probe_fma: %s chains in registers, CTAs of 256 threads; best over 1, 2, 4 CTAs per SM "
                        "and 8, 16, 32 chains per thread; CUDA events; per-SM rate at the median SM clock of the "
                        "timed region" % ("DFMA" if p_prec == B.GE_F64 else "FFMA")}

    ms_per_step = elapsed_ms / args.steps
    updates = float(N_POINTS) * GE_STEPS
    value = updates * world / (ms_per_step / 1e3)
    n_launch = launches_per_solve(args.kernel, depth)
    n_tiled = (GE_STEPS + depth - 1) // depth if args.kernel in ("temporal", "temporal_df") else n_launch
    launch_ms = ms_per_step / n_tiled  # the dominant kernel's average launch (prescale time included for DF)

    # ---- under torchrun: the batch sharded by problem, and config 2 as one
    # solve split over the ranks (every rank takes part) ---------------------
    batched_sharded = split_solve = None
    if dist is not None and not args.no_variants:
        batched_sharded = measure_batch_sharded(B, torch, inputs, dev, dist, rank, world, 3, 2)
        split_solve = measure_split_solve(B, torch, inputs, dev, dist, rank, world)

    if rank != 0:
        B.ge_destroy(ctx)
        if dist is not None:
            dist.destroy_process_group()
        return 0

    # ---- roofline of the dominant kernel ----------------------------------
    bytes_per_update = 8 if prec == B.GE_F64 else 4
    if args.kernel == "canonical":
        flops_per_update = 7.0    # one multiply and three multiply-adds, Eqs. (cc)/(dd)
    elif args.kernel == "onestep":
        flops_per_update = 4.0    # entry and exit multiply-adds (a one-step launch has no block step)
    elif prec == B.GE_F32_COMP:
        flops_per_update = 6.0    # normalised block map + Kahan sum, FP32
    else:
        flops_per_update = 2.0    # one multiply-add per point and step (right-hand-side form)
    alu_peak = 2.0 * FMA_PER_CLK[args.precision] * SMS * sm_max_mhz * 1e6  # flop/s
    if args.subdomain > 1:
        # width-k sweeps: three dependent DP operations per point (Saul'yev A / B)
        flops_per_update = 6.0
        sweep_steps = GE_STEPS / n_launch
        achieved = flops_per_update * N_POINTS * sweep_steps / (launch_ms / 1e3)
        roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": alu_peak / 1e12, "unit": "TFLOP/s",
                    "frac": achieved / alu_peak, "traffic": None,
                    "peak_source": "derived: %g FMA/clk/SM x %d SMs x %.0f MHz"
                    % (FMA_PER_CLK[args.precision], SMS, sm_max_mhz),
                    "kernel": "sweep_tb_kernel" if args.kernel == "temporal" else "sweep_smem_kernel"}
    elif args.kernel == "temporal_df":
        ops = DF_OPS_PER_UPDATE[two_r_is_fp32(R)]
        peak_ops = 128.0 * SMS * sm_max_mhz * 1e6
        achieved = ops * N_POINTS * (GE_STEPS / n_tiled) / (launch_ms / 1e3)
        kname = "tb_df_kernel<%s>" % ("false" if two_r_is_fp32(R) else "true")
        roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                    "unit": "T FP32-pipe instructions/s", "frac": achieved / peak_ops,
                    "traffic": measured_traffic(kname),
                    "algorithmic_bytes_per_launch": 2 * bytes_per_update * N_POINTS,
                    "ops_per_update": ops,
                    "peak_source": "derived: 128 FP32 instructions/clk/SM x %d SMs x %.0f MHz" % (SMS, sm_max_mhz),
                    "kernel": kname}
    elif args.kernel == "temporal":
        updates_per_launch = N_POINTS * (GE_STEPS / n_launch)
        # FP64: a build-fixed share of the interior updates runs as exact FP64
        # multiply-adds on the integer pipes; the FP64 unit does the rest
        int_share = B.ge_fp64_int_share() if prec == B.GE_F64 else 0.0
        unit_flops_per_update = flops_per_update * (1.0 - int_share)
        achieved = unit_flops_per_update * updates_per_launch / (launch_ms / 1e3)
        kname = "tb_kernel<%s>" % ("double" if prec == B.GE_F64 else "float")
        traffic = measured_traffic(kname) if (prec == B.GE_F64 and depth == 48) else None
        if prec == B.GE_F32_COMP:
            work = "normalised block map + Kahan sum"
        elif int_share > 0:
            work = ("one multiply-add per point and step (right-hand-side form); %.0f %% of the interior updates "
                    "as exact FP64 multiply-adds on the integer pipes, the rest on the FP64 unit (achieved and "
                    "frac count the FP64 unit's share)" % (100 * int_share))
        else:
            work = "one multiply-add per point and step (right-hand-side form)"
        roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": alu_peak / 1e12,
                    "unit": "TFLOP/s", "frac": achieved / alu_peak,
                    "traffic": traffic, "algorithmic_bytes_per_launch": 2 * bytes_per_update * N_POINTS,
                    "kernel": kname,
                    # achieved = executed_flops_per_update x updates_per_launch / launch_ms
                    "executed_flops_per_update": unit_flops_per_update,
                    "executed_work": work,
                    "int_pipe_share": int_share,
                    "updates_per_launch": updates_per_launch, "launch_ms": launch_ms,
                    # peak = 2 flops x FMA/clk/SM x SMs x max SM clock
                    "peak_source": "derived: 2 flops x %g FMA/clk/SM x %d SMs (device attribute) x %.0f MHz "
                                   "(max SM clock); the probe below measures the same ceiling in this run"
                                   % (FMA_PER_CLK[args.precision], SMS, sm_max_mhz),
                    "method_flops_per_update": METHOD_FLOPS_PER_UPDATE if prec == B.GE_F64 else None,
                    "method_bytes_per_update": 2 * bytes_per_update}
        if probe is not None:
            roofline["peak_probe"] = probe["flops_per_s"] / 1e12
            roofline["frac_of_probe"] = achieved / probe["flops_per_s"]
            if int_share > 0:
                # every update's multiply-add against the FP64 unit's measured
                # ceiling: above 1 is what the integer pipes add
                roofline["all_updates_frac_of_probe"] = (flops_per_update * updates_per_launch
                                                         / (launch_ms / 1e3) / probe["flops_per_s"])
    else:
        # one step per launch: report the roofline that binds (HBM bytes or
        # the ALU), with the other fraction beside it
        byt = 2.0 * bytes_per_update * N_POINTS
        achieved = byt / (launch_ms / 1e3)
        hbm_frac = achieved / (hbm_gbs * 1e9)
        flops = flops_per_update * N_POINTS / (launch_ms / 1e3)
        alu_frac = flops / alu_peak
        kname = "canon_kernel" if args.kernel == "canonical" else "tb_kernel (1 step/launch)"
        if alu_frac >= hbm_frac:
            roofline = {"bound": "alu", "achieved": flops / 1e12, "peak": alu_peak / 1e12, "unit": "TFLOP/s",
                        "frac": alu_frac, "traffic": None, "hbm_frac": hbm_frac,
                        "peak_source": "derived: %g FMA/clk/SM x %d SMs x %.0f MHz"
                        % (FMA_PER_CLK[args.precision], SMS, sm_max_mhz), "kernel": kname}
        else:
            roofline = {"bound": "hbm", "achieved": achieved / 1e9, "peak": hbm_gbs, "unit": "GB/s",
                        "frac": hbm_frac, "traffic": None, "alu_frac": alu_frac,
                        "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)", "kernel": kname}
    hbm_roof_updates = hbm_gbs * 1e9 / (2.0 * bytes_per_update)
    # effective HBM fraction: the updates/s over the one-step HBM roofline
    # (method bytes per update over the measured copy bandwidth)
    roofline["hbm_effective_frac"] = value / world / hbm_roof_updates
    # HBM fraction from the bytes the dominant kernel actually moves (ncu DRAM counters per launch)
    hbm_actual = None
    if roofline.get("traffic"):
        steps_per_launch = GE_STEPS / n_tiled
        gbs = roofline["traffic"] / (launch_ms / 1e3) / 1e9
        hbm_actual = {"bytes_per_launch": roofline["traffic"], "steps_per_launch": steps_per_launch,
                      "bytes_per_step": roofline["traffic"] / steps_per_launch, "achieved_gbs": gbs,
                      "peak_gbs": hbm_gbs, "frac": gbs / hbm_gbs,
                      "source": "dram__bytes_read.sum + dram__bytes_write.sum of one launch (profiles/traffic.txt) "
                                "over the live average launch time"}

    # ---- accuracy against the oracle (sampled) ----------------------------
    idx = sample_indices(N_POINTS)
    scale = float(np.max(np.abs(u0)))
    acc, want = None, None
    if not args.no_accuracy or not args.no_variants:
        want = oracle_reference(u0, idx)
        acc = errors(got[idx], want, scale) if args.subdomain == 1 else {
            "skipped": "width k > 1: the sampled reference is the k = 1 scheme (the width-k path is checked "
                       "bit for bit against the oracle's width-k step in the tests)"}

    # ---- end to end through the public API with host buffers --------------
    e2e = {"value": None, "unit": UNIT, "skipped": "--no-e2e"}
    if not args.no_e2e:
        try:
            e2e = measure_e2e(B, torch, u0, prec, kern, depth, args.steps, world)
        except Exception as exc:  # report, never hide
            e2e = {"value": None, "unit": UNIT, "error": str(exc)}

    # ---- variants: one-step kernels and FP32 paths -------------------------
    variants = {}
    if not args.no_variants:
        flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

        def flush():
            flush_buf.fill_(1)
        for vp, vk, vd in (("f64", "temporal_df", 96), ("f64", "temporal_df", 1), ("f64", "onestep", 1),
                           ("f64", "canonical", 1),
                           ("f32", "temporal", 128), ("f32c", "temporal", 64), ("f32", "onestep", 1),
                           ("f64", "subdomain16", 8), ("f64", "subdomain16_onestep", 1)):
            if (vp, vk) == (args.precision, args.kernel) and (vd == depth or vk not in ("temporal", "temporal_df")):
                continue
            p2 = {"f64": B.GE_F64, "f32": B.GE_F32, "f32c": B.GE_F32_COMP}[vp]
            width = 16 if vk.startswith("subdomain16") else 1
            # width 16: `depth` steps per launch on a tile in shared memory, or one launch per step
            k2 = {"temporal": B.GE_KERNEL_TEMPORAL, "temporal_df": B.GE_KERNEL_TEMPORAL_DF,
                  "onestep": B.GE_KERNEL_ONESTEP, "canonical": B.GE_KERNEL_CANONICAL,
                  "subdomain16": B.GE_KERNEL_TEMPORAL, "subdomain16_onestep": B.GE_KERNEL_CANONICAL}[vk]
            x2 = torch.from_numpy(u0).to(dev, dtype=B.dtype_of(p2))
            with torch.cuda.stream(stream):
                c2 = B.ge_create(N_POINTS, R, 0.0, 0.0, p2, x2, stream=stream)
                B.ge_set_kernel(c2, k2, vd)
                B.ge_set_subdomain_width(c2, width)
                ms = time_solver(B, torch, c2, x2, 2, 1, stream, flush=flush)
                o2 = torch.empty_like(x2)
                B.ge_read_state(c2, o2)
                B.ge_sync(c2)
                B.ge_destroy(c2)
            bpu = 8 if p2 == B.GE_F64 else 4
            upd_s = updates / (ms / 1e3)
            ent = {"updates_per_s": upd_s, "ms_per_step": ms,
                   "hbm_roofline_frac_1step": upd_s / (hbm_gbs * 1e9 / (2.0 * bpu)),
                   "launches_per_step": launches_per_solve(vk, vd)}
            if width == 1:
                ent.update(errors(o2.cpu().numpy().astype(np.float64)[idx], want, scale))
            else:
                ent["scheme"] = "sub-domain width k = 16 (the paper's 32-node sub-domain couples)"
            if vk == "temporal_df":
                ops = DF_OPS_PER_UPDATE[two_r_is_fp32(R)]
                ent.update({"arithmetic": "double-float on the FP32 pipes (FP64 storage and API)",
                            "ops_per_update": ops,
                            "alu_frac": ops * upd_s / (128.0 * SMS * sm_max_mhz * 1e6),
                            "vs_f64_temporal": upd_s / value if args.kernel == "temporal" else None})
            variants[f"{vp}_{vk}" + (f"_d{vd}" if vk.startswith("temporal") or vk == "subdomain16" else "")] = ent
            del x2, o2
        del flush_buf

    # ---- batched workload (many uneven problems, one graph per solve) ------
    batched = None
    if not args.no_variants and world == 1:
        batched = measure_batch(B, torch, inputs, dev, 3, 2)

    # ---- learned surrogate with the GE fallback ----------------------------
    surrogate = sweep = None
    if not args.no_surrogate and world == 1:
        surrogate = measure_surrogate(B, torch, inputs, args.sno_train_steps)
        if not args.no_sno_sweep:
            sweep = measure_surrogate_k_sweep(B, torch, inputs, args.sno_train_steps)

    # ---- CPU baseline: the oracle on a bounded sample -----------------------
    cpu = None
    if not args.no_cpu:
        import oracle
        t0 = time.perf_counter()
        oracle.run(u0, R, 0.0, 0.0, CPU_SAMPLE_STEPS)
        t_cpu = time.perf_counter() - t0
        cpu = {"value": N_POINTS * CPU_SAMPLE_STEPS / t_cpu, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{CPU_SAMPLE_STEPS} GE steps over the full N=2^24 grid (serial FP64 C)",
               "seconds": t_cpu}
        try:
            v_all, cores, wall = oracle_all_cores(u0, R, CPU_SAMPLE_STEPS)
            cpu_all = {"value": v_all, "unit": UNIT, "cores": cores, "kind": "oracle",
                       "sample": f"{CPU_SAMPLE_STEPS} GE steps over the full N=2^24 grid, the serial oracle on "
                                 f"one dependency-cone window per core ({cores} spawned processes)",
                       "seconds": wall}
        except Exception as exc:  # reported, not fatal: the one-core baseline stands
            cpu_all = {"unavailable": f"{type(exc).__name__}: {exc}"}
    else:
        cpu_all = None

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.precision if args.precision != "f32c" else "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N_POINTS, "r": R, "ge_steps": GE_STEPS,
                   "precision": args.precision, "kernel": args.kernel, "depth": depth,
                   "parallelism": f"independent problem per GPU x{world}",
                   "l2": "inputs larger than L2 (two %d MB state buffers); no flush"
                         % (N_POINTS * bytes_per_update >> 20)},
        "roofline": roofline,
        "hbm_actual": hbm_actual,
        "hbm_roofline_frac_effective": value / world / hbm_roof_updates,
        "cpu_baseline": cpu,
        "cpu_baseline_all_cores": cpu_all,
        "paper_context": PAPER_CONTEXT,
        "e2e": e2e,
        "gpu_launches": n_launch * args.steps,
        "kernel_ms_per_launch": launch_ms,
        "clocks": clocks,
        "alu_probe": probe,
        "accuracy": acc,
        "variants": variants,
        "batched": batched,
        "batched_sharded": batched_sharded,
        "split_solve": split_solve,
        "surrogate": surrogate,
        "surrogate_k_sweep": sweep,
    }
    B.ge_destroy(ctx)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
