"""Benchmark: high-order NPFs of an n = 120 block-structured system, orders 3 and 4.

One step = one npf_compute(order=4) through the C ABI: the order-3 and order-4 modal
contractions (Algorithm 2 steps 1-11), the Khatri-Rao reductions (steps 12-19) and the NPF finish
(step 20), on inputs already resident in device memory. Metric: modal-tensor entries per second,
entries = n^4 + n^5 per step (every h^i_{p_1..p_N} of both orders, counted densely).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--precision P]

Multi-GPU (torchrun, one process per GPU): by default the upper-index rows of the one n = 120
system are split over the ranks (paper_2509_08968_gb300.shard.sharded_npf: each rank forms its rows
of Psi_3 and Psi_4, one NCCL all-reduce of the n x n terms, the NPF finish), "scaling": "strong";
with --replicas each rank computes its own system (seed = rank) with no collective on the data
path, "scaling": "weak". value = all ranks' entries / max time.
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

N_STATES = 120
ORDERS = (3, 4)
# name -> (n, orders)
WORKLOADS = {"n120": (120, (3, 4)), "n60": (60, (3, 4)), "n120o3": (120, (3,)),
             "batch256": (None, (2, 3)), "surrogate": (40, (2, 3)), "swing120": (120, (3, 4))}
METRIC = "modal-tensor entries/s & % roofline, split-prec vs native FP64 at rel err <=1e-10"


def entries_per_step(n, orders=None):
    return sum(n ** (N + 1) for N in (ORDERS if orders is None else orders))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def code_hash(paths):
    """SHA-256 of source files with their comments and whitespace removed: edits that leave the
    code itself unchanged keep the hash."""
    import hashlib
    import re
    h = hashlib.sha256()
    for path in paths:
        with open(path, encoding="utf-8") as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)   # block comments
        text = re.sub(r"//[^\n]*", " ", text)                   # line comments
        h.update("".join(text.split()).encode())
    return h.hexdigest()


def measured_traffic(kernel, workload):
    """DRAM bytes (read + write) per launch of `kernel` on `workload` from the committed ncu
    capture profiles/dram_<kernel>_<workload>.json, or None when there is none or when the kernel
    sources' code no longer hashes to the captured build's."""
    p = os.path.join(ROOT, "profiles", f"dram_{kernel}_{workload}.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    current = code_hash([os.path.join(ROOT, src) for src in d["sources"]])
    return d["traffic_per_launch"] if current == d["code_sha256"] else None


class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 4 + k and r[4 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate(dist, t, units):
    """Whole-job view of one rank's step: (max of t over ranks, sum of units over ranks). Every
    rank works on its own problem (weak scaling), so this pair is the only exchange; on NCCL the
    values travel on the GPU, on gloo on the host."""
    if dist is None:
        return t, units
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    tm = torch.tensor([float(t)], dtype=torch.float64, device=dev)
    us = torch.tensor([float(units)], dtype=torch.float64, device=dev)
    dist.all_reduce(tm, op=dist.ReduceOp.MAX)
    dist.all_reduce(us, op=dist.ReduceOp.SUM)
    return float(tm.item()), float(us.item())


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def workload_config(n, orders, precision, swing=False, modes=None):
    """The `config` of a single-system workload line (both arms)."""
    from math import comb
    return {"workload": (f"n={n} swing model ({n // 2} machines, ring + random lines), NPF orders "
                         f"{', '.join(map(str, orders))}, derivative tensors generated on the GPU")
                        if swing else
                        (f"n={n} block-structured system ({n // 4} blocks x 4 states), NPF orders "
                         f"{', '.join(map(str, orders))}, packed symmetric tensors 30% N(0,1)"),
            "n": n, "orders": list(orders), "precision": precision,
            "entries_per_step": sum((modes or n) ** (N + 1) for N in orders),
            # distinct entries (h is symmetric in its lower indices): what the method forms
            "unique_entries_per_step": sum((modes or n) * comb((modes or n) + N - 1, N)
                                           for N in orders),
            "modes": modes or n,
            "l2": "inputs larger than L2 (packed order-4 tensor 8.7 GB)"}


def fp64_equivalent(n, m, orders, ms):
    """The whole step as the dense FP64 work of Algorithm 2: F(n, N) = 2n(4N + 6) real flops per
    entry of the dense m^(N+1) modal tensor (one real x complex and N complex x complex products of
    length n, and the Khatri-Rao step). The method forms only non-decreasing tuples (up to N!
    fewer), so this is the rate a dense FP64 code would need, not work the GPU executes; the
    measured comparison with the native FP64 form is the `vs_fp64` object."""
    F = {N: 2 * n * (4 * N + 6) for N in orders}
    flops = sum(m ** (N + 1) * F[N] for N in orders)
    tflops = flops / (ms * 1e-3) / 1e12
    return {"flops_per_entry": {str(N): F[N] for N in orders}, "tflops": tflops,
            "note": "dense-count rate; only sorted tuples are formed, so not comparable with a "
                    "pipe's peak"}


def measure_fp64_peak(reps=5, size=4096):
    """Dense FP64 rate of this GPU: torch.matmul on float64 size^3 (cuBLAS DGEMM), best of
    `reps` back-to-back products timed with CUDA events, with the SM clock sampled meanwhile."""
    import torch
    a = torch.randn(size, size, dtype=torch.float64, device="cuda")
    b = torch.randn(size, size, dtype=torch.float64, device="cuda")
    c = a @ b
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b, out=c)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    clk = clocks.stop()
    del a, b, c
    return {"tflops": 2.0 * size ** 3 / (best * 1e-3) / 1e12,
            "how": f"torch.matmul float64 {size}^3 (cuBLAS DGEMM), best of {reps}, CUDA events",
            "sm_mhz": clk.get("sm_mhz"), "reasons": clk.get("reasons")}


def cpu_baseline(seconds_budget=20.0):
    """The CPU oracle as it stands on the host cores: order-3 modal contraction plus reduction
    of the n = 120 system for as many leading p_1 values as fit the time budget."""
    import npf_synth as S
    import oracle
    sysm = S.config_n120(0, orders=(3,))
    n, N = N_STATES, 3
    oracle.build()
    t0 = time.perf_counter()
    done = 0
    while done < n and time.perf_counter() - t0 < seconds_budget:
        oracle.psiN_partial(sysm.tensors[N], n, N, sysm.U, sysm.V, sysm.lam, done, done + 1)
        done += 1
    dt = time.perf_counter() - t0
    ents = done * n ** N            # h^i_{p_1 p_2 p_3} for the sampled p_1
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": ents / dt, "unit": "entries/s", "cores": cores, "kind": "oracle",
            "sample": f"order-3 share of the n=120 orders-3+4 workload only: contraction + "
                      f"reduction for p_1 in [0,{done}) ({ents} entries, {dt:.1f} s); one order-4 "
                      f"p_1 slice alone is n^4 entries (~1 min on 16 cores), beyond the sample's "
                      f"budget, and costs ~5/4 as much per entry"}


def cpu_baseline_one_core(seconds_budget=8.0):
    """The same sample on one host core (OMP_NUM_THREADS=1 in a child process, since the
    oracle's OpenMP runtime reads it at start-up)."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample",
                        str(seconds_budget)], env=env, capture_output=True, text=True,
                       timeout=600)
    if r.returncode:
        return {"error": r.stderr[-300:]}
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_reference(args):
    """The CPU oracle on the default workload's config: every step is a bounded sample of it (the
    order-3 contraction and reduction for the leading p_1 values that fit the step's budget), the
    value its entries per second."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    budget = min(20.0, 150.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_baseline(seconds_budget=min(budget, 2.0))
    vals, secs = [], []
    cb = None
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        cb = cpu_baseline(seconds_budget=budget)
        secs.append(time.perf_counter() - t0)
        vals.append(cb["value"])
    v = statistics.median(vals)
    cb["value"] = v
    cb["sample_ms_per_step"] = statistics.median(secs) * 1e3
    config = workload_config(N_STATES, ORDERS, "fp64 (CPU oracle)")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "entries/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            # a whole step of the workload at the sampled rate (each timed step is a sample)
            "ms_per_step": config["entries_per_step"] / v * 1e3,
            "ms_per_step_kind": "extrapolated: entries_per_step / sampled rate (each timed step "
                                "is a bounded sample, cpu_baseline.sample_ms_per_step)",
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config,
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "entries/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="split_bf16", choices=["split_bf16", "fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--replicas", action="store_true",
                    help="multi-GPU: one independent system per rank (weak scaling) instead of the "
                         "row-sharded system")
    ap.add_argument("--no-fp64", action="store_true",
                    help="skip the native-FP64 comparison and the DGEMM peak measurement")
    ap.add_argument("--cpu-sample", type=float, default=0.0, help=argparse.SUPPRESS)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--tile-n", type=int, default=0,
                    help="complex columns per tensor-core tile (16/32/48/64; 0 = library default)")
    ap.add_argument("--modes", type=int, default=0,
                    help="critical-mode subset: the m least-damped modes (0 = all modes)")
    ap.add_argument("--mem-budget", type=float, default=0.0,
                    help="device memory for intermediates in GB (0 = the library default, 80%% of "
                         "free memory); small values keep profiler captures small")
    ap.add_argument("--workload", default="n120", choices=list(WORKLOADS),
                    help="n120: the measured configuration; the others are small cases for "
                         "profiler captures")
    args = ap.parse_args()
    if args.cpu_sample:
        print(json.dumps(cpu_baseline(seconds_budget=args.cpu_sample)))
        return 0
    if args.impl == "reference":
        return run_reference(args)

    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import npf_synth as S
    import paper_2509_08968_gb300 as npf
    from paper_2509_08968_gb300 import build
    build.build()
    if args.workload == "batch256":
        return run_batch(args, world, rank, local, dist)
    if args.workload == "surrogate":
        return run_surrogate(args, world, rank, local, dist)

    global N_STATES, ORDERS
    N_STATES, ORDERS = WORKLOADS[args.workload]
    swing = args.workload.startswith("swing")
    # several GPUs: the rows of one system split over the ranks, unless replicas are asked for
    sharded = world > 1 and not args.replicas and not args.modes
    seed = 0 if sharded else rank
    if swing:   # tensors generated on the GPU from a 60-machine swing model
        model = S.swing_model(N_STATES // 2, seed)
        sysm = S.swing_system(model)
    else:
        sysm = S.config_blocks(N_STATES, seed, orders=ORDERS)
    n = sysm.n
    stream = torch.cuda.current_stream()
    plan = npf.Plan(sysm.lam, sysm.U, sysm.V, max(ORDERS), precision=args.precision,
                    stream=stream.cuda_stream)
    if args.tile_n:
        plan.set_option(npf.OPT_TILE_N, args.tile_n)
    if args.mem_budget:
        plan.set_option(npf.OPT_MEM_BUDGET, args.mem_budget * 2**30)
    subset = None
    if args.modes and args.modes < n:
        # least damped first (largest real part), ties by index
        subset = np.argsort(-sysm.lam.real, kind="stable")[:args.modes]
        plan.set_mode_subset(subset)
    if swing:
        for N in ORDERS:
            plan.set_tensor_swing(N, model)
    else:
        dev_tensors = {N: torch.from_numpy(sysm.tensors[N]).cuda() for N in ORDERS}
        for N in ORDERS:
            plan.set_tensor(N, dev_tensors[N])
    out = torch.empty((n, n), dtype=torch.complex128, device="cuda")
    from paper_2509_08968_gb300 import shard
    lo, hi = shard.row_ranges(n, world)[rank] if sharded else (0, n)

    def step():
        if sharded:
            shard.sharded_npf(plan, ORDERS, dist, out=out)
        else:
            plan.compute(max(ORDERS), out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- timed region: inputs resident in HBM
    plan.set_option(npf.OPT_PROFILE, 1)
    plan.profile(reset=True)
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = npf.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = npf.launch_count() - l0
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    prof = plan.profile(reset=True)
    plan.set_option(npf.OPT_PROFILE, 0)
    m_modes = len(subset) if subset is not None else n
    ents_rank = sum(m_modes ** (N + 1) for N in ORDERS)   # h^i_p with i, p in the modes used
    if sharded:
        ents_rank = ents_rank * (hi - lo) // n             # this rank's upper indices i
    ms, ents = aggregate(dist, ms, ents_rank)
    value = ents / (ms * 1e-3)

    # ---- roofline of the dominant kernel (live CUDA-event durations of the timed steps)
    peaks, src = measured_peaks()
    roof = None
    if prof:
        name, (cnt, tot_ms) = max(prof.items(), key=lambda kv: kv[1][1])
        work, kind = algorithmic_work_per_step(name, n, args.precision, m_modes)
        if work is not None:
            per_launch = work * args.steps / cnt
            avg_ms = tot_ms / cnt
            if kind == "flops" and name.startswith("fp64"):
                # FP64 pipe: this GPU's DGEMM rate measured in this run
                fp64_peak = measure_fp64_peak()
                peak = fp64_peak["tflops"]
                achieved = per_launch / (avg_ms * 1e-3) / 1e12
                bound, unit = "alu", "TFLOP/s"   # DFMA on the FP64 pipe
                psrc = (f"fp64 measured: {fp64_peak['how']}, SM clock {fp64_peak['sm_mhz']} MHz")
            elif kind == "flops":
                peak = peaks.get("bf16_tflops_sustained", 1700.0)
                achieved = per_launch / (avg_ms * 1e-3) / 1e12
                bound, unit, psrc = "tensor", "TFLOP/s", f"bf16 sustained ({src})"
            else:
                peak = peaks.get("hbm_gbs", 6800.0)
                achieved = per_launch / (avg_ms * 1e-3) / 1e9
                bound, unit, psrc = "hbm", "GB/s", f"hbm copy ({src})"
            roof = {"kernel": name, "bound": bound, "achieved": achieved, "peak": peak,
                    "unit": unit, "frac": achieved / peak,
                    "traffic": (measured_traffic(name, args.workload)
                                if args.precision == "split_bf16" and not (args.tile_n or args.modes)
                                else None),
                    "peak_source": psrc,
                    "launches": cnt, "avg_ms": avg_ms,
                    "share": tot_ms / sum(v[1] for v in prof.values())}

    # ---- error of the timed call against the oracle's stored values (n = 120 system, seed 0)
    rel_err = None
    if args.workload == "n120" and rank == 0 and subset is None:
        rel_err = stored_oracle_errors(plan, out, args.precision)

    # ---- the same box, same run: the native-FP64 form against the timed form on order 3
    vs_fp64 = None
    if (not args.no_fp64 and args.precision != "fp64" and not swing and subset is None
            and args.workload in ("n120", "n60") and rank == 0):
        vs_fp64 = compare_fp64(npf, sysm, plan, dev_tensors[3], stream, args.workload)

    # ---- end to end through the C ABI from pinned host buffers
    e2e = None
    if not args.no_e2e:
        host_out = torch.empty((n, n), dtype=torch.complex128).pin_memory()
        d2h = int(host_out.numel() * 16)
        if swing:   # the step's inputs are the model parameters; tensors generated on the GPU
            h2d = 8 * (3 * model.m + 2 * model.m * model.m) * len(ORDERS)
            how = "per step: model parameters uploaded, tensors generated on the GPU"

            def e2e_run(k):
                for _ in range(k):
                    for N in ORDERS:
                        plan.set_tensor_swing(N, model)
                    plan.compute(max(ORDERS), host_out)
        else:
            host_t = {N: torch.from_numpy(sysm.tensors[N]).pin_memory() for N in ORDERS}
            h2d = sum(int(t.numel() * 8) for t in host_t.values())
            how = ("per step: packed tensors from pinned host memory, step s + 1's uploading "
                   "during step s (npf_compute_prefetch); the first step's upload is not hidden")

            def e2e_run(k):
                if sharded:   # every rank uploads the whole tensors and forms its rows
                    for _ in range(k):
                        for N in ORDERS:
                            plan.set_tensor(N, host_t[N])
                        shard.sharded_npf(plan, ORDERS, dist, out=host_out)
                    return
                for N in ORDERS:
                    plan.set_tensor(N, host_t[N])
                for s_ in range(k):
                    plan.compute_prefetch(max(ORDERS), host_out, host_t if s_ + 1 < k else None)

        e2e_run(2)   # warm-up (allocates the staging buffers)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        steps_e2e = max(2, min(args.steps, 5))
        t0 = time.perf_counter()
        e2e_run(steps_e2e)
        torch.cuda.synchronize()
        dt, e_all = aggregate(dist, (time.perf_counter() - t0) / steps_e2e, ents_rank)
        if sharded:
            h2d, d2h = h2d * world, d2h * world
            how = "per step: every rank uploads the packed tensors from pinned host memory"
        e2e = {"value": e_all / dt, "unit": "entries/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": dt * 1e3,
               "steps": steps_e2e, "inputs": how}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()
        cpu["one_core"] = cpu_baseline_one_core()

    if rank == 0:
        config = workload_config(n, ORDERS, args.precision, swing, m_modes)
        config["parallelism"] = (f"rows of one system over {world} GPUs, one NCCL all-reduce of the "
                                 f"n x n terms per step" if sharded else
                                 f"{world} independent systems (one per GPU)" if world > 1 else
                                 "one GPU")
        line = {
            "metric": METRIC, "value": value, "unit": "entries/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "strong" if sharded else "weak",
            "vs_baseline": None,
            "dtype": DTYPES[args.precision],
            "data": "synthetic",
            "config": config,
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk, "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in prof.items()},
            "fp64_equivalent": fp64_equivalent(n, m_modes, ORDERS, ms),
            "rel_err": rel_err, "vs_fp64": vs_fp64,
        }
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    plan.close()
    return 0


GOLDEN = os.path.join(ROOT, "tests", "golden")
TOLERANCE = {"split_bf16": 1e-10, "fp32": 1e-5, "fp64": 1e-12}


def _rel(got, ref):
    return float(np.linalg.norm((got - ref).ravel()) / np.linalg.norm(ref.ravel()))


def stored_oracle_errors(plan, out, precision):
    """Relative Frobenius error of the timed call's NPF (the last step's output) and of the
    plan's Psi_3 and Psi_4 terms against values the complex128 CPU oracle wrote once for this
    system (tests/golden, written by tests/golden/make_golden.py)."""
    res = {"reference": "complex128 CPU oracle, stored (tests/golden)",
           "bar": TOLERANCE[precision]}
    files = {"psi3": ("n120_seed0_order3.npz", 3), "psi4": ("n120_seed0_order4.npz", 4)}
    for key, (fname, N) in files.items():
        path = os.path.join(GOLDEN, fname)
        if os.path.exists(path):
            res[key] = _rel(plan.term(N), np.load(path)[key])
    path = os.path.join(GOLDEN, "n120_seed0_npf34.npz")
    if os.path.exists(path):
        res["npf"] = _rel(out.cpu().numpy(), np.load(path)["npf"])
    return res


def compare_fp64(npf, sysm, plan, t3, stream, workload):
    """npf_compute(3) (order 3 alone) of the timed form and of the native-FP64 form on the same
    system, timed back to back with CUDA events on the library's stream, their errors against the
    stored oracle Psi_3 (n = 120), the FP64 mode-product kernel's rate and this GPU's measured
    DGEMM rate (the FP64 roof)."""
    import torch
    n = sysm.n
    out = torch.empty((n, n), dtype=torch.complex128, device="cuda")

    def timed(p, reps, warm):
        for _ in range(warm):
            p.compute(3, out)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            p.compute(3, out)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    split_ms = timed(plan, 5, 3)
    res = {"workload": f"n={n}, order 3 alone (npf_compute(3)), inputs resident",
           "split_ms": split_ms}
    with npf.Plan(sysm.lam, sysm.U, sysm.V, 3, precision="fp64",
                  stream=stream.cuda_stream) as p64:
        p64.set_tensor(3, t3)
        p64.set_option(npf.OPT_PROFILE, 1)
        fp64_ms = timed(p64, 2, 1)
        prof = p64.profile(reset=True)
        gold = os.path.join(GOLDEN, "n120_seed0_order3.npz")
        if workload == "n120" and os.path.exists(gold):
            ref = np.load(gold)["psi3"]
            res["split_rel_err_psi3"] = _rel(plan.term(3), ref)
            res["fp64_rel_err_psi3"] = _rel(p64.term(3), ref)
    res["fp64_ms"] = fp64_ms
    res["speedup"] = fp64_ms / split_ms
    peak = measure_fp64_peak()
    res["fp64_peak"] = peak
    if "fp64_mode_product" in prof:
        cnt, tot = prof["fp64_mode_product"]
        flops = (3 - 1) * n ** 5 * 8 * 3 / cnt      # 3 timed calls (1 warm-up + 2)
        achieved = flops / (tot / cnt * 1e-3) / 1e12
        res["fp64_mode_product"] = {"achieved_tflops": achieved, "frac_of_dgemm": achieved / peak["tflops"]}
    return res


def run_batch(args, world, rank, local, dist):
    """256 independent systems, n ~ U{20..80} (even), orders drawn from {2, 3}, about 5% of the
    ordered mode pairs within 1e-3 of a resonance; one npf_batch_compute per step (one recorded
    CUDA graph, tile widths autotuned). Metric: sum over systems of n^(N+1) per second."""
    import torch
    import npf_synth as S
    import paper_2509_08968_gb300 as npf
    systems = S.batch_systems(count=256, seed=rank)
    plans, orders, outs = [], [], []
    for sysm, N in systems:
        p = npf.Plan(sysm.lam, sysm.U, sysm.V, N, precision=args.precision)
        p.set_option(npf.OPT_TILE_N, args.tile_n)   # 0 = autotuned
        p.set_tensor(N, torch.from_numpy(sysm.tensors[N]).cuda())
        plans.append(p)
        orders.append(N)
        outs.append(torch.empty((sysm.n, sysm.n), dtype=torch.complex128, device="cuda"))
    ents = sum(s.n ** (N + 1) for s, N in systems)

    def step():
        npf.batch_compute(plans, orders, outs)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = npf.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()          # returns after its graph and copies have finished
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = npf.launch_count() - l0
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms, ents_all = aggregate(dist, ms, ents)
    value = ents_all / (ms * 1e-3)

    # whole-step tensor roofline: algorithmic (sorted-tuple, unpadded) BF16 flops of every system
    from math import comb
    pairs = PAIRS[args.precision]
    useful = executed = 0.0
    tiles = {}
    for s, N in systems:
        n = s.n
        f = n * comb(n + N - 1, N) * n * 4
        f += sum(n * comb(n + c - 1, c) * a_part(n, N, c) * n * 8 for c in range(1, N))
        f += n * comb(n + N - 1, N) * n * 8 + n * comb(n + N - 1, N) * n * 8
        f *= pairs
        t = args.tile_n or npf.tuned_tile(n, N, args.precision) or 64
        tiles[f"n{n}o{N}"] = t
        # padded tile shape: the row radix (32 / 64 / 128 >= n) per innermost row index, K' in
        # chunks of 32, t columns
        rad = 32 if n <= 32 else 64 if n <= 64 else 128
        r = (rad / n) * (32 * -(-2 * n // 32) / (2 * n)) * (t * -(-n // t) / n)
        useful += f
        executed += f * r
    peaks, src = measured_peaks()
    peak = peaks.get("bf16_tflops_sustained", 1700.0)
    achieved = useful / (ms * 1e-3) / 1e12
    roof = None
    if args.precision != "fp64":
        roof = {"kernel": "whole step (all systems)", "bound": "tensor", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "peak_source": f"bf16 sustained ({src})"}

    e2e = None
    if not args.no_e2e:
        host_t = [torch.from_numpy(s.tensors[N]).pin_memory() for s, N in systems]
        host_o = [torch.empty((s.n, s.n), dtype=torch.complex128).pin_memory() for s, _ in systems]
        h2d = sum(int(t.numel() * 8) for t in host_t)
        d2h = sum(int(o.numel() * 16) for o in host_o)

        def e2e_step():
            for p, N, t in zip(plans, orders, host_t):
                p.set_tensor(N, t)
            npf.batch_compute(plans, orders, host_o)

        e2e_step()
        steps_e2e = max(1, min(args.steps, 3))
        t0 = time.perf_counter()
        for _ in range(steps_e2e):
            e2e_step()
        dt, e_all = aggregate(dist, (time.perf_counter() - t0) / steps_e2e, ents)
        e2e = {"value": e_all / dt, "unit": "entries/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": dt * 1e3}
    if rank == 0:
        ns = [s.n for s, _ in systems]
        line = {
            "metric": METRIC, "value": value, "unit": "entries/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[args.precision], "data": "synthetic",
            "config": {"workload": "256 systems, n ~ U{20..80} (even), orders U{2,3}, ~5% of mode "
                                   "pairs within 1e-3 of resonance, one recorded graph per step",
                       "systems": len(systems), "n_min": min(ns), "n_max": max(ns),
                       "entries_per_step": ents, "precision": args.precision,
                       "padding_fraction_est": 1.0 - useful / executed if executed else None,
                       "tiles": tiles,
                       "l2": "inputs larger than L2 (packed tensors and scratch ~GBs)"},
            "roofline": roof, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
            "cpu_baseline": None,
        }
        print(json.dumps(line))
    for p in plans:
        p.close()
    if dist:
        dist.destroy_process_group()
    return 0


def run_surrogate(args, world, rank, local, dist):
    """Learned surrogate over a family of operating points (n = 40, orders 2 and 3): 4096
    training labels and 512 held-out labels from the plain method, an ensemble of five BF16 MLPs
    4 -> 256 -> 256 -> 256 -> 64 trained by the library, then one step = gated prediction of the
    512 held-out points (members' spread > 5% -> plain method). Metric: queries per second."""
    import torch
    import npf_synth as S
    from paper_2509_08968_gb300 import surrogate as SG
    fam = S.surrogate_family(40, rank)
    lam_ref = np.linalg.eigvals(fam.A(fam.p0))
    solver = SG.PlainSolver(fam, 3, lam_ref, slots=256, precision=args.precision)
    idx = SG.top_indices(solver.npf(fam.p0[None])[0], 64)
    solver.indices = idx
    Ptr = S.operating_points(fam, 4096, 2 * rank)
    Pte = S.operating_points(fam, 512, 2 * rank + 1)
    t0 = time.perf_counter()
    Ytr = solver.values(Ptr)
    t_label = time.perf_counter() - t0
    solver.values(Pte)                       # records the 256-system graph for this pool
    t0 = time.perf_counter()
    Yte = solver.values(Pte)
    t_plain = time.perf_counter() - t0
    sur = SG.Surrogate(fam, idx, [4, 256, 256, 256, 64], ensemble=5, seed=0)
    t0 = time.perf_counter()
    hist = sur.fit(Ptr, Ytr, epochs=300, batch=256, lr=1e-3, seed=0)
    t_train = time.perf_counter() - t0
    for _ in range(max(3, args.warmup)):
        sur.gated(Pte, solver, 0.05)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    from paper_2509_08968_gb300 import launch_count
    l0 = launch_count()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        out, spread, fb = sur.gated(Pte, solver, 0.05)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / args.steps
    launches = launch_count() - l0
    clk = clocks.stop()
    dt, q_all = aggregate(dist, dt, len(Pte))
    mean, _, _ = sur.predict(Pte, 0.05)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sur.predict(Pte, 0.05)
    t_sur = (time.perf_counter() - t0) / args.steps
    rel = np.abs(out - Yte) / Yte
    rel_ungated = np.abs(mean - Yte) / Yte
    if rank == 0:
        line = {
            "metric": "surrogate queries/s (gated at 5% ensemble spread, plain-method fallback)",
            "value": q_all / dt, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16 (MLP), " + DTYPES[args.precision]
            + " (fallback)", "data": "synthetic",
            "config": {"workload": "operating-point family n=40, NPF order 3 (A2, A3), p = (load "
                                   "scale U[0.6,1.2], 3 gains U[0.5,2]), top-64 |NPF|, 4096 train "
                                   "+ 512 held-out, ensemble 5 x MLP 4-256-256-256-64",
                       "l2": "small working set (latency-bound MLP), no L2 flush"},
            "surrogate": {"plain_queries_per_s": len(Pte) / t_plain,
                          "ungated_queries_per_s": len(Pte) / t_sur,
                          "speedup_gated_vs_plain": t_plain / dt,
                          "fallback_rate": float(fb.mean()),
                          # accepted rows whose worst output misses the 5% gate
                          "gate_miss_rate": float(((rel.max(axis=1) > 0.05) & ~fb).sum()
                                                  / max(1, int((~fb).sum()))),
                          "heldout_rel_err_gated": {"median": float(np.median(rel)),
                                                    "p95": float(np.percentile(rel, 95)),
                                                    "max": float(rel.max())},
                          "heldout_rel_err_ungated": {"median": float(np.median(rel_ungated)),
                                                      "p95": float(np.percentile(rel_ungated, 95)),
                                                      "max": float(rel_ungated.max())},
                          "train_s": t_train, "train_loss_first_last": [float(hist[0]),
                                                                        float(hist[-1])],
                          "label_queries_per_s": len(Ptr) / t_label},
            "roofline": None, "cpu_baseline": None,
            "e2e": {"value": q_all / dt, "unit": "queries/s", "h2d_bytes_per_step": 512 * 4 * 4,
                    "d2h_bytes_per_step": 512 * (64 * 4 + 8)},
            "gpu_launches": launches, "clocks": clk,
        }
        print(json.dumps(line))
    sur.close()
    solver.close()
    if dist:
        dist.destroy_process_group()
    return 0


DTYPES = {"split_bf16": "bf16x6-split (fp64-emulating)", "fp32": "bf16x4-split", "fp64": "f64"}
PAIRS = {"split_bf16": 21, "fp32": 10, "fp64": 1}    # BF16 slice pairs s + t < S (S = 6 / 4)
SLICES = {"split_bf16": 6, "fp32": 4, "fp64": 0}


def a_part(n, N, c):
    """Lower-input index tuples (a's) formed by contraction c: the innermost a is dense, shared
    a's are dense too except a pair of them, which is formed non-decreasing."""
    from math import comb
    sa = N - c - 1
    return (comb(n + 1, 2) if sa == 2 else n ** sa) * n


def algorithmic_work_per_step(name, n, precision, m=None):
    """Algorithmic work of every launch of `name` in one step, as (amount, kind).

    Tensor kernels (kind "flops"): executed BF16 tensor flops of the work the symmetric method
    needs -- only non-decreasing lower-index tuples are formed, indices unpadded (n, not 128);
    a complex multiply-add over K is 8 real flops, times the slice pairs. Per order N with
    C(m, r) = binomial:
      split_upper_contraction : C(n+N-1,N) packed tuples x n (i) x n (j) x 4 (real x complex)
      split_mode_product      : sum_{c=1..N-1} n (i) x C(n+c-1,c) (sorted p's) x A_c (a's)
                                x n (K) x 8, A_c = n^(N-c), except that two shared a's are
                                formed non-decreasing only: A_c = C(n+1,2) n when N-c-1 = 2
      split_mode_divide       : n (i) x C(n+N-1,N) x n (K) x 8
      split_reduce            : n (i) x C(n+N-1,N) (sorted rows x p_N >= p_{N-1}) x n (k) x 8
    Memory kernels (kind "bytes"): split_expand, per upper index i, gathers the n 32-byte digit
    records of every sorted prefix (a_1..a_{N-1}) once (C(n+N-2, N-1) prefixes) and writes S
    planes x 4 bytes per operand entry of every row whose shared a's are non-decreasing
    (C(n+N-3, N-2) x n rows of n entries): n (i) x [C(n+N-2,N-1) n 32 + C(n+N-3,N-2) n^2 4 S].
    """
    from math import comb
    pairs = PAIRS[precision]
    m = n if m is None else m          # modes in use (a critical-mode subset); states stay n
    tot = 0
    for N in ORDERS:
        if name == "split_upper_contraction":
            tot += comb(n + N - 1, N) * m * n * 4 * pairs
        elif name == "split_mode_product":
            tot += sum(m * comb(m + c - 1, c) * a_part(n, N, c) * n * 8 for c in range(1, N)) * pairs
        elif name == "split_mode_divide":
            tot += m * comb(m + N - 1, N) * n * 8 * pairs
        elif name == "split_reduce":
            tot += m * comb(m + N - 1, N) * n * 8 * pairs
        elif name == "split_expand":
            tot += m * (comb(n + N - 2, N - 1) * n * 32 +
                        comb(n + N - 3, N - 2) * n * n * 4 * SLICES[precision])
        elif name == "fp64_mode_product":
            tot += (N - 1) * n ** (N + 2) * 8
        else:
            return None, None
    return tot, ("bytes" if name == "split_expand" else "flops")


if __name__ == "__main__":
    sys.exit(main())
