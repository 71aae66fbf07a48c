"""Benchmark: high-order NPFs of an n = 120 block-structured system, orders 3 and 4.

One step = one npf_compute(order=4) through the C ABI: the order-3 and order-4 modal
contractions (Algorithm 2 steps 1-11), the Khatri-Rao reductions (steps 12-19) and the NPF finish
(step 20), on inputs already resident in device memory. Metric: modal-tensor entries per second,
entries = n^4 + n^5 per step (every h^i_{p_1..p_N} of both orders, counted densely).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--precision P]

Multi-GPU (torchrun, one process per GPU): each rank computes its own system (seed = rank),
no collective on the data path ("scaling": "weak"); value = all ranks' entries / max time.
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
WORKLOADS = {"n120": (120, (3, 4)), "n60": (60, (3, 4)), "n120o3": (120, (3,))}
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


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


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
            "sample": f"order-3 contraction + reduction, n=120, p_1 in [0,{done}) "
                      f"({ents} entries, {dt:.1f} s)"}


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        pass
    vals = []
    cb = None
    for _ in range(max(1, args.steps)):
        cb = cpu_baseline(seconds_budget=min(20.0, 150.0 / max(1, args.steps)))
        vals.append(cb["value"])
    v = statistics.median(vals)
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "entries/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "n=120 block-structured system, order 3 sample (CPU oracle)",
                       "n": N_STATES, "orders": [3]},
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
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--tile-n", type=int, default=0,
                    help="complex columns per tensor-core tile (16/32/64; 0 = library default)")
    ap.add_argument("--workload", default="n120", choices=list(WORKLOADS),
                    help="n120: the measured configuration; the others are small cases for "
                         "profiler captures")
    args = ap.parse_args()
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

    global N_STATES, ORDERS
    N_STATES, ORDERS = WORKLOADS[args.workload]
    sysm = S.config_blocks(N_STATES, rank, orders=ORDERS)
    n = sysm.n
    stream = torch.cuda.current_stream()
    plan = npf.Plan(sysm.lam, sysm.U, sysm.V, max(ORDERS), precision=args.precision,
                    stream=stream.cuda_stream)
    if args.tile_n:
        plan.set_option(npf.OPT_TILE_N, args.tile_n)
    dev_tensors = {N: torch.from_numpy(sysm.tensors[N]).cuda() for N in ORDERS}
    for N in ORDERS:
        plan.set_tensor(N, dev_tensors[N])
    out = torch.empty((n, n), dtype=torch.complex128, device="cuda")

    def step():
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
    if dist:
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ents = entries_per_step(n) * world
    value = ents / (ms * 1e-3)

    # ---- roofline of the dominant kernel (live CUDA-event durations of the timed steps)
    peaks, src = measured_peaks()
    roof = None
    if prof:
        name, (cnt, tot_ms) = max(prof.items(), key=lambda kv: kv[1][1])
        work, kind = algorithmic_work_per_step(name, n, args.precision)
        if work is not None:
            per_launch = work * args.steps / cnt
            avg_ms = tot_ms / cnt
            if kind == "flops":
                peak = peaks.get("bf16_tflops_sustained", 1700.0)
                achieved = per_launch / (avg_ms * 1e-3) / 1e12
                bound, unit, psrc = "tensor", "TFLOP/s", f"bf16 sustained ({src})"
            else:
                peak = peaks.get("hbm_gbs", 6800.0)
                achieved = per_launch / (avg_ms * 1e-3) / 1e9
                bound, unit, psrc = "hbm", "GB/s", f"hbm copy ({src})"
            roof = {"kernel": name, "bound": bound, "achieved": achieved, "peak": peak,
                    "unit": unit, "frac": achieved / peak, "traffic": None, "peak_source": psrc,
                    "launches": cnt, "avg_ms": avg_ms,
                    "share": tot_ms / sum(v[1] for v in prof.values())}

    # ---- end to end through the C ABI from pinned host buffers
    e2e = None
    if not args.no_e2e:
        host_t = {N: torch.from_numpy(sysm.tensors[N]).pin_memory() for N in ORDERS}
        host_out = torch.empty((n, n), dtype=torch.complex128).pin_memory()
        h2d = sum(int(t.numel() * 8) for t in host_t.values())
        d2h = int(host_out.numel() * 16)

        def e2e_step():
            for N in ORDERS:
                plan.set_tensor(N, host_t[N])
            plan.compute(max(ORDERS), host_out)

        e2e_step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        steps_e2e = max(1, min(args.steps, 3))
        t0 = time.perf_counter()
        for _ in range(steps_e2e):
            e2e_step()
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / steps_e2e
        e2e = {"value": entries_per_step(n) * world / dt, "unit": "entries/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": dt * 1e3}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "entries/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"split_bf16": "bf16x5-split (fp64-emulating)", "fp32": "bf16x3-split",
                      "fp64": "f64"}[args.precision],
            "data": "synthetic",
            "config": {"workload": f"n={n} block-structured system ({n // 4} blocks x 4 states), "
                                   f"NPF orders {', '.join(map(str, ORDERS))}, packed symmetric "
                                   "tensors 30% N(0,1)",
                       "n": n, "orders": list(ORDERS), "precision": args.precision,
                       "entries_per_step": entries_per_step(n),
                       "l2": "inputs larger than L2 (packed order-4 tensor 8.7 GB)"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk, "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in prof.items()},
        }
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    plan.close()
    return 0


PAIRS = {"split_bf16": 21, "fp32": 6, "fp64": 1}     # BF16 slice pairs s + t < S (S = 6 / 3)
SLICES = {"split_bf16": 6, "fp32": 3, "fp64": 0}


def algorithmic_work_per_step(name, n, precision):
    """Algorithmic work of every launch of `name` in one step, as (amount, kind).

    Tensor kernels (kind "flops"): executed BF16 tensor flops of the work the symmetric method
    needs -- only non-decreasing lower-index tuples are formed, indices unpadded (n, not 128);
    a complex multiply-add over K is 8 real flops, times the slice pairs. Per order N with
    C(m, r) = binomial:
      split_upper_contraction : C(n+N-1,N) packed tuples x n (i) x n (j) x 4 (real x complex)
      split_mode_product      : sum_{c=1..N-1} n (i) x C(n+c-1,c) (sorted p's) x n^(N-c) (a's)
                                x n (K) x 8
      split_mode_divide       : n (i) x C(n+N-1,N) x n (K) x 8
      split_reduce            : n (i) x C(n+N-2,N-1) (rows) x n (k) x n (K) x 8
    Memory kernels (kind "bytes"): split_expand gathers one 32-byte digit record and writes
    S planes x 4 bytes per dense operand entry: n (i) x n^N x (32 + 4 S).
    """
    from math import comb
    pairs = PAIRS[precision]
    tot = 0
    for N in ORDERS:
        if name == "split_upper_contraction":
            tot += comb(n + N - 1, N) * n * n * 4 * pairs
        elif name == "split_mode_product":
            tot += sum(n * comb(n + c - 1, c) * n ** (N - c) * n * 8 for c in range(1, N)) * pairs
        elif name == "split_mode_divide":
            tot += n * comb(n + N - 1, N) * n * 8 * pairs
        elif name == "split_reduce":
            tot += n * comb(n + N - 2, N - 1) * n * n * 8 * pairs
        elif name == "split_expand":
            tot += n * n ** N * (32 + 4 * SLICES[precision])
        elif name == "fp64_mode_product":
            tot += (N - 1) * n ** (N + 2) * 8
        else:
            return None, None
    return tot, ("bytes" if name == "split_expand" else "flops")


if __name__ == "__main__":
    sys.exit(main())
