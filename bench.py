#!/usr/bin/env python3
"""Benchmark: TS4 steps/s and HBM GB/s at N=28 (dipolar XXZ chain, complex64).

One "step" is one TS4 step U4(tau) applied in place to the 2^28-amplitude state
(all rotation layers and diagonal slots), i.e. one call of ts_step(tau, 1).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--prec c64|c128]

N > 1 runs N independent replicas (one process per GPU under torchrun): the path
has no exchange step, so value = total steps of all replicas / max time.
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TS4 steps/s and HBM GB/s (% of peak) at N=28, complex64 vs complex128 at stated err"
WORKLOAD = "N=28 open chain, dipolar XXZ (J^z=1/|i-j|^3, J^x=J^y=-J^z/2, 378 bonds), " \
           "random-phase state with spin 1 up, tau=0.01"
TAU = 0.01


KERNEL_SOURCES = ("paper_1305_0036_gb300/csrc/ts4_tile.cuh", "paper_1305_0036_gb300/csrc/ts4_kernels.cuh",
                  "paper_1305_0036_gb300/csrc/ts4_common.cuh")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_tile_traffic.txt")


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def measured_traffic(N):
    """DRAM bytes per complex64 k_tile launch from the committed ncu summary, scaled to 2^N
    amplitudes; None when the kernel sources changed since the counters were taken."""
    try:
        kv = {}
        with open(TRAFFIC_FILE) as f:
            for line in f:
                line = line.strip()
                if line and not line.startswith("#"):
                    k, v = line.split(None, 1)
                    kv[k] = v.strip()
        if kv.get("source_sha256") != kernel_source_hash():
            return None
        n0 = int(kv["spins"])
        return float(kv["dram_bytes_per_launch"]) * 2.0 ** (N - n0)
    except Exception:
        return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """Samples nvidia-smi clocks every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, v):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- CPU oracle baseline

def oracle_sample(nsteps=1):
    """Times the oracle on a bounded sample and scales it to the N=28 step.

    The oracle's U4 step is 40 global rotations (N 2^{N-1} pair updates each) and
    30 diagonal phases (2^N states x (N(N-1)/2 + N) terms each).  Both are timed at
    N=20 on the same dipolar chain; the N=28 step time is their sum scaled by the
    exact operation-count ratios.
    """
    import numpy as np
    import oracle
    from paper_1305_0036_gb300 import workloads as W
    n = 20
    s = W.dipolar_chain(n)
    H = oracle.Hamiltonian(n, s.Jx, s.Jy, s.Jz, hz=s.hz)
    psi = W.random_phase_state(n, 1)
    t0 = time.perf_counter()
    for _ in range(nsteps):
        psi = oracle.ts4(psi, H, TAU, 1)
    t_step20 = (time.perf_counter() - t0) / nsteps
    t0 = time.perf_counter()
    oracle.rotate_all(psi, n, oracle.X)
    t_rot = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.phase(psi, n, s.Jz, s.hz, TAU)
    t_ph = time.perf_counter() - t0
    N = 28
    rot_scale = (N * 2 ** (N - 1)) / (n * 2 ** (n - 1))
    ph_scale = (2 ** N * (N * (N - 1) / 2 + N)) / (2 ** n * (n * (n - 1) / 2 + n))
    model20 = 40 * t_rot + 30 * t_ph
    # the remainder of the measured N=20 step (scales, copies) scales like the rotations
    rest = max(t_step20 - model20, 0.0)
    t28 = 40 * t_rot * rot_scale + 30 * t_ph * ph_scale + rest * rot_scale
    return {"t_step_n20_s": t_step20, "t_step_n28_s": t28, "cores": oracle.num_threads(),
            "sample": f"{nsteps} oracle U4 step(s) of the N=20 dipolar chain ({t_step20:.2f} s/step) plus one "
                      "rotation layer and one phase at N=20, scaled to N=28 by the oracle's operation counts"}


def run_reference(args, ws, rank):
    if rank != 0:
        return
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        oracle_sample(1)
    t0 = time.perf_counter()
    t28 = []
    info = None
    for _ in range(args.steps):
        info = oracle_sample(1)
        t28.append(info["t_step_n28_s"])
    wall = time.perf_counter() - t0
    ms = 1000 * statistics.mean(t28)
    v = 1000.0 / ms
    line = {"metric": METRIC, "value": v, "unit": "TS4 steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "N": 28, "prec": "c128 (oracle, FP64 CPU)"},
            "cpu_baseline": {"value": v, "unit": "TS4 steps/s", "cores": info["cores"], "kind": "oracle",
                             "sample": info["sample"]},
            "e2e": {"value": v, "unit": "TS4 steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm

def run_ours(args, ws, rank, local):
    import numpy as np
    import torch
    from paper_1305_0036_gb300 import build
    build.build()
    from paper_1305_0036_gb300 import ts4, workloads as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    s = W.dipolar_chain(args.spins)
    N = s.N
    prec = args.prec
    npdt = np.complex64 if prec == "c64" else np.complex128
    amp = 8 if prec == "c64" else 16
    state_bytes = amp << N
    psi0 = W.random_phase_state(N, W.SEED_BASE + 3, npdt)
    host = torch.from_numpy(psi0).pin_memory()
    del psi0

    ctx = ts4.Context.from_system(s, prec=prec, device=dev)
    if args.tile:
        ctx.set_schedule(ts4.TS_KERNEL_FUSED, args.tile, args.cbits)
    sched = ctx.schedule()
    ctx.set_state_host_ptr(host.data_ptr())
    stream = ctx.stream
    for _ in range(args.warmup):
        ctx.step(TAU, 1)
    torch.cuda.synchronize(dev)

    # ---- device-timed region: K steps, state resident in HBM (2 GiB >> L2)
    clocks = Clocks(local)
    launches0 = ctx.launches()
    barrier(ws)
    torch.cuda.synchronize(dev)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # the job: K chained TS4 steps in one ts_step call (adjacent P_z slots of consecutive steps
    # merge, so a step costs 20 (g - 1) passes plus one final pass per call); the call builds
    # its K-step schedule inside the timed region, as a user's call would
    e0.record(stream)
    ctx.step(TAU, args.steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_total = e0.elapsed_time(e1)
    clk = clocks.stop()
    barrier(ws)
    launches = ctx.launches() - launches0
    ms_total = max_over_ranks(ws, ms_total)
    ms_step = ms_total / args.steps
    value = ws * args.steps / (ms_total / 1000.0)

    passes = sched["passes_per_step"]
    groups = sched["groups"]
    # roofline of the dominant kernel (the fused pass): algorithmic bytes per launch =
    # one read + one write of the state per rotation layer, a launch completing
    # 1/(g-1) of a layer; duration = timed region / pass launches
    pass_launches = 1 + args.steps * passes          # fused passes of the chained call
    avg_pass_ms = ms_total / max(pass_launches, 1)
    alg_bytes_launch = 2 * state_bytes / max(groups - 1, 1)
    achieved = alg_bytes_launch / (avg_pass_ms / 1000.0) / 1e9
    peak, peak_kind = peaks()
    eff_gbs = 40 * state_bytes / (ms_step / 1000.0) / 1e9
    dram_gbs = passes * 2 * state_bytes / (ms_step / 1000.0) / 1e9

    # ---- end to end through the public API with host buffers:
    # ts_set_state from pinned host memory, then every step ts_step + ts_observe(TS_NORM),
    # with the calls chained (ts_set_chaining: each call's final pass runs inside the next
    # call; the norm accounts for it exactly).  One untimed round first, like the warm-up of
    # the device-timed region.
    ctx.set_chaining(True)
    tw = time.perf_counter()
    ctx.set_state_host_ptr(host.data_ptr())
    warm_upload_ms = 1000.0 * (time.perf_counter() - tw)
    ctx.step(TAU, 1)
    ctx.norm()
    torch.cuda.synchronize(dev)
    barrier(ws)
    t0 = time.perf_counter()
    ctx.set_state_host_ptr(host.data_ptr())
    t_up = time.perf_counter()
    norm = 1.0
    for _ in range(args.steps):
        ctx.step(TAU, 1)
        norm = ctx.norm()
    t1 = time.perf_counter()
    e2e_s = max_over_ranks(ws, t1 - t0)
    e2e_value = ws * args.steps / e2e_s
    e2e_upload_ms = 1000.0 * (t_up - t0)
    e2e_step_ms = 1000.0 * (t1 - t_up) / args.steps

    line = {
        "metric": METRIC, "value": value, "unit": "TS4 steps/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": prec, "data": "synthetic",
        "config": {"workload": WORKLOAD if N == 28 else WORKLOAD.replace("N=28", f"N={N}"), "N": N, "prec": prec, "tile_bits": sched["tile_bits"],
                   "coalesce_bits": sched["coalesce_bits"], "groups": groups, "passes_per_step": passes,
                   "l2": f"state {state_bytes / 2**20:.0f} MiB vs 129 MB L2" +
                         (" (larger: no flush needed)" if state_bytes > 2 * 129e6 else " (NOT larger than L2)"),
                   "parallelism": f"replicas x{ws}",
                   "timed_call": f"one ts_step(tau, {args.steps}): {args.steps} chained TS4 steps"},
        "hbm": {"effective_gbs": eff_gbs, "effective_frac": eff_gbs / peak,
                "pass_traffic_gbs": dram_gbs, "pass_traffic_frac": dram_gbs / peak},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": measured_traffic(N) if prec == "c64" else None, "peak_kind": peak_kind,
                     "kernel": "k_tile", "alg_bytes_per_launch": alg_bytes_launch,
                     "avg_launch_ms": avg_pass_ms},
        "e2e": {"value": e2e_value, "unit": "TS4 steps/s", "h2d_bytes_per_step": state_bytes / args.steps,
                "d2h_bytes_per_step": 8, "final_norm": norm,
                "calls": "ts_set_state(host), then per step ts_step(tau, 1) + ts_observe(TS_NORM), chained",
                "upload_ms": e2e_upload_ms, "untimed_upload_ms": warm_upload_ms,
                "step_plus_norm_ms": e2e_step_ms},
        "gpu_launches": launches,
        "clocks": clk,
    }
    ctx.close()

    if args.compare_c128 and prec == "c64":
        c = ts4.Context.from_system(s, prec="c128", device=dev)
        c.set_state(np.asarray(host.numpy(), dtype=np.complex128))
        c.step(TAU, 1)
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k = 2
        a.record(c.stream)
        c.step(TAU, k)
        b.record(c.stream)
        torch.cuda.synchronize(dev)
        ms128 = a.elapsed_time(b) / k
        # complex128 is bound by the FP64 pipes, not by HBM: per amplitude and step the 20 layers
        # take N butterfly stages of 2 FP64 adds each, and the 21 slots 3 complex multiplies of
        # 4 FP64 instructions each (FMA counted once).  Peak: the nominal 1.25 TFLOP/s of FP64
        # = 0.625e12 FP64 FMA instructions/s.
        fp64_inst = float(2 ** N) * (20 * N * 2 + 21 * 12)
        fp64_rate = fp64_inst / (ms128 / 1000.0) / 1e12
        line["c128"] = {"value": 1000.0 / ms128, "unit": "TS4 steps/s", "ms_per_step": ms128,
                        "effective_gbs": 40 * (16 << N) / (ms128 / 1000.0) / 1e9,
                        "roofline": {"bound": "alu", "achieved": fp64_rate, "peak": 0.625,
                                     "unit": "T FP64 instructions/s", "frac": fp64_rate / 0.625,
                                     "peak_kind": "nominal FP64 rate (1.25 TFLOP/s)"}}
        c.close()

    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        info = oracle_sample(4)
        # the same sample on one core (one U4 step at N=20 instead of four)
        oracle.set_num_threads(1)
        one = oracle_sample(1)
        oracle.set_num_threads(info["cores"])
        line["cpu_baseline"] = {"value": 1.0 / info["t_step_n28_s"], "unit": "TS4 steps/s",
                                "cores": info["cores"], "kind": "oracle", "sample": info["sample"],
                                "single_thread": {"value": 1.0 / one["t_step_n28_s"], "cores": one["cores"],
                                                  "sample": one["sample"]}}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="c64", choices=["c64", "c128"])
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--cbits", type=int, default=0)
    ap.add_argument("--compare-c128", action="store_true", default=True)
    ap.add_argument("--no-compare-c128", dest="compare_c128", action="store_false")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--spins", type=int, default=28,
                    help="chain length N (28 is the benchmark; smaller N only for profiling captures)")
    args = ap.parse_args()
    ws, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
