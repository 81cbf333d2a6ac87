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

# The oracle's U4 step (Sec. 2: U4 = five U2's, each U2 = U1(t/2) then U1^dag(-t/2), each U1 three
# parts; a z part is one Z-like phase, an x or y part is a global rotation, a phase, the inverse
# rotation and an exact 2^-N scale) is, operation by operation:
ORACLE_U4_PHASES, ORACLE_U4_ROTATIONS, ORACLE_U4_SCALES = 30, 40, 20


class OracleSample:
    """Times the FP64 CPU oracle, as it stands, on the benchmark's own N=28 state, in place.

    The three kinds of operation of its U4 step are timed at full size: a Z-like phase
    (O(N^2) bond terms per amplitude), a global rotation (N spins x 2^(N-1) pair updates) and
    the exact 2^-N scale.  The U4 step time is 30 phases + 40 rotations + 20 scales, the exact
    operation count of the oracle's U4.
    """

    def __init__(self, N=28):
        import numpy as np
        import oracle
        from paper_1305_0036_gb300 import workloads as W
        self.np, self.oracle, self.N = np, oracle, N
        self.lib = oracle.lib()
        s = W.dipolar_chain(N)
        self.J = np.ascontiguousarray(s.Jz)
        self.h = np.ascontiguousarray(s.hz)
        self.psi = W.random_phase_state(N, W.SEED_BASE + 3)   # complex128, 2^N amplitudes
        self.cores = oracle.num_threads()

    def phase(self):
        t0 = time.perf_counter()
        self.lib.oracle_phase(self.psi.ctypes.data, self.N, self.J.ctypes.data, self.h.ctypes.data, TAU)
        return time.perf_counter() - t0

    def rotation_and_scale(self):
        t0 = time.perf_counter()
        self.lib.oracle_rotate_all(self.psi.ctypes.data, self.N, self.oracle.X)
        t1 = time.perf_counter()
        self.lib.oracle_scale(self.psi.ctypes.data, self.N, 2.0 ** (-self.N / 2))
        return t1 - t0, time.perf_counter() - t1

    @staticmethod
    def u4_seconds(t_phase, t_rot, t_scale):
        return ORACLE_U4_PHASES * t_phase + ORACLE_U4_ROTATIONS * t_rot + ORACLE_U4_SCALES * t_scale

    def u1_measured(self):
        """One real oracle U1 on the same state (for checking the composition: U1 = 3 phases +
        4 rotations + 2 scales)."""
        import oracle
        from paper_1305_0036_gb300 import workloads as W
        s = W.dipolar_chain(self.N)
        H = oracle.Hamiltonian(self.N, s.Jx, s.Jy, s.Jz, hz=s.hz)
        t0 = time.perf_counter()
        self.lib.oracle_apply(self.psi.ctypes.data, self.N, *H.args(), 1, TAU)
        return time.perf_counter() - t0


SAMPLE_TEXT = ("the FP64 oracle at N=28 on the benchmark's own dipolar chain and state (complex128, 4 GiB, "
               "in place): {what}; TS4 step = 30 Z-like phases + 40 global rotations + 20 exact scales "
               "(the operation count of the oracle's U4)")


def run_reference(args, ws, rank):
    if rank != 0:
        return
    import oracle
    oracle.build()
    smp = OracleSample(28)
    # the phase (about a minute of one core's work per 2^24 amplitudes) is timed once, in the
    # first warm-up step; every step times a global rotation and a scale
    t_phase = smp.phase()
    for _ in range(args.warmup):
        smp.rotation_and_scale()
    rots, scs, walls = [], [], []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        w0 = time.perf_counter()
        r, c = smp.rotation_and_scale()
        walls.append(time.perf_counter() - w0)
        rots.append(r)
        scs.append(c)
    wall = time.perf_counter() - t0
    t_u4 = OracleSample.u4_seconds(t_phase, statistics.mean(rots), statistics.mean(scs))
    v = 1.0 / t_u4
    sample = SAMPLE_TEXT.format(what=f"each step times one global rotation and one scale "
                                     f"({1000 * statistics.mean(rots):.0f} + {1000 * statistics.mean(scs):.0f} ms), "
                                     f"the phase was timed once before them ({t_phase:.2f} s)")
    line = {"metric": METRIC, "value": v, "unit": "TS4 steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * statistics.mean(walls), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "N": 28, "prec": "c128 (oracle, FP64 CPU)"},
            "ms_per_step_is": "wall time of one timed sample (one global rotation + one scale at N=28)",
            "ts4_step_s": t_u4,
            "parts_s": {"phase": t_phase, "rotation": statistics.mean(rots), "scale": statistics.mean(scs)},
            "cpu_baseline": {"value": v, "unit": "TS4 steps/s", "cores": smp.cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "TS4 steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm

def accuracy_vs_c128(ts4, torch, ctx64, ctx128):
    """complex64 against complex128 after the same steps from the same state (Sec. 4.2's
    accuracy figures): state difference, norm drift, largest S^z difference."""
    a = ctx64.psi.to(torch.complex128)
    d = a - ctx128.psi
    l2 = float(torch.linalg.vector_norm(d).item())
    mx = float(d.abs().max().item())
    del a, d
    n64, n128 = ctx64.norm(), ctx128.norm()
    dsz = float(abs(ctx64.sz() - ctx128.sz()).max())
    return {"l2": l2, "max_abs": mx, "norm_drift_c64": abs(n64 - 1.0), "norm_drift_c128": abs(n128 - 1.0),
            "max_abs_dSz": dsz}


def oracle_cross_check(ts4):
    """The benchmark's schedules against the FP64 oracle where it runs in seconds: the N=23
    dipolar chain with the tile shapes of both arms (12-bit tiles; 3 coalescing spins for
    complex64, 2 for complex128), which give 3 bit groups and the slot-less middle pass as at
    N=28; 2 TS4 steps of tau = 0.01 from the random-phase state."""
    import numpy as np
    import oracle
    from paper_1305_0036_gb300 import workloads as W
    N, n = 23, 2
    s = W.dipolar_chain(N)
    psi0 = W.random_phase_state(N, W.SEED_BASE + 3)
    ref = oracle.ts4(psi0, oracle.Hamiltonian(N, s.Jx, s.Jy, s.Jz, hz=s.hz), TAU, n)
    out = {"N": N, "steps": n, "workload": "dipolar XXZ chain, random-phase state"}
    for prec, tile, cb in (("c64", 12, 3), ("c128", 12, 2)):
        c = ts4.Context.from_system(s, prec=prec)
        c.set_schedule(ts4.TS_KERNEL_FUSED, tile, cb)
        c.set_state(psi0)
        c.step(TAU, n)
        sch = c.schedule()
        d = c.get_state().astype(np.complex128) - ref
        c.close()
        out[prec] = {"max_abs": float(np.abs(d).max()), "l2": float(np.linalg.norm(d)),
                     "tile_bits": sch["tile_bits"], "coalesce_bits": sch["coalesce_bits"], "groups": sch["groups"]}
    return out


def config4_ensemble(ts4, torch, dev, steps):
    """Config 4: 256 Haar states, 64 each at N = 16, 18, 20, 22 (XYZ chains 1.0/0.8/0.5, fields
    uniform in [-1, 1]), tau = 0.02, complex64, autotuned tile; ms per ensemble step over one
    ts_batch_step(tau, steps) graph launch."""
    from paper_1305_0036_gb300 import workloads as W
    cfg = W.config(3)
    systems, k = cfg["systems"], cfg["states_per_system"]
    b = ts4.Batch(systems, [k] * len(systems), prec="c64", device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(cfg["state_seed"])
    for i, s in enumerate(systems):
        z = torch.randn((k, 1 << s.N), dtype=torch.complex64, device=dev, generator=g)
        z /= torch.linalg.vector_norm(z, dim=1, keepdim=True)
        b.set_states(i, z)
        del z
    tune_ms = b.autotune(cfg["tau"], reps=2)
    sch = b.schedule()
    b.step(cfg["tau"], 2)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    b.step(cfg["tau"], steps)
    e1.record(b.stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    norms = b.norms()
    amps = sum(k << s.N for s in systems)
    out = {"workload": "256 Haar states, 64 each at N=16/18/20/22, XYZ chains (1.0, 0.8, 0.5), h~U[-1,1], "
                       "tau=0.02, complex64", "ms_per_ensemble_step": ms, "steps_timed": steps,
           "timed_call": f"one ts_batch_step(tau, {steps}) (one CUDA graph launch)",
           "effective_gbs": 40 * 8 * amps / (ms / 1000.0) / 1e9, "tile_bits": sch["tile_bits"],
           "coalesce_bits": sch["coalesce_bits"], "autotune_best_ms": tune_ms,
           "max_norm_drift": float(abs(norms - 1.0).max())}
    b.close()
    return out


def config2_ladder(ts4, torch, dev):
    """Config 2: the 2x12 ladder (J^a_ij i.i.d. U[-1, 1], h i.i.d. U[-1/2, 1/2]), Neel state,
    tau = 0.02, 1000 steps: complex64 timed over one ts_step(tau, 1000) call, against the same
    run in complex128 (S^z and norm drift; targets 1e-5)."""
    from paper_1305_0036_gb300 import workloads as W
    cfg = W.config(1)
    s = cfg["system"]
    out = {"workload": "N=24 two-leg ladder 2x12, J^a~U[-1,1], h~U[-0.5,0.5], Neel state, tau=0.02, "
                       "1000 steps, complex64 vs complex128", "steps": cfg["nsteps"]}
    res = {}
    for prec in ("c64", "c128"):
        c = ts4.Context.from_system(s, prec=prec, device=dev)
        c.set_basis_state(cfg["state"][1])
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(c.stream)
        c.step(cfg["tau"], cfg["nsteps"])
        e1.record(c.stream)
        torch.cuda.synchronize(dev)
        res[prec] = (e0.elapsed_time(e1) / cfg["nsteps"], c.norm(), c.sz())
        c.close()
    out["ms_per_step_c64"] = res["c64"][0]
    out["ms_per_step_c128"] = res["c128"][0]
    out["norm_drift_c64"] = abs(res["c64"][1] - 1.0)
    out["norm_drift_c128"] = abs(res["c128"][1] - 1.0)
    out["max_abs_dSz"] = float(abs(res["c64"][2] - res["c128"][2]).max())
    out["targets"] = {"max_abs_dSz": 1e-5, "norm_drift_c64": 1e-5}
    return out


def config5_capacity(ts4, torch, dev, steps):
    """Config 5: N=33 XYZ chain (1.0, 0.8, 0.5), h=0.1, Neel state, tau=0.02, complex64 (64 GiB
    state in place); ms per TS4 step over one ts_step(tau, steps) call."""
    from paper_1305_0036_gb300 import workloads as W
    cfg = W.config(4)
    s = cfg["system"]
    N = s.N
    ctx = ts4.Context.from_system(s, prec="c64", device=dev)
    ctx.set_basis_state(cfg["state"][1])
    ctx.step(cfg["tau"], 1)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    ctx.step(cfg["tau"], steps)
    e1.record(ctx.stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    sch = ctx.schedule()
    norm = ctx.norm()
    state_bytes = 8 << N
    out = {"workload": "N=33 open XYZ chain (1.0, 0.8, 0.5), h=0.1, Neel state, tau=0.02, complex64",
           "ms_per_step": ms, "steps_timed": steps, "state_gib": state_bytes / 2 ** 30,
           "groups": sch["groups"], "passes_per_step": sch["passes_per_step"],
           "effective_gbs": 40 * state_bytes / (ms / 1000.0) / 1e9,
           "pass_traffic_gbs": sch["passes_per_step"] * 2 * state_bytes / (ms / 1000.0) / 1e9,
           "norm_drift": abs(norm - 1.0)}
    ctx.close()
    return out


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
    ctx.flush()          # the state after K steps from psi_0, for the accuracy figures below

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

    if args.compare_c128 and prec == "c64":
        # the complex128 arm: the same K steps from the same state (the complex64 initial state
        # converted exactly), one ts_step(tau, K) call timed with events
        c = ts4.Context.from_system(s, prec="c128", device=dev)
        c.set_state(np.asarray(host.numpy(), dtype=np.complex128))
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(c.stream)
        c.step(TAU, args.steps)
        b.record(c.stream)
        torch.cuda.synchronize(dev)
        ms128 = a.elapsed_time(b) / args.steps
        # complex128 is bound by the FP64 pipes, not by HBM: per amplitude and step the 20 layers
        # take N butterfly stages of 2 FP64 adds each, and the 21 slots 3 complex multiplies of
        # 4 FP64 instructions each (FMA counted once).  Peak: the nominal 1.25 TFLOP/s of FP64
        # = 0.625e12 FP64 FMA instructions/s.
        fp64_inst = float(2 ** N) * (20 * N * 2 + 21 * 12)
        fp64_rate = fp64_inst / (ms128 / 1000.0) / 1e12
        line["c128"] = {"value": 1000.0 / ms128, "unit": "TS4 steps/s", "ms_per_step": ms128,
                        "steps_timed": args.steps, "speedup_of_c64": (1000.0 / ms_step) / (1000.0 / ms128),
                        "effective_gbs": 40 * (16 << N) / (ms128 / 1000.0) / 1e9,
                        "roofline": {"bound": "alu", "achieved": fp64_rate, "peak": 0.625,
                                     "unit": "T FP64 instructions/s", "frac": fp64_rate / 0.625,
                                     "peak_kind": "nominal FP64 rate (1.25 TFLOP/s)"}}
        # accuracy of the benchmarked complex64 run (its end-to-end leg: K chained one-step calls
        # from psi_0) against the complex128 run; targets 1e-5 for S^z and the norm drift
        err = accuracy_vs_c128(ts4, torch, ctx, c)
        err.update({"vs": f"complex128 GPU run (parity with the FP64 oracle: 1e-12), same state, same {args.steps} steps",
                    "steps": args.steps, "targets": {"max_abs_dSz": 1e-5, "norm_drift_c64": 1e-5}})
        line["err"] = err
        c.close()
    ctx.close()
    del host
    torch.cuda.empty_cache()

    if rank == 0 and ws == 1 and not args.no_oracle_check:
        line["err_vs_oracle"] = oracle_cross_check(ts4)
    if not args.no_configs and N == 28:
        line["config2"] = config2_ladder(ts4, torch, dev)
        torch.cuda.empty_cache()
        line["config4"] = config4_ensemble(ts4, torch, dev, 20)
        torch.cuda.empty_cache()
        line["config5"] = config5_capacity(ts4, torch, dev, 2)
        torch.cuda.empty_cache()

    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        smp = OracleSample(28)
        t_ph = smp.phase()
        t_rot, t_sc = smp.rotation_and_scale()
        t_u4 = OracleSample.u4_seconds(t_ph, t_rot, t_sc)
        line["cpu_baseline"] = {"value": 1.0 / t_u4, "unit": "TS4 steps/s", "cores": smp.cores, "kind": "oracle",
                                "sample": SAMPLE_TEXT.format(what=f"one phase ({t_ph:.2f} s), one global rotation "
                                                                  f"({t_rot:.2f} s) and one scale ({t_sc:.3f} s) timed"),
                                "ts4_step_s": t_u4}
        if args.validate_cpu_model:
            t_u1 = smp.u1_measured()
            model = 3 * t_ph + 4 * t_rot + 2 * t_sc
            line["cpu_baseline"]["u1_check"] = {"measured_s": t_u1, "composed_s": model,
                                                "residual": t_u1 / model - 1.0}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_phase_table_ab(args):
    """The paper's phase-table mode (Sec. 3.1) against bit tests and the fused pass: ms per TS4
    step of the dipolar chain at each N in --ab-sizes, for both precisions (one JSON line)."""
    import torch
    from paper_1305_0036_gb300 import build
    build.build()
    from paper_1305_0036_gb300 import ts4, workloads as W
    torch.cuda.set_device(0)
    rows = []
    for N in args.ab_sizes:
        s = W.dipolar_chain(N)
        for prec in ("c64", "c128"):
            row = {"N": N, "prec": prec}
            for mode in ("fused", "basic_bits", "basic_tables"):
                ctx = ts4.Context.from_system(s, prec=prec)
                if mode != "fused":
                    ctx.set_schedule(ts4.TS_KERNEL_BASIC, 0, 0)
                if mode == "basic_tables":
                    ctx.set_phase_tables(True)
                ctx.set_basis_state(W.neel_index(N))
                ctx.step(TAU, 1)
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                n = args.ab_steps
                a.record(ctx.stream)
                ctx.step(TAU, n)
                b.record(ctx.stream)
                torch.cuda.synchronize()
                row[mode + "_ms"] = a.elapsed_time(b) / n
                ctx.close()
                torch.cuda.empty_cache()
            rows.append(row)
    print(json.dumps({"phase_table_ab": rows, "workload": "dipolar XXZ chain, Neel state, tau=0.01",
                      "tables": "complex64: 3 x 2^N floats; complex128: 3 x 2^N doubles"}), flush=True)


def run_pass_times(args):
    """Time per amplitude and pass with the state in L2 (N <= 23: at most 64 MB) and in HBM (N >= 25),
    complex64 dipolar chain, default schedule: the whole step with CUDA events, and each kind of
    k_tile launch from CUPTI activity records (torch.profiler; kernels back to back on one stream,
    no cache flush between them).  Kinds: slot passes and passes without a slot of compiled
    shapes, and the builds that follow the step list at run time (first and last pass of a call).
    One JSON line."""
    import numpy as np
    import torch
    from torch.profiler import ProfilerActivity, profile
    from paper_1305_0036_gb300 import build
    build.build()
    from paper_1305_0036_gb300 import ts4, workloads as W
    torch.cuda.set_device(0)
    # the first profiling session of a process can come back without kernel records: open one
    # on a throwaway launch first
    with profile(activities=[ProfilerActivity.CUDA]):
        torch.ones(1024, device="cuda").mul_(2.0)
        torch.cuda.synchronize()
    rows = []
    for N in args.pt_sizes:
        ctx = ts4.Context.from_system(W.dipolar_chain(N), prec="c64")
        ctx.set_state(W.random_phase_state(N, W.SEED_BASE + 3, np.complex64))
        sch = ctx.schedule()
        ctx.step(TAU, 2)
        torch.cuda.synchronize()
        n = 40 if N < 26 else 10
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(ctx.stream)
        ctx.step(TAU, n)
        b.record(ctx.stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / n
        row = {"N": N, "state_mb": 2 ** N * 8 / 1e6, "groups": sch["groups"],
               "passes_per_step": sch["passes_per_step"], "ms_per_step": ms,
               "ps_per_amp_pass": ms * 1e9 / 2 ** N / sch["passes_per_step"]}
        with profile(activities=[ProfilerActivity.CUDA]) as prof:
            ctx.step(TAU, 4)
            torch.cuda.synchronize()
        kinds = {}
        for ev in prof.events():
            if ev.device_type != torch.autograd.DeviceType.CUDA or "k_tile<" not in ev.name:
                continue
            if "PassShape" not in ev.name:
                kind = "run-time build"
            elif "k_tile<float, 12, 5, true" in ev.name:
                kind = "slot pass"
            else:
                kind = "pass without slot"
            t = ev.device_time if hasattr(ev, "device_time") else ev.cuda_time
            k = kinds.setdefault(kind, [0, 0.0])
            k[0] += 1
            k[1] += t
        row["kernels"] = {k: {"launches": v[0], "mean_us": v[1] / v[0], "ps_per_amp": v[1] / v[0] * 1e6 / 2 ** N}
                          for k, v in sorted(kinds.items())}
        rows.append(row)
        ctx.close()
        torch.cuda.empty_cache()
    print(json.dumps({"pass_times": rows, "workload": "dipolar XXZ chain, random-phase state, tau=0.01, complex64",
                      "l2_mb": 129}), flush=True)


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
    ap.add_argument("--no-oracle-check", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the config-4 and config-5 lines")
    ap.add_argument("--validate-cpu-model", action="store_true",
                    help="also time one real oracle U1 at N=28 against its composition from the parts")
    ap.add_argument("--phase-table-ab", action="store_true",
                    help="time the paper's phase-table mode against bit tests and the fused pass instead")
    ap.add_argument("--ab-sizes", type=int, nargs="+", default=[22, 26, 28])
    ap.add_argument("--ab-steps", type=int, default=1)
    ap.add_argument("--pass-times", action="store_true",
                    help="time each kind of pass per amplitude at the sizes in --pt-sizes instead")
    ap.add_argument("--pt-sizes", type=int, nargs="+", default=[22, 23, 24, 25, 26, 28])
    ap.add_argument("--spins", type=int, default=28,
                    help="chain length N (28 is the benchmark; smaller N only for profiling captures)")
    args = ap.parse_args()
    ws, rank, local = dist_init()
    if args.phase_table_ab:
        run_phase_table_ab(args)
        return
    if args.pass_times:
        run_pass_times(args)
        return
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
