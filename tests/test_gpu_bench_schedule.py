"""Oracle parity for the exact schedules the benchmark times (Secs. 3.3-3.4 tiling on top of
the Sec. 2 decomposition), checked amplitude by amplitude.

The benchmark runs complex64 with 12-bit tiles and 3 coalescing spins, and complex128 with
12-bit tiles and 2 coalescing spins.  At N=28 both give three bit groups: the 12 low spins,
visited in the middle of the zigzag by a pass without a slot (the kernel build without the
slot code), and two window groups whose passes apply the slots and rotate their group twice.
The same kernel instances and the same zigzag appear at N=22 and N=23 with the same tile
shapes, where the FP64 oracle finishes in seconds: N=22 has two 5-spin windows (one register
chunk each), N=23 a 6-spin window (two chunks) and a 5-spin one.  N=27 has the window geometry
of N=28 itself (an 8-spin window that keeps the 4 lowest spins, 128-byte runs, and a 7-spin
one); there the oracle runs two steps.

Tolerances
  complex128: max_s |dpsi_s| <= 1e-12 (the bound stated for the FP64 path).
  complex64, whole vector: ||dpsi||_2 <= L (N + 8) u, u = 2^-24, L = rotation layers: every
    layer sends each amplitude through N rounded butterflies and at most about 8 rounded
    slot multiplications, each a relative error of at most u; worst-case linear sum over the
    layers for a unit-norm state.
  complex64, per amplitude: max_s |dpsi_s| <= c L (N + 8) u max_s |psi_s|, c = sqrt(2 ln 2^(N+1)).
    The rounding errors of one layer have, per amplitude, at most (N + 8) u times the size of
    the values being rounded, i.e. an RMS of at most (N + 8) u RMS(psi) <= (N + 8) u max|psi|
    (the passes are unitary up to exact powers of two, so the intermediate vectors of these
    random states have the same size distribution as the state).  Later layers spread each
    layer's errors into a random-like vector, whose largest entry exceeds its RMS by at most
    the Gaussian tail factor c of 2^N samples; the layers add at most linearly.  A single
    amplitude (or a tile) that is wrong by a few parts in 1e4 of the largest amplitude fails
    this check even where the L2 bound would let it through.

The observed errors are printed (run with -s to see them) next to their bounds.
"""
import functools

import numpy as np
import pytest

import oracle
from paper_1305_0036_gb300 import workloads as W

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
NSTEPS = 20


def _ham(s):
    return oracle.Hamiltonian(s.N, s.Jx, s.Jy, s.Jz, hz=s.hz, hx=s.hx, hy=s.hy)


def _system(kind, N):
    if kind == "random":
        return W.random_system(N, 900 + N, transverse=True), W.haar_state(N, 950 + N), 0.05
    return W.dipolar_chain(N), W.random_phase_state(N, W.SEED_BASE + 3), 0.01


@functools.lru_cache(maxsize=None)
def _oracle_run(kind, N, nsteps=NSTEPS, c64_start=False):
    s, psi0, tau = _system(kind, N)
    if c64_start:      # the initial state as complex64 holds it (what the complex64 runs start from)
        psi0 = psi0.astype(np.complex64).astype(np.complex128)
    return oracle.ts4(psi0, _ham(s), tau, nsteps)


def _bounds_c64(N, layers, ref):
    l2 = layers * (N + 8) * U32
    tail = np.sqrt(2.0 * np.log(2.0 ** (N + 1)))
    return l2, tail * l2 * np.abs(ref).max()


def _run(ts4, s, psi0, tau, prec, tile, cbits, chained, nsteps=NSTEPS):
    ctx = ts4.Context.from_system(s, prec=prec)
    ctx.set_schedule(ts4.TS_KERNEL_FUSED, tile, cbits)
    sched = ctx.schedule()
    ctx.set_state(psi0)
    if chained:
        # one-step calls: each call's final pass runs inside the next call; the norm read
        # after each call accounts for the held-back pass without running it
        ctx.set_chaining(True)
        for _ in range(nsteps):
            ctx.step(tau, 1)
            assert abs(ctx.norm() - 1.0) <= 1e-4
    else:
        ctx.step(tau, nsteps)
    got = ctx.get_state().astype(np.complex128)
    ctx.close()
    return got, sched


def _check_plan(ts4, N, prec, tile, cbits, nsteps=NSTEPS):
    """The plan has three bit groups and middle passes without a slot (the no-slot kernel)."""
    groups, passes = ts4.ts_plan(N, ts4.TS_C64 if prec == "c64" else ts4.TS_C128, tile, cbits, 4, nsteps)
    assert len(groups) == 3
    assert groups[0] == dict(c=0, w=0, h=12)
    middle = [p for p in passes if p["slot"] < 0]
    assert middle and all(p["group"] == 0 for p in middle)
    assert len(passes) == 1 + 20 * nsteps * 2
    return groups


@pytest.mark.parametrize("kind,N", [("random", 22), ("random", 23), ("dipolar", 22)])
@pytest.mark.parametrize("chained", [False, True])
def test_bench_schedule_c64_matches_oracle(ts4, kind, N, chained):
    s, psi0, tau = _system(kind, N)
    ref = _oracle_run(kind, N)
    _check_plan(ts4, N, "c64", 12, 3)
    got, sched = _run(ts4, s, psi0.astype(np.complex64), tau, "c64", 12, 3, chained)
    assert (sched["tile_bits"], sched["coalesce_bits"], sched["groups"]) == (12, 3, 3)
    l2_bound, el_bound = _bounds_c64(N, 20 * NSTEPS + 1, ref)
    # the initial state is rounded to complex64 before the run: that rounding is part of dpsi
    err = got - ref
    l2, el = np.linalg.norm(err), np.abs(err).max()
    print(f"\nc64 {kind} N={N} chained={chained}: ||dpsi||_2 = {l2:.3e} (bound {l2_bound:.3e}), "
          f"max|dpsi| = {el:.3e} (bound {el_bound:.3e}, max|psi| = {np.abs(ref).max():.3e})")
    assert l2 <= l2_bound, l2
    assert el <= el_bound, el


@pytest.mark.parametrize("chained", [False, True])
def test_bench_schedule_c128_matches_oracle(ts4, chained):
    """The complex128 arm's default schedule (12-bit tiles, 2 coalescing spins, 3 groups)."""
    N = 23
    s, psi0, tau = _system("random", N)
    ref = _oracle_run("random", N)
    _check_plan(ts4, N, "c128", 0, 0)
    got, sched = _run(ts4, s, psi0, tau, "c128", 0, 0, chained)
    assert (sched["tile_bits"], sched["coalesce_bits"], sched["groups"]) == (12, 2, 3)
    el = np.abs(got - ref).max()
    print(f"\nc128 random N={N} chained={chained}: max|dpsi| = {el:.3e} (bound 1e-12)")
    assert el <= 1e-12, el


def test_bench_window_geometry_n27_c64_matches_oracle(ts4):
    """N=27 dipolar chain with the benchmark's complex64 schedule: its first window group is
    that of N=28 (8 spins plus the 4 lowest, 128-byte runs); two steps against the oracle."""
    N, n = 27, 2
    s, psi0, tau = _system("dipolar", N)
    groups = _check_plan(ts4, N, "c64", 12, 3, n)
    assert groups[1] == dict(c=4, w=12, h=8) and groups[2] == dict(c=5, w=20, h=7)
    ref = _oracle_run("dipolar", N, n, c64_start=True)
    got, sched = _run(ts4, s, psi0.astype(np.complex64), tau, "c64", 12, 3, False, n)
    assert (sched["tile_bits"], sched["coalesce_bits"], sched["groups"]) == (12, 3, 3)
    l2_bound, el_bound = _bounds_c64(N, 20 * n + 1, ref)
    err = got - ref
    l2, el = np.linalg.norm(err), np.abs(err).max()
    print(f"\nc64 dipolar N={N}: ||dpsi||_2 = {l2:.3e} (bound {l2_bound:.3e}), "
          f"max|dpsi| = {el:.3e} (bound {el_bound:.3e})")
    assert l2 <= l2_bound, l2
    assert el <= el_bound, el
    # complex128 with its default schedule (2 coalescing spins: windows of 8 and 7 spins)
    got128, sched = _run(ts4, s, psi0.astype(np.complex64).astype(np.complex128), tau, "c128", 0, 0, False, n)
    assert (sched["tile_bits"], sched["coalesce_bits"], sched["groups"]) == (12, 2, 3)
    el128 = np.abs(got128 - _oracle_run("dipolar", N, n, c64_start=True)).max()
    print(f"c128 dipolar N={N}: max|dpsi| = {el128:.3e} (bound 1e-12)")
    assert el128 <= 1e-12, el128


def test_bench_instance_n28_one_step_matches_oracle(ts4):
    """The benchmark's own instance at full size: N=28 dipolar chain, Eq. A.1 state, tau = 0.01,
    the default complex64 schedule (12-bit tiles, 3 coalescing spins, windows of 8 spins plus
    the 4 lowest), one TS4 step (41 passes: every pass kind of the timed run) against one FP64
    oracle step (about three minutes on 16 cores, 8 GiB of host memory)."""
    N = 28
    s = W.dipolar_chain(N)
    psi0 = W.random_phase_state(N, W.SEED_BASE + 3, np.complex64)
    groups = _check_plan(ts4, N, "c64", 0, 0, 1)
    assert groups[1] == dict(c=4, w=12, h=8) and groups[2] == dict(c=4, w=20, h=8)
    ctx = ts4.Context.from_system(s, prec="c64")
    ctx.set_state(psi0)
    ctx.step(0.01, 1)
    got = ctx.get_state()
    ctx.close()
    ref = oracle.ts4(psi0.astype(np.complex128), _ham(s), 0.01, 1)
    l2_bound, el_bound = _bounds_c64(N, 21, ref)
    err = got.astype(np.complex128)
    err -= ref
    l2, el = np.linalg.norm(err), np.abs(err).max()
    print(f"\nc64 dipolar N=28 (bench instance), 1 step: ||dpsi||_2 = {l2:.3e} (bound {l2_bound:.3e}), "
          f"max|dpsi| = {el:.3e} (bound {el_bound:.3e})")
    assert l2 <= l2_bound, l2
    assert el <= el_bound, el
