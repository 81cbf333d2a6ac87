"""Batched ensemble (several systems of uneven N, many states each) against the
oracle and against single-state runs of the same library; the persistent ensemble
kernel's one launch per step and its bounded dependency waits."""
import numpy as np
import pytest

import oracle
from paper_1305_0036_gb300 import workloads as W

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24




def _ham(s):
    return oracle.Hamiltonian(s.N, s.Jx, s.Jy, s.Jz, hz=s.hz, hx=s.hx, hy=s.hy)


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_small_batch_matches_oracle(ts4, prec):
    systems = [W.xyz_chain(n, 1.0, 0.8, 0.5, seed=900 + n) for n in (12, 13, 15)]
    nst = [3, 2, 2]
    b = ts4.Batch(systems, nst, prec=prec)
    b.set_schedule(12, 2)
    init = []
    for i, (s, k) in enumerate(zip(systems, nst)):
        a = np.stack([W.haar_state(s.N, 1000 + 10 * i + j) for j in range(k)])
        init.append(a)
        b.set_states(i, a)
    nsteps, tau = 3, 0.05
    b.step(tau, nsteps)
    for i, (s, k) in enumerate(zip(systems, nst)):
        got = b.get_states(i).astype(np.complex128)
        for j in range(k):
            ref = oracle.ts4(init[i][j], _ham(s), tau, nsteps)
            if prec == "c128":
                assert np.abs(got[j] - ref).max() <= 1e-12
            else:
                assert np.linalg.norm(got[j] - ref) <= 20 * nsteps * (s.N + 8) * U32
    norms = b.norms()
    assert np.all(np.abs(norms - 1) <= (1e-12 if prec == "c128" else 1e-5))
    # a second call replays the cached graph: one persistent kernel launch per step call
    l0 = b.launches()
    b.step(tau, nsteps)
    b.status()
    assert b.launches() - l0 == 1
    b.close()


def test_ensemble_many_steps_uneven_passes_match_oracle(ts4):
    """Systems with 1, 2 and 3 bit groups (different numbers of passes per step: 20, 20, 40)
    over 12 steps, so that the per-state counters order thousands of dependent tiles."""
    systems = [W.xyz_chain(12, 1.0, 0.8, 0.5, seed=41), W.random_system(16, 42, transverse=False),
               W.xyz_chain(21, 1.0, 0.8, 0.5, seed=43)]
    nst = [5, 3, 1]
    b = ts4.Batch(systems, nst, prec="c128")
    b.set_schedule(12, 4)
    init = []
    for i, (s, k) in enumerate(zip(systems, nst)):
        a = np.stack([W.haar_state(s.N, 2000 + 10 * i + j) for j in range(k)])
        init.append(a)
        b.set_states(i, a)
    nsteps, tau = 12, 0.04
    b.step(tau, nsteps)
    for i, (s, k) in enumerate(zip(systems, nst)):
        got = b.get_states(i)
        for j in sorted({0, k - 1}):
            ref = oracle.ts4(init[i][j], _ham(s), tau, nsteps)
            assert np.abs(got[j] - ref).max() <= 1e-12, (i, j)
    b.close()


def test_ensemble_wait_timeout_is_reported_and_recoverable(ts4):
    """Every dependency wait made to run out (a device flag that nothing sets): the launch
    ends by itself, the timeout is reported once, and the batch works again afterwards."""
    systems = [W.xyz_chain(12, 1.0, 0.8, 0.5, seed=51), W.xyz_chain(14, 1.0, 0.8, 0.5, seed=52)]
    nst = [2, 2]
    b = ts4.Batch(systems, nst, prec="c64")
    b.set_schedule(12, 2)
    init = [np.stack([W.haar_state(s.N, 3000 + 10 * i + j, np.complex64) for j in range(k)])
            for i, (s, k) in enumerate(zip(systems, nst))]
    for i in range(2):
        b.set_states(i, init[i])
    b.set_wait(0.05, hold=True)
    b.step(0.05, 2)
    with pytest.raises(ts4.TS4Error) as e:
        b.status()
    assert e.value.status == ts4.TS_ERR_TIMEOUT
    b.status()                      # reported once
    b.set_wait(2.0, hold=False)
    for i in range(2):
        b.set_states(i, init[i])
    b.step(0.05, 2)
    for i, (s, k) in enumerate(zip(systems, nst)):
        got = b.get_states(i).astype(np.complex128)
        for j in range(k):
            ref = oracle.ts4(init[i][j].astype(np.complex128), _ham(s), 0.05, 2)
            assert np.linalg.norm(got[j] - ref) <= 40 * (s.N + 8) * U32
    with pytest.raises(ts4.TS4Error) as e:
        b.set_wait(0.0)
    assert e.value.status == ts4.TS_ERR_ARG
    b.close()


def test_config4_ensemble_against_single_state_runs(ts4):
    """256 Haar states (64 each at N = 16, 18, 20, 22), XYZ chains, tau = 0.02, 200 steps,
    complex64, one graph launch; sampled states checked against single-state runs."""
    cfg = W.config(3)
    systems, k = cfg["systems"], cfg["states_per_system"]
    b = ts4.Batch(systems, [k] * len(systems), prec="c64")
    init = []
    for i, s in enumerate(systems):
        a = np.stack([W.haar_state(s.N, cfg["state_seed"] * 1000 + 100 * i + j, np.complex64) for j in range(k)])
        init.append(a)
        b.set_states(i, a)
    b.step(cfg["tau"], cfg["nsteps"])
    norms = b.norms()
    assert np.all(np.abs(norms - 1) <= 1e-4), np.abs(norms - 1).max()
    szs = b.sz()
    # the two smallest systems' first states against the FP64 oracle after the whole run
    for i in (0, 1):
        s = systems[i]
        got = b.get_states(i)[0].astype(np.complex128)
        ref = oracle.ts4(init[i][0].astype(np.complex128), _ham(s), cfg["tau"], cfg["nsteps"])
        L = 20 * cfg["nsteps"] + 1
        assert np.linalg.norm(got - ref) <= L * (s.N + 8) * U32
        assert np.abs(got - ref).max() <= np.sqrt(2 * np.log(2.0 ** (s.N + 1))) * L * (s.N + 8) * U32 * np.abs(ref).max()
        np.testing.assert_allclose(szs[i][0], oracle.sz(ref, s.N), atol=2 * L * (s.N + 8) * U32)
    for i, s in enumerate(systems):
        got = b.get_states(i)
        for j in (0, k - 1):
            c = ts4.Context.from_system(s, prec="c64")
            c.set_state(init[i][j])
            c.step(cfg["tau"], cfg["nsteps"])
            single = c.get_state()
            np.testing.assert_allclose(c.sz(), szs[i][j], atol=1e-6)
            c.close()
            # Same formula in both runs, but the batched and the single-state kernels are
            # compiled separately and the compiler may fuse a multiply and an add in one and
            # not in the other.  Those roundings (<= 2^-24 relative, unbiased) add up like a
            # random walk over the ~20 (N + 8) rounded operations per amplitude and step.
            tol = 4.0 * np.sqrt(20 * cfg["nsteps"] * (s.N + 8)) * U32
            assert np.linalg.norm(got[j].astype(np.complex128) - single) <= tol
    b.close()
