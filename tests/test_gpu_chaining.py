"""Chained step calls (ts_set_chaining): the final pass of each call is held back and run
inside the next call's first pass (Sec. 2: adjacent P_z halves merge), and every other use of
the state runs it first.  Checked against the FP64 oracle and against unchained runs."""
import numpy as np
import pytest

import oracle
from paper_1305_0036_gb300 import workloads as W

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


def _ham(s):
    return oracle.Hamiltonian(s.N, s.Jx, s.Jy, s.Jz, hz=s.hz, hx=s.hx, hy=s.hy)


def test_one_step_calls_with_norm_reads_match_the_oracle_c128(ts4):
    """Six one-step calls on three bit groups, the norm read after each (no flush: its value
    accounts for the held-back pass), S^z after the third (a flush), then the state."""
    N = 17
    s = W.random_system(N, 31, transverse=True)
    psi0 = W.haar_state(N, 32)
    H = _ham(s)
    ctx = ts4.Context.from_system(s, prec="c128")
    ctx.set_schedule(ts4.TS_KERNEL_FUSED, 11, 6)
    ctx.set_chaining(True)
    ctx.set_state(psi0)
    assert ctx.schedule()["groups"] == 3
    ref = psi0
    for k in range(6):
        ctx.step(0.04, 1)
        ref = oracle.ts4(ref, H, 0.04, 1)
        assert abs(ctx.norm() - 1.0) <= 1e-12
        if k == 2:
            np.testing.assert_allclose(ctx.sz(), oracle.sz(ref, N), atol=1e-12)
    assert np.abs(ctx.get_state() - ref).max() <= 1e-12
    ctx.close()


def test_chained_calls_equal_one_chained_call_c64(ts4):
    N = 20
    s = W.xyz_chain(N, 1.0, 0.8, 0.5, seed=33)
    psi0 = W.haar_state(N, 34, np.complex64)
    a = ts4.Context.from_system(s, prec="c64")
    a.set_chaining(True)
    a.set_state(psi0)
    for _ in range(5):
        a.step(0.02, 1)
        a.norm()
    b = ts4.Context.from_system(s, prec="c64")
    b.set_state(psi0)
    b.step(0.02, 5)
    got, want = a.get_state().astype(np.complex128), b.get_state().astype(np.complex128)
    assert np.linalg.norm(got - want) <= 2 * 20 * 5 * (N + 8) * U32
    a.close()
    b.close()


def test_mixed_orders_and_step_lengths_match_the_oracle(ts4):
    """Chaining across different tau and orders: the held-back P_z merges with the next
    call's first slot whatever its length; order 1 takes it in but holds nothing back."""
    N = 15
    s = W.random_system(N, 35, transverse=True)
    psi0 = W.haar_state(N, 36)
    H = _ham(s)
    ctx = ts4.Context.from_system(s, prec="c128")
    ctx.set_chaining(True)
    ctx.set_state(psi0)
    ctx.step(0.03, 2)
    ctx.step(-0.05, 1)
    ctx.step_order(2, 0.02, 2)
    ctx.step_order(1, 0.01, 1)
    ctx.step(0.03, 1)
    ref = oracle.ts4(psi0, H, 0.03, 2)
    ref = oracle.ts4(ref, H, -0.05, 1)
    ref = oracle.apply(oracle.apply(ref, H, 2, 0.02), H, 2, 0.02)
    ref = oracle.apply(ref, H, 1, 0.01)
    ref = oracle.ts4(ref, H, 0.03, 1)
    assert np.abs(ctx.get_state() - ref).max() <= 1e-12
    ctx.close()


def test_state_changes_flush_or_drop_the_held_back_pass(ts4):
    N = 16
    s = W.random_system(N, 37, transverse=True)
    psi0 = W.haar_state(N, 38)
    psi1 = W.haar_state(N, 39)
    H = _ham(s)
    ctx = ts4.Context.from_system(s, prec="c128")
    ctx.set_chaining(True)
    # a new state drops it
    ctx.set_state(psi0)
    ctx.step(0.05, 1)
    ctx.set_state(psi1)
    assert np.array_equal(ctx.get_state(), psi1)
    # new fields flush it first: the held-back slot belongs to the old Hamiltonian
    ctx.step(0.05, 1)
    hx = np.linspace(-0.3, 0.3, N)
    ts4.ts_set_transverse_fields(ctx.ctx, hx, None, N)
    ctx.step(0.05, 1)
    H2 = oracle.Hamiltonian(N, s.Jx, s.Jy, s.Jz, hz=s.hz, hx=hx, hy=np.zeros(N))
    ref = oracle.ts4(oracle.ts4(psi1, H, 0.05, 1), H2, 0.05, 1)
    assert np.abs(ctx.get_state() - ref).max() <= 1e-12
    # a new tile shape flushes it too; so does turning chaining off
    ctx.step(0.05, 1)
    ctx.set_schedule(ts4.TS_KERNEL_FUSED, 12, 3)
    ctx.step(0.05, 1)
    ctx.set_chaining(False)
    ref = oracle.ts4(ref, H2, 0.05, 2)
    assert np.abs(ctx.get_state() - ref).max() <= 1e-12
    ctx.close()
