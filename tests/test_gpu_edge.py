"""GPU edge cases: the smallest systems, degenerate step counts and angles, and the N=2 case
in which TS4 is exact (all three bond terms of one pair commute, Sec. 2).

Tolerances as in test_gpu_parity.py: complex128 max |diff| <= 1e-12; complex64
||diff||_2 <= L (N + 8) 2^-24 for L Walsh-Hadamard layers.
"""
import numpy as np
import pytest

import oracle
from paper_1305_0036_gb300 import workloads as W

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _ham(s):
    return oracle.Hamiltonian(s.N, s.Jx, s.Jy, s.Jz, hz=s.hz, hx=s.hx, hy=s.hy)


def _run(ts4, s, psi0, tau, nsteps, prec):
    ctx = ts4.Context.from_system(s, prec=prec)
    ctx.set_state(psi0)
    ctx.step(tau, nsteps)
    out = ctx.get_state().astype(np.complex128)
    ctx.close()
    return out


@pytest.mark.parametrize("N", [1, 2, 3, 5, 7])
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_smallest_systems_match_oracle(ts4, N, prec):
    """Below the tile size the library runs the per-layer kernels; N=1 has no bonds at all."""
    s = W.random_system(N, 40 + N, transverse=True)
    psi0 = W.haar_state(N, 50 + N)
    nsteps, tau = 3, 0.09
    ref = oracle.ts4(psi0, _ham(s), tau, nsteps)
    got = _run(ts4, s, psi0, tau, nsteps, prec)
    if prec == "c128":
        assert np.abs(got - ref).max() <= 1e-12
    else:
        assert np.linalg.norm(got - ref) <= 20 * nsteps * (N + 8) * U32


def test_two_spins_without_field_is_exact(ts4):
    """N=2, h=0: S^x S^x, S^y S^y and S^z S^z of one pair commute, so every Trotter-Suzuki
    order gives e^{-i n tau H} exactly; compared with the dense matrix exponential."""
    expm = pytest.importorskip("scipy.linalg").expm
    from tests.dense_ref import part_matrix
    s = W.xyz_chain(2, 0.9, -0.4, 1.3, h=0.0)
    H = sum(part_matrix(s, a) for a in range(3))
    psi0 = W.haar_state(2, 7)
    tau, n = 0.3, 5
    exact = expm(-1j * n * tau * H) @ psi0
    got = _run(ts4, s, psi0, tau, n, "c128")
    assert np.abs(got - exact).max() <= 1e-13


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_zero_steps_leave_the_state_untouched(ts4, prec):
    N = 14
    s = W.random_system(N, 3, transverse=True)
    psi0 = W.haar_state(N, 4, np.complex128 if prec == "c128" else np.complex64)
    got = _run(ts4, s, psi0, 0.05, 0, prec)
    assert np.array_equal(got, psi0.astype(np.complex128))


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_zero_tau_is_the_identity_up_to_rounding(ts4, prec):
    """U4(0) = 1: the rotations still run (with their exact 2^-N scalings) and the phases are 1."""
    N = 17
    s = W.random_system(N, 5, transverse=True)
    psi0 = W.haar_state(N, 6)
    nsteps = 2
    got = _run(ts4, s, psi0, 0.0, nsteps, prec)
    if prec == "c128":
        assert np.abs(got - psi0).max() <= 1e-12
    else:
        assert np.linalg.norm(got - psi0) <= 20 * nsteps * (N + 8) * U32


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_backward_steps_undo_forward_steps(ts4, prec):
    """U4 is palindromic, so U4(-tau)^n U4(tau)^n = 1 (the echo of Sec. 4.2), here on a
    three-group fused schedule with uneven windows."""
    N = 23
    s = W.random_system(N, 8, transverse=True)
    psi0 = W.haar_state(N, 9)
    ctx = ts4.Context.from_system(s, prec=prec)
    ctx.set_state(psi0)
    n = 4
    ctx.step(0.05, n)
    ctx.step(-0.05, n)
    got = ctx.get_state().astype(np.complex128)
    assert ctx.schedule()["groups"] == 3
    ctx.close()
    if prec == "c128":
        assert np.abs(got - psi0).max() <= 1e-12
    else:
        assert np.linalg.norm(got - psi0) <= 2 * 20 * n * (N + 8) * U32
