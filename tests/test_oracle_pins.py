"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics.

None of these compares the oracle with itself: each checks it against a
closed form, a worked example printed in the paper, an identity the paper
states, dense-matrix brute force, exact diagonalisation, or an invariant.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1305_0036_gb300 import workloads as W
from tests.dense_ref import DenseTS, exact_evolution, full_matrix, part_matrix

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# spin operators in the (up, down) order of Eq. 5, written out here
SX_UD = np.array([[0, 1], [1, 0]]) / 2
SY_UD = np.array([[0, -1j], [1j, 0]]) / 2
SZ_UD = np.array([[1, 0], [0, -1]]) / 2


def _sys(N, seed, transverse=False, density=1.0):
    return W.random_system(N, seed, transverse=transverse, density=density)


def _ham(s):
    return oracle.Hamiltonian(s.N, s.Jx, s.Jy, s.Jz, hz=s.hz, hx=s.hx, hy=s.hy)


# ------------------------------------------------------------------ Eq. 5 identities

def test_rotation_identities_eq5():
    """(R^y)^dag S^x R^y = S^z and (R^x)^dag S^y R^x = S^z with the oracle's own matrices."""
    Ry = oracle.rotation_matrix(oracle.Y) / np.sqrt(2)
    Rx = oracle.rotation_matrix(oracle.X) / np.sqrt(2)
    np.testing.assert_allclose(Ry.conj().T @ SX_UD @ Ry, SZ_UD, atol=1e-15)
    np.testing.assert_allclose(Rx.conj().T @ SY_UD @ Rx, SZ_UD, atol=1e-15)
    # the paper's printed matrices (Eq. 5)
    np.testing.assert_allclose(Ry * np.sqrt(2), [[1, -1], [1, 1]])
    np.testing.assert_allclose(Rx * np.sqrt(2), [[1, 1j], [1j, 1]])
    # the dagger forms are the inverses (times the sqrt2^2 = 2 of the unnormalised pair)
    for r, rd in ((oracle.X, oracle.XDAG), (oracle.Y, oracle.YDAG)):
        np.testing.assert_allclose(oracle.rotation_matrix(r) @ oracle.rotation_matrix(rd), 2 * np.eye(2))


def test_zz_phase_values_eq9():
    """Eq. 9: the ZZ term of one bond is +J/4 on aligned spins and -J/4 on anti-aligned ones."""
    J = np.zeros((2, 2))
    J[0, 1] = 0.8
    for s, e in ((0b00, 0.2), (0b01, -0.2), (0b10, -0.2), (0b11, 0.2)):
        assert oracle.zlike_energy(s, 2, J) == pytest.approx(e, abs=1e-16)
    h = np.array([0.3, -0.5])
    # S^z = +1/2 for bit 1: state 0b01 has spin 1 up, spin 2 down
    assert oracle.zlike_energy(0b01, 2, np.zeros((2, 2)), h) == pytest.approx(0.15 + 0.25)


# ------------------------------------------------------------------ Sec. 3.2 worked example

def test_pairing_worked_example_sec32():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "pairs_spin2_N4.txt")) if l.strip() and l[0] != "#"]
    expected = [(int(a, 2), int(b, 2)) for a, b in rows]
    got = []
    for p in range(8):
        lo = oracle.pair_low(p, 1)               # spin 2 = bit 1
        got.append((lo, lo + (1 << 1)))
    assert got == expected


def test_single_spin_rotation_touches_only_its_pairs():
    """Rotating spin j mixes each amplitude only with its partner differing in bit j-1."""
    N = 5
    psi = W.haar_state(N, 7)
    out = oracle.rotate_spin(psi, N, 3, oracle.YDAG)
    M = oracle.rotation_matrix(oracle.YDAG)
    for s in range(1 << N):
        up, dn = (s | 8), (s & ~8)
        vec = M @ np.array([psi[up], psi[dn]])
        assert out[s] == pytest.approx(vec[0] if s & 8 else vec[1], abs=1e-15)


# ------------------------------------------------------------------ P3: one layer on a basis state

@pytest.mark.parametrize("which,mat", [
    (oracle.XDAG, [[1, -1j], [-1j, 1]]), (oracle.X, [[1, 1j], [1j, 1]]),
    (oracle.YDAG, [[1, 1], [-1, 1]]), (oracle.Y, [[1, -1], [1, 1]])])
def test_layer_on_basis_state_is_product_state(which, mat):
    """(x)_j M |s> is the product of the single-spin columns of M (written from Eq. 5)."""
    N, s = 6, 0b101101
    out = oracle.rotate_all(W.basis_state(N, s), N, which)
    M_ud = np.array(mat, dtype=complex)
    # column in basis-index order (down, up) of M applied to the single-spin state of bit j
    cols = []
    for j in range(N):
        col_ud = M_ud[:, 0] if (s >> j) & 1 else M_ud[:, 1]
        cols.append(np.array([col_ud[1], col_ud[0]]))     # reorder to (down, up)
    expected = cols[N - 1]
    for j in range(N - 2, -1, -1):
        expected = np.kron(expected, cols[j])
    np.testing.assert_allclose(out, expected, atol=1e-15)


# ------------------------------------------------------------------ P1: N = 2 is exact

def test_n2_ts4_equals_exact_bell_basis():
    """For N = 2 without fields the three parts commute, so U4(tau) = e^{-i tau H}.
    The exact propagator is written in the Bell basis with eigenvalues worked out by hand:
    E(Phi+-) = (+-Jx -+ Jy + Jz)/4,  E(Psi+-) = (+-Jx +- Jy - Jz)/4."""
    jx, jy, jz = 0.9, -0.4, 0.65
    J = lambda v: np.array([[0.0, v], [0.0, 0.0]])
    H = oracle.Hamiltonian(2, J(jx), J(jy), J(jz))
    r2 = np.sqrt(2)
    # basis index: bit 0 = spin 1, bit 1 = spin 2; |up up> = 3, |down down> = 0
    phi_p = np.array([1, 0, 0, 1]) / r2
    phi_m = np.array([-1, 0, 0, 1]) / r2
    psi_p = np.array([0, 1, 1, 0]) / r2
    psi_m = np.array([0, 1, -1, 0]) / r2
    E = {0: (jx - jy + jz) / 4, 1: (-jx + jy + jz) / 4, 2: (jx + jy - jz) / 4, 3: (-jx - jy - jz) / 4}
    vecs = [phi_p, phi_m, psi_p, psi_m]
    tau = 0.37
    psi0 = W.haar_state(2, 3)
    exact = sum(np.exp(-1j * tau * E[k]) * v * np.vdot(v, psi0) for k, v in enumerate(vecs))
    np.testing.assert_allclose(oracle.ts4(psi0, H, tau, 1), exact, atol=1e-14)
    np.testing.assert_allclose(oracle.ts4(psi0, H, tau / 7, 7), exact, atol=1e-14)


# ------------------------------------------------------------------ P2: Ising special case

def test_ising_closed_form():
    """J^x = J^y = 0: every rotation cancels its inverse and TS4^n = exp(-i n tau H_z) exactly."""
    N = 9
    s = _sys(N, 11)
    Hz = np.diag(part_matrix(type(s)(s.name, N, 0 * s.Jx, 0 * s.Jy, s.Jz, s.hz), 2)).real
    H = oracle.Hamiltonian(N, 0 * s.Jx, 0 * s.Jy, s.Jz, hz=s.hz)
    psi0 = W.haar_state(N, 5)
    n, tau = 13, 0.21
    np.testing.assert_allclose(oracle.ts4(psi0, H, tau, n), np.exp(-1j * n * tau * Hz) * psi0, atol=1e-13)


# ------------------------------------------------------------------ P4: dense brute force

@pytest.mark.parametrize("N,seed,transverse", [(3, 1, False), (5, 2, True), (6, 3, False)])
def test_u1_u2_u4_match_dense_matrices(N, seed, transverse):
    s = _sys(N, seed, transverse=transverse)
    H = _ham(s)
    D = DenseTS(s)
    psi0 = W.haar_state(N, seed + 100)
    t = 0.29
    np.testing.assert_allclose(oracle.apply(psi0, H, 1, t), D.u1(t) @ psi0, atol=1e-13)
    np.testing.assert_allclose(oracle.apply(psi0, H, 2, t), D.u2(t) @ psi0, atol=1e-13)
    np.testing.assert_allclose(oracle.apply(psi0, H, 4, t), D.u4(t) @ psi0, atol=1e-13)
    U = D.u4(t)
    np.testing.assert_allclose(oracle.ts4(psi0, H, t, 5), np.linalg.matrix_power(U, 5) @ psi0, atol=1e-13)


def test_each_part_matches_dense_exponential():
    """exp(-itH_a) = R exp(-itH~) R^dag (Eqs. 7, 10) for each a, against expm of the dense part."""
    from scipy.linalg import expm
    N = 5
    s = _sys(N, 21, transverse=True)
    psi0 = W.haar_state(N, 22)
    J = (s.Jx, s.Jy, s.Jz)
    h = (s.hx, s.hy, s.hz)
    for a in range(3):
        got = oracle.part(psi0, N, a, J[a], h[a], 0.41)
        np.testing.assert_allclose(got, expm(-0.41j * part_matrix(s, a)) @ psi0, atol=1e-13)


# ------------------------------------------------------------------ P5: exact diagonalisation

def _global_error(s, psi0, T, order, nsteps):
    H = _ham(s)
    psi = psi0.copy()
    for _ in range(nsteps):
        psi = oracle.apply(psi, H, order, T / nsteps)
    return np.abs(psi - exact_evolution(s, psi0, T)).max()


@pytest.mark.parametrize("order", [1, 2, 4])
def test_global_error_slope_vs_exact_diagonalisation(order):
    """Global error at fixed T falls as tau^order (order 1, 2 and 4 of Sec. 2)."""
    N = 7
    s = _sys(N, 31, transverse=True)
    psi0 = W.haar_state(N, 32)
    T = 1.2
    steps = [6, 12, 24] if order == 4 else [24, 48, 96]
    errs = [_global_error(s, psi0, T, order, n) for n in steps]
    slopes = [np.log2(errs[k] / errs[k + 1]) for k in range(len(errs) - 1)]
    for sl in slopes:
        assert abs(sl - order) < 0.3, (errs, slopes)


def test_ts4_close_to_exact_at_small_tau():
    N = 8
    s = _sys(N, 41)
    psi0 = W.haar_state(N, 42)
    err = _global_error(s, psi0, 1.0, 4, 50)
    assert err < 1e-7


# ------------------------------------------------------------------ P6: invariants

def test_norm_conserved_to_1e13_over_100_steps():
    N = 10
    s = _sys(N, 51, transverse=True)
    psi = oracle.ts4(W.haar_state(N, 52), _ham(s), 0.05, 100)
    assert abs(oracle.norm(psi, N) - 1.0) < 1e-13


def test_loschmidt_echo_returns_to_initial_state():
    """U4 is palindromic, so U4(-tau)^n U4(tau)^n = 1 and the echo (Eq. 11, Sigma = 0) is 1."""
    N = 9
    s = W.ring_heisenberg(N)
    H = _ham(s)
    psi0 = W.random_phase_state(N, 61)
    fwd = oracle.ts4(psi0, H, 0.03, 40)
    back = oracle.ts4(fwd, H, -0.03, 40)
    assert np.abs(back - psi0).max() < 1e-13
    assert abs(1.0 - oracle.echo(psi0, back, N)) < 1e-13
    assert abs(1.0 - oracle.echo(psi0, fwd, N)) > 1e-3     # the forward state did move


def test_sz_total_violation_scales_as_tau4_for_xxz():
    """XXZ conserves S^z_tot exactly; TS4 leaks amplitude out of the initial magnetisation
    sector only through the splitting, with amplitude ~ tau^4, so <S^z_tot> (second order
    in the leaked amplitude) moves as tau^8."""
    N = 8
    s = W.xyz_chain(N, 1.0, 1.0, 0.6, seed=71)
    H = _ham(s)
    psi0 = W.basis_state(N, W.neel_index(N))
    outside = np.array([bin(k).count("1") != N // 2 for k in range(1 << N)])
    T = 2.0
    leak, mz = [], []
    for n in (5, 10, 20):
        psi = oracle.ts4(psi0, H, T / n, n)
        leak.append(np.linalg.norm(psi[outside]))
        mz.append(abs(oracle.sz(psi, N).sum()))
    for k in range(2):
        assert 14 < leak[k] / leak[k + 1] < 18, leak
    assert 150 < mz[0] / mz[1] < 350, mz


def test_energy_drift_scales_as_tau4():
    N = 8
    s = _sys(N, 81)
    H = _ham(s)
    psi0 = W.haar_state(N, 82)
    e0 = oracle.energy(psi0, H)
    drift = []
    for n in (10, 20):
        drift.append(abs(oracle.energy(oracle.ts4(psi0, H, 3.0 / n, n), H) - e0))
    ratio = drift[0] / drift[1]
    assert 10 < ratio < 24, (drift, ratio)


# ------------------------------------------------------------------ observables by definition

def test_observables_match_dense():
    N = 6
    s = _sys(N, 91, transverse=True)
    psi = W.haar_state(N, 92)
    Hm = full_matrix(s)
    assert oracle.energy(psi, _ham(s)) == pytest.approx(np.vdot(psi, Hm @ psi).real, abs=1e-13)
    np.testing.assert_allclose(oracle.apply_hamiltonian(psi, _ham(s)), Hm @ psi, atol=1e-13)
    from tests.dense_ref import SZ, site_op
    sz = [np.vdot(psi, site_op(SZ, j, N) @ psi).real for j in range(N)]
    np.testing.assert_allclose(oracle.sz(psi, N), sz, atol=1e-14)
    assert oracle.norm(psi, N) == pytest.approx(1.0, abs=1e-14)
    phi = W.haar_state(N, 93)
    assert oracle.overlap(phi, psi, N) == pytest.approx(np.vdot(phi, psi), abs=1e-14)


def test_correlations_match_dense():
    """<S^a_i S^a_j> and <S^x_j>, <S^y_j> against Kronecker-product operators on a random state."""
    N = 5
    psi = W.haar_state(N, 94)
    from tests.dense_ref import SX, SY, SZ, site_op
    C, mx, my = oracle.correlations(psi, N)
    for a, op in (("x", SX), ("y", SY), ("z", SZ)):
        for i in range(N):
            for j in range(N):
                want = np.vdot(psi, site_op(op, i, N) @ (site_op(op, j, N) @ psi)).real
                assert C[a][i, j] == pytest.approx(want, abs=1e-14), (a, i, j)
    np.testing.assert_allclose(mx, [np.vdot(psi, site_op(SX, j, N) @ psi).real for j in range(N)], atol=1e-14)
    np.testing.assert_allclose(my, [np.vdot(psi, site_op(SY, j, N) @ psi).real for j in range(N)], atol=1e-14)


def test_correlations_closed_forms():
    """Product states: every spin along +x, along +y, and a Neel state along z."""
    N = 3
    # |+x> = (|up> + |down>)/sqrt 2 on every site
    plus = np.ones(1 << N, dtype=complex) / np.sqrt(1 << N)
    C, mx, my = oracle.correlations(plus, N)
    np.testing.assert_allclose(mx, 0.5, atol=1e-15)
    np.testing.assert_allclose(my, 0.0, atol=1e-15)
    np.testing.assert_allclose(C["x"], 0.25, atol=1e-15)
    np.testing.assert_allclose(C["z"] - np.diag(np.diag(C["z"])), 0.0, atol=1e-15)
    # |+y> = (|up> + i |down>)/sqrt 2: bit 1 (up) carries 1, bit 0 (down) carries i
    k = np.arange(1 << N)
    amp = np.prod([np.where((k >> b) & 1, 1.0, 1j) for b in range(N)], axis=0) / np.sqrt(1 << N)
    C, mx, my = oracle.correlations(amp, N)
    np.testing.assert_allclose(my, 0.5, atol=1e-15)
    np.testing.assert_allclose(mx, 0.0, atol=1e-15)
    np.testing.assert_allclose(C["y"], 0.25, atol=1e-15)
    # Neel |up down up> along z: <S^z_i S^z_j> = +-1/4, no transverse order
    neel = np.zeros(1 << N, dtype=complex)
    neel[0b101] = 1.0
    C, mx, my = oracle.correlations(neel, N)
    assert C["z"][0, 1] == -0.25 and C["z"][0, 2] == 0.25 and C["z"][1, 1] == 0.25
    np.testing.assert_allclose(C["x"] - np.diag(np.diag(C["x"])), 0.0, atol=1e-15)
    np.testing.assert_allclose(mx, 0.0, atol=1e-15)


def test_suzuki_coefficient():
    a = oracle.suzuki_a()
    assert a == pytest.approx(0.41449077179437573, abs=1e-16)
    assert 4 * a + (1 - 4 * a) == pytest.approx(1.0)
    # the third-order error term cancels: 4 a^3 + (1-4a)^3 = 0
    assert 4 * a ** 3 + (1 - 4 * a) ** 3 == pytest.approx(0.0, abs=1e-15)
