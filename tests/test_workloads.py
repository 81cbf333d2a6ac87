"""The seeded input generators: shapes, determinism and the structure of each workload."""
import numpy as np

from paper_1305_0036_gb300 import workloads as W


def test_ladder_shape_and_determinism():
    a, b = W.ladder(12), W.ladder(12)
    assert a.N == 24 and a.meta["bonds"] == 12 + 2 * 11
    for M in (a.Jx, a.Jy, a.Jz):
        assert np.count_nonzero(M) == 34
        assert np.all(np.tril(M) == 0) and np.all(np.abs(M) <= 1)
    np.testing.assert_array_equal(a.Jz, b.Jz)
    assert np.all(np.abs(a.hz) <= 0.5)


def test_dipolar_chain_couplings():
    s = W.dipolar_chain(28)
    assert np.count_nonzero(s.Jz) == 378
    assert s.Jz[0, 1] == 1.0 and s.Jz[3, 5] == 1 / 8
    np.testing.assert_array_equal(s.Jx, -s.Jz / 2)
    np.testing.assert_array_equal(s.Jy, s.Jx)


def test_neel_indices():
    assert W.neel_index(4) == 0b0101
    # 2x2 ladder: sites (r,l) -> bit 2r+l; up iff r+l even: (0,0) and (1,1) -> bits 0 and 3
    assert W.neel_ladder_index(2) == 0b1001


def test_random_phase_state_eq_a1():
    N = 6
    psi = W.random_phase_state(N, 3)
    assert np.all(psi[0::2] == 0)                         # spin 1 is up
    np.testing.assert_allclose(np.abs(psi[1::2]), 2 ** (-(N - 1) / 2))
    np.testing.assert_array_equal(psi, W.random_phase_state(N, 3))


def test_haar_state_normalised():
    psi = W.haar_state(10, 1)
    assert abs(np.vdot(psi, psi).real - 1) < 1e-14


def test_configs_build():
    c = W.config(0)
    assert c["system"].N == 12 and c["prec"] == "c128"
    c = W.config(3)
    assert [s.N for s in c["systems"]] == [16, 18, 20, 22]
    c = W.config(4)
    assert c["system"].N == 33 and np.all(c["system"].hz == 0.1)
