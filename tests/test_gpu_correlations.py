"""Two-spin correlations <S^a_i S^a_j> and transverse magnetisations <S^x_j>, <S^y_j>
(ts_observe TS_SZSZ, TS_SXSX, TS_SYSY, TS_SX, TS_SY) against the operators applied
explicitly to the same state on the host.

Conventions of the library (Sec. 3.2): spin j is bit j-1 of the basis index, bit 1 = up,
S = sigma/2.  sigma^x flips a bit; sigma^y flips it with a factor -i when the result is up
and +i when it is down (sigma^y |up> = i |down>, sigma^y |down> = -i |up>).
"""
import numpy as np
import pytest

from paper_1305_0036_gb300 import workloads as W

U32 = 2.0 ** -24


def _flip(N, psi, mask):
    idx = np.arange(1 << N) ^ mask
    return psi[idx]


def _ysign(N, i):
    """Factor of sigma^y_i on the component whose index s is the result: -i if bit i of s is 1."""
    bits = (np.arange(1 << N) >> i) & 1
    return np.where(bits == 1, -1j, 1j)


def reference(N, psi):
    """Explicit <S^a_i S^a_j> (a = z, x, y) and <S^x_j>, <S^y_j> of a normalised state."""
    w = np.abs(psi) ** 2
    bits = [((np.arange(1 << N) >> i) & 1) - 0.5 for i in range(N)]
    C = {a: np.zeros((N, N)) for a in "zxy"}
    for i in range(N):
        for j in range(N):
            if i == j:
                for a in "zxy":
                    C[a][i, j] = 0.25 * w.sum()
                continue
            C["z"][i, j] = (w * bits[i] * bits[j]).sum()
            m = (1 << i) | (1 << j)
            C["x"][i, j] = 0.25 * np.vdot(psi, _flip(N, psi, m)).real
            C["y"][i, j] = 0.25 * np.vdot(psi, _ysign(N, i) * _ysign(N, j) * _flip(N, psi, m)).real
    mx = np.array([0.5 * np.vdot(psi, _flip(N, psi, 1 << i)).real for i in range(N)])
    my = np.array([0.5 * np.vdot(psi, _ysign(N, i) * _flip(N, psi, 1 << i)).real for i in range(N)])
    return C, mx, my


def test_reference_pins():
    """The host reference itself: closed forms on product states."""
    N = 3
    # all spins up along +x: |+x> = (|up> + |down>)/sqrt 2 on every site
    plus = np.ones(1 << N, dtype=complex) / np.sqrt(1 << N)
    C, mx, my = reference(N, plus)
    np.testing.assert_allclose(mx, 0.5, atol=1e-15)
    np.testing.assert_allclose(my, 0.0, atol=1e-15)
    np.testing.assert_allclose(C["x"], 0.25, atol=1e-15)
    np.testing.assert_allclose(C["z"] - np.diag(np.diag(C["z"])), 0.0, atol=1e-15)
    # all spins up along +y: |+y> = (|up> + i |down>)/sqrt 2; bit 1 = up carries 1, bit 0 carries i
    s = np.arange(1 << N)
    amp = np.prod([np.where((s >> k) & 1, 1.0, 1j) for k in range(N)], axis=0) / np.sqrt(1 << N)
    C, mx, my = reference(N, amp)
    np.testing.assert_allclose(my, 0.5, atol=1e-15)
    np.testing.assert_allclose(mx, 0.0, atol=1e-15)
    np.testing.assert_allclose(C["y"], 0.25, atol=1e-15)
    # Neel state along z: <S^z_i S^z_j> = +-1/4
    neel = np.zeros(1 << N, dtype=complex)
    neel[0b101] = 1.0
    C, _, _ = reference(N, neel)
    assert C["z"][0, 1] == -0.25 and C["z"][0, 2] == 0.25


@pytest.mark.gpu
@pytest.mark.parametrize("prec,N,tb", [("c128", 13, 12), ("c64", 14, 12), ("c64", 17, 12)])
def test_correlations_match_explicit_operators(ts4, prec, N, tb):
    s = W.random_system(N, 900 + N, transverse=True)
    ctx = ts4.Context.from_system(s, prec=prec)
    ctx.set_schedule(ts4.TS_KERNEL_FUSED, tb, 2)
    ctx.set_state(W.haar_state(N, 910 + N))
    ctx.step(0.05, 3)
    psi = ctx.get_state().astype(np.complex128)
    C, mx, my = reference(N, psi)
    # c128: rounding only; c64: the frame rotation adds N rounded butterflies per amplitude
    tol = 1e-12 if prec == "c128" else 8 * (N + 4) * U32
    for a in "zxy":
        np.testing.assert_allclose(ctx.correlations(a), C[a], atol=tol, err_msg=a)
    np.testing.assert_allclose(ctx.magnetization("x"), mx, atol=tol)
    np.testing.assert_allclose(ctx.magnetization("y"), my, atol=tol)
    # the z magnetisation agrees with the correlation row sums' single-site form
    np.testing.assert_allclose(ctx.magnetization("z"), [(np.abs(psi) ** 2 * (((np.arange(1 << N) >> i) & 1) - 0.5)).sum()
                                                        for i in range(N)], atol=tol)
    ctx.close()


@pytest.mark.gpu
def test_correlations_high_bits_and_small_states(ts4):
    """Pairs among the bits above one reduction range (2^13 amplitudes) and a state smaller than a range."""
    for N, tb in ((20, 12), (11, 11)):
        s = W.random_system(N, 950 + N)
        ctx = ts4.Context.from_system(s, prec="c128")
        if N >= 12:
            ctx.set_schedule(ts4.TS_KERNEL_FUSED, tb, 2)
        ctx.set_state(W.haar_state(N, 960 + N))
        psi = ctx.get_state()
        w = np.abs(psi) ** 2
        bits = [((np.arange(1 << N) >> i) & 1) - 0.5 for i in range(N)]
        Cz = ctx.correlations("z")
        for i, j in ((0, N - 1), (N - 2, N - 1), (3, 15 % N), (12 % N, 13 % N)):
            if i != j:
                assert abs(Cz[i, j] - (w * bits[i] * bits[j]).sum()) <= 1e-12
        ctx.close()
