"""Two-spin correlations <S^a_i S^a_j> and transverse magnetisations <S^x_j>, <S^y_j>
(ts_observe TS_SZSZ, TS_SXSX, TS_SYSY, TS_SX, TS_SY) against the FP64 oracle's
definitions (the spin operators applied to the same state; pinned by closed forms and by
Kronecker-product operators in test_oracle_pins.py).

Conventions of the library (Sec. 3.2): spin j is bit j-1 of the basis index, bit 1 = up,
S = sigma/2.
"""
import numpy as np
import pytest

import oracle
from paper_1305_0036_gb300 import workloads as W

U32 = 2.0 ** -24


@pytest.mark.gpu
@pytest.mark.parametrize("prec,N,tb", [("c128", 13, 12), ("c64", 14, 12), ("c64", 17, 12)])
def test_correlations_match_explicit_operators(ts4, prec, N, tb):
    s = W.random_system(N, 900 + N, transverse=True)
    ctx = ts4.Context.from_system(s, prec=prec)
    ctx.set_schedule(ts4.TS_KERNEL_FUSED, tb, 2)
    ctx.set_state(W.haar_state(N, 910 + N))
    ctx.step(0.05, 3)
    psi = ctx.get_state().astype(np.complex128)
    C, mx, my = oracle.correlations(psi, N)
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
