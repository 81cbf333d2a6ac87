"""Dense-matrix references for small N (test infrastructure).

Everything here is built from Kronecker products of 2x2 spin operators with
numpy and scipy, with no code shared with the oracle or the CUDA library:
  - H_a (a = x, y, z) as 2^N x 2^N matrices (Eq. 1, bonds i < j, S = sigma/2);
  - U1, U2, U4 of Sec. 2 composed from scipy.linalg.expm of those matrices;
  - the exact evolution e^{-iTH} by exact diagonalisation (numpy eigh).
The single-spin basis order here is the basis-index order (down = bit 0,
up = bit 1); the kron order puts spin N (the highest bit) leftmost so that
row/column indices equal basis indices.
"""
from functools import reduce

import numpy as np
from scipy.linalg import expm

# single-spin operators in basis-index order (|down>, |up>)
SX = np.array([[0, 1], [1, 0]], dtype=complex) / 2
SY = np.array([[0, 1j], [-1j, 0]], dtype=complex) / 2   # sigma^y|up> = i|down>, sigma^y|down> = -i|up>
SZ = np.array([[-1, 0], [0, 1]], dtype=complex) / 2
OPS = (SX, SY, SZ)


def site_op(single, j, N):
    """single acting on bit j (spin j+1) of an N-spin system."""
    mats = [np.eye(2, dtype=complex)] * N
    mats[N - 1 - j] = single
    return reduce(np.kron, mats)


def part_matrix(sys, a):
    """H_a = sum_{i<j} J^a_ij S^a_i S^a_j + sum_i h^a_i S^a_i as a dense matrix."""
    N = sys.N
    J = (sys.Jx, sys.Jy, sys.Jz)[a]
    h = (sys.hx, sys.hy, sys.hz)[a]
    dim = 1 << N
    Hm = np.zeros((dim, dim), dtype=complex)
    ops = [site_op(OPS[a], j, N) for j in range(N)]
    for i in range(N):
        for j in range(i + 1, N):
            if J[i, j] != 0.0:
                Hm += J[i, j] * ops[i] @ ops[j]
        if h is not None and h[i] != 0.0:
            Hm += h[i] * ops[i]
    return Hm


def full_matrix(sys):
    return part_matrix(sys, 0) + part_matrix(sys, 1) + part_matrix(sys, 2)


class DenseTS:
    """U1, U2, U4 of Sec. 2 from the exponentials of the three dense parts."""

    def __init__(self, sys):
        self.H = [part_matrix(sys, a) for a in range(3)]

    def u1(self, t):
        ex = [expm(-1j * t * Ha) for Ha in self.H]
        return ex[0] @ ex[1] @ ex[2]            # e^{-itHx} e^{-itHy} e^{-itHz}

    def u2(self, t):
        return self.u1(-t / 2).conj().T @ self.u1(t / 2)

    def u4(self, t):
        a = 1.0 / (4.0 - 4.0 ** (1.0 / 3.0))
        A, B = self.u2(a * t), self.u2((1 - 4 * a) * t)
        return A @ A @ B @ A @ A


def exact_evolution(sys, psi0, T):
    """e^{-iTH} psi0 by exact diagonalisation."""
    w, V = np.linalg.eigh(full_matrix(sys))
    return V @ (np.exp(-1j * w * T) * (V.conj().T @ psi0))
