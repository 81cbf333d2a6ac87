"""Seeded synthetic inputs shaped like the workloads of Dente et al. (Sec. 4).

This module only draws couplings, fields and initial states.  It holds none of
the method's arithmetic, so both the CUDA library's tests and the CPU oracle
may use it.  The paper publishes no dataset: its accuracy runs (Sec. 4.2) use
one-dimensional chains and rings of N = 16-22 spins, Heisenberg couplings,
double-quantum variants and random-phase initial states (Eq. A.1).  The
generators below produce stand-ins of those shapes, every one from a fixed
seed through ``numpy.random.default_rng``.

Conventions: spin j (1-based) is bit j-1 of the basis index, bit 1 = up.
Coupling matrices are N*N float64 with the bond (i, j), i < j, stored at
[i, j]; the lower triangle and the diagonal are zero.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 1305036


@dataclass
class System:
    """A spin Hamiltonian: couplings J^x, J^y, J^z (N*N) and fields (length N)."""
    name: str
    N: int
    Jx: np.ndarray
    Jy: np.ndarray
    Jz: np.ndarray
    hz: np.ndarray
    hx: np.ndarray | None = None
    hy: np.ndarray | None = None
    meta: dict = field(default_factory=dict)


def _zeros(N):
    return np.zeros((N, N), dtype=np.float64)


def _bond(J, i, j, v):
    a, b = (i, j) if i < j else (j, i)
    J[a, b] = v


def ring_heisenberg(N: int = 12, J: float = 1.0) -> System:
    """Periodic ring, isotropic nearest-neighbour Heisenberg J^x = J^y = J^z = J, no field."""
    Jx = _zeros(N)
    for i in range(N):
        _bond(Jx, i, (i + 1) % N, J)
    return System(f"ring{N}_heisenberg", N, Jx, Jx.copy(), Jx.copy(), np.zeros(N))


def ladder(L: int = 12, seed: int = SEED_BASE + 2, jmax: float = 1.0, hmax: float = 0.5) -> System:
    """Two-leg ladder 2 x L with open ends; site (rung r, leg l) is spin 2r + l + 1 (bit 2r + l).

    Rung bonds (2r, 2r+1) and leg bonds (2r+l, 2r+2+l); every bond draws its own
    J^x, J^y, J^z i.i.d. uniform in [-jmax, jmax]; h_i uniform in [-hmax, hmax].
    """
    N = 2 * L
    rng = np.random.default_rng(seed)
    bonds = [(2 * r, 2 * r + 1) for r in range(L)]
    bonds += [(2 * r + l, 2 * r + 2 + l) for r in range(L - 1) for l in range(2)]
    Js = [_zeros(N) for _ in range(3)]
    for (i, j) in bonds:
        v = rng.uniform(-jmax, jmax, size=3)
        for a in range(3):
            _bond(Js[a], i, j, v[a])
    hz = rng.uniform(-hmax, hmax, size=N)
    return System(f"ladder2x{L}", N, *Js, hz, meta={"bonds": len(bonds), "seed": seed})


def dipolar_chain(N: int = 28) -> System:
    """Open chain with all-to-all XXZ couplings J^z_ij = 1/|i-j|^3, J^x = J^y = -J^z/2, no field."""
    Jz = _zeros(N)
    for i in range(N):
        for j in range(i + 1, N):
            Jz[i, j] = 1.0 / (j - i) ** 3
    return System(f"dipolar{N}", N, -Jz / 2, -Jz / 2, Jz, np.zeros(N),
                  meta={"bonds": N * (N - 1) // 2})


def xyz_chain(N: int, jx: float = 1.0, jy: float = 0.8, jz: float = 0.5,
              h: float | None = None, seed: int | None = None, hmax: float = 1.0,
              periodic: bool = False) -> System:
    """Nearest-neighbour XYZ chain; the field is the constant h, or uniform in [-hmax, hmax] from seed."""
    Js = [_zeros(N) for _ in range(3)]
    nb = N if periodic else N - 1
    for i in range(nb):
        for a, v in enumerate((jx, jy, jz)):
            _bond(Js[a], i, (i + 1) % N, v)
    if h is not None:
        hz = np.full(N, float(h))
    elif seed is not None:
        hz = np.random.default_rng(seed).uniform(-hmax, hmax, size=N)
    else:
        hz = np.zeros(N)
    return System(f"xyz{N}", N, *Js, hz, meta={"seed": seed})


def random_system(N: int, seed: int, jmax: float = 1.0, hmax: float = 0.5,
                  transverse: bool = False, density: float = 1.0) -> System:
    """All-to-all random couplings (each bond present with probability `density`), for tests."""
    rng = np.random.default_rng(seed)
    Js = [_zeros(N) for _ in range(3)]
    for i in range(N):
        for j in range(i + 1, N):
            if rng.uniform() < density:
                v = rng.uniform(-jmax, jmax, size=3)
                for a in range(3):
                    Js[a][i, j] = v[a]
    hz = rng.uniform(-hmax, hmax, size=N)
    hx = rng.uniform(-hmax, hmax, size=N) if transverse else None
    hy = rng.uniform(-hmax, hmax, size=N) if transverse else None
    return System(f"random{N}_s{seed}", N, *Js, hz, hx, hy, meta={"seed": seed})


# ---------------------------------------------------------------- initial states

def neel_index(N: int) -> int:
    """|up down up down ...>: spin 1 (bit 0) up, alternating."""
    return sum(1 << k for k in range(0, N, 2))


def neel_ladder_index(L: int) -> int:
    """Bipartite Neel state of the 2 x L ladder: site (r, l) up iff r + l is even."""
    return sum(1 << (2 * r + l) for r in range(L) for l in range(2) if (r + l) % 2 == 0)


def basis_state(N: int, s: int, dtype=np.complex128) -> np.ndarray:
    psi = np.zeros(1 << N, dtype=dtype)
    psi[s] = 1.0
    return psi


def random_phase_state(N: int, seed: int, dtype=np.complex128) -> np.ndarray:
    """Eq. A.1: spin 1 up, times an equal-weight superposition of the 2^{N-1} configurations
    of the other spins with phases phi_j uniform in [0, 2 pi)."""
    rng = np.random.default_rng(seed)
    n = 1 << (N - 1)
    phi = rng.uniform(0.0, 2.0 * np.pi, size=n)
    amp = np.exp(1j * phi) / np.sqrt(n)
    psi = np.zeros(1 << N, dtype=dtype)
    psi[1::2] = amp.astype(dtype)            # bit 0 (spin 1) = 1
    return psi


def haar_state(N: int, seed: int, dtype=np.complex128) -> np.ndarray:
    """i.i.d. complex Gaussian amplitudes, normalised (a Haar-random pure state)."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(1 << N) + 1j * rng.standard_normal(1 << N)
    z /= np.sqrt(np.vdot(z, z).real)
    return z.astype(dtype)


# ---------------------------------------------------------------- the five workloads

def config(idx: int) -> dict:
    """The benchmark workloads (0-based index), as plain dicts of inputs."""
    if idx == 0:
        s = ring_heisenberg(12)
        return dict(system=s, state=("basis", neel_index(12)), tau=0.01, nsteps=100, prec="c128")
    if idx == 1:
        s = ladder(12)
        return dict(system=s, state=("basis", neel_ladder_index(12)), tau=0.02, nsteps=1000, prec="c64")
    if idx == 2:
        s = dipolar_chain(28)
        return dict(system=s, state=("random_phase", SEED_BASE + 3), tau=0.01, nsteps=500, prec="c64")
    if idx == 3:
        systems = [xyz_chain(n, 1.0, 0.8, 0.5, seed=SEED_BASE + 4 * 100 + n) for n in (16, 18, 20, 22)]
        return dict(systems=systems, states_per_system=64, state_seed=SEED_BASE + 4, tau=0.02,
                    nsteps=200, prec="c64")
    if idx == 4:
        s = xyz_chain(33, 1.0, 0.8, 0.5, h=0.1)
        return dict(system=s, state=("basis", neel_index(33)), tau=0.02, nsteps=200, prec="c64")
    raise ValueError(idx)


def make_state(spec, N: int, dtype=np.complex128) -> np.ndarray:
    kind, arg = spec
    if kind == "basis":
        return basis_state(N, arg, dtype)
    if kind == "random_phase":
        return random_phase_state(N, arg, dtype)
    if kind == "haar":
        return haar_state(N, arg, dtype)
    raise ValueError(kind)
