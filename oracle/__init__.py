"""Python binding of the FP64 CPU oracle (oracle/ts4_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` import this module; the CUDA library never does.
The oracle restates Sec. 2 of Dente et al. (TS4 of the XYZ decomposition) in
plain C; see the header comment of ts4_oracle.c for the conventions.

All state vectors are numpy complex128 arrays of length 2^N in basis-index
order (spin j is bit j-1, bit 1 = up).  Coupling matrices are N*N float64
(upper triangle i<j read), fields are length-N float64 or None.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ts4_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

XDAG, X, YDAG, Y = 0, 1, 2, 3

CFLAGS = ["-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11",
          # identical results on x86 and Arm: no FMA contraction; finite complex
          # products are the same with or without the C99 Annex-G inf/nan fix-ups
          "-ffp-contract=off", "-fcx-limited-range"]


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (seconds). Returns its path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i, d, i64, u64 = ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.c_uint64
            sig = {
                "oracle_rotation_matrix": (None, [i, P]),
                "oracle_pair_low": (u64, [u64, i]),
                "oracle_rotate_spin": (None, [P, i, i, i]),
                "oracle_rotate_all": (None, [P, i, i]),
                "oracle_scale": (None, [P, i, d]),
                "oracle_zlike_energy": (d, [u64, i, P, P]),
                "oracle_phase": (None, [P, i, P, P, d]),
                "oracle_part": (None, [P, i, i, P, P, d]),
                "oracle_suzuki_a": (d, []),
                "oracle_apply": (None, [P, i, P, P, P, P, P, P, i, d]),
                "oracle_ts4": (None, [P, i, P, P, P, P, P, P, d, i64]),
                "oracle_norm": (d, [P, i]),
                "oracle_sz": (None, [P, i, P]),
                "oracle_overlap": (None, [P, P, i, P]),
                "oracle_apply_hamiltonian": (None, [P, P, i, P, P, P, P, P, P]),
                "oracle_energy": (d, [P, i, P, P, P, P, P, P]),
                "oracle_correlations": (None, [P, i, P, P, P, P, P]),
                "oracle_num_threads": (i, []),
                "oracle_set_num_threads": (None, [i]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _state(psi, N):
    a = np.ascontiguousarray(psi, dtype=np.complex128)
    if a.shape != (1 << N,):
        raise ValueError(f"state must have 2^{N} amplitudes, got {a.shape}")
    return a


def _mat(J, N):
    return np.ascontiguousarray(np.asarray(J, dtype=np.float64).reshape(N, N))


def _vec(h, N):
    return None if h is None else np.ascontiguousarray(np.asarray(h, dtype=np.float64).reshape(N))


class Hamiltonian:
    """Couplings J^x, J^y, J^z (N*N) and fields h^x, h^y, h^z (N or None)."""

    def __init__(self, N, Jx, Jy, Jz, hz=None, hx=None, hy=None):
        self.N = int(N)
        self.Jx, self.Jy, self.Jz = _mat(Jx, N), _mat(Jy, N), _mat(Jz, N)
        self.hx, self.hy, self.hz = _vec(hx, N), _vec(hy, N), _vec(hz, N)

    def args(self):
        return (_ptr(self.Jx), _ptr(self.Jy), _ptr(self.Jz),
                _ptr(self.hx), _ptr(self.hy), _ptr(self.hz))


def rotation_matrix(which: int) -> np.ndarray:
    """The unnormalised (sqrt2 x) rotation matrix in (up, down) order."""
    out = np.zeros(8)
    lib().oracle_rotation_matrix(which, _ptr(out))
    return (out[0::2] + 1j * out[1::2]).reshape(2, 2)


def pair_low(p: int, b: int) -> int:
    return int(lib().oracle_pair_low(p, b))


def suzuki_a() -> float:
    return float(lib().oracle_suzuki_a())


def rotate_spin(psi, N, b, which):
    a = _state(psi, N).copy()
    lib().oracle_rotate_spin(_ptr(a), N, b, which)
    return a


def rotate_all(psi, N, which):
    a = _state(psi, N).copy()
    lib().oracle_rotate_all(_ptr(a), N, which)
    return a


def zlike_energy(s, N, J, h=None):
    return float(lib().oracle_zlike_energy(s, N, _ptr(_mat(J, N)), _ptr(_vec(h, N))))


def phase(psi, N, J, h, t):
    a = _state(psi, N).copy()
    lib().oracle_phase(_ptr(a), N, _ptr(_mat(J, N)), _ptr(_vec(h, N)), float(t))
    return a


def part(psi, N, alpha, J, h, t):
    a = _state(psi, N).copy()
    lib().oracle_part(_ptr(a), N, alpha, _ptr(_mat(J, N)), _ptr(_vec(h, N)), float(t))
    return a


def apply(psi, H: Hamiltonian, order: int, t: float):
    """One application of U1(t), U2(t) or U4(t)."""
    a = _state(psi, H.N).copy()
    lib().oracle_apply(_ptr(a), H.N, *H.args(), int(order), float(t))
    return a


def ts4(psi, H: Hamiltonian, tau: float, nsteps: int):
    """nsteps TS4 steps: U4(tau)^nsteps psi (a new array)."""
    a = _state(psi, H.N).copy()
    lib().oracle_ts4(_ptr(a), H.N, *H.args(), float(tau), int(nsteps))
    return a


def norm(psi, N):
    return float(lib().oracle_norm(_ptr(_state(psi, N)), N))


def sz(psi, N):
    out = np.zeros(N)
    lib().oracle_sz(_ptr(_state(psi, N)), N, _ptr(out))
    return out


def overlap(a, b, N):
    out = np.zeros(2)
    lib().oracle_overlap(_ptr(_state(a, N)), _ptr(_state(b, N)), N, _ptr(out))
    return complex(out[0], out[1])


def echo(psi0, psi, N):
    """Loschmidt echo |<psi0|psi>|^2 (Eq. 11)."""
    return abs(overlap(psi0, psi, N)) ** 2


def apply_hamiltonian(psi, H: Hamiltonian):
    a = _state(psi, H.N)
    out = np.zeros_like(a)
    lib().oracle_apply_hamiltonian(_ptr(a), _ptr(out), H.N, *H.args())
    return out


def energy(psi, H: Hamiltonian):
    return float(lib().oracle_energy(_ptr(_state(psi, H.N)), H.N, *H.args()))


def correlations(psi, N):
    """Two-spin correlations <S^a_i S^a_j> (a = "z", "x", "y": N x N arrays, diagonal =
    norm/4) and the transverse magnetisations <S^x_j>, <S^y_j>, by direct action of the spin
    operators: returns (C, mx, my) with C a dict of the three matrices."""
    a = _state(psi, N)
    czz, cxx, cyy = np.zeros((N, N)), np.zeros((N, N)), np.zeros((N, N))
    mx, my = np.zeros(N), np.zeros(N)
    lib().oracle_correlations(_ptr(a), N, _ptr(czz), _ptr(cxx), _ptr(cyy), _ptr(mx), _ptr(my))
    return {"z": czz, "x": cxx, "y": cyy}, mx, my


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's parallel loops from now on (for timing it on one core)."""
    lib().oracle_set_num_threads(int(n))
