"""Thin ctypes binding of libts4.so (include/ts4.h): argument marshalling only.

Every computation runs in the CUDA library; nothing here touches amplitudes.
Importing this module loads the library and raises ImportError if it is
missing (build it with ``paper_1305_0036_gb300.build.build()``): there is no
CPU fallback.  torch supplies device memory (tensors bound as the state and
work buffers) and the CUDA stream.

The functions mirror the C ABI one to one (ts_create, ts_step, ...); the
``Context`` class wraps them for convenience.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libts4.so")

TS_OK, TS_ERR_ARG, TS_ERR_OOM, TS_ERR_CUDA, TS_ERR_TIMEOUT, TS_ERR_STATE = 0, -1, -2, -3, -4, -5
TS_C64, TS_C128 = 0, 1
TS_NORM, TS_ENERGY, TS_SZ, TS_ECHO, TS_OVERLAP = 1, 2, 3, 4, 5
TS_SZSZ, TS_SXSX, TS_SYSY, TS_SX, TS_SY = 6, 7, 8, 9, 10
TS_KERNEL_FUSED, TS_KERNEL_BASIC = 0, 1
_STATUS = {0: "TS_OK", -1: "TS_ERR_ARG", -2: "TS_ERR_OOM", -3: "TS_ERR_CUDA", -4: "TS_ERR_TIMEOUT",
           -5: "TS_ERR_STATE"}

# every entry point declared in include/ts4.h, with its ctypes signature
_P, _I, _D, _I64, _U64, _SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.c_uint64, ctypes.c_size_t
SIGNATURES = {
    "ts_create": (_I, [ctypes.POINTER(_P), _I, _P, _P, _P, _P, _I, _P]),
    "ts_set_transverse_fields": (_I, [_P, _P, _P]),
    "ts_bind_buffers": (_I, [_P, _P, _P, _P, _SZ]),
    "ts_set_state": (_I, [_P, _P, _I]),
    "ts_set_basis_state": (_I, [_P, _U64]),
    "ts_save_reference": (_I, [_P]),
    "ts_step": (_I, [_P, _D, _I64]),
    "ts_step_order": (_I, [_P, _I, _D, _I64]),
    "ts_observe": (_I, [_P, _I, _P]),
    "ts_get_state": (_I, [_P, _P, _I]),
    "ts_destroy": (_I, [_P]),
    "ts_last_error": (ctypes.c_char_p, [_P]),
    "ts_set_schedule": (_I, [_P, _I, _I, _I]),
    "ts_get_schedule": (_I, [_P, _P, _P, _P, _P, _P]),
    "ts_step_bound": (_D, [_P]),
    "ts_step_bound_host": (_D, [_I, _P, _P, _P, _P, _P, _P]),
    "ts_tile_global_index": (_U64, [_I, _I, _I, _I, _U64, _U64]),
    "ts_plan": (_I, [_I, _I, _I, _I, _I, _I64, _I, _P, _I, _P, _P, _I64, _P]),
    "ts_set_chaining": (_I, [_P, _I]),
    "ts_flush": (_I, [_P]),
    "ts_kernel_launches": (_I64, [_P]),
    "ts_reduce_sz_static": (_I, [_P, _I, _I, _P, _P]),
    "ts_autotune": (_I, [_P, _D, _I, ctypes.c_char_p, _P]),
    "ts_set_phase_tables": (_I, [_P, _I]),
    "ts_batch_create": (_I, [ctypes.POINTER(_P), _I, _P, _P, _P, _P, _P, _P, _I, _P]),
    "ts_batch_bind_states": (_I, [_P, _I, _P, _SZ]),
    "ts_batch_set_states": (_I, [_P, _I, _P, _I]),
    "ts_batch_get_states": (_I, [_P, _I, _P, _I]),
    "ts_batch_set_schedule": (_I, [_P, _I, _I]),
    "ts_batch_get_schedule": (_I, [_P, _P, _P]),
    "ts_batch_autotune": (_I, [_P, _D, _I, ctypes.c_char_p, _P]),
    "ts_batch_step": (_I, [_P, _D, _I64]),
    "ts_batch_status": (_I, [_P]),
    "ts_batch_set_wait": (_I, [_P, _D, _I]),
    "ts_batch_observe": (_I, [_P, _I, _P]),
    "ts_batch_kernel_launches": (_I64, [_P]),
    "ts_batch_last_error": (ctypes.c_char_p, [_P]),
    "ts_batch_destroy": (_I, [_P]),
    "ts_version": (ctypes.c_char_p, []),
}


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build the CUDA library first "
                          "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = load()


class TS4Error(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


def _check(st, ctx=None):
    if st != TS_OK:
        msg = _lib.ts_last_error(ctx).decode() if ctx else ""
        raise TS4Error(st, msg)


def _mat(J, N):
    return np.ascontiguousarray(np.asarray(J, dtype=np.float64).reshape(N, N))


def _vec(h, N):
    return None if h is None else np.ascontiguousarray(np.asarray(h, dtype=np.float64).reshape(N))


def _p(a):
    return None if a is None else a.ctypes.data


# ---------------------------------------------------------------- C-named wrappers

def ts_create(N, Jx, Jy, Jz, h=None, prec=TS_C64, stream=None):
    Jx, Jy, Jz, h = _mat(Jx, N), _mat(Jy, N), _mat(Jz, N), _vec(h, N)
    out = _P()
    _check(_lib.ts_create(ctypes.byref(out), int(N), _p(Jx), _p(Jy), _p(Jz), _p(h), int(prec), stream))
    return out


def ts_set_transverse_fields(ctx, hx, hy, N):
    hx, hy = _vec(hx, N), _vec(hy, N)
    _check(_lib.ts_set_transverse_fields(ctx, _p(hx), _p(hy)), ctx)


def ts_bind_buffers(ctx, psi_ptr, ref_ptr, scratch_ptr, nbytes):
    _check(_lib.ts_bind_buffers(ctx, psi_ptr, ref_ptr, scratch_ptr, int(nbytes)), ctx)


def ts_set_state(ctx, ptr, on_device):
    _check(_lib.ts_set_state(ctx, ptr, int(on_device)), ctx)


def ts_set_basis_state(ctx, s):
    _check(_lib.ts_set_basis_state(ctx, int(s)), ctx)


def ts_save_reference(ctx):
    _check(_lib.ts_save_reference(ctx), ctx)


def ts_step(ctx, tau, nsteps):
    _check(_lib.ts_step(ctx, float(tau), int(nsteps)), ctx)


def ts_step_order(ctx, order, tau, nsteps):
    _check(_lib.ts_step_order(ctx, int(order), float(tau), int(nsteps)), ctx)


def ts_observe(ctx, what, n_out):
    out = np.zeros(n_out, dtype=np.float64)
    _check(_lib.ts_observe(ctx, int(what), out.ctypes.data), ctx)
    return out


def ts_get_state(ctx, ptr, on_device):
    _check(_lib.ts_get_state(ctx, ptr, int(on_device)), ctx)


def ts_destroy(ctx):
    _check(_lib.ts_destroy(ctx))


def ts_last_error(ctx):
    return _lib.ts_last_error(ctx).decode()


def ts_set_schedule(ctx, kernel, tile_bits=0, coalesce_bits=0):
    _check(_lib.ts_set_schedule(ctx, int(kernel), int(tile_bits), int(coalesce_bits)), ctx)


def ts_get_schedule(ctx):
    v = [ctypes.c_int() for _ in range(5)]
    _check(_lib.ts_get_schedule(ctx, *[ctypes.byref(x) for x in v]), ctx)
    return dict(zip(("kernel", "tile_bits", "coalesce_bits", "groups", "passes_per_step"), [x.value for x in v]))


def ts_step_bound(ctx):
    return float(_lib.ts_step_bound(ctx))


def ts_step_bound_host(N, Jx, Jy, Jz, hx=None, hy=None, hz=None):
    """The Eq. 4 time-step bound from the couplings, on the host (no GPU)."""
    Jx, Jy, Jz = _mat(Jx, N), _mat(Jy, N), _mat(Jz, N)
    hx, hy, hz = _vec(hx, N), _vec(hy, N), _vec(hz, N)
    return float(_lib.ts_step_bound_host(int(N), _p(Jx), _p(Jy), _p(Jz), _p(hx), _p(hy), _p(hz)))


def ts_tile_global_index(N, c, w, h, f, e):
    return int(_lib.ts_tile_global_index(int(N), int(c), int(w), int(h), int(f), int(e)))


class PlanGroup(ctypes.Structure):
    _fields_ = [("c", ctypes.c_int), ("w", ctypes.c_int), ("h", ctypes.c_int)]


class PlanPass(ctypes.Structure):
    _fields_ = [("group", ctypes.c_int), ("slot", ctypes.c_int), ("rot_before", ctypes.c_uint64),
                ("rot_after", ctypes.c_uint64), ("dup", ctypes.c_int)]


def ts_plan(N, prec=TS_C64, tile_bits=0, coalesce_bits=0, order=4, nsteps=1, chain=0):
    """The fused-pass plan (host only, no GPU): a list of group dicts and a list of pass dicts.
    chain: bit 1 = the call continues a held-back pass, bit 2 = it holds back its final pass."""
    ng, npass = ctypes.c_int(), ctypes.c_int64()
    st = _lib.ts_plan(int(N), int(prec), int(tile_bits), int(coalesce_bits), int(order), int(nsteps), int(chain),
                      None, 0, ctypes.byref(ng), None, 0, ctypes.byref(npass))
    if st:
        raise TS4Error(st, "ts_plan: invalid arguments")
    G = (PlanGroup * max(ng.value, 1))()
    P = (PlanPass * max(npass.value, 1))()
    _check(_lib.ts_plan(int(N), int(prec), int(tile_bits), int(coalesce_bits), int(order), int(nsteps), int(chain),
                        ctypes.cast(G, _P), ng.value, ctypes.byref(ng), ctypes.cast(P, _P), npass.value,
                        ctypes.byref(npass)), None)
    groups = [dict(c=g.c, w=g.w, h=g.h) for g in G[:ng.value]]
    passes = [dict(group=p.group, slot=p.slot, rot_before=int(p.rot_before), rot_after=int(p.rot_after),
                   dup=p.dup) for p in P[:npass.value]]
    return groups, passes


def ts_kernel_launches(ctx):
    return int(_lib.ts_kernel_launches(ctx))


def ts_reduce_sz_static(psi_ptr, N, prec, out_ptr, stream=None):
    """Norm and <S^z_j> of a device state into a device buffer of N + 1 doubles, with no allocation."""
    _check(_lib.ts_reduce_sz_static(psi_ptr, int(N), int(prec), out_ptr, stream))


def ts_version():
    return _lib.ts_version().decode()


def _bcheck(st, b):
    if st != TS_OK:
        raise TS4Error(st, _lib.ts_batch_last_error(b).decode() if b else "")


class Batch:
    """An ensemble of states of several systems (uneven N) evolved together.

    systems: list of objects with N, Jx, Jy, Jz, hz; nstates: states per system.
    Device memory for the states comes from torch (one tensor per system).
    """

    def __init__(self, systems, nstates, prec="c64", stream=None, device=None):
        import torch
        self.torch = torch
        self.systems = list(systems)
        self.nstates = [int(k) for k in nstates]
        self.prec = TS_C64 if prec in ("c64", TS_C64) else TS_C128
        self.dtype = torch.complex64 if self.prec == TS_C64 else torch.complex128
        self.device = torch.device(device or "cuda")
        n = len(self.systems)
        Ns = (ctypes.c_int * n)(*[s.N for s in self.systems])
        self._keep = []
        def arr(attr):
            ptrs = []
            for s in self.systems:
                a = getattr(s, attr)
                if a is None:
                    ptrs.append(None)
                    continue
                a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
                self._keep.append(a)
                ptrs.append(a.ctypes.data)
            return (ctypes.c_void_p * n)(*ptrs)
        Jx, Jy, Jz, hz = arr("Jx"), arr("Jy"), arr("Jz"), arr("hz")
        ks = (ctypes.c_int * n)(*self.nstates)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            out = _P()
            _check(_lib.ts_batch_create(ctypes.byref(out), n, ctypes.cast(Ns, _P), ctypes.cast(Jx, _P),
                                        ctypes.cast(Jy, _P), ctypes.cast(Jz, _P), ctypes.cast(hz, _P),
                                        ctypes.cast(ks, _P), self.prec, ctypes.c_void_p(self.stream.cuda_stream)))
            self.b = out
            self.states = [torch.empty((k, 1 << s.N), dtype=self.dtype, device=self.device)
                           for s, k in zip(self.systems, self.nstates)]
        for i, t in enumerate(self.states):
            _bcheck(_lib.ts_batch_bind_states(self.b, i, t.data_ptr(), t.numel() * t.element_size()), self.b)

    def set_states(self, i, amps):
        """amps: (nstates_i, 2^N_i) numpy array or device tensor."""
        if isinstance(amps, self.torch.Tensor) and amps.is_cuda:
            a = amps.to(self.dtype).contiguous()
            _bcheck(_lib.ts_batch_set_states(self.b, i, a.data_ptr(), 1), self.b)
        else:
            a = np.ascontiguousarray(np.asarray(amps), dtype=np.complex64 if self.prec == TS_C64 else np.complex128)
            _bcheck(_lib.ts_batch_set_states(self.b, i, a.ctypes.data, 0), self.b)

    def get_states(self, i):
        a = np.empty((self.nstates[i], 1 << self.systems[i].N),
                     dtype=np.complex64 if self.prec == TS_C64 else np.complex128)
        _bcheck(_lib.ts_batch_get_states(self.b, i, a.ctypes.data, 0), self.b)
        return a

    def set_schedule(self, tile_bits=0, coalesce_bits=0):
        _bcheck(_lib.ts_batch_set_schedule(self.b, int(tile_bits), int(coalesce_bits)), self.b)

    def schedule(self):
        tb, cb = ctypes.c_int(), ctypes.c_int()
        _bcheck(_lib.ts_batch_get_schedule(self.b, ctypes.byref(tb), ctypes.byref(cb)), self.b)
        return {"tile_bits": tb.value, "coalesce_bits": cb.value}

    def autotune(self, tau, reps=2, cache_path=None):
        """Brute-force search of the ensemble's tile shape (library side); returns the best ms
        per ensemble step, or -1 when the shape came from the cache file."""
        ms = ctypes.c_double(0.0)
        _bcheck(_lib.ts_batch_autotune(self.b, float(tau), int(reps),
                                       cache_path.encode() if cache_path else None, ctypes.byref(ms)), self.b)
        return ms.value

    def step(self, tau, nsteps=1):
        _bcheck(_lib.ts_batch_step(self.b, float(tau), int(nsteps)), self.b)

    def status(self):
        """Waits for the queued work; raises TS4Error(TS_ERR_TIMEOUT) if a dependency wait ran out."""
        _bcheck(_lib.ts_batch_status(self.b), self.b)

    def set_wait(self, limit_s=2.0, hold=False):
        """Bound of every dependency wait of the ensemble kernel; hold=True tests the timeout path."""
        _bcheck(_lib.ts_batch_set_wait(self.b, float(limit_s), 1 if hold else 0), self.b)

    def norms(self):
        out = np.zeros(sum(self.nstates))
        _bcheck(_lib.ts_batch_observe(self.b, TS_NORM, out.ctypes.data), self.b)
        return out

    def sz(self):
        out = np.zeros(sum(k * s.N for s, k in zip(self.systems, self.nstates)))
        _bcheck(_lib.ts_batch_observe(self.b, TS_SZ, out.ctypes.data), self.b)
        res, o = [], 0
        for s, k in zip(self.systems, self.nstates):
            res.append(out[o:o + k * s.N].reshape(k, s.N))
            o += k * s.N
        return res

    def launches(self):
        return int(_lib.ts_batch_kernel_launches(self.b))

    def close(self):
        if getattr(self, "b", None):
            _lib.ts_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- convenience wrapper

class Context:
    """One state vector of N spins on the current CUDA device, evolved by TS4.

    Device memory comes from torch: the state (and, lazily, the echo reference
    and the energy scratch) are torch tensors bound to the library.
    """

    def __init__(self, N, Jx, Jy, Jz, h=None, prec="c64", hx=None, hy=None, stream=None, device=None):
        import torch
        self.torch = torch
        self.N = int(N)
        self.prec = TS_C64 if prec in ("c64", TS_C64) else TS_C128
        self.dtype = torch.complex64 if self.prec == TS_C64 else torch.complex128
        self.device = torch.device(device or "cuda")
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.ctx = ts_create(self.N, Jx, Jy, Jz, h, self.prec, ctypes.c_void_p(self.stream.cuda_stream))
            if hx is not None or hy is not None:
                ts_set_transverse_fields(self.ctx, hx, hy, self.N)
            self.psi = torch.empty(1 << self.N, dtype=self.dtype, device=self.device)
        self.ref = None        # echo reference, allocated on first use
        self.scratch = None    # energy work buffer, allocated on first use
        self.nbytes = self.psi.numel() * self.psi.element_size()
        ts_bind_buffers(self.ctx, self.psi.data_ptr(), None, None, self.nbytes)

    def _aux(self, name):
        if getattr(self, name) is None:
            t = self.torch.empty_like(self.psi)
            setattr(self, name, t)
            ts_bind_buffers(self.ctx, self.psi.data_ptr(), t.data_ptr() if name == "ref" else None,
                            t.data_ptr() if name == "scratch" else None, self.nbytes)

    @classmethod
    def from_system(cls, sys, prec="c64", **kw):
        return cls(sys.N, sys.Jx, sys.Jy, sys.Jz, sys.hz, prec=prec, hx=sys.hx, hy=sys.hy, **kw)

    def set_state(self, amps):
        """amps: a numpy array (host) or a torch tensor on the device, 2^N amplitudes."""
        torch = self.torch
        if isinstance(amps, torch.Tensor) and amps.is_cuda:
            a = amps.to(self.dtype).contiguous()
            ts_set_state(self.ctx, a.data_ptr(), 1)
            self._keep = a
        else:
            npdt = np.complex64 if self.prec == TS_C64 else np.complex128
            a = np.ascontiguousarray(np.asarray(amps), dtype=npdt)
            if a.shape != (1 << self.N,):
                raise ValueError("state must hold 2^N amplitudes")
            ts_set_state(self.ctx, a.ctypes.data, 0)

    def set_state_host_ptr(self, ptr):
        ts_set_state(self.ctx, ptr, 0)

    def set_basis_state(self, s):
        ts_set_basis_state(self.ctx, s)

    def save_reference(self):
        self._aux("ref")
        ts_save_reference(self.ctx)

    def step(self, tau, nsteps=1):
        ts_step(self.ctx, tau, nsteps)

    def set_chaining(self, enable=True):
        """Hold back the final pass of each step call until the next one (library side)."""
        _check(_lib.ts_set_chaining(self.ctx, 1 if enable else 0), self.ctx)

    def flush(self):
        """Run a held-back final pass, so that the bound state buffer holds the state."""
        _check(_lib.ts_flush(self.ctx), self.ctx)

    def step_order(self, order, tau, nsteps=1):
        ts_step_order(self.ctx, order, tau, nsteps)

    def norm(self):
        return float(ts_observe(self.ctx, TS_NORM, 1)[0])

    def energy(self):
        self._aux("scratch")
        return float(ts_observe(self.ctx, TS_ENERGY, 1)[0])

    def sz(self):
        return ts_observe(self.ctx, TS_SZ, self.N)

    def magnetization(self, axis="z"):
        """<S^axis_j> for j = 1..N (axis x or y uses a rotated scratch copy)."""
        if axis == "z":
            return self.sz()
        self._aux("scratch")
        return ts_observe(self.ctx, {"x": TS_SX, "y": TS_SY}[axis], self.N)

    def correlations(self, axis="z"):
        """<S^axis_i S^axis_j> as an N x N array (axis x or y uses a rotated scratch copy)."""
        if axis != "z":
            self._aux("scratch")
        what = {"z": TS_SZSZ, "x": TS_SXSX, "y": TS_SYSY}[axis]
        return ts_observe(self.ctx, what, self.N * self.N).reshape(self.N, self.N)

    def echo(self):
        return float(ts_observe(self.ctx, TS_ECHO, 1)[0])

    def overlap(self):
        o = ts_observe(self.ctx, TS_OVERLAP, 2)
        return complex(o[0], o[1])

    def get_state(self):
        """The state as a numpy array on the host."""
        npdt = np.complex64 if self.prec == TS_C64 else np.complex128
        out = np.empty(1 << self.N, dtype=npdt)
        ts_get_state(self.ctx, out.ctypes.data, 0)
        return out

    def set_schedule(self, kernel=TS_KERNEL_FUSED, tile_bits=0, coalesce_bits=0):
        ts_set_schedule(self.ctx, kernel, tile_bits, coalesce_bits)

    def schedule(self):
        return ts_get_schedule(self.ctx)

    def set_phase_tables(self, enable=True):
        """The paper's 2^N energy tables for the basic kernel (A/B comparison)."""
        _check(_lib.ts_set_phase_tables(self.ctx, 1 if enable else 0), self.ctx)

    def autotune(self, tau, reps=2, cache_path=None):
        """Brute-force search of the tile shape (library side); returns the best ms per step."""
        self._aux("scratch")
        ms = ctypes.c_double(0.0)
        _check(_lib.ts_autotune(self.ctx, float(tau), int(reps),
                                cache_path.encode() if cache_path else None, ctypes.byref(ms)), self.ctx)
        return ms.value

    def step_bound(self):
        return ts_step_bound(self.ctx)

    def launches(self):
        return ts_kernel_launches(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            ts_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
