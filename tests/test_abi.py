"""The C ABI: the library loads, exports every entry point of include/ts4.h,
rejects bad arguments before touching the GPU, and maps tiles the way the
paper's worked examples do (Secs. 3.3-3.4).  No GPU compute here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ts4.h")
GOLDEN = os.path.join(ROOT, "tests", "golden")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^TS4_API[^(]*?\b(ts_\w+)\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1305_0036_gb300 import build
    build.build()
    from paper_1305_0036_gb300 import ts4
    return ts4


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("ts_create", "ts_set_state", "ts_step", "ts_observe", "ts_get_state", "ts_destroy",
              "ts_save_reference", "ts_set_basis_state", "ts_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(lib.LIB_PATH)
    for name in _declared():
        assert hasattr(raw, name), name
    assert set(_declared()) == set(lib.SIGNATURES), "binding and header disagree"


def test_version(lib):
    assert "sm_103a" in lib.ts_version()


def test_invalid_arguments_rejected_before_any_cuda_call(lib):
    import numpy as np
    J = np.zeros((4, 4))
    out = ctypes.c_void_p()
    for N in (0, 35, -3):
        st = lib._lib.ts_create(ctypes.byref(out), N, J.ctypes.data, J.ctypes.data, J.ctypes.data, None, 0, None)
        assert st == lib.TS_ERR_ARG
    assert lib._lib.ts_create(ctypes.byref(out), 4, None, J.ctypes.data, J.ctypes.data, None, 0, None) == lib.TS_ERR_ARG
    assert lib._lib.ts_create(None, 4, J.ctypes.data, J.ctypes.data, J.ctypes.data, None, 0, None) == lib.TS_ERR_ARG
    bad = J.copy()
    bad[0, 1] = float("nan")
    with pytest.raises(lib.TS4Error) as e:
        lib.ts_create(4, bad, J, J)
    assert e.value.status == lib.TS_ERR_ARG
    with pytest.raises(lib.TS4Error) as e:
        lib.ts_create(4, J, J, J, h=[0, 0, float("inf"), 0])
    assert e.value.status == lib.TS_ERR_ARG
    with pytest.raises(lib.TS4Error):
        lib.ts_create(4, J, J, J, prec=7)


def test_null_context_calls_are_rejected(lib):
    for name, args in (("ts_step", (0.1, 1)), ("ts_save_reference", ()), ("ts_set_basis_state", (0,))):
        assert getattr(lib._lib, name)(None, *args) == lib.TS_ERR_ARG
    assert lib._lib.ts_destroy(None) == lib.TS_OK
    assert lib.ts_last_error(None) == ""


def test_tile_mapping_matches_block_tables_sec34(lib):
    """Blocks rotating spins {1,2} hold 4 consecutive states; blocks rotating {3,4} hold
    states at stride 4 (the two tables of Sec. 3.4 for N = 4)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "block_tables_N4.txt")) if l.strip() and l[0] != "#"]
    for r in rows:
        spins = r[0].split("=")[1]
        block = int(r[1].split("=")[1])
        states = [int(x) for x in r[2:]]
        if spins == "1,2":      # tile = bits [0,2): c = 0, window w = 0, h = 2
            got = [lib.ts_tile_global_index(4, 0, 0, 2, block, e) for e in range(4)]
        else:                   # tile = bits [2,4): c = 0, w = 2, h = 2
            got = [lib.ts_tile_global_index(4, 0, 2, 2, block, e) for e in range(4)]
        assert got == states, (r, got)


def test_tile_mapping_closed_set_sec33(lib):
    """F = {spin 1, spin 3} fixed to (down, up); the block's states are closed under
    flipping spins 2 and 4.  Tile = bit 1 (c=0,w=1,h=1) would fix bits 0, 2, 3; instead
    take the window [1, 4) and check the members with bit 2 = 1 and bit 0 = 0."""
    lines = [l.strip() for l in open(os.path.join(GOLDEN, "closed_set_N4_F13.txt")) if l.strip() and l[0] != "#"]
    expected = sorted(int(x, 2) for x in lines)
    # block f fixes bit 0 (spin 1) = 0; the window holds bits 1..3; keep members with bit 2 = 1
    members = [lib.ts_tile_global_index(4, 0, 1, 3, 0, e) for e in range(8)]
    got = sorted(m for m in members if (m >> 2) & 1)
    assert got == expected


def test_tile_mapping_is_a_partition(lib):
    """For every group shape, the blocks' tiles cover each basis index exactly once."""
    N = 9
    for (c, w, h) in ((0, 0, 5), (2, 5, 3), (3, 4, 5), (1, 8, 1)):
        seen = []
        for f in range(1 << (N - c - h)):
            seen += [lib.ts_tile_global_index(N, c, w, h, f, e) for e in range(1 << (c + h))]
        assert sorted(seen) == list(range(1 << N))


def test_step_bound_host_is_eq4(lib):
    """Eq. 4: [max_{j,k} (sum_a (h^a_j/2)^2 + sum_a (J^a_jk/4)^2)^(1/2)]^-1, on closed forms."""
    import numpy as np
    J = np.zeros((2, 2))
    J[0, 1] = 1.0
    # one isotropic bond, no field: 3 (1/4)^2 = 3/16
    assert lib.ts_step_bound_host(2, J, J, J) == pytest.approx(4 / np.sqrt(3), rel=1e-15)
    # a z-field of 1 on spin 1 adds (1/2)^2 to that spin's terms: 3/16 + 4/16
    assert lib.ts_step_bound_host(2, J, J, J, hz=[1.0, 0.0]) == pytest.approx(4 / np.sqrt(7), rel=1e-15)
    # transverse fields count alike; the lower triangle is ignored
    Jl = J.T.copy()
    assert lib.ts_step_bound_host(2, J + Jl, J, J, hx=[0.0, 2.0]) == pytest.approx(1 / np.sqrt(1 + 3 / 16), rel=1e-15)
    # the dipolar chain: nearest neighbours J^z = 1, J^x = J^y = -1/2 give 6/64
    from paper_1305_0036_gb300 import workloads as W
    s = W.dipolar_chain(28)
    assert lib.ts_step_bound_host(28, s.Jx, s.Jy, s.Jz, hz=s.hz) == pytest.approx(8 / np.sqrt(6), rel=1e-15)
    # no Hamiltonian: no time scale
    Z = np.zeros((3, 3))
    assert lib.ts_step_bound_host(3, Z, Z, Z) == float("inf")
    assert lib._lib.ts_step_bound_host(0, Z.ctypes.data, Z.ctypes.data, Z.ctypes.data, None, None, None) == -1.0
    assert lib._lib.ts_step_bound_host(3, None, Z.ctypes.data, Z.ctypes.data, None, None, None) == -1.0
