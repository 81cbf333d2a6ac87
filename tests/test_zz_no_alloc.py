"""The allocation-free reduction entry point (ts_reduce_sz_static).

It serves callers that cannot allocate device memory where they need the norm
and <S^z_j> (hosts whose device memory is handed out by their own allocator,
plug-ins that must not grow the device footprint, loops that must not allocate
once started): the caller passes a device state and a device output buffer,
and the library's only scratch is a fixed static device array.  The test calls
it through the C ABI on two calls in a row (the second reuses the static array
left by the first) and checks both against the FP64 oracle's norm and <S^z>
of the same state, downloaded and converted exactly to complex128, and against
ts_observe.  It lives in a file that pytest collects last, so that a run that
stops at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1305_0036_gb300 import workloads as W

pytestmark = pytest.mark.gpu


# tolerances: complex128 sums in FP64 (order 2^N u_64 of the total at worst); complex64 sums
# exact squares of the FP32 components in double-float per thread, then FP64 (order 1e-11)
@pytest.mark.parametrize("prec,N,tol", [("c64", 18, 1e-11), ("c128", 15, 1e-13), ("c64", 9, 1e-11),
                                        ("c64", 24, 1e-11)])
def test_static_reduction_matches_oracle_twice(prec, N, tol):
    import torch
    from paper_1305_0036_gb300 import build
    build.build()
    from paper_1305_0036_gb300 import ts4

    torch.cuda.set_device(0)
    s = W.random_system(N, 500 + N)
    ctx = ts4.Context.from_system(s, prec=prec)
    ctx.set_state(W.haar_state(N, 600 + N))
    ctx.step(0.05, 1)
    psi = ctx.get_state().astype(np.complex128)
    ref_norm = oracle.norm(psi, N)
    ref_sz = oracle.sz(psi, N)
    out = torch.full((N + 1,), float("nan"), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(ctx.stream.cuda_stream)
    p = ts4.TS_C64 if prec == "c64" else ts4.TS_C128
    for call in range(2):
        out.fill_(float("nan"))
        ts4.ts_reduce_sz_static(ctx.psi.data_ptr(), N, p, out.data_ptr(), stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        print(f"\n{prec} N={N} call {call}: |dnorm| = {abs(got[0] - ref_norm):.2e}, "
              f"max|dSz| = {np.abs(got[1:] - ref_sz).max():.2e}")
        assert abs(got[0] - ref_norm) <= tol, (call, got[0], ref_norm)
        np.testing.assert_allclose(got[1:], ref_sz, rtol=0, atol=tol)
    # the context's own reductions give the same numbers
    assert abs(ctx.norm() - ref_norm) <= tol
    np.testing.assert_allclose(ctx.sz(), ref_sz, rtol=0, atol=tol)
    ctx.close()


def test_static_reduction_rejects_bad_arguments():
    from paper_1305_0036_gb300 import build
    build.build()
    from paper_1305_0036_gb300 import ts4
    with pytest.raises(ts4.TS4Error) as e:
        ts4.ts_reduce_sz_static(None, 10, ts4.TS_C64, None)
    assert e.value.status == ts4.TS_ERR_ARG
    with pytest.raises(ts4.TS4Error) as e:
        ts4.ts_reduce_sz_static(1 << 20, 35, ts4.TS_C64, 1 << 20)
    assert e.value.status == ts4.TS_ERR_ARG
