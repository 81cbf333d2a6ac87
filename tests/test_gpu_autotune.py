"""The autotuner (brute-force search of the tile shape, Sec. 3.4) and its cache file."""
import numpy as np
import pytest

from paper_1305_0036_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_autotune_picks_a_shape_keeps_the_state_and_caches(tmp_path):
    from paper_1305_0036_gb300 import build
    build.build()
    from paper_1305_0036_gb300 import ts4
    s = W.xyz_chain(20, 1.0, 0.8, 0.5, seed=5)
    ctx = ts4.Context.from_system(s, prec="c64")
    psi0 = W.haar_state(20, 6, np.complex64)
    ctx.set_state(psi0)
    cache = str(tmp_path / "tune.txt")
    ms = ctx.autotune(0.02, reps=1, cache_path=cache)
    assert ms > 0
    sch = ctx.schedule()
    assert sch["kernel"] == ts4.TS_KERNEL_FUSED and sch["tile_bits"] in (12, 13, 14)
    np.testing.assert_array_equal(ctx.get_state(), psi0)        # the search ran on a copy
    line = open(cache).read().split()
    assert int(line[1]) == 20 and int(line[3]) == sch["tile_bits"] and int(line[4]) == sch["coalesce_bits"]
    ctx2 = ts4.Context.from_system(s, prec="c64")
    ctx2.set_state(psi0)
    assert ctx2.autotune(0.02, reps=1, cache_path=cache) == -1.0   # taken from the cache
    assert ctx2.schedule() == sch
    ctx.close()
    ctx2.close()
