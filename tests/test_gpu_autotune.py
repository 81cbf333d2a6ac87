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


def test_batch_autotune_picks_a_shape_keeps_the_states_and_caches(tmp_path):
    """The ensemble autotuner (config 4's autotuned tile): trials on the ensemble's own
    buffers, states restored afterwards, the winner cached under the ensemble's key."""
    from paper_1305_0036_gb300 import build
    build.build()
    from paper_1305_0036_gb300 import ts4
    systems = [W.xyz_chain(n, 1.0, 0.8, 0.5, seed=60 + n) for n in (14, 16)]
    nst = [3, 2]
    states = [np.stack([W.haar_state(s.N, 70 + 10 * i + j, np.complex64) for j in range(k)])
              for i, (s, k) in enumerate(zip(systems, nst))]
    b = ts4.Batch(systems, nst, prec="c64")
    for i, a in enumerate(states):
        b.set_states(i, a)
    cache = str(tmp_path / "tune.txt")
    ms = b.autotune(0.02, reps=1, cache_path=cache)
    assert ms > 0
    sch = b.schedule()
    assert sch["tile_bits"] in (12, 13, 14) and 1 <= sch["coalesce_bits"] <= 4
    for i, a in enumerate(states):
        np.testing.assert_array_equal(b.get_states(i), a)     # restored after the trials
    line = open(cache).read().split()
    assert int(line[1]) < 0 and int(line[3]) == sch["tile_bits"] and int(line[4]) == sch["coalesce_bits"]
    b2 = ts4.Batch(systems, nst, prec="c64")
    for i, a in enumerate(states):
        b2.set_states(i, a)
    assert b2.autotune(0.02, reps=1, cache_path=cache) == -1.0   # taken from the cache
    assert b2.schedule() == sch
    # the tuned ensemble still evolves correctly: one step against single-state runs
    b2.step(0.02, 1)
    c = ts4.Context.from_system(systems[1], prec="c64")
    c.set_state(states[1][1])
    c.step(0.02, 1)
    assert np.linalg.norm(b2.get_states(1)[1].astype(np.complex128) - c.get_state()) <= 1e-5
    c.close()
    b.close()
    b2.close()
