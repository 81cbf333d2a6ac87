"""The fused-pass plan (host logic, no GPU): bit groups and the order of passes, rotations
and slots (Secs. 3.3-3.4 on top of the Sec. 2 decomposition), checked by replaying it.

Replay rules (what makes the plan compute the decomposition):
  * the groups partition the N spins: group 0 is the TB lowest spins, the others are
    contiguous windows above it, and a window tile keeps TB - h of the lowest spins;
  * every rotation of a pass covers exactly its group's spins, each once;
  * slot k may run only after every group has finished layer k (k rotations each), and
    a group may start layer k + 1 only after slot k ran;
  * all layers and all slots run, the last slot after the last layer.
"""
import pytest

LAYERS_PER_STEP = {1: 3, 2: 4, 4: 20}


@pytest.fixture(scope="module")
def ts4():
    from paper_1305_0036_gb300 import build
    build.build()
    from paper_1305_0036_gb300 import ts4 as m
    return m


def _mask(lo, n):
    return ((1 << n) - 1) << lo


def replay(groups, passes, layers, state=None, slot_base=0, complete=True):
    """Replays one call's passes; state carries (layers done per group, last slot) across
    chained calls, whose slot k is global slot slot_base + k."""
    g = len(groups)
    gmask = [_mask(gr["w"], gr["h"]) for gr in groups]
    if state is None:
        state = {"done": [0] * g, "last_slot": -1}
    done = state["done"]     # layers finished per group
    for p in passes:
        gi = p["group"]
        assert p["dup"] == 0
        for side in ("rot_before", "rot_after"):
            m = p[side]
            if side == "rot_after" and p["slot"] < 0:
                assert m == 0
                continue
            if side == "rot_after":
                # the slot sits between the two sides
                k = slot_base + p["slot"]
                assert k == state["last_slot"] + 1, (k, state["last_slot"])
                assert all(d == k for d in done), (k, done)
                state["last_slot"] = k
            if m == 0:
                continue
            assert m == gmask[gi], (side, hex(m), hex(gmask[gi]))
            assert state["last_slot"] == done[gi], "rotation before the slot of its layer"
            done[gi] += 1
    if complete:
        assert done == [slot_base + layers] * g
        assert state["last_slot"] == slot_base + layers
    return state


@pytest.mark.parametrize("N,tb,cb", [(12, 12, 3), (14, 12, 2), (17, 12, 3), (20, 12, 3), (23, 12, 2),
                                     (23, 12, 7), (25, 12, 3), (28, 12, 3), (28, 12, 7), (28, 13, 3),
                                     (28, 14, 4), (32, 12, 3), (33, 12, 3), (34, 12, 3)])
@pytest.mark.parametrize("order", [4, 2, 1])
def test_plan_replays_to_the_full_decomposition(ts4, N, tb, cb, order):
    nsteps = 2
    groups, passes = ts4.ts_plan(N, ts4.TS_C64, tb, cb, order, nsteps)
    # groups partition the spins
    assert groups[0] == dict(c=0, w=0, h=tb)
    w = tb
    for gr in groups[1:]:
        assert gr["w"] == w and 1 <= gr["h"] <= tb - cb and gr["c"] + gr["h"] == tb
        w += gr["h"]
    assert w == N
    g = len(groups)
    layers = LAYERS_PER_STEP[order] * nsteps
    assert len(passes) == (layers + 1 if g == 1 else 1 + layers * (g - 1))
    replay(groups, passes, layers)


def test_largest_group_never_carries_a_slot_with_three_or_more_groups(ts4):
    groups, passes = ts4.ts_plan(28, ts4.TS_C64, 12, 3, 4, 3)
    assert len(groups) == 3
    assert all(p["slot"] < 0 for p in passes if p["group"] == 0)
    # and every other pass with a slot rotates its group twice (the zigzag ends), except
    # the first and the last pass of the run
    for p in passes[1:-1]:
        if p["slot"] >= 0:
            assert p["rot_before"] and p["rot_after"]


def test_complex128_plan_uses_four_register_bits(ts4):
    groups, passes = ts4.ts_plan(23, ts4.TS_C128, 11, 2, 4, 1)
    replay(groups, passes, 20)
    assert len(groups) == 3


def test_a_broken_plan_fails_the_replay(ts4):
    """The replay is not vacuous: a pass dropped, two swapped, or a slot moved all fail."""
    groups, passes = ts4.ts_plan(25, ts4.TS_C64, 12, 3, 4, 1)
    with pytest.raises(AssertionError):
        replay(groups, passes[:-2] + passes[-1:], 20)
    swapped = list(passes)
    swapped[3], swapped[4] = swapped[4], swapped[3]
    with pytest.raises(AssertionError):
        replay(groups, swapped, 20)
    moved = [dict(p) for p in passes]
    k = next(i for i, p in enumerate(moved) if p["slot"] == 5)
    moved[k]["slot"] = 6
    with pytest.raises(AssertionError):
        replay(groups, moved, 20)


def test_plan_rejects_bad_arguments(ts4):
    for args in [(11, ts4.TS_C64, 12, 3, 4, 1),     # N below the tile
                 (35, ts4.TS_C64, 12, 3, 4, 1),     # N above 34
                 (20, ts4.TS_C64, 15, 3, 4, 1),     # tile not provided
                 (20, ts4.TS_C64, 12, 8, 4, 1),     # coalescing wider than tile - register bits
                 (20, ts4.TS_C64, 12, 3, 3, 1),     # order 3
                 (20, ts4.TS_C64, 12, 3, 4, 0)]:    # no steps
        with pytest.raises(ts4.TS4Error):
            ts4.ts_plan(*args)


@pytest.mark.parametrize("N,tb,cb", [(17, 12, 3), (23, 12, 2), (23, 12, 7), (28, 12, 3), (28, 12, 7), (33, 12, 3)])
@pytest.mark.parametrize("order", [4, 2])
def test_chained_calls_replay_as_one_run(ts4, N, tb, cb, order):
    """Calls with chaining (ts_set_chaining): the first holds back its final pass, the middle
    ones continue and hold back, the last continues and completes.  Replayed in sequence
    with global slot numbers, they must form the full decomposition of all their layers."""
    steps = [1, 2, 1]
    chains = [2, 3, 1]
    state, base, groups = None, 0, None
    for n, ch in zip(steps, chains):
        groups, passes = ts4.ts_plan(N, ts4.TS_C64, tb, cb, order, n, chain=ch)
        layers = LAYERS_PER_STEP[order] * n
        last = ch == 1
        state = replay(groups, passes, layers, state, slot_base=base, complete=last)
        if not last:
            # exactly the final pass is missing: one group one layer short, its last slot pending
            short = [i for i, d in enumerate(state["done"]) if d == base + layers - 1]
            assert len(short) == 1 and short[0] == (1 if len(groups) >= 3 else 0)
            assert state["last_slot"] == base + layers - 1
        base += layers
    assert state["done"] == [base] * len(groups)


def test_chaining_needs_two_groups(ts4):
    with pytest.raises(ts4.TS4Error):
        ts4.ts_plan(12, ts4.TS_C64, 12, 3, 4, 1, chain=2)


def test_default_coalescing_width(ts4):
    """Defaults: 3 coalescing spins for complex64, one fewer where that saves a bit group."""
    def widths(N):
        groups, _ = ts4.ts_plan(N, ts4.TS_C64, 12, 0, 4, 1)
        return [12 - gr["h"] for gr in groups[1:]]
    assert widths(22) == [2]                 # 2 spins: one window of 10 instead of two
    assert widths(28) == [4, 4]              # 2 windows either way: keep 3 (windows of 8)
    assert widths(20) == [4]                 # one window of 8 with 3 spins already
    groups, _ = ts4.ts_plan(23, ts4.TS_C128, 12, 0, 4, 1)
    assert len(groups) == 3                  # complex128 never goes below 2 spins
