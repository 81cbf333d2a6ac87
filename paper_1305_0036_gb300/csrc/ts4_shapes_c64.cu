// Compiled pass shapes of complex64 12-bit tiles (32 amplitudes per thread, register chunks of
// 5 bits) for the fused pass of Secs. 3.3-3.4.  A pass of one of these shapes runs a build of
// k_tile whose step list is a template list (see PassShape in ts4_tile.cuh): same arithmetic in
// the same order as the run-time step loop, without its branches.  The shapes are those of the
// passes that make up long runs of the default schedules:
//   slot passes (rotate the group, slot, rotate again) of window groups of 4..10 spins (their
//   tiles keep the lowest spins) and of the group of the 12 lowest spins (two bit groups);
//   passes without a slot of the 12 lowest spins (the middle of three bit groups) and of
//   windows of 7 and 8 spins (four bit groups, N = 33, 34).
// The slot-factor form of the usual small angles and the 32-bit element offsets of N <= 32 are
// compiled in as well (MODE, NARROW of k_tile); passes with other values take the builds that
// read them at run time.
#include "ts4_tile.cuh"

namespace ts4 {

namespace {
using SlotWin4 = PassShape<0, Step<0, 0, 4, 1, 0, 4>>;
using SlotWin5 = PassShape<0, Step<0, 0, 5, 1, 0, 5>>;
using SlotWin6 = PassShape<0, Step<0, 0, 5, 0, 0, 0>, Step<1, 0, 1, 1, 0, 1>, Step<0, 0, 0, 0, 0, 5>>;
using SlotWin7 = PassShape<0, Step<0, 0, 5, 0, 0, 0>, Step<1, 0, 2, 1, 0, 2>, Step<0, 0, 0, 0, 0, 5>>;
using SlotWin8 = PassShape<0, Step<0, 0, 5, 0, 0, 0>, Step<1, 0, 3, 1, 0, 3>, Step<0, 0, 0, 0, 0, 5>>;
using SlotWin9 = PassShape<0, Step<0, 0, 5, 0, 0, 0>, Step<1, 0, 4, 1, 0, 4>, Step<0, 0, 0, 0, 0, 5>>;
using SlotWin10 = PassShape<0, Step<0, 0, 5, 0, 0, 0>, Step<1, 0, 5, 1, 0, 5>, Step<0, 0, 0, 0, 0, 5>>;
using SlotLow12 = PassShape<1, Step<1, 0, 5, 0, 0, 0>, Step<0, 0, 5, 0, 0, 0>, Step<2, 3, 5, 1, 3, 5>,
                            Step<0, 0, 0, 0, 0, 5>, Step<1, 0, 0, 0, 0, 5>>;
using RotLow12 = PassShape<1, Step<1, 0, 5, 0, 0, 0>, Step<0, 0, 5, 0, 0, 0>, Step<2, 3, 5, 0, 0, 0>>;
using RotWin7 = PassShape<0, Step<0, 0, 5, 0, 0, 0>, Step<1, 0, 2, 0, 0, 0>>;
using RotWin8 = PassShape<0, Step<0, 0, 5, 0, 0, 0>, Step<1, 0, 3, 0, 0, 0>>;
} // namespace

template <>
bool launch_shaped<float, 12, 5>(cudaStream_t st, void *psi, const TileArgs &a, const void *tabs, uint64_t nblk,
                                 cudaError_t *err)
{
    using R = float;
    // slot passes: the short-series factor (|y| <= 0.05, the usual case) compiled in, then any
    // factor form read at run time
    return launch_if_shape<R, 12, 5, true, SlotWin8, 0>(st, psi, a, tabs, nblk, err) ||
           launch_if_shape<R, 12, 5, false, RotLow12>(st, psi, a, tabs, nblk, err) ||
           launch_if_shape<R, 12, 5, true, SlotWin7, 0>(st, psi, a, tabs, nblk, err) ||
           launch_if_shape<R, 12, 5, true, SlotWin6, 0>(st, psi, a, tabs, nblk, err) ||
           launch_if_shape<R, 12, 5, true, SlotWin5, 0>(st, psi, a, tabs, nblk, err) ||
           launch_if_shape<R, 12, 5, true, SlotWin9, 0>(st, psi, a, tabs, nblk, err) ||
           launch_if_shape<R, 12, 5, true, SlotWin10, 0>(st, psi, a, tabs, nblk, err) ||
           launch_if_shape<R, 12, 5, true, SlotWin4, 0>(st, psi, a, tabs, nblk, err) ||
           launch_if_shape<R, 12, 5, true, SlotLow12, 0>(st, psi, a, tabs, nblk, err) ||
           launch_if_shape<R, 12, 5, true, SlotWin8>(st, psi, a, tabs, nblk, err) ||
           launch_if_shape<R, 12, 5, true, SlotWin7>(st, psi, a, tabs, nblk, err) ||
           launch_if_shape<R, 12, 5, true, SlotWin6>(st, psi, a, tabs, nblk, err) ||
           launch_if_shape<R, 12, 5, true, SlotWin5>(st, psi, a, tabs, nblk, err) ||
           launch_if_shape<R, 12, 5, true, SlotWin9>(st, psi, a, tabs, nblk, err) ||
           launch_if_shape<R, 12, 5, true, SlotWin10>(st, psi, a, tabs, nblk, err) ||
           launch_if_shape<R, 12, 5, true, SlotWin4>(st, psi, a, tabs, nblk, err) ||
           launch_if_shape<R, 12, 5, true, SlotLow12>(st, psi, a, tabs, nblk, err) ||
           // N = 33, 34 (64-bit offsets): the slot passes of their 7- and 8-spin windows
           launch_if_shape<R, 12, 5, true, SlotWin7, 0, 0>(st, psi, a, tabs, nblk, err) ||
           launch_if_shape<R, 12, 5, true, SlotWin8, 0, 0>(st, psi, a, tabs, nblk, err) ||
           launch_if_shape<R, 12, 5, true, SlotWin7, -1, 0>(st, psi, a, tabs, nblk, err) ||
           launch_if_shape<R, 12, 5, true, SlotWin8, -1, 0>(st, psi, a, tabs, nblk, err) ||
           // four bit groups (N = 33, 34): window passes without a slot, 32- or 64-bit offsets
           launch_if_shape<R, 12, 5, false, RotWin7, -1, 1>(st, psi, a, tabs, nblk, err) ||
           launch_if_shape<R, 12, 5, false, RotWin8, -1, 1>(st, psi, a, tabs, nblk, err) ||
           launch_if_shape<R, 12, 5, false, RotWin7, -1, 0>(st, psi, a, tabs, nblk, err) ||
           launch_if_shape<R, 12, 5, false, RotWin8, -1, 0>(st, psi, a, tabs, nblk, err) ||
           launch_if_shape<R, 12, 5, false, RotLow12, -1, 0>(st, psi, a, tabs, nblk, err);
}

} // namespace ts4
