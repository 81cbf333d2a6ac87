// Compiled pass shapes of complex128 12-bit tiles (16 amplitudes per thread, register chunks of
// 4 bits) for the fused pass of Secs. 3.3-3.4 (see ts4_shapes_c64.cu): slot passes of window
// groups of 6..8 spins and passes without a slot of the 12 lowest spins -- the passes of the
// default complex128 schedules at N = 23..28.
#include "ts4_tile.cuh"

namespace ts4 {

namespace {
using SlotWin6 = PassShape<0, Step<0, 0, 4, 0, 0, 0>, Step<1, 0, 2, 1, 0, 2>, Step<0, 0, 0, 0, 0, 4>>;
using SlotWin7 = PassShape<0, Step<0, 0, 4, 0, 0, 0>, Step<1, 0, 3, 1, 0, 3>, Step<0, 0, 0, 0, 0, 4>>;
using SlotWin8 = PassShape<0, Step<0, 0, 4, 0, 0, 0>, Step<1, 0, 4, 1, 0, 4>, Step<0, 0, 0, 0, 0, 4>>;
using RotLow12 = PassShape<1, Step<1, 0, 4, 0, 0, 0>, Step<0, 0, 4, 0, 0, 0>, Step<2, 0, 4, 0, 0, 0>>;
} // namespace

template <>
bool launch_shaped<double, 12, 4>(cudaStream_t st, void *psi, const TileArgs &a, const void *tabs, uint64_t nblk,
                                  cudaError_t *err)
{
    using R = double;
    return launch_if_shape<R, 12, 4, true, SlotWin8>(st, psi, a, tabs, nblk, err) ||
           launch_if_shape<R, 12, 4, false, RotLow12>(st, psi, a, tabs, nblk, err) ||
           launch_if_shape<R, 12, 4, true, SlotWin7>(st, psi, a, tabs, nblk, err) ||
           launch_if_shape<R, 12, 4, true, SlotWin6>(st, psi, a, tabs, nblk, err);
}

} // namespace ts4
