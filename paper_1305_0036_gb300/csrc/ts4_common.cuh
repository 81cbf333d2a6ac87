// Shared definitions of the CUDA TS4 library: complex arithmetic on float2 /
// double2, the diagonal "slot" descriptors, tile geometry, and the device
// copies of the Hamiltonian.
//
// Formulation used on the GPU (derived from Sec. 2, Eqs. 5, 9, 10):
// every rotation layer of a U2 -- X^dag, Y^dag X, X^dag Y, X, in time order --
// factors per spin as D_L W D_R, with W = [[1, 1], [1, -1]] (basis order
// down, up) and diagonal D_L, D_R.  Products of the per-spin diagonals over all
// spins depend only on popcount(s), so they fold into the diagonal phases that
// sit between consecutive layers.  One U2(t) is then, in time order,
//   (-i)^pc P_z(t/2) . W . 2^{-N/2} i^pc P_y(t/2) . W . 2^{-N/2} P_x(t)
//   . W . 2^{-N/2} (-i)^pc P_y(t/2) . W . 2^{-N/2} i^pc P_z(t/2)
// where P_a(t) = exp(-i t E_a(s)), E_a(s) = sum_{i<j} J^a_ij s_i s_j / 4
// + sum_i h^a_i s_i / 2 (s = +-1 from the bits), pc = popcount(s), and W acts
// on every spin.  (Two constant phases e^{-+i pi N / 4} cancel between the
// P_x and the second P_y slot.)  Consecutive U2's merge their P_z slots.
// So the GPU only ever applies unnormalised Walsh-Hadamard butterflies
// (a + b, a - b) and diagonal slots.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ts4 {

template <typename R> struct CT;
template <> struct CT<float> { using T = float2; };
template <> struct CT<double> { using T = double2; };

__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

// a * i^k, exact (swap and sign changes only), branch-free: k is often different
// in the lanes of a warp
template <typename C> __host__ __device__ __forceinline__ C cmul_ipow(C a, int k)
{
    const bool sw = (k & 1) != 0, ng = (k & 2) != 0;
    const auto x = sw ? -a.y : a.x;   // times i: (x, y) -> (-y, x)
    const auto y = sw ? a.x : a.y;
    C r;
    r.x = ng ? -x : x;                // times -1
    r.y = ng ? -y : y;
    return r;
}

// Unnormalised butterfly W on a pair (x0 = bit 0, x1 = bit 1): (x0 + x1, x0 - x1),
// with the packed FP32x2 instructions (one per complex add; a - b as a + b * (-1),
// which rounds once like the plain subtraction).
__device__ __forceinline__ void bfly(float2 &a, float2 &b)
{
    const float2 s = __fadd2_rn(a, b);
    const float2 d = __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
    a = s;
    b = d;
}
__device__ __forceinline__ void bfly(double2 &a, double2 &b)
{
    double2 s = cadd(a, b), d = csub(a, b);
    a = s;
    b = d;
}

// Knuth's two-sum: s + err = a + b exactly.  Written with the _rn intrinsics, which the
// compiler never fuses into multiply-adds, so the transform stays error-free.
__device__ __forceinline__ float2 two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return make_float2(s, err);
}

// e^{-i pi x}: angles on the device are carried in half-turns (units of pi),
// already reduced in FP64, so CUDA's sincospi needs no large-argument path.
__device__ __forceinline__ float2 cexpm_pi(float x)
{
    float s, c;
    sincospif(x, &s, &c);
    return make_float2(c, -s);
}
__device__ __forceinline__ double2 cexpm_pi(double x)
{
    double s, c;
    sincospi(x, &s, &c);
    return make_double2(c, -s);
}

// theta / pi reduced to [-1, 1] (i.e. theta mod 2 pi, in half-turns), in FP64
__host__ __device__ __forceinline__ double halfturns_2pi(double th)
{
    const double inv_pi = 0.31830988618379067153776752674503;
    const double x = th * inv_pi;
    return x - 2.0 * rint(0.5 * x);
}

// One diagonal factor between two Walsh-Hadamard layers:
//   psi_s <- mag 2^{-scale_exp} * i^{pcq * popcount(s)} * exp(-i (t E_alpha(s) + th0)) * psi_s
struct Slot {
    double t;       // time multiplying E_alpha (0: no Hamiltonian part)
    double th0;     // constant angle (global phase left over by a layer factorisation)
    double mag;     // extra magnitude: 1, or 2^{-1/2} when N * layers is odd
    int alpha;      // 0 = x, 1 = y, 2 = z couplings / fields
    int pcq;        // 0..3
    int scale_exp;  // exact power-of-two scale
    int pad;
    double scale;   // mag 2^{-scale_exp} (host-computed: no FP64 arithmetic in the kernels)
    float scale_f;  // the same, rounded to FP32
    float srel;     // scale / scale_f - 1, the rounding of scale_f (0 unless mag = sqrt 1/2)
};

// Device copies of the Hamiltonian, FP64:
//   Jq[a*N*N + i*N + j] = J^a_{min(i,j), max(i,j)} / 4 for i != j, 0 on the diagonal (symmetric)
//   hh[a*N + i]         = h^a_i / 2
struct HamDev {
    const double *Jq;
    const double *hh;
    int N;
};

// A tile is the global bits [0, c) and [w, w + h); local bit order: window first.
struct TileGeom {
    int c, w, h;
};

__host__ __device__ __forceinline__ uint64_t tile_global_index(int c, int w, int h, uint64_t f, uint64_t e)
{
    const uint64_t win = e & ((UINT64_C(1) << h) - 1);
    const uint64_t low = e >> h;                                   // c bits
    const int nf_lo = w - c;                                       // fixed bits between the runs
    const uint64_t f_lo = f & ((UINT64_C(1) << nf_lo) - 1);
    const uint64_t f_hi = f >> nf_lo;
    return low | (f_lo << c) | (win << w) | (f_hi << (w + h));
}

__host__ __device__ __forceinline__ bool in_tile(int bit, int c, int w, int h)
{
    return bit < c || (bit >= w && bit < w + h);
}

} // namespace ts4
