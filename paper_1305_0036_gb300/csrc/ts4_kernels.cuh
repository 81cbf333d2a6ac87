// CUDA kernels of the TS4 library (sm_103a).
//
//   k_wht_bit     one butterfly per thread on one spin over the whole state
//                 (the paper's "GPU-Basic" kernel, Sec. 3.3 first paragraph)
//   k_slot_basic  one diagonal slot per element, E(s) from bit tests (Sec. 3.1)
//   (the fused tile pass k_tile is in ts4_tile.cuh; this file holds the step
//   descriptors and per-pass tables it shares with the host)
//   k_sum_*       FP64-accumulating reductions for the observables (Sec. 4.2)
#pragma once

#include "ts4_common.cuh"

#include <utility>

namespace ts4 {

// ------------------------------------------------------------------ basic kernels

template <typename C>
__global__ void k_wht_bit(C *__restrict__ psi, uint64_t npairs, int b)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npairs; p += stride) {
        const uint64_t lo = p & ((UINT64_C(1) << b) - 1);
        const uint64_t n0 = ((p >> b) << (b + 1)) | lo;
        const uint64_t n1 = n0 | (UINT64_C(1) << b);
        C x0 = psi[n0], x1 = psi[n1];
        bfly(x0, x1);
        psi[n0] = x0;
        psi[n1] = x1;
    }
}

// E_alpha(s) = sum_{i<j} J^a_ij s_i s_j / 4 + sum_i h^a_i s_i / 2, from the FP64 tables.
__device__ __forceinline__ double energy_bits(uint64_t s, const double *__restrict__ Jq,
                                              const double *__restrict__ hh, int N)
{
    double e = 0.0;
    for (int i = 0; i < N; i++) {
        const double si = ((s >> i) & 1) ? 1.0 : -1.0;
        double r = hh[i];
        for (int j = i + 1; j < N; j++) {
            const double v = Jq[i * N + j];
            if (v != 0.0)
                r += v * (((s >> j) & 1) ? 1.0 : -1.0);
        }
        e += si * r;
    }
    return e;
}

template <typename R>
__global__ void k_slot_basic(typename CT<R>::T *__restrict__ psi, uint64_t dim, HamDev ham, Slot sl)
{
    using C = typename CT<R>::T;
    const double *Jq = ham.Jq + (size_t)sl.alpha * ham.N * ham.N;
    const double *hh = ham.hh + (size_t)sl.alpha * ham.N;
    const double scale = sl.scale;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < dim; s += stride) {
        double th = sl.th0;
        if (sl.t != 0.0)
            th += sl.t * energy_bits(s, Jq, hh, ham.N);
        // the factor is formed and applied in FP64 for both precisions: a complex64 factor
        // near 1 would be off the unit circle by a rounding error that depends only on the
        // energy level, which acts on the norm coherently over many steps
        double2 f = cexpm_pi(halfturns_2pi(th));
        f.x *= scale;
        f.y *= scale;
        f = cmul_ipow(f, sl.pcq * __popcll(s));
        const C x = psi[s];
        const double2 y = cmul(make_double2((double)x.x, (double)x.y), f);
        C r;
        r.x = (R)y.x;
        r.y = (R)y.y;
        psi[s] = r;
    }
}

// The paper's phase-table mode (Sec. 3.1): E_alpha(s) for every basis state, stored once
// (FP32, 4 bytes per state and alpha), so that a slot reads its angle instead of forming it
// from the bits.  Kept for the A/B comparison with the bit-test and the fused kernels.
static __global__ void k_energy_table(float *__restrict__ E, uint64_t dim, HamDev ham, int alpha)
{
    const double *Jq = ham.Jq + (size_t)alpha * ham.N * ham.N;
    const double *hh = ham.hh + (size_t)alpha * ham.N;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < dim; s += stride)
        E[s] = (float)energy_bits(s, Jq, hh, ham.N);
}

// One slot from the energy table: as k_slot_basic, with E_alpha(s) read from E.
template <typename R>
__global__ void k_slot_table(typename CT<R>::T *__restrict__ psi, const float *__restrict__ E, uint64_t dim, Slot sl)
{
    using C = typename CT<R>::T;
    const double scale = sl.scale;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < dim; s += stride) {
        const double th = sl.th0 + sl.t * (double)E[s];
        double2 f = cexpm_pi(halfturns_2pi(th));
        f.x *= scale;
        f.y *= scale;
        f = cmul_ipow(f, sl.pcq * __popcll(s));
        const C x = psi[s];
        const double2 y = cmul(make_double2((double)x.x, (double)x.y), f);
        C r;
        r.x = (R)y.x;
        r.y = (R)y.y;
        psi[s] = r;
    }
}

// ------------------------------------------------------------------ fused tile pass: descriptors

struct StepDesc {
    uint8_t k;          // chunk: register window starts at min(k * RB, TB - RB)
    uint8_t r0lo, r0hi; // register bits rotated before the slot
    uint8_t ph;         // 1: apply the pass's slot
    uint8_t r1lo, r1hi; // register bits rotated after the slot
    uint8_t pad0, pad1;
};

constexpr int kMaxSteps = 16;

// Per-(slot, tile geometry, register chunk) tables, built on the host in FP64 and
// rounded to R.  Angle unit: radians for complex64, half-turns for complex128.
// With A_lm = t J^a_{pos l, pos m} / 4 on the tile's local bits, W the register
// window of the layout that applies the slot, and s = +-1 the local bits of thread
// `tid`'s base index in that layout (its thread bits; the register bits are 0):
//   TP[tid]     = sum over thread-bit pairs m < l of A_ml s_m s_l
//   TC[b][tid]  = sum over thread bits m of A_{W+b, m} s_m        (b < RB)
//   QK[j]       c64:  (q(j), 0) with q(j) = sum over register-bit pairs l < m of A s_l s_m
//               c128: exp(-i q(j)) i^{pcq popcount(j)}
// The per-frame terms (the frame angle and the fields on the tile spins) are
// computed on the device once per schedule (k_frame_terms in ts4_tile.cuh).
template <typename R, int TB, int RB> struct PassTab {
    R TP[1 << (TB - RB)];
    R TC[RB][1 << (TB - RB)];
    typename CT<R>::T QK[1 << RB];
};

// Butterflies of register bit B on all 2^RB registers (register indices are template
// constants: the compiler must not fall back to run-time indexing of the array).
template <int B, typename C, int N, int... J>
__device__ __forceinline__ void wht_bit(C (&x)[N], std::integer_sequence<int, J...>)
{
    ((void)((J & (1 << B)) ? 0 : (bfly(x[J], x[J | (1 << B)]), 0)), ...);
}

// Register bits [LO, HI), straight-line.
template <int LO, int HI, typename C, int N> __device__ __forceinline__ void wht_fixed(C (&x)[N])
{
    if constexpr (LO < HI) {
        wht_bit<LO>(x, std::make_integer_sequence<int, N>{});
        wht_fixed<LO + 1, HI>(x);
    }
}
template <int RB, int LO, int HI, typename C, int N> __device__ __forceinline__ void wht_dispatch_hi(C (&x)[N], int hi)
{
    if constexpr (HI <= RB) {
        if (hi == HI)
            wht_fixed<LO, HI>(x);
        else
            wht_dispatch_hi<RB, LO, HI + 1>(x, hi);
    }
}
template <int RB, int LO, typename C, int N> __device__ __forceinline__ void wht_dispatch_lo(C (&x)[N], int lo, int hi)
{
    if constexpr (LO < RB) {
        if (lo == LO)
            wht_dispatch_hi<RB, LO, LO + 1>(x, hi);
        else
            wht_dispatch_lo<RB, LO + 1>(x, lo, hi);
    }
}

// Rotates register bits [lo, hi) (a run-time range, uniform across the block): one branch
// tree selects a straight-line block for the range.  Testing each bit at run time instead
// costs 20% more instructions per pass (measured).
template <int RB, typename C> __device__ __forceinline__ void wht_regs(C (&x)[1 << RB], int lo, int hi)
{
    wht_dispatch_lo<RB, 0>(x, lo, hi);
}

// ------------------------------------------------------------------ reductions (FP64)

template <typename T> __device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double norm2(float2 a) { return (double)a.x * a.x + (double)a.y * a.y; }
__device__ __forceinline__ double norm2(double2 a) { return a.x * a.x + a.y * a.y; }

// Block sums of several values; the results land in dst[0..K) (shared memory).
template <int K, typename T> __device__ void block_sum(T (&v)[K], T *__restrict__ dst)
{
    __shared__ T red[32][K];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; k++)
        v[k] = warp_sum(v[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; k++)
            red[wid][k] = v[k];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < K; k++) {
            T s = (lane < nw) ? red[lane][k] : T(0);
            s = warp_sum(s);
            if (lane == 0)
                dst[k] = s;
        }
    }
    __syncthreads();
}

// Per-thread sums over the 32 amplitudes p[j * stride], j < 32 (those with j < n):
// tot = sum |psi|^2 and low[b] = sum over j with bit b of j set (b < 5).
// complex64: squares and pairwise sums in FP32 (error <= 5 u of the thread's
// total), converted once to FP64; complex128: FP64 throughout.
template <typename C, typename A>
__device__ __forceinline__ void thread_sums32(const C *__restrict__ p, int stride, int n, A &tot, A (&low)[5])
{
    A q[32];
#pragma unroll
    for (int j = 0; j < 32; j++) {
        C a;
        a.x = 0;
        a.y = 0;
        if (j < n)
            a = p[(size_t)j * stride];
        q[j] = (A)a.x * (A)a.x + (A)a.y * (A)a.y;
    }
    // sum over the elements with bit b set = pairwise tree over the 16 such elements
#pragma unroll
    for (int b = 0; b < 5; b++) {
        A t[16];
        int k = 0;
#pragma unroll
        for (int j = 0; j < 32; j++)
            if ((j >> b) & 1)
                t[k++] = q[j];
#pragma unroll
        for (int w = 8; w >= 1; w >>= 1)
#pragma unroll
            for (int i = 0; i < w; i++)
                t[i] = t[i] + t[i + w];
        low[b] = t[0];
    }
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1)
#pragma unroll
        for (int i = 0; i < w; i++)
            q[i] = q[i] + q[i + w];
    tot = q[0];
}

template <typename C> struct AccOf;
template <> struct AccOf<float2> { using T = float; };
template <> struct AccOf<double2> { using T = double; };

// Per block: [0] = sum |psi|^2, [1..] = sum |psi_s|^2 bit_i(s) for i < N  (stride N+1).
// Each block iteration covers 2^13 consecutive amplitudes; its 14 sums are formed in
// the precision of the amplitudes (complex64: FP32 pairwise per thread and across
// the block, relative error ~1e-6 of that range's weight) and added to FP64 totals.
template <typename C>
__global__ void __launch_bounds__(256) k_sum_sz(const C *__restrict__ psi, int N, double *__restrict__ part)
{
    using A = typename AccOf<C>::T;
    constexpr int LB = 5;
    const uint64_t dim = UINT64_C(1) << N;
    __shared__ double acc_sh[64];
    for (int i = threadIdx.x; i < 64; i += blockDim.x)
        acc_sh[i] = 0.0;
    __syncthreads();
    const uint64_t per_block = (uint64_t)blockDim.x << LB;
    const int RBITS = 5 + 8;              // bits resolved inside one block range (blockDim = 256)
    // amplitude base + (j << 8) + tid: thread bits are global bits 0..7 (coalesced),
    // the 32 per-thread values are global bits 8..12
    for (uint64_t base = (uint64_t)blockIdx.x * per_block; base < dim; base += (uint64_t)gridDim.x * per_block) {
        A tot = A(0), low[LB] = {A(0), A(0), A(0), A(0), A(0)};
        const uint64_t s0 = base + threadIdx.x;
        if (s0 < dim) {
            const uint64_t rem = (dim - s0 + 255) >> 8;       // elements s0 + 256 j below dim
            const int n = rem < 32 ? (int)rem : 32;
            thread_sums32<C, A>(psi + s0, 256, n, tot, low);
        }
        A v[1 + 8 + LB];
        v[0] = tot;
#pragma unroll
        for (int b = 0; b < 8; b++)
            v[1 + b] = ((threadIdx.x >> b) & 1) ? tot : A(0);
#pragma unroll
        for (int b = 0; b < LB; b++)
            v[1 + 8 + b] = low[b];
        __shared__ A bs[1 + 8 + LB];
        block_sum<1 + 8 + LB>(v, bs);
        if (threadIdx.x == 0) {
            acc_sh[0] += (double)bs[0];
            for (int i = 0; i < N && i < RBITS; i++)
                acc_sh[1 + i] += (double)bs[1 + i];
            for (int i = RBITS; i < N; i++)
                if ((base >> i) & 1)
                    acc_sh[1 + i] += (double)bs[0];
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i <= N; i += blockDim.x)
        part[(size_t)blockIdx.x * (N + 1) + i] = acc_sh[i];
}

// Joint bit weights for two-spin correlations.  Per block, FP64, stride K = 1 + N + N(N-1)/2:
//   [0] = sum_s w(s),  [1 + i] = sum_s w(s) b_i(s),  [1 + N + pair(i, j)] = sum_s w(s) b_i(s) b_j(s)
// with w(s) = |psi_s|^2, b_i the bits of s and pair(i, j) (i < j) the row-major index of the
// strict upper triangle.  Each block iteration covers 2^13 consecutive amplitudes: thread bits
// are global bits 0..7, the 32 per-thread amplitudes global bits 8..12, the higher bits are
// constant over the range.  The 92 in-range sums (total, 13 singles, 78 pairs) are formed in the
// amplitudes' precision and added, with the constant high bits, to FP64 totals.
__host__ __device__ constexpr int pair_index(int i, int j, int N) { return i * N - i * (i + 1) / 2 + (j - i - 1); }

template <typename C>
__global__ void __launch_bounds__(256) k_sum_pairs(const C *__restrict__ psi, int N, double *__restrict__ part)
{
    using A = typename AccOf<C>::T;
    constexpr int LB = 5, TBITS = 8, RBITS = LB + TBITS;
    constexpr int NV = 1 + RBITS + RBITS * (RBITS - 1) / 2;   // 92
    const int K = 1 + N + N * (N - 1) / 2;
    const uint64_t dim = UINT64_C(1) << N;
    extern __shared__ double acc_sh[];                       // K doubles
    __shared__ A bs[NV];
    __shared__ A red16[16];
    for (int i = threadIdx.x; i < K; i += blockDim.x)
        acc_sh[i] = 0.0;
    __syncthreads();
    const uint64_t per_block = (uint64_t)blockDim.x << LB;
    const int nin = N < RBITS ? N : RBITS;                   // bits inside one range
    for (uint64_t base = (uint64_t)blockIdx.x * per_block; base < dim; base += (uint64_t)gridDim.x * per_block) {
        // per-thread sums over its 32 amplitudes: total, per register bit, per register-bit pair
        A q[32];
        const uint64_t s0 = base + threadIdx.x;
#pragma unroll
        for (int j = 0; j < 32; j++) {
            C a;
            a.x = 0;
            a.y = 0;
            const uint64_t s = s0 + ((uint64_t)j << TBITS);
            if (s < dim)
                a = psi[s];
            q[j] = (A)a.x * (A)a.x + (A)a.y * (A)a.y;
        }
        A tot = A(0), low[LB], low2[LB * (LB - 1) / 2];
#pragma unroll
        for (int b = 0; b < LB; b++)
            low[b] = A(0);
#pragma unroll
        for (int k = 0; k < LB * (LB - 1) / 2; k++)
            low2[k] = A(0);
#pragma unroll
        for (int j = 0; j < 32; j++) {
            tot += q[j];
#pragma unroll
            for (int b = 0; b < LB; b++)
                if ((j >> b) & 1)
                    low[b] += q[j];
            int k = 0;
#pragma unroll
            for (int b1 = 0; b1 < LB; b1++)
#pragma unroll
                for (int b2 = b1 + 1; b2 < LB; b2++, k++)
                    if (((j >> b1) & 1) && ((j >> b2) & 1))
                        low2[k] += q[j];
        }
        // the block's 92 sums, 16 at a time (register pressure); local bit l is thread bit l
        // (l < 8) or register bit l - 8
        const uint32_t t = threadIdx.x;
        auto value = [&](int k) -> A {
            if (k == 0)
                return tot;
            if (k <= RBITS) {
                const int l = k - 1;
                return l < TBITS ? (((t >> l) & 1) ? tot : A(0)) : low[l - TBITS];
            }
            int r = k - 1 - RBITS, l1 = 0;
            while (r >= RBITS - 1 - l1) {
                r -= RBITS - 1 - l1;
                l1++;
            }
            const int l2 = l1 + 1 + r;
            if (l2 < TBITS)
                return (((t >> l1) & 1) && ((t >> l2) & 1)) ? tot : A(0);
            if (l1 < TBITS)
                return ((t >> l1) & 1) ? low[l2 - TBITS] : A(0);
            return low2[pair_index(l1 - TBITS, l2 - TBITS, LB)];
        };
#pragma unroll
        for (int r0 = 0; r0 < NV; r0 += 16) {
            A v[16];
#pragma unroll
            for (int i = 0; i < 16; i++)
                v[i] = (r0 + i < NV) ? value(r0 + i) : A(0);
            block_sum<16>(v, red16);
            if (threadIdx.x < 16 && r0 + (int)threadIdx.x < NV)
                bs[r0 + threadIdx.x] = red16[threadIdx.x];
        }
        __syncthreads();
        // add to the FP64 totals; the bits above the range are those of base
        for (int e = threadIdx.x; e < K; e += blockDim.x) {
            double add;
            if (e == 0) {
                add = (double)bs[0];
            } else if (e <= N) {
                const int i = e - 1;
                add = i < nin ? (double)bs[1 + i] : (((base >> i) & 1) ? (double)bs[0] : 0.0);
            } else {
                // invert the pair index
                int r = e - 1 - N, i = 0;
                while (r >= N - 1 - i) {
                    r -= N - 1 - i;
                    i++;
                }
                const int j = i + 1 + r;
                if (j < nin)
                    add = (double)bs[1 + RBITS + pair_index(i, j, RBITS)];
                else if (i < nin)
                    add = ((base >> j) & 1) ? (double)bs[1 + i] : 0.0;
                else
                    add = (((base >> i) & 1) && ((base >> j) & 1)) ? (double)bs[0] : 0.0;
            }
            acc_sh[e] += add;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < K; i += blockDim.x)
        part[(size_t)blockIdx.x * K + i] = acc_sh[i];
}

// Per block: sum |psi|^2 over a grid-stride range; per thread FP32 (complex64) pairwise
// sums of 32 amplitudes added to an FP64 running total, one FP64 block reduction.
template <typename C>
__global__ void __launch_bounds__(256) k_sum_norm(const C *__restrict__ psi, int N, double *__restrict__ part)
{
    using A = typename AccOf<C>::T;
    const uint64_t dim = UINT64_C(1) << N;
    const uint64_t per_block = (uint64_t)blockDim.x << 5;
    double run = 0.0;
    for (uint64_t base = (uint64_t)blockIdx.x * per_block; base < dim; base += (uint64_t)gridDim.x * per_block) {
        const uint64_t s0 = base + threadIdx.x;
        if (s0 < dim) {
            const uint64_t rem = (dim - s0 + 255) >> 8;
            const int n = rem < 32 ? (int)rem : 32;
            A q[32];
#pragma unroll
            for (int j = 0; j < 32; j++) {
                C a;
                a.x = 0;
                a.y = 0;
                if (j < n)
                    a = psi[s0 + (size_t)j * 256];
                q[j] = (A)a.x * (A)a.x + (A)a.y * (A)a.y;
            }
#pragma unroll
            for (int w = 16; w >= 1; w >>= 1)
#pragma unroll
                for (int i = 0; i < w; i++)
                    q[i] = q[i] + q[i + w];
            run += (double)q[0];
        }
    }
    double v[1] = {run};
    __shared__ double bs[1];
    block_sum<1>(v, bs);
    if (threadIdx.x == 0)
        part[blockIdx.x] = bs[0];
}

// Per block: sum |psi_s|^2 * E_alpha(s) * wscale
template <typename C>
__global__ void k_sum_diag_energy(const C *__restrict__ psi, uint64_t dim, HamDev ham, int alpha,
                                  double *__restrict__ part)
{
    const double *Jq = ham.Jq + (size_t)alpha * ham.N * ham.N;
    const double *hh = ham.hh + (size_t)alpha * ham.N;
    double v[1] = {0.0};
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < dim; s += stride)
        v[0] += norm2(psi[s]) * energy_bits(s, Jq, hh, ham.N);
    __shared__ double bs[1];
    block_sum<1>(v, bs);
    if (threadIdx.x == 0)
        part[blockIdx.x] = bs[0];
}

// Per block: sum conj(a_s) b_s as (re, im)
template <typename C>
__global__ void k_sum_overlap(const C *__restrict__ a, const C *__restrict__ b, uint64_t dim,
                              double *__restrict__ part)
{
    double v[2] = {0.0, 0.0};
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < dim; s += stride) {
        const C x = a[s], y = b[s];
        v[0] += (double)x.x * y.x + (double)x.y * y.y;
        v[1] += (double)x.x * y.y - (double)x.y * y.x;
    }
    __shared__ double bs[2];
    block_sum<2>(v, bs);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = bs[0];
        part[2 * blockIdx.x + 1] = bs[1];
    }
}

// Final stage: out[k] = sum over nblk blocks of part[b * K + k], fixed order.
static __global__ void k_sum_final(const double *__restrict__ part, int nblk, int K, double *__restrict__ out)
{
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblk; b++)
            s += part[(size_t)b * K + k];
        out[k] = s;
    }
}

template <typename C>
__global__ void k_set_basis(C *__restrict__ psi, uint64_t dim, uint64_t s0)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < dim; s += stride) {
        C z;
        z.x = (s == s0) ? 1 : 0;
        z.y = 0;
        psi[s] = z;
    }
}

} // namespace ts4
