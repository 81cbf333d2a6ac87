// CUDA kernels of the TS4 library (sm_103a).
//
//   k_wht_bit     one butterfly per thread on one spin over the whole state
//                 (the paper's "GPU-Basic" kernel, Sec. 3.3 first paragraph)
//   k_slot_basic  one diagonal slot per element, E(s) from bit tests (Sec. 3.1)
//   (the fused tile pass k_tile is in ts4_tile.cuh; this file holds the step
//   descriptors and per-pass tables it shares with the host)
//   k_sum_*       reductions for the observables (Sec. 4.2), FP64-grade accumulation
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

// The paper's phase-table mode (Sec. 3.1): E_alpha(s) for every basis state, stored once, so
// that a slot reads its angle instead of forming it from the bits.  E is the table's type:
// double for complex128 (8 bytes per state and alpha, the paper's FP64 tables), float for
// complex64 (4 bytes).  Kept for the A/B comparison with the bit-test and the fused kernels.
template <typename E>
__global__ void k_energy_table(E *__restrict__ tab, uint64_t dim, HamDev ham, int alpha)
{
    const double *Jq = ham.Jq + (size_t)alpha * ham.N * ham.N;
    const double *hh = ham.hh + (size_t)alpha * ham.N;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < dim; s += stride)
        tab[s] = (E)energy_bits(s, Jq, hh, ham.N);
}

// One slot from the energy table: as k_slot_basic, with E_alpha(s) read from the table.
template <typename R, typename E>
__global__ void k_slot_table(typename CT<R>::T *__restrict__ psi, const E *__restrict__ tab, uint64_t dim, Slot sl)
{
    using C = typename CT<R>::T;
    const double scale = sl.scale;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < dim; s += stride) {
        const double th = sl.th0 + sl.t * (double)tab[s];
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

// ---- accumulation of |psi_s|^2 at FP64-grade accuracy
// complex64: the square of an FP32 component is exact as its product plus the FMA residual, and
// a thread keeps its sums as unevaluated float pairs hi + lo ("double-float"): two_sum keeps the
// rounding of every addition in lo, so a sum of n terms is off by about n u^2 (u = 2^-24) of its
// value instead of n u.  GB300's FP64 pipe is too narrow for one FP64 addition per amplitude at
// HBM speed (about 0.4 ms per operation per amplitude at N = 28, more than the 0.3 ms read), while
// these FP32 operations fit under the read.  Per-thread results are converted to FP64 (exactly:
// hi and lo are floats) and reduced across the block and the grid in FP64.
// complex128: plain FP64 throughout.
struct DF {
    float hi, lo;
};

template <typename C> struct SqAcc;
template <> struct SqAcc<float2> {
    DF v;
    __device__ __forceinline__ void zero() { v.hi = v.lo = 0.0f; }
    __device__ __forceinline__ void add_sq(float2 a)
    {
        const float p1 = __fmul_rn(a.x, a.x), e1 = __fmaf_rn(a.x, a.x, -p1);
        const float p2 = __fmul_rn(a.y, a.y), e2 = __fmaf_rn(a.y, a.y, -p2);
        const float2 s = two_sum(p1, p2);
        const float2 h = two_sum(v.hi, s.x);
        v.hi = h.x;
        v.lo = __fadd_rn(v.lo, __fadd_rn(h.y, __fadd_rn(s.y, __fadd_rn(e1, e2))));
    }
    __device__ __forceinline__ void add(const SqAcc &o)
    {
        const float2 h = two_sum(v.hi, o.v.hi);
        v.hi = h.x;
        v.lo = __fadd_rn(v.lo, __fadd_rn(h.y, o.v.lo));
    }
    // this minus o, for o an earlier value of the same running sum (the difference is formed
    // from the exact hi difference and the lo terms)
    __device__ __forceinline__ SqAcc minus(const SqAcc &o) const
    {
        SqAcc r;
        const float2 h = two_sum(v.hi, -o.v.hi);
        r.v.hi = h.x;
        r.v.lo = __fadd_rn(h.y, __fsub_rn(v.lo, o.v.lo));
        return r;
    }
    // moves the rounding in lo back under hi (keeps |lo| <= ulp(hi) / 2 over long sums)
    __device__ __forceinline__ void renorm()
    {
        const float s = __fadd_rn(v.hi, v.lo);
        v.lo = __fsub_rn(v.lo, __fsub_rn(s, v.hi));
        v.hi = s;
    }
    __device__ __forceinline__ double value() const { return (double)v.hi + (double)v.lo; }
};
template <> struct SqAcc<double2> {
    double v;
    __device__ __forceinline__ void zero() { v = 0.0; }
    __device__ __forceinline__ void add_sq(double2 a) { v += a.x * a.x + a.y * a.y; }
    __device__ __forceinline__ void add(const SqAcc &o) { v += o.v; }
    __device__ __forceinline__ SqAcc minus(const SqAcc &o) const
    {
        SqAcc r;
        r.v = v - o.v;
        return r;
    }
    __device__ __forceinline__ void renorm() {}
    __device__ __forceinline__ double value() const { return v; }
};

// Geometry of the |psi|^2 reductions: a range is 2^12 consecutive amplitudes; in a range the
// 256 threads take global bits 0..7 (coalesced loads) and the 16 amplitudes of a thread global
// bits 8..11.
constexpr int kSumTBits = 8, kSumJBits = 4, kSumRangeBits = kSumTBits + kSumJBits;
// Varying range bits one block of k_sum_sz may span (its span of ranges is at most 2^12).
constexpr int kSumMaxVar = 12;

__host__ __device__ constexpr uint64_t sum_ranges(int N)
{
    return N > kSumRangeBits ? (UINT64_C(1) << (N - kSumRangeBits)) : UINT64_C(1);
}

// Number of blocks for k_sum_sz: a power of two that divides the ranges, at most `cap` (a
// power of two), and large enough that every block spans at most 2^kSumMaxVar ranges.
__host__ __device__ inline unsigned sum_sz_blocks(int N, unsigned cap)
{
    const uint64_t R = sum_ranges(N);
    uint64_t b = R < cap ? R : cap;
    while (R / b > (UINT64_C(1) << kSumMaxVar))
        b <<= 1;
    return (unsigned)b;
}

// Per block: part[b (N + 1)] = sum |psi_s|^2 and part[b (N + 1) + 1 + i] = sum |psi_s|^2 bit_i(s)
// over the block's amplitudes (<S^z_i> = the second minus half the first, Sec. 4.2).
// gridDim.x = sum_sz_blocks(N, cap): block b covers the contiguous span of S = 2^m ranges from
// b S, so range bits m and above are the same for the whole block.  Per thread: one accumulator
// per register index j (global bits 8..11), a running total, and, for each of the m varying
// range bits, the sum of the totals of the ranges that set it (each range's total is the
// difference of the running total before and after it).
template <typename C>
__global__ void __launch_bounds__(256) k_sum_sz(const C *__restrict__ psi, int N, double *__restrict__ part)
{
    constexpr int NJ = 1 << kSumJBits;
    constexpr int NV = 1 + kSumRangeBits + kSumMaxVar;
    const uint64_t dim = UINT64_C(1) << N;
    const uint64_t span = sum_ranges(N) / gridDim.x;
    const int m = 63 - __clzll((long long)span);            // span = 2^m
    const uint64_t r0 = (uint64_t)blockIdx.x * span;
    const uint32_t t = threadIdx.x;
    SqAcc<C> acc[NJ], tot, hv[kSumMaxVar];
#pragma unroll
    for (int j = 0; j < NJ; j++)
        acc[j].zero();
    tot.zero();
#pragma unroll
    for (int k = 0; k < kSumMaxVar; k++)
        hv[k].zero();
    for (uint64_t rr = 0; rr < span; rr++) {
        const uint64_t s0 = ((r0 + rr) << kSumRangeBits) + t;
        const SqAcc<C> before = tot;
        C a[NJ];
#pragma unroll
        for (int j = 0; j < NJ; j++) {
            const uint64_t s = s0 + ((uint64_t)j << kSumTBits);
            a[j].x = 0;
            a[j].y = 0;
            if (s < dim)
                a[j] = psi[s];
        }
#pragma unroll
        for (int j = 0; j < NJ; j++) {
            acc[j].add_sq(a[j]);
            tot.add_sq(a[j]);
        }
        tot.renorm();
        const SqAcc<C> it = tot.minus(before);
#pragma unroll
        for (int k = 0; k < kSumMaxVar; k++)
            if (k < m && ((rr >> k) & 1)) {
                hv[k].add(it);
                hv[k].renorm();
            }
#pragma unroll
        for (int j = 0; j < NJ; j++)
            acc[j].renorm();
    }
    // the thread's sums in FP64: total, thread bits, register bits, varying range bits
    double v[NV];
    const double T = tot.value();
    v[0] = T;
#pragma unroll
    for (int b = 0; b < kSumTBits; b++)
        v[1 + b] = ((t >> b) & 1) ? T : 0.0;
#pragma unroll
    for (int b = 0; b < kSumJBits; b++) {
        SqAcc<C> lb;
        lb.zero();
#pragma unroll
        for (int j = 0; j < NJ; j++)
            if ((j >> b) & 1)
                lb.add(acc[j]);
        v[1 + kSumTBits + b] = lb.value();
    }
#pragma unroll
    for (int k = 0; k < kSumMaxVar; k++)
        v[1 + kSumRangeBits + k] = hv[k].value();
    __shared__ double bs[NV];
    block_sum<NV>(v, bs);
    for (int i = threadIdx.x; i <= N; i += blockDim.x) {
        double r;
        if (i == 0)
            r = bs[0];
        else if (i - 1 < kSumRangeBits)
            r = bs[i];                                           // thread and register bits
        else if (i - 1 - kSumRangeBits < m)
            r = bs[i];                                           // range bits that vary in the span
        else
            r = ((r0 >> (i - 1 - kSumRangeBits)) & 1) ? bs[0] : 0.0;   // constant over the span
        part[(size_t)blockIdx.x * (N + 1) + i] = r;
    }
}

// Joint bit weights for two-spin correlations.  Per block, FP64, stride K = 1 + N + N(N-1)/2:
//   [0] = sum_s w(s),  [1 + i] = sum_s w(s) b_i(s),  [1 + N + pair(i, j)] = sum_s w(s) b_i(s) b_j(s)
// with w(s) = |psi_s|^2, b_i the bits of s and pair(i, j) (i < j) the row-major index of the
// strict upper triangle.  Each block iteration covers 2^13 consecutive amplitudes: thread bits
// are global bits 0..7, the 32 per-thread amplitudes global bits 8..12, the higher bits are
// constant over the range.  The 92 in-range sums (total, 13 singles, 78 pairs) are formed in
// FP64 (for both precisions: these correlations are read rarely, so the FP64 rate does not
// matter) and added, with the constant high bits, to the block's FP64 totals.
__host__ __device__ constexpr int pair_index(int i, int j, int N) { return i * N - i * (i + 1) / 2 + (j - i - 1); }

template <typename C>
__global__ void __launch_bounds__(256) k_sum_pairs(const C *__restrict__ psi, int N, double *__restrict__ part)
{
    using A = double;
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

// Per block: sum |psi|^2 over a grid-stride set of ranges (the geometry of k_sum_sz); each
// thread keeps two running sums of the accumulator type above, one FP64 block reduction.
template <typename C>
__global__ void __launch_bounds__(256) k_sum_norm(const C *__restrict__ psi, int N, double *__restrict__ part)
{
    constexpr int NJ = 1 << kSumJBits;
    const uint64_t dim = UINT64_C(1) << N;
    const uint64_t R = sum_ranges(N);
    SqAcc<C> s0, s1;
    s0.zero();
    s1.zero();
    for (uint64_t r = blockIdx.x; r < R; r += gridDim.x) {
        const uint64_t b = (r << kSumRangeBits) + threadIdx.x;
        C a[NJ];
#pragma unroll
        for (int j = 0; j < NJ; j++) {
            const uint64_t s = b + ((uint64_t)j << kSumTBits);
            a[j].x = 0;
            a[j].y = 0;
            if (s < dim)
                a[j] = psi[s];
        }
#pragma unroll
        for (int j = 0; j < NJ; j += 2) {
            s0.add_sq(a[j]);
            s1.add_sq(a[j + 1]);
        }
        s0.renorm();
        s1.renorm();
    }
    double v[1] = {s0.value() + s1.value()};
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
