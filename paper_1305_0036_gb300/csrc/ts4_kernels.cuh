// CUDA kernels of the TS4 library (sm_103a).
//
//   k_wht_bit     one butterfly per thread on one spin over the whole state
//                 (the paper's "GPU-Basic" kernel, Sec. 3.3 first paragraph)
//   k_slot_basic  one diagonal slot per element, E(s) from bit tests (Sec. 3.1)
//   k_pass        fused tile pass: a thread block holds 2^TB amplitudes whose
//                 other spins are fixed by the block index (Secs. 3.3-3.4),
//                 rotates the window spins in registers, 2^RB amplitudes per
//                 thread, applies a diagonal slot between two layers, and
//                 writes the tile back: one HBM round trip per pass
//   k_sum_*       FP64-accumulating reductions for the observables (Sec. 4.2)
#pragma once

#include "ts4_common.cuh"

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
    const double scale = ldexp(sl.mag, -sl.scale_exp);
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

// ------------------------------------------------------------------ fused tile pass

// Bank swizzle of the shared-memory tile: the 16-byte (8-byte amplitudes) or
// 8-slot (16-byte amplitudes) bank group of element e is XORed with its higher
// nibbles, so that a warp reading 32 amplitudes that differ in any 4 (3)
// consecutive local bits hits distinct banks.  XOR-linear: phys(a ^ b) =
// phys(a) ^ phys(b).
template <int ES> __host__ __device__ constexpr uint32_t phys(uint32_t e)
{
    return ES == 8 ? (e ^ (((e >> 4) ^ (e >> 8) ^ (e >> 12) ^ (e >> 16)) & 15u))
                   : (e ^ (((e >> 3) ^ (e >> 6) ^ (e >> 9) ^ (e >> 12) ^ (e >> 15)) & 7u));
}

struct StepDesc {
    uint8_t k;          // chunk: register window starts at min(k * RB, TB - RB)
    uint8_t r0lo, r0hi; // register bits rotated before the slot
    uint8_t ph;         // 1: apply the pass's slot
    uint8_t r1lo, r1hi; // register bits rotated after the slot
    uint8_t pad0, pad1;
};

constexpr int kMaxSteps = 16;

struct PassArgs {
    int c, w, h;  // tile geometry (global bits [0,c) and [w,w+h))
    int nsteps;
    StepDesc steps[kMaxSteps];
    Slot slot;
    int has_slot;
    int tab;      // index of the slot's local tables
    HamDev ham;
};

// Per-(slot, geometry) tables, built on the host in FP64 (angles in units of pi):
//   A[l*TB+m] = t * J^a_{pos l, pos m} / (4 pi) for the tile's local bits (symmetric)
//   QK[j]     = exp(-i sum_{l<m in chunk} A s_l s_m) * i^{pcq popcount(j)} for
//               the register chunk of the step that applies the slot
template <typename R, int TB, int RB> struct PassTab {
    R A[TB * TB];
    typename CT<R>::T QK[1 << RB];
};

template <int RB, typename C> __device__ __forceinline__ void wht_regs(C (&x)[1 << RB], int lo, int hi)
{
#pragma unroll
    for (int b = 0; b < RB; b++) {
        if (b >= lo && b < hi) {
#pragma unroll
            for (int j = 0; j < (1 << RB); j++)
                if (!(j & (1 << b)))
                    bfly(x[j], x[j | (1 << b)]);
        }
    }
}

template <typename R, int TB, int RB> struct PassShared {
    R A[TB * TB];
    R g[TB];
    typename CT<R>::T QK[1 << RB];
    R thFF;
    int pcF;
};

// Factors of the slot for one thread's 2^RB amplitudes (local index base | j << W):
//   F(j) = 2^{-e} i^{pcq pc(s)} exp(-i theta(s)),
//   theta = theta_FF + sum_{l in tile} s_l g_l + sum_{l<m in tile} A_lm s_l s_m.
// Everything that depends on the thread's own bits (base) is summed once per
// thread: theta = ang + sum_{b<RB} s_b cb_b + q(j); then
//   F(j) = flo[j mod 2^LO] * fhi[j >> LO] * QK[j]
// with flo, fhi products of exp(-+i cb_b) over the low / high register bits and
// QK[j] = exp(-i q(j)) i^{pcq popcount(j)} from the per-slot table.
template <typename R, int RB> struct SlotFactors {
    static constexpr int LO = RB - 2;
    typename CT<R>::T flo[1 << LO];
    typename CT<R>::T fhi[4];
};

template <typename R, int TB, int RB, int W>
__device__ __forceinline__ void slot_factors(SlotFactors<R, RB> &F, uint32_t base,
                                             const PassShared<R, TB, RB> &sh, int pcq, R scale)
{
    using C = typename CT<R>::T;
    constexpr int LO = RB - 2;
    R ang = sh.thFF;
    R cb[RB];
#pragma unroll
    for (int b = 0; b < RB; b++)
        cb[b] = sh.g[W + b];
#pragma unroll
    for (int m = 0; m < TB; m++) {
        if (m >= W && m < W + RB)
            continue;
        const R sm = ((base >> m) & 1u) ? R(1) : R(-1);
        ang += sm * sh.g[m];
#pragma unroll
        for (int l = m + 1; l < TB; l++) {
            if (l >= W && l < W + RB)
                continue;
            const R sl = ((base >> l) & 1u) ? R(1) : R(-1);
            ang += (sm * sl) * sh.A[m * TB + l];
        }
#pragma unroll
        for (int b = 0; b < RB; b++)
            cb[b] += sm * sh.A[(W + b) * TB + m];
    }
    C eb = cexpm_pi(ang);
    eb.x *= scale;
    eb.y *= scale;
    eb = cmul_ipow(eb, pcq * (sh.pcF + __popc(base)));
    F.flo[0] = eb;
#pragma unroll
    for (int b = 0; b < LO; b++) {
        const C ub = cexpm_pi(cb[b]);
#pragma unroll
        for (int k = 0; k < (1 << b); k++) {
            const C v = F.flo[k];
            F.flo[k] = cmul(v, cconj(ub));
            F.flo[k | (1 << b)] = cmul(v, ub);
        }
    }
    const C a1 = cexpm_pi(cb[LO]), b1 = cexpm_pi(cb[LO + 1]);
    const C a0 = cconj(a1), b0 = cconj(b1);
    F.fhi[0] = cmul(a0, b0);
    F.fhi[1] = cmul(a1, b0);
    F.fhi[2] = cmul(a0, b1);
    F.fhi[3] = cmul(a1, b1);
}

template <typename R, int TB, int RB, int K, bool PH>
__device__ __forceinline__ void run_step(typename CT<R>::T *tile, const StepDesc &d,
                                         const PassShared<R, TB, RB> &sh, int pcq, R scale)
{
    using C = typename CT<R>::T;
    constexpr int ES = sizeof(C);
    constexpr int W = (K * RB < TB - RB) ? K * RB : TB - RB;
    constexpr int LO = RB - 2;
    const uint32_t tid = threadIdx.x;
    const uint32_t base = (tid & ((1u << W) - 1)) | ((tid >> W) << (W + RB));
    const uint32_t pb = phys<ES>(base);
    SlotFactors<R, RB> F;
    if constexpr (PH)
        slot_factors<R, TB, RB, W>(F, base, sh, pcq, scale);
    C x[1 << RB];
#pragma unroll
    for (int j = 0; j < (1 << RB); j++)
        x[j] = tile[pb ^ phys<ES>((uint32_t)j << W)];
    wht_regs<RB>(x, d.r0lo, d.r0hi);
    if constexpr (PH) {
#pragma unroll
        for (int j = 0; j < (1 << RB); j++)
            x[j] = cmul(x[j], cmul(cmul(F.flo[j & ((1 << LO) - 1)], F.fhi[j >> LO]), sh.QK[j]));
    }
    wht_regs<RB>(x, d.r1lo, d.r1hi);
#pragma unroll
    for (int j = 0; j < (1 << RB); j++)
        tile[pb ^ phys<ES>((uint32_t)j << W)] = x[j];
}

// 128 registers per thread at most: as many blocks per SM as that allows
template <int NT> constexpr int min_blocks() { return (512 / NT) > 0 ? (512 / NT) : 1; }

template <typename R, int TB, int RB>
__global__ void __launch_bounds__(1 << (TB - RB), min_blocks<(1 << (TB - RB))>())
k_pass(typename CT<R>::T *__restrict__ psi, const __grid_constant__ PassArgs a,
       const PassTab<R, TB, RB> *__restrict__ tabs)
{
    using C = typename CT<R>::T;
    constexpr int ES = sizeof(C);
    constexpr int NT = 1 << (TB - RB);
    constexpr int NE = 1 << TB;
    constexpr int NR = 1 << RB;
    constexpr int PER_VEC = 16 / ES;         // amplitudes per 16-byte vector
    constexpr int NV = NE / PER_VEC / NT;    // vectors per thread
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tile = reinterpret_cast<C *>(smem_raw);
    __shared__ PassShared<R, TB, RB> sh;

    const int tid = threadIdx.x;
    const uint64_t f = blockIdx.x;
    const int c = a.c, w = a.w, h = a.h;
    const uint64_t gbase = tile_global_index(c, w, h, f, 0);
    const uint32_t cm = (1u << c) - 1u;
    // local index step between the two amplitudes of one 16-byte vector
    const uint32_t estep = (c >= 1) ? (1u << h) : 1u;

    // ---- load: 16-byte vectors, consecutive threads on consecutive addresses (two batches)
#pragma unroll
    for (int half = 0; half < 2; half++) {
        constexpr int NH = NV / 2;
        float4 v[NH];
#pragma unroll
        for (int q = 0; q < NH; q++) {
            const uint32_t u = (uint32_t)((half * NH + q) * NT + tid) * PER_VEC;
            const uint64_t gi = gbase | (u & cm) | ((uint64_t)(u >> c) << w);
            v[q] = __ldcs(reinterpret_cast<const float4 *>(psi + gi));
        }
#pragma unroll
        for (int q = 0; q < NH; q++) {
            const uint32_t u = (uint32_t)((half * NH + q) * NT + tid) * PER_VEC;
            const uint32_t e = (u >> c) | ((u & cm) << h);
            if constexpr (PER_VEC == 2) {
                const float2 *p = reinterpret_cast<const float2 *>(&v[q]);
                reinterpret_cast<float2 *>(tile)[phys<ES>(e)] = p[0];
                reinterpret_cast<float2 *>(tile)[phys<ES>(e + estep)] = p[1];
            } else {
                reinterpret_cast<float4 *>(tile)[phys<ES>(e)] = v[q];
            }
        }
    }

    // ---- per-block part of the slot, FP64 (fixed spins of this block)
    int pcq = 0;
    R scale = R(1);
    if (a.has_slot) {
        const int N = a.ham.N;
        const int al = a.slot.alpha;
        const double t = a.slot.t;
        const double *Jq = a.ham.Jq + (size_t)al * N * N;
        const double *hh = a.ham.hh + (size_t)al * N;
        pcq = a.slot.pcq;
        scale = (R)ldexp(a.slot.mag, -a.slot.scale_exp);
        if (tid < TB) {
            const int pos = (tid < h) ? (w + tid) : (tid - h);
            double acc = hh[pos];
            for (int j = 0; j < N; j++)
                if (!in_tile(j, c, w, h))
                    acc += Jq[pos * N + j] * (((gbase >> j) & 1) ? 1.0 : -1.0);
            sh.g[tid] = (R)(t * acc * 0.31830988618379067153776752674503);
        } else if (tid >= 32 && tid < 64) {
            const int lane = tid - 32;
            double acc = 0.0;
            for (int i = lane; i < N; i += 32) {
                if (in_tile(i, c, w, h))
                    continue;
                double r = hh[i];
                for (int j = i + 1; j < N; j++)
                    if (!in_tile(j, c, w, h))
                        r += Jq[i * N + j] * (((gbase >> j) & 1) ? 1.0 : -1.0);
                acc += (((gbase >> i) & 1) ? 1.0 : -1.0) * r;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) {
                sh.thFF = (R)halfturns_2pi(t * acc + a.slot.th0);
                sh.pcF = __popcll(gbase);
            }
        }
        const PassTab<R, TB, RB> *tb = tabs + a.tab;
        for (int k = tid; k < TB * TB; k += NT)
            sh.A[k] = tb->A[k];
        if (tid < NR)
            sh.QK[tid] = tb->QK[tid];
    }
    __syncthreads();

    // ---- register-chunk steps
    for (int s = 0; s < a.nsteps; s++) {
        const StepDesc d = a.steps[s];
        switch (d.k * 2 + (d.ph ? 1 : 0)) {
        case 0: run_step<R, TB, RB, 0, false>(tile, d, sh, pcq, scale); break;
        case 1: run_step<R, TB, RB, 0, true>(tile, d, sh, pcq, scale); break;
        case 2: run_step<R, TB, RB, 1, false>(tile, d, sh, pcq, scale); break;
        case 3: run_step<R, TB, RB, 1, true>(tile, d, sh, pcq, scale); break;
        case 4: run_step<R, TB, RB, 2, false>(tile, d, sh, pcq, scale); break;
        case 5: run_step<R, TB, RB, 2, true>(tile, d, sh, pcq, scale); break;
        case 6: run_step<R, TB, RB, 3, false>(tile, d, sh, pcq, scale); break;
        default: run_step<R, TB, RB, 3, true>(tile, d, sh, pcq, scale); break;
        }
        __syncthreads();
    }

    // ---- store
#pragma unroll
    for (int k = 0; k < NV; k++) {
        const uint32_t u = (uint32_t)(k * NT + tid) * PER_VEC;
        const uint32_t e = (u >> c) | ((u & cm) << h);
        const uint64_t gi = gbase | (u & cm) | ((uint64_t)(u >> c) << w);
        float4 v;
        if constexpr (PER_VEC == 2) {
            float2 *p = reinterpret_cast<float2 *>(&v);
            p[0] = reinterpret_cast<const float2 *>(tile)[phys<ES>(e)];
            p[1] = reinterpret_cast<const float2 *>(tile)[phys<ES>(e + estep)];
        } else {
            v = reinterpret_cast<const float4 *>(tile)[phys<ES>(e)];
        }
        __stcs(reinterpret_cast<float4 *>(psi + gi), v);
    }
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

// Block sums of several FP64 values; results land in out[0..K) of block 0's thread 0 view.
template <int K> __device__ void block_sum(double (&v)[K], double *__restrict__ dst)
{
    __shared__ double red[32][K];
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
            double s = (lane < nw) ? red[lane][k] : 0.0;
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
__device__ __forceinline__ void thread_sums32(const C *__restrict__ p, int stride, int n, double &tot,
                                              double (&low)[5])
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
        low[b] = (double)t[0];
    }
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1)
#pragma unroll
        for (int i = 0; i < w; i++)
            q[i] = q[i] + q[i + w];
    tot = (double)q[0];
}

template <typename C> struct AccOf;
template <> struct AccOf<float2> { using T = float; };
template <> struct AccOf<double2> { using T = double; };

// Per block: [0] = sum |psi|^2, [1..] = sum |psi_s|^2 bit_i(s) for i < N  (stride N+1)
template <typename C>
__global__ void __launch_bounds__(256) k_sum_sz(const C *__restrict__ psi, int N, double *__restrict__ part)
{
    // each block iteration covers a contiguous range of 2^13 amplitudes (256 threads x 32)
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
        double tot = 0.0, low[LB] = {0, 0, 0, 0, 0};
        const uint64_t s0 = base + threadIdx.x;
        if (s0 < dim) {
            const uint64_t rem = (dim - s0 + 255) >> 8;       // elements s0 + 256 j below dim
            const int n = rem < 32 ? (int)rem : 32;
            thread_sums32<C, typename AccOf<C>::T>(psi + s0, 256, n, tot, low);
        }
        double v[1 + 8 + LB];
        v[0] = tot;
#pragma unroll
        for (int b = 0; b < 8; b++)
            v[1 + b] = ((threadIdx.x >> b) & 1) ? tot : 0.0;
#pragma unroll
        for (int b = 0; b < LB; b++)
            v[1 + 8 + b] = low[b];
        __shared__ double bs[1 + 8 + LB];
        block_sum<1 + 8 + LB>(v, bs);
        if (threadIdx.x == 0) {
            acc_sh[0] += bs[0];
            for (int i = 0; i < N && i < RBITS; i++)
                acc_sh[1 + i] += bs[1 + i];
            for (int i = RBITS; i < N; i++)
                if ((base >> i) & 1)
                    acc_sh[1 + i] += bs[0];
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i <= N; i += blockDim.x)
        part[(size_t)blockIdx.x * (N + 1) + i] = acc_sh[i];
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
