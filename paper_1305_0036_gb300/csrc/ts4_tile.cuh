// Fused tile pass, register-resident (Secs. 3.3-3.4 redesigned for sm_103a).
//
// A thread block owns one tile of 2^TB amplitudes: the tile's local bits are the
// window spins [w, w + h) (local bits [0, h)) and the c = TB - h lowest spins
// (local bits [h, TB)); the block index fixes every other spin.  Each thread
// keeps 2^RB amplitudes in registers.  A "layout" says which RB local bits are
// the register index; the others are spread over the 32 lanes and the warps.
// Butterflies on register bits need no data movement; to rotate other bits the
// tile is transposed to another layout through shared memory.
//
// Layouts: chunk k holds the local bits [W_k, W_k + RB), W_k = min(k RB, TB - RB).
// One chunk (1 for the lowest-spin group, 0 for the others) is also the I/O
// layout: its lanes are chosen (on the host) among the globally lowest bits of
// the tile so that the global loads and stores of one warp instruction cover
// consecutive addresses.
//
// Shared memory holds the transposed tile at padded positions
//   P(e) = e + (e >> 5) + (e >> 10)        (8-byte amplitudes, bank pair P mod 16)
//   P(e) = e + (e >> 4) + (e >> 8)         (16-byte amplitudes, 16-byte slot P mod 8)
// P is additive over disjoint bit sets, so the address of register j is the
// thread's base plus a compile-time offset, and the lanes of every layout are
// chosen so that the bank contributions of their low bits are distinct powers
// of two: every warp access is conflict-free.
#pragma once

#include <utility>

#include "ts4_kernels.cuh"

#include <type_traits>

namespace ts4 {

template <int ES> __host__ __device__ constexpr uint32_t padidx(uint32_t e)
{
    return ES == 8 ? e + (e >> 5) + (e >> 10) : e + (e >> 4) + (e >> 8);
}
template <int ES> __host__ __device__ constexpr int bank_contrib(int k)
{
    return (int)(padidx<ES>(1u << k) & (ES == 8 ? 15u : 7u));
}

// Thread-bit order (lanes first, then warps) of chunk layout W: the first
// (ES == 8 ? 4 : 3) lane bits take distinct nonzero bank contributions.
template <int TB, int RB, int ES> struct ChunkLayout {
    int bits[TB - RB];
    __host__ __device__ constexpr ChunkLayout(int W) : bits{}
    {
        const int need = ES == 8 ? 4 : 3;
        bool used[32] = {};
        int n = 0;
        int seen = 0;  // bitmask of contributions taken
        for (int k = 0; k < TB && n < need; k++) {
            if (k >= W && k < W + RB)
                continue;
            const int cb = bank_contrib<ES>(k);
            if (cb != 0 && !(seen & cb)) {
                seen |= cb;
                bits[n++] = k;
                used[k] = true;
            }
        }
        for (int k = 0; k < TB; k++) {
            if ((k >= W && k < W + RB) || used[k])
                continue;
            bits[n++] = k;
        }
    }
};

template <int TB, int RB> __host__ __device__ constexpr int chunk_w(int k)
{
    return (k * RB < TB - RB) ? k * RB : TB - RB;
}

// I/O layout (the register bits of chunk `chunk`), computed on the host for each group.
struct IOLayout {
    uint8_t bits[16];   // thread bit t -> local bit (lanes first)
    int chunk;          // 0 or 1
};

struct TileArgs {
    int c, w, h;
    int nsteps;
    StepDesc steps[kMaxSteps];
    Slot slot;
    int has_slot;
    int tab;
    int exact_sincos;   // c64 per-amplitude factor: 0 if |y| <= 0.05, 1 if |y| <= 0.5, 2 otherwise (sincospif)
    IOLayout io;
    HamDev ham;
    const double *theta; // per frame f: (t E_FF(f) + th0) / pi reduced to [-1, 1]  (k_frame_terms)
    const void *gfield;  // per frame f: g_l(f) for the TB tile spins, R precision  (k_frame_terms)
    const uint4 *iomap;  // per thread of the I/O layout: (global offset lo, hi, local base, 0)
    uint64_t gst[8];     // global offset of each register bit of the I/O layout
    int ens_shape;       // ensemble kernel: index of the compiled shape of this pass (0 = none)
};

// The frame-dependent parts of a slot's angle, for every tile f of a geometry
// (c, w, h) with TB = c + h local spins (local bit l is global spin pos(l)):
//   theta[f]       = (t E_FF(f) + th0) / pi reduced mod 2, E_FF = the field and
//                    coupling terms among the spins outside the tile;
//   g[f * TB + l]  = t (h_{pos l} / 2 + sum_{m outside} J_{pos l, m} sigma_m(f) / 4) * unit
//                    (unit = 1 for radians, 1/pi for half-turns).
// FP64 throughout, once per schedule; a pass reads TB + 2 words per block.
template <typename R>
__global__ void k_frame_terms(const double *__restrict__ Jq, const double *__restrict__ hh, int N, int c, int w,
                              int h, double t, double th0, double unit, uint64_t nframes, double *__restrict__ theta,
                              R *__restrict__ g)
{
    const int TB = c + h;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t f = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; f < nframes; f += stride) {
        const uint64_t gb = tile_global_index(c, w, h, f, 0);
        double acc = 0.0;
        for (int i = 0; i < N; i++) {
            if (in_tile(i, c, w, h))
                continue;
            double r = hh[i];
            for (int j = i + 1; j < N; j++)
                if (!in_tile(j, c, w, h))
                    r += Jq[i * N + j] * (((gb >> j) & 1) ? 1.0 : -1.0);
            acc += (((gb >> i) & 1) ? 1.0 : -1.0) * r;
        }
        theta[f] = halfturns_2pi(t * acc + th0);
        for (int l = 0; l < TB; l++) {
            const int i = l < h ? w + l : l - h;
            double r = hh[i];
            for (int m = 0; m < N; m++)
                if (!in_tile(m, c, w, h))
                    r += Jq[i * N + m] * (((gb >> m) & 1) ? 1.0 : -1.0);
            g[f * TB + l] = (R)(t * r * unit);
        }
    }
}

// Per-(slot, group) tables: PassTab (host-built in FP64, see ts4_kernels.cuh)
template <typename R, int TB, int RB> using TileTab = PassTab<R, TB, RB>;

// Per-thread factors of a complex64 slot with 2^RB registers; the register index j splits
// into its low RB - 2 bits (Lo) and its top 2 bits (Hi).
template <int RB> struct SlotThreadC64 {
    static constexpr int LB = RB - 2;
    float2 R[4];  // T i^{pcq p}, p = popcount of the register index mod 4 (i^4 = 1)
    float Lo[1 << LB];
    float Hi[4];
    float kT;          // |T (1 + kT)| = |scale| to ~1e-14: the FP32 magnitude error of T, removed
};

struct SlotThreadC128 {
    double2 flo[4];
    double2 fhi[4];
};

// The per-thread factors live in shared memory between their computation and the
// slot step, one array per field ([field][thread]), so that a warp reading one
// field touches consecutive words: an array of the structs above (stride 104 or
// 128 bytes) would put several lanes of a warp on the same bank.
template <int NT, int RB> struct SlotSoA64 {
    static constexpr int LB = RB - 2;
    float2 R[4][NT];
    float Lo[1 << LB][NT];
    float Hi[4][NT];
    float kT[NT];

    __device__ __forceinline__ void put(int t, const SlotThreadC64<RB> &o)
    {
#pragma unroll
        for (int k = 0; k < 4; k++)
            R[k][t] = o.R[k];
#pragma unroll
        for (int k = 0; k < (1 << LB); k++)
            Lo[k][t] = o.Lo[k];
#pragma unroll
        for (int k = 0; k < 4; k++)
            Hi[k][t] = o.Hi[k];
        kT[t] = o.kT;
    }
};

template <int NT> struct SlotSoA128 {
    double2 flo[4][NT];
    double2 fhi[4][NT];

    __device__ __forceinline__ void put(int t, const SlotThreadC128 &o)
    {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            flo[k][t] = o.flo[k];
            fhi[k][t] = o.fhi[k];
        }
    }
};

template <typename R, int TB, int RB> struct TileShared {
    // per-thread slot factors, computed before the tile occupies the registers
    typename std::conditional<sizeof(R) == 4, SlotSoA64<1 << (TB - RB), RB>, SlotSoA128<1 << (TB - RB)>>::type th_f;
    R g[TB];
    typename CT<R>::T Q[1 << RB];
    float th_hi, th_lo;  // c64: block angle in half-turns as a float pair
    double th;           // c128: block angle in half-turns
    int pcF;
};

// sin and cos of pi r for |r| <= 1/4 (plus rounding), without branches: x = pi r with
// pi split into two floats (x to ~1e-15 relative), then the Taylor series of sin to
// x^13 and of cos to x^14 (truncation below 3e-14 for |x| <= pi/4 + 1e-6).  The
// caller removes the magnitude error of the rounded pair, so only the angle matters.
__device__ __forceinline__ void sincos_quarter(float r, float &sn, float &cs)
{
    const float pi_hi = 3.14159274101257324f, pi_lo = -8.74227766e-8f;   // pi = pi_hi + pi_lo
    const float x = fmaf(r, pi_hi, r * pi_lo);
    const float x2 = x * x;
    float ps = fmaf(x2, 1.0f / 6227020800.0f, -1.0f / 39916800.0f);
    ps = fmaf(x2, ps, 1.0f / 362880.0f);
    ps = fmaf(x2, ps, -1.0f / 5040.0f);
    ps = fmaf(x2, ps, 1.0f / 120.0f);
    ps = fmaf(x2, ps, -1.0f / 6.0f);
    sn = fmaf(x * x2, ps, x);
    float pc = fmaf(x2, -1.0f / 87178291200.0f, 1.0f / 479001600.0f);
    pc = fmaf(x2, pc, -1.0f / 3628800.0f);
    pc = fmaf(x2, pc, 1.0f / 40320.0f);
    pc = fmaf(x2, pc, -1.0f / 720.0f);
    pc = fmaf(x2, pc, 1.0f / 24.0f);
    pc = fmaf(x2, pc, -0.5f);
    cs = fmaf(x2, pc, 1.0f);
}

__host__ __device__ constexpr int popc_c(int v) { return v ? (v & 1) + popc_c(v >> 1) : 0; }


// c64 slot, one factor per amplitude:
//   F(j) = T_thread * e^{-i y_j} * i^{pcq popcount(j)},
//   T_thread = 2^{-e} i^{pcq (pcF + popcount(base))} e^{-i pi X}, X = block + thread angle
//   y_j = sum_b s_b(j) c_b + q(j)  (small: |y| <= 0.5 unless exact_sincos)
// Rounding happens per amplitude (no table of rounded factors shared by many
// amplitudes), so the errors do not build up coherently over the steps.

// Per-thread part, for the register window W of the layout that applies the slot
// (compile-time W: only the thread's own bits enter the unrolled sums).
template <int TB, int RB, int W>
__device__ __forceinline__ void slot_thread_c64_w(SlotThreadC64<RB> &o, uint32_t base, const TileShared<float, TB, RB> &sh,
                                                  int pcq, float scale, float srel, float tp, const float (&tc)[RB])
{
    constexpr uint32_t chunk = ((1u << RB) - 1u) << W;
    // the couplings among the thread's own bits (tp, tc) come from the pass table;
    // the frame fields g_l depend on the block
    float sacc = tp;
    float cb[RB];
#pragma unroll
    for (int b = 0; b < RB; b++)
        cb[b] = sh.g[W + b] + tc[b];
#pragma unroll
    for (int m = 0; m < TB; m++) {
        if ((chunk >> m) & 1u)
            continue;
        const float sm = ((base >> m) & 1u) ? 1.0f : -1.0f;
        sacc = fmaf(sm, sh.g[m], sacc);
    }
    // thread angle in half-turns, reduced exactly: X = th_hi + th_lo + sacc / pi
    const float2 s1 = two_sum(sh.th_hi, __fmul_rn(sacc, 0.31830988618379067f));
    const float q = rintf(2.0f * s1.x);
    const float r = fmaf(-0.5f, q, s1.x) + (s1.y + sh.th_lo);
    float sn, cs;
    sincos_quarter(r, sn, cs);
    const int kt = (pcq * (sh.pcF + __popc(base)) - (int)q) & 3;
    const float2 T = cmul_ipow(make_float2(cs * scale, -sn * scale), kt);
    // magnitude error d = cs^2 + sn^2 - 1 of the FP32 pair, to ~1e-14 (exact products by FMA;
    // cs^2 in [1/2, 1] so cs^2 - 1 is exact); (1 - d/2) restores unit magnitude
    {
        const float p1 = __fmul_rn(cs, cs), e1 = fmaf(cs, cs, -p1);
        const float p2 = __fmul_rn(sn, sn), e2 = fmaf(sn, sn, -p2);
        const float d = ((p1 - 1.0f) + p2) + (e1 + e2);
        o.kT = fmaf(-0.5f, d, srel);
    }
    // the factor of register j is T i^{pcq popcount(j)} e^{-i y_j}: keep T i^{pcq p} for
    // p = 0..3 (the power of i repeats with period 4 in the popcount)
#pragma unroll
    for (int p = 0; p < 4; p++)
        o.R[p] = cmul_ipow(T, (pcq * p) & 3);
    constexpr int LB = RB - 2;
    o.Lo[0] = 0.0f;
#pragma unroll
    for (int b = 0; b < LB; b++)
#pragma unroll
        for (int k = 0; k < (1 << b); k++) {
            const float v = o.Lo[k];
            o.Lo[k] = v - cb[b];
            o.Lo[k | (1 << b)] = v + cb[b];
        }
    o.Hi[0] = -cb[LB] - cb[LB + 1];
    o.Hi[1] = cb[LB] - cb[LB + 1];
    o.Hi[2] = -cb[LB] + cb[LB + 1];
    o.Hi[3] = cb[LB] + cb[LB + 1];
}

template <int TB, int RB>
__device__ __forceinline__ void slot_thread_c64(SlotThreadC64<RB> &o, uint32_t base, int k,
                                                const TileShared<float, TB, RB> &sh, int pcq, float scale,
                                                float srel, float tp, const float (&tc)[RB])
{
    switch (k) {
    case 0: slot_thread_c64_w<TB, RB, chunk_w<TB, RB>(0)>(o, base, sh, pcq, scale, srel, tp, tc); break;
    case 1: slot_thread_c64_w<TB, RB, chunk_w<TB, RB>(1)>(o, base, sh, pcq, scale, srel, tp, tc); break;
    case 2: slot_thread_c64_w<TB, RB, chunk_w<TB, RB>(2)>(o, base, sh, pcq, scale, srel, tp, tc); break;
    default: slot_thread_c64_w<TB, RB, chunk_w<TB, RB>(3)>(o, base, sh, pcq, scale, srel, tp, tc); break;
    }
}

// e^{-iy} = (1 + c) - i s with s = sin y and c = cos y - 1, kept on the unit circle:
// mode 0 (|y| <= 0.05): Taylor series of cos y - 1 to y^6 and of sin y to y^5; the
//   magnitude error of the exact pair, 2 c_err + 2 s s_err, is below 2e-14, and the FP32
//   rounding of c (|c| <= 1.25e-3) adds about 1e-10;
// mode 1 (|y| <= 0.5): series to y^10 / y^11, then the magnitude error d = 2c + c^2 + s^2
//   is removed to first order;
// mode 2 (any y): CUDA's sincospif, then the same correction.
template <int MODE> __device__ __forceinline__ void unit_factor(float y, float &c, float &s)
{
    const float y2 = y * y;
    if constexpr (MODE == 0) {
        c = y2 * fmaf(y2, fmaf(y2, -1.0f / 720.0f, 1.0f / 24.0f), -0.5f);
        s = fmaf(y * y2, fmaf(y2, 1.0f / 120.0f, -1.0f / 6.0f), y);
    } else {
        if constexpr (MODE == 1) {
            float pc = fmaf(y2, -1.0f / 3628800.0f, 1.0f / 40320.0f);
            pc = fmaf(y2, pc, -1.0f / 720.0f);
            pc = fmaf(y2, pc, 1.0f / 24.0f);
            pc = fmaf(y2, pc, -0.5f);
            c = y2 * pc;
            float ps = fmaf(y2, -1.0f / 39916800.0f, 1.0f / 362880.0f);
            ps = fmaf(y2, ps, -1.0f / 5040.0f);
            ps = fmaf(y2, ps, 1.0f / 120.0f);
            ps = fmaf(y2, ps, -1.0f / 6.0f);
            s = fmaf(y * y2, ps, y);
        } else {
            float cc;
            sincospif(y * 0.31830988618379067f, &s, &cc);
            c = cc - 1.0f;
        }
        const float d = fmaf(s, s, fmaf(c, c, 2.0f * c));
        c = fmaf(-0.5f, d, c);
        s = fmaf(-0.5f * d, s, s);
    }
}

// Per-amplitude factors: x_j <- x_j R[popcount j] (1 + kT)((1 + c_j) - i s_j).  Every
// factor has unit magnitude to ~1e-10 times the exact scale; the one FP32 rounding left per
// component is that of the full product, which changes from step to step and does not
// build up.
// One amplitude, register index J (compile-time: every table index below is a constant).
template <int MODE, int J, int NT, int RB>
__device__ __forceinline__ void slot_c64_one(float2 &xj, const SlotSoA64<NT, RB> &o, int t,
                                             const float2 *__restrict__ Q, float kT)
{
    constexpr int P = popc_c(J), LB = RB - 2;
    const float y = (o.Lo[J & ((1 << LB) - 1)][t] + o.Hi[J >> LB][t]) + Q[J].x;
    float c, s;
    unit_factor<MODE>(y, c, s);
    // fold T's magnitude correction: (1 + kT)((1 + c) - i s), cross terms included (they
    // carry the sign of kT for every amplitude of a thread, i.e. they repeat each step)
    const float ct = fmaf(c, kT, c + kT);
    const float st = fmaf(s, kT, s);
    // x R (1 + ct - i st) = x R + x u with u = R (ct - i st) small.  The O(1) products enter
    // the FMA chain last, so each component is rounded once at full size.  Rounding x R
    // first and then applying the near-unit factor loses the sub-ulp magnitude correction
    // whenever c and s are small, and that loss repeats every step: it made the norm drift
    // by -1e-8 per step on the 2x12 ladder.
    const float2 r = o.R[P & 3][t];
    const float2 u = make_float2(fmaf(r.x, ct, r.y * st), fmaf(r.y, ct, -r.x * st));
    xj = make_float2(fmaf(xj.x, r.x, fmaf(-xj.y, r.y, fmaf(xj.x, u.x, -xj.y * u.y))),
                     fmaf(xj.x, r.y, fmaf(xj.y, r.x, fmaf(xj.x, u.y, xj.y * u.x))));
}

template <int MODE, int NT, int RB, int... J>
__device__ __forceinline__ void slot_c64_apply_seq(float2 (&x)[sizeof...(J)], const SlotSoA64<NT, RB> &o, int t,
                                                   const float2 *__restrict__ Q, std::integer_sequence<int, J...>)
{
    const float kT = o.kT[t];
    (slot_c64_one<MODE, J, NT, RB>(x[J], o, t, Q, kT), ...);
}

template <int RB, int MODE, int NT>
__device__ __forceinline__ void slot_c64_apply(float2 (&x)[1 << RB], const SlotSoA64<NT, RB> &o, int t,
                                               const float2 *__restrict__ Q)
{
    slot_c64_apply_seq<MODE, NT, RB>(x, o, t, Q, std::make_integer_sequence<int, (1 << RB)>{});
}

template <int RB, int NT>
__device__ __forceinline__ void slot_c64(float2 (&x)[1 << RB], const SlotSoA64<NT, RB> &o, int t,
                                         const float2 *__restrict__ Q, int mode)
{
    if (mode == 0)
        slot_c64_apply<RB, 0>(x, o, t, Q);
    else if (mode == 1)
        slot_c64_apply<RB, 1>(x, o, t, Q);
    else
        slot_c64_apply<RB, 2>(x, o, t, Q);
}

// c128 slot: per-thread factors (errors ~1e-16; table of the in-chunk terms).
template <int TB, int RB>
__device__ __forceinline__ void slot_thread_c128(SlotThreadC128 &o, uint32_t base, int W,
                                                 const TileShared<double, TB, RB> &sh, int pcq, double scale,
                                                 double tp, const double (&tc)[RB])
{
    double ang = sh.th + tp;
    double cb[RB];
#pragma unroll
    for (int b = 0; b < RB; b++)
        cb[b] = sh.g[W + b] + tc[b];
    const uint32_t chunk = ((1u << RB) - 1u) << W;
    for (int m = 0; m < TB; m++) {
        if ((chunk >> m) & 1u)
            continue;
        ang = fma(((base >> m) & 1u) ? 1.0 : -1.0, sh.g[m], ang);
    }
    double2 eb = cexpm_pi(ang);
    eb.x *= scale;
    eb.y *= scale;
    eb = cmul_ipow(eb, pcq * (sh.pcF + __popc(base)));
    static_assert(RB == 4, "c128 factors assume 4 register bits");
    o.flo[0] = eb;
#pragma unroll
    for (int b = 0; b < 2; b++) {
        const double2 ub = cexpm_pi(cb[b]);
#pragma unroll
        for (int k = 0; k < (1 << b); k++) {
            const double2 v = o.flo[k];
            o.flo[k] = cmul(v, cconj(ub));
            o.flo[k | (1 << b)] = cmul(v, ub);
        }
    }
    const double2 a1 = cexpm_pi(cb[2]), b1 = cexpm_pi(cb[3]);
    const double2 a0 = cconj(a1), b0 = cconj(b1);
    o.fhi[0] = cmul(a0, b0);
    o.fhi[1] = cmul(a1, b0);
    o.fhi[2] = cmul(a0, b1);
    o.fhi[3] = cmul(a1, b1);
}

template <int NT, int... J>
__device__ __forceinline__ void slot_c128_seq(double2 (&x)[16], const SlotSoA128<NT> &o, int t,
                                              const double2 *__restrict__ Q, std::integer_sequence<int, J...>)
{
    ((x[J] = cmul(x[J], cmul(cmul(o.flo[J & 3][t], o.fhi[J >> 2][t]), Q[J]))), ...);
}

template <int NT>
__device__ __forceinline__ void slot_c128(double2 (&x)[16], const SlotSoA128<NT> &o, int t,
                                          const double2 *__restrict__ Q)
{
    slot_c128_seq(x, o, t, Q, std::make_integer_sequence<int, 16>{});
}

// ---- compile-time pass shapes
// A pass is a list of steps: in chunk layout K, rotate the register bits [R0LO, R0HI), apply the
// slot if PH, rotate [R1LO, R1HI) (the run-time StepDesc).  The shapes of the passes that make up
// almost all of a long run are also compiled as template lists: the step loop, the chunk
// switches and the butterfly-range dispatch then vanish, and the compiler schedules across the
// steps of a pass.  RuntimeShape keeps the run-time loop for every other pass.
template <int K_, int R0LO_, int R0HI_, int PH_, int R1LO_, int R1HI_> struct Step {
    static constexpr int K = K_, R0LO = R0LO_, R0HI = R0HI_, PH = PH_, R1LO = R1LO_, R1HI = R1HI_;
};
template <int KIO_, typename... S> struct PassShape {
    static constexpr int KIO = KIO_;
    static constexpr int NS = (int)sizeof...(S);
    static constexpr int KPH = (0 + ... + (S::PH ? S::K : 0));   // chunk of the step with the slot
    // the group's window size h: the highest local bit the steps rotate, plus one
    template <int TB, int RB> static constexpr int h()
    {
        int m = 0;
        ((m = (chunk_w<TB, RB>(S::K) + (S::R0HI > S::R1HI ? S::R0HI : S::R1HI)) > m
                  ? chunk_w<TB, RB>(S::K) + (S::R0HI > S::R1HI ? S::R0HI : S::R1HI)
                  : m),
         ...);
        return m;
    }
};

// The I/O layout (thread bit -> local bit) of a tile whose group has h window spins, as the host
// builds it (make_io in ts4_api.cu).  It depends on (h, TB, RB, ES) only: the TB - h lowest
// spins always sort before the window spins, wherever the window sits.  Compiled shapes form the
// thread's local base and global offset from it with a few bit operations instead of reading
// the per-group table; the host launches them only when this layout equals the table's.
template <int TB, int RB, int ES> struct StaticIO {
    uint8_t bits[16];
    __host__ __device__ constexpr StaticIO(int h, int io_chunk) : bits{}
    {
        const int W = io_chunk == 0 ? 0 : (RB < TB - RB ? RB : TB - RB);
        int tb[32] = {};
        int ntb = 0;
        for (int l = h; l < TB; l++)      // the lowest spins (global positions 0 .. TB - h - 1)
            if (l < W || l >= W + RB)
                tb[ntb++] = l;
        for (int l = 0; l < h; l++)       // then the window spins
            if (l < W || l >= W + RB)
                tb[ntb++] = l;
        int set[5] = {}, lanes[32] = {};
        bool in_set[32] = {}, in_lanes[32] = {};
        int ns = 0, seen = 0;
        for (int i = 0; i < ntb && ns < 5; i++)
            if (tb[i] >= h) {
                set[ns++] = tb[i];
                in_set[tb[i]] = true;
                seen |= contrib(tb[i]);
            }
        for (int i = 0; i < ntb; i++)
            if (ns < 5 && !in_set[tb[i]] && contrib(tb[i]) && !(seen & contrib(tb[i]))) {
                set[ns++] = tb[i];
                in_set[tb[i]] = true;
                seen |= contrib(tb[i]);
            }
        for (int i = 0; i < ntb; i++)
            if (ns < 5 && !in_set[tb[i]]) {
                set[ns++] = tb[i];
                in_set[tb[i]] = true;
            }
        const int need = ES == 8 ? 4 : 3;
        int n = 0, got = 0;
        for (int i = 0; i < ns; i++)
            if (n < need && contrib(set[i]) && !(got & contrib(set[i]))) {
                lanes[n++] = set[i];
                in_lanes[set[i]] = true;
                got |= contrib(set[i]);
            }
        for (int i = 0; i < ns; i++)
            if (!in_lanes[set[i]]) {
                lanes[n++] = set[i];
                in_lanes[set[i]] = true;
            }
        for (int l = 0; l < TB; l++)
            if ((l < W || l >= W + RB) && !in_lanes[l])
                lanes[n++] = l;
        for (int i = 0; i < n && i < 16; i++)
            bits[i] = (uint8_t)lanes[i];
    }
    static __host__ __device__ constexpr int contrib(int k)
    {
        const uint32_t e = 1u << k;
        const uint32_t p = ES == 8 ? e + (e >> 5) + (e >> 10) : e + (e >> 4) + (e >> 8);
        return (int)(p & (ES == 8 ? 15u : 7u));
    }
    // host check against the layout the schedule built
    bool equals(const uint8_t *b) const
    {
        for (int t = 0; t < TB - RB; t++)
            if (bits[t] != b[t])
                return false;
        return true;
    }
};
struct RuntimeShape {};
template <typename T> struct TypeTag {
    using type = T;
};

// Host check: does the pass described by (kio, steps) have shape SH?
template <int I, typename... S> struct ShapeMatch;
template <int I> struct ShapeMatch<I> {
    static bool ok(const StepDesc *) { return true; }
};
template <int I, typename S0, typename... S> struct ShapeMatch<I, S0, S...> {
    static bool ok(const StepDesc *d)
    {
        return d[I].k == S0::K && d[I].r0lo == S0::R0LO && d[I].r0hi == S0::R0HI && d[I].ph == S0::PH &&
               d[I].r1lo == S0::R1LO && d[I].r1hi == S0::R1HI && ShapeMatch<I + 1, S...>::ok(d);
    }
};
template <typename SH> struct ShapeOf;
template <int KIO, typename... S> struct ShapeOf<PassShape<KIO, S...>> {
    static bool matches(int kio, int nsteps, const StepDesc *d)
    {
        return kio == KIO && nsteps == (int)sizeof...(S) && ShapeMatch<0, S...>::ok(d);
    }
};

template <typename R, int TB, int RB> struct TileKernel {
    using C = typename CT<R>::T;
    static constexpr int ES = sizeof(C);
    static constexpr int NT = 1 << (TB - RB);
    static constexpr int NR = 1 << RB;
    static constexpr int NTB = TB - RB;                // thread bits
    static constexpr int NCH = (TB + RB - 1) / RB;     // chunks
    static constexpr uint32_t SMEM_ELEMS = padidx<ES>((1u << TB) - 1) + 1;

    // local base index of this thread in chunk layout K (K != 1)
    template <int K> static __device__ __forceinline__ uint32_t chunk_base(uint32_t tid)
    {
        constexpr ChunkLayout<TB, RB, ES> L(chunk_w<TB, RB>(K));
        uint32_t b = 0;
#pragma unroll
        for (int t = 0; t < NTB; t++)
            b |= ((tid >> t) & 1u) << L.bits[t];
        return b;
    }

    // register j of layout K lives at pbase + P(j << W): a compile-time offset per j
    template <int K, int... J>
    static __device__ __forceinline__ void store_seq(C *sm, uint32_t pbase, const C (&x)[NR],
                                                     std::integer_sequence<int, J...>)
    {
        constexpr int W = chunk_w<TB, RB>(K);
        ((sm[pbase + padidx<ES>((uint32_t)J << W)] = x[J]), ...);
    }
    template <int K, int... J>
    static __device__ __forceinline__ void load_seq(const C *sm, uint32_t pbase, C (&x)[NR],
                                                    std::integer_sequence<int, J...>)
    {
        constexpr int W = chunk_w<TB, RB>(K);
        ((x[J] = sm[pbase + padidx<ES>((uint32_t)J << W)]), ...);
    }
    // global index of register J in the I/O layout: the thread's index with the bits of
    // the register window (offsets gst[b]) that J sets
    template <int J>
    static __device__ __forceinline__ uint64_t gidx(uint64_t gthr, const uint64_t (&gst)[RB])
    {
        uint64_t gi = gthr;
#pragma unroll
        for (int b = 0; b < RB; b++)
            if ((J >> b) & 1)
                gi |= gst[b];
        return gi;
    }
    // loads of the tile: streaming (__ldcs), or through L2 only (__ldcg) when the data were
    // written by other thread blocks of the same launch (the persistent ensemble kernel), so
    // that no stale L1 line can be hit
    template <bool CG> static __device__ __forceinline__ C ld_amp(const C *p)
    {
        if constexpr (CG)
            return __ldcg(p);
        else
            return __ldcs(p);
    }
    template <bool CG, int... J>
    static __device__ __forceinline__ void gload(const C *__restrict__ psi, uint64_t gthr, const uint64_t (&gst)[RB],
                                                 C (&x)[NR], std::integer_sequence<int, J...>)
    {
        ((x[J] = ld_amp<CG>(psi + gidx<J>(gthr, gst))), ...);
    }
    template <int... J>
    static __device__ __forceinline__ void gstore(C *__restrict__ psi, uint64_t gthr, const uint64_t (&gst)[RB],
                                                  const C (&x)[NR], std::integer_sequence<int, J...>)
    {
        (__stcs(psi + gidx<J>(gthr, gst), x[J]), ...);
    }
    // the same with 32-bit element offsets from the thread's base pointer (states of at
    // most 2^32 amplitudes): one integer add tree and one wide multiply-add per address
    template <int J> static __device__ __forceinline__ uint32_t goff32(const uint32_t (&gst)[RB])
    {
        uint32_t o = 0;
#pragma unroll
        for (int b = 0; b < RB; b++)
            if ((J >> b) & 1)
                o += gst[b];
        return o;
    }
    template <bool CG, int... J>
    static __device__ __forceinline__ void gload32(const C *__restrict__ p, const uint32_t (&gst)[RB], C (&x)[NR],
                                                   std::integer_sequence<int, J...>)
    {
        ((x[J] = ld_amp<CG>(p + goff32<J>(gst))), ...);
    }
    template <int... J>
    static __device__ __forceinline__ void gstore32(C *__restrict__ p, const uint32_t (&gst)[RB], const C (&x)[NR],
                                                    std::integer_sequence<int, J...>)
    {
        (__stcs(p + goff32<J>(gst), x[J]), ...);
    }
    template <int K> static __device__ __forceinline__ void store_chunk(C *sm, uint32_t pbase, const C (&x)[NR])
    {
        store_seq<K>(sm, pbase, x, std::make_integer_sequence<int, NR>{});
    }
    template <int K> static __device__ __forceinline__ void load_chunk(const C *sm, uint32_t pbase, C (&x)[NR])
    {
        load_seq<K>(sm, pbase, x, std::make_integer_sequence<int, NR>{});
    }

    static __device__ __forceinline__ void apply_slot(C (&x)[NR], const TileShared<R, TB, RB> &sh, int mode)
    {
        if constexpr (sizeof(R) == 4)
            slot_c64<RB>(x, sh.th_f, threadIdx.x, sh.Q, mode);
        else
            slot_c128(x, sh.th_f, threadIdx.x, sh.Q);
    }
    // MODE >= 0: the complex64 factor's series form fixed at compile time
    template <int MODE>
    static __device__ __forceinline__ void apply_slot_m(C (&x)[NR], const TileShared<R, TB, RB> &sh, int mode)
    {
        if constexpr (sizeof(R) == 4 && MODE >= 0)
            slot_c64_apply<RB, MODE>(x, sh.th_f, threadIdx.x, sh.Q);
        else
            apply_slot(x, sh, mode);
    }

    // the steps of a compile-time shape (see PassShape), from layout CUR; back to KIO at the end.
    // FIRST: no transpose yet in this pass.  The transpose buffer has then been untouched since
    // the barrier that ends the pass's prologue (and, in a persistent kernel, since the barrier
    // between tiles), so the first transpose needs no barrier before its stores.
    template <int CUR, int KIO, bool SLOT, int MODE, bool FIRST, typename BaseOf, typename SH>
    static __device__ __forceinline__ void run_shape(C (&x)[NR], C *sm, const BaseOf &base_of, const SH &sh, int mode)
    {
        if constexpr (CUR != KIO) {
            if constexpr (!FIRST)
                __syncthreads();
            store_chunk<CUR>(sm, padidx<ES>(base_of(CUR)), x);
            __syncthreads();
            load_chunk<KIO>(sm, padidx<ES>(base_of(KIO)), x);
        }
    }
    template <int CUR, int KIO, bool SLOT, int MODE, bool FIRST, typename BaseOf, typename SH, typename S0,
              typename... Rest>
    static __device__ __forceinline__ void run_shape(C (&x)[NR], C *sm, const BaseOf &base_of, const SH &sh, int mode)
    {
        if constexpr (S0::K != CUR) {
            if constexpr (!FIRST)
                __syncthreads();
            store_chunk<CUR>(sm, padidx<ES>(base_of(CUR)), x);
            __syncthreads();
            load_chunk<S0::K>(sm, padidx<ES>(base_of(S0::K)), x);
        }
        wht_fixed<S0::R0LO, S0::R0HI>(x);
        if constexpr (SLOT && S0::PH)
            apply_slot_m<MODE>(x, sh, mode);
        wht_fixed<S0::R1LO, S0::R1HI>(x);
        run_shape<S0::K, KIO, SLOT, MODE, FIRST && (S0::K == CUR), BaseOf, SH, Rest...>(x, sm, base_of, sh, mode);
    }
    template <bool SLOT, int MODE, typename BaseOf, typename SH, int KIO, typename... S>
    static __device__ __forceinline__ void run_pass_shape(C (&x)[NR], C *sm, const BaseOf &base_of, const SH &sh,
                                                          int mode, PassShape<KIO, S...>)
    {
        run_shape<KIO, KIO, SLOT, MODE, true, BaseOf, SH, S...>(x, sm, base_of, sh, mode);
    }
};

// One tile f of the state psi through the pass described by a.
// SLOT = false compiles a pass without a slot (the middle passes): no slot tables, no
// per-thread factors in shared memory, fewer registers, so more blocks per SM.
// CG = true loads the tile through L2 only (see ld_amp).
template <typename SH> struct ShapeTraits {
    static constexpr bool runtime = false;
    static constexpr int KIO = SH::KIO, KPH = SH::KPH;
};
template <> struct ShapeTraits<RuntimeShape> {
    static constexpr bool runtime = true;
    static constexpr int KIO = 0, KPH = 0;
};

// SHAPE: RuntimeShape follows a.steps at run time; a PassShape compiles the pass's steps (the
// caller launches it only for passes of that shape, which always carry the slot when SLOT).
// MODE (the complex64 factor's series form, a.exact_sincos) and NARROW (32-bit element offsets,
// N <= 32) are fixed at compile time when >= 0, read from a otherwise.
// sh_ext: shared-memory slot state provided by the caller (a kernel that inlines several builds
// of this function passes one block so that each build does not reserve its own); NULL = own.
template <typename R, int TB, int RB, bool SLOT, bool CG = false, typename SHAPE = RuntimeShape, int MODE = -1,
          int NARROW = -1, bool EXT_SH = false>
__device__ __forceinline__ void tile_pass(typename CT<R>::T *__restrict__ psi, const TileArgs &a,
                                          const TileTab<R, TB, RB> *__restrict__ tabs, uint64_t f,
                                          void *sh_ext = nullptr)
{
    using K = TileKernel<R, TB, RB>;
    using C = typename CT<R>::T;
    using ST = ShapeTraits<SHAPE>;
    constexpr int NR = K::NR, ES = K::ES;
    const int kio = ST::runtime ? a.io.chunk : ST::KIO;
    const bool has_slot = ST::runtime ? (a.has_slot != 0) : SLOT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *sm = reinterpret_cast<C *>(smem_raw);
    using TSH = typename std::conditional<SLOT, TileShared<R, TB, RB>, char>::type;
    __shared__ typename std::conditional<EXT_SH, char, TSH>::type sh_store;
    TSH &sh = EXT_SH ? *reinterpret_cast<TSH *>(sh_ext) : reinterpret_cast<TSH &>(sh_store);

    const uint32_t tid = threadIdx.x;
    const int c = a.c, w = a.w, h = a.h;
    const uint64_t gbase = tile_global_index(c, w, h, f, 0);

    // ---- the slot's per-block terms and per-pass tables: a few words per thread,
    // requested before the tile so that they do not queue behind its loads
    static_assert(TB <= 32 && K::NT > 32, "prologue thread mapping");
    R gv = R(0), tp = R(0), tc[RB];
    double thv = 0.0;
    C qv = C();
#pragma unroll
    for (int b = 0; b < RB; b++)
        tc[b] = R(0);
    if constexpr (SLOT) {
        if (has_slot) {
            const TileTab<R, TB, RB> *tb = tabs + a.tab;
            if (tid < TB)
                gv = static_cast<const R *>(a.gfield)[f * TB + tid];
            if (tid == 32)
                thv = a.theta[f];
            tp = tb->TP[tid];
#pragma unroll
            for (int b = 0; b < RB; b++)
                tc[b] = tb->TC[b][tid];
            if (tid < NR)
                qv = tb->QK[tid];
        }
    }

    // ---- I/O layout: this thread's local base and global offset (host table) and the
    // global offsets of the register bits
    uint32_t base_io;
    uint64_t gthr;
    if constexpr (!ST::runtime) {
        // compiled shape: the I/O layout is known at compile time (StaticIO); the local base is
        // a scatter of the thread index, its global offset the window bits shifted to w and the
        // lowest spins below them
        constexpr int H = SHAPE::template h<TB, RB>();
        constexpr StaticIO<TB, RB, ES> sio(H, SHAPE::KIO);
        uint32_t bl = 0;
#pragma unroll
        for (int t = 0; t < K::NTB; t++)
            bl |= ((tid >> t) & 1u) << sio.bits[t];
        base_io = bl;
        gthr = gbase | ((uint64_t)(bl & ((1u << H) - 1u)) << w) | (uint64_t)(bl >> H);
    } else {
        const uint4 iom = a.iomap[tid];
        base_io = iom.z;
        gthr = gbase | ((uint64_t)iom.y << 32 | iom.x);
    }
    uint64_t gst[RB];
#pragma unroll
    for (int b = 0; b < RB; b++)
        gst[b] = a.gst[b];

    const uint32_t b0 = kio == 0 ? base_io : K::template chunk_base<0>(tid);
    const uint32_t b1 = kio == 1 ? base_io : K::template chunk_base<1>(tid);
    const uint32_t b2 = (K::NCH > 2) ? K::template chunk_base<2>(tid) : 0u;
    const uint32_t b3 = (K::NCH > 3) ? K::template chunk_base<3>(tid) : 0u;
    auto base_of = [&](int k) { return k == 0 ? b0 : k == 1 ? b1 : k == 2 ? b2 : b3; };
    // ---- issue the tile's loads first: the slot set-up below runs under their latency
    const bool narrow = NARROW >= 0 ? (NARROW != 0) : (a.ham.N <= 32);   // element offsets fit in 32 bits
    uint32_t gst32[RB];
#pragma unroll
    for (int b = 0; b < RB; b++)
        gst32[b] = (uint32_t)gst[b];
    C x[NR];
    if (narrow)
        K::template gload32<CG>(psi + gthr, gst32, x, std::make_integer_sequence<int, NR>{});
    else
        K::template gload<CG>(psi, gthr, gst, x, std::make_integer_sequence<int, NR>{});

    // ---- per-block part of the slot into shared memory
    int pcq = 0;
    R scale = R(1);
    float srel = 0.0f;                 // exact scale / rounded scale - 1 (c64: sqrt 1/2 is not exact)
    const int mode = MODE >= 0 ? MODE : a.exact_sincos;   // c64 factor: 0 tiny |y|, 1 small |y|, 2 any
    if constexpr (SLOT) {
        if (has_slot) {
            pcq = a.slot.pcq;
            if constexpr (sizeof(R) == 4) {
                scale = a.slot.scale_f;
                srel = a.slot.srel;
            } else {
                scale = a.slot.scale;
            }
            if (tid < TB)
                sh.g[tid] = gv;
            if (tid == 32) {
                sh.th = thv;
                sh.th_hi = (float)thv;
                sh.th_lo = (float)(thv - (double)(float)thv);
                sh.pcF = __popcll(gbase);
            }
            if (tid < NR)
                sh.Q[tid] = qv;
        }
    }
    __syncthreads();

    // ---- per-thread slot factors, computed before the tile occupies the registers
    if constexpr (SLOT) {
        if (has_slot) {
            int kph = ST::KPH;
            if constexpr (ST::runtime) {
                for (int s = 0; s < a.nsteps; s++)
                    if (a.steps[s].ph)
                        kph = a.steps[s].k;
            }
            if constexpr (sizeof(R) == 4) {
                SlotThreadC64<RB> o;
                slot_thread_c64<TB, RB>(o, base_of(kph), kph, sh, pcq, (float)scale, srel, tp, tc);
                sh.th_f.put(tid, o);
            } else {
                SlotThreadC128 o;
                slot_thread_c128<TB, RB>(o, base_of(kph), chunk_w<TB, RB>(kph), sh, pcq, (double)scale, tp, tc);
                sh.th_f.put(tid, o);
            }
        }
    }

    // ---- steps: transpose to the step's chunk layout when it changes
    if constexpr (!ST::runtime) {
        K::template run_pass_shape<SLOT, MODE>(x, sm, base_of, sh, mode, SHAPE{});
    } else {
    int cur = kio;
    for (int s = 0; s < a.nsteps; s++) {
        const StepDesc d = a.steps[s];
        const int k = d.k;
        if (k != cur) {
            __syncthreads();
            const uint32_t pc = padidx<ES>(base_of(cur));
            switch (cur) {
            case 0: K::template store_chunk<0>(sm, pc, x); break;
            case 1: K::template store_chunk<1>(sm, pc, x); break;
            case 2: K::template store_chunk<2>(sm, pc, x); break;
            default: K::template store_chunk<3>(sm, pc, x); break;
            }
            __syncthreads();
            const uint32_t pn = padidx<ES>(base_of(k));
            switch (k) {
            case 0: K::template load_chunk<0>(sm, pn, x); break;
            case 1: K::template load_chunk<1>(sm, pn, x); break;
            case 2: K::template load_chunk<2>(sm, pn, x); break;
            default: K::template load_chunk<3>(sm, pn, x); break;
            }
            cur = k;
        }
        wht_regs<RB>(x, d.r0lo, d.r0hi);
        if constexpr (SLOT) {
            if (d.ph)
                K::apply_slot(x, sh, mode);
        }
        wht_regs<RB>(x, d.r1lo, d.r1hi);
    }
    if (cur != kio) {
        __syncthreads();
        const uint32_t pc = padidx<ES>(base_of(cur));
        switch (cur) {
        case 0: K::template store_chunk<0>(sm, pc, x); break;
        case 1: K::template store_chunk<1>(sm, pc, x); break;
        case 2: K::template store_chunk<2>(sm, pc, x); break;
        default: K::template store_chunk<3>(sm, pc, x); break;
        }
        __syncthreads();
        if (kio == 0)
            K::template load_chunk<0>(sm, padidx<ES>(base_io), x);
        else
            K::template load_chunk<1>(sm, padidx<ES>(base_io), x);
    }
    }

    // ---- store in the I/O layout
    // (opaque copies: keeps the compiler from holding the 2^RB load addresses live
    // across the whole pass)
    asm volatile("mov.b64 %0, %0;" : "+l"(gthr));
    if (narrow) {
#pragma unroll
        for (int b = 0; b < RB; b++)
            asm volatile("mov.b32 %0, %0;" : "+r"(gst32[b]));
        K::gstore32(psi + gthr, gst32, x, std::make_integer_sequence<int, NR>{});
    } else {
#pragma unroll
        for (int b = 0; b < RB; b++)
            asm volatile("mov.b64 %0, %0;" : "+l"(gst[b]));
        K::gstore(psi, gthr, gst, x, std::make_integer_sequence<int, NR>{});
    }
}

// Resident blocks per SM the register allocation is sized for: about twice the tile's
// registers per thread, i.e. 4 blocks of 128 threads (c64, 32 amplitudes, 128 registers),
// 4 blocks of 256 threads (c64, 16 amplitudes, 64 registers), 2 blocks of 256 threads
// (c128, 16 amplitudes, 128 registers), ... within the SM's 64K registers.
__host__ __device__ constexpr int tile_min_blocks(int thread_bits, int reg_elems)
{
    // 2^RB amplitudes per thread take reg_elems = 2^RB x (8 or 16 bytes) / 4 registers;
    // budget about twice that per thread
    return (65536 / (2 * reg_elems)) >> thread_bits > 0 ? (65536 / (2 * reg_elems)) >> thread_bits : 1;
}

template <typename R, int TB, int RB, bool SLOT, typename SHAPE = RuntimeShape, int MODE = -1, int NARROW = -1>
__global__ void __launch_bounds__(1 << (TB - RB), tile_min_blocks(TB - RB, (int)(sizeof(typename CT<R>::T) / 4) << RB))
k_tile(typename CT<R>::T *__restrict__ psi, const __grid_constant__ TileArgs a,
       const TileTab<R, TB, RB> *__restrict__ tabs)
{
    tile_pass<R, TB, RB, SLOT, false, SHAPE, MODE, NARROW>(psi, a, tabs, blockIdx.x);
}

// Launch of a pass through a compiled shape (ts4_shapes_*.cu): returns false if no compiled
// shape of this tile matches the pass, else launches it and sets *err.
template <typename R, int TB, int RB>
bool launch_shaped(cudaStream_t st, void *psi, const TileArgs &a, const void *tabs, uint64_t nblk, cudaError_t *err)
{
    return false;
}
template <> bool launch_shaped<float, 12, 5>(cudaStream_t, void *, const TileArgs &, const void *, uint64_t, cudaError_t *);
template <> bool launch_shaped<double, 12, 4>(cudaStream_t, void *, const TileArgs &, const void *, uint64_t, cudaError_t *);

// Host: the pass's group has the window size of SHAPE and the I/O layout StaticIO gives it, so the
// compiled build may form its I/O addresses without the table.
template <typename R, int TB, int RB, typename SHAPE> bool shape_io_ok(const TileArgs &a)
{
    constexpr int H = SHAPE::template h<TB, RB>();
    constexpr int ES = (int)sizeof(typename CT<R>::T);
    if (a.h != H || a.c != TB - H)
        return false;
    const StaticIO<TB, RB, ES> sio(H, SHAPE::KIO);
    return sio.equals(a.io.bits);
}

// One compiled shape: launches k_tile<..., SHAPE, MODE, NARROW> if the pass has that shape, that
// slot-factor form (MODE, slot passes of complex64 only; -1 = any) and that offset width
// (NARROW: 1 for N <= 32, 0 above).
template <typename R, int TB, int RB, bool SLOT, typename SHAPE, int MODE = -1, int NARROW = 1>
bool launch_if_shape(cudaStream_t st, void *psi, const TileArgs &a, const void *tabs, uint64_t nblk, cudaError_t *err)
{
    if ((a.has_slot != 0) != SLOT || !ShapeOf<SHAPE>::matches(a.io.chunk, a.nsteps, a.steps))
        return false;
    if ((MODE >= 0 && a.exact_sincos != MODE) || ((a.ham.N <= 32) != (NARROW != 0)))
        return false;
    if (!shape_io_ok<R, TB, RB, SHAPE>(a))
        return false;
    using K = TileKernel<R, TB, RB>;
    constexpr size_t smem = sizeof(typename CT<R>::T) * K::SMEM_ELEMS;
    cudaError_t e = cudaFuncSetAttribute(k_tile<R, TB, RB, SLOT, SHAPE, MODE, NARROW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        k_tile<R, TB, RB, SLOT, SHAPE, MODE, NARROW><<<(unsigned)nblk, K::NT, smem, st>>>(
            (typename CT<R>::T *)psi, a, (const TileTab<R, TB, RB> *)tabs);
        e = cudaGetLastError();
    }
    *err = e;
    return true;
}

// Compiled shapes the ensemble kernel dispatches to (complex64, 12-bit tiles): the slot passes
// of two bit groups, i.e. of the 12 lowest spins and of windows of 4, 6, 8 and 10 spins (the
// systems of N = 16, 18, 20, 22 with 2 coalescing spins).  ens_shape: 1 + the index in this list.
namespace ens {
using Low12 = PassShape<1, Step<1, 0, 5, 0, 0, 0>, Step<0, 0, 5, 0, 0, 0>, Step<2, 3, 5, 1, 3, 5>,
                        Step<0, 0, 0, 0, 0, 5>, Step<1, 0, 0, 0, 0, 5>>;
using Win4 = PassShape<0, Step<0, 0, 4, 1, 0, 4>>;
using Win6 = PassShape<0, Step<0, 0, 5, 0, 0, 0>, Step<1, 0, 1, 1, 0, 1>, Step<0, 0, 0, 0, 0, 5>>;
using Win8 = PassShape<0, Step<0, 0, 5, 0, 0, 0>, Step<1, 0, 3, 1, 0, 3>, Step<0, 0, 0, 0, 0, 5>>;
using Win10 = PassShape<0, Step<0, 0, 5, 0, 0, 0>, Step<1, 0, 5, 1, 0, 5>, Step<0, 0, 0, 0, 0, 5>>;
} // namespace ens

// Host: the ensemble shape of a complex64 12-bit pass (0 if none), N <= 32 and a slot required.
inline int ensemble_shape_id(const TileArgs &a)
{
    if (!a.has_slot || a.ham.N > 32)
        return 0;
    auto ok = [&](auto tag) {
        using SH = typename decltype(tag)::type;
        return ShapeOf<SH>::matches(a.io.chunk, a.nsteps, a.steps) && shape_io_ok<float, 12, 5, SH>(a);
    };
    if (ok(TypeTag<ens::Low12>{}))
        return 1;
    if (ok(TypeTag<ens::Win4>{}))
        return 2;
    if (ok(TypeTag<ens::Win6>{}))
        return 3;
    if (ok(TypeTag<ens::Win8>{}))
        return 4;
    if (ok(TypeTag<ens::Win10>{}))
        return 5;
    return 0;
}

// Persistent ensemble kernel: every pass of every state of every system of a batch in one
// launch (the typical-state ensembles of App. A).
//
// Work items are chunks of up to 2^chunk_shift tiles of one state in one pass, in pass-major
// order: all items of pass p of every state come before any item of pass p + 1.  A block takes
// the next item from a global ticket counter (it fetches its following ticket as soon as it
// starts an item, so that the atomic's latency hides behind the item's tiles).  A tile of pass
// p reads amplitudes that every tile of pass p - 1 of its state wrote (the passes rotate
// different bit groups), so an item first waits until its state's counter of completed tiles
// reaches p x (tiles per pass); after its tiles the block adds their number.  A block only
// waits for items with smaller tickets, and the smallest unfinished ticket is always held by a
// block that is working on it (a block holding a fetched-ahead ticket is still working on a
// smaller one), so the launch always progresses, whatever the number of resident blocks.
// Every wait is bounded in time (%globaltimer): when it runs out, the block sets the sticky
// status word and returns, and every other block returns before its next item, so the launch
// ends and the host reports TS_ERR_TIMEOUT.
struct BatchSys {
    void *psi;           // nstates x 2^n amplitudes
    const void *tabs;    // this system's per-slot tables
    int n;
    int tile_shift;      // log2 tiles per state
    int chunk_shift;     // log2 tiles per work item (<= tile_shift)
    uint32_t block_start; // first work item of this system within its pass
    uint32_t state_base;  // index of the system's first state among all states of the batch
    int active;          // 0: this system has no pass at this index
};

struct BatchSync {
    unsigned long long *ticket;   // next work item (zero at launch)
    unsigned long long *done;     // per state: tiles completed, over all passes (zero at launch)
    int *status;                  // sticky: nonzero after a dependency wait ran out
    const int *hold_flag;         // a device word that nothing writes (test of the timeout path)
    const uint64_t *pstart;       // first work item of each pass; pstart[npass] = all items
    uint64_t limit_ns;            // longest dependency wait
    int npass;
    int hold;                     // nonzero: every wait also waits for *hold_flag (never set)
};

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits until *cnt >= need (and, with sy.hold, for the flag nothing sets).  Bounded: gives up
// after sy.limit_ns nanoseconds or 2^22 polls (at most ~9 s with the 2 us back-off), or as
// soon as another block gave up.
__device__ __forceinline__ bool wait_count(const unsigned long long *cnt, unsigned long long need, const BatchSync &sy)
{
    const uint64_t t0 = global_ns();
    unsigned sleep_ns = 32;
    for (uint32_t it = 0; it < (1u << 22); it++) {
        const unsigned long long v = *(volatile const unsigned long long *)cnt;
        if (v >= need && !(sy.hold && *(volatile const int *)sy.hold_flag == 0)) {
            __threadfence();   // acquire: the counted tiles' stores are visible from here on
            return true;
        }
        if (*(volatile const int *)sy.status != 0)
            return false;
        if (global_ns() - t0 > sy.limit_ns)
            break;
        __nanosleep(sleep_ns);
        if (sleep_ns < 2048)
            sleep_ns *= 2;
    }
    atomicExch(sy.status, 1);
    return false;
}

template <typename R, int TB, int RB>
__global__ void __launch_bounds__(1 << (TB - RB), tile_min_blocks(TB - RB, (int)(sizeof(typename CT<R>::T) / 4) << RB))
k_tile_ensemble(const BatchSys *__restrict__ sys, const TileArgs *__restrict__ args, int nsys, const BatchSync sy)
{
    __shared__ int w_go, w_pass, w_sys, w_ntiles;
    __shared__ uint32_t w_state;
    __shared__ uint64_t w_tile0;
    __shared__ TileShared<R, TB, RB> sh_ens;   // slot state shared by the inlined pass builds
    const uint64_t total = sy.pstart[sy.npass];
    unsigned long long next = 0;   // thread 0: the ticket fetched ahead
    int pass_hint = 0;             // thread 0: tickets only grow, so the pass search starts here
    if (threadIdx.x == 0)
        next = atomicAdd(sy.ticket, 1ull);
    for (;;) {
        __syncthreads();   // the previous item's shared-memory reads are done
        if (threadIdx.x == 0) {
            int go = 0;
            const unsigned long long t = next;
            if (t < total && *(volatile const int *)sy.status == 0) {
                next = atomicAdd(sy.ticket, 1ull);
                int p = pass_hint;
                while (p + 1 < sy.npass && sy.pstart[p + 1] <= t)
                    p++;
                pass_hint = p;
                const BatchSys *row = sys + (size_t)p * nsys;
                const uint32_t local = (uint32_t)(t - sy.pstart[p]);
                int s = 0;
                while (s + 1 < nsys && row[s + 1].block_start <= local)
                    s++;
                if (row[s].active) {
                    const int per_state = row[s].tile_shift - row[s].chunk_shift;   // log2 items per state
                    const uint32_t li = local - row[s].block_start;
                    const uint32_t state = li >> per_state;
                    w_pass = p;
                    w_sys = s;
                    w_state = state;
                    w_tile0 = (uint64_t)(li & ((1u << per_state) - 1u)) << row[s].chunk_shift;
                    w_ntiles = 1 << row[s].chunk_shift;
                    const unsigned long long need = (unsigned long long)p << row[s].tile_shift;
                    go = wait_count(sy.done + row[s].state_base + state, need, sy) ? 1 : 0;
                }
            }
            w_go = go;
        }
        __syncthreads();
        if (!w_go)
            return;
        const int p = w_pass, s = w_sys, nt = w_ntiles;
        const uint32_t state = w_state;
        const uint64_t f0 = w_tile0;
        const BatchSys &bs = sys[(size_t)p * nsys + s];
        typename CT<R>::T *psi = reinterpret_cast<typename CT<R>::T *>(bs.psi) + ((uint64_t)state << bs.n);
        const TileArgs &a = args[(size_t)p * nsys + s];
        const TileTab<R, TB, RB> *tabs = reinterpret_cast<const TileTab<R, TB, RB> *>(bs.tabs);
        // a pass without a slot (the middle passes of three or more bit groups) runs the code
        // path compiled without the slot machinery, as ts_step's separate kernel build does;
        // complex64 12-bit passes of a compiled shape run that build (ens_shape)
        auto tiles = [&](auto shape_tag) {
            using SH = typename decltype(shape_tag)::type;
            for (int k = 0; k < nt; k++) {
                if (k)
                    __syncthreads();
                tile_pass<R, TB, RB, true, true, SH, -1, 1, true>(psi, a, tabs, f0 + k, &sh_ens);
            }
        };
        bool done_shape = false;
        if constexpr (sizeof(R) == 4 && TB == 12 && RB == 5) {
            done_shape = true;
            switch (a.ens_shape) {
            case 1: tiles(TypeTag<ens::Low12>{}); break;
            case 2: tiles(TypeTag<ens::Win4>{}); break;
            case 3: tiles(TypeTag<ens::Win6>{}); break;
            case 4: tiles(TypeTag<ens::Win8>{}); break;
            case 5: tiles(TypeTag<ens::Win10>{}); break;
            default: done_shape = false; break;
            }
        }
        if (done_shape) {
        } else if (a.has_slot) {
            for (int k = 0; k < nt; k++) {
                if (k)
                    __syncthreads();   // the previous tile's shared-memory reads are done
                tile_pass<R, TB, RB, true, true, RuntimeShape, -1, -1, true>(psi, a, tabs, f0 + k, &sh_ens);
            }
        } else {
            for (int k = 0; k < nt; k++) {
                if (k)
                    __syncthreads();
                tile_pass<R, TB, RB, false, true>(psi, a, tabs, f0 + k);
            }
        }
        __syncthreads();   // every thread's stores come before thread 0's fence and count
        if (threadIdx.x == 0) {
            __threadfence();   // release (cumulative over the block's stores seen at the barrier)
            atomicAdd(sy.done + bs.state_base + state, (unsigned long long)nt);
        }
    }
}

} // namespace ts4
