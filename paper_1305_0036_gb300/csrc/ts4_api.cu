// Host side of the TS4 library: the C ABI of include/ts4.h, the context, the
// schedule builder (slots and bit-group passes) and the launches.
//
// Schedule (Sec. 2 and Secs. 3.3-3.4):
//   * ts_step expands U4(tau)^n into L = 20 n Walsh-Hadamard layers and L + 1
//     diagonal slots (see ts4_common.cuh for the slot algebra).
//   * The fused kernel covers the N spins with g bit groups: G_1 = the TB
//     lowest spins, then windows of at most TB - s higher spins, each tile also
//     keeping the s lowest spins so that it reads runs of 2^s consecutive
//     amplitudes (Sec. 3.4, "coalescing").  A layer is done when every group
//     has been rotated; the slot that follows is applied inside the pass of the
//     layer's last group, which then starts the next layer on the same group
//     (groups are visited in alternating order).  Passes per chained TS4 step:
//     20 (g - 1).
#include "../../include/ts4.h"
#include "ts4_tile.cuh"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <map>
#include <string>
#include <tuple>
#include <vector>

using namespace ts4;

namespace {

struct Buf {
    void *p = nullptr;
    bool own = false;
};

struct HostSlot {
    double t = 0.0, th0 = 0.0, mag = 1.0;
    int alpha = 2, pcq = 0, scale_exp = 0;
    Slot dev() const
    {
        Slot s;
        s.t = t;
        s.th0 = th0;
        s.mag = mag;
        s.alpha = alpha;
        s.pcq = pcq;
        s.scale_exp = scale_exp;
        s.pad = 0;
        s.scale = std::ldexp(mag, -scale_exp);
        s.scale_f = (float)s.scale;
        s.srel = (float)(s.scale / (double)s.scale_f - 1.0);
        return s;
    }
};

struct Group {
    int c, w, h;
};

struct HostPass {
    int group = 0;
    int nsteps = 0;
    StepDesc steps[kMaxSteps];
    int slot = -1;      // slot index or -1
    int phase_k = 0;    // chunk of the step that applies the slot
    int tab = -1;
    int ymode = 0;      // c64 per-amplitude factor: 0 |y| <= 0.05, 1 |y| <= 0.5, 2 sincospif
    size_t theta_off = 0; // first frame of this pass's (slot, group) in Schedule::dtheta / dgfield
};

struct Schedule {
    // key
    int order = 0;
    double tau = 0.0;
    int64_t n = -1;
    int kernel = -1, TB = 0, cbits = 0, slot0_pcq = -1, mode = 0;
    int shape = 0;        // SHAPE_* flags: how the pass list differs from make_passes
    int tail_group = 0;   // SHAPE_TAIL_ONLY: the group of the single pass
    // content
    std::vector<HostSlot> slots;
    std::vector<Group> groups;
    std::vector<IOLayout> io;      // per group
    std::vector<HostPass> passes;
    std::vector<unsigned char> tabs;    // host image of the PassTab array
    size_t tab_size = 0;
    void *dtab = nullptr;                // device copy, owned by this schedule
    size_t dtab_cap = 0;
    std::vector<uint4> iomap;            // per group, per thread: I/O-layout offset and base (host image)
    void *dmap = nullptr;                // device copy
    size_t dmap_cap = 0;                 // bytes
    double *dtheta = nullptr;            // frame angles of every (slot, group), owned by this schedule
    void *dgfield = nullptr;             // fields g_l per frame (TB values of the kernel's precision), same allocation
    size_t dtheta_cap = 0;               // bytes of the allocation
};

// Frees S's device tables once the stream's queued passes (which read them) are done.
void release_tables(Schedule &S, cudaStream_t st)
{
    if (S.dtab || S.dtheta || S.dmap)
        cudaStreamSynchronize(st);
    if (S.dmap)
        cudaFree(S.dmap);
    S.dmap = nullptr;
    S.dmap_cap = 0;
    if (S.dtab)
        cudaFree(S.dtab);
    if (S.dtheta)
        cudaFree(S.dtheta);
    S.dtab = nullptr;
    S.dtab_cap = 0;
    S.dtheta = nullptr;
    S.dgfield = nullptr;
    S.dtheta_cap = 0;
}

// Drops the pass list and tables of S (keeps nothing cached).
void reset_schedule(Schedule &S, cudaStream_t st)
{
    release_tables(S, st);
    S = Schedule();
}

constexpr int kMaxN = 34;
// largest host read-back of one reduction: the joint bit weights of k_sum_pairs
constexpr int kMaxOut = 1 + kMaxN + kMaxN * (kMaxN - 1) / 2;

} // namespace

struct ts_ctx {
    int N = 0;
    ts_prec prec = TS_C64;
    cudaStream_t stream = nullptr;
    int device = 0;
    int sms = 0;
    std::vector<double> Jq;   // [3][N][N] symmetric, J/4
    std::vector<double> hh;   // [3][N], h/2
    std::vector<double> Jraw[3];
    std::vector<double> hraw[3];
    double *dJq = nullptr, *dhh = nullptr;
    void *dE = nullptr;       // phase-table mode: E_x, E_y, E_z per basis state (3 x 2^N doubles for
                              // complex128, floats for complex64), or NULL
    Buf psi, ref, scratch;
    bool ref_valid = false;
    double *dpart = nullptr;
    size_t part_cap = 0;      // doubles
    double *hout = nullptr;   // pinned, kMaxOut doubles
    int kernel = TS_KERNEL_FUSED;
    int TB = 0, RB = 0, cbits = 0;
    Schedule sched;       // last ts_step schedule
    Schedule sched_obs;   // frame rotation used by TS_ENERGY
    // The final pass of the last ts_step (the last layer's rotation of group tail_group, then
    // the P_z slot tail_slot), held back so that the next ts_step runs it inside its first
    // pass, as a chained run does; any use of the state other than the next step or the norm
    // runs it first (flush_tail).
    bool chain = false;   // ts_set_chaining: hold back the final pass of each ts_step
    bool tail_pending = false;
    HostSlot tail_slot;
    int tail_group = 0;
    int tail_h = 0;       // spins that rotation covers: the norm grows by 2^tail_h through it
    Schedule sched_tail;  // that pass alone
    std::string err;
    int64_t launches = 0;
};

namespace {

ts_status fail(ts_ctx *ctx, ts_status st, const std::string &msg)
{
    if (ctx)
        ctx->err = msg;
    return st;
}

ts_status cuda_fail(ts_ctx *ctx, cudaError_t e, const char *where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(ctx, e == cudaErrorMemoryAllocation ? TS_ERR_OOM : TS_ERR_CUDA, m);
}

#define TS_CUDA(ctx, call)                                                                        \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return cuda_fail((ctx), e_, #call);                                                   \
    } while (0)

size_t amp_bytes(const ts_ctx *ctx) { return ctx->prec == TS_C64 ? 8 : 16; }
uint64_t dim_of(const ts_ctx *ctx) { return UINT64_C(1) << ctx->N; }
size_t state_bytes(const ts_ctx *ctx) { return (size_t)dim_of(ctx) * amp_bytes(ctx); }

// ------------------------------------------------------------ kernel shapes

// Register bits per precision and the tile sizes this build provides.
int reg_bits(ts_prec p) { return p == TS_C64 ? 5 : 4; }
bool tile_supported(ts_prec p, int tb)
{
    return p == TS_C64 ? (tb >= 12 && tb <= 14) : (tb >= 11 && tb <= 13);
}
int default_tile(ts_prec) { return 12; }  // fastest at N=28 on GB300 for both precisions (measured)
int default_cbits(ts_prec p) { return p == TS_C64 ? 3 : 2; }

template <typename R, int TB, int RB, bool SLOT, typename SHAPE = RuntimeShape>
cudaError_t launch_tile_s(cudaStream_t st, void *psi, const TileArgs &a, const void *tabs, uint64_t nblk)
{
    using K = TileKernel<R, TB, RB>;
    constexpr size_t smem = sizeof(typename CT<R>::T) * K::SMEM_ELEMS;
    cudaError_t e = cudaFuncSetAttribute(k_tile<R, TB, RB, SLOT, SHAPE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess)
        return e;
    k_tile<R, TB, RB, SLOT, SHAPE><<<(unsigned)nblk, K::NT, smem, st>>>((typename CT<R>::T *)psi, a,
                                                                         (const TileTab<R, TB, RB> *)tabs);
    return cudaGetLastError();
}

// Passes whose shape is compiled (ts4_shapes_*.cu) run that build; the others follow their step
// list at run time.  Passes without a slot run a kernel compiled without the slot machinery.
template <typename R, int TB, int RB>
cudaError_t launch_tile_t(cudaStream_t st, void *psi, const TileArgs &a, const void *tabs, uint64_t nblk)
{
    cudaError_t e = cudaSuccess;
    if (launch_shaped<R, TB, RB>(st, psi, a, tabs, nblk, &e))
        return e;
    return a.has_slot ? launch_tile_s<R, TB, RB, true>(st, psi, a, tabs, nblk)
                      : launch_tile_s<R, TB, RB, false>(st, psi, a, tabs, nblk);
}

cudaError_t launch_tile(const ts_ctx *ctx, int TB, void *psi, const TileArgs &a, const void *tabs, uint64_t nblk)
{
    if (ctx->prec == TS_C64) {
        switch (TB) {
        case 12: return launch_tile_t<float, 12, 5>(ctx->stream, psi, a, tabs, nblk);
        case 13: return launch_tile_t<float, 13, 5>(ctx->stream, psi, a, tabs, nblk);
        default: return launch_tile_t<float, 14, 5>(ctx->stream, psi, a, tabs, nblk);
        }
    }
    switch (TB) {
    case 11: return launch_tile_t<double, 11, 4>(ctx->stream, psi, a, tabs, nblk);
    case 12: return launch_tile_t<double, 12, 4>(ctx->stream, psi, a, tabs, nblk);
    default: return launch_tile_t<double, 13, 4>(ctx->stream, psi, a, tabs, nblk);
    }
}

template <typename R, int TB, int RB> size_t tab_size_t() { return sizeof(PassTab<R, TB, RB>); }

size_t tab_size(ts_prec p, int TB)
{
    if (p == TS_C64) {
        switch (TB) {
        case 12: return tab_size_t<float, 12, 5>();
        case 13: return tab_size_t<float, 13, 5>();
        default: return tab_size_t<float, 14, 5>();
        }
    }
    switch (TB) {
    case 11: return tab_size_t<double, 11, 4>();
    case 12: return tab_size_t<double, 12, 4>();
    default: return tab_size_t<double, 13, 4>();
    }
}

// Host FP64 construction of the per-(slot, group, chunk) tables of the tile kernel
// (PassTab: the couplings among each thread's own bits, TP and TC, and the in-chunk
// table QK).  The thread's bits are those of its base index in the layout of the
// step that applies the slot: the I/O layout when that is the I/O chunk, the
// chunk layout otherwise -- the same mapping from thread index to local bits as the
// kernel's base_of().
template <typename R, int TB, int RB>
void build_tab_t(unsigned char *dst, const ts_ctx *ctx, const HostSlot &sl, const Group &g, const IOLayout &io,
                 int phase_k)
{
    using C = typename CT<R>::T;
    constexpr int NT = 1 << (TB - RB), ES = sizeof(C);
    std::vector<unsigned char> buf(sizeof(PassTab<R, TB, RB>), 0);
    PassTab<R, TB, RB> &tb = *reinterpret_cast<PassTab<R, TB, RB> *>(buf.data());
    const int N = ctx->N;
    const double *Jq = ctx->Jq.data() + (size_t)sl.alpha * N * N;
    auto pos = [&](int l) { return l < g.h ? g.w + l : l - g.h; };
    std::vector<double> A(TB * TB, 0.0);
    for (int l = 0; l < TB; l++)
        for (int m = 0; m < TB; m++)
            if (l != m)
                A[l * TB + m] = sl.t * Jq[pos(l) * N + pos(m)];
    const bool f32 = sizeof(R) == 4;
    const double unit = f32 ? 1.0 : 1.0 / M_PI;
    const int W = chunk_w<TB, RB>(phase_k);
    // thread bits of the slot's layout
    int tbits[TB - RB];
    if (phase_k == io.chunk) {
        for (int t = 0; t < TB - RB; t++)
            tbits[t] = io.bits[t];
    } else {
        const ChunkLayout<TB, RB, ES> L(W);
        for (int t = 0; t < TB - RB; t++)
            tbits[t] = L.bits[t];
    }
    for (int tid = 0; tid < NT; tid++) {
        double sgn[TB - RB];
        for (int t = 0; t < TB - RB; t++)
            sgn[t] = ((tid >> t) & 1) ? 1.0 : -1.0;
        double tp = 0.0;
        for (int u = 0; u < TB - RB; u++)
            for (int v = u + 1; v < TB - RB; v++)
                tp += A[tbits[u] * TB + tbits[v]] * sgn[u] * sgn[v];
        tb.TP[tid] = (R)(tp * unit);
        for (int b = 0; b < RB; b++) {
            double tc = 0.0;
            for (int u = 0; u < TB - RB; u++)
                tc += A[(W + b) * TB + tbits[u]] * sgn[u];
            tb.TC[b][tid] = (R)(tc * unit);
        }
    }
    for (int j = 0; j < (1 << RB); j++) {
        double q = 0.0;
        for (int l = 0; l < RB; l++)
            for (int m = l + 1; m < RB; m++) {
                const double sl_ = ((j >> l) & 1) ? 1.0 : -1.0;
                const double sm_ = ((j >> m) & 1) ? 1.0 : -1.0;
                q += A[(W + l) * TB + (W + m)] * sl_ * sm_;
            }
        C z;
        if (f32) {
            z.x = (R)q;
            z.y = (R)0;
        } else {
            double re = std::cos(q), im = -std::sin(q);
            const int k = (sl.pcq * __builtin_popcount((unsigned)j)) & 3;
            for (int r = 0; r < k; r++) { // multiply by i
                double t = re;
                re = -im;
                im = t;
            }
            z.x = (R)re;
            z.y = (R)im;
        }
        tb.QK[j] = z;
    }
    std::memcpy(dst, buf.data(), buf.size());
}

void build_tab(unsigned char *dst, const ts_ctx *ctx, int TB, const HostSlot &sl, const Group &g, const IOLayout &io,
               int phase_k)
{
    if (ctx->prec == TS_C64) {
        switch (TB) {
        case 12: return build_tab_t<float, 12, 5>(dst, ctx, sl, g, io, phase_k);
        case 13: return build_tab_t<float, 13, 5>(dst, ctx, sl, g, io, phase_k);
        default: return build_tab_t<float, 14, 5>(dst, ctx, sl, g, io, phase_k);
        }
    }
    switch (TB) {
    case 11: return build_tab_t<double, 11, 4>(dst, ctx, sl, g, io, phase_k);
    case 12: return build_tab_t<double, 12, 4>(dst, ctx, sl, g, io, phase_k);
    default: return build_tab_t<double, 13, 4>(dst, ctx, sl, g, io, phase_k);
    }
}

// Upper bound of |y_j| (radians) in the c64 per-amplitude factor of a slot on tile group g:
// every per-thread coefficient is at most |t| (|h/2| + sum |J/4|) of its spin; RB of them
// plus the in-chunk quadratic terms.
// Bound on |y_j|, the per-amplitude remainder of the slot angle in the tile kernel:
// y_j collects the terms of t E_alpha that involve the RB register spins of the
// step that applies the slot (tile bits W .. W + RB - 1 of group g), each with a
// sign, so |y_j| <= |t| sum over those spins of (|hh_i| + sum_m |Jq_im|).
double slot_y_bound(const ts_ctx *ctx, const HostSlot &sl, const Group &g, int TB, int RB, int phase_k)
{
    const int N = ctx->N;
    const double *Jq = ctx->Jq.data() + (size_t)sl.alpha * N * N;
    const double *hh = ctx->hh.data() + (size_t)sl.alpha * N;
    const int W = std::min(phase_k * RB, TB - RB);
    double bound = 0.0;
    for (int b = 0; b < RB; b++) {
        const int l = W + b;
        const int i = l < g.h ? g.w + l : l - g.h;
        double r = std::fabs(hh[i]);
        for (int m = 0; m < N; m++)
            r += std::fabs(Jq[i * N + m]);
        bound += r;
    }
    return std::fabs(sl.t) * bound;
}

// I/O layout of a group.  The 5 lanes must hold the globally lowest bits of the
// tile (the c lowest spins, then window spins when c < 5) so that one warp
// instruction covers consecutive addresses; their order is free, and the first
// 4 (3 for 16-byte amplitudes) are ordered to give distinct shared-memory bank
// contributions, so that the transposes from and to this layout are
// conflict-free whenever the bits allow it.
IOLayout make_io(const Group &g, int TB, int RB, int ES, int io_chunk)
{
    IOLayout io;
    std::memset(&io, 0, sizeof(io));
    io.chunk = io_chunk;
    const int W = io_chunk == 0 ? 0 : (RB < TB - RB ? RB : TB - RB);
    auto gp = [&](int l) { return l < g.h ? g.w + l : l - g.h; };
    auto contrib = [&](int k) {
        const uint32_t e = 1u << k;
        const uint32_t p = ES == 8 ? e + (e >> 5) + (e >> 10) : e + (e >> 4) + (e >> 8);
        return (int)(p & (ES == 8 ? 15u : 7u));
    };
    std::vector<int> tb;
    for (int l = 0; l < TB; l++)
        if (l < W || l >= W + RB)
            tb.push_back(l);
    std::sort(tb.begin(), tb.end(), [&](int a, int b) { return gp(a) < gp(b); });
    auto has = [](const std::vector<int> &v, int l) { return std::find(v.begin(), v.end(), l) != v.end(); };
    // the lane set: contiguous bits first (lowest global positions), then window bits
    // that add new bank contributions, then any
    std::vector<int> set;
    int seen = 0;
    for (int l : tb)
        if (gp(l) < g.c && (int)set.size() < 5) {
            set.push_back(l);
            seen |= contrib(l);
        }
    for (int l : tb)
        if ((int)set.size() < 5 && !has(set, l) && contrib(l) && !(seen & contrib(l))) {
            set.push_back(l);
            seen |= contrib(l);
        }
    for (int l : tb)
        if ((int)set.size() < 5 && !has(set, l))
            set.push_back(l);
    // order within the set: distinct nonzero contributions first
    const int need = ES == 8 ? 4 : 3;
    std::vector<int> lanes;
    int got = 0;
    for (int l : set)
        if ((int)lanes.size() < need && contrib(l) && !(got & contrib(l))) {
            lanes.push_back(l);
            got |= contrib(l);
        }
    for (int l : set)
        if (!has(lanes, l))
            lanes.push_back(l);
    int n = 0;
    for (int l : lanes)
        io.bits[n++] = (uint8_t)l;
    std::vector<int> rest;
    for (int l = 0; l < TB; l++)
        if ((l < W || l >= W + RB) && !has(lanes, l))
            io.bits[n++] = (uint8_t)l;
    return io;
}

// ------------------------------------------------------------ slots (Sec. 2)

int half_scale(int N, int k) { return (k & 1) ? N / 2 : N - N / 2; }

// Slots of U4(tau)^n (order 4), U2(tau)^n (order 2) or U1(tau)^n (order 1).
std::vector<HostSlot> make_slots(int N, int order, double tau, int64_t n)
{
    std::vector<HostSlot> s;
    HostSlot z;
    if (order == 4 || order == 2) {
        const double p = 1.0 / (4.0 - std::cbrt(4.0));
        const double c4[5] = {p, p, 1.0 - 4.0 * p, p, p};
        const int per = (order == 4) ? 5 : 1;
        const int64_t U = n * per;
        auto tu = [&](int64_t u) { return (order == 4 ? c4[u % 5] : 1.0) * tau; };
        s.reserve((size_t)(4 * U + 1));
        z.t = tu(0) / 2;
        z.alpha = 2;
        z.pcq = 3;
        s.push_back(z);
        for (int64_t u = 0; u < U; u++) {
            const double t = tu(u);
            const int64_t k = 4 * u;
            HostSlot a;
            a.t = t / 2; a.alpha = 1; a.pcq = 1; a.scale_exp = half_scale(N, (int)((k + 1) & 1));
            s.push_back(a);
            HostSlot b;
            b.t = t; b.alpha = 0; b.pcq = 0; b.scale_exp = half_scale(N, (int)((k + 2) & 1));
            s.push_back(b);
            HostSlot c;
            c.t = t / 2; c.alpha = 1; c.pcq = 3; c.scale_exp = half_scale(N, (int)((k + 3) & 1));
            s.push_back(c);
            HostSlot d;
            d.alpha = 2;
            d.scale_exp = half_scale(N, (int)((k + 4) & 1));
            if (u + 1 < U) {
                d.t = (t + tu(u + 1)) / 2;
                d.pcq = 0;
            } else {
                d.t = t / 2;
                d.pcq = 1;
            }
            s.push_back(d);
        }
    } else {
        // U1(tau) = e^{-i tau H_x} e^{-i tau H_y} e^{-i tau H_z}: layers X^dag, Y^dag X, Y
        z.t = tau;
        z.alpha = 2;
        z.pcq = 3;
        s.push_back(z);
        for (int64_t u = 0; u < n; u++) {
            const int64_t k = 3 * u;
            HostSlot a;
            a.t = tau; a.alpha = 1; a.pcq = 1; a.scale_exp = half_scale(N, (int)((k + 1) & 1));
            s.push_back(a);
            HostSlot b;
            b.t = tau; b.alpha = 0; b.pcq = 1; b.th0 = M_PI * N / 4.0;
            b.scale_exp = half_scale(N, (int)((k + 2) & 1));
            s.push_back(b);
            HostSlot c;
            c.alpha = 2;
            c.scale_exp = half_scale(N, (int)((k + 3) & 1));
            if (u + 1 < n) {
                c.t = tau;
                c.pcq = 1;
            } else {
                c.t = 0.0;
                c.pcq = 2;
            }
            s.push_back(c);
        }
    }
    // with N * layers odd the powers of two fall short by sqrt 2: fold it into the last slot
    const int64_t L = (int64_t)s.size() - 1;
    if ((N & 1) && (L & 1))
        s.back().mag = std::sqrt(0.5);
    return s;
}

// ------------------------------------------------------------ groups and passes

std::vector<Group> make_groups(int N, int TB, int cbits)
{
    std::vector<Group> g;
    if (N <= TB) {
        g.push_back({0, 0, N});
        return g;
    }
    g.push_back({0, 0, TB});
    const int rest = N - TB;
    const int hmax = TB - cbits;
    const int ng = (rest + hmax - 1) / hmax;
    const int base = rest / ng, extra = rest % ng;
    int w = TB;
    for (int k = 0; k < ng; k++) {
        const int hk = base + (k < extra ? 1 : 0);
        g.push_back({TB - hk, w, hk});
        w += hk;
    }
    return g;
}

// Default coalescing width for N spins and TB-bit tiles: the precision's default (64-byte
// runs), or one bit less (32-byte runs, still whole sectors) when that saves a bit group,
// i.e. one pass per layer.
int default_cbits_for(ts_prec p, int N, int TB)
{
    const int cb = default_cbits(p);
    if (N <= TB || cb - 1 < 2)
        return cb;
    return make_groups(N, TB, cb - 1).size() < make_groups(N, TB, cb).size() ? cb - 1 : cb;
}

// The same for an ensemble: the width that minimises the amplitude-passes of all its states
// (ties keep the precision's default).
int default_cbits_batch(ts_prec p, int TB, const std::vector<int> &N, const std::vector<int> &nstates)
{
    const int cb0 = default_cbits(p);
    auto cost = [&](int cb) {
        double c = 0.0;
        for (size_t s = 0; s < N.size(); s++) {
            const int g = N[s] <= TB ? 1 : (int)make_groups(N[s], TB, cb).size();
            c += (double)nstates[s] * std::ldexp(1.0, N[s]) * (g > 1 ? g - 1 : 1);
        }
        return c;
    };
    return (cb0 - 1 >= 2 && cost(cb0 - 1) < cost(cb0)) ? cb0 - 1 : cb0;
}

struct ChunkInfo {
    int n;
    int lo[8], hi[8];
};

ChunkInfo chunks_of(int h, int TB, int RB)
{
    ChunkInfo ci;
    ci.n = (h + RB - 1) / RB;
    for (int k = 0; k < ci.n; k++) {
        const int W = (k * RB < TB - RB) ? k * RB : TB - RB;
        ci.lo[k] = k * RB - W;
        ci.hi[k] = ((k + 1) * RB < h ? (k + 1) * RB : h) - W;
    }
    return ci;
}

enum PassKind { P_PHASE_ROT, P_ROT, P_ROT_PHASE_ROT, P_ROT_PHASE, P_PHASE };

// Chunk whose register bits the I/O layout of group g uses: the lanes must sit on the
// globally lowest bits of the tile, which for the lowest group (c == 0) are the first
// RB local bits, so there the registers take chunk 1; otherwise the lowest bits are the
// c coalescing bits (local bits h..TB-1) and the registers take chunk 0.
int io_chunk(const Group &g) { return g.c == 0 ? 1 : 0; }

// One pass over group g.  The layer's chunks are visited starting from the I/O chunk
// (the tile arrives and leaves in that layout), so a pass that rotates the group twice
// around a slot costs 4 transposes for three chunks instead of 6:
// io, a, b | slot | b, a, io.
HostPass make_pass(int gi, const Group &g, PassKind kind, int slot, int TB, int RB)
{
    HostPass p;
    p.group = gi;
    p.slot = slot;
    ChunkInfo ci = chunks_of(g.h, TB, RB);
    const int n = ci.n;
    const int kio = io_chunk(g) < n ? io_chunk(g) : 0;
    int ord[8];
    ord[0] = kio;
    for (int k = 0, m = 1; k < n; k++)
        if (k != kio)
            ord[m++] = k;
    auto add = [&](int k, bool r0, bool ph, bool r1) {
        StepDesc d;
        std::memset(&d, 0, sizeof(d));
        d.k = (uint8_t)k;
        d.r0lo = (uint8_t)(r0 ? ci.lo[k] : 0);
        d.r0hi = (uint8_t)(r0 ? ci.hi[k] : 0);
        d.ph = ph ? 1 : 0;
        d.r1lo = (uint8_t)(r1 ? ci.lo[k] : 0);
        d.r1hi = (uint8_t)(r1 ? ci.hi[k] : 0);
        if (ph)
            p.phase_k = k;
        p.steps[p.nsteps++] = d;
    };
    switch (kind) {
    case P_PHASE_ROT:
        add(ord[0], false, true, true);
        for (int i = 1; i < n; i++)
            add(ord[i], true, false, false);
        break;
    case P_ROT:
        for (int i = 0; i < n; i++)
            add(ord[i], true, false, false);
        break;
    case P_ROT_PHASE_ROT:
        for (int i = 0; i < n - 1; i++)
            add(ord[i], true, false, false);
        add(ord[n - 1], true, true, true);
        for (int i = n - 2; i >= 0; i--)
            add(ord[i], false, false, true);
        break;
    case P_ROT_PHASE:
        for (int i = 1; i < n; i++)
            add(ord[i], true, false, false);
        add(ord[0], true, true, false);
        break;
    case P_PHASE:
        add(ord[0], false, true, false);
        break;
    }
    return p;
}

// Passes for L layers and slots 0..L (slot 0 before the first layer).
std::vector<HostPass> make_passes(const std::vector<Group> &G, int64_t L, int TB, int RB)
{
    std::vector<HostPass> P;
    const int g = (int)G.size();
    if (g == 1) {
        P.reserve((size_t)L + 1);
        for (int64_t l = 0; l < L; l++)
            P.push_back(make_pass(0, G[0], P_PHASE_ROT, (int)l, TB, RB));
        P.push_back(make_pass(0, G[0], P_PHASE, (int)L, TB, RB));
        return P;
    }
    // Visiting order of the groups: the two ends of the zigzag carry the slots and rotate
    // their group twice, so the largest group (group 0, TB bits) goes between them when
    // there are three or more groups: its single rotation per layer then runs in a pass
    // without a slot, and the double rotations fall on the smaller window groups.
    std::vector<int> perm(g);
    for (int k = 0; k < g; k++)
        perm[k] = k;
    if (g >= 3)
        std::swap(perm[0], perm[1]);
    P.reserve((size_t)(1 + L * (g - 1)));
    P.push_back(make_pass(perm[0], G[perm[0]], P_PHASE_ROT, 0, TB, RB));
    for (int64_t l = 1; l <= L; l++) {
        // layer l visits the groups forward when l is odd, backward when even
        std::vector<int> ord(g);
        for (int k = 0; k < g; k++)
            ord[k] = perm[(l & 1) ? k : g - 1 - k];
        for (int k = 1; k < g - 1; k++)
            P.push_back(make_pass(ord[k], G[ord[k]], P_ROT, -1, TB, RB));
        const int last = ord[g - 1];
        if (l < L)
            P.push_back(make_pass(last, G[last], P_ROT_PHASE_ROT, (int)l, TB, RB));
        else
            P.push_back(make_pass(last, G[last], P_ROT_PHASE, (int)l, TB, RB));
    }
    return P;
}

// ------------------------------------------------------------ buffers

ts_status ensure_buf(ts_ctx *ctx, Buf &b, const char *what)
{
    if (b.p)
        return TS_OK;
    size_t freeb = 0, totb = 0;
    TS_CUDA(ctx, cudaMemGetInfo(&freeb, &totb));
    if (state_bytes(ctx) > freeb)
        return fail(ctx, TS_ERR_OOM, std::string(what) + ": state of " + std::to_string(state_bytes(ctx)) +
                                         " bytes does not fit in free device memory");
    cudaError_t e = cudaMalloc(&b.p, state_bytes(ctx));
    if (e != cudaSuccess) {
        b.p = nullptr;
        return cuda_fail(ctx, e, what);
    }
    b.own = true;
    return TS_OK;
}

void free_buf(Buf &b)
{
    if (b.p && b.own)
        cudaFree(b.p);
    b.p = nullptr;
    b.own = false;
}

ts_status ensure_part(ts_ctx *ctx, size_t doubles)
{
    if (ctx->part_cap >= doubles)
        return TS_OK;
    if (ctx->dpart)
        cudaFree(ctx->dpart);
    ctx->dpart = nullptr;
    TS_CUDA(ctx, cudaMalloc(&ctx->dpart, doubles * sizeof(double)));
    ctx->part_cap = doubles;
    return TS_OK;
}

// ------------------------------------------------------------ execution

HamDev ham_dev(const ts_ctx *ctx)
{
    HamDev h;
    h.Jq = ctx->dJq;
    h.hh = ctx->dhh;
    h.N = ctx->N;
    return h;
}

unsigned grid_for(const ts_ctx *ctx, uint64_t work, int threads)
{
    uint64_t blocks = (work + threads - 1) / threads;
    const uint64_t cap = (uint64_t)ctx->sms * 16;
    if (blocks > cap)
        blocks = cap;
    return (unsigned)(blocks ? blocks : 1);
}

ts_status run_basic(ts_ctx *ctx, void *buf, const std::vector<HostSlot> &slots)
{
    const uint64_t dim = dim_of(ctx);
    const unsigned gs = grid_for(ctx, dim, 256), gp = grid_for(ctx, dim / 2, 256);
    const HamDev hd = ham_dev(ctx);
    for (size_t k = 0; k < slots.size(); k++) {
        if (k > 0) {
            for (int b = 0; b < ctx->N; b++) {
                if (ctx->prec == TS_C64)
                    k_wht_bit<float2><<<gp, 256, 0, ctx->stream>>>((float2 *)buf, dim / 2, b);
                else
                    k_wht_bit<double2><<<gp, 256, 0, ctx->stream>>>((double2 *)buf, dim / 2, b);
                ctx->launches++;
            }
        }
        const Slot sl = slots[k].dev();
        if (ctx->dE) {
            if (ctx->prec == TS_C64)
                k_slot_table<float, float><<<gs, 256, 0, ctx->stream>>>(
                    (float2 *)buf, static_cast<const float *>(ctx->dE) + (size_t)sl.alpha * dim, dim, sl);
            else
                k_slot_table<double, double><<<gs, 256, 0, ctx->stream>>>(
                    (double2 *)buf, static_cast<const double *>(ctx->dE) + (size_t)sl.alpha * dim, dim, sl);
        } else if (ctx->prec == TS_C64) {
            k_slot_basic<float><<<gs, 256, 0, ctx->stream>>>((float2 *)buf, dim, hd, sl);
        } else {
            k_slot_basic<double><<<gs, 256, 0, ctx->stream>>>((double2 *)buf, dim, hd, sl);
        }
        ctx->launches++;
        TS_CUDA(ctx, cudaGetLastError());
    }
    return TS_OK;
}

// Builds the fused schedule for the slots in S: groups, passes, per-group I/O
// layouts, and one table per distinct (slot values, group, phase chunk).
// Pass-list shapes: the first pass also completes the previous call's last layer on its
// group (the slot is then the merged P_z of both calls); the last pass is held back; or the
// held-back pass alone.
enum { SHAPE_HEAD_MERGED = 1, SHAPE_TAIL_DEFERRED = 2, SHAPE_TAIL_ONLY = 4 };

// Two consecutive P_z slots as one (Sec. 2: P_z(a) P_z(b) = P_z(a + b)); the scale and the
// powers of i multiply as well.
HostSlot merge_z(const HostSlot &a, const HostSlot &b)
{
    HostSlot m = b;
    m.t = a.t + b.t;
    m.th0 = a.th0 + b.th0;
    m.pcq = (a.pcq + b.pcq) & 3;
    m.scale_exp = a.scale_exp + b.scale_exp;
    m.mag = a.mag * b.mag;
    return m;
}

// make_passes with a shape applied: the held-back pass alone; or the first pass also running
// the previous call's held-back rotation before its (merged) slot; and/or the last pass held back.
std::vector<HostPass> shaped_passes(const std::vector<Group> &G, int64_t L, int TB, int RB, int shape,
                                    int tail_group)
{
    std::vector<HostPass> P = make_passes(G, L, TB, RB);
    if (shape & SHAPE_TAIL_ONLY) {
        P.assign(1, make_pass(tail_group, G[(size_t)tail_group], P_ROT_PHASE, 0, TB, RB));
        return P;
    }
    if (shape & SHAPE_HEAD_MERGED) {
        const int g0 = P.front().group;
        P.front() = make_pass(g0, G[(size_t)g0], P_ROT_PHASE_ROT, 0, TB, RB);
    }
    if (shape & SHAPE_TAIL_DEFERRED)
        P.pop_back();
    return P;
}

bool same_slot(const HostSlot &a, const HostSlot &b)
{
    return a.t == b.t && a.th0 == b.th0 && a.mag == b.mag && a.alpha == b.alpha && a.pcq == b.pcq &&
           a.scale_exp == b.scale_exp;
}

ts_status prepare_fused(ts_ctx *ctx, Schedule &S)
{
    const int RB = ctx->RB, TB = ctx->TB;
    const int ES = (int)amp_bytes(ctx);
    S.groups = make_groups(ctx->N, TB, ctx->cbits);
    S.io.clear();
    for (size_t gi = 0; gi < S.groups.size(); gi++)
        S.io.push_back(make_io(S.groups[gi], TB, RB, ES, io_chunk(S.groups[gi])));
    // per group and thread of the I/O layout: global offset of its base and its local base
    const int NT = 1 << (TB - RB);
    S.iomap.assign(S.groups.size() * (size_t)NT, make_uint4(0, 0, 0, 0));
    for (size_t gi = 0; gi < S.groups.size(); gi++) {
        const Group &g = S.groups[gi];
        auto gpos = [&](int l) { return l < g.h ? g.w + l : l - g.h; };
        for (int tid = 0; tid < NT; tid++) {
            uint32_t base = 0;
            uint64_t off = 0;
            for (int t = 0; t < TB - RB; t++)
                if ((tid >> t) & 1) {
                    base |= 1u << S.io[gi].bits[t];
                    off |= UINT64_C(1) << gpos(S.io[gi].bits[t]);
                }
            S.iomap[gi * NT + tid] = make_uint4((uint32_t)off, (uint32_t)(off >> 32), base, 0);
        }
    }
    const int64_t L = (int64_t)S.slots.size() - 1;
    S.passes = shaped_passes(S.groups, L, TB, RB, S.shape, S.tail_group);
    S.tab_size = tab_size(ctx->prec, TB);
    std::map<std::tuple<double, int, int, int, int>, int> seen;
    S.tabs.clear();
    for (auto &p : S.passes) {
        if (p.slot < 0)
            continue;
        const HostSlot &sl = S.slots[p.slot];
        if (ctx->prec == TS_C64) {
            const double yb = slot_y_bound(ctx, sl, S.groups[p.group], TB, RB, p.phase_k);
            p.ymode = yb <= 0.05 ? 0 : (yb <= 0.5 ? 1 : 2);
        }
        auto key = std::make_tuple(sl.t, sl.alpha, sl.pcq, p.group, p.phase_k);
        auto it = seen.find(key);
        if (it != seen.end()) {
            p.tab = it->second;
            continue;
        }
        const int idx = (int)seen.size();
        seen[key] = idx;
        p.tab = idx;
        S.tabs.resize((size_t)(idx + 1) * S.tab_size);
        build_tab(S.tabs.data() + (size_t)idx * S.tab_size, ctx, TB, sl, S.groups[p.group], S.io[p.group], p.phase_k);
    }
    // frame terms: per distinct (slot, group), one angle and TB fields per tile
    struct ThetaJob {
        const HostSlot *sl;
        int group;
        size_t off;
    };
    std::vector<ThetaJob> jobs;
    std::map<std::tuple<double, int, double, int>, size_t> seen_th;
    size_t ntheta = 0;
    for (auto &p : S.passes) {
        if (p.slot < 0)
            continue;
        const HostSlot &sl = S.slots[p.slot];
        auto key = std::make_tuple(sl.t, sl.alpha, sl.th0, p.group);
        auto it = seen_th.find(key);
        if (it != seen_th.end()) {
            p.theta_off = it->second;
            continue;
        }
        const Group &g = S.groups[p.group];
        p.theta_off = ntheta;
        seen_th[key] = ntheta;
        jobs.push_back({&sl, p.group, ntheta});
        ntheta += (size_t)1 << (ctx->N - (g.c + g.h));
    }
    const size_t rsize = ctx->prec == TS_C64 ? sizeof(float) : sizeof(double);
    const size_t frame_bytes = ntheta * (sizeof(double) + (size_t)TB * rsize);
    if (S.tabs.size() > S.dtab_cap || frame_bytes > S.dtheta_cap) {
        release_tables(S, ctx->stream);
        if (!S.tabs.empty()) {
            TS_CUDA(ctx, cudaMalloc(&S.dtab, S.tabs.size()));
            S.dtab_cap = S.tabs.size();
        }
        if (frame_bytes) {
            TS_CUDA(ctx, cudaMalloc(&S.dtheta, frame_bytes));
            S.dtheta_cap = frame_bytes;
        }
    }
    S.dgfield = S.dtheta ? static_cast<void *>(S.dtheta + ntheta) : nullptr;
    if (!S.tabs.empty())
        TS_CUDA(ctx, cudaMemcpyAsync(S.dtab, S.tabs.data(), S.tabs.size(), cudaMemcpyHostToDevice, ctx->stream));
    const size_t map_bytes = S.iomap.size() * sizeof(uint4);
    if (map_bytes > S.dmap_cap) {
        if (S.dmap) {
            TS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
            cudaFree(S.dmap);
            S.dmap = nullptr;
            S.dmap_cap = 0;
        }
        TS_CUDA(ctx, cudaMalloc(&S.dmap, map_bytes));
        S.dmap_cap = map_bytes;
    }
    TS_CUDA(ctx, cudaMemcpyAsync(S.dmap, S.iomap.data(), map_bytes, cudaMemcpyHostToDevice, ctx->stream));
    for (const auto &j : jobs) {
        const Group &g = S.groups[j.group];
        const int N = ctx->N;
        const uint64_t nframes = UINT64_C(1) << (N - (g.c + g.h));
        const unsigned blocks = (unsigned)std::min<uint64_t>((nframes + 127) / 128, (uint64_t)ctx->sms * 8);
        const double *Jq = ctx->dJq + (size_t)j.sl->alpha * N * N;
        const double *hh = ctx->dhh + (size_t)j.sl->alpha * N;
        if (ctx->prec == TS_C64)
            k_frame_terms<float><<<blocks, 128, 0, ctx->stream>>>(Jq, hh, N, g.c, g.w, g.h, j.sl->t, j.sl->th0, 1.0,
                                                                  nframes, S.dtheta + j.off,
                                                                  static_cast<float *>(S.dgfield) + j.off * TB);
        else
            k_frame_terms<double><<<blocks, 128, 0, ctx->stream>>>(Jq, hh, N, g.c, g.w, g.h, j.sl->t, j.sl->th0,
                                                                   1.0 / M_PI, nframes, S.dtheta + j.off,
                                                                   static_cast<double *>(S.dgfield) + j.off * TB);
        ctx->launches++;
        TS_CUDA(ctx, cudaGetLastError());
    }
    // the host image must stay valid until the copy is done
    TS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return TS_OK;
}

// Fields of the first frame of a (slot, group) whose angles start at frame offset off.
const void *gfield_at(const ts_ctx *ctx, const Schedule &S, size_t off)
{
    if (ctx->prec == TS_C64)
        return static_cast<const float *>(S.dgfield) + off * ctx->TB;
    return static_cast<const double *>(S.dgfield) + off * ctx->TB;
}

// The I/O layout of group gi: the per-thread table and the register bits' global offsets.
void set_io_args(TileArgs &a, const ts_ctx *ctx, const Schedule &S, int gi)
{
    const int TB = ctx->TB, RB = ctx->RB, NT = 1 << (TB - RB);
    const Group &g = S.groups[gi];
    a.iomap = static_cast<const uint4 *>(S.dmap) + (size_t)gi * NT;
    const int W = S.io[gi].chunk == 0 ? 0 : (RB < TB - RB ? RB : TB - RB);
    for (int b = 0; b < RB; b++) {
        const int l = W + b;
        a.gst[b] = UINT64_C(1) << (l < g.h ? g.w + l : l - g.h);
    }
}

ts_status run_fused(ts_ctx *ctx, void *buf, const Schedule &S)
{
    const HamDev hd = ham_dev(ctx);
    for (const auto &p : S.passes) {
        const Group &g = S.groups[p.group];
        TileArgs a;
        std::memset(&a, 0, sizeof(a));
        a.c = g.c;
        a.w = g.w;
        a.h = g.h;
        a.nsteps = p.nsteps;
        std::memcpy(a.steps, p.steps, sizeof(p.steps));
        a.has_slot = p.slot >= 0;
        if (p.slot >= 0)
            a.slot = S.slots[p.slot].dev();
        a.tab = p.tab < 0 ? 0 : p.tab;
        a.exact_sincos = p.ymode;
        a.io = S.io[p.group];
        a.ham = hd;
        a.theta = p.slot >= 0 ? S.dtheta + p.theta_off : nullptr;
        a.gfield = p.slot >= 0 ? gfield_at(ctx, S, p.theta_off) : nullptr;
        set_io_args(a, ctx, S, p.group);
        const uint64_t nblk = UINT64_C(1) << (ctx->N - (g.c + g.h));
        cudaError_t e = launch_tile(ctx, ctx->TB, buf, a, S.dtab, nblk);
        ctx->launches++;
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "fused pass launch");
    }
    return TS_OK;
}

bool fused_usable(const ts_ctx *ctx) { return ctx->kernel == TS_KERNEL_FUSED && ctx->N >= ctx->TB; }

// Runs the layers of `slots` on buf with the selected kernel.  The schedule is
// cached under `key` so that repeated calls reuse the pass list and tables.
ts_status run_slots(ts_ctx *ctx, Schedule &S, void *buf, int order, double tau, int64_t n, int mode,
                    const std::vector<HostSlot> &slots, int shape = 0, int tail_group = 0)
{
    // small N: the fused kernel needs a full tile; take the largest provided tile <= N
    const int keepTB = ctx->TB;
    if (ctx->kernel == TS_KERNEL_FUSED && ctx->N < ctx->TB && tile_supported(ctx->prec, ctx->N))
        ctx->TB = ctx->N;
    ts_status st = TS_OK;
    if (!fused_usable(ctx)) {
        st = run_basic(ctx, buf, slots);
    } else {
        const bool hit = S.order == order && S.tau == tau && S.n == n && S.kernel == ctx->kernel &&
                         S.TB == ctx->TB && S.cbits == ctx->cbits && S.mode == mode && S.shape == shape &&
                         S.tail_group == tail_group && !S.slots.empty() && same_slot(S.slots[0], slots[0]);
        if (!hit) {
            // keep the device table buffer for reuse, rebuild everything else
            void *keep = S.dtab;
            const size_t keep_cap = S.dtab_cap;
            double *keep_th = S.dtheta;
            const size_t keep_th_cap = S.dtheta_cap;  // (dgfield is re-derived by prepare_fused)
            void *keep_map = S.dmap;
            const size_t keep_map_cap = S.dmap_cap;
            S = Schedule();
            S.dtab = keep;
            S.dtab_cap = keep_cap;
            S.dtheta = keep_th;
            S.dtheta_cap = keep_th_cap;
            S.dmap = keep_map;
            S.dmap_cap = keep_map_cap;
            S.slots = slots;
            S.shape = shape;
            S.tail_group = tail_group;
            st = prepare_fused(ctx, S);
            if (st == TS_OK) {
                S.shape = shape;
                S.tail_group = tail_group;
                S.order = order;
                S.tau = tau;
                S.n = n;
                S.kernel = ctx->kernel;
                S.TB = ctx->TB;
                S.cbits = ctx->cbits;
                S.mode = mode;
            } else {
                reset_schedule(S, ctx->stream);
            }
        }
        if (st == TS_OK)
            st = run_fused(ctx, buf, S);
    }
    ctx->TB = keepTB;
    return st;
}

// Runs the held-back final pass of the last ts_step (if any) on the state.
ts_status flush_tail(ts_ctx *ctx)
{
    if (!ctx->tail_pending)
        return TS_OK;
    ctx->tail_pending = false;
    const std::vector<HostSlot> one(1, ctx->tail_slot);
    return run_slots(ctx, ctx->sched_tail, ctx->psi.p, 0, 0.0, 0, 0, one, SHAPE_TAIL_ONLY, ctx->tail_group);
}

// ------------------------------------------------------------ reductions

ts_status finish_sum(ts_ctx *ctx, int nblk, int K, double *out)
{
    if (K > kMaxOut)
        return fail(ctx, TS_ERR_ARG, "reduction larger than the read-back buffer");
    // partial sums live in dpart[0 .. nblk*K); the final sums go after them
    double *dfin = ctx->dpart + (size_t)nblk * K;
    k_sum_final<<<1, 64, 0, ctx->stream>>>(ctx->dpart, nblk, K, dfin);
    ctx->launches++;
    TS_CUDA(ctx, cudaGetLastError());
    TS_CUDA(ctx, cudaMemcpyAsync(ctx->hout, dfin, K * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    TS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    std::memcpy(out, ctx->hout, K * sizeof(double));
    return TS_OK;
}

unsigned red_blocks(const ts_ctx *ctx, uint64_t work_per_block)
{
    uint64_t b = (dim_of(ctx) + work_per_block - 1) / work_per_block;
    const uint64_t cap = (uint64_t)ctx->sms * 4;
    if (b > cap)
        b = cap;
    return (unsigned)(b ? b : 1);
}

ts_status sum_sz(ts_ctx *ctx, const void *buf, double *norm_and_p /* N+1 */)
{
    const int K = ctx->N + 1;
    const unsigned nb = sum_sz_blocks(ctx->N, 512);
    ts_status st = ensure_part(ctx, (size_t)nb * K + K);
    if (st)
        return st;
    if (ctx->prec == TS_C64)
        k_sum_sz<float2><<<nb, 256, 0, ctx->stream>>>((const float2 *)buf, ctx->N, ctx->dpart);
    else
        k_sum_sz<double2><<<nb, 256, 0, ctx->stream>>>((const double2 *)buf, ctx->N, ctx->dpart);
    ctx->launches++;
    TS_CUDA(ctx, cudaGetLastError());
    return finish_sum(ctx, (int)nb, K, norm_and_p);
}

ts_status sum_norm(ts_ctx *ctx, const void *buf, double *out)
{
    const unsigned nb = red_blocks(ctx, UINT64_C(1) << kSumRangeBits);
    ts_status st = ensure_part(ctx, (size_t)nb + 1);
    if (st)
        return st;
    if (ctx->prec == TS_C64)
        k_sum_norm<float2><<<nb, 256, 0, ctx->stream>>>((const float2 *)buf, ctx->N, ctx->dpart);
    else
        k_sum_norm<double2><<<nb, 256, 0, ctx->stream>>>((const double2 *)buf, ctx->N, ctx->dpart);
    ctx->launches++;
    TS_CUDA(ctx, cudaGetLastError());
    return finish_sum(ctx, (int)nb, 1, out);
}

ts_status sum_diag(ts_ctx *ctx, const void *buf, int alpha, double *out)
{
    const unsigned nb = red_blocks(ctx, 256 * 8);
    ts_status st = ensure_part(ctx, (size_t)nb + 1);
    if (st)
        return st;
    if (ctx->prec == TS_C64)
        k_sum_diag_energy<float2><<<nb, 256, 0, ctx->stream>>>((const float2 *)buf, dim_of(ctx), ham_dev(ctx), alpha,
                                                               ctx->dpart);
    else
        k_sum_diag_energy<double2><<<nb, 256, 0, ctx->stream>>>((const double2 *)buf, dim_of(ctx), ham_dev(ctx),
                                                                alpha, ctx->dpart);
    ctx->launches++;
    TS_CUDA(ctx, cudaGetLastError());
    return finish_sum(ctx, (int)nb, 1, out);
}

ts_status sum_overlap(ts_ctx *ctx, const void *a, const void *b, double *out2)
{
    const unsigned nb = red_blocks(ctx, 256 * 8);
    ts_status st = ensure_part(ctx, (size_t)nb * 2 + 2);
    if (st)
        return st;
    if (ctx->prec == TS_C64)
        k_sum_overlap<float2><<<nb, 256, 0, ctx->stream>>>((const float2 *)a, (const float2 *)b, dim_of(ctx),
                                                           ctx->dpart);
    else
        k_sum_overlap<double2><<<nb, 256, 0, ctx->stream>>>((const double2 *)a, (const double2 *)b, dim_of(ctx),
                                                            ctx->dpart);
    ctx->launches++;
    TS_CUDA(ctx, cudaGetLastError());
    return finish_sum(ctx, (int)nb, 2, out2);
}

// <H_a> for a = x (pcq 2: Y^dag = 2^{-N/2} W (-1)^pc) or y (pcq 3: X^dag = 2^{-N/2} D W (-i)^pc):
// one Walsh-Hadamard layer on a copy, then sum |phi_s|^2 E_a(s) 2^{-N}.
// Copies the state into the scratch buffer rotated into the eigenbasis of S^x (alpha = 0)
// or S^y (alpha = 1): one Walsh-Hadamard layer between two diagonal slots, so that
// |scratch_s|^2 2^-N is the probability of the x or y configuration s (bit 1 = +1/2).
ts_status frame_copy(ts_ctx *ctx, int alpha)
{
    ts_status st = ensure_buf(ctx, ctx->scratch, "observable scratch buffer");
    if (st)
        return st;
    TS_CUDA(ctx, cudaMemcpyAsync(ctx->scratch.p, ctx->psi.p, state_bytes(ctx), cudaMemcpyDeviceToDevice, ctx->stream));
    std::vector<HostSlot> sl(2);
    sl[0].t = 0.0;
    sl[0].pcq = alpha == 0 ? 2 : 3;
    sl[1].t = 0.0;
    return run_slots(ctx, ctx->sched_obs, ctx->scratch.p, 0, 0.0, 1, 10 + alpha, sl);
}

// Joint bit weights of a state (k_sum_pairs): out[0] = total, out[1 + i] singles,
// out[1 + N + pair(i, j)] pairs.
ts_status sum_pairs(ts_ctx *ctx, const void *buf, double *out)
{
    const int N = ctx->N;
    const int K = 1 + N + N * (N - 1) / 2;
    const unsigned nb = red_blocks(ctx, 256 * 32);
    ts_status st = ensure_part(ctx, (size_t)nb * K + K);
    if (st)
        return st;
    const size_t smem = (size_t)K * sizeof(double);
    if (ctx->prec == TS_C64)
        k_sum_pairs<float2><<<nb, 256, smem, ctx->stream>>>((const float2 *)buf, N, ctx->dpart);
    else
        k_sum_pairs<double2><<<nb, 256, smem, ctx->stream>>>((const double2 *)buf, N, ctx->dpart);
    ctx->launches++;
    TS_CUDA(ctx, cudaGetLastError());
    return finish_sum(ctx, (int)nb, K, out);
}

// <S^a_i S^a_j> = sum_s w(s) (b_i - 1/2)(b_j - 1/2) from the joint bit weights, times wscale.
void pairs_to_correlations(int N, const double *v, double wscale, double *out)
{
    for (int i = 0; i < N; i++) {
        out[i * N + i] = 0.25 * v[0] * wscale;
        for (int j = i + 1; j < N; j++) {
            const double pij = v[1 + N + pair_index(i, j, N)];
            const double c = (pij - 0.5 * (v[1 + i] + v[1 + j]) + 0.25 * v[0]) * wscale;
            out[i * N + j] = c;
            out[j * N + i] = c;
        }
    }
}

ts_status rotated_energy(ts_ctx *ctx, int alpha, double *out)
{
    ts_status st = frame_copy(ctx, alpha);
    if (st)
        return st;
    double v = 0.0;
    st = sum_diag(ctx, ctx->scratch.p, alpha, &v);
    if (st)
        return st;
    *out = std::ldexp(v, -ctx->N);
    return TS_OK;
}

// The time-step bound of Eq. 4 (the inverse of the largest local second moment of H), from
// the raw couplings (N*N row-major, upper triangle) and fields of each axis.
double step_bound_of(int N, const std::vector<double> (&J)[3], const std::vector<double> (&h)[3])
{
    double mx = 0.0;
    for (int j = 0; j < N; j++) {
        double hs = 0.0;
        for (int a = 0; a < 3; a++)
            hs += (h[a][j] / 2) * (h[a][j] / 2);
        for (int k = 0; k < N; k++) {
            if (k == j)
                continue;
            double js = 0.0;
            for (int a = 0; a < 3; a++) {
                const double v = (j < k) ? J[a][j * N + k] : J[a][k * N + j];
                js += (v / 4) * (v / 4);
            }
            const double m = hs + js;
            if (m > mx)
                mx = m;
        }
        if (N == 1 && hs > mx)
            mx = hs;
    }
    return mx > 0.0 ? 1.0 / std::sqrt(mx) : INFINITY;
}

bool finite_all(const double *p, size_t n)
{
    for (size_t i = 0; i < n; i++)
        if (!std::isfinite(p[i]))
            return false;
    return true;
}

} // namespace

// ================================================================== C ABI

extern "C" {

const char *ts_version(void) { return "ts4-gb300 0.1 (sm_103a)"; }

const char *ts_last_error(const ts_ctx *ctx) { return ctx ? ctx->err.c_str() : ""; }

int64_t ts_kernel_launches(const ts_ctx *ctx) { return ctx ? ctx->launches : 0; }

uint64_t ts_tile_global_index(int N, int c, int w, int h, uint64_t f, uint64_t e)
{
    (void)N;
    return tile_global_index(c, w, h, f, e);
}

ts_status ts_plan(int N, ts_prec prec, int tile_bits, int coalesce_bits, int order, int64_t nsteps, int chain,
                  ts_plan_group *groups, int max_groups, int *ngroups, ts_plan_pass *passes, int64_t max_passes,
                  int64_t *npasses)
{
    if (!ngroups || !npasses || N < 1 || N > kMaxN || (prec != TS_C64 && prec != TS_C128) ||
        (order != 1 && order != 2 && order != 4) || nsteps < 1 || chain < 0 || chain > 3)
        return TS_ERR_ARG;
    const int TB = tile_bits ? tile_bits : default_tile(prec);
    const int RB = reg_bits(prec);
    const int cb = coalesce_bits ? coalesce_bits : default_cbits_for(prec, N, TB);
    if (!tile_supported(prec, TB) || N < TB || cb < 1 || cb > TB - RB)
        return TS_ERR_ARG;
    const std::vector<Group> G = make_groups(N, TB, cb);
    if (chain && G.size() < 2)
        return TS_ERR_ARG;
    const int64_t L = (int64_t)make_slots(N, order, 0.01, nsteps).size() - 1;
    // chain bit 1: the call continues a held-back pass; bit 2: it holds back its final pass
    const int shape = ((chain & 1) ? SHAPE_HEAD_MERGED : 0) | ((chain & 2) ? SHAPE_TAIL_DEFERRED : 0);
    const std::vector<HostPass> P = shaped_passes(G, L, TB, RB, shape, 0);
    *ngroups = (int)G.size();
    *npasses = (int64_t)P.size();
    for (int i = 0; i < (int)G.size() && groups && i < max_groups; i++)
        groups[i] = ts_plan_group{G[i].c, G[i].w, G[i].h};
    for (int64_t p = 0; p < (int64_t)P.size() && passes && p < max_passes; p++) {
        const HostPass &hp = P[(size_t)p];
        const Group &g = G[(size_t)hp.group];
        uint64_t side[2] = {0, 0};
        int dup = 0, after = 0;
        // register bits [lo, hi) of chunk k: tile-local bits W_k + b, W_k = min(k RB, TB - RB)
        auto rotate = [&](int k, int lo, int hi) {
            const int W = (k * RB < TB - RB) ? k * RB : TB - RB;
            for (int b = lo; b < hi; b++) {
                const int l = W + b;                               // tile-local bit
                const int pos = l < g.h ? g.w + l : l - g.h;       // global spin
                const uint64_t m = UINT64_C(1) << pos;
                if (side[after] & m)
                    dup = 1;
                side[after] |= m;
            }
        };
        for (int s = 0; s < hp.nsteps; s++) {
            const StepDesc &d = hp.steps[s];
            rotate(d.k, d.r0lo, d.r0hi);
            if (d.ph)
                after = 1;
            rotate(d.k, d.r1lo, d.r1hi);
        }
        passes[p] = ts_plan_pass{hp.group, hp.slot, side[0], side[1], dup};
    }
    return TS_OK;
}

ts_status ts_create(ts_ctx **out, int N, const double *Jx, const double *Jy, const double *Jz, const double *h,
                    ts_prec prec, void *cuda_stream)
{
    if (!out)
        return TS_ERR_ARG;
    *out = nullptr;
    if (N < 1 || N > kMaxN || !Jx || !Jy || !Jz || (prec != TS_C64 && prec != TS_C128))
        return TS_ERR_ARG;
    const double *J[3] = {Jx, Jy, Jz};
    for (int a = 0; a < 3; a++)
        if (!finite_all(J[a], (size_t)N * N))
            return TS_ERR_ARG;
    if (h && !finite_all(h, (size_t)N))
        return TS_ERR_ARG;
    ts_ctx *ctx = new (std::nothrow) ts_ctx();
    if (!ctx)
        return TS_ERR_OOM;
    ctx->N = N;
    ctx->prec = prec;
    ctx->stream = (cudaStream_t)cuda_stream;
    ctx->Jq.assign((size_t)3 * N * N, 0.0);
    ctx->hh.assign((size_t)3 * N, 0.0);
    for (int a = 0; a < 3; a++) {
        ctx->Jraw[a].assign(J[a], J[a] + (size_t)N * N);
        ctx->hraw[a].assign((size_t)N, 0.0);
        for (int i = 0; i < N; i++)
            for (int j = i + 1; j < N; j++) {
                const double v = J[a][i * N + j] / 4.0;
                ctx->Jq[(size_t)a * N * N + i * N + j] = v;
                ctx->Jq[(size_t)a * N * N + j * N + i] = v;
            }
    }
    if (h)
        for (int i = 0; i < N; i++) {
            ctx->hraw[2][i] = h[i];
            ctx->hh[2 * N + i] = h[i] / 2.0;
        }
    ctx->RB = reg_bits(prec);
    ctx->TB = default_tile(prec);
    ctx->cbits = default_cbits_for(prec, N, ctx->TB);
    ts_status st = TS_OK;
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e == cudaSuccess)
        e = cudaMalloc(&ctx->dJq, ctx->Jq.size() * sizeof(double));
    if (e == cudaSuccess)
        e = cudaMalloc(&ctx->dhh, ctx->hh.size() * sizeof(double));
    if (e == cudaSuccess)
        e = cudaMemcpy(ctx->dJq, ctx->Jq.data(), ctx->Jq.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(ctx->dhh, ctx->hh.data(), ctx->hh.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMallocHost(&ctx->hout, kMaxOut * sizeof(double));
    if (e != cudaSuccess) {
        st = (e == cudaErrorMemoryAllocation) ? TS_ERR_OOM : TS_ERR_CUDA;
        ts_destroy(ctx);
        return st;
    }
    *out = ctx;
    return TS_OK;
}

ts_status ts_set_transverse_fields(ts_ctx *ctx, const double *hx, const double *hy)
{
    if (!ctx)
        return TS_ERR_ARG;
    const int N = ctx->N;
    if ((hx && !finite_all(hx, N)) || (hy && !finite_all(hy, N)))
        return fail(ctx, TS_ERR_ARG, "ts_set_transverse_fields: non-finite field");
    const ts_status fst = flush_tail(ctx);   // the held-back slot belongs to the old H
    if (fst)
        return fst;
    for (int i = 0; i < N; i++) {
        ctx->hraw[0][i] = hx ? hx[i] : 0.0;
        ctx->hraw[1][i] = hy ? hy[i] : 0.0;
        ctx->hh[0 * N + i] = hx ? hx[i] / 2.0 : 0.0;
        ctx->hh[1 * N + i] = hy ? hy[i] / 2.0 : 0.0;
    }
    TS_CUDA(ctx, cudaMemcpyAsync(ctx->dhh, ctx->hh.data(), ctx->hh.size() * sizeof(double), cudaMemcpyHostToDevice,
                                 ctx->stream));
    TS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    reset_schedule(ctx->sched, ctx->stream);
    reset_schedule(ctx->sched_obs, ctx->stream);
    reset_schedule(ctx->sched_tail, ctx->stream);
    if (ctx->dE) {   // the phase tables hold the old fields: rebuild them
        ts_set_phase_tables(ctx, 0);
        return ts_set_phase_tables(ctx, 1);
    }
    return TS_OK;
}

ts_status ts_bind_buffers(ts_ctx *ctx, void *psi, void *ref, void *scratch, size_t bytes_each)
{
    if (!ctx)
        return TS_ERR_ARG;
    if (!psi)
        return fail(ctx, TS_ERR_ARG, "ts_bind_buffers: psi is NULL");
    if (bytes_each < state_bytes(ctx))
        return fail(ctx, TS_ERR_ARG, "ts_bind_buffers: buffers hold fewer than 2^N amplitudes");
    for (void *p : {psi, ref, scratch})
        if (p && ((uintptr_t)p & 255))
            return fail(ctx, TS_ERR_ARG, "ts_bind_buffers: buffer not 256-byte aligned");
    if (psi != ctx->psi.p)
        ctx->tail_pending = false;
    free_buf(ctx->psi);
    ctx->psi.p = psi;
    if (ref) {
        free_buf(ctx->ref);
        ctx->ref.p = ref;
        ctx->ref_valid = false;
    }
    if (scratch) {
        free_buf(ctx->scratch);
        ctx->scratch.p = scratch;
    }
    return TS_OK;
}

ts_status ts_set_state(ts_ctx *ctx, const void *amps, int on_device)
{
    if (!ctx || !amps)
        return ctx ? fail(ctx, TS_ERR_ARG, "ts_set_state: NULL amplitudes") : TS_ERR_ARG;
    ts_status st = ensure_buf(ctx, ctx->psi, "state buffer");
    if (st)
        return st;
    ctx->tail_pending = false;
    TS_CUDA(ctx, cudaMemcpyAsync(ctx->psi.p, amps, state_bytes(ctx),
                                 on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
    if (!on_device)
        TS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return TS_OK;
}

ts_status ts_set_basis_state(ts_ctx *ctx, uint64_t s)
{
    if (!ctx)
        return TS_ERR_ARG;
    if (s >= dim_of(ctx))
        return fail(ctx, TS_ERR_ARG, "ts_set_basis_state: index out of range");
    ts_status st = ensure_buf(ctx, ctx->psi, "state buffer");
    if (st)
        return st;
    ctx->tail_pending = false;
    const unsigned g = grid_for(ctx, dim_of(ctx), 256);
    if (ctx->prec == TS_C64)
        k_set_basis<float2><<<g, 256, 0, ctx->stream>>>((float2 *)ctx->psi.p, dim_of(ctx), s);
    else
        k_set_basis<double2><<<g, 256, 0, ctx->stream>>>((double2 *)ctx->psi.p, dim_of(ctx), s);
    ctx->launches++;
    TS_CUDA(ctx, cudaGetLastError());
    return TS_OK;
}

ts_status ts_save_reference(ts_ctx *ctx)
{
    if (!ctx)
        return TS_ERR_ARG;
    if (!ctx->psi.p)
        return fail(ctx, TS_ERR_STATE, "ts_save_reference: no state set");
    ts_status st = flush_tail(ctx);
    if (st)
        return st;
    st = ensure_buf(ctx, ctx->ref, "reference buffer");
    if (st)
        return st;
    TS_CUDA(ctx, cudaMemcpyAsync(ctx->ref.p, ctx->psi.p, state_bytes(ctx), cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->ref_valid = true;
    return TS_OK;
}

ts_status ts_step_order(ts_ctx *ctx, int order, double tau, int64_t nsteps)
{
    if (!ctx)
        return TS_ERR_ARG;
    if (!std::isfinite(tau) || nsteps < 0 || (order != 1 && order != 2 && order != 4))
        return fail(ctx, TS_ERR_ARG, "ts_step: tau must be finite, nsteps >= 0, order in {1, 2, 4}");
    if (!ctx->psi.p)
        return fail(ctx, TS_ERR_STATE, "ts_step: no state set");
    if (nsteps == 0)
        return TS_OK;
    {
        // Eq. 4: the step must be small against the largest local time scale of H
        const double bound = step_bound_of(ctx->N, ctx->Jraw, ctx->hraw);
        if (std::fabs(tau) >= bound) {
            char msg[200];
            std::snprintf(msg, sizeof(msg),
                          "warning: |tau| = %.6g is not small against the Eq. 4 time scale %.6g of this "
                          "Hamiltonian; the Trotter-Suzuki error may be large", std::fabs(tau), bound);
            ctx->err = msg;
        }
    }
    std::vector<HostSlot> slots = make_slots(ctx->N, order, tau, nsteps);
    // With chaining on, consecutive calls run like one chained call (Sec. 2: the P_z halves of
    // adjacent U2s merge): a held-back final pass of the previous call is merged into this
    // call's first pass, and with an even number of layers (orders 2 and 4) this call's final
    // pass is held back in turn.  Both ends of such a run sit on the first group of the zigzag.
    const bool fused = fused_usable(ctx);
    std::vector<Group> G;
    if (fused)
        G = make_groups(ctx->N, ctx->TB, ctx->cbits);
    const int ng = (int)G.size();
    const int first = ng >= 3 ? 1 : 0;
    int shape = 0;
    if (ctx->tail_pending) {
        if (fused && ng >= 2 && ctx->tail_group == first) {
            slots[0] = merge_z(ctx->tail_slot, slots[0]);
            shape |= SHAPE_HEAD_MERGED;
            ctx->tail_pending = false;
        } else {
            const ts_status fst = flush_tail(ctx);
            if (fst)
                return fst;
        }
    }
    const bool defer = ctx->chain && fused && ng >= 2 && (order == 2 || order == 4);
    if (defer)
        shape |= SHAPE_TAIL_DEFERRED;
    const ts_status st = run_slots(ctx, ctx->sched, ctx->psi.p, order, tau, nsteps, 0, slots, shape, 0);
    if (st == TS_OK && defer) {
        ctx->tail_pending = true;
        ctx->tail_slot = slots.back();
        ctx->tail_group = first;
        ctx->tail_h = G[(size_t)first].h;
    }
    return st;
}

ts_status ts_step(ts_ctx *ctx, double tau, int64_t nsteps) { return ts_step_order(ctx, 4, tau, nsteps); }

ts_status ts_set_chaining(ts_ctx *ctx, int enable)
{
    if (!ctx)
        return TS_ERR_ARG;
    ctx->chain = enable != 0;
    return enable ? TS_OK : flush_tail(ctx);
}

ts_status ts_flush(ts_ctx *ctx)
{
    if (!ctx)
        return TS_ERR_ARG;
    return flush_tail(ctx);
}

ts_status ts_observe(ts_ctx *ctx, int what, double *out)
{
    if (!ctx || !out)
        return ctx ? fail(ctx, TS_ERR_ARG, "ts_observe: NULL output") : TS_ERR_ARG;
    if (!ctx->psi.p)
        return fail(ctx, TS_ERR_STATE, "ts_observe: no state set");
    const int N = ctx->N;
    ts_status st = TS_OK;
    if (what == TS_NORM) {
        // a held-back pass is a Walsh-Hadamard rotation of tail_h spins (norm x 2^tail_h, the
        // butterflies are unnormalised) and a diagonal slot of modulus mag 2^-scale_exp
        st = sum_norm(ctx, ctx->psi.p, out);
        if (st == TS_OK && ctx->tail_pending) {
            const double m = std::ldexp(ctx->tail_slot.mag, -ctx->tail_slot.scale_exp);
            out[0] *= std::ldexp(m * m, ctx->tail_h);
        }
        return st;
    }
    st = flush_tail(ctx);
    if (st)
        return st;
    switch (what) {
    case TS_NORM:
        return sum_norm(ctx, ctx->psi.p, out);
    case TS_SZ: {
        std::vector<double> v(N + 1);
        st = sum_sz(ctx, ctx->psi.p, v.data());
        if (!st)
            for (int i = 0; i < N; i++)
                out[i] = v[1 + i] - 0.5 * v[0];
        return st;
    }
    case TS_ECHO:
    case TS_OVERLAP: {
        if (!ctx->ref_valid)
            return fail(ctx, TS_ERR_STATE, "ts_observe: no reference saved (ts_save_reference)");
        double ov[2];
        st = sum_overlap(ctx, ctx->ref.p, ctx->psi.p, ov);
        if (st)
            return st;
        if (what == TS_ECHO)
            out[0] = ov[0] * ov[0] + ov[1] * ov[1];
        else {
            out[0] = ov[0];
            out[1] = ov[1];
        }
        return TS_OK;
    }
    case TS_SZSZ:
    case TS_SXSX:
    case TS_SYSY: {
        const int alpha = what == TS_SXSX ? 0 : (what == TS_SYSY ? 1 : 2);
        const void *buf = ctx->psi.p;
        double wscale = 1.0;
        if (alpha < 2) {
            st = frame_copy(ctx, alpha);
            if (st)
                return st;
            buf = ctx->scratch.p;
            wscale = std::ldexp(1.0, -N);
        }
        std::vector<double> v(1 + N + N * (N - 1) / 2);
        st = sum_pairs(ctx, buf, v.data());
        if (!st)
            pairs_to_correlations(N, v.data(), wscale, out);
        return st;
    }
    case TS_SX:
    case TS_SY: {
        st = frame_copy(ctx, what == TS_SX ? 0 : 1);
        if (st)
            return st;
        std::vector<double> v(N + 1);
        st = sum_sz(ctx, ctx->scratch.p, v.data());
        if (!st)
            for (int i = 0; i < N; i++)
                out[i] = std::ldexp(v[1 + i] - 0.5 * v[0], -N);
        return st;
    }
    case TS_ENERGY: {
        double ez = 0.0, ex = 0.0, ey = 0.0;
        st = sum_diag(ctx, ctx->psi.p, 2, &ez);
        if (!st)
            st = rotated_energy(ctx, 0, &ex);
        if (!st)
            st = rotated_energy(ctx, 1, &ey);
        if (!st)
            out[0] = ex + ey + ez;
        return st;
    }
    default:
        return fail(ctx, TS_ERR_ARG, "ts_observe: unknown observable");
    }
}

ts_status ts_get_state(ts_ctx *ctx, void *amps, int on_device)
{
    if (!ctx || !amps)
        return ctx ? fail(ctx, TS_ERR_ARG, "ts_get_state: NULL destination") : TS_ERR_ARG;
    if (!ctx->psi.p)
        return fail(ctx, TS_ERR_STATE, "ts_get_state: no state set");
    const ts_status fst = flush_tail(ctx);
    if (fst)
        return fst;
    TS_CUDA(ctx, cudaMemcpyAsync(amps, ctx->psi.p, state_bytes(ctx),
                                 on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    if (!on_device)
        TS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return TS_OK;
}

ts_status ts_destroy(ts_ctx *ctx)
{
    if (!ctx)
        return TS_OK;
    cudaStreamSynchronize(ctx->stream);
    free_buf(ctx->psi);
    free_buf(ctx->ref);
    free_buf(ctx->scratch);
    if (ctx->dJq)
        cudaFree(ctx->dJq);
    if (ctx->dhh)
        cudaFree(ctx->dhh);
    if (ctx->dpart)
        cudaFree(ctx->dpart);
    release_tables(ctx->sched, ctx->stream);
    release_tables(ctx->sched_obs, ctx->stream);
    release_tables(ctx->sched_tail, ctx->stream);
    if (ctx->hout)
        cudaFreeHost(ctx->hout);
    if (ctx->dE)
        cudaFree(ctx->dE);
    delete ctx;
    return TS_OK;
}

ts_status ts_set_phase_tables(ts_ctx *ctx, int enable)
{
    if (!ctx)
        return TS_ERR_ARG;
    if (!enable) {
        if (ctx->dE) {
            cudaStreamSynchronize(ctx->stream);
            cudaFree(ctx->dE);
        }
        ctx->dE = nullptr;
        return TS_OK;
    }
    if (ctx->dE)
        return TS_OK;
    const uint64_t dim = dim_of(ctx);
    const size_t esize = ctx->prec == TS_C64 ? sizeof(float) : sizeof(double);
    const size_t bytes = 3 * (size_t)dim * esize;
    size_t freeb = 0, totb = 0;
    TS_CUDA(ctx, cudaMemGetInfo(&freeb, &totb));
    if (bytes > freeb)
        return fail(ctx, TS_ERR_OOM, "ts_set_phase_tables: the three 2^N tables do not fit");
    TS_CUDA(ctx, cudaMalloc(&ctx->dE, bytes));
    const HamDev hd = ham_dev(ctx);
    const unsigned gs = grid_for(ctx, dim, 256);
    for (int a = 0; a < 3; a++) {
        if (ctx->prec == TS_C64)
            k_energy_table<float><<<gs, 256, 0, ctx->stream>>>(static_cast<float *>(ctx->dE) + (size_t)a * dim,
                                                               dim, hd, a);
        else
            k_energy_table<double><<<gs, 256, 0, ctx->stream>>>(static_cast<double *>(ctx->dE) + (size_t)a * dim,
                                                                dim, hd, a);
        ctx->launches++;
    }
    TS_CUDA(ctx, cudaGetLastError());
    TS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return TS_OK;
}

ts_status ts_set_schedule(ts_ctx *ctx, int kernel, int tile_bits, int coalesce_bits)
{
    if (!ctx)
        return TS_ERR_ARG;
    if (kernel != TS_KERNEL_FUSED && kernel != TS_KERNEL_BASIC)
        return fail(ctx, TS_ERR_ARG, "ts_set_schedule: unknown kernel");
    const int tb = tile_bits ? tile_bits : default_tile(ctx->prec);
    const int cb = coalesce_bits ? coalesce_bits : default_cbits_for(ctx->prec, ctx->N, tb);
    if (!tile_supported(ctx->prec, tb))
        return fail(ctx, TS_ERR_ARG, "ts_set_schedule: tile size not provided for this precision");
    if (cb < 1 || cb > tb - ctx->RB)
        return fail(ctx, TS_ERR_ARG, "ts_set_schedule: coalescing bits must be in [1, tile_bits - reg_bits]");
    const ts_status fst = flush_tail(ctx);   // the held-back pass uses the current tiles
    if (fst)
        return fst;
    ctx->kernel = kernel;
    ctx->TB = tb;
    ctx->cbits = cb;
    reset_schedule(ctx->sched, ctx->stream);
    reset_schedule(ctx->sched_obs, ctx->stream);
    reset_schedule(ctx->sched_tail, ctx->stream);
    return TS_OK;
}

ts_status ts_get_schedule(const ts_ctx *ctx, int *kernel, int *tile_bits, int *coalesce_bits, int *groups,
                          int *passes_per_step)
{
    if (!ctx)
        return TS_ERR_ARG;
    int tb = ctx->TB;
    if (ctx->kernel == TS_KERNEL_FUSED && ctx->N < tb && tile_supported(ctx->prec, ctx->N))
        tb = ctx->N;
    const bool fused = ctx->kernel == TS_KERNEL_FUSED && ctx->N >= tb;
    const int g = fused ? (int)make_groups(ctx->N, tb, ctx->cbits).size() : 0;
    if (kernel)
        *kernel = fused ? TS_KERNEL_FUSED : TS_KERNEL_BASIC;
    if (tile_bits)
        *tile_bits = fused ? tb : 0;
    if (coalesce_bits)
        *coalesce_bits = fused ? ctx->cbits : 0;
    if (groups)
        *groups = g;
    if (passes_per_step)
        *passes_per_step = fused ? (g == 1 ? 20 : 20 * (g - 1)) : 20 * ctx->N + 20;
    return TS_OK;
}

double ts_step_bound(const ts_ctx *ctx)
{
    if (!ctx)
        return 0.0;
    return step_bound_of(ctx->N, ctx->Jraw, ctx->hraw);
}

double ts_step_bound_host(int N, const double *Jx, const double *Jy, const double *Jz, const double *hx,
                          const double *hy, const double *hz)
{
    if (N < 1 || N > kMaxN || !Jx || !Jy || !Jz)
        return -1.0;
    std::vector<double> J[3], h[3];
    const double *Js[3] = {Jx, Jy, Jz}, *hs[3] = {hx, hy, hz};
    for (int a = 0; a < 3; a++) {
        J[a].assign(Js[a], Js[a] + (size_t)N * N);
        h[a].assign((size_t)N, 0.0);
        if (hs[a])
            h[a].assign(hs[a], hs[a] + N);
    }
    return step_bound_of(N, J, h);
}

} // extern "C"

// ================================================================== batched ensemble
//
// Many states of several systems (uneven N) advance together: one launch of the
// persistent kernel k_tile_ensemble runs every pass of every state of a
// ts_batch_step (per-state completion counters order the passes of a state), and
// that launch, with the resets of its counters, is captured into one CUDA graph
// and replayed.

struct ts_batch {
    int nsys = 0;
    ts_prec prec = TS_C64;
    cudaStream_t stream = nullptr;       // the caller's stream: graphs are launched here
    cudaStream_t cap = nullptr;          // private stream used only to capture the graph
    int TB = 0, cbits = 0;
    std::vector<ts_ctx *> sys;       // couplings and schedule of each system
    std::vector<int> nstates;
    std::vector<Buf> psi;            // nstates x 2^N amplitudes per system
    // device copies of the per-pass launch arguments
    BatchSys *dsys = nullptr;
    TileArgs *dargs = nullptr;
    size_t dcap = 0;                 // entries
    std::vector<uint64_t> blocks;    // work items (chunks of tiles) per pass index
    uint64_t *dpstart = nullptr;     // first work item of each pass (npass + 1)
    size_t pstart_cap = 0;           // entries
    // synchronisation words of the persistent kernel: ticket, per-state counters, status
    unsigned long long *dsync = nullptr;
    size_t sync_cap = 0;             // counters (ticket + states)
    int *dstatus = nullptr;          // [0] sticky status, [1] the word nothing writes
    int *hstatus = nullptr;          // pinned copy of the status after each launch
    double wait_limit_s = 2.0;       // longest dependency wait of a launch
    int hold = 0;                    // test of the timeout path
    unsigned grid = 0;               // persistent blocks: SMs x resident blocks per SM
    // cached graph of the last (tau, nsteps)
    cudaGraphExec_t gexec = nullptr;
    double g_tau = 0.0;
    int64_t g_n = -1;
    int64_t g_nodes = 0;
    double *dpart = nullptr;
    size_t part_cap = 0;
    double *hout = nullptr;
    std::string err;
    int64_t launches = 0;
};

namespace {

ts_status bfail(ts_batch *b, ts_status st, const std::string &msg)
{
    if (b)
        b->err = msg;
    return st;
}

#define TS_BCUDA(b, call)                                                                         \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return bfail((b), e_ == cudaErrorMemoryAllocation ? TS_ERR_OOM : TS_ERR_CUDA,         \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                     \
    } while (0)

// Tiles per work item of the persistent ensemble kernel: 2^3 (fewer ticket atomics and
// counter updates per tile; a state's pass always splits into whole items).
constexpr int kEnsembleChunkShift = 3;

size_t batch_state_bytes(const ts_batch *b, int s)
{
    return (size_t)b->nstates[s] * state_bytes(b->sys[s]);
}

template <typename R, int TB, int RB>
cudaError_t launch_batch_t(const ts_batch *b, const BatchSync &sy, bool attr, unsigned *grid)
{
    using K = TileKernel<R, TB, RB>;
    constexpr size_t smem = sizeof(typename CT<R>::T) * K::SMEM_ELEMS;
    if (attr) {
        cudaError_t e = cudaFuncSetAttribute(k_tile_ensemble<R, TB, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess)
            return e;
        int per_sm = 0, dev = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile_ensemble<R, TB, RB>, K::NT, smem);
        if (e == cudaSuccess)
            e = cudaGetDevice(&dev);
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        *grid = (unsigned)(std::max(per_sm, 1) * std::max(sms, 1));
        return e;
    }
    k_tile_ensemble<R, TB, RB><<<*grid, K::NT, smem, b->stream>>>(b->dsys, b->dargs, b->nsys, sy);
    return cudaGetLastError();
}

// attr: set the kernel's shared-memory attribute and size the persistent grid; otherwise launch.
cudaError_t launch_batch(ts_batch *b, const BatchSync &sy, bool attr)
{
    unsigned *g = &b->grid;
    if (b->prec == TS_C64) {
        switch (b->TB) {
        case 12: return launch_batch_t<float, 12, 5>(b, sy, attr, g);
        case 13: return launch_batch_t<float, 13, 5>(b, sy, attr, g);
        default: return launch_batch_t<float, 14, 5>(b, sy, attr, g);
        }
    }
    switch (b->TB) {
    case 11: return launch_batch_t<double, 11, 4>(b, sy, attr, g);
    case 12: return launch_batch_t<double, 12, 4>(b, sy, attr, g);
    default: return launch_batch_t<double, 13, 4>(b, sy, attr, g);
    }
}

void batch_drop_graph(ts_batch *b)
{
    if (b->gexec)
        cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    b->g_n = -1;
}

// Builds every system's schedule for U4(tau)^n, the per-pass launch arguments, and
// captures the launches into a CUDA graph.
ts_status batch_prepare(ts_batch *b, double tau, int64_t n)
{
    batch_drop_graph(b);
    size_t maxp = 0;
    for (int s = 0; s < b->nsys; s++) {
        ts_ctx *c = b->sys[s];
        c->TB = b->TB;
        c->cbits = b->cbits;
        c->kernel = TS_KERNEL_FUSED;
        reset_schedule(c->sched, b->stream);
        c->sched.slots = make_slots(c->N, 4, tau, n);
        ts_status st = prepare_fused(c, c->sched);
        if (st)
            return bfail(b, st, std::string("system schedule: ") + c->err);
        maxp = std::max(maxp, c->sched.passes.size());
    }
    const size_t need = maxp * (size_t)b->nsys;
    if (need > b->dcap) {
        if (b->dsys)
            cudaFree(b->dsys);
        if (b->dargs)
            cudaFree(b->dargs);
        b->dsys = nullptr;
        b->dargs = nullptr;
        b->dcap = 0;
        TS_BCUDA(b, cudaMalloc(&b->dsys, need * sizeof(BatchSys)));
        TS_BCUDA(b, cudaMalloc(&b->dargs, need * sizeof(TileArgs)));
        b->dcap = need;
    }
    std::vector<BatchSys> hs(need);
    std::vector<TileArgs> ha(need);
    b->blocks.assign(maxp, 0);
    for (size_t p = 0; p < maxp; p++) {
        uint32_t start = 0;
        for (int s = 0; s < b->nsys; s++) {
            ts_ctx *c = b->sys[s];
            const Schedule &S = c->sched;
            BatchSys &bs = hs[p * b->nsys + s];
            TileArgs &a = ha[p * b->nsys + s];
            std::memset(&bs, 0, sizeof(bs));
            std::memset(&a, 0, sizeof(a));
            bs.psi = b->psi[s].p;
            bs.tabs = S.dtab;
            bs.n = c->N;
            bs.tile_shift = c->N - b->TB;
            bs.chunk_shift = std::min(bs.tile_shift, kEnsembleChunkShift);
            bs.block_start = start;
            bs.state_base = 0;
            for (int q = 0; q < s; q++)
                bs.state_base += (uint32_t)b->nstates[q];
            bs.active = p < S.passes.size();
            if (!bs.active)
                continue;
            const HostPass &hp = S.passes[p];
            const Group &g = S.groups[hp.group];
            a.c = g.c;
            a.w = g.w;
            a.h = g.h;
            a.nsteps = hp.nsteps;
            std::memcpy(a.steps, hp.steps, sizeof(hp.steps));
            a.has_slot = hp.slot >= 0;
            if (hp.slot >= 0)
                a.slot = S.slots[hp.slot].dev();
            a.tab = hp.tab < 0 ? 0 : hp.tab;
            a.exact_sincos = hp.ymode;
            a.io = S.io[hp.group];
            a.ham = ham_dev(c);
            a.theta = hp.slot >= 0 ? S.dtheta + hp.theta_off : nullptr;
            a.gfield = hp.slot >= 0 ? gfield_at(c, S, hp.theta_off) : nullptr;
            set_io_args(a, c, S, hp.group);
            a.ens_shape = (b->prec == TS_C64 && b->TB == 12) ? ensemble_shape_id(a) : 0;
            start += (uint32_t)((uint64_t)b->nstates[s] << (bs.tile_shift - bs.chunk_shift));
        }
        b->blocks[p] = start;
    }
    // first work item of every pass, and the synchronisation words
    std::vector<uint64_t> pst(maxp + 1, 0);
    for (size_t p = 0; p < maxp; p++)
        pst[p + 1] = pst[p] + b->blocks[p];
    if (pst.size() > b->pstart_cap) {
        if (b->dpstart)
            cudaFree(b->dpstart);
        b->dpstart = nullptr;
        b->pstart_cap = 0;
        TS_BCUDA(b, cudaMalloc(&b->dpstart, pst.size() * sizeof(uint64_t)));
        b->pstart_cap = pst.size();
    }
    size_t nst = 0;
    for (int s = 0; s < b->nsys; s++)
        nst += (size_t)b->nstates[s];
    if (1 + nst > b->sync_cap) {
        if (b->dsync)
            cudaFree(b->dsync);
        b->dsync = nullptr;
        b->sync_cap = 0;
        TS_BCUDA(b, cudaMalloc(&b->dsync, (1 + nst) * sizeof(unsigned long long)));
        b->sync_cap = 1 + nst;
    }
    if (!b->dstatus) {
        TS_BCUDA(b, cudaMalloc(&b->dstatus, 2 * sizeof(int)));
        TS_BCUDA(b, cudaMemsetAsync(b->dstatus, 0, 2 * sizeof(int), b->stream));
    }
    if (!b->hstatus) {
        TS_BCUDA(b, cudaHostAlloc(&b->hstatus, sizeof(int), cudaHostAllocDefault));
        *b->hstatus = 0;
    }
    TS_BCUDA(b, cudaMemcpyAsync(b->dsys, hs.data(), need * sizeof(BatchSys), cudaMemcpyHostToDevice, b->stream));
    TS_BCUDA(b, cudaMemcpyAsync(b->dargs, ha.data(), need * sizeof(TileArgs), cudaMemcpyHostToDevice, b->stream));
    TS_BCUDA(b, cudaMemcpyAsync(b->dpstart, pst.data(), pst.size() * sizeof(uint64_t), cudaMemcpyHostToDevice,
                                b->stream));
    TS_BCUDA(b, cudaStreamSynchronize(b->stream));
    BatchSync sy;
    sy.ticket = b->dsync;
    sy.done = b->dsync + 1;
    sy.status = b->dstatus;
    sy.hold_flag = b->dstatus + 1;
    sy.pstart = b->dpstart;
    sy.limit_ns = (uint64_t)(b->wait_limit_s * 1e9);
    sy.npass = (int)maxp;
    sy.hold = b->hold;
    TS_BCUDA(b, launch_batch(b, sy, true));
    // capture the whole evolution into one graph: reset the ticket and the per-state counters,
    // run the persistent kernel, copy the status out
    cudaGraph_t graph = nullptr;
    // (the legacy default stream cannot be captured: record on a private stream)
    TS_BCUDA(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    const cudaStream_t user = b->stream;
    b->stream = b->cap;
    cudaError_t ce = cudaMemsetAsync(b->dsync, 0, (1 + nst) * sizeof(unsigned long long), b->cap);
    if (ce == cudaSuccess && pst[maxp] > 0)
        ce = launch_batch(b, sy, false);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(b->hstatus, b->dstatus, sizeof(int), cudaMemcpyDeviceToHost, b->cap);
    b->stream = user;
    cudaError_t ee = cudaStreamEndCapture(b->cap, &graph);
    if (ce != cudaSuccess || ee != cudaSuccess) {
        if (graph)
            cudaGraphDestroy(graph);
        return bfail(b, TS_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce != cudaSuccess ? ce : ee));
    }
    size_t nodes = 0;
    cudaGraphGetNodes(graph, nullptr, &nodes);
    cudaError_t ie = cudaGraphInstantiate(&b->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
        b->gexec = nullptr;
        return bfail(b, TS_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
    }
    b->g_tau = tau;
    b->g_n = n;
    b->g_nodes = pst[maxp] > 0 ? 1 : 0;   // kernel launches per replay (the other nodes are copies)
    (void)nodes;
    return TS_OK;
}

// Waits for the batch's queued work; TS_ERR_TIMEOUT (once) if a dependency wait of the
// persistent kernel ran out since the last check.
ts_status batch_check(ts_batch *b)
{
    TS_BCUDA(b, cudaStreamSynchronize(b->stream));
    if (b->hstatus && *b->hstatus) {
        *b->hstatus = 0;
        TS_BCUDA(b, cudaMemsetAsync(b->dstatus, 0, sizeof(int), b->stream));
        TS_BCUDA(b, cudaStreamSynchronize(b->stream));
        return bfail(b, TS_ERR_TIMEOUT, "ts_batch_step: a dependency wait of the ensemble kernel ran out; the "
                                        "states are undefined until they are set again");
    }
    return TS_OK;
}

} // namespace

extern "C" {

ts_status ts_batch_create(ts_batch **out, int nsys, const int *N, const double *const *Jx, const double *const *Jy,
                          const double *const *Jz, const double *const *h, const int *nstates, ts_prec prec,
                          void *cuda_stream)
{
    if (!out)
        return TS_ERR_ARG;
    *out = nullptr;
    if (nsys < 1 || !N || !Jx || !Jy || !Jz || !nstates || (prec != TS_C64 && prec != TS_C128))
        return TS_ERR_ARG;
    ts_batch *b = new (std::nothrow) ts_batch();
    if (!b)
        return TS_ERR_OOM;
    b->nsys = nsys;
    b->prec = prec;
    b->stream = (cudaStream_t)cuda_stream;
    b->TB = default_tile(prec);
    b->cbits = default_cbits(prec);
    int nmin = 64;
    for (int s = 0; s < nsys; s++) {
        if (nstates[s] < 1) {
            ts_batch_destroy(b);
            return TS_ERR_ARG;
        }
        ts_ctx *c = nullptr;
        ts_status st = ts_create(&c, N[s], Jx[s], Jy[s], Jz[s], h ? h[s] : nullptr, prec, cuda_stream);
        if (st) {
            ts_batch_destroy(b);
            return st;
        }
        b->sys.push_back(c);
        b->nstates.push_back(nstates[s]);
        b->psi.push_back(Buf());
        nmin = std::min(nmin, N[s]);
    }
    if (!tile_supported(prec, b->TB) || nmin < b->TB) {
        // the smallest system sets the largest usable tile
        int tb = std::min(b->TB, nmin);
        if (!tile_supported(prec, tb)) {
            ts_batch_destroy(b);
            return TS_ERR_ARG;
        }
        b->TB = tb;
    }
    {
        std::vector<int> ns(N, N + nsys), ks(nstates, nstates + nsys);
        b->cbits = default_cbits_batch(prec, b->TB, ns, ks);
    }
    TS_BCUDA(b, cudaMallocHost(&b->hout, (kMaxN + 8) * sizeof(double)));
    TS_BCUDA(b, cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    *out = b;
    return TS_OK;
}

ts_status ts_batch_bind_states(ts_batch *b, int sys, void *dev, size_t bytes)
{
    if (!b || sys < 0 || sys >= b->nsys || !dev)
        return b ? bfail(b, TS_ERR_ARG, "ts_batch_bind_states: bad system or pointer") : TS_ERR_ARG;
    if (bytes < batch_state_bytes(b, sys) || ((uintptr_t)dev & 255))
        return bfail(b, TS_ERR_ARG, "ts_batch_bind_states: buffer too small or not 256-byte aligned");
    free_buf(b->psi[sys]);
    b->psi[sys].p = dev;
    batch_drop_graph(b);
    return TS_OK;
}

static ts_status batch_ensure(ts_batch *b, int s)
{
    if (b->psi[s].p)
        return TS_OK;
    cudaError_t e = cudaMalloc(&b->psi[s].p, batch_state_bytes(b, s));
    if (e != cudaSuccess) {
        b->psi[s].p = nullptr;
        return bfail(b, TS_ERR_OOM, "ts_batch: state buffer allocation failed");
    }
    b->psi[s].own = true;
    batch_drop_graph(b);
    return TS_OK;
}

ts_status ts_batch_set_states(ts_batch *b, int sys, const void *amps, int on_device)
{
    if (!b || sys < 0 || sys >= b->nsys || !amps)
        return b ? bfail(b, TS_ERR_ARG, "ts_batch_set_states: bad system or pointer") : TS_ERR_ARG;
    ts_status st = batch_ensure(b, sys);
    if (st)
        return st;
    TS_BCUDA(b, cudaMemcpyAsync(b->psi[sys].p, amps, batch_state_bytes(b, sys),
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, b->stream));
    if (!on_device)
        TS_BCUDA(b, cudaStreamSynchronize(b->stream));
    return TS_OK;
}

ts_status ts_batch_get_states(ts_batch *b, int sys, void *amps, int on_device)
{
    if (!b || sys < 0 || sys >= b->nsys || !amps || !b->psi[sys].p)
        return b ? bfail(b, TS_ERR_ARG, "ts_batch_get_states: bad system, pointer or no state") : TS_ERR_ARG;
    TS_BCUDA(b, cudaMemcpyAsync(amps, b->psi[sys].p, batch_state_bytes(b, sys),
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream));
    if (!on_device)
        return batch_check(b);
    return TS_OK;
}

ts_status ts_batch_set_schedule(ts_batch *b, int tile_bits, int coalesce_bits)
{
    if (!b)
        return TS_ERR_ARG;
    int nmin = 64;
    for (auto *c : b->sys)
        nmin = std::min(nmin, c->N);
    const int tb = tile_bits ? tile_bits : std::min(default_tile(b->prec), nmin);
    std::vector<int> ns, ks;
    for (int s = 0; s < b->nsys; s++) {
        ns.push_back(b->sys[(size_t)s]->N);
        ks.push_back(b->nstates[(size_t)s]);
    }
    const int cb = coalesce_bits ? coalesce_bits : default_cbits_batch(b->prec, tb, ns, ks);
    if (!tile_supported(b->prec, tb) || tb > nmin || cb < 1 || cb > tb - reg_bits(b->prec))
        return bfail(b, TS_ERR_ARG, "ts_batch_set_schedule: tile not provided or larger than the smallest system");
    b->TB = tb;
    b->cbits = cb;
    batch_drop_graph(b);
    return TS_OK;
}

ts_status ts_batch_step(ts_batch *b, double tau, int64_t nsteps)
{
    if (!b)
        return TS_ERR_ARG;
    if (!std::isfinite(tau) || nsteps < 0)
        return bfail(b, TS_ERR_ARG, "ts_batch_step: tau must be finite and nsteps >= 0");
    for (int s = 0; s < b->nsys; s++)
        if (!b->psi[s].p)
            return bfail(b, TS_ERR_STATE, "ts_batch_step: a system has no states set");
    if (nsteps == 0)
        return TS_OK;
    if (b->hstatus && *b->hstatus)   // an earlier launch gave up: report it before more work
        return batch_check(b);
    if (!b->gexec || b->g_tau != tau || b->g_n != nsteps) {
        ts_status st = batch_prepare(b, tau, nsteps);
        if (st)
            return st;
    }
    TS_BCUDA(b, cudaGraphLaunch(b->gexec, b->stream));
    b->launches += b->g_nodes;
    return TS_OK;
}

ts_status ts_batch_status(ts_batch *b)
{
    if (!b)
        return TS_ERR_ARG;
    return batch_check(b);
}

ts_status ts_batch_set_wait(ts_batch *b, double limit_s, int hold)
{
    if (!b)
        return TS_ERR_ARG;
    if (!(limit_s > 0.0) || !std::isfinite(limit_s) || limit_s > 8.0)
        return bfail(b, TS_ERR_ARG, "ts_batch_set_wait: the limit must be in (0, 8] seconds");
    b->wait_limit_s = limit_s;
    b->hold = hold != 0;
    batch_drop_graph(b);
    return TS_OK;
}

ts_status ts_batch_observe(ts_batch *b, int what, double *out)
{
    if (!b || !out)
        return b ? bfail(b, TS_ERR_ARG, "ts_batch_observe: NULL output") : TS_ERR_ARG;
    if (what != TS_NORM && what != TS_SZ)
        return bfail(b, TS_ERR_ARG, "ts_batch_observe: only TS_NORM and TS_SZ are batched");
    {
        const ts_status cs = batch_check(b);
        if (cs)
            return cs;
    }
    size_t o = 0;
    for (int s = 0; s < b->nsys; s++) {
        ts_ctx *c = b->sys[s];
        if (!b->psi[s].p)
            return bfail(b, TS_ERR_STATE, "ts_batch_observe: a system has no states set");
        const size_t sb = state_bytes(c);
        for (int k = 0; k < b->nstates[s]; k++) {
            std::vector<double> v(c->N + 1);
            ts_status st = sum_sz(c, (const char *)b->psi[s].p + (size_t)k * sb, v.data());
            if (st)
                return bfail(b, st, c->err);
            b->launches += 2;
            if (what == TS_NORM)
                out[o++] = v[0];
            else
                for (int j = 0; j < c->N; j++)
                    out[o++] = v[1 + j] - 0.5 * v[0];
        }
    }
    return TS_OK;
}

int64_t ts_batch_kernel_launches(const ts_batch *b) { return b ? b->launches : 0; }

const char *ts_batch_last_error(const ts_batch *b) { return b ? b->err.c_str() : ""; }

ts_status ts_batch_destroy(ts_batch *b)
{
    if (!b)
        return TS_OK;
    cudaStreamSynchronize(b->stream);
    batch_drop_graph(b);
    for (auto &p : b->psi)
        free_buf(p);
    for (auto *c : b->sys)
        ts_destroy(c);
    if (b->dsys)
        cudaFree(b->dsys);
    if (b->dargs)
        cudaFree(b->dargs);
    if (b->dpstart)
        cudaFree(b->dpstart);
    if (b->dsync)
        cudaFree(b->dsync);
    if (b->dstatus)
        cudaFree(b->dstatus);
    if (b->hstatus)
        cudaFreeHost(b->hstatus);
    if (b->hout)
        cudaFreeHost(b->hout);
    if (b->cap)
        cudaStreamDestroy(b->cap);
    delete b;
    return TS_OK;
}

} // extern "C"

// ================================================================== autotuner
//
// Sec. 3.4 (last paragraph): no rotation schedule is best for every size, so the
// paper searched them by brute force and stored the winners in a file.  Here the
// search space is the tile size and the coalescing bits of the fused kernel.

namespace {

std::string device_name()
{
    int dev = 0;
    cudaDeviceProp p;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess)
        return "unknown";
    std::string n = p.name;
    for (auto &ch : n)
        if (ch == ' ')
            ch = '_';
    return n;
}

// Cache file lines: "<gpu> <N> <prec> <tile_bits> <coalesce_bits> <ms_per_step>"
bool tune_lookup(const char *path, const std::string &gpu, int N, int prec, int *tb, int *cb)
{
    FILE *f = path ? std::fopen(path, "r") : nullptr;
    if (!f)
        return false;
    char g[256];
    int n, p, t, c;
    double ms;
    bool found = false;
    while (std::fscanf(f, "%255s %d %d %d %d %lf", g, &n, &p, &t, &c, &ms) == 6)
        if (gpu == g && n == N && p == prec) {
            *tb = t;
            *cb = c;
            found = true;
        }
    std::fclose(f);
    return found;
}

void tune_store(const char *path, const std::string &gpu, int N, int prec, int tb, int cb, double ms)
{
    FILE *f = path ? std::fopen(path, "a") : nullptr;
    if (!f)
        return;
    std::fprintf(f, "%s %d %d %d %d %.6f\n", gpu.c_str(), N, prec, tb, cb, ms);
    std::fclose(f);
}

} // namespace

extern "C" {

ts_status ts_autotune(ts_ctx *ctx, double tau, int reps, const char *cache_path, double *best_ms)
{
    if (!ctx || !std::isfinite(tau) || reps < 1)
        return ctx ? fail(ctx, TS_ERR_ARG, "ts_autotune: tau must be finite and reps >= 1") : TS_ERR_ARG;
    if (!ctx->psi.p)
        return fail(ctx, TS_ERR_STATE, "ts_autotune: no state set");
    const ts_status fst = flush_tail(ctx);   // the tile shape may change
    if (fst)
        return fst;
    const std::string gpu = device_name();
    int tb = 0, cb = 0;
    if (tune_lookup(cache_path, gpu, ctx->N, (int)ctx->prec, &tb, &cb) && tile_supported(ctx->prec, tb) &&
        ctx->N >= tb) {
        if (best_ms)
            *best_ms = -1.0;
        return ts_set_schedule(ctx, TS_KERNEL_FUSED, tb, cb);
    }
    ts_status st = ensure_buf(ctx, ctx->scratch, "autotune scratch buffer");
    if (st)
        return st;
    const int keep_k = ctx->kernel, keep_tb = ctx->TB, keep_cb = ctx->cbits;
    double best = 1e300;
    int btb = keep_tb, bcb = keep_cb;
    cudaEvent_t e0, e1;
    TS_CUDA(ctx, cudaEventCreate(&e0));
    TS_CUDA(ctx, cudaEventCreate(&e1));
    const int tbs64[3] = {12, 13, 14}, tbs128[3] = {11, 12, 13};
    for (int i = 0; i < 3 && !st; i++) {
        const int t = ctx->prec == TS_C64 ? tbs64[i] : tbs128[i];
        if (ctx->N < t)
            continue;
        for (int c = 1; c <= 4 && !st; c++) {
            if (c > t - ctx->RB)
                continue;
            ctx->kernel = TS_KERNEL_FUSED;
            ctx->TB = t;
            ctx->cbits = c;
            Schedule trial;
            const std::vector<HostSlot> slots = make_slots(ctx->N, 4, tau, 1);
            if (cudaMemcpyAsync(ctx->scratch.p, ctx->psi.p, state_bytes(ctx), cudaMemcpyDeviceToDevice,
                                ctx->stream) != cudaSuccess) {
                st = TS_ERR_CUDA;
                break;
            }
            st = run_slots(ctx, trial, ctx->scratch.p, 4, tau, 1, 0, slots);   // warm-up and schedule build
            if (!st && cudaEventRecord(e0, ctx->stream) != cudaSuccess)
                st = TS_ERR_CUDA;
            for (int r = 0; r < reps && !st; r++)
                st = run_slots(ctx, trial, ctx->scratch.p, 4, tau, 1, 0, slots);
            if (!st && (cudaEventRecord(e1, ctx->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
                st = TS_ERR_CUDA;
            float ms = 0.f;
            if (!st && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms / reps < best) {
                best = ms / reps;
                btb = t;
                bcb = c;
            }
            reset_schedule(trial, ctx->stream);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->kernel = keep_k;
    ctx->TB = keep_tb;
    ctx->cbits = keep_cb;
    if (st)
        return fail(ctx, st, "ts_autotune: a trial failed: " + ctx->err);
    if (best_ms)
        *best_ms = best;
    tune_store(cache_path, gpu, ctx->N, (int)ctx->prec, btb, bcb, best);
    return ts_set_schedule(ctx, TS_KERNEL_FUSED, btb, bcb);
}

ts_status ts_batch_get_schedule(const ts_batch *b, int *tile_bits, int *coalesce_bits)
{
    if (!b)
        return TS_ERR_ARG;
    if (tile_bits)
        *tile_bits = b->TB;
    if (coalesce_bits)
        *coalesce_bits = b->cbits;
    return TS_OK;
}

ts_status ts_batch_autotune(ts_batch *b, double tau, int reps, const char *cache_path, double *best_ms)
{
    if (!b)
        return TS_ERR_ARG;
    if (!std::isfinite(tau) || reps < 1)
        return bfail(b, TS_ERR_ARG, "ts_batch_autotune: tau must be finite and reps >= 1");
    for (int s = 0; s < b->nsys; s++)
        if (!b->psi[s].p)
            return bfail(b, TS_ERR_STATE, "ts_batch_autotune: a system has no states set");
    // cache key: -(FNV-1a of the (N, nstates) list), so that it never equals a system size
    uint32_t h = 2166136261u;
    auto mix = [&h](uint32_t v) {
        for (int k = 0; k < 4; k++) {
            h ^= (v >> (8 * k)) & 0xffu;
            h *= 16777619u;
        }
    };
    int nmin = 64;
    std::vector<size_t> bytes(b->nsys);
    size_t total = 0;
    for (int s = 0; s < b->nsys; s++) {
        mix((uint32_t)b->sys[s]->N);
        mix((uint32_t)b->nstates[s]);
        nmin = std::min(nmin, b->sys[s]->N);
        bytes[s] = state_bytes(b->sys[s]) * (size_t)b->nstates[s];
        total += bytes[s];
    }
    const int key = -(int)(h & 0x7fffffffu);
    const std::string gpu = device_name();
    int tb = 0, cb = 0;
    if (tune_lookup(cache_path, gpu, key, (int)b->prec, &tb, &cb) && tile_supported(b->prec, tb) && tb <= nmin) {
        if (best_ms)
            *best_ms = -1.0;
        return ts_batch_set_schedule(b, tb, cb);
    }
    // the trials run on the ensemble's buffers: keep a device copy of every state
    void *save = nullptr;
    cudaError_t ce = cudaMalloc(&save, total);
    if (ce != cudaSuccess)
        return bfail(b, ce == cudaErrorMemoryAllocation ? TS_ERR_OOM : TS_ERR_CUDA,
                     "ts_batch_autotune: no room for a copy of the states");
    size_t off = 0;
    for (int s = 0; s < b->nsys && ce == cudaSuccess; s++) {
        ce = cudaMemcpyAsync((char *)save + off, b->psi[s].p, bytes[s], cudaMemcpyDeviceToDevice, b->stream);
        off += bytes[s];
    }
    const int keep_tb = b->TB, keep_cb = b->cbits;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ce == cudaSuccess)
        ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess)
        ce = cudaEventCreate(&e1);
    ts_status st = ce == cudaSuccess ? TS_OK : TS_ERR_CUDA;
    double best = 1e300;
    int btb = keep_tb, bcb = keep_cb;
    const int tbs64[3] = {12, 13, 14}, tbs128[3] = {11, 12, 13};
    for (int i = 0; i < 3 && !st; i++) {
        const int t = b->prec == TS_C64 ? tbs64[i] : tbs128[i];
        if (t > nmin)
            continue;
        for (int c = 1; c <= 4 && !st; c++) {
            if (c > t - reg_bits(b->prec))
                continue;
            st = ts_batch_set_schedule(b, t, c);
            if (!st)
                st = ts_batch_step(b, tau, 1);   // graph capture and warm-up
            if (!st && cudaEventRecord(e0, b->stream) != cudaSuccess)
                st = TS_ERR_CUDA;
            for (int r = 0; r < reps && !st; r++)
                st = ts_batch_step(b, tau, 1);
            if (!st && (cudaEventRecord(e1, b->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
                st = TS_ERR_CUDA;
            float ms = 0.f;
            if (!st && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms / reps < best) {
                best = ms / reps;
                btb = t;
                bcb = c;
            }
        }
    }
    const std::string trial_err = b->err;
    // the states as they were
    off = 0;
    cudaError_t re = cudaSuccess;
    for (int s = 0; s < b->nsys && re == cudaSuccess; s++) {
        re = cudaMemcpyAsync(b->psi[s].p, (char *)save + off, bytes[s], cudaMemcpyDeviceToDevice, b->stream);
        off += bytes[s];
    }
    if (re == cudaSuccess)
        re = cudaStreamSynchronize(b->stream);
    if (re == cudaSuccess && !st)
        st = batch_check(b);
    cudaFree(save);
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    if (re != cudaSuccess)
        return bfail(b, TS_ERR_CUDA, std::string("ts_batch_autotune: restoring the states: ") + cudaGetErrorString(re));
    if (st) {
        ts_batch_set_schedule(b, keep_tb, keep_cb);
        return bfail(b, st, "ts_batch_autotune: a trial failed: " + trial_err);
    }
    if (best_ms)
        *best_ms = best;
    tune_store(cache_path, gpu, key, (int)b->prec, btb, bcb, best);
    return ts_batch_set_schedule(b, btb, bcb);
}

} // extern "C"
