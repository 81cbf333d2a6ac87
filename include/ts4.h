/*
 * ts4.h -- C ABI of the GB300 (sm_103a) fourth-order Trotter-Suzuki solver for
 * spin-1/2 dynamics (Dente, Bederian, Zangara, Pastawski, "GPU accelerated
 * Trotter-Suzuki solver for quantum spin dynamics").
 *
 * The library evolves the full 2^N-amplitude state vector of
 *     H = sum_{i<j} sum_{a=x,y,z} J^a_ij S^a_i S^a_j + sum_i h^a_i S^a_i      (Eq. 1)
 * with the TS4 step of the XYZ decomposition (Sec. 2):
 *     U4(tau) = U2(p tau)^2 U2((1-4p) tau) U2(p tau)^2,  p = 1/(4 - 4^{1/3}),
 *     U2(t)   = U1^dag(-t/2) U1(t/2),  U1(t) = e^{-itH_x} e^{-itH_y} e^{-itH_z},
 * where e^{-itH_x} = Y e^{-itH~_x} Y^dag and e^{-itH_y} = X e^{-itH~_y} X^dag
 * map the X and Y parts onto diagonal Z-like phases (Eqs. 5, 7, 9, 10).
 *
 * Conventions
 *   - Spin j (1-based) is bit j-1 of the basis index; bit 1 is spin up
 *     (S^z = +1/2) (Sec. 3.2: spins are enumerated from right to left).
 *   - S = sigma/2.  Couplings are N*N row-major float64 matrices; only the
 *     upper triangle (i < j) is read (each bond once; the diagonal and the lower
 *     triangle are ignored).  Fields are length-N float64 vectors.
 *   - The partition order inside U1 is (H_x, H_y, H_z); H_a holds the a-a
 *     couplings and the a-fields.  The state is in the computational (Z) basis
 *     before and after every ts_step call.
 *   - Amplitudes: TS_C64 = interleaved float32 (re, im) pairs (8 bytes per
 *     amplitude); TS_C128 = interleaved float64 pairs (16 bytes).  2^N of them,
 *     in basis-index order.
 *
 * Threading and streams
 *   Every call is ordered on the CUDA stream given to ts_create (NULL = the
 *   legacy default stream).  ts_step and ts_set_basis_state only enqueue work;
 *   ts_observe, ts_get_state (to host) and ts_set_state (from host) wait for
 *   their own copies.  A context must not be used from two host threads at once.
 *
 * Errors
 *   Every entry point returns a ts_status; none aborts or throws.  The text of
 *   the last error of a context is available from ts_last_error.  A CUDA error
 *   raised by a kernel may surface at a later call (TS_ERR_CUDA).
 *
 * Memory ownership
 *   Inputs passed by pointer are copied; the caller keeps ownership.  Device
 *   buffers bound with ts_bind_buffers remain owned by the caller (for example
 *   torch tensors) and must outlive the context; any buffer not bound is
 *   allocated by the library with cudaMalloc on first use and freed by
 *   ts_destroy.
 */
#ifndef TS4_H
#define TS4_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TS4_API __attribute__((visibility("default")))
#else
#define TS4_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ts_ctx ts_ctx;

typedef enum {
    TS_OK = 0,
    TS_ERR_ARG = -1,     /* invalid argument (size, pointer, non-finite tau, ...) */
    TS_ERR_OOM = -2,     /* device memory exhausted or the state does not fit */
    TS_ERR_CUDA = -3,    /* a CUDA runtime call or kernel failed */
    TS_ERR_TIMEOUT = -4, /* a bounded device-side wait gave up (batched mode) */
    TS_ERR_STATE = -5    /* call out of order (e.g. echo without a saved reference) */
} ts_status;

typedef enum {
    TS_C64 = 0,  /* complex64 state, FP32 butterflies; angles formed in FP64 */
    TS_C128 = 1  /* complex128 state, FP64 throughout */
} ts_prec;

/* Observables for ts_observe (Sec. 4.2). */
enum {
    TS_NORM = 1,   /* sum_s |psi_s|^2                                    -> 1 double */
    TS_ENERGY = 2, /* <psi|H|psi> = <H_x> + <H_y> + <H_z>                -> 1 double */
    TS_SZ = 3,     /* <S^z_j> for j = 1..N                               -> N doubles */
    TS_ECHO = 4,   /* Loschmidt echo |<psi_0|psi>|^2 (Eq. 11, Sigma = 0)
                      against the reference saved by ts_save_reference   -> 1 double */
    TS_OVERLAP = 5, /* <psi_0|psi> as (re, im)                           -> 2 doubles */
    /* Two-spin correlations <S^a_i S^a_j> for all i, j (the paper measures local
     * polarisations and the echo, Sec. 4.2; these extend them to correlation
     * functions).  Row-major N x N, symmetric, diagonal = norm / 4.  The x and y
     * cases rotate a scratch copy of the state into the a eigenbasis (one
     * Walsh-Hadamard layer with diagonal phases, as for TS_ENERGY). */
    TS_SZSZ = 6,   /* <S^z_i S^z_j>                                      -> N*N doubles */
    TS_SXSX = 7,   /* <S^x_i S^x_j>                                      -> N*N doubles */
    TS_SYSY = 8,   /* <S^y_i S^y_j>                                      -> N*N doubles */
    TS_SX = 9,     /* <S^x_j> for j = 1..N                               -> N doubles */
    TS_SY = 10     /* <S^y_j> for j = 1..N                               -> N doubles */
};

/* Kernels for the rotation layers (ts_set_schedule). */
enum {
    TS_KERNEL_FUSED = 0, /* tiled pass kernel: one HBM round trip per bit group  */
    TS_KERNEL_BASIC = 1  /* one launch per spin and per phase (the paper's GPU-Basic) */
};

/*
 * Creates a context for N spins (1 <= N <= 34).
 *   Jx, Jy, Jz  N*N row-major couplings J^a_ij (upper triangle read), host memory.
 *   h           N z-fields h^z_i, host memory, or NULL for no field.
 *   prec        TS_C64 or TS_C128.
 *   cuda_stream cudaStream_t to order all work on, or NULL.
 * Uploads the couplings (FP64) and allocates small device tables.  The state
 * buffer itself is bound (ts_bind_buffers) or allocated on first use, so a
 * context can be created before deciding where the 2^N amplitudes live.
 * Errors: TS_ERR_ARG (N out of range, NULL out/J, non-finite entries),
 * TS_ERR_CUDA, TS_ERR_OOM.
 */
TS4_API ts_status ts_create(ts_ctx **out, int N, const double *Jx, const double *Jy, const double *Jz,
                    const double *h, ts_prec prec, void *cuda_stream);

/*
 * Adds transverse fields h^x_i, h^y_i (host, length N; either may be NULL for
 * zero).  They join H_x and H_y and are rotated with them (Eqs. 6-7).
 */
TS4_API ts_status ts_set_transverse_fields(ts_ctx *ctx, const double *hx, const double *hy);

/*
 * Binds caller-owned device buffers (each of 2^N amplitudes of the context's
 * precision, 256-byte aligned): psi holds the state; ref (may be NULL) holds
 * the echo reference; scratch (may be NULL) is used by TS_ENERGY.  Buffers
 * previously allocated by the library are freed.  Errors: TS_ERR_ARG for a
 * NULL psi, a size below 2^N amplitudes or a misaligned pointer.
 */
TS4_API ts_status ts_bind_buffers(ts_ctx *ctx, void *psi, void *ref, void *scratch, size_t bytes_each);

/* Copies 2^N amplitudes into the state (from host memory if on_device == 0). */
TS4_API ts_status ts_set_state(ts_ctx *ctx, const void *amps, int on_device);

/* Sets the state to the computational basis state |s> (Eq. 2 with one c_i = 1). */
TS4_API ts_status ts_set_basis_state(ts_ctx *ctx, uint64_t s);

/* Copies the current state into the echo reference psi_0 (Eq. 11). */
TS4_API ts_status ts_save_reference(ts_ctx *ctx);

/*
 * Advances the state by nsteps TS4 steps of length tau: psi <- U4(tau)^nsteps psi
 * (Sec. 2).  tau < 0 runs backwards (U4(-tau) = U4(tau)^{-1}, used for the
 * Loschmidt echo of Sec. 4.2).  Asynchronous.  Errors: TS_ERR_ARG (non-finite
 * tau, nsteps < 0), TS_ERR_OOM, TS_ERR_CUDA.
 */
TS4_API ts_status ts_step(ts_ctx *ctx, double tau, int64_t nsteps);

/*
 * Lower-order variants (Sec. 2): order 1 applies U1(tau), order 2 applies
 * U2(tau), order 4 is ts_step.  nsteps applications.
 */
TS4_API ts_status ts_step_order(ts_ctx *ctx, int order, double tau, int64_t nsteps);

/*
 * Chaining of consecutive ts_step calls (Sec. 2: the final P_z half of one U2 and the first of
 * the next merge into one slot).  With enable != 0, each ts_step / ts_step_order of order 2
 * or 4 on the fused kernel holds back its final pass (the last layer's rotation of one bit
 * group and the closing P_z slot); the next step call runs it inside its own first pass, so
 * a loop of one-step calls costs what one chained call costs (20 (g - 1) passes per TS4 step
 * instead of 20 (g - 1) + 1).  While a pass is held back, the state buffer does not yet hold
 * the evolved state: ts_get_state, ts_observe (all but TS_NORM, whose value accounts for
 * the held-back pass exactly: a Walsh-Hadamard gain and a slot scale), ts_save_reference,
 * ts_set_schedule, ts_set_transverse_fields, ts_autotune and ts_flush run it first;
 * ts_set_state, ts_set_basis_state and binding a new state buffer drop it.  Callers that
 * read a bound state buffer directly call ts_flush first.  enable = 0 (the default) runs
 * any held-back pass and turns chaining off.
 * Errors: TS_ERR_ARG (NULL context), TS_ERR_CUDA.
 */
TS4_API ts_status ts_set_chaining(ts_ctx *ctx, int enable);

/* Runs a held-back final pass (see ts_set_chaining), if any.  Errors: TS_ERR_ARG, TS_ERR_CUDA. */
TS4_API ts_status ts_flush(ts_ctx *ctx);

/*
 * Evaluates an observable (TS_NORM, TS_ENERGY, TS_SZ, TS_ECHO, TS_OVERLAP, ...)
 * into host memory `out` (sizes above).  Sums are accumulated in FP64; for
 * complex64 norms and <S^z> each thread first sums exact squares of the FP32
 * components in double-float (pairs of floats), whose error is of order
 * 1e-11 relative, then the threads' sums are added in FP64.
 * Synchronises the context's stream.  TS_ECHO/TS_OVERLAP without a saved
 * reference return TS_ERR_STATE.
 */
TS4_API ts_status ts_observe(ts_ctx *ctx, int what, double *out);

/* Copies the state out (to host memory if on_device == 0). */
TS4_API ts_status ts_get_state(ts_ctx *ctx, void *amps, int on_device);

/* Frees everything the library allocated.  NULL is accepted. */
TS4_API ts_status ts_destroy(ts_ctx *ctx);

/* Text of the last error or warning of ctx (never NULL; "" if none).  ctx may be NULL. */
TS4_API const char *ts_last_error(const ts_ctx *ctx);

/*
 * Selects the rotation kernel and its tile shape (Secs. 3.3-3.4; the paper
 * searched these by brute force per N, Sec. 3.4 last paragraph).
 *   kernel          TS_KERNEL_FUSED or TS_KERNEL_BASIC
 *   tile_bits       log2 of the amplitudes one thread block holds (0 = default)
 *   coalesce_bits   the s lowest spins every block keeps, so that each block
 *                   touches runs of 2^s consecutive amplitudes (0 = default: 3 for
 *                   complex64 and 2 for complex128, 64-byte runs, or 2 for complex64
 *                   when that needs one bit group fewer at this N)
 * Runs a pass held back by chaining first (ts_set_chaining).
 * Errors: TS_ERR_ARG for a shape this build does not provide.
 */
TS4_API ts_status ts_set_schedule(ts_ctx *ctx, int kernel, int tile_bits, int coalesce_bits);

/*
 * Reports the schedule in use: kernel, tile bits, coalescing bits, number of
 * bit groups g, and HBM passes per TS4 step when chained (20 (g - 1) for the
 * fused kernel).  Any pointer may be NULL.
 */
TS4_API ts_status ts_get_schedule(const ts_ctx *ctx, int *kernel, int *tile_bits, int *coalesce_bits,
                          int *groups, int *passes_per_step);

/*
 * The time-step bound of Eq. 4: returns
 *   [ max_{j,k} ( sum_a (h^a_j/2)^2 + sum_a (J^a_jk/4)^2 )^{1/2} ]^{-1}
 * for the context's Hamiltonian (infinity when H = 0); steps should satisfy
 * |tau| << this value.  ts_step and ts_step_order accept larger steps but record a
 * warning in ts_last_error (text starting "warning: ") when |tau| is at least
 * this bound; they still return TS_OK.
 */
TS4_API double ts_step_bound(const ts_ctx *ctx);

/*
 * The same bound from the couplings directly, on the host only (no device, no
 * context): Jx, Jy, Jz are N*N row-major (upper triangle read), hx, hy, hz length
 * N or NULL.  Returns -1 for N outside [1, 34] or a NULL coupling matrix.
 */
TS4_API double ts_step_bound_host(int N, const double *Jx, const double *Jy, const double *Jz, const double *hx,
                                  const double *hy, const double *hz);

/*
 * Global basis index of local amplitude e of thread block f for a tile made of
 * the global bits [0, c) and [w, w + h) (Secs. 3.3-3.4: the block index fixes
 * the other spins).  Local bits [0, h) are the window, local bits [h, h + c)
 * the c lowest spins.  Host-side copy of the mapping the kernels use; exported
 * so that it can be checked against the paper's block tables.
 */
TS4_API uint64_t ts_tile_global_index(int N, int c, int w, int h, uint64_t f, uint64_t e);

/*
 * The fused-pass plan, computed on the host without a GPU (Secs. 3.3-3.4: the bit
 * groups and the order in which one pass per group applies the rotation layers and
 * the diagonal slots of Sec. 2).  For nsteps chained steps of the given order
 * (1, 2 or 4) at N spins with the given tile and coalescing bits (0 = defaults) and
 * precision (which fixes the register bits of a tile):
 *   groups[i]  the bit groups: the tile holds global bits [0, c) and [w, w + h);
 *              group 0 is the TB lowest spins (c = 0);
 *   passes[p]  per kernel launch, in launch order: its group, the slot it applies
 *              (index into the slot list, -1 for none), and the global spins it
 *              rotates before and after the slot (rot_before holds every rotation of
 *              a pass without a slot); dup = 1 if some spin would be rotated twice on
 *              the same side of the slot (never, for a valid plan).
 * The slot list of an isolated run has layers + 1 entries (20 layers per TS4 step,
 * 4 per U2 step, 3 per U1 step).  chain (see ts_set_chaining): bit 1 = the call
 * continues a held-back pass of the previous call (its first pass then also rotates
 * its group before its slot 0, the merged P_z); bit 2 = the call holds back its final
 * pass (the plan omits it).  chain != 0 needs at least two bit groups.  Arrays are caller-owned; at most max_groups /
 * max_passes entries are written, the counts are always returned (call with NULL
 * arrays and 0 to size them).
 * Errors: TS_ERR_ARG (N outside [1, 34], N smaller than the tile, an unsupported
 * tile or coalescing width, order not 1, 2 or 4, nsteps < 1, chain outside [0, 3] or
 * chain with one group, NULL counts).
 */
typedef struct { int c, w, h; } ts_plan_group;
typedef struct {
    int group;
    int slot;
    uint64_t rot_before;
    uint64_t rot_after;
    int dup;
} ts_plan_pass;
TS4_API ts_status ts_plan(int N, ts_prec prec, int tile_bits, int coalesce_bits, int order, int64_t nsteps,
                          int chain, ts_plan_group *groups, int max_groups, int *ngroups, ts_plan_pass *passes,
                          int64_t max_passes, int64_t *npasses);

/*
 * The paper's phase-table mode (Sec. 3.1: the energies of every basis state are
 * precomputed once and each phase reads them), kept for an A/B comparison with
 * the bit-test slots.  enable != 0 builds three tables E_x, E_y, E_z of 2^N
 * entries each on the device: doubles for complex128 (24 bytes per basis state,
 * as in the paper; N = 28: 6 GiB), floats for complex64 (12 bytes per basis
 * state; N = 28: 3 GiB).  The basic kernel (TS_KERNEL_BASIC) then reads its slot
 * angles from them.  The fused kernel forms its angles from the bits and ignores
 * the tables.  enable = 0 frees them.  The tables follow later
 * ts_set_transverse_fields calls.
 * Errors: TS_ERR_OOM if the tables do not fit, TS_ERR_CUDA.
 */
TS4_API ts_status ts_set_phase_tables(ts_ctx *ctx, int enable);

/*
 * Autotuner (Sec. 3.4, last paragraph: the best rotation schedule depends on the
 * system size, so the paper searched it by brute force and stored the winners in
 * a file).  Times one TS4 step of length tau, reps times, on a scratch copy of the
 * current state for every tile size and coalescing width this build provides,
 * and selects the fastest for this context (ts_get_schedule reports it).  The
 * state itself is not changed.  cache_path (may be NULL): a text file of lines
 * "<gpu> <N> <prec> <tile_bits> <coalesce_bits> <ms_per_step>"; a matching
 * line is used instead of searching (best_ms is then -1), and a new result is
 * appended.  best_ms (may be NULL) receives the best time per step in ms.
 * Errors: TS_ERR_ARG, TS_ERR_STATE (no state), TS_ERR_OOM, TS_ERR_CUDA.
 */
TS4_API ts_status ts_autotune(ts_ctx *ctx, double tau, int reps, const char *cache_path, double *best_ms);

/*
 * Norm and <S^z_j> of a caller-owned device state, computed without allocating
 * any device memory.  The paper has no counterpart: this entry point serves
 * callers that cannot call cudaMalloc where they need these numbers -- hosts
 * whose device memory is owned by their own pool allocator, plug-ins that must
 * not grow the device footprint, loops that must not allocate once started.
 *   psi_dev  2^N amplitudes of precision prec, device memory (read only).  A
 *            state buffer bound to a context with chaining on (ts_set_chaining)
 *            lacks the held-back final pass: call ts_flush on that context first.
 *   out_dev  N + 1 doubles of device memory owned by the caller:
 *            out[0] = sum_s |psi_s|^2, out[1 + j] = sum_s |psi_s|^2 (bit_j(s) - 1/2)
 *            = <S^z_{j+1}>; sums accumulated as in ts_observe.
 *   cuda_stream  stream to enqueue on (NULL = legacy default stream); no host
 *            synchronisation.
 * Scratch: a static device array of 1024 x 35 doubles (about 280 KB), held by
 * every device that loads the library until exit.  Its device address is set up
 * on the first call made with a device current; make that first call before any
 * stream capture.  All calls share the array, so calls that overlap on the GPU
 * race.  Errors: TS_ERR_ARG (N outside [1, 34], a NULL pointer, an unknown
 * precision), TS_ERR_CUDA.
 */
TS4_API ts_status ts_reduce_sz_static(const void *psi_dev, int N, ts_prec prec, double *out_dev, void *cuda_stream);

/* ------------------------------------------------------------------ batched ensemble
 * Many independent states of several systems of uneven N advance together:
 * system k has N[k] spins, couplings Jx[k], Jy[k], Jz[k] (N[k]*N[k], upper
 * triangle), z-fields h[k] (or NULL) and nstates[k] states stored one after the
 * other (nstates[k] x 2^N[k] amplitudes).  This is the ensemble use of the
 * method for typical-state averages (App. A: random-phase states stand in for
 * the infinite-temperature density matrix).  Every system uses the same tile
 * size.  A whole ts_batch_step is one launch of a persistent kernel: its blocks
 * take the (pass, state, tile) work items in pass-major order from a counter, and
 * a tile waits until every tile of the previous pass of its state has finished
 * (per-state counters in device memory).  Every such wait is bounded in time
 * (ts_batch_set_wait; 2 s by default); when one runs out the launch ends early
 * and the next ts_batch_status, ts_batch_observe, ts_batch_get_states (to host)
 * or ts_batch_step returns TS_ERR_TIMEOUT.  The launch and the resets of its
 * counters are captured into one CUDA graph, replayed until tau or nsteps change.
 */
typedef struct ts_batch ts_batch;

/* Errors: TS_ERR_ARG (no systems, a NULL array, nstates < 1, a system smaller
 * than the smallest tile this build provides), TS_ERR_OOM, TS_ERR_CUDA. */
TS4_API ts_status ts_batch_create(ts_batch **out, int nsys, const int *N, const double *const *Jx,
                                  const double *const *Jy, const double *const *Jz, const double *const *h,
                                  const int *nstates, ts_prec prec, void *cuda_stream);

/* Binds caller-owned device memory (>= nstates x 2^N amplitudes, 256-byte aligned) for system sys. */
TS4_API ts_status ts_batch_bind_states(ts_batch *b, int sys, void *dev, size_t bytes);

/* Copies nstates x 2^N amplitudes of system sys in (host memory if on_device == 0). */
TS4_API ts_status ts_batch_set_states(ts_batch *b, int sys, const void *amps, int on_device);

/* Copies the states of system sys out (host memory if on_device == 0). */
TS4_API ts_status ts_batch_get_states(ts_batch *b, int sys, void *amps, int on_device);

/* Tile bits and coalescing bits for every system (0 = default; the default width is the one
 * that minimises the ensemble's amplitude-passes); the tile may not exceed the smallest N. */
TS4_API ts_status ts_batch_set_schedule(ts_batch *b, int tile_bits, int coalesce_bits);

/* The ensemble's tile bits and coalescing bits (either pointer may be NULL). */
TS4_API ts_status ts_batch_get_schedule(const ts_batch *b, int *tile_bits, int *coalesce_bits);

/*
 * Autotuner for the ensemble (Sec. 3.4's brute-force schedule search, applied to
 * the whole batch): times reps ts_batch_step(tau, 1) graph launches for every tile
 * size this build provides up to the smallest N and every coalescing width 1..4,
 * and keeps the fastest.  The trials run on the ensemble's own buffers after a
 * device copy of every state has been taken; the states are copied back at the
 * end, so they are unchanged.  cache_path (may be NULL): the same file format as
 * ts_autotune, with the N field set to -(a 31-bit FNV-1a hash of the (N, nstates)
 * list of the systems); a matching line is used instead of searching (best_ms is
 * then -1) and a new result is appended.  best_ms (may be NULL) receives the best
 * time per ensemble step in ms.
 * Errors: TS_ERR_ARG, TS_ERR_STATE (a system has no states), TS_ERR_OOM (no room
 * for the copy of the states), TS_ERR_CUDA.
 */
TS4_API ts_status ts_batch_autotune(ts_batch *b, double tau, int reps, const char *cache_path, double *best_ms);

/* nsteps TS4 steps of length tau for every state: one CUDA graph launch holding one
 * kernel launch (Sec. 2).  Asynchronous.  Errors: TS_ERR_ARG, TS_ERR_STATE (a system
 * has no states), TS_ERR_TIMEOUT (an earlier launch gave up; reported once), TS_ERR_CUDA. */
TS4_API ts_status ts_batch_step(ts_batch *b, double tau, int64_t nsteps);

/* Waits for the batch's queued work.  TS_ERR_TIMEOUT, reported once, if a dependency
 * wait of a launch ran out since the last report (the states are then undefined until
 * they are set again); TS_OK otherwise. */
TS4_API ts_status ts_batch_status(ts_batch *b);

/* Bounds every dependency wait of the ensemble kernel to limit_s seconds (0 < limit_s
 * <= 8; default 2; a wait also gives up after 2^22 polls).  hold != 0 makes every wait also wait for a device flag that
 * nothing sets, so that each one runs out: a test of the timeout path, which leaves
 * the device usable (the kernel returns; no fault, no endless wait).
 * Errors: TS_ERR_ARG. */
TS4_API ts_status ts_batch_set_wait(ts_batch *b, double limit_s, int hold);

/* TS_NORM (one double per state) or TS_SZ (N[k] doubles per state), systems in
 * order, states in order; synchronises the stream. */
TS4_API ts_status ts_batch_observe(ts_batch *b, int what, double *out);

/* Kernels launched so far (one per ts_batch_step; plus the reductions of ts_batch_observe). */
TS4_API int64_t ts_batch_kernel_launches(const ts_batch *b);

/* Text of the last error of b (never NULL). */
TS4_API const char *ts_batch_last_error(const ts_batch *b);

/* Frees everything the library allocated for the batch; NULL is accepted. */
TS4_API ts_status ts_batch_destroy(ts_batch *b);

/* Number of CUDA kernels this context has launched so far. */
TS4_API int64_t ts_kernel_launches(const ts_ctx *ctx);

/* Library version string. */
TS4_API const char *ts_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TS4_H */
