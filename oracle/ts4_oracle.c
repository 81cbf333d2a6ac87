/*
 * FP64 CPU oracle for the fourth-order Trotter-Suzuki (TS4) evolution of the
 * XYZ decomposition (Dente, Bederian, Zangara, Pastawski, "GPU accelerated
 * Trotter-Suzuki solver for quantum spin dynamics", Sec. 2).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA library is checked against.  Only the test suite, the smoke check and
 * the benchmark's CPU-baseline leg load it; the library never links it, and it
 * shares no source, header, table or helper with the CUDA path.
 *
 * It is deliberately plain and slow: every operator of Sec. 2 is applied in
 * the order the paper writes it, with no blocking, no fusion and no
 * reordering.
 *
 * Conventions (readings of the paper, listed with reasons in the design notes):
 *   - spin j (1-based) is bit j-1 of the basis index; bit 1 is spin up
 *     (S^z = +1/2), bit 0 is spin down (Sec. 3.2 and its footnote: spins are
 *     enumerated from right to left, n_up = n_down + 2^j);
 *   - S = sigma/2 (Eq. 9 gives the ZZ phases as +-J/4);
 *   - H = sum_{i<j} sum_a J^a_ij S^a_i S^a_j + sum_i sum_a h^a_i S^a_i (Eq. 1
 *     with each bond counted once and the diagonal j = k dropped);
 *   - the partition of Eq. 3 is (H1, H2, H3) = (H_x, H_y, H_z), where H_a holds
 *     the a-a couplings and the a-fields (Eqs. 7 and 10 rotate both together);
 *   - 2x2 matrices are written in the basis order (up, down), the order in
 *     which the identities under Eq. 5 hold.
 *
 * Functions follow the paper's steps:
 *   oracle_rotate_all   one global rotation X, X^dag, Y or Y^dag (Eq. 5), as
 *                       2^{N-1} independent pair updates per spin (Sec. 3.2)
 *   oracle_phase        the diagonal factor exp(-i t E(s)) of a Z-like part
 *                       (Eq. 9, and the z-field factor of Eq. 7)
 *   oracle_part         exp(-i t H_a): a Z-like phase conjugated by Y (a = x)
 *                       or X (a = y), Eqs. 7 and 10; H_z needs no rotation
 *   oracle_u1           U1(t) = e^{-itH_x} e^{-itH_y} e^{-itH_z}    (Eq. 3)
 *   oracle_u2           U2(t) = U1^dag(-t/2) U1(t/2)                 (Sec. 2)
 *   oracle_u4           U4(t) = U2(at)U2(at)U2((1-4a)t)U2(at)U2(at) (Sec. 2)
 * and the observables of Sec. 4.2 by their definitions (norm, <S^z_i>, <H>
 * by direct application of the Pauli operators, overlap for the echo Eq. 11,
 * two-spin correlations and transverse magnetisations).
 *
 * Amplitudes are C99 double complex, 2^N of them, in basis-index order.
 */
#include <complex.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

enum { ORACLE_XDAG = 0, ORACLE_X = 1, ORACLE_YDAG = 2, ORACLE_Y = 3 };

/*
 * Unnormalised rotation matrices, i.e. sqrt(2) times the global-rotation
 * factors of Eq. 5, in the basis order (up, down):
 *   R^x_{-pi/2} = [[1, i], [i, 1]] / sqrt2      R^y_{pi/2} = [[1, -1], [1, 1]] / sqrt2
 * Every entry is 0, +-1 or +-i, so applying them is exact up to the rounding
 * of one addition; the product of a rotation and its inverse is therefore 2
 * per spin, and each conjugation is followed by the exact scale 2^{-N}.
 */
static void rotation_matrix(int which, cplx m[2][2])
{
    switch (which) {
    case ORACLE_XDAG: /* (R^x_{-pi/2})^dagger */
        m[0][0] = 1; m[0][1] = -I; m[1][0] = -I; m[1][1] = 1; break;
    case ORACLE_X: /* R^x_{-pi/2} */
        m[0][0] = 1; m[0][1] = I; m[1][0] = I; m[1][1] = 1; break;
    case ORACLE_YDAG: /* (R^y_{pi/2})^dagger */
        m[0][0] = 1; m[0][1] = 1; m[1][0] = -1; m[1][1] = 1; break;
    default: /* ORACLE_Y: R^y_{pi/2} */
        m[0][0] = 1; m[0][1] = -1; m[1][0] = 1; m[1][1] = 1; break;
    }
}

/* Entries of the unnormalised matrix as (re, im) pairs, row-major, (up, down) order. */
void oracle_rotation_matrix(int which, double *out8)
{
    cplx m[2][2];
    rotation_matrix(which, m);
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 2; c++) {
            out8[4 * r + 2 * c] = creal(m[r][c]);
            out8[4 * r + 2 * c + 1] = cimag(m[r][c]);
        }
}

/*
 * Index of the p-th basis state whose bit b is 0 (spin down), p in [0, 2^{N-1}).
 * Its partner with the same spin up is this index + 2^b (Sec. 3.2).
 */
uint64_t oracle_pair_low(uint64_t p, int b)
{
    uint64_t low = p & ((UINT64_C(1) << b) - 1);
    return ((p >> b) << (b + 1)) | low;
}

/*
 * Applies the unnormalised 2x2 matrix of `which` to the single spin j
 * (bit b = j-1): for every pair (n_down, n_up = n_down + 2^b) the vector
 * (psi[n_up], psi[n_down]) is multiplied by the matrix (Sec. 3.2).
 */
void oracle_rotate_spin(cplx *psi, int N, int b, int which)
{
    cplx m[2][2];
    rotation_matrix(which, m);
    const int64_t npairs = (int64_t)1 << (N - 1);
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < npairs; p++) {
        uint64_t n_dn = oracle_pair_low((uint64_t)p, b);
        uint64_t n_up = n_dn | (UINT64_C(1) << b);
        cplx up = psi[n_up], dn = psi[n_dn];
        psi[n_up] = m[0][0] * up + m[0][1] * dn;
        psi[n_dn] = m[1][0] * up + m[1][1] * dn;
    }
}

/* The global rotation X = (x)_j R^x_j (or X^dag, Y, Y^dag), unnormalised: every spin in turn. */
void oracle_rotate_all(cplx *psi, int N, int which)
{
    for (int b = 0; b < N; b++)
        oracle_rotate_spin(psi, N, b, which);
}

void oracle_scale(cplx *psi, int N, double f)
{
    const int64_t dim = (int64_t)1 << N;
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < dim; s++)
        psi[s] *= f;
}

/*
 * Eigenvalue of the Z-like operator sum_{i<j} J_ij S^z_i S^z_j + sum_i h_i S^z_i
 * on the basis state s, with S^z = sigma/2 and sigma = +1 for bit 1 (Eq. 9).
 * J is N*N row-major and only its upper triangle (i < j) is read; h may be NULL.
 */
double oracle_zlike_energy(uint64_t s, int N, const double *J, const double *h)
{
    double e = 0.0;
    for (int i = 0; i < N; i++) {
        double si = ((s >> i) & 1) ? 1.0 : -1.0;
        for (int j = i + 1; j < N; j++) {
            double sj = ((s >> j) & 1) ? 1.0 : -1.0;
            e += J[i * N + j] * si * sj / 4.0;
        }
        if (h)
            e += h[i] * si / 2.0;
    }
    return e;
}

/* Diagonal factor exp(-i t E(s)) on every basis state (Eq. 9 with U = e^{-itH}). */
void oracle_phase(cplx *psi, int N, const double *J, const double *h, double t)
{
    const int64_t dim = (int64_t)1 << N;
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < dim; s++)
        psi[s] *= cexp(-I * t * oracle_zlike_energy((uint64_t)s, N, J, h));
}

/*
 * exp(-i t H_a) for a = 0 (x), 1 (y), 2 (z).
 *   H_z is diagonal: one phase.
 *   H_x = Y H~ Y^dag and H_y = X H~ X^dag, where H~ is the same sum with every
 *   S^a replaced by S^z (Eqs. 7 and 10), so exp(-itH_a) = R exp(-itH~) R^dag:
 *   rotate with R^dag, apply the phase, rotate back with R, then undo the two
 *   sqrt(2)^N factors of the unnormalised matrices with the exact 2^{-N}.
 */
void oracle_part(cplx *psi, int N, int a, const double *J, const double *h, double t)
{
    if (a == 2) {
        oracle_phase(psi, N, J, h, t);
        return;
    }
    int rdag = (a == 0) ? ORACLE_YDAG : ORACLE_XDAG;
    int r = (a == 0) ? ORACLE_Y : ORACLE_X;
    oracle_rotate_all(psi, N, rdag);
    oracle_phase(psi, N, J, h, t);
    oracle_rotate_all(psi, N, r);
    oracle_scale(psi, N, ldexp(1.0, -N));
}

/* The Hamiltonian: three N*N coupling matrices and three N-field vectors (any may be NULL for fields). */
typedef struct {
    int N;
    const double *J[3];
    const double *h[3];
} oracle_ham;

/* U1(t) = e^{-itH_x} e^{-itH_y} e^{-itH_z} (Eq. 3): the rightmost factor acts first. */
static void u1(cplx *psi, const oracle_ham *H, double t)
{
    oracle_part(psi, H->N, 2, H->J[2], H->h[2], t);
    oracle_part(psi, H->N, 1, H->J[1], H->h[1], t);
    oracle_part(psi, H->N, 0, H->J[0], H->h[0], t);
}

/* U1^dag(-t) = e^{-itH_z} e^{-itH_y} e^{-itH_x}: the same parts in reverse order. */
static void u1_dag_neg(cplx *psi, const oracle_ham *H, double t)
{
    oracle_part(psi, H->N, 0, H->J[0], H->h[0], t);
    oracle_part(psi, H->N, 1, H->J[1], H->h[1], t);
    oracle_part(psi, H->N, 2, H->J[2], H->h[2], t);
}

/* U2(t) = U1^dag(-t/2) U1(t/2) (Sec. 2): U1(t/2) acts first. */
static void u2(cplx *psi, const oracle_ham *H, double t)
{
    u1(psi, H, t / 2.0);
    u1_dag_neg(psi, H, t / 2.0);
}

/* The Suzuki coefficient a = 1/(4 - 4^{1/3}) of U4 (Sec. 2). */
double oracle_suzuki_a(void)
{
    return 1.0 / (4.0 - cbrt(4.0));
}

/* U4(t) = U2(at) U2(at) U2((1-4a)t) U2(at) U2(at) (Sec. 2). */
static void u4(cplx *psi, const oracle_ham *H, double t)
{
    const double a = oracle_suzuki_a();
    u2(psi, H, a * t);
    u2(psi, H, a * t);
    u2(psi, H, (1.0 - 4.0 * a) * t);
    u2(psi, H, a * t);
    u2(psi, H, a * t);
}

static oracle_ham make_ham(int N, const double *Jx, const double *Jy, const double *Jz,
                           const double *hx, const double *hy, const double *hz)
{
    oracle_ham H;
    H.N = N;
    H.J[0] = Jx; H.J[1] = Jy; H.J[2] = Jz;
    H.h[0] = hx; H.h[1] = hy; H.h[2] = hz;
    return H;
}

/* One application of U1(t), U2(t) or U4(t) (order = 1, 2 or 4). */
void oracle_apply(cplx *psi, int N, const double *Jx, const double *Jy, const double *Jz,
                  const double *hx, const double *hy, const double *hz, int order, double t)
{
    oracle_ham H = make_ham(N, Jx, Jy, Jz, hx, hy, hz);
    if (order == 1)
        u1(psi, &H, t);
    else if (order == 2)
        u2(psi, &H, t);
    else
        u4(psi, &H, t);
}

/* nsteps TS4 steps of length tau: psi <- U4(tau)^nsteps psi. */
void oracle_ts4(cplx *psi, int N, const double *Jx, const double *Jy, const double *Jz,
                const double *hx, const double *hy, const double *hz, double tau, int64_t nsteps)
{
    oracle_ham H = make_ham(N, Jx, Jy, Jz, hx, hy, hz);
    for (int64_t k = 0; k < nsteps; k++)
        u4(psi, &H, tau);
}

/* ---------------- observables, by definition ---------------- */

double oracle_norm(const cplx *psi, int N)
{
    const int64_t dim = (int64_t)1 << N;
    double acc = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : acc)
    for (int64_t s = 0; s < dim; s++)
        acc += creal(psi[s]) * creal(psi[s]) + cimag(psi[s]) * cimag(psi[s]);
    return acc;
}

/* <S^z_j> for every spin: sum_s |psi_s|^2 (bit_j(s) - 1/2). */
void oracle_sz(const cplx *psi, int N, double *out)
{
    const int64_t dim = (int64_t)1 << N;
    for (int j = 0; j < N; j++) {
        double acc = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : acc)
        for (int64_t s = 0; s < dim; s++) {
            double p = creal(psi[s]) * creal(psi[s]) + cimag(psi[s]) * cimag(psi[s]);
            acc += p * ((((uint64_t)s >> j) & 1) ? 0.5 : -0.5);
        }
        out[j] = acc;
    }
}

/* <a|b> = sum_s conj(a_s) b_s, returned as (re, im). */
void oracle_overlap(const cplx *a, const cplx *b, int N, double *out2)
{
    const int64_t dim = (int64_t)1 << N;
    double re = 0.0, im = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : re, im)
    for (int64_t s = 0; s < dim; s++) {
        cplx z = conj(a[s]) * b[s];
        re += creal(z);
        im += cimag(z);
    }
    out2[0] = re;
    out2[1] = im;
}

/*
 * out = H psi by direct action of the spin operators on basis states (Eq. 1),
 * with S = sigma/2 and, on (up, down):
 *   sigma^x flips the spin;  sigma^y|up> = i|down>, sigma^y|down> = -i|up>;
 *   sigma^z|up> = |up>, sigma^z|down> = -|down>.
 * Written as a gather: (H psi)[s] = sum over terms of <s|term|s'> psi[s'].
 */
void oracle_apply_hamiltonian(const cplx *psi, cplx *out, int N, const double *Jx, const double *Jy,
                              const double *Jz, const double *hx, const double *hy, const double *hz)
{
    const int64_t dim = (int64_t)1 << N;
#pragma omp parallel for schedule(static)
    for (int64_t si = 0; si < dim; si++) {
        uint64_t s = (uint64_t)si;
        cplx acc = 0.0;
        for (int i = 0; i < N; i++) {
            uint64_t mi = UINT64_C(1) << i;
            int bi = (int)((s >> i) & 1);
            double sgi = bi ? 1.0 : -1.0;
            for (int j = i + 1; j < N; j++) {
                uint64_t mj = UINT64_C(1) << j;
                int bj = (int)((s >> j) & 1);
                double sgj = bj ? 1.0 : -1.0;
                cplx flipped = psi[s ^ mi ^ mj];
                /* sigma^x sigma^x: both spins flipped, amplitude 1 */
                acc += Jx[i * N + j] / 4.0 * flipped;
                /* sigma^y sigma^y: <s|sy sy|s'> = (-1) if the two spins of s are equal, else +1 */
                acc += Jy[i * N + j] / 4.0 * ((bi == bj) ? -1.0 : 1.0) * flipped;
                /* sigma^z sigma^z: diagonal */
                acc += Jz[i * N + j] / 4.0 * sgi * sgj * psi[s];
            }
            if (hx)
                acc += hx[i] / 2.0 * psi[s ^ mi];
            if (hy) /* <s|sigma^y|s^mi>: s down -> from up: i ; s up -> from down: -i */
                acc += hy[i] / 2.0 * (bi ? -I : I) * psi[s ^ mi];
            if (hz)
                acc += hz[i] / 2.0 * sgi * psi[s];
        }
        out[s] = acc;
    }
}

/* <psi|H|psi> (real part; H is Hermitian). */
double oracle_energy(const cplx *psi, int N, const double *Jx, const double *Jy, const double *Jz,
                     const double *hx, const double *hy, const double *hz)
{
    const int64_t dim = (int64_t)1 << N;
    cplx *hpsi = (cplx *)malloc(sizeof(cplx) * (size_t)dim);
    if (!hpsi)
        return NAN;
    oracle_apply_hamiltonian(psi, hpsi, N, Jx, Jy, Jz, hx, hy, hz);
    double ov[2];
    oracle_overlap(psi, hpsi, N, ov);
    free(hpsi);
    return ov[0];
}

/*
 * Two-spin correlations and one-spin expectations of psi by direct action of the spin
 * operators on basis states (the conventions of oracle_apply_hamiltonian):
 *   czz, cxx, cyy  N x N row-major, <S^a_i S^a_j> for i != j; the diagonal is
 *                  <(S^a_i)^2> = <psi|psi>/4;
 *   mx, my         <S^x_j> and <S^y_j>, j = 1..N.
 * These extend the local polarisations and the echo of Sec. 4.2 to correlation functions.
 */
void oracle_correlations(const cplx *psi, int N, double *czz, double *cxx, double *cyy, double *mx, double *my)
{
    const int64_t dim = (int64_t)1 << N;
    const double nrm = oracle_norm(psi, N);
    for (int i = 0; i < N; i++) {
        const uint64_t mi = UINT64_C(1) << i;
        double ax = 0.0, ay = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : ax, ay)
        for (int64_t si = 0; si < dim; si++) {
            uint64_t s = (uint64_t)si;
            int bi = (int)((s >> i) & 1);
            cplx f = conj(psi[s]) * psi[s ^ mi];
            /* <s|sigma^x|s^mi> = 1;  <s|sigma^y|s^mi> = -i if spin i of s is up, +i if down */
            ax += creal(f);
            ay += creal((bi ? -I : I) * f);
        }
        mx[i] = 0.5 * ax;
        my[i] = 0.5 * ay;
        czz[i * N + i] = cxx[i * N + i] = cyy[i * N + i] = 0.25 * nrm;
        for (int j = i + 1; j < N; j++) {
            const uint64_t mj = UINT64_C(1) << j;
            double zz = 0.0, xx = 0.0, yy = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : zz, xx, yy)
            for (int64_t si = 0; si < dim; si++) {
                uint64_t s = (uint64_t)si;
                int bi = (int)((s >> i) & 1), bj = (int)((s >> j) & 1);
                double w = creal(psi[s]) * creal(psi[s]) + cimag(psi[s]) * cimag(psi[s]);
                zz += w * (bi ? 0.5 : -0.5) * (bj ? 0.5 : -0.5);
                cplx f = conj(psi[s]) * psi[s ^ mi ^ mj];
                xx += 0.25 * creal(f);
                /* sigma^y sigma^y: -1 if the two spins of s are equal, +1 otherwise */
                yy += 0.25 * ((bi == bj) ? -1.0 : 1.0) * creal(f);
            }
            czz[i * N + j] = czz[j * N + i] = zz;
            cxx[i * N + j] = cxx[j * N + i] = xx;
            cyy[i * N + j] = cyy[j * N + i] = yy;
        }
    }
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the following parallel loops (n >= 1); used to time the oracle on one core. */
void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1)
        omp_set_num_threads(n);
#else
    (void)n;
#endif
}
