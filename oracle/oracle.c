/*
 * Plain FP64 CPU oracle for state-vector simulation (test infrastructure).
 *
 * This file is TEST INFRASTRUCTURE. Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it. It shares no code,
 * header, table or helper with the GPU library and includes none of them.
 *
 * Everything here is written for obviousness, not speed: one thread, double
 * complex arithmetic, loops over the whole 2^n vector, Neumaier-compensated
 * sums. Qubit q is bit q of the amplitude index (little-endian), so the
 * amplitude of basis string b_{n-1}...b_0 sits at index sum_q b_q 2^q.
 *
 * Paper sections followed (arXiv 2304.14969):
 *  - Sec. II (exact simulation): the ket |psi_C> = C|psi_0> is computed by
 *    applying the gates of C one at a time in the Schroedinger picture.
 *  - Sec. II.E, Eq. (qft)/(dft): the QFT maps amplitudes x_k to
 *    y_j = N^{-1/2} sum_k x_k w^{jk}, w = exp(2 pi i / N); orc_dft_sample
 *    evaluates that definition for one output index.
 *  - Sec. III.A, Eq. (schmidt)/(sdrp) and the four steps after it: the SDRP
 *    check computes the Bloch vector r = (<X_q>, <Y_q>, <Z_q>), the rounding
 *    error eps = (1 - |r|)/2, and when eps <= p/2 rotates r onto the |0> pole,
 *    post-selects |0>, and rotates back.
 *  - Sec. III.B, Eq. (fid_model): F = prod_j (1 - eps_j).
 *  - Sec. III.B, Eq. (fid_exact): F_exact = |<psi_approx|psi_exact>|^2.
 *  - Sec. III.C: the U(theta, phi, lambda) single-qubit gate.
 *
 * All-core build: the same file compiled with -fopenmp (liboracle_mt.so)
 * splits the iterations of the index loops across the host's threads; the
 * only differences are the "omp" pragmas below. Element-wise loops give
 * bit-identical results; each thread keeps its own compensated partial sums,
 * merged (compensated) at the end, so sums agree with the one-thread build
 * to within the compensated sums' error. The one-thread build is the
 * oracle the pins check; the all-core build is checked against it.
 *
 * Pins: every function here is checked by the CPU tests against closed
 * forms, library routines (numpy FFT, numpy kron-built matrices), brute
 * force on tiny inputs and identities; see tests/test_oracle_*.py.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* Gate kinds understood by the oracle (its own numbering). */
enum {
    OG_H = 1, OG_X = 2, OG_Y = 3, OG_Z = 4, OG_S = 5, OG_T = 6,
    OG_SQRTX = 7, OG_SQRTY = 8, OG_SQRTW = 9, OG_U3 = 10, OG_PHASE = 11,
    OG_RZ = 12, OG_MAT1 = 13,
    OG_CP = 32, OG_SWAP = 33, OG_FSIM = 34, OG_MAT2 = 35
};

#define ORC_MAXCTRL 6

/* One gate. q[0] is the target of a one-qubit gate; for a two-qubit gate
 * q[0] is bit 0 and q[1] bit 1 of the 4x4 matrix's row/column index.
 * Controls apply to one-qubit kinds: the gate acts only on the part of the
 * state where bit ctrl[j] equals cval[j] for every j. mat holds an explicit
 * matrix (row-major, re/im interleaved) for OG_MAT1/OG_MAT2. */
typedef struct {
    int32_t kind;
    int32_t q[2];
    int32_t nctrl;
    int32_t ctrl[ORC_MAXCTRL];
    int32_t cval[ORC_MAXCTRL];
    double prm[4];
    double mat[32];
} orc_gate;

/* One SDRP decision of orc_sdrp_run. */
typedef struct {
    int32_t gate;     /* index of the two-qubit gate after which it ran */
    int32_t qubit;    /* global qubit id checked */
    int32_t action;   /* 0 keep, 1 rounded (eps <= p/2), 2 exact separation */
    int32_t pad;
    double eps;
    double r[3];
} orc_decision;

/* ---------------------------------------------------------------- sums */

/* Neumaier-compensated running sum. */
typedef struct { double s, c; } nsum;

static void nsum_add(nsum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}

static double nsum_get(const nsum *a) { return a->s + a->c; }

#ifdef _OPENMP
#include <omp.h>
/* Merges a thread's partial sum into another (all-core build only). */
static void nsum_merge(nsum *out, const nsum *in)
{
    nsum_add(out, in->s);
    nsum_add(out, in->c);
}
#pragma omp declare reduction(nplus : nsum : nsum_merge(&omp_out, &omp_in)) initializer(omp_priv = (nsum){ 0, 0 })
#endif

/* Threads the index loops use: 1 in the one-thread build. */
int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------- gate matrices */

/* Writes the gate's matrix (2x2 for one-qubit kinds, 4x4 for two-qubit
 * kinds) into m, row-major. Returns the matrix dimension, 0 if unknown. */
int orc_gate_matrix(const orc_gate *g, cplx *m)
{
    const double r2 = 1.0 / sqrt(2.0);
    double th, ph, la;
    switch (g->kind) {
    case OG_H:
        m[0] = r2; m[1] = r2; m[2] = r2; m[3] = -r2;
        return 2;
    case OG_X:
        m[0] = 0; m[1] = 1; m[2] = 1; m[3] = 0;
        return 2;
    case OG_Y:
        m[0] = 0; m[1] = -I; m[2] = I; m[3] = 0;
        return 2;
    case OG_Z:
        m[0] = 1; m[1] = 0; m[2] = 0; m[3] = -1;
        return 2;
    case OG_S:
        m[0] = 1; m[1] = 0; m[2] = 0; m[3] = I;
        return 2;
    case OG_T:
        m[0] = 1; m[1] = 0; m[2] = 0; m[3] = cexp(I * M_PI / 4.0);
        return 2;
    case OG_SQRTX:
    case OG_SQRTY:
    case OG_SQRTW: {
        /* sqrt(P) = ((1+i) I + (1-i) P) / 2 for a Pauli-like P with P^2 = I. */
        cplx P[4];
        if (g->kind == OG_SQRTX) { P[0] = 0; P[1] = 1; P[2] = 1; P[3] = 0; }
        else if (g->kind == OG_SQRTY) { P[0] = 0; P[1] = -I; P[2] = I; P[3] = 0; }
        else { /* W = (X + Y)/sqrt(2) */
            P[0] = 0; P[1] = (1.0 - I) * r2; P[2] = (1.0 + I) * r2; P[3] = 0;
        }
        for (int k = 0; k < 4; k++) {
            cplx id = (k == 0 || k == 3) ? 1.0 : 0.0;
            m[k] = ((1.0 + I) * id + (1.0 - I) * P[k]) / 2.0;
        }
        return 2;
    }
    case OG_U3:
        /* Sec. III.C: U(theta, phi, lambda). */
        th = g->prm[0]; ph = g->prm[1]; la = g->prm[2];
        m[0] = cos(th / 2.0);
        m[1] = -cexp(I * la) * sin(th / 2.0);
        m[2] = cexp(I * ph) * sin(th / 2.0);
        m[3] = cexp(I * (ph + la)) * cos(th / 2.0);
        return 2;
    case OG_PHASE:
        m[0] = 1; m[1] = 0; m[2] = 0; m[3] = cexp(I * g->prm[0]);
        return 2;
    case OG_RZ:
        m[0] = cexp(-I * g->prm[0] / 2.0); m[1] = 0; m[2] = 0;
        m[3] = cexp(I * g->prm[0] / 2.0);
        return 2;
    case OG_MAT1:
        for (int k = 0; k < 4; k++) m[k] = g->mat[2 * k] + I * g->mat[2 * k + 1];
        return 2;
    case OG_CP:
        for (int k = 0; k < 16; k++) m[k] = 0;
        m[0] = 1; m[5] = 1; m[10] = 1; m[15] = cexp(I * g->prm[0]);
        return 4;
    case OG_SWAP:
        for (int k = 0; k < 16; k++) m[k] = 0;
        m[0 * 4 + 0] = 1; m[1 * 4 + 2] = 1; m[2 * 4 + 1] = 1; m[3 * 4 + 3] = 1;
        return 4;
    case OG_FSIM:
        /* fSim(theta, phi) on the basis |00>,|01>,|10>,|11>. */
        th = g->prm[0]; ph = g->prm[1];
        for (int k = 0; k < 16; k++) m[k] = 0;
        m[0] = 1;
        m[1 * 4 + 1] = cos(th); m[1 * 4 + 2] = -I * sin(th);
        m[2 * 4 + 1] = -I * sin(th); m[2 * 4 + 2] = cos(th);
        m[3 * 4 + 3] = cexp(-I * ph);
        return 4;
    case OG_MAT2:
        for (int k = 0; k < 16; k++) m[k] = g->mat[2 * k] + I * g->mat[2 * k + 1];
        return 4;
    default:
        return 0;
    }
}

static int controls_hold(const orc_gate *g, uint64_t i)
{
    for (int j = 0; j < g->nctrl; j++)
        if ((int)((i >> g->ctrl[j]) & 1u) != g->cval[j]) return 0;
    return 1;
}

/* ------------------------------------------------------- gate apply */

/* psi <- U psi on target t, restricted to indices where the controls hold. */
void orc_apply_1q(cplx *psi, int n, const cplx *u, int t, const orc_gate *ctl)
{
    uint64_t N = (uint64_t)1 << n, bt = (uint64_t)1 << t;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (uint64_t i = 0; i < N; i++) {
        if (i & bt) continue;
        if (ctl && !controls_hold(ctl, i)) continue;
        cplx a = psi[i], b = psi[i | bt];
        psi[i] = u[0] * a + u[1] * b;
        psi[i | bt] = u[2] * a + u[3] * b;
    }
}

/* psi <- U psi with U 4x4 on (q0 = local bit 0, q1 = local bit 1). */
void orc_apply_2q(cplx *psi, int n, const cplx *u, int q0, int q1)
{
    uint64_t N = (uint64_t)1 << n, b0 = (uint64_t)1 << q0, b1 = (uint64_t)1 << q1;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (uint64_t i = 0; i < N; i++) {
        if ((i & b0) || (i & b1)) continue;
        uint64_t idx[4] = { i, i | b0, i | b1, i | b0 | b1 };
        cplx v[4], w[4];
        for (int r = 0; r < 4; r++) v[r] = psi[idx[r]];
        for (int r = 0; r < 4; r++) {
            w[r] = 0;
            for (int c = 0; c < 4; c++) w[r] += u[r * 4 + c] * v[c];
        }
        for (int r = 0; r < 4; r++) psi[idx[r]] = w[r];
    }
}

/* psi <- U psi with U of size 2^k x 2^k on qubits[0..k-1] (k <= 8); qubits[b]
 * is bit b of U's row/column index. Gather, multiply, scatter. */
void orc_apply_kq(cplx *psi, int n, int k, const int *qubits, const cplx *u)
{
    if (k < 1 || k > 8) return;
    uint64_t N = (uint64_t)1 << n, D = (uint64_t)1 << k, mask = 0;
    for (int b = 0; b < k; b++) mask |= (uint64_t)1 << qubits[b];
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (uint64_t i = 0; i < N; i++) {
        if (i & mask) continue;
        uint64_t idx[256];
        cplx v[256], w[256];
        for (uint64_t l = 0; l < D; l++) {
            uint64_t j = i;
            for (int b = 0; b < k; b++)
                if ((l >> b) & 1u) j |= (uint64_t)1 << qubits[b];
            idx[l] = j;
            v[l] = psi[j];
        }
        for (uint64_t r = 0; r < D; r++) {
            w[r] = 0;
            for (uint64_t c = 0; c < D; c++) w[r] += u[r * D + c] * v[c];
        }
        for (uint64_t l = 0; l < D; l++) psi[idx[l]] = w[l];
    }
}

/* Applies one gate record. Returns 0 on success, -1 on an unknown kind. */
int orc_apply_gate(cplx *psi, int n, const orc_gate *g)
{
    cplx m[16];
    int d = orc_gate_matrix(g, m);
    if (d == 2) orc_apply_1q(psi, n, m, g->q[0], g->nctrl ? g : NULL);
    else if (d == 4) orc_apply_2q(psi, n, m, g->q[0], g->q[1]);
    else return -1;
    return 0;
}

int orc_apply_circuit(cplx *psi, int n, const orc_gate *g, int ng)
{
    for (int k = 0; k < ng; k++)
        if (orc_apply_gate(psi, n, &g[k])) return -1;
    return 0;
}

/* ------------------------------------------------- dense check (n <= 8) */

/* Full 2^n x 2^n matrix of one gate, built element by element: entry
 * (row, col) is nonzero only when row and col agree on every qubit the
 * gate does not act on. Independent of the index-pair loops above. */
int orc_dense_gate(int n, const orc_gate *g, cplx *G)
{
    cplx m[16];
    int d = orc_gate_matrix(g, m);
    if (d == 0 || n > 10) return -1;
    uint64_t N = (uint64_t)1 << n;
    uint64_t act = (uint64_t)1 << g->q[0];
    if (d == 4) act |= (uint64_t)1 << g->q[1];
    for (uint64_t r = 0; r < N; r++) {
        for (uint64_t c = 0; c < N; c++) {
            cplx e = 0;
            if ((r & ~act) == (c & ~act)) {
                int lr, lc;
                if (d == 2) {
                    lr = (int)((r >> g->q[0]) & 1u);
                    lc = (int)((c >> g->q[0]) & 1u);
                } else {
                    lr = (int)(((r >> g->q[0]) & 1u) | (((r >> g->q[1]) & 1u) << 1));
                    lc = (int)(((c >> g->q[0]) & 1u) | (((c >> g->q[1]) & 1u) << 1));
                }
                if (g->nctrl && !controls_hold(g, r)) e = (lr == lc) ? 1.0 : 0.0;
                else e = m[lr * d + lc];
            }
            G[r * N + c] = e;
        }
    }
    return 0;
}

/* Product of the dense gate matrices, last gate leftmost. */
int orc_dense_circuit(int n, const orc_gate *g, int ng, cplx *M)
{
    if (n > 10) return -1;
    uint64_t N = (uint64_t)1 << n;
    cplx *G = malloc(N * N * sizeof(cplx)), *T = malloc(N * N * sizeof(cplx));
    for (uint64_t r = 0; r < N; r++)
        for (uint64_t c = 0; c < N; c++) M[r * N + c] = (r == c) ? 1.0 : 0.0;
    for (int k = 0; k < ng; k++) {
        if (orc_dense_gate(n, &g[k], G)) { free(G); free(T); return -1; }
        for (uint64_t r = 0; r < N; r++)
            for (uint64_t c = 0; c < N; c++) {
                cplx s = 0;
                for (uint64_t x = 0; x < N; x++) s += G[r * N + x] * M[x * N + c];
                T[r * N + c] = s;
            }
        memcpy(M, T, N * N * sizeof(cplx));
    }
    free(G); free(T);
    return 0;
}

/* ---------------------------------------------------------- reductions */

double orc_norm2(const cplx *psi, int n)
{
    uint64_t N = (uint64_t)1 << n;
    nsum s = { 0, 0 };
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(nplus : s)
#endif
    for (uint64_t i = 0; i < N; i++) nsum_add(&s, creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]));
    return nsum_get(&s);
}

void orc_probs(const cplx *psi, int n, double *p)
{
    uint64_t N = (uint64_t)1 << n;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (uint64_t i = 0; i < N; i++) p[i] = creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
}

/* Probability that qubit q reads 1 (unnormalised state: divided by norm). */
double orc_prob1(const cplx *psi, int n, int q)
{
    uint64_t N = (uint64_t)1 << n;
    nsum one = { 0, 0 }, all = { 0, 0 };
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(nplus : one, all)
#endif
    for (uint64_t i = 0; i < N; i++) {
        double a = creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
        nsum_add(&all, a);
        if ((i >> q) & 1u) nsum_add(&one, a);
    }
    return nsum_get(&one) / nsum_get(&all);
}

/* <a|b> = sum_i conj(a_i) b_i. */
void orc_inner(const cplx *a, const cplx *b, int n, double out[2])
{
    uint64_t N = (uint64_t)1 << n;
    nsum re = { 0, 0 }, im = { 0, 0 };
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(nplus : re, im)
#endif
    for (uint64_t i = 0; i < N; i++) {
        cplx z = conj(a[i]) * b[i];
        nsum_add(&re, creal(z));
        nsum_add(&im, cimag(z));
    }
    out[0] = nsum_get(&re);
    out[1] = nsum_get(&im);
}

/* Sec. III.A step 1: Bloch vector of qubit q, r = (<X>, <Y>, <Z>) of the
 * reduced state rho_q = Tr_{not q} |psi><psi| / <psi|psi>. With a_i the
 * amplitudes where bit q = 0 and b_i their partners with bit q = 1:
 * rho_q[1][0] = sum_i b_i conj(a_i), <X> = 2 Re rho_q[1][0],
 * <Y> = 2 Im rho_q[1][0], <Z> = rho_q[0][0] - rho_q[1][1]. */
void orc_bloch(const cplx *psi, int n, int q, double r[3])
{
    uint64_t N = (uint64_t)1 << n, bq = (uint64_t)1 << q;
    nsum r00 = { 0, 0 }, r11 = { 0, 0 }, sre = { 0, 0 }, sim = { 0, 0 };
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(nplus : r00, r11, sre, sim)
#endif
    for (uint64_t i = 0; i < N; i++) {
        if (i & bq) continue;
        cplx a = psi[i], b = psi[i | bq];
        cplx s = b * conj(a);
        nsum_add(&r00, creal(a) * creal(a) + cimag(a) * cimag(a));
        nsum_add(&r11, creal(b) * creal(b) + cimag(b) * cimag(b));
        nsum_add(&sre, creal(s));
        nsum_add(&sim, cimag(s));
    }
    double tr = nsum_get(&r00) + nsum_get(&r11);
    r[0] = 2.0 * nsum_get(&sre) / tr;
    r[1] = 2.0 * nsum_get(&sim) / tr;
    r[2] = (nsum_get(&r00) - nsum_get(&r11)) / tr;
}

/* ------------------------------------------------------ DFT definition */

/* Eq. (dft): y_j = N^{-1/2} sum_k x_k exp(2 pi i j k / N), evaluated for
 * one output index j straight from the definition. j k mod N is taken in
 * exact integer arithmetic before the angle is formed. */
void orc_dft_sample(const cplx *x, int n, uint64_t j, double out[2])
{
    uint64_t N = (uint64_t)1 << n;
    nsum re = { 0, 0 }, im = { 0, 0 };
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(nplus : re, im)
#endif
    for (uint64_t k = 0; k < N; k++) {
        uint64_t m = (j * k) & (N - 1);
        double ang = 2.0 * M_PI * (double)m / (double)N;
        cplx z = x[k] * cexp(I * ang);
        nsum_add(&re, creal(z));
        nsum_add(&im, cimag(z));
    }
    out[0] = nsum_get(&re) / sqrt((double)N);
    out[1] = nsum_get(&im) / sqrt((double)N);
}

/* --------------------------------------------------------------- SDRP */

/* Sec. III.A steps 2-4 for qubit q: rotate the Bloch vector r onto the |0>
 * pole with a local unitary V, post-select |0> on q and renormalise by the
 * computed norm, then rotate back with V^dagger. The net effect is the
 * projection of Eq. (sdrp) onto |phi>_q, the dominant Schmidt branch.
 * |phi> = (cos(th/2), e^{i ph} sin(th/2)) with th = acos(r_z/|r|),
 * ph = atan2(r_y, r_x); for |r| below 1e-15 the +z direction is used. */
void orc_sdrp_project(cplx *psi, int n, int q, const double r[3])
{
    double len = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    double th = 0.0, ph = 0.0;
    if (len >= 1e-15) {
        double c = r[2] / len;
        if (c > 1.0) c = 1.0;
        if (c < -1.0) c = -1.0;
        th = acos(c);
        ph = atan2(r[1], r[0]);
    }
    cplx f0 = cos(th / 2.0), f1 = cexp(I * ph) * sin(th / 2.0);
    /* V has rows <phi| and <phi_perp|, so V|phi> = |0>. */
    cplx V[4] = { conj(f0), conj(f1), -f1, f0 };
    cplx Vd[4] = { conj(V[0]), conj(V[2]), conj(V[1]), conj(V[3]) };
    uint64_t N = (uint64_t)1 << n, bq = (uint64_t)1 << q;
    orc_apply_1q(psi, n, V, q, NULL);                 /* step 2: rotate */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (uint64_t i = 0; i < N; i++)                  /* step 3: post-select |0> */
        if (i & bq) psi[i] = 0;
    double s = sqrt(orc_norm2(psi, n));
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (uint64_t i = 0; i < N; i++) psi[i] /= s;
    orc_apply_1q(psi, n, Vd, q, NULL);                /* step 4: rotate back */
}

/* ------------------------------------------- two-qubit subsystems (SDRP) */

/* Reduced density matrix of the pair (qa, qb) of psi, normalised:
 * rho[x * 4 + y] = sum over the other qubits of psi[.. x ..] conj(psi[.. y ..])
 * / <psi|psi>, where x = bit qa + 2 bit qb of the index. */
void orc_rho2(const cplx *psi, int n, int qa, int qb, cplx rho[16])
{
    uint64_t N = (uint64_t)1 << n, ba = (uint64_t)1 << qa, bb = (uint64_t)1 << qb;
    nsum re[16], im[16];
    for (int k = 0; k < 16; k++) { re[k].s = re[k].c = 0; im[k].s = im[k].c = 0; }
    for (uint64_t i = 0; i < N; i++) {
        if ((i & ba) || (i & bb)) continue;
        uint64_t idx[4] = { i, i | ba, i | bb, i | ba | bb };
        for (int x = 0; x < 4; x++)
            for (int y = 0; y < 4; y++) {
                cplx z = psi[idx[x]] * conj(psi[idx[y]]);
                nsum_add(&re[x * 4 + y], creal(z));
                nsum_add(&im[x * 4 + y], cimag(z));
            }
    }
    double tr = nsum_get(&re[0]) + nsum_get(&re[5]) + nsum_get(&re[10]) + nsum_get(&re[15]);
    for (int k = 0; k < 16; k++) rho[k] = (nsum_get(&re[k]) + I * nsum_get(&im[k])) / tr;
}

/* Eigenvalues (ascending in w[0..3]) and unit eigenvectors (columns of
 * vec, vec[r * 4 + c] = component r of vector c) of a Hermitian 4 x 4 H.
 * The cyclic Jacobi method (Jacobi 1846; see Golub and Van Loan, Matrix
 * Computations, Sec. 8.5) runs on the real symmetric 8 x 8 embedding
 * M = [[Re H, -Im H], [Im H, Re H]]: each eigenvalue of H appears twice
 * in M, and an eigenvector (x, y) of M gives the eigenvector x + i y of H. */
void orc_herm4_eig(const cplx H[16], double w[4], cplx vec[16])
{
    double A[8][8], V[8][8];
    for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++) {
            A[r][c] = creal(H[r * 4 + c]);
            A[r][c + 4] = -cimag(H[r * 4 + c]);
            A[r + 4][c] = cimag(H[r * 4 + c]);
            A[r + 4][c + 4] = creal(H[r * 4 + c]);
        }
    for (int r = 0; r < 8; r++)
        for (int c = 0; c < 8; c++) V[r][c] = r == c ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = 0, diag = 0;
        for (int p = 0; p < 8; p++) {
            diag += A[p][p] * A[p][p];
            for (int q = p + 1; q < 8; q++) off += A[p][q] * A[p][q];
        }
        if (off <= 1e-34 * diag || off == 0.0) break;
        for (int p = 0; p < 8; p++)
            for (int q = p + 1; q < 8; q++) {
                if (A[p][q] == 0.0) continue;
                /* rotation J (J_pp = J_qq = c, J_pq = s, J_qp = -s) with
                 * (J^T A J)_pq = 0: t = tan(theta) is the smaller root of
                 * t^2 + 2 tau t - 1 = 0, tau = (A_qq - A_pp) / (2 A_pq) */
                double tau = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(tau * tau + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < 8; k++) {   /* A <- A J */
                    double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - sn * akq;
                    A[k][q] = sn * akp + c * akq;
                }
                for (int k = 0; k < 8; k++) {   /* A <- J^T A */
                    double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - sn * aqk;
                    A[q][k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < 8; k++) {   /* V <- V J */
                    double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - sn * vkq;
                    V[k][q] = sn * vkp + c * vkq;
                }
            }
    }
    /* the 8 eigenvalues in ascending order; each of H's comes twice: take
     * every other one, with the eigenvector of the first of each pair */
    int ord[8];
    for (int k = 0; k < 8; k++) ord[k] = k;
    for (int a = 0; a < 8; a++)
        for (int b = a + 1; b < 8; b++)
            if (A[ord[b]][ord[b]] < A[ord[a]][ord[a]]) { int t = ord[a]; ord[a] = ord[b]; ord[b] = t; }
    for (int e = 0; e < 4; e++) {
        int k = ord[2 * e];
        w[e] = 0.5 * (A[ord[2 * e]][ord[2 * e]] + A[ord[2 * e + 1]][ord[2 * e + 1]]);
        double nrm = 0;
        for (int r = 0; r < 4; r++) nrm += V[r][k] * V[r][k] + V[r + 4][k] * V[r + 4][k];
        nrm = sqrt(nrm);
        for (int r = 0; r < 4; r++) vec[r * 4 + e] = (V[r][k] + I * V[r + 4][k]) / nrm;
    }
}

/* The SDRP projection generalised to the pair (qa, qb): psi <- (|phi><phi|
 * on the pair, identity on the rest) psi, renormalised by the computed norm
 * (phi: four amplitudes, index bit qa + 2 bit qb). */
void orc_sdrp_project2(cplx *psi, int n, int qa, int qb, const cplx phi[4])
{
    uint64_t N = (uint64_t)1 << n, ba = (uint64_t)1 << qa, bb = (uint64_t)1 << qb;
    for (uint64_t i = 0; i < N; i++) {
        if ((i & ba) || (i & bb)) continue;
        uint64_t idx[4] = { i, i | ba, i | bb, i | ba | bb };
        cplx ov = 0;
        for (int x = 0; x < 4; x++) ov += conj(phi[x]) * psi[idx[x]];
        for (int x = 0; x < 4; x++) psi[idx[x]] = phi[x] * ov;
    }
    double s = sqrt(orc_norm2(psi, n));
    for (uint64_t i = 0; i < N; i++) psi[i] /= s;
}

/* Projects qubit q onto the Z eigenstate |v> (post-selects bit q = v and
 * renormalises by the computed norm). */
void orc_project_z(cplx *psi, int n, int q, int v)
{
    uint64_t N = (uint64_t)1 << n, bq = (uint64_t)1 << q;
    for (uint64_t i = 0; i < N; i++)
        if (((i & bq) != 0) != (v != 0)) psi[i] = 0;
    double s = sqrt(orc_norm2(psi, n));
    for (uint64_t i = 0; i < N; i++) psi[i] /= s;
}

/* Sec. II.B (unobservable optimisations, Table I "eliminates Z-basis
 * eigenstate controls"): the Z-eigenstate value of qubit q if it is a
 * subsystem of its own and its probability of the other value is at most
 * tau (returns 0 or 1, the eigenvalue's bit), else -1. A nonzero
 * probability of the other value is projected away first. */
static int z_eigen(cplx *psi, int n, const int *sys, int q, double tau)
{
    int members = 0;
    for (int x = 0; x < n; x++) members += sys[x] == sys[q];
    if (members != 1) return -1;
    double p1 = orc_prob1(psi, n, q);
    int v = p1 <= tau ? 0 : (1.0 - p1 <= tau ? 1 : -1);
    if (v >= 0 && (v == 0 ? p1 : 1.0 - p1) != 0.0) orc_project_z(psi, n, q, v);
    return v;
}

/* Runs a circuit with SDRP rounding on the full state vector (no
 * factorisation). psi must hold a product state on entry (normally
 * |0...0>); every qubit starts in its own subsystem.
 *
 * Subsystem bookkeeping is membership only: a two-qubit gate (or a
 * controlled one-qubit gate) merges the subsystems of its qubits, except a
 * SWAP, which only exchanges the two qubits' memberships; after a merge,
 * every qubit of the merged subsystem is checked in ascending global id,
 * one after the other, while that subsystem still holds two or more
 * qubits. A check computes r and eps = (1 - |r|)/2; eps <= p/2 (p > 0) rounds
 * (F <- F (1 - eps), Eq. fid_model); otherwise eps <= tau separates the
 * qubit exactly without touching F; otherwise the qubit stays. A rounded
 * or separated qubit becomes a subsystem of its own.
 *
 * force (optional, nforce entries): when given, only the listed
 * (gate, qubit) checks run, in the listed order, instead of the
 * exhaustive schedule. force_action (optional, nforce entries, only with
 * force): entry j >= 0 replaces the decision of check j (0 keep, 1 round,
 * 2 separate exactly) while r and eps are still computed and logged; -1
 * decides by eps as above. This replays another run's decisions, so that a
 * decision taken the other way at a near-tie (eps within rounding of p/2
 * or tau) does not hide the rest of the trajectory from the comparison.
 *
 * unobservable != 0 applies Sec. II.B's rule before each controlled
 * one-qubit gate and each controlled phase: a control (either qubit of a
 * CP) that is a one-qubit subsystem in a Z eigenstate, to within tau, is
 * first projected onto that eigenstate (fidelity >= 1 - tau, not entered
 * into F, as an exact separation); a control holding the value the gate
 * waits for is dropped, one holding the other value removes the gate. The
 * gate is still applied to the full vector, where it now acts exactly as
 * its reduced form; only the qubits it still couples merge, so a gate
 * reduced to a local one merges nothing and triggers no checks.
 * *nunobs_out (optional) counts the gates removed or reduced.
 *
 * pairs != 0 adds a two-qubit check after the one-qubit checks of a gate
 * that couples exactly two qubits (a, b): if a and b are still in one
 * subsystem of three or more qubits, rho of the pair gives eps = 1 -
 * (largest eigenvalue), the rounding error of the pair's dominant Schmidt
 * branch; eps <= p/2 rounds (F <- F (1 - eps)) and eps <= tau separates
 * exactly, projecting onto that branch's pair state, after which the pair is
 * a subsystem of its own. Its log entry has qubit a, pad 1 + b, and r the
 * three largest eigenvalues in descending order.
 *
 * Returns the number of decisions written to log (capped at logcap). */
int orc_sdrp_run(cplx *psi, int n, const orc_gate *g, int ng, double p, double tau,
                 const int32_t *force, int nforce, const int32_t *force_action, int unobservable, int pairs,
                 double *F_out, int *nround_out, int *nunobs_out, orc_decision *log, int logcap)
{
    int sys[64];
    int nextsys = n;
    for (int q = 0; q < n; q++) sys[q] = q;
    double F = 1.0;
    int nround = 0, nlog = 0, fpos = 0, nunobs = 0;

    for (int k = 0; k < ng; k++) {
        const orc_gate *gk = &g[k];
        /* qubits the gate still couples after the unobservable rule */
        int keep_q[ORC_MAXCTRL + 2], nkeep = -1, removed = 0;
        if (unobservable && (gk->kind == OG_CP || (gk->nctrl > 0 && gk->kind < OG_CP))) {
            nkeep = 0;
            if (gk->kind == OG_CP) {
                /* diag(1,1,1,e^{i theta}) is symmetric: either qubit may act as the control */
                int e0 = z_eigen(psi, n, sys, gk->q[0], tau);
                int e1 = e0 < 0 ? z_eigen(psi, n, sys, gk->q[1], tau) : -1;
                if (e0 >= 0 || e1 >= 0) {
                    int v = e0 >= 0 ? e0 : e1;
                    if (v == 0) removed = 1;
                    else keep_q[nkeep++] = e0 >= 0 ? gk->q[1] : gk->q[0];
                } else {
                    keep_q[nkeep++] = gk->q[0];
                    keep_q[nkeep++] = gk->q[1];
                }
            } else {
                keep_q[nkeep++] = gk->q[0];
                for (int j = 0; j < gk->nctrl; j++) {
                    int e = z_eigen(psi, n, sys, gk->ctrl[j], tau);
                    if (e < 0) {
                        keep_q[nkeep++] = gk->ctrl[j];
                        continue;
                    }
                    if (e != gk->cval[j]) removed = 1;
                }
            }
            const int orig = gk->kind == OG_CP ? 2 : 1 + gk->nctrl;   /* qubits the gate couples as written */
            if (removed || nkeep < orig) nunobs++;
        }
        if (orc_apply_gate(psi, n, gk)) return -1;
        if (nkeep >= 0 && (removed || nkeep < 2)) continue;   /* removed or local: nothing merges */
        if (gk->kind == OG_SWAP) {
            /* a SWAP entangles nothing: the two qubits trade subsystems */
            int t = sys[gk->q[0]];
            sys[gk->q[0]] = sys[gk->q[1]];
            sys[gk->q[1]] = t;
            continue;
        }
        int two = 0, a = -1, b = -1;
        cplx m[16];
        int d = orc_gate_matrix(gk, m);
        if (d == 4) { two = 1; a = gk->q[0]; b = gk->q[1]; }
        else if (gk->nctrl > 0) { two = 1; a = gk->q[0]; b = gk->ctrl[0]; }
        if (!two) continue;
        /* merge subsystems of every qubit the gate touches */
        int keep = sys[a], drop = sys[b];
        if (nkeep >= 2) {
            /* merge only the qubits the reduced gate still couples */
            keep = sys[keep_q[0]];
            for (int j = 1; j < nkeep; j++) {
                int dj = sys[keep_q[j]];
                for (int q = 0; q < n; q++) if (sys[q] == dj) sys[q] = keep;
            }
        } else {
            for (int q = 0; q < n; q++) if (sys[q] == drop) sys[q] = keep;
            for (int j = 1; j < gk->nctrl; j++) {
                int dj = sys[gk->ctrl[j]];
                for (int q = 0; q < n; q++) if (sys[q] == dj) sys[q] = keep;
            }
        }

        int cand[64], cact[64], ncand = 0;
        if (force) {
            while (fpos < nforce && force[2 * fpos] == k) {
                cact[ncand] = force_action ? force_action[fpos] : -1;
                cand[ncand++] = force[2 * fpos++ + 1];
            }
        } else {
            for (int q = 0; q < n; q++) if (sys[q] == keep) { cact[ncand] = -1; cand[ncand++] = q; }
        }
        for (int c = 0; c < ncand; c++) {
            int q = cand[c], members = 0;
            for (int x = 0; x < n; x++) if (sys[x] == sys[q]) members++;
            if (members < 2) continue;
            double r[3];
            orc_bloch(psi, n, q, r);
            double len = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
            double eps = (1.0 - len) / 2.0;
            int action = 0;
            if (p > 0.0 && eps <= p / 2.0) action = 1;   /* p = 0: exact simulation, nothing rounds */
            else if (eps <= tau) action = 2;
            if (cact[c] >= 0) action = cact[c];
            if (action) {
                orc_sdrp_project(psi, n, q, r);
                if (action == 1) { F *= (1.0 - eps); nround++; }
                sys[q] = nextsys++;
            }
            if (nlog < logcap) {
                log[nlog].gate = k; log[nlog].qubit = q; log[nlog].action = action;
                log[nlog].pad = 0; log[nlog].eps = eps;
                log[nlog].r[0] = r[0]; log[nlog].r[1] = r[1]; log[nlog].r[2] = r[2];
            }
            nlog++;
        }
        if (pairs) {
            /* the two qubits the gate couples (after the unobservable rule) */
            int pa = -1, pb = -1;
            if (nkeep >= 0) {
                if (nkeep == 2) { pa = keep_q[0]; pb = keep_q[1]; }
            } else if (d == 4) {
                pa = gk->q[0]; pb = gk->q[1];
            } else if (gk->nctrl == 1) {
                pa = gk->q[0]; pb = gk->ctrl[0];
            }
            int members = 0;
            if (pa >= 0 && sys[pa] == sys[pb])
                for (int x = 0; x < n; x++) members += sys[x] == sys[pa];
            if (members >= 3) {
                cplx rho[16], vec[16], phi[4];
                double w[4];
                orc_rho2(psi, n, pa, pb, rho);
                orc_herm4_eig(rho, w, vec);
                double eps = 1.0 - w[3];
                int action = 0;
                if (p > 0.0 && eps <= p / 2.0) action = 1;
                else if (eps <= tau) action = 2;
                if (action) {
                    for (int x = 0; x < 4; x++) phi[x] = vec[x * 4 + 3];
                    orc_sdrp_project2(psi, n, pa, pb, phi);
                    if (action == 1) { F *= (1.0 - eps); nround++; }
                    sys[pa] = sys[pb] = nextsys++;
                }
                if (nlog < logcap) {
                    log[nlog].gate = k; log[nlog].qubit = pa; log[nlog].action = action;
                    log[nlog].pad = 1 + pb; log[nlog].eps = eps;
                    log[nlog].r[0] = w[3]; log[nlog].r[1] = w[2]; log[nlog].r[2] = w[1];
                }
                nlog++;
            }
        }
    }
    *F_out = F;
    *nround_out = nround;
    if (nunobs_out) *nunobs_out = nunobs;
    return nlog;
}
