// Approximate mode: SDRP rounding on a factorised ket (arXiv 2304.14969,
// Sec. II.A and Sec. III.A-B).
//
// The ket is kept as a tensor product of subsystem kets (Sec. II.A, "as
// factorized as possible"); every subsystem lives in its own device buffer
// with local bit b holding global qubit qs[b]. A two-qubit gate spanning two
// subsystems first composes them (Kronecker product); a SWAP is a relabel
// (Table I). After every entangling gate the qubits of the touched subsystem
// are checked in ascending global id: the Bloch sums of all its qubits come
// from one tiled FP64 reduction, a one-thread kernel forms
// r = (<X>, <Y>, <Z>), eps = (1 - |r|)/2 (step 2) and picks the first
// candidate with eps <= p/2 (SDRP rounding, Eq. sdrp) or eps <= tau (exact
// separation); that qubit is projected onto the dominant Schmidt branch
// |phi> (steps 2-4 collapse to <phi|_q applied to the subsystem, then an
// FP64 renormalisation) and becomes a one-qubit subsystem holding |phi>.
// F <- F (1 - eps) for each rounding (Eq. fid_model). Candidates after the
// rounded one are checked again on the new, smaller subsystem.
//
// Optionally (opts->unobservable, Sec. II.B and Table I) a controlled gate
// whose control is a one-qubit subsystem in a Z eigenstate is removed or
// reduced before anything is composed: the control's two amplitudes are
// read back, a probability of the other value of at most tau projects it
// onto the eigenstate, and the gate then drops that control (value as
// required) or is removed (value opposite); a controlled phase may use
// either qubit as the control. A gate left on one qubit runs locally and
// entangles nothing, so no check follows it.
//
// Optionally (opts->pairs) the rounding also acts on two-qubit subsystems:
// after the one-qubit checks of a gate coupling exactly two qubits a, b
// that still share a subsystem of three or more qubits, one FP64 reduction
// gives the pair's 4 x 4 reduced density matrix, a complex Jacobi
// iteration on the host its eigenvalues, and eps = 1 - lambda_max decides
// (eps <= p/2 rounds, eps <= tau separates exactly): the subsystem is
// projected onto the top eigenvector |phi> of the pair, which becomes a
// two-qubit subsystem holding |phi>.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>

#include "qsim_internal.h"

namespace qs {

qsim_status validate_circuit(const qsim_circuit *c);
qsim_status mlp_infer_device(const qsim_mlp *m, const float *d_x, int rows, float *d_out, cudaStream_t st);
int mlp_nfeat(const qsim_mlp *m);

// Features of a candidate qubit for the proposal network (all known on the
// host before any reduction runs): the Bloch vector and its length from the
// qubit's last check (stale by design: the fresh one is what a check
// costs), its rounding error then, gates on it since (one- and two-qubit),
// gates since its last check, whether that check separated it, the
// subsystem size relative to n, p, and a constant.
static const int kFeat = 12;
struct QubitHist {
    double r[3] = {0, 0, 1};
    int g1 = 0, g2 = 0, last = -1, sep = 0;
};

static void features(const QubitHist &h, int gate, int m, int n, double p, float *f)
{
    double len = std::sqrt(h.r[0] * h.r[0] + h.r[1] * h.r[1] + h.r[2] * h.r[2]);
    f[0] = (float)h.r[0];
    f[1] = (float)h.r[1];
    f[2] = (float)h.r[2];
    f[3] = (float)len;
    f[4] = (float)((1.0 - len) / 2.0);
    f[5] = (float)h.g1 / 8.0f;
    f[6] = (float)h.g2 / 8.0f;
    f[7] = (float)(h.last < 0 ? gate + 1 : gate - h.last) / 64.0f;
    f[8] = (float)h.sep;
    f[9] = (float)m / (float)n;
    f[10] = (float)p;
    f[11] = 1.0f;
}

template <typename R> struct AV;
template <> struct AV<float> { using T = float2; };
template <> struct AV<double> { using T = double2; };

// C[ia + (ib << ma)] = A[ia] * B[ib]
template <typename R>
__global__ void k_kron(const typename AV<R>::T *__restrict__ A, int ma, const typename AV<R>::T *__restrict__ B,
                       uint64_t nb, typename AV<R>::T *__restrict__ Cc)
{
    uint64_t total = nb << ma, stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        auto a = A[i & ((1ull << ma) - 1)];
        auto b = B[i >> ma];
        typename AV<R>::T o;
        o.x = a.x * b.x - a.y * b.y;
        o.y = a.x * b.y + a.y * b.x;
        Cc[i] = o;
    }
}

// dst[j] = conj(f0) src[j with bit b = 0] + conj(f1) src[j with bit b = 1]
template <typename R>
__global__ void k_project(const typename AV<R>::T *__restrict__ src, int b, uint64_t nout, double f0r, double f0i,
                          double f1r, double f1i, typename AV<R>::T *__restrict__ dst)
{
    const R c0r = (R)f0r, c0i = (R)-f0i, c1r = (R)f1r, c1i = (R)-f1i;
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x, lo = (1ull << b) - 1;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nout; j += stride) {
        uint64_t i0 = ((j & ~lo) << 1) | (j & lo);
        auto x = src[i0], y = src[i0 | (1ull << b)];
        typename AV<R>::T o;
        o.x = c0r * x.x - c0i * x.y + c1r * y.x - c1i * y.y;
        o.y = c0r * x.y + c0i * x.x + c1r * y.y + c1i * y.x;
        dst[j] = o;
    }
}

template <typename R>
__global__ void k_put2(typename AV<R>::T *__restrict__ d, double a0r, double a0i, double a1r, double a1i)
{
    d[0].x = (R)a0r;
    d[0].y = (R)a0i;
    d[1].x = (R)a1r;
    d[1].y = (R)a1i;
}

// The 16 FP64 sums of a pair's reduced density matrix (unnormalised) over
// the quads of a subsystem ket (pair bits ba, bb): |a_x|^2 for x = 0..3,
// then Re and Im of a_x conj(a_y) for the six x < y, x = bit ba + 2 bit bb.
// One row of 16 partial sums per CTA.
constexpr int kRhoThreads = 128;
template <typename R>
__global__ void __launch_bounds__(kRhoThreads) k_rho2(const typename AV<R>::T *__restrict__ a, int ba, int bb,
                                                       uint64_t nquads, double *__restrict__ part)
{
    double acc[16];
#pragma unroll
    for (int k = 0; k < 16; k++) acc[k] = 0.0;
    const int lo = ba < bb ? ba : bb, hi = ba < bb ? bb : ba;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nquads; j += stride) {
        // insert zero bits at lo, then hi
        uint64_t i = ((j >> lo) << (lo + 1)) | (j & ((1ull << lo) - 1));
        i = ((i >> hi) << (hi + 1)) | (i & ((1ull << hi) - 1));
        double xr[4], xi[4];
#pragma unroll
        for (int x = 0; x < 4; x++) {
            const auto v = a[i | ((uint64_t)(x & 1) << ba) | ((uint64_t)(x >> 1) << bb)];
            xr[x] = (double)v.x;
            xi[x] = (double)v.y;
        }
#pragma unroll
        for (int x = 0; x < 4; x++) acc[x] += xr[x] * xr[x] + xi[x] * xi[x];
        int k = 4;
#pragma unroll
        for (int x = 0; x < 4; x++)
#pragma unroll
            for (int y = x + 1; y < 4; y++) {
                // a_x conj(a_y)
                acc[k++] += xr[x] * xr[y] + xi[x] * xi[y];
                acc[k++] += xi[x] * xr[y] - xr[x] * xi[y];
            }
    }
    __shared__ double sh[kRhoThreads / 32][16];
#pragma unroll
    for (int k = 0; k < 16; k++) {
        double v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 16) {
        double v = 0;
        for (int w = 0; w < kRhoThreads / 32; w++) v += sh[w][threadIdx.x];
        part[(size_t)blockIdx.x * 16 + threadIdx.x] = v;
    }
}

// Four complex amplitudes of a pair state (index bit a + 2 bit b).
struct Pair4 {
    double re[4], im[4];
};

// dst[j] = sum_x conj(phi_x) src[j with the pair bits (ba, bb) = x]: the
// subsystem ket projected onto <phi| of the pair (m - 2 qubits out).
template <typename R>
__global__ void k_project2(const typename AV<R>::T *__restrict__ src, int ba, int bb, uint64_t nout, const Pair4 ph,
                           typename AV<R>::T *__restrict__ dst)
{
    const double *pr = ph.re, *pi = ph.im;
    const int lo = ba < bb ? ba : bb, hi = ba < bb ? bb : ba;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nout; j += stride) {
        uint64_t i = ((j >> lo) << (lo + 1)) | (j & ((1ull << lo) - 1));
        i = ((i >> hi) << (hi + 1)) | (i & ((1ull << hi) - 1));
        double orr = 0, oi = 0;
#pragma unroll
        for (int x = 0; x < 4; x++) {
            const auto v = src[i | ((uint64_t)(x & 1) << ba) | ((uint64_t)(x >> 1) << bb)];
            // conj(phi_x) v
            orr += pr[x] * (double)v.x + pi[x] * (double)v.y;
            oi += pr[x] * (double)v.y - pi[x] * (double)v.x;
        }
        typename AV<R>::T o;
        o.x = (R)orr;
        o.y = (R)oi;
        dst[j] = o;
    }
}

template <typename R>
__global__ void k_put4(typename AV<R>::T *__restrict__ d, const Pair4 ph)
{
    for (int x = 0; x < 4; x++) {
        d[x].x = (R)ph.re[x];
        d[x].y = (R)ph.im[x];
    }
}

// Eigenvalues (ascending) and unit eigenvectors (columns) of a Hermitian
// 4 x 4 by cyclic complex Jacobi rotations: for the entry h_pq = r e^{i f},
// G = [[c, s e^{i f}], [-s e^{-i f}, c]] on (p, q), with t = s / c the
// smaller root of t^2 + 2 tau t - 1 = 0, tau = (h_qq - h_pp) / (2 r), makes
// (G^H H G)_pq = 0; V accumulates the G.
static void herm4_jacobi(cd H[4][4], double w[4], cd V[4][4])
{
    for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++) V[r][c] = r == c ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 60; sweep++) {
        double off = 0, dg = 0;
        for (int p = 0; p < 4; p++) {
            dg += std::norm(H[p][p]);
            for (int q = p + 1; q < 4; q++) off += std::norm(H[p][q]);
        }
        if (off == 0.0 || off <= 1e-34 * dg) break;
        for (int p = 0; p < 4; p++)
            for (int q = p + 1; q < 4; q++) {
                const double r = std::abs(H[p][q]);
                if (r == 0.0) continue;
                const cd e = H[p][q] / r;   // e^{i f}
                const double tau = (H[q][q].real() - H[p][p].real()) / (2.0 * r);
                const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(tau * tau + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
                const cd gpq = sn * e, gqp = -sn * std::conj(e);
                for (int k = 0; k < 4; k++) {   // H <- H G
                    const cd hp = H[k][p], hq = H[k][q];
                    H[k][p] = c * hp + gqp * hq;
                    H[k][q] = gpq * hp + c * hq;
                }
                for (int k = 0; k < 4; k++) {   // H <- G^H H
                    const cd hp = H[p][k], hq = H[q][k];
                    H[p][k] = c * hp + std::conj(gqp) * hq;
                    H[q][k] = std::conj(gpq) * hp + c * hq;
                }
                for (int k = 0; k < 4; k++) {   // V <- V G
                    const cd vp = V[k][p], vq = V[k][q];
                    V[k][p] = c * vp + gqp * vq;
                    V[k][q] = gpq * vp + c * vq;
                }
            }
    }
    int ord[4] = {0, 1, 2, 3};
    std::sort(ord, ord + 4, [&](int x, int y) { return H[x][x].real() < H[y][y].real(); });
    cd Vs[4][4];
    for (int e = 0; e < 4; e++) {
        w[e] = H[ord[e]][ord[e]].real();
        for (int r = 0; r < 4; r++) Vs[r][e] = V[r][ord[e]];
    }
    for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++) V[r][c] = Vs[r][c];
}

struct Decide {
    int32_t first;       // index into the candidate list of the first acted-on qubit, or ncand
    int32_t action;      // 1 rounded, 2 exact, 0 none
    int32_t examined;
    int32_t pad;
    double eps[64];
    double r[64][3];
    double phi[4];       // |phi> of the acted-on qubit (re0, im0, re1, im1)
    int32_t nsel;        // MLP rounds: candidates the network proposed (rows of the scored list)
    int32_t pad2;
    int32_t sel[64];
};

// Sec. III.A step 2 in FP64 on the device: for candidates in order, r from
// the Bloch sums, eps = (1 - |r|)/2, stop at the first eps <= p/2 (round) or
// eps <= tau (exact separation). |phi> = (cos(th/2), e^{i ph} sin(th/2)),
// th = acos(r_z/|r|), ph = atan2(r_y, r_x); +z when |r| < 1e-15.
__global__ void k_decide(const double *__restrict__ sums, const int *__restrict__ cand, int ncand, double p,
                         double tau, Decide *__restrict__ out, const int *__restrict__ d_ncand)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (d_ncand) ncand = *d_ncand;
    out->first = ncand;
    out->action = 0;
    int k = 0;
    for (; k < ncand; k++) {
        const double *s = sums + 4 * cand[k];
        double tr = s[0] + s[1];
        double r0 = 2.0 * s[2] / tr, r1 = 2.0 * s[3] / tr, r2 = (s[0] - s[1]) / tr;
        double len = sqrt(r0 * r0 + r1 * r1 + r2 * r2);
        double eps = (1.0 - len) / 2.0;
        out->eps[k] = eps;
        out->r[k][0] = r0;
        out->r[k][1] = r1;
        out->r[k][2] = r2;
        int act = (p > 0.0 && eps <= p / 2.0) ? 1 : (eps <= tau ? 2 : 0);   // p = 0 rounds nothing
        if (act) {
            double th = 0.0, ph = 0.0;
            if (len >= 1e-15) {
                double cz = fmin(1.0, fmax(-1.0, r2 / len));
                th = acos(cz);
                ph = atan2(r1, r0);
            }
            double ch = cos(th / 2.0), sh = sin(th / 2.0);
            out->phi[0] = ch;
            out->phi[1] = 0.0;
            out->phi[2] = cos(ph) * sh;
            out->phi[3] = sin(ph) * sh;
            out->first = k;
            out->action = act;
            k++;
            break;
        }
    }
    out->examined = k;
}

// Proposal step of an MLP check round, on the device so that the round
// needs one host synchronisation, as an exhaustive one: of the `rows`
// scored qubits (ascending ids, local bits loc[]), those with logit > 0,
// the top_m by logit (ties to the lower row), in ascending order: their
// local bits go to cand[], their count to *ncand (0: the round's Bloch
// passes and decisions do nothing), their rows to out->sel.
__global__ void k_mlp_select(const float *__restrict__ logit, const int *__restrict__ loc, int rows, int top_m,
                             int *__restrict__ cand, int *__restrict__ ncand, Decide *__restrict__ out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    uint64_t chosen = 0;
    int nsel = 0;
    while (nsel < top_m) {
        int best = -1;
        for (int i = 0; i < rows; i++)
            if (!((chosen >> i) & 1) && logit[i] > 0.f && (best < 0 || logit[i] > logit[best])) best = i;
        if (best < 0) break;
        chosen |= 1ull << best;
        nsel++;
    }
    int k = 0;
    for (int i = 0; i < rows; i++)
        if ((chosen >> i) & 1) {
            out->sel[k] = i;
            cand[k++] = loc[i];
        }
    out->nsel = k;
    *ncand = k;
}

namespace {

struct Sub {
    std::vector<int> qs;   // local bit -> global qubit
    void *d = nullptr;
    size_t bytes = 0;
};

struct Run {
    int n = 0;
    qsim_dtype dt = QSIM_C64;
    cudaStream_t st = nullptr;
    size_t es = 8;
    double budget = 0;
    size_t cur = 0, peak = 0;
    std::vector<std::unique_ptr<Sub>> subs;
    std::vector<int> sys_of;  // global qubit -> index in subs
    Scratch sc;
    double *d_sums = nullptr;
    int *d_cand = nullptr;
    int *d_loc = nullptr;       // MLP rounds: local bits of the scored qubits, then the count
    Decide *d_dec = nullptr, *h_dec = nullptr;
    double *h_amp2 = nullptr;   // pinned: two amplitudes of a one-qubit factor (re, im each)
    int64_t bloch_passes = 0;

    ~Run()
    {
        cudaStreamSynchronize(st);
        for (auto &s : subs)
            if (s && s->d) cudaFree(s->d);
        if (d_sums) cudaFree(d_sums);
        if (d_cand) cudaFree(d_cand);
        if (d_loc) cudaFree(d_loc);
        if (d_dec) cudaFree(d_dec);
        if (h_dec) cudaFreeHost(h_dec);
        if (h_amp2) cudaFreeHost(h_amp2);
        free_scratch(sc);
    }

    qsim_status alloc(Sub &s, int m)
    {
        s.bytes = es << m;
        QS_CUDA(cudaMallocAsync(&s.d, s.bytes, st));
        cur += s.bytes;
        peak = std::max(peak, cur);
        return QSIM_OK;
    }
    void release(Sub &s)
    {
        if (s.d) cudaFreeAsync(s.d, st);
        cur -= s.bytes;
        s.d = nullptr;
        s.bytes = 0;
    }

    qsim_state view(Sub &s)
    {
        qsim_state v;
        v.n = (int)s.qs.size();
        v.dt = dt;
        v.stream = st;
        v.amps = s.d;
        v.owned = false;
        v.l2p.resize(v.n);
        for (int b = 0; b < v.n; b++) v.l2p[b] = b;
        return v;
    }

    int local(const Sub &s, int q) const
    {
        for (size_t b = 0; b < s.qs.size(); b++)
            if (s.qs[b] == q) return (int)b;
        return -1;
    }

    // merge subsystem j into i (i keeps its low bits)
    qsim_status compose(int i, int j)
    {
        Sub &A = *subs[i], &B = *subs[j];
        int ma = (int)A.qs.size(), mb = (int)B.qs.size();
        size_t nb = es << (ma + mb);
        if ((double)(cur + nb) > budget) return fail(QSIM_E_BUDGET, "composing %d+%d qubits exceeds the budget", ma, mb);
        Sub C;
        C.qs = A.qs;
        C.qs.insert(C.qs.end(), B.qs.begin(), B.qs.end());
        QS_TRY(alloc(C, ma + mb));
        uint64_t total = 1ull << (ma + mb);
        int grid = default_grid(total, 256);
        if (dt == QSIM_C64)
            k_kron<float><<<grid, 256, 0, st>>>((const float2 *)A.d, ma, (const float2 *)B.d, 1ull << mb, (float2 *)C.d);
        else
            k_kron<double><<<grid, 256, 0, st>>>((const double2 *)A.d, ma, (const double2 *)B.d, 1ull << mb,
                                                 (double2 *)C.d);
        QS_CUDA(cudaGetLastError());
        release(A);
        release(B);
        A = C;
        C.d = nullptr;
        for (int q : A.qs) sys_of[q] = i;
        subs[j].reset();
        return QSIM_OK;
    }

    // Z-eigenstate value of qubit q (0 or 1) if it is a one-qubit subsystem
    // whose probability of the other value is at most tau, else -1; an
    // eigenstate within tau is made exact (the factor projected onto it,
    // keeping its phase).
    qsim_status z_eigen(int q, double tau, int *out)
    {
        *out = -1;
        Sub &S = *subs[sys_of[q]];
        if (S.qs.size() != 1) return QSIM_OK;
        if (dt == QSIM_C64) {
            float f[4];
            QS_CUDA(cudaMemcpyAsync(f, S.d, sizeof f, cudaMemcpyDeviceToHost, st));
            QS_CUDA(cudaStreamSynchronize(st));
            for (int i = 0; i < 4; i++) h_amp2[i] = f[i];
        } else {
            QS_CUDA(cudaMemcpyAsync(h_amp2, S.d, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
            QS_CUDA(cudaStreamSynchronize(st));
        }
        const double a2 = h_amp2[0] * h_amp2[0] + h_amp2[1] * h_amp2[1];
        const double b2 = h_amp2[2] * h_amp2[2] + h_amp2[3] * h_amp2[3];
        const double p1 = b2 / (a2 + b2);
        if (p1 <= tau) *out = 0;
        else if (1.0 - p1 <= tau) *out = 1;
        else return QSIM_OK;
        if (*out == 0 && b2 != 0.0) {
            const double ra = std::sqrt(a2);
            if (dt == QSIM_C64) k_put2<float><<<1, 1, 0, st>>>((float2 *)S.d, h_amp2[0] / ra, h_amp2[1] / ra, 0, 0);
            else k_put2<double><<<1, 1, 0, st>>>((double2 *)S.d, h_amp2[0] / ra, h_amp2[1] / ra, 0, 0);
            QS_CUDA(cudaGetLastError());
        } else if (*out == 1 && a2 != 0.0) {
            const double rb = std::sqrt(b2);
            if (dt == QSIM_C64) k_put2<float><<<1, 1, 0, st>>>((float2 *)S.d, 0, 0, h_amp2[2] / rb, h_amp2[3] / rb);
            else k_put2<double><<<1, 1, 0, st>>>((double2 *)S.d, 0, 0, h_amp2[2] / rb, h_amp2[3] / rb);
            QS_CUDA(cudaGetLastError());
        }
        return QSIM_OK;
    }

    // reduced density matrix of the pair (qubits qa, qb) of subsystem i,
    // normalised, rho[x][y] with x = bit qa + 2 bit qb (FP64)
    qsim_status pair_rho(int i, int qa, int qb, cd rho[4][4])
    {
        Sub &S = *subs[i];
        const int m = (int)S.qs.size();
        const int ba = local(S, qa), bb = local(S, qb);
        const uint64_t nquads = 1ull << (m - 2);
        const int grid = (int)std::min<uint64_t>((nquads + kRhoThreads - 1) / kRhoThreads, 256);
        QS_TRY(ensure_scratch(sc, (size_t)grid * 16 + 64));
        if (dt == QSIM_C64)
            k_rho2<float><<<grid, kRhoThreads, 0, st>>>((const float2 *)S.d, ba, bb, nquads, sc.d);
        else
            k_rho2<double><<<grid, kRhoThreads, 0, st>>>((const double2 *)S.d, ba, bb, nquads, sc.d);
        QS_CUDA(cudaGetLastError());
        std::vector<double> part((size_t)grid * 16);
        QS_CUDA(cudaMemcpyAsync(part.data(), sc.d, part.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        QS_CUDA(cudaStreamSynchronize(st));
        double v[16] = {0};
        for (int b = 0; b < grid; b++)
            for (int k = 0; k < 16; k++) v[k] += part[(size_t)b * 16 + k];
        const double tr = v[0] + v[1] + v[2] + v[3];
        if (!(tr > 0)) return fail(QSIM_E_CUDA, "pair check on a ket of zero norm");
        for (int x = 0; x < 4; x++) rho[x][x] = v[x] / tr;
        int k = 4;
        for (int x = 0; x < 4; x++)
            for (int y = x + 1; y < 4; y++) {
                rho[x][y] = cd(v[k], v[k + 1]) / tr;
                rho[y][x] = std::conj(rho[x][y]);
                k += 2;
            }
        bloch_passes++;
        return QSIM_OK;
    }

    // projects the pair (qa, qb) of subsystem i onto phi (index bit qa + 2
    // bit qb) and splits it off as a two-qubit subsystem
    qsim_status split2(int i, int qa, int qb, const cd phi[4])
    {
        Sub &S = *subs[i];
        const int m = (int)S.qs.size();
        const int ba = local(S, qa), bb = local(S, qb);
        Sub R;
        for (int b = 0; b < m; b++)
            if (b != ba && b != bb) R.qs.push_back(S.qs[b]);
        QS_TRY(alloc(R, m - 2));
        const uint64_t nout = 1ull << (m - 2);
        const int grid = default_grid(nout, 256);
        Pair4 ph;
        for (int x = 0; x < 4; x++) {
            ph.re[x] = phi[x].real();
            ph.im[x] = phi[x].imag();
        }
        if (dt == QSIM_C64)
            k_project2<float><<<grid, 256, 0, st>>>((const float2 *)S.d, ba, bb, nout, ph, (float2 *)R.d);
        else
            k_project2<double><<<grid, 256, 0, st>>>((const double2 *)S.d, ba, bb, nout, ph, (double2 *)R.d);
        QS_CUDA(cudaGetLastError());
        release(S);
        S = R;
        R.d = nullptr;
        for (int q : S.qs) sys_of[q] = i;
        // renormalise by the computed FP64 norm (Sec. III.A step 3)
        qsim_state v = view(S);
        v.red = sc;
        double nrm = 0;
        qsim_status stt = reduce_norm(&v, &nrm);
        sc = v.red;
        v.red = Scratch();
        QS_TRY(stt);
        if (!(nrm > 0)) return fail(QSIM_E_CUDA, "projected ket has zero norm");
        QS_CUDA(launch_scale(S.d, dt, nout, 1.0 / std::sqrt(nrm), st));
        // the pair's new subsystem holds |phi> (local bit 0 = qa, 1 = qb)
        auto F = std::make_unique<Sub>();
        F->qs = {qa, qb};
        QS_TRY(alloc(*F, 2));
        if (dt == QSIM_C64) k_put4<float><<<1, 1, 0, st>>>((float2 *)F->d, ph);
        else k_put4<double><<<1, 1, 0, st>>>((double2 *)F->d, ph);
        QS_CUDA(cudaGetLastError());
        subs.push_back(std::move(F));
        sys_of[qa] = sys_of[qb] = (int)subs.size() - 1;
        return QSIM_OK;
    }

    // projects qubit at local bit b of subsystem i onto phi and splits it off
    qsim_status split(int i, int b, const double phi[4])
    {
        Sub &S = *subs[i];
        int m = (int)S.qs.size();
        int q = S.qs[b];
        Sub R;
        R.qs = S.qs;
        R.qs.erase(R.qs.begin() + b);
        QS_TRY(alloc(R, m - 1));
        uint64_t nout = 1ull << (m - 1);
        int grid = default_grid(nout, 256);
        if (dt == QSIM_C64)
            k_project<float><<<grid, 256, 0, st>>>((const float2 *)S.d, b, nout, phi[0], phi[1], phi[2], phi[3],
                                                  (float2 *)R.d);
        else
            k_project<double><<<grid, 256, 0, st>>>((const double2 *)S.d, b, nout, phi[0], phi[1], phi[2], phi[3],
                                                   (double2 *)R.d);
        QS_CUDA(cudaGetLastError());
        release(S);
        S = R;
        R.d = nullptr;
        // renormalise by the computed FP64 norm (Sec. III.A step 3)
        qsim_state v = view(S);
        v.red = sc;
        double nrm = 0;
        qsim_status stt = reduce_norm(&v, &nrm);
        sc = v.red;
        v.red = Scratch();
        QS_TRY(stt);
        if (!(nrm > 0)) return fail(QSIM_E_CUDA, "projected ket has zero norm");
        QS_CUDA(launch_scale(S.d, dt, 1ull << (m - 1), 1.0 / std::sqrt(nrm), st));
        // the new one-qubit factor
        auto F = std::make_unique<Sub>();
        F->qs = {q};
        QS_TRY(alloc(*F, 1));
        if (dt == QSIM_C64) k_put2<float><<<1, 1, 0, st>>>((float2 *)F->d, phi[0], phi[1], phi[2], phi[3]);
        else k_put2<double><<<1, 1, 0, st>>>((double2 *)F->d, phi[0], phi[1], phi[2], phi[3]);
        QS_CUDA(cudaGetLastError());
        subs.push_back(std::move(F));
        sys_of[q] = (int)subs.size() - 1;
        return QSIM_OK;
    }
};

}  // namespace
}  // namespace qs

using namespace qs;

extern "C" qsim_status qsim_approx_run(const qsim_circuit *c, double p, const qsim_approx_opts *opts,
                                       qsim_approx_result *res)
{
    clear_error();
    QS_TRY(validate_circuit(c));
    if (!res) return fail(QSIM_E_INVAL, "result is NULL");
    if (!(p >= 0.0 && p <= 1.0)) return fail(QSIM_E_INVAL, "p=%g outside [0, 1]", p);
    qsim_approx_opts o{};
    if (opts) o = *opts;
    if (o.dtype != QSIM_C64 && o.dtype != QSIM_C128) return fail(QSIM_E_INVAL, "unknown dtype");
    if (o.schedule == QSIM_SCHED_MLP) {
        if (!o.mlp) return fail(QSIM_E_INVAL, "MLP schedule needs opts->mlp");
        if (mlp_nfeat(o.mlp) != kFeat) return fail(QSIM_E_INVAL, "the proposal MLP must take %d features", kFeat);
        if (o.top_m < 1) return fail(QSIM_E_INVAL, "top_m must be >= 1");
    }
    if (o.schedule < 0 || o.schedule > 2) return fail(QSIM_E_INVAL, "unknown schedule %d", o.schedule);
    if (o.schedule == QSIM_SCHED_FORCED && o.nforce > 0 && !o.force) return fail(QSIM_E_INVAL, "force is NULL");
    if (o.state_out && c->n > 30) return fail(QSIM_E_INVAL, "state_out needs n <= 30");
    memset(res, 0, sizeof *res);
    res->budget_gate = -1;
    auto t0 = std::chrono::steady_clock::now();

    Run R;
    R.n = c->n;
    R.dt = (qsim_dtype)o.dtype;
    R.es = R.dt == QSIM_C64 ? 8 : 16;
    R.st = (cudaStream_t)o.stream;
    R.budget = o.budget_bytes > 0 ? o.budget_bytes : 64.0 * (1ull << 30);
    double tau = o.tau > 0 ? o.tau : (R.dt == QSIM_C64 ? 1e-6 : 1e-13);
    const int n = c->n;
    R.sys_of.resize(n);
    QS_CUDA(cudaMalloc(&R.d_sums, 4 * sizeof(double) * 64));
    QS_CUDA(cudaMalloc(&R.d_cand, sizeof(int) * 64));
    QS_CUDA(cudaMalloc(&R.d_loc, sizeof(int) * 65));
    QS_CUDA(cudaMalloc(&R.d_dec, sizeof(Decide)));
    QS_CUDA(cudaMallocHost(&R.h_dec, sizeof(Decide)));
    QS_CUDA(cudaMallocHost(&R.h_amp2, 4 * sizeof(double)));
    for (int q = 0; q < n; q++) {
        auto s = std::make_unique<Sub>();
        s->qs = {q};
        QS_TRY(R.alloc(*s, 1));
        if (R.dt == QSIM_C64) k_put2<float><<<1, 1, 0, R.st>>>((float2 *)s->d, 1, 0, 0, 0);
        else k_put2<double><<<1, 1, 0, R.st>>>((double2 *)s->d, 1, 0, 0, 0);
        R.subs.push_back(std::move(s));
        R.sys_of[q] = q;
    }
    QS_CUDA(cudaGetLastError());

    std::vector<QubitHist> hist(n);
    float *d_feat = nullptr, *d_logit = nullptr;
    std::vector<float> hfeat, hlogit;
    if (o.schedule == QSIM_SCHED_MLP) {
        QS_CUDA(cudaMalloc(&d_feat, sizeof(float) * kFeat * 64));
        QS_CUDA(cudaMalloc(&d_logit, sizeof(float) * 64));
    }
    struct Free {
        float *a, *b;
        ~Free() { if (a) cudaFree(a); if (b) cudaFree(b); }
    } free_mlp{d_feat, d_logit};
    int64_t n_ent = 0, ntrace = 0;
    double F = 1.0;
    int64_t nlog = 0, nround = 0, nexact = 0, nchecks = 0, nunobs = 0;
    int maxsub = 1, fpos = 0;
    qsim_status status = QSIM_OK;
    for (int k = 0; k < c->ngates && status == QSIM_OK; k++) {
        const qsim_gate &g = c->gates[k];
        cd m[16];
        int d = gate_matrix(g, c->matrices, c->nmatrix_doubles, m);
        if (g.kind == QSIM_G_SWAP) {
            int a = g.q0, b = g.q1, ia = R.sys_of[a], ib = R.sys_of[b];
            Sub &A = *R.subs[ia], &B = *R.subs[ib];
            A.qs[R.local(A, a)] = -1;
            B.qs[R.local(B, b)] = a;
            A.qs[R.local(A, -1)] = b;
            R.sys_of[a] = ib;
            R.sys_of[b] = ia;
            continue;
        }
        // Sec. II.B: Z-eigenstate controls removed, or the gate removed
        qsim_gate gr = g;       // the gate as reduced
        bool removed = false;
        if (o.unobservable && (g.kind == QSIM_G_CP || (d == 2 && g.ncontrols > 0))) {
            bool reduced = false;
            if (g.kind == QSIM_G_CP) {
                int e0 = -1, e1 = -1;
                QS_TRY(R.z_eigen(g.q0, tau, &e0));
                if (e0 < 0) QS_TRY(R.z_eigen(g.q1, tau, &e1));
                if (e0 >= 0 || e1 >= 0) {
                    reduced = true;
                    const int v = e0 >= 0 ? e0 : e1;
                    if (v == 0) {
                        removed = true;
                    } else {
                        // CP with one qubit in |1>: the phase diag(1, e^{i theta}) on the other
                        gr.kind = QSIM_G_PHASE;
                        gr.q0 = e0 >= 0 ? g.q1 : g.q0;
                        gr.q1 = -1;
                        gr.ncontrols = 0;
                        d = gate_matrix(gr, c->matrices, c->nmatrix_doubles, m);
                    }
                }
            } else {
                gr.ncontrols = 0;
                gr.control_values = 0;
                for (int j = 0; j < g.ncontrols; j++) {
                    int e = -1;
                    QS_TRY(R.z_eigen(g.controls[j], tau, &e));
                    if (e < 0) {
                        if ((g.control_values >> j) & 1) gr.control_values |= 1u << gr.ncontrols;
                        gr.controls[gr.ncontrols++] = g.controls[j];
                        continue;
                    }
                    reduced = true;
                    if (e != (int)((g.control_values >> j) & 1)) removed = true;
                }
            }
            if (reduced) nunobs++;
        }
        if (removed) {
            hist[g.q0].g1++;
            continue;
        }
        std::vector<int> touched;
        touched.push_back(gr.q0);
        if (d == 4) touched.push_back(gr.q1);
        for (int j = 0; j < gr.ncontrols; j++) touched.push_back(gr.controls[j]);
        int si = R.sys_of[touched[0]];
        for (size_t j = 1; j < touched.size() && status == QSIM_OK; j++) {
            int sj = R.sys_of[touched[j]];
            if (sj != si) {
                status = R.compose(si, sj);
                if (status == QSIM_E_BUDGET) res->budget_gate = k;
            }
        }
        if (status != QSIM_OK) break;
        Sub &S = *R.subs[si];
        maxsub = std::max(maxsub, (int)S.qs.size());
        qsim_state v = R.view(S);
        if (d == 2) {
            uint64_t cmask = 0, cval = 0;
            for (int j = 0; j < gr.ncontrols; j++) {
                uint64_t bb = bit(R.local(S, gr.controls[j]));
                cmask |= bb;
                if ((gr.control_values >> j) & 1) cval |= bb;
            }
            QS_CUDA(launch_gate1(&v, m, R.local(S, gr.q0), cmask, cval));
        } else if (gr.kind == QSIM_G_CP) {
            QS_CUDA(launch_cphase(&v, R.local(S, gr.q0), R.local(S, gr.q1), gr.params[0]));
        } else {
            QS_CUDA(launch_gate2(&v, m, R.local(S, gr.q0), R.local(S, gr.q1)));
        }
        if (touched.size() < 2) {
            hist[gr.q0].g1++;
            continue;
        }
        for (int q : touched) hist[q].g2++;
        n_ent++;

        // ---- checks (Sec. III.A) on the touched subsystem
        std::vector<int> cand;
        if (o.schedule == QSIM_SCHED_FORCED) {
            while (fpos < o.nforce && o.force[2 * fpos] == k) cand.push_back(o.force[2 * fpos++ + 1]);
        } else {
            cand = R.subs[si]->qs;
            std::sort(cand.begin(), cand.end());
        }
        const bool mlp_round = o.schedule == QSIM_SCHED_MLP && cand.size() >= 2 &&
                               !(o.fallback_every > 0 && n_ent % o.fallback_every == 0) &&
                               !(o.exhaustive_from > 0 && (int)cand.size() >= o.exhaustive_from);
        // trace rows: features of the candidates before this check round
        std::vector<float> tf;
        if (o.trace_features && o.schedule != QSIM_SCHED_MLP) {
            tf.assign(cand.size() * kFeat, 0.f);
            int msz = (int)R.subs[si]->qs.size();
            for (size_t i = 0; i < cand.size(); i++) features(hist[cand[i]], k, msz, n, p, &tf[i * kFeat]);
        }
        // the decisions of one check round (D) on candidates cand[ci ..]
        auto consume = [&](const Decide &D, size_t ci, int sidx, Sub &Sq) -> qsim_status {
            for (int e = 0; e < D.examined; e++) {
                int qq = cand[ci + e];
                int act = (e == D.first) ? D.action : 0;
                if (!tf.empty()) {
                    if (ntrace < o.trace_cap) {
                        memcpy(o.trace_features + ntrace * kFeat, &tf[(ci + e) * kFeat], sizeof(float) * kFeat);
                        if (o.trace_labels) o.trace_labels[ntrace] = (act == 1);
                    }
                    ntrace++;
                }
                QubitHist &hq = hist[qq];
                hq.r[0] = D.r[e][0];
                hq.r[1] = D.r[e][1];
                hq.r[2] = D.r[e][2];
                hq.g1 = hq.g2 = 0;
                hq.last = k;
                hq.sep = act != 0;
                if (act) {
                    double len = std::sqrt(hq.r[0] * hq.r[0] + hq.r[1] * hq.r[1] + hq.r[2] * hq.r[2]);
                    for (int z = 0; z < 3 && len > 0; z++) hq.r[z] /= len;
                }
                if (o.log && nlog < o.log_cap) {
                    qsim_decision &L = o.log[nlog];
                    L.gate = k;
                    L.qubit = qq;
                    L.action = act;
                    L.reserved = 0;
                    L.eps = D.eps[e];
                    for (int z = 0; z < 3; z++) L.r[z] = D.r[e][z];
                }
                nlog++;
                nchecks++;
            }
            if (D.action == 0) return QSIM_OK;
            double phi[4] = {D.phi[0], D.phi[1], D.phi[2], D.phi[3]};
            int qa = cand[ci + D.first];
            if (D.action == 1) {
                F *= (1.0 - D.eps[D.first]);
                nround++;
            } else {
                nexact++;
            }
            QS_TRY(R.split(sidx, R.local(Sq, qa), phi));
            return QSIM_OK;
        };
        size_t ci = 0;
        if (mlp_round) {
            // score every qubit of the subsystem (up to 64, ascending), let the
            // device keep the top_m predicted to round (logit > 0) and check
            // them: one host synchronisation for the whole round
            std::vector<int> rows_q = cand;
            if (rows_q.size() > 64) rows_q.resize(64);
            const int rows = (int)rows_q.size();
            Sub &S0 = *R.subs[si];
            hfeat.assign((size_t)rows * kFeat, 0.f);
            std::vector<int> loc_all(rows);
            for (int i = 0; i < rows; i++) {
                features(hist[rows_q[i]], k, (int)S0.qs.size(), n, p, &hfeat[(size_t)i * kFeat]);
                loc_all[i] = R.local(S0, rows_q[i]);
            }
            QS_CUDA(cudaMemcpyAsync(d_feat, hfeat.data(), sizeof(float) * hfeat.size(), cudaMemcpyHostToDevice, R.st));
            QS_CUDA(cudaMemcpyAsync(R.d_loc, loc_all.data(), sizeof(int) * rows, cudaMemcpyHostToDevice, R.st));
            QS_TRY(mlp_infer_device(o.mlp, d_feat, rows, d_logit, R.st));
            k_mlp_select<<<1, 1, 0, R.st>>>(d_logit, R.d_loc, rows, o.top_m, R.d_cand, R.d_loc + 64, R.d_dec);
            QS_CUDA(cudaGetLastError());
            int passes = 0;
            QS_TRY(bloch_sums_device(S0.d, R.dt, (int)S0.qs.size(), R.st, R.sc, R.d_loc + 64, R.d_sums, &passes));
            k_decide<<<1, 1, 0, R.st>>>(R.d_sums, R.d_cand, 0, p, tau, R.d_dec, R.d_loc + 64);
            QS_CUDA(cudaGetLastError());
            QS_CUDA(cudaMemcpyAsync(R.h_dec, R.d_dec, sizeof(Decide), cudaMemcpyDeviceToHost, R.st));
            QS_CUDA(cudaStreamSynchronize(R.st));
            const Decide &D = *R.h_dec;
            cand.clear();
            for (int i = 0; i < D.nsel; i++) cand.push_back(rows_q[D.sel[i]]);
            if (D.nsel > 0) {
                R.bloch_passes += passes;
                QS_TRY(consume(D, 0, si, S0));
                ci = D.examined;
            }
        }
        while (ci < cand.size()) {
            // skip candidates whose subsystem is a single qubit now
            int q = cand[ci];
            Sub &Sq = *R.subs[R.sys_of[q]];
            if (Sq.qs.size() < 2) {
                ci++;
                continue;
            }
            int sidx = R.sys_of[q];
            // the run of following candidates in the same subsystem
            std::vector<int> loc;
            size_t cj = ci;
            while (cj < cand.size() && R.sys_of[cand[cj]] == sidx && loc.size() < 64) loc.push_back(R.local(Sq, cand[cj++]));
            int passes = 0;
            QS_TRY(bloch_sums_device(Sq.d, R.dt, (int)Sq.qs.size(), R.st, R.sc, nullptr, R.d_sums, &passes));
            R.bloch_passes += passes;
            QS_CUDA(cudaMemcpyAsync(R.d_cand, loc.data(), sizeof(int) * loc.size(), cudaMemcpyHostToDevice, R.st));
            k_decide<<<1, 1, 0, R.st>>>(R.d_sums, R.d_cand, (int)loc.size(), p, tau, R.d_dec, nullptr);
            QS_CUDA(cudaGetLastError());
            QS_CUDA(cudaMemcpyAsync(R.h_dec, R.d_dec, sizeof(Decide), cudaMemcpyDeviceToHost, R.st));
            QS_CUDA(cudaStreamSynchronize(R.st));
            const Decide &D = *R.h_dec;
            QS_TRY(consume(D, ci, sidx, Sq));
            ci += D.examined;
        }
        // ---- two-qubit-subsystem check of the gate's pair (opts->pairs)
        if (o.pairs && touched.size() == 2) {
            const int qa = touched[0], qb = touched[1];
            const int sp = R.sys_of[qa];
            if (sp == R.sys_of[qb] && R.subs[sp]->qs.size() >= 3) {
                cd rho[4][4], V[4][4];
                double w[4];
                QS_TRY(R.pair_rho(sp, qa, qb, rho));
                herm4_jacobi(rho, w, V);
                const double eps = 1.0 - w[3];
                int act = 0;
                if (p > 0.0 && eps <= p / 2.0) act = 1;
                else if (eps <= tau) act = 2;
                if (o.log && nlog < o.log_cap) {
                    qsim_decision &L = o.log[nlog];
                    L.gate = k;
                    L.qubit = qa;
                    L.action = act;
                    L.reserved = 1 + qb;
                    L.eps = eps;
                    L.r[0] = w[3];
                    L.r[1] = w[2];
                    L.r[2] = w[1];
                }
                nlog++;
                nchecks++;
                if (act) {
                    if (act == 1) {
                        F *= (1.0 - eps);
                        nround++;
                    } else {
                        nexact++;
                    }
                    cd phi[4] = {V[0][3], V[1][3], V[2][3], V[3][3]};
                    QS_TRY(R.split2(sp, qa, qb, phi));
                }
            }
        }
    }
    res->fidelity_model = F;
    res->n_rounds = nround;
    res->n_exact = nexact;
    res->n_checks = nchecks;
    res->n_bloch_passes = R.bloch_passes;
    res->peak_bytes = (int64_t)R.peak;
    res->n_log = nlog;
    res->n_trace = ntrace;
    res->max_subsystem_qubits = maxsub;
    res->n_unobservable = nunobs;
    if (status != QSIM_OK) {
        res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        return status;
    }
    // ---- expand the factors into the full ket (validation, Eq. fid_exact)
    if (o.state_out) {
        std::vector<int> live;
        for (size_t i = 0; i < R.subs.size(); i++)
            if (R.subs[i]) live.push_back((int)i);
        R.budget = 1e300;
        for (size_t j = 1; j < live.size(); j++) QS_TRY(R.compose(live[0], live[j]));
        Sub &A = *R.subs[live[0]];
        std::vector<int> to(n);
        for (int b = 0; b < n; b++) to[b] = A.qs[b];
        void *tmp = nullptr;
        QS_CUDA(cudaMallocAsync(&tmp, A.bytes, R.st));
        QS_CUDA(launch_permute(A.d, tmp, R.dt, n, to.data(), R.st));
        QS_CUDA(cudaMemcpyAsync(o.state_out, tmp, A.bytes, cudaMemcpyDeviceToHost, R.st));
        cudaFreeAsync(tmp, R.st);
    }
    QS_CUDA(cudaStreamSynchronize(R.st));
    res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return QSIM_OK;
}
