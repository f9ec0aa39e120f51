// Per-gate kernels: one HBM pass per gate (the plain baseline path).
//
// Sec. II of arXiv 2304.14969: a gate on k qubits updates every group of
// 2^k amplitudes whose indices differ only in those qubits. Work items are
// numbered densely and expanded to amplitude indices by inserting the
// gate's qubit bits (zeros) at their positions, so no thread idles on an
// index the gate does not touch. Consecutive work items map to consecutive
// amplitudes in every stream, which keeps loads coalesced; complex64 pairs
// are moved as 16-byte vectors when the lowest qubit is untouched.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <cuda_runtime.h>

#include "qsim_internal.h"

namespace qs {

template <typename R> struct Vec2;
template <> struct Vec2<float> { using T = float2; };
template <> struct Vec2<double> { using T = double2; };

template <typename R> struct M2 { R re[4], im[4]; };
template <typename R> struct M4 { R re[16], im[16]; };

__device__ __forceinline__ uint64_t expand_bits(uint64_t w, const InsSpec &ins)
{
#pragma unroll
    for (int j = 0; j < 12; j++) {
        if (j < ins.npos) {
            int p = ins.pos[j];
            uint64_t lo = w & ((1ull << p) - 1);
            w = ((w >> p) << (p + 1)) | lo;
        }
    }
    return w;
}

int num_sms()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 152;
    }
    return sms;
}

int default_grid(uint64_t work, int threads)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 152;
    }
    uint64_t blocks = (work + threads - 1) / threads;
    uint64_t cap = (uint64_t)sms * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

template <typename R>
__device__ __forceinline__ void cmul_acc(R &ore, R &oim, R ure, R uim, R xre, R xim)
{
    ore = fma(ure, xre, ore);
    ore = fma(-uim, xim, ore);
    oim = fma(ure, xim, oim);
    oim = fma(uim, xre, oim);
}

// One-qubit gate. Each work item is one pair (i, i | tbit).
template <typename R>
__global__ void k_gate1(typename Vec2<R>::T *__restrict__ a, uint64_t nwork, InsSpec ins,
                        uint64_t setmask, uint64_t tbit, M2<R> u)
{
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwork; w += stride) {
        uint64_t i0 = expand_bits(w, ins) | setmask, i1 = i0 | tbit;
        auto x = a[i0], y = a[i1];
        R r0 = 0, m0 = 0, r1 = 0, m1 = 0;
        cmul_acc(r0, m0, u.re[0], u.im[0], x.x, x.y);
        cmul_acc(r0, m0, u.re[1], u.im[1], y.x, y.y);
        cmul_acc(r1, m1, u.re[2], u.im[2], x.x, x.y);
        cmul_acc(r1, m1, u.re[3], u.im[3], y.x, y.y);
        x.x = r0; x.y = m0; y.x = r1; y.y = m1;
        a[i0] = x;
        a[i1] = y;
    }
}

// complex64 variant: each work item covers two neighbouring pairs (bit 0 of
// the index is untouched by the gate), moved as float4.
__global__ void k_gate1_c64v(float4 *__restrict__ a4, uint64_t nwork, InsSpec ins, uint64_t setmask,
                             uint64_t tbit, M2<float> u)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    auto apply = [&](float4 x, float4 y, float4 &o0, float4 &o1) {
        o0 = make_float4(0, 0, 0, 0);
        o1 = o0;
        cmul_acc(o0.x, o0.y, u.re[0], u.im[0], x.x, x.y);
        cmul_acc(o0.x, o0.y, u.re[1], u.im[1], y.x, y.y);
        cmul_acc(o0.z, o0.w, u.re[0], u.im[0], x.z, x.w);
        cmul_acc(o0.z, o0.w, u.re[1], u.im[1], y.z, y.w);
        cmul_acc(o1.x, o1.y, u.re[2], u.im[2], x.x, x.y);
        cmul_acc(o1.x, o1.y, u.re[3], u.im[3], y.x, y.y);
        cmul_acc(o1.z, o1.w, u.re[2], u.im[2], x.z, x.w);
        cmul_acc(o1.z, o1.w, u.re[3], u.im[3], y.z, y.w);
    };
    uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // four work items per iteration: eight 16-byte loads in flight per thread
    for (; w + 3 * stride < nwork; w += 4 * stride) {
        uint64_t i0[4];
        float4 x[4], y[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            i0[k] = expand_bits((w + k * stride) << 1, ins) | setmask;
            x[k] = a4[i0[k] >> 1];
            y[k] = a4[(i0[k] | tbit) >> 1];
        }
#pragma unroll
        for (int k = 0; k < 4; k++) {
            float4 o0, o1;
            apply(x[k], y[k], o0, o1);
            a4[i0[k] >> 1] = o0;
            a4[(i0[k] | tbit) >> 1] = o1;
        }
    }
    for (; w < nwork; w += stride) {
        const uint64_t i0 = expand_bits(w << 1, ins) | setmask, i1 = i0 | tbit;
        float4 o0, o1;
        apply(a4[i0 >> 1], a4[i1 >> 1], o0, o1);
        a4[i0 >> 1] = o0;
        a4[i1 >> 1] = o1;
    }
}

// Dense two-qubit gate: each work item is one quad.
template <typename R>
__global__ void k_gate2(typename Vec2<R>::T *__restrict__ a, uint64_t nwork, InsSpec ins, uint64_t b0,
                        uint64_t b1, M4<R> u)
{
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwork; w += stride) {
        uint64_t base = expand_bits(w, ins);
        uint64_t idx[4] = {base, base | b0, base | b1, base | b0 | b1};
        R xr[4], xi[4];
#pragma unroll
        for (int c = 0; c < 4; c++) {
            auto v = a[idx[c]];
            xr[c] = v.x;
            xi[c] = v.y;
        }
#pragma unroll
        for (int r = 0; r < 4; r++) {
            R orr = 0, oi = 0;
#pragma unroll
            for (int c = 0; c < 4; c++) cmul_acc(orr, oi, u.re[r * 4 + c], u.im[r * 4 + c], xr[c], xi[c]);
            typename Vec2<R>::T o;
            o.x = orr;
            o.y = oi;
            a[idx[r]] = o;
        }
    }
}

// Controlled phase: multiplies the amplitudes with both bits set.
template <typename R>
__global__ void k_cphase(typename Vec2<R>::T *__restrict__ a, uint64_t nwork, InsSpec ins, uint64_t both,
                         R cr, R ci)
{
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwork; w += stride) {
        uint64_t i = expand_bits(w, ins) | both;
        auto v = a[i];
        R re = v.x * cr - v.y * ci;
        R im = v.x * ci + v.y * cr;
        v.x = re;
        v.y = im;
        a[i] = v;
    }
}

// complex64, neither qubit is qubit 0: each work item is an adjacent pair
// of affected amplitudes (one 16-byte access), four items in flight; ins
// holds qubit 0 as well as the two qubits.
__global__ void k_cphase_c64v(float4 *__restrict__ a4, uint64_t nwork, InsSpec ins, uint64_t both, float cr,
                              float ci)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    auto rot = [&](float4 v) {
        return make_float4(v.x * cr - v.y * ci, v.x * ci + v.y * cr, v.z * cr - v.w * ci, v.z * ci + v.w * cr);
    };
    uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; w + 3 * stride < nwork; w += 4 * stride) {
        uint64_t i[4];
        float4 v[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            i[k] = (expand_bits(w + k * stride, ins) | both) >> 1;
            v[k] = a4[i[k]];
        }
#pragma unroll
        for (int k = 0; k < 4; k++) a4[i[k]] = rot(v[k]);
    }
    for (; w < nwork; w += stride) {
        const uint64_t i = (expand_bits(w, ins) | both) >> 1;
        a4[i] = rot(a4[i]);
    }
}

template <typename R>
__global__ void k_swap(typename Vec2<R>::T *__restrict__ a, uint64_t nwork, InsSpec ins, uint64_t ba,
                       uint64_t bb)
{
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwork; w += stride) {
        uint64_t i = expand_bits(w, ins);
        auto x = a[i | ba], y = a[i | bb];
        a[i | ba] = y;
        a[i | bb] = x;
    }
}

template <typename R>
__global__ void k_set_basis(typename Vec2<R>::T *__restrict__ a, uint64_t N, uint64_t x)
{
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        typename Vec2<R>::T v;
        v.x = (i == x) ? R(1) : R(0);
        v.y = 0;
        a[i] = v;
    }
}

template <typename R>
__global__ void k_scale(typename Vec2<R>::T *__restrict__ a, uint64_t N, R f)
{
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        auto v = a[i];
        v.x *= f;
        v.y *= f;
        a[i] = v;
    }
}

// dst[perm(i)] = src[i] where bit q of i moves to bit new_of_old[q].
// Qubit permutation (relabel materialised in memory), tiled: a tile is the
// 2^s amplitudes spanned by S = qubits 0..4, the source qubits that move
// to positions 0..4, and further low qubits up to s = min(n, 10). It is
// read with consecutive threads on source qubits 0..4 and written with
// consecutive threads on destination qubits 0..4 (both coalesced) through
// a shared-memory tile whose index e (compressed over S) is stored at
// e ^ ((e >> 5) & 31): conflict-free for reads, and for writes whenever
// the lanes' source bits fold onto distinct low bits (e.g. bit reversal).
struct PermTile {
    int s;               // tile qubits
    int nrest;           // other qubits
    int rest[40];        // their source positions, ascending
    int rest_to[40];     // their destination positions
    uint64_t srcLo[32], srcHi[32];   // source offset of tile index e: low 5 / high bits of e
    uint64_t dstLo[32], dstHi[32];   // destination offset of destination tile index f
    uint16_t eLo[32], eHi[32];       // tile index e of destination tile index f
};

template <typename R>
__global__ void __launch_bounds__(256) k_permute(const typename Vec2<R>::T *__restrict__ src,
                                                 typename Vec2<R>::T *__restrict__ dst, uint64_t ntiles,
                                                 const __grid_constant__ PermTile P)
{
    using V = typename Vec2<R>::T;
    __shared__ V tile[1024];
    __shared__ uint64_t sLo[32], sHi[32], dLo[32], dHi[32];
    __shared__ uint16_t eLo[32], eHi[32];
    if (threadIdx.x < 32) {
        sLo[threadIdx.x] = P.srcLo[threadIdx.x];
        sHi[threadIdx.x] = P.srcHi[threadIdx.x];
        dLo[threadIdx.x] = P.dstLo[threadIdx.x];
        dHi[threadIdx.x] = P.dstHi[threadIdx.x];
        eLo[threadIdx.x] = P.eLo[threadIdx.x];
        eHi[threadIdx.x] = P.eHi[threadIdx.x];
    }
    __syncthreads();
    const uint32_t T = 1u << P.s;
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        uint64_t sb = 0, db = 0;
        for (int i = 0; i < P.nrest; i++)
            if ((t >> i) & 1) {
                sb |= 1ull << P.rest[i];
                db |= 1ull << P.rest_to[i];
            }
        for (uint32_t e = threadIdx.x; e < T; e += blockDim.x)
            tile[e ^ ((e >> 5) & 31)] = src[sb | sLo[e & 31] | sHi[e >> 5]];
        __syncthreads();
        for (uint32_t f = threadIdx.x; f < T; f += blockDim.x) {
            const uint32_t e = eLo[f & 31] | eHi[f >> 5];
            dst[db | dLo[f & 31] | dHi[f >> 5]] = tile[e ^ ((e >> 5) & 31)];
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ launchers

static InsSpec make_ins(std::vector<int> pos)
{
    std::sort(pos.begin(), pos.end());
    InsSpec s;
    s.npos = (int)pos.size();
    for (int j = 0; j < s.npos; j++) s.pos[j] = pos[j];
    return s;
}

template <typename R> static M2<R> to_m2(const cd u[4])
{
    M2<R> m;
    for (int k = 0; k < 4; k++) { m.re[k] = (R)u[k].real(); m.im[k] = (R)u[k].imag(); }
    return m;
}

template <typename R> static M4<R> to_m4(const cd u[16])
{
    M4<R> m;
    for (int k = 0; k < 16; k++) { m.re[k] = (R)u[k].real(); m.im[k] = (R)u[k].imag(); }
    return m;
}

static const int kThreads = 256;

cudaError_t launch_gate1(qsim_state *s, const cd u[4], int t, uint64_t cmask, uint64_t cval)
{
    std::vector<int> pos{t};
    for (int q = 0; q < s->n; q++)
        if (cmask & bit(q)) pos.push_back(q);
    InsSpec ins = make_ins(pos);
    uint64_t nwork = s->N() >> ins.npos;
    bool low_free = (ins.pos[0] != 0);
    if (s->dt == QSIM_C64) {
        if (low_free && nwork >= 2) {
            uint64_t nw = nwork / 2;
            k_gate1_c64v<<<default_grid(nw, kThreads), kThreads, 0, s->stream>>>(
                (float4 *)s->amps, nw, ins, cval, bit(t), to_m2<float>(u));
        } else {
            k_gate1<float><<<default_grid(nwork, kThreads), kThreads, 0, s->stream>>>(
                (float2 *)s->amps, nwork, ins, cval, bit(t), to_m2<float>(u));
        }
    } else {
        k_gate1<double><<<default_grid(nwork, kThreads), kThreads, 0, s->stream>>>(
            (double2 *)s->amps, nwork, ins, cval, bit(t), to_m2<double>(u));
    }
    return cudaGetLastError();
}

cudaError_t launch_gate2(qsim_state *s, const cd u[16], int q0, int q1)
{
    InsSpec ins = make_ins({q0, q1});
    uint64_t nwork = s->N() >> 2;
    if (s->dt == QSIM_C64)
        k_gate2<float><<<default_grid(nwork, kThreads), kThreads, 0, s->stream>>>(
            (float2 *)s->amps, nwork, ins, bit(q0), bit(q1), to_m4<float>(u));
    else
        k_gate2<double><<<default_grid(nwork, kThreads), kThreads, 0, s->stream>>>(
            (double2 *)s->amps, nwork, ins, bit(q0), bit(q1), to_m4<double>(u));
    return cudaGetLastError();
}

cudaError_t launch_cphase(qsim_state *s, int q0, int q1, double theta)
{
    InsSpec ins = make_ins({q0, q1});
    uint64_t nwork = s->N() >> 2;
    double c = std::cos(theta), sn = std::sin(theta);
    if (s->dt == QSIM_C64 && q0 != 0 && q1 != 0 && nwork >= 2) {
        // ins also holds qubit 0 so that work items enumerate pairs (2i, 2i+1)
        InsSpec ins0 = make_ins({0, q0, q1});
        const uint64_t nw = s->N() >> 3;
        k_cphase_c64v<<<default_grid(nw, kThreads), kThreads, 0, s->stream>>>(
            (float4 *)s->amps, nw, ins0, bit(q0) | bit(q1), (float)c, (float)sn);
    } else if (s->dt == QSIM_C64)
        k_cphase<float><<<default_grid(nwork, kThreads), kThreads, 0, s->stream>>>(
            (float2 *)s->amps, nwork, ins, bit(q0) | bit(q1), (float)c, (float)sn);
    else
        k_cphase<double><<<default_grid(nwork, kThreads), kThreads, 0, s->stream>>>(
            (double2 *)s->amps, nwork, ins, bit(q0) | bit(q1), c, sn);
    return cudaGetLastError();
}

cudaError_t launch_swap(qsim_state *s, int q0, int q1)
{
    InsSpec ins = make_ins({q0, q1});
    uint64_t nwork = s->N() >> 2;
    if (s->dt == QSIM_C64)
        k_swap<float><<<default_grid(nwork, kThreads), kThreads, 0, s->stream>>>(
            (float2 *)s->amps, nwork, ins, bit(q0), bit(q1));
    else
        k_swap<double><<<default_grid(nwork, kThreads), kThreads, 0, s->stream>>>(
            (double2 *)s->amps, nwork, ins, bit(q0), bit(q1));
    return cudaGetLastError();
}

cudaError_t launch_set_basis(qsim_state *s, uint64_t x)
{
    uint64_t N = s->N();
    if (s->dt == QSIM_C64)
        k_set_basis<float><<<default_grid(N, kThreads), kThreads, 0, s->stream>>>((float2 *)s->amps, N, x);
    else
        k_set_basis<double><<<default_grid(N, kThreads), kThreads, 0, s->stream>>>((double2 *)s->amps, N, x);
    return cudaGetLastError();
}

cudaError_t launch_scale(void *amps, qsim_dtype dt, uint64_t N, double f, cudaStream_t st)
{
    if (dt == QSIM_C64)
        k_scale<float><<<default_grid(N, kThreads), kThreads, 0, st>>>((float2 *)amps, N, (float)f);
    else
        k_scale<double><<<default_grid(N, kThreads), kThreads, 0, st>>>((double2 *)amps, N, f);
    return cudaGetLastError();
}

cudaError_t launch_permute(const void *src, void *dst, qsim_dtype dt, int n, const int *new_of_old,
                           cudaStream_t st)
{
    // S: qubits 0..4, the source qubits moving to 0..4, then low qubits up to s
    std::vector<int> S;
    auto add = [&](int q) {
        if (q < n && std::find(S.begin(), S.end(), q) == S.end()) S.push_back(q);
    };
    for (int q = 0; q < std::min(n, 5); q++) add(q);
    for (int q = 0; q < n; q++)
        if (new_of_old[q] < 5) add(q);
    const int s = std::min(n, 10);
    for (int q = 0; q < n && (int)S.size() < s; q++) add(q);
    if ((int)S.size() > 10) return cudaErrorInvalidValue;
    std::sort(S.begin(), S.end());
    PermTile P;
    memset(&P, 0, sizeof P);
    P.s = (int)S.size();
    for (int q = 0; q < n; q++)
        if (std::find(S.begin(), S.end(), q) == S.end()) {
            P.rest[P.nrest] = q;
            P.rest_to[P.nrest++] = new_of_old[q];
        }
    // destination tile qubits, ascending; f indexes them
    std::vector<int> D;
    for (int q : S) D.push_back(new_of_old[q]);
    std::sort(D.begin(), D.end());
    auto src_off = [&](uint32_t e) {
        uint64_t o = 0;
        for (int j = 0; j < P.s; j++)
            if ((e >> j) & 1) o |= 1ull << S[j];
        return o;
    };
    auto dst_off = [&](uint32_t f) {
        uint64_t o = 0;
        for (int j = 0; j < P.s; j++)
            if ((f >> j) & 1) o |= 1ull << D[j];
        return o;
    };
    auto e_of_f = [&](uint32_t f) {
        uint32_t e = 0;
        for (int j = 0; j < P.s; j++)
            if ((f >> j) & 1) {
                // destination qubit D[j] holds source qubit S[i] with new_of_old[S[i]] == D[j]
                for (int i = 0; i < P.s; i++)
                    if (new_of_old[S[i]] == D[j]) e |= 1u << i;
            }
        return e;
    };
    for (uint32_t x = 0; x < 32; x++) {
        P.srcLo[x] = src_off(x);
        P.srcHi[x] = src_off(x << 5);
        P.dstLo[x] = dst_off(x);
        P.dstHi[x] = dst_off(x << 5);
        P.eLo[x] = (uint16_t)e_of_f(x);
        P.eHi[x] = (uint16_t)e_of_f(x << 5);
    }
    const uint64_t ntiles = 1ull << (n - P.s);
    const int grid = (int)std::min<uint64_t>(ntiles, (uint64_t)num_sms() * 8);
    if (dt == QSIM_C64)
        k_permute<float><<<grid, 256, 0, st>>>((const float2 *)src, (float2 *)dst, ntiles, P);
    else
        k_permute<double><<<grid, 256, 0, st>>>((const double2 *)src, (double2 *)dst, ntiles, P);
    return cudaGetLastError();
}

}  // namespace qs
