// FP64 reductions over a ket: norm, P(q = 1), inner product, Bloch vectors,
// probabilities.
//
// Sec. III.A (arXiv 2304.14969) needs the reduced one-qubit state rho_q of
// each checked qubit, i.e. r = (<X_q>, <Y_q>, <Z_q>), and a normalised ket;
// Eq. (fid_exact) needs <psi_approx|psi_exact>. All cross-element sums are
// carried in FP64. For complex64 kets each thread first sums runs of 8
// terms in FP32 (the products of FP32 amplitudes are FP32 numbers anyway)
// and adds each run to an FP64 accumulator; this keeps the FP64 pipe, which
// is narrow on this part, off the critical path while the sum itself stays
// FP64. complex128 kets are summed in FP64 throughout.
//
// Each kernel writes one row of M partial sums per CTA; a one-CTA kernel
// adds the rows in FP64 and the result is copied to pinned host memory.
#include <algorithm>
#include <cuda_runtime.h>

#include "qsim_internal.h"

namespace qs {

static const int kRedThreads = 256;
static const int kMaxRedBlocks = 152 * 8;

template <typename R> struct V2T;
template <> struct V2T<float> { using T = float2; };
template <> struct V2T<double> { using T = double2; };

template <int M>
__device__ __forceinline__ void block_write(double (&acc)[M], double *__restrict__ partial)
{
    __shared__ double sh[M][kRedThreads / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int m = 0; m < M; m++) {
        double v = acc[m];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sh[m][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < M) {
        double v = 0;
        for (int w = 0; w < kRedThreads / 32; w++) v += sh[threadIdx.x][w];
        partial[(size_t)blockIdx.x * M + threadIdx.x] = v;
    }
}

template <int M>
__global__ void __launch_bounds__(256) k_red_final(const double *__restrict__ partial, int rows,
                                                   double *__restrict__ out)
{
    // one CTA of 256 threads; warp w adds the columns m = w, w + 8, ...: each
    // lane adds every 32nd row, then a warp-shuffle tree adds the 32 lanes
    // (FP64; no block-wide barrier, so the columns proceed in parallel)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int m = warp; m < M; m += nw) {
        double v = 0;
        for (int r = lane; r < rows; r += 32) v += partial[(size_t)r * M + m];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) out[m] = v;
    }
}

// ---- norm: sum |psi_i|^2
template <typename R>
__global__ void k_red_norm(const typename V2T<R>::T *__restrict__ a, uint64_t N, double *partial)
{
    double acc[1] = {0};
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
    if constexpr (sizeof(R) == 4) {
        // 16-byte loads, consecutive lanes on consecutive amplitude pairs;
        // runs of 8 terms in FP32 (four loads in flight per thread)
        const float4 *a4 = (const float4 *)a;
        const uint64_t N4 = N / 2;
        uint64_t i = tid;
        for (; i + 3 * nt < N4; i += 4 * nt) {
            float4 v[4];
#pragma unroll
            for (int j = 0; j < 4; j++) v[j] = a4[i + j * nt];
            float run = 0;
#pragma unroll
            for (int j = 0; j < 4; j++) {
                run = fmaf(v[j].x, v[j].x, run);
                run = fmaf(v[j].y, v[j].y, run);
                run = fmaf(v[j].z, v[j].z, run);
                run = fmaf(v[j].w, v[j].w, run);
            }
            acc[0] += (double)run;
        }
        for (; i < N4; i += nt) {
            const float4 v = a4[i];
            acc[0] += (double)(v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w);
        }
        if ((N & 1) && tid == 0) {
            const auto v = a[N - 1];
            acc[0] += (double)v.x * v.x + (double)v.y * v.y;
        }
    } else {
        for (uint64_t i = tid; i < N; i += nt) {
            const auto v = a[i];
            acc[0] += v.x * v.x + v.y * v.y;
        }
    }
    block_write<1>(acc, partial);
}

// ---- P(q = 1): partial[0] = sum over bit q = 1, partial[1] = total.
// complex64: 16-byte loads (amplitude pairs 2i, 2i+1), consecutive lanes on
// consecutive pairs, four loads in flight; runs of 8 terms in FP32.
template <typename R>
__global__ void k_red_prob1(const typename V2T<R>::T *__restrict__ a, uint64_t N, uint64_t qb, double *partial)
{
    double acc[2] = {0, 0};
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
    if constexpr (sizeof(R) == 4) {
        const float4 *a4 = (const float4 *)a;
        const uint64_t N4 = N / 2;
        uint64_t i = tid;
        for (; i + 3 * nt < N4; i += 4 * nt) {
            float4 v[4];
#pragma unroll
            for (int j = 0; j < 4; j++) v[j] = a4[i + j * nt];
            float one = 0.f, all = 0.f;
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const uint64_t e = 2 * (i + j * nt);
                const float p0 = v[j].x * v[j].x + v[j].y * v[j].y, p1 = v[j].z * v[j].z + v[j].w * v[j].w;
                all += p0 + p1;
                one += ((e & qb) ? p0 : 0.f) + (((e + 1) & qb) ? p1 : 0.f);
            }
            acc[0] += (double)one;
            acc[1] += (double)all;
        }
        for (; i < N4; i += nt) {
            const float4 v = a4[i];
            const uint64_t e = 2 * i;
            const float p0 = v.x * v.x + v.y * v.y, p1 = v.z * v.z + v.w * v.w;
            acc[1] += (double)(p0 + p1);
            acc[0] += (double)(((e & qb) ? p0 : 0.f) + (((e + 1) & qb) ? p1 : 0.f));
        }
        if ((N & 1) && tid == 0) {
            const auto v = a[N - 1];
            const double p = (double)v.x * v.x + (double)v.y * v.y;
            acc[1] += p;
            if ((N - 1) & qb) acc[0] += p;
        }
    } else {
        for (uint64_t i = tid; i < N; i += nt) {
            const auto v = a[i];
            const double p = v.x * v.x + v.y * v.y;
            acc[1] += p;
            if (i & qb) acc[0] += p;
        }
    }
    block_write<2>(acc, partial);
}

// ---- <a|b> = sum conj(a_i) b_i (complex64: as above, two streams)
template <typename R>
__global__ void k_red_inner(const typename V2T<R>::T *__restrict__ a, const typename V2T<R>::T *__restrict__ b,
                            uint64_t N, double *partial)
{
    double acc[2] = {0, 0};
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
    if constexpr (sizeof(R) == 4) {
        const float4 *a4 = (const float4 *)a, *b4 = (const float4 *)b;
        const uint64_t N4 = N / 2;
        uint64_t i = tid;
        for (; i + 1 * nt < N4; i += 2 * nt) {
            float4 x[2], y[2];
#pragma unroll
            for (int j = 0; j < 2; j++) {
                x[j] = a4[i + j * nt];
                y[j] = b4[i + j * nt];
            }
            float re = 0.f, im = 0.f;
#pragma unroll
            for (int j = 0; j < 2; j++) {
                re = fmaf(x[j].x, y[j].x, fmaf(x[j].y, y[j].y, re));
                re = fmaf(x[j].z, y[j].z, fmaf(x[j].w, y[j].w, re));
                im = fmaf(x[j].x, y[j].y, fmaf(-x[j].y, y[j].x, im));
                im = fmaf(x[j].z, y[j].w, fmaf(-x[j].w, y[j].z, im));
            }
            acc[0] += (double)re;
            acc[1] += (double)im;
        }
        for (; i < N4; i += nt) {
            const float4 x = a4[i], y = b4[i];
            acc[0] += (double)(x.x * y.x + x.y * y.y + x.z * y.z + x.w * y.w);
            acc[1] += (double)(x.x * y.y - x.y * y.x + x.z * y.w - x.w * y.z);
        }
        if ((N & 1) && tid == 0) {
            const auto x = a[N - 1], y = b[N - 1];
            acc[0] += (double)x.x * y.x + (double)x.y * y.y;
            acc[1] += (double)x.x * y.y - (double)x.y * y.x;
        }
    } else {
        for (uint64_t i = tid; i < N; i += nt) {
            const auto x = a[i], y = b[i];
            acc[0] += x.x * y.x + x.y * y.y;
            acc[1] += x.x * y.y - x.y * y.x;
        }
    }
    block_write<2>(acc, partial);
}

// ---- Bloch sums of one qubit over pairs (a = bit 0, b = bit 1):
// partial = [sum |a|^2, sum |b|^2, Re sum conj(a) b, Im sum conj(a) b]
template <typename R>
__global__ void k_red_bloch(const typename V2T<R>::T *__restrict__ a, uint64_t npairs, int q, double *partial)
{
    double acc[4] = {0, 0, 0, 0};
    uint64_t qb = 1ull << q, lomask = qb - 1;
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x * 4;
    for (uint64_t base = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4; base < npairs; base += stride) {
        R s0 = 0, s1 = 0, sr = 0, si = 0;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            uint64_t w = base + j;
            if (w < npairs) {
                uint64_t i0 = ((w & ~lomask) << 1) | (w & lomask);
                auto x = a[i0];
                auto y = a[i0 | qb];
                s0 = fma(x.x, x.x, fma(x.y, x.y, s0));
                s1 = fma(y.x, y.x, fma(y.y, y.y, s1));
                sr = fma(x.x, y.x, fma(x.y, y.y, sr));
                si = fma(x.x, y.y, fma(-x.y, y.x, si));
            }
        }
        acc[0] += (double)s0;
        acc[1] += (double)s1;
        acc[2] += (double)sr;
        acc[3] += (double)si;
    }
    block_write<4>(acc, partial);
}

// ---- Bloch sums of several qubits in one pass. Each CTA iteration stages a
// tile of 2^t amplitudes whose index bits are the physical qubits tq[0..t-1]
// (tq[0..c-1] = 0..c-1, so every tile row is a contiguous run), then for
// each tile qubit j accumulates [sum_{bit 1} |psi|^2, Re S_j, Im S_j] and, for
// j == 0 only, the total sum |psi|^2. Output row per CTA: 1 + 3t doubles.
static const int kTileRow = 1 + 3 * 16;   // partial row of the tiled Bloch pass

struct TileSpec {
    int n, t, c;
    int tq[16];       // tile qubits, tq[0..c-1] = 0..c-1, rest ascending
    InsSpec ins;      // high tile qubits to insert when expanding a tile id
    uint32_t wmask;   // tile qubits whose sums this pass reports
};

__device__ __forceinline__ uint64_t tile_expand(uint64_t w, const InsSpec &ins)
{
    for (int j = 0; j < ins.npos; j++) {
        int p = ins.pos[j];
        uint64_t lo = w & ((1ull << p) - 1);
        w = ((w >> p) << (p + 1)) | lo;
    }
    return w;
}

// End of a tiled Bloch pass, called by every thread of every CTA after the
// CTA's partial row (kTileRow doubles, ncol of them used) is written: the
// last CTA to finish (ticket, which wraps back to 0 with it) adds the rows in
// FP64 and writes [sum_{bit0}|psi|^2, sum_{bit1}|psi|^2, Re S, Im S] of qubit
// tq[j] at out[4 tq[j]] for every tile qubit j the pass reports (ts.wmask).
__device__ __forceinline__ void bloch_last_cta(const double *partial, int ncol, const TileSpec &ts,
                                               double *__restrict__ out, unsigned *__restrict__ ticket)
{
    __shared__ unsigned s_last;
    __shared__ double comb[kTileRow];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicInc(ticket, gridDim.x - 1) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int m = warp; m < ncol; m += nw) {
        double x = 0;
        for (int r = lane; r < (int)gridDim.x; r += 32) x += __ldcg(&partial[(size_t)r * kTileRow + m]);
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) comb[m] = x;
    }
    __syncthreads();
    const int j = threadIdx.x;
    if (j < ts.t && ((ts.wmask >> j) & 1)) {
        const int q = ts.tq[j];
        const double total = comb[0], one = comb[1 + 3 * j];
        out[4 * q + 0] = total - one;
        out[4 * q + 1] = one;
        out[4 * q + 2] = comb[2 + 3 * j];
        out[4 * q + 3] = comb[3 + 3 * j];
    }
}

template <typename R>
__global__ void k_red_bloch_tile(const typename V2T<R>::T *__restrict__ a, TileSpec ts, double *partial,
                                 const int *__restrict__ gate, double *__restrict__ out, unsigned *__restrict__ ticket)
{
    if (gate && *gate == 0) return;   // nothing to check (the sums are not read)
    extern __shared__ __align__(16) unsigned char smraw[];
    typename V2T<R>::T *tile = (typename V2T<R>::T *)smraw;
    const int t = ts.t, c = ts.c;
    const uint64_t T = 1ull << t, runlen = 1ull << c;
    const uint64_t ntiles = 1ull << (ts.n - t);
    __shared__ double bacc[kTileRow];
    for (int m = threadIdx.x; m < kTileRow; m += blockDim.x) bacc[m] = 0;
    double tot = 0;

    for (uint64_t tid = blockIdx.x; tid < ntiles; tid += gridDim.x) {
        // tile base: insert zeros at the high tile qubits, after the low c bits
        uint64_t base = tile_expand(tid << c, ts.ins);
        __syncthreads();
        for (uint64_t e = threadIdx.x; e < T; e += blockDim.x) {
            uint64_t run = e >> c, off = e & (runlen - 1);
            uint64_t idx = base | off;
            for (int j = c; j < t; j++)
                if ((run >> (j - c)) & 1) idx |= 1ull << ts.tq[j];
            tile[e] = a[idx];
        }
        __syncthreads();
        // total |psi|^2
        {
            R run = 0;
            for (uint64_t e = threadIdx.x; e < T; e += blockDim.x) {
                auto v = tile[e];
                run = fma(v.x, v.x, fma(v.y, v.y, run));
            }
            tot += (double)run;
        }
        for (int j = 0; j < t; j++) {
            R s1 = 0, sr = 0, si = 0;
            uint64_t jb = 1ull << j, lom = jb - 1;
            for (uint64_t w = threadIdx.x; w < T / 2; w += blockDim.x) {
                uint64_t e0 = ((w & ~lom) << 1) | (w & lom);
                auto x = tile[e0];
                auto y = tile[e0 | jb];
                s1 = fma(y.x, y.x, fma(y.y, y.y, s1));
                sr = fma(x.x, y.x, fma(x.y, y.y, sr));
                si = fma(x.x, y.y, fma(-x.y, y.x, si));
            }
            double d1 = s1, dr = sr, di = si;
            for (int o = 16; o > 0; o >>= 1) {
                d1 += __shfl_down_sync(0xffffffffu, d1, o);
                dr += __shfl_down_sync(0xffffffffu, dr, o);
                di += __shfl_down_sync(0xffffffffu, di, o);
            }
            if ((threadIdx.x & 31) == 0) {
                atomicAdd(&bacc[1 + 3 * j], d1);
                atomicAdd(&bacc[2 + 3 * j], dr);
                atomicAdd(&bacc[3 + 3 * j], di);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_down_sync(0xffffffffu, tot, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&bacc[0], tot);
    __syncthreads();
    for (int m = threadIdx.x; m < kTileRow; m += blockDim.x) partial[(size_t)blockIdx.x * kTileRow + m] = bacc[m];
    bloch_last_cta(partial, 1 + 3 * t, ts, out, ticket);
}

// Compensated accumulator: FP32 (hi, lo) pair kept with TwoSum (Knuth), so
// that thousands of per-tile runs add up to near-FP64 accuracy without the
// FP64 pipe; FP64 for complex128 kets.
template <typename R> struct CAcc;
template <> struct CAcc<float> {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        const float s = hi + x, bp = s - hi;
        lo += (hi - (s - bp)) + (x - bp);
        hi = s;
    }
    __device__ __forceinline__ double get() const { return (double)hi + (double)lo; }
};
template <> struct CAcc<double> {
    double hi = 0.0;
    __device__ __forceinline__ void add(double x) { hi += x; }
    __device__ __forceinline__ double get() const { return hi; }
};

// A pair of values of the ket's precision handled together: for FP32 one
// 64-bit register pair and the packed FP32x2 instructions (one instruction
// for two multiply-adds), for FP64 two scalars.
struct PkF {
    unsigned long long u;
};
struct PkD {
    double x, y;
};
template <typename R> struct PkT;
template <> struct PkT<float> { using T = PkF; };
template <> struct PkT<double> { using T = PkD; };

__device__ __forceinline__ PkF pk(float a, float b)
{
    PkF r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.u) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ PkD pk(double a, double b) { return PkD{a, b}; }
__device__ __forceinline__ float2 upk(PkF p)
{
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(p.u));
    return make_float2(a, b);
}
__device__ __forceinline__ double2 upk(PkD p) { return make_double2(p.x, p.y); }
__device__ __forceinline__ PkF fma2(PkF a, PkF b, PkF c)
{
    PkF r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.u) : "l"(a.u), "l"(b.u), "l"(c.u));
    return r;
}
__device__ __forceinline__ PkD fma2(PkD a, PkD b, PkD c) { return PkD{fma(a.x, b.x, c.x), fma(a.y, b.y, c.y)}; }
__device__ __forceinline__ PkF add2(PkF a, PkF b)
{
    PkF r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.u) : "l"(a.u), "l"(b.u));
    return r;
}
__device__ __forceinline__ PkD add2(PkD a, PkD b) { return PkD{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ PkF sub2(PkF a, PkF b)
{
    PkF r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.u) : "l"(a.u), "l"(b.u));
    return r;
}
__device__ __forceinline__ PkD sub2(PkD a, PkD b) { return PkD{a.x - b.x, a.y - b.y}; }

// CAcc for a pair: TwoSum on both halves at once (FP32x2), plain FP64 sums
// for complex128 kets.
template <typename R> struct CAcc2;
template <> struct CAcc2<float> {
    PkF hi = pk(0.f, 0.f), lo = pk(0.f, 0.f);
    __device__ __forceinline__ void add(PkF x)
    {
        const PkF s = add2(hi, x), bp = sub2(s, hi);
        lo = add2(lo, add2(sub2(hi, sub2(s, bp)), sub2(x, bp)));
        hi = s;
    }
    __device__ __forceinline__ double2 get() const
    {
        const float2 h = upk(hi), l = upk(lo);
        return make_double2((double)h.x + (double)l.x, (double)h.y + (double)l.y);
    }
};
template <> struct CAcc2<double> {
    PkD hi = PkD{0.0, 0.0};
    __device__ __forceinline__ void add(PkD x) { hi = add2(hi, x); }
    __device__ __forceinline__ double2 get() const { return upk(hi); }
};

// Bloch sums of the 12 tile qubits of every tile (t = 12, c = 4: tile qubits
// 0..3 and eight high ones), same partial-row format as k_red_bloch_tile.
//
// Tiles stream through a ring of kBlochStages shared-memory stages filled by
// 16-byte cp.async copies, so kBlochStages - 1 tiles are in flight while one
// is summed and registers hold only the accumulators and one slice of 16
// amplitudes. A stage keeps a tile as 256 runs of 16 consecutive amplitudes
// (tile bits 0..3); run r sits at byte r * (16 B + 16): the 16-byte pad
// staggers the runs across the shared-memory banks, which makes the copies
// and the three read patterns below free of bank conflicts. The copies of a
// warp cover whole runs (one 128- or 256-byte line each).
//
// Thread th then takes three slices of 16 amplitudes: its own run (register
// bits = tile bits 0..3, tile bits 4..11 = th), then those with register
// bits = tile bits 4..7 and 8..11. Each slice gives, for its four tile
// qubits, S = sum over bit = 0 of conj(psi_i) psi_{i + 2^q}, in runs of 8
// terms in the ket's precision added into compensated accumulators. The
// first slice also gives the run total |psi|^2 and, for LOW, the sums over
// bit = 1 of |psi|^2 of the tile qubits 0..3. That sum for a high tile qubit
// 4 + b is the sum of the run totals of the threads whose bit b is set, so
// it is formed once, in the block reduction. LOW = false skips the low
// qubits (an earlier pass over the same ket has them). Each CTA writes one
// partial row; the last CTA to finish adds the rows and writes the sums of
// the qubits the pass reports.
static const int kBlochStages = 3;

template <typename R>
struct BlochGeom {
    static constexpr int kB = 2 * (int)sizeof(R);   // bytes per amplitude
    static constexpr int kRun = 16 * kB;             // bytes of a run
    static constexpr int kRunPad = kRun + 16;        // stage stride of a run
    static constexpr int kStage = 256 * kRunPad;     // bytes of a stage
    static constexpr int kGran = kRun / 16;          // 16-byte granules per run
    static constexpr int kSmem = kBlochStages * kStage;
};

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <typename R, bool LOW>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 2 : 1)
    k_red_bloch_pipe(const typename V2T<R>::T *__restrict__ a, const __grid_constant__ TileSpec ts,
                     double *partial, const int *__restrict__ gate, double *__restrict__ out,
                     unsigned *__restrict__ ticket)
{
    if (gate && *gate == 0) return;   // nothing to check (the sums are not read)
    using V = typename V2T<R>::T;
    using G = BlochGeom<R>;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ uint64_t hh[16];   // ket offset of the run-index bits above the ones a thread fixes
    const int th = threadIdx.x, lane = th & 31, warp = th >> 5;
    // copy k of thread th moves granule th % kGran of run k * (256 / kGran) + th / kGran
    constexpr int kLoBits = G::kGran == 8 ? 5 : 4;   // run-index bits fixed by th
    if (th < G::kGran) {
        uint64_t h = 0;
        for (int b = 0; b < 8 - kLoBits; b++)
            if ((th >> b) & 1) h |= 1ull << ts.tq[4 + kLoBits + b];
        hh[th] = h * (uint64_t)G::kB;
    }
    uint64_t hlo = 0;
    for (int b = 0; b < kLoBits; b++)
        if (((th / G::kGran) >> b) & 1) hlo |= 1ull << ts.tq[4 + b];
    const unsigned char *src0 = (const unsigned char *)a + hlo * G::kB + (th % G::kGran) * 16;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smraw);
    const uint32_t dst0 = sbase + (th / G::kGran) * G::kRunPad + (th % G::kGran) * 16;
    constexpr uint32_t kDstStep = (256 / G::kGran) * G::kRunPad;
    __syncthreads();

    const uint64_t ntiles = 1ull << (ts.n - 12);
    const uint64_t cnt = ntiles > blockIdx.x ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    // ket index of the next tile to issue: the tile id's bits deposited into the
    // non-tile bit positions (nonTile); the next id of this CTA is gridDim.x on,
    // added with carries running through the tile positions (set to one)
    uint64_t nonTile = ((1ull << ts.n) - 1) & ~0xfull;
    for (int j = 0; j < 8; j++) nonTile &= ~(1ull << ts.tq[4 + j]);
    const uint64_t step = tile_expand((uint64_t)gridDim.x << 4, ts.ins);
    uint64_t nextBase = tile_expand((uint64_t)blockIdx.x << 4, ts.ins);
    auto issue = [&](uint64_t i) {
        const uint64_t base = nextBase * G::kB;
        nextBase = ((nextBase | ~nonTile) + step) & nonTile;
        const uint32_t d = dst0 + (uint32_t)(i % kBlochStages) * G::kStage;
#pragma unroll
        for (int k = 0; k < G::kGran; k++) cp_async16(d + k * kDstStep, src0 + base + hh[k]);
    };
#pragma unroll
    for (int s = 0; s < kBlochStages - 1; s++) {
        if (s < cnt) issue(s);
        cp_async_commit();
    }

    using P = typename PkT<R>::T;
    CAcc<R> aT;                       // run totals
    CAcc<R> aS1[LOW ? 4 : 1];         // sum over bit = 1 of |psi|^2, tile qubits 0..3
    CAcc2<R> aS[LOW ? 12 : 8];        // (Re S, Im S) of tile qubit j (index j - 4 without LOW)
    constexpr int kOff = LOW ? 0 : 4;
    // without LOW the run sums of an even tile are held and added together with
    // the next tile's (runs of 16 terms), which halves the compensated adds
    P hS[LOW ? 1 : 8];
    bool hold = false, paired = false;
    V v[16];
    // S_j = sum over pairs of conj(x) y = (x.x y.x + x.y y.y) + i (x.x y.y - x.y y.x):
    // two packed products per pair, x (.) y and x (.) (y.y, y.x), split at the end
    auto pair_sums = [&](int j0) {
        P ys[16];
#pragma unroll
        for (int r = 1; r < 16; r++) ys[r] = pk(v[r].y, v[r].x);
#pragma unroll
        for (int j = 0; j < 4; j++) {
            P q1 = pk((R)0, (R)0), q2 = pk((R)0, (R)0);
#pragma unroll
            for (int r = 0; r < 16; r++) {
                if (r & (1 << j)) continue;
                const P x = pk(v[r].x, v[r].y), y = pk(v[r | (1 << j)].x, v[r | (1 << j)].y);
                q1 = fma2(x, y, q1);
                q2 = fma2(x, ys[r | (1 << j)], q2);
            }
            const auto a1 = upk(q1), a2 = upk(q2);
            const P sri = pk(a1.x + a1.y, a2.x - a2.y);
            const int k = j0 + j - kOff;
            if constexpr (LOW) {
                aS[k].add(sri);
            } else if (hold) {
                hS[k] = sri;
            } else {
                aS[k].add(paired ? add2(hS[k], sri) : sri);
            }
        }
    };
    const uint32_t offA = (uint32_t)th * G::kRunPad;
    const uint32_t offB = (uint32_t)(th >> 4) * 16 * G::kRunPad + (th & 15) * G::kB;
    const uint32_t offC = (uint32_t)(th >> 4) * G::kRunPad + (th & 15) * G::kB;

    for (uint64_t i = 0; i < cnt; i++) {
        cp_async_wait<kBlochStages - 2>();   // this thread's copies of tile i have landed
        __syncthreads();                     // everyone's have, and tile i - 1 is read
        if (i + kBlochStages - 1 < cnt) issue(i + kBlochStages - 1);
        cp_async_commit();
        const unsigned char *st = smraw + (size_t)(i % kBlochStages) * G::kStage;
        hold = !(i & 1) && i + 1 < cnt;
        paired = (i & 1);
        // slice 1: own run
        if constexpr (sizeof(R) == 4) {
#pragma unroll
            for (int g = 0; g < 8; g++) {
                const float4 w = *(const float4 *)(st + offA + g * 16);
                v[2 * g] = make_float2(w.x, w.y);
                v[2 * g + 1] = make_float2(w.z, w.w);
            }
        } else {
#pragma unroll
            for (int r = 0; r < 16; r++) v[r] = *(const V *)(st + offA + r * 16);
        }
        {
            if constexpr (LOW) {
                R p[16];
#pragma unroll
                for (int r = 0; r < 16; r++) p[r] = fma(v[r].x, v[r].x, v[r].y * v[r].y);
                R tot = 0;
#pragma unroll
                for (int r = 0; r < 16; r++) tot += p[r];
                aT.add(tot);
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    R s1 = 0;
#pragma unroll
                    for (int r = 0; r < 16; r++)
                        if (r & (1 << j)) s1 += p[r];
                    aS1[j].add(s1);
                }
            } else {
                P t2 = pk((R)0, (R)0);
#pragma unroll
                for (int r = 0; r < 16; r++) {
                    const P x = pk(v[r].x, v[r].y);
                    t2 = fma2(x, x, t2);
                }
                const auto tt = upk(t2);
                aT.add(tt.x + tt.y);
            }
        }
        if constexpr (LOW) pair_sums(0);
        // slice 2: register bits = tile bits 4..7
#pragma unroll
        for (int r = 0; r < 16; r++) v[r] = *(const V *)(st + offB + r * G::kRunPad);
        pair_sums(4);
        // slice 3: register bits = tile bits 8..11
#pragma unroll
        for (int r = 0; r < 16; r++) v[r] = *(const V *)(st + offC + r * 16 * G::kRunPad);
        pair_sums(8);
    }
    cp_async_wait<0>();
    __syncthreads();   // the stages are free: the block reduction uses them

    // block reduction (FP64) into this CTA's partial row
    double *red = (double *)smraw;   // [8 warps][kTileRow]
    const double tot = aT.get();
    auto put = [&](int m, double x) {
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[warp * kTileRow + m] = x;
    };
    put(0, tot);
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const double2 sj = LOW ? aS[LOW ? j : 0].get() : make_double2(0.0, 0.0);
        put(1 + 3 * j, LOW ? aS1[LOW ? j : 0].get() : 0.0);
        put(2 + 3 * j, sj.x);
        put(3 + 3 * j, sj.y);
    }
#pragma unroll
    for (int j = 4; j < 12; j++) {
        const double2 sj = aS[j - kOff].get();
        put(1 + 3 * j, ((th >> (j - 4)) & 1) ? tot : 0.0);
        put(2 + 3 * j, sj.x);
        put(3 + 3 * j, sj.y);
    }
    __syncthreads();
    for (int m = th; m < kTileRow; m += blockDim.x) {
        double x = 0;
        if (m < 37)
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) x += red[w * kTileRow + m];
        partial[(size_t)blockIdx.x * kTileRow + m] = x;
    }

    bloch_last_cta(partial, 37, ts, out, ticket);
}

template <typename R>
__global__ void k_probs(const typename V2T<R>::T *__restrict__ a, uint64_t N, double *__restrict__ out)
{
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        auto v = a[i];
        double re = v.x, im = v.y;
        out[i] = re * re + im * im;
    }
}

// ------------------------------------------------------------- host side

qsim_status ensure_scratch(Scratch &sc, size_t doubles)
{
    if (sc.cap >= doubles) return QSIM_OK;
    free_scratch(sc);
    // one more slot past the capacity holds the tiled Bloch pass's ticket,
    // which no other user of the scratch writes; it starts at 0
    QS_CUDA(cudaMalloc(&sc.d, (doubles + 1) * sizeof(double)));
    QS_CUDA(cudaMallocHost(&sc.h, 64 * sizeof(double)));
    const double zero = 0.0;
    QS_CUDA(cudaMemcpy(sc.d + doubles, &zero, sizeof(double), cudaMemcpyHostToDevice));
    sc.cap = doubles;
    return QSIM_OK;
}

void free_scratch(Scratch &sc)
{
    if (sc.d) cudaFree(sc.d);
    if (sc.h) cudaFreeHost(sc.h);
    sc.d = nullptr;
    sc.h = nullptr;
    sc.cap = 0;
}

static int red_blocks(uint64_t items)
{
    uint64_t b = (items + kRedThreads - 1) / kRedThreads;
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(b, kMaxRedBlocks));
}

// Final FP64 combine of `rows` x M partials into red.h[0..M-1] (syncs).
template <int M>
static qsim_status finish(qsim_state *s, int rows)
{
    double *dout = s->red.d + (size_t)kMaxRedBlocks * 64;
    k_red_final<M><<<1, 256, 0, s->stream>>>(s->red.d, rows, dout);
    QS_CUDA(cudaGetLastError());
    QS_CUDA(cudaMemcpyAsync(s->red.h, dout, M * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    err_fetch(s);
    QS_CUDA(cudaStreamSynchronize(s->stream));
    return err_check(s);
}

static qsim_status ensure_red(qsim_state *s)
{
    return ensure_scratch(s->red, (size_t)kMaxRedBlocks * 64 + 64);
}

qsim_status reduce_norm(qsim_state *s, double *out)
{
    QS_TRY(ensure_red(s));
    uint64_t N = s->N();
    int blocks = red_blocks((N + 7) / 8);
    if (s->dt == QSIM_C64)
        k_red_norm<float><<<blocks, kRedThreads, 0, s->stream>>>((const float2 *)s->amps, N, s->red.d);
    else
        k_red_norm<double><<<blocks, kRedThreads, 0, s->stream>>>((const double2 *)s->amps, N, s->red.d);
    QS_CUDA(cudaGetLastError());
    QS_TRY(finish<1>(s, blocks));
    *out = s->red.h[0];
    return QSIM_OK;
}

qsim_status reduce_prob1(qsim_state *s, int q, double *p1, double *total)
{
    QS_TRY(ensure_red(s));
    uint64_t N = s->N();
    int blocks = red_blocks((N + 7) / 8);
    if (s->dt == QSIM_C64)
        k_red_prob1<float><<<blocks, kRedThreads, 0, s->stream>>>((const float2 *)s->amps, N, bit(q), s->red.d);
    else
        k_red_prob1<double><<<blocks, kRedThreads, 0, s->stream>>>((const double2 *)s->amps, N, bit(q), s->red.d);
    QS_CUDA(cudaGetLastError());
    QS_TRY(finish<2>(s, blocks));
    *p1 = s->red.h[0];
    *total = s->red.h[1];
    return QSIM_OK;
}

qsim_status reduce_inner(qsim_state *a, qsim_state *b, double out[2])
{
    QS_TRY(ensure_red(a));
    uint64_t N = a->N();
    int blocks = red_blocks((N + 7) / 8);
    if (a->stream != b->stream) QS_CUDA(cudaStreamSynchronize(b->stream));
    if (a->dt == QSIM_C64)
        k_red_inner<float><<<blocks, kRedThreads, 0, a->stream>>>((const float2 *)a->amps, (const float2 *)b->amps, N,
                                                                  a->red.d);
    else
        k_red_inner<double><<<blocks, kRedThreads, 0, a->stream>>>((const double2 *)a->amps,
                                                                   (const double2 *)b->amps, N, a->red.d);
    QS_CUDA(cudaGetLastError());
    QS_TRY(finish<2>(a, blocks));
    out[0] = a->red.h[0];
    out[1] = a->red.h[1];
    return QSIM_OK;
}

qsim_status reduce_bloch(qsim_state *s, int q, double out4[4])
{
    QS_TRY(ensure_red(s));
    uint64_t np = s->N() / 2;
    int blocks = red_blocks((np + 3) / 4);
    if (s->dt == QSIM_C64)
        k_red_bloch<float><<<blocks, kRedThreads, 0, s->stream>>>((const float2 *)s->amps, np, q, s->red.d);
    else
        k_red_bloch<double><<<blocks, kRedThreads, 0, s->stream>>>((const double2 *)s->amps, np, q, s->red.d);
    QS_CUDA(cudaGetLastError());
    QS_TRY(finish<4>(s, blocks));
    for (int k = 0; k < 4; k++) out4[k] = s->red.h[k];
    return QSIM_OK;
}

// Bloch sums of all n qubits of a ket into d_out[4n] (device), without a
// host sync. n < 12: one pass with every qubit in the tile. n >= 12: P =
// ceil((n - 4)/8) passes of 12 tile qubits, the 4 lowest (reported by the
// first pass) and 8 high ones; high qubit number i (ascending) goes to pass
// i mod P, so that every pass holds a few of the highest qubits and a tile's
// runs spread over few memory pages; a pass with fewer than 8 of its own
// fills its tile with low high qubits of other passes (not reported).
qsim_status bloch_sums_device(const void *amps, qsim_dtype dt, int n, cudaStream_t stream, Scratch &sc, const int *d_gate,
                              double *d_out, int *passes)
{
    QS_TRY(ensure_scratch(sc, (size_t)kMaxRedBlocks * 64 + 64));
    std::vector<TileSpec> specs;
    if (n < 12) {
        TileSpec ts;
        ts.n = n;
        ts.t = n;
        ts.c = std::min(n, 4);
        for (int j = 0; j < n; j++) ts.tq[j] = j;
        ts.ins.npos = n - ts.c;
        for (int j = 0; j < n - ts.c; j++) ts.ins.pos[j] = ts.c + j;
        ts.wmask = (1u << n) - 1;
        specs.push_back(ts);
    } else {
        const int h = n - 4, P = (h + 7) / 8;
        for (int p = 0; p < P; p++) {
            std::vector<int> own, high;
            for (int i = p; i < h; i += P) own.push_back(4 + i);
            high = own;
            for (int q = 4; q < n && (int)high.size() < 8; q++)
                if (std::find(high.begin(), high.end(), q) == high.end()) high.push_back(q);
            std::sort(high.begin(), high.end());
            TileSpec ts;
            ts.n = n;
            ts.t = 12;
            ts.c = 4;
            for (int j = 0; j < 4; j++) ts.tq[j] = j;
            ts.wmask = p == 0 ? 0xfu : 0u;
            for (int j = 0; j < 8; j++) {
                ts.tq[4 + j] = high[j];
                ts.ins.pos[j] = high[j];
                if (std::find(own.begin(), own.end(), high[j]) != own.end()) ts.wmask |= 1u << (4 + j);
            }
            ts.ins.npos = 8;
            specs.push_back(ts);
        }
    }
    int np = 0;
    unsigned *ticket = (unsigned *)(sc.d + sc.cap);   // see ensure_scratch
    for (const TileSpec &ts : specs) {
        const uint64_t ntiles = 1ull << (n - ts.t);
        int blocks;
        if (ts.t == 12) {
            // pipelined tile pass (256 threads x 16 amplitudes, cp.async stage ring);
            // complex64: two CTAs per SM, complex128: one
            static bool attr = false;
            if (!attr) {
                cudaFuncSetAttribute(k_red_bloch_pipe<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     BlochGeom<float>::kSmem);
                cudaFuncSetAttribute(k_red_bloch_pipe<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     BlochGeom<float>::kSmem);
                cudaFuncSetAttribute(k_red_bloch_pipe<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     BlochGeom<double>::kSmem);
                cudaFuncSetAttribute(k_red_bloch_pipe<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     BlochGeom<double>::kSmem);
                attr = true;
            }
            const bool low = np == 0;
            if (dt == QSIM_C64) {
                blocks = (int)std::min<uint64_t>(ntiles, 2 * (uint64_t)num_sms());
                const size_t smem = BlochGeom<float>::kSmem;
                if (low)
                    k_red_bloch_pipe<float, true><<<blocks, 256, smem, stream>>>((const float2 *)amps, ts, sc.d, d_gate,
                                                                                  d_out, ticket);
                else
                    k_red_bloch_pipe<float, false><<<blocks, 256, smem, stream>>>((const float2 *)amps, ts, sc.d,
                                                                                   d_gate, d_out, ticket);
            } else {
                blocks = (int)std::min<uint64_t>(ntiles, (uint64_t)num_sms());
                const size_t smem = BlochGeom<double>::kSmem;
                if (low)
                    k_red_bloch_pipe<double, true><<<blocks, 256, smem, stream>>>((const double2 *)amps, ts, sc.d,
                                                                                   d_gate, d_out, ticket);
                else
                    k_red_bloch_pipe<double, false><<<blocks, 256, smem, stream>>>((const double2 *)amps, ts, sc.d,
                                                                                    d_gate, d_out, ticket);
            }
        } else {
            blocks = (int)std::min<uint64_t>(ntiles, kMaxRedBlocks);
            size_t smem = ((size_t)1 << ts.t) * (dt == QSIM_C64 ? 8 : 16);
            if (dt == QSIM_C64)
                k_red_bloch_tile<float><<<blocks, kRedThreads, smem, stream>>>((const float2 *)amps, ts, sc.d, d_gate,
                                                                               d_out, ticket);
            else
                k_red_bloch_tile<double><<<blocks, kRedThreads, smem, stream>>>((const double2 *)amps, ts, sc.d,
                                                                                 d_gate, d_out, ticket);
        }
        QS_CUDA(cudaGetLastError());
        np++;
    }
    if (passes) *passes = np;
    return QSIM_OK;
}

// Host copy of the per-physical-qubit Bloch sums (synchronises).
qsim_status reduce_bloch_all(qsim_state *s, double *sums)
{
    // the 4n sums go to the state's scratch, past the partial rows and the combine row
    const size_t at = (size_t)kMaxRedBlocks * 64 + 64;
    QS_TRY(ensure_scratch(s->red, at + 4 * (size_t)s->n));
    double *d = s->red.d + at;
    QS_TRY(bloch_sums_device(s->amps, s->dt, s->n, s->stream, s->red, nullptr, d, nullptr));
    QS_CUDA(cudaMemcpyAsync(sums, d, 4 * sizeof(double) * s->n, cudaMemcpyDeviceToHost, s->stream));
    QS_CUDA(cudaStreamSynchronize(s->stream));
    return QSIM_OK;
}

qsim_status probs_to_device(qsim_state *s, double *d_out)
{
    uint64_t N = s->N();
    if (s->dt == QSIM_C64)
        k_probs<float><<<default_grid(N, 256), 256, 0, s->stream>>>((const float2 *)s->amps, N, d_out);
    else
        k_probs<double><<<default_grid(N, 256), 256, 0, s->stream>>>((const double2 *)s->amps, N, d_out);
    QS_CUDA(cudaGetLastError());
    return QSIM_OK;
}

}  // namespace qs
