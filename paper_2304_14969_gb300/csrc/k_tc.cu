// Dense k-qubit block on the 5th-generation tensor cores (tcgen05), k <= 6.
//
// Table I of arXiv 2304.14969 ("coalesced gates ... single traversal"):
// a run of gates fused into one 2^k x 2^k unitary U is a dense contraction
// of U with the ket viewed as a (2^k) x (2^n / 2^k) matrix of groups. With
// the real embedding
//     [Re y]   [Re U  -Im U] [Re x]
//     [Im y] = [Im U   Re U] [Im x]
// interleaved as rows 2r + {re, im}, the product is a real GEMM
// D (128 x N) = A (128 x 128) * B (128 x N) for k = 6; blocks with k < 6 are
// padded with identity qubits (U (x) I), so every block uses M = K = 128.
//
// Precision: the 3-product split x = x_hi + x_lo of both operands
// (a_hi b_hi + a_hi b_lo + a_lo b_hi, FP32 accumulation in TMEM), with
// TF32 parts (kind::tf32) or BF16 parts (kind::f16 with BF16 inputs).
//
// One CTA = one warpgroup (128 threads). A (hi, lo) is staged once per CTA
// in shared memory in the canonical K-major no-swizzle layout (8-row x
// 16-byte core matrices, K-adjacent core matrices 128 B apart). Per
// iteration the CTA gathers N groups, splits them into B_hi / B_lo (same
// layout, rows = groups), one thread issues the 3 x K/kstep MMAs into a
// 128 x N FP32 accumulator in TMEM and commits to an mbarrier, every thread
// waits (bounded), each warp reads its 32 TMEM lanes (rows), the tile goes
// through shared memory and back to HBM coalesced.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "qsim_internal.h"
#include "tc_ptx.cuh"

namespace qs {

static const int kTcThreads = 128;
// Splits the pair (re, im) into hi and lo parts and stores each part as
// one paired store (the two K-adjacent elements of a row).
template <int ES>
__device__ __forceinline__ void split_store2(unsigned char *hi, unsigned char *lo, uint32_t off, float2 x)
{
    if constexpr (ES == 4) {
        uint32_t h0, h1;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h0) : "f"(x.x));
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h1) : "f"(x.y));
        *(uint2 *)(hi + off) = make_uint2(h0, h1);
        *(float2 *)(lo + off) = make_float2(x.x - __uint_as_float(h0), x.y - __uint_as_float(h1));
    } else {
        __nv_bfloat162 h = __floats2bfloat162_rn(x.x, x.y);
        float2 hf = __bfloat1622float2(h);
        *(__nv_bfloat162 *)(hi + off) = h;
        *(__nv_bfloat162 *)(lo + off) = __floats2bfloat162_rn(x.x - hf.x, x.y - hf.y);
    }
}

// PREC: 1 = 3xTF32 (ES 4), 2 = BF16x3 (ES 2); N = 64 groups per iteration
// (BF16x3 fits two CTAs per SM)
template <int PREC>
__global__ void __launch_bounds__(kTcThreads, PREC == 1 ? 1 : 2) k_tc_block(float2 *__restrict__ a, uint64_t ngroups, TcSpec ts,
                                                            const unsigned char *__restrict__ Ag, int *err)
{
    constexpr int ES = PREC == 1 ? 4 : 2;
    constexpr int N = 64;
    constexpr int KSTEP = PREC == 1 ? 8 : 16;          // K per instruction
    constexpr uint32_t A_BYTES = kTcRows * kTcRows * ES;
    constexpr uint32_t B_BYTES = N * kTcRows * ES;
    constexpr int SROW = kTcRows + 2;                  // padded staging row (floats)
    constexpr uint32_t SBO = (uint32_t)(kTcRows / (16 / ES)) * 128u;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *Ahi = sm, *Alo = sm + A_BYTES, *Bhi = sm + 2 * A_BYTES, *Blo = Bhi + B_BYTES;
    float *stage = (float *)Bhi;                       // D staging reuses the B region
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    __shared__ uint64_t s_spread[64];   // physical offset of block index l
    __shared__ int s_pos[6];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid < 64) {
        uint64_t o = 0;
#pragma unroll
        for (int b = 0; b < 6; b++)
            if ((tid >> b) & 1) o |= 1ull << ts.q[b];
        s_spread[tid] = o;
    }
    if (tid < 6) s_pos[tid] = ts.ins.pos[tid];

    // A (hi, lo) arrives in its final byte layout
    {
        const int4 *src = (const int4 *)Ag;
        int4 *dst = (int4 *)Ahi;
        for (uint32_t i = tid; i < 2 * A_BYTES / 16; i += kTcThreads) dst[i] = src[i];
    }
    if (tid == 0) {
        s_fail = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "r"((uint32_t)N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = (1u << 4) | ((PREC == 1 ? 2u : 1u) << 7) | ((PREC == 1 ? 2u : 1u) << 10) |
                           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
    uint32_t phase = 0;

    // Thread -> work ownership: group row nn = tid % N of each iteration and
    // block elements l = l0 + j * (threads / N). The loads of iteration i+1
    // are issued right after iteration i's operands are stored, so they are
    // in flight during i's MMAs, TMEM reads and write-back.
    const int nn = tid % N;
    constexpr int LPER = 64 / (kTcThreads / N);
    const int l0 = tid / N;
    const uint32_t rowoff = (uint32_t)(nn >> 3) * SBO + (uint32_t)(nn & 7) * 16u;
    auto group_base = [&](uint64_t g) {
        uint64_t base = g;
#pragma unroll
        for (int j = 0; j < 6; j++) {
            const int p = s_pos[j];
            base = ((base >> p) << (p + 1)) | (base & ((1ull << p) - 1));
        }
        return base;
    };
    const uint64_t gstride = (uint64_t)gridDim.x * N;
    float2 vin[LPER];
    uint64_t g0 = (uint64_t)blockIdx.x * N;
    uint64_t base = group_base(g0 + nn);
    bool gok = g0 + nn < ngroups;
#pragma unroll
    for (int j = 0; j < LPER; j++)
        vin[j] = gok ? a[base | s_spread[l0 + j * (kTcThreads / N)]] : make_float2(0.f, 0.f);

    for (; g0 < ngroups; g0 += gstride) {
        // ---- deferred phases of this group (pre-diagonal), then split the
        // loaded groups into the B operands
        if (ts.pd_off) {
            // per block bit b: e_b = exp(2 pi i T_b(group)); element factor is
            // the product of e_b over the set bits of l = l0 + j * step
            float er[6], ei[6];
#pragma unroll
            for (int b = 0; b < 6; b++) {
                uint64_t tt = 0;
                for (int e = ts.pd_off[b]; e < ts.pd_off[b + 1]; e++)
                    if ((base >> ts.pd_bit[e]) & 1) tt += ts.pd_tw[e];
                float f = (float)(int64_t)tt * 5.42101086242752217e-20f, sn, cs;
                sincospif(2.0f * f, &sn, &cs);
                ei[b] = sn;
                er[b] = cs;
            }
            constexpr int STEP = kTcThreads / N;
            // factors for the low log2(STEP) bits come from l0, the rest from j
            float br = 1.f, bi = 0.f;
#pragma unroll
            for (int b = 0; b < 6; b++)
                if ((1 << b) < STEP && ((l0 >> b) & 1)) {
                    const float xr = br * er[b] - bi * ei[b];
                    bi = br * ei[b] + bi * er[b];
                    br = xr;
                }
            constexpr int SH = STEP == 1 ? 0 : (STEP == 2 ? 1 : 2);
            float fr[LPER], fi[LPER];
            fr[0] = br;
            fi[0] = bi;
            // f[m + 2^bb] = f[m] * e[SH + bb] (constant indices: registers, not local memory)
            constexpr int LB = LPER == 64 ? 6 : LPER == 32 ? 5 : LPER == 16 ? 4 : 3;
#pragma unroll
            for (int bb = 0; bb < LB; bb++) {
#pragma unroll
                for (int m = 0; m < (1 << bb); m++) {
                    fr[m + (1 << bb)] = fr[m] * er[SH + bb] - fi[m] * ei[SH + bb];
                    fi[m + (1 << bb)] = fr[m] * ei[SH + bb] + fi[m] * er[SH + bb];
                }
            }
#pragma unroll
            for (int j = 0; j < LPER; j++) {
                const float2 x = vin[j];
                vin[j] = make_float2(x.x * fr[j] - x.y * fi[j], x.x * fi[j] + x.y * fr[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < LPER; j++) {
            const int l = l0 + j * (kTcThreads / N);
            split_store2<ES>(Bhi, Blo, rowoff + (uint32_t)((2 * l) / (16 / ES)) * 128u +
                                           (uint32_t)((2 * l) % (16 / ES)) * ES, vin[j]);
        }
        // ---- prefetch the next iteration's groups
        const uint64_t cur_base = base;
        const bool cur_ok = gok;
        {
            const uint64_t gn = g0 + gstride + nn;
            gok = gn < ngroups;
            base = gok ? group_base(gn) : 0;
#pragma unroll
            for (int j = 0; j < LPER; j++)
                vin[j] = gok ? a[base | s_spread[l0 + j * (kTcThreads / N)]] : make_float2(0.f, 0.f);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        // ---- D = A_hi B_hi + A_hi B_lo + A_lo B_hi
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t ah = smem_addr(Ahi), al = smem_addr(Alo), bh = smem_addr(Bhi), bl = smem_addr(Blo);
            uint32_t accum = 0;
            for (int part = 0; part < 3; part++) {
                const uint32_t abase = part == 2 ? al : ah, bbase = part == 1 ? bl : bh;
                for (int kk = 0; kk < kTcRows / KSTEP; kk++) {
                    const uint32_t koff = (uint32_t)kk * 256u;   // two K-adjacent core matrices per step
                    mma_issue(tmem, smem_desc(abase + koff, 128u, SBO), smem_desc(bbase + koff, 128u, SBO), idesc,
                              accum, PREC == 1);
                    accum = 1;
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_addr(&mbar)));
        }
        if (!mbar_wait(smem_addr(&mbar), phase)) {
            s_fail = 1;
            atomicExch(err, 1);
        }
        phase ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;");
        __syncthreads();
        if (s_fail) break;
        // ---- TMEM -> registers -> staging (row m = this thread's lane)
        const int m = warp * 32 + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < N; c0 += 32) {
            uint32_t r[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            tmem_ld32(taddr, r);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 32; j++) stage[(c0 + j) * SROW + m] = __uint_as_float(r[j]);
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        // ---- write the N groups back (same thread -> group ownership)
        if (cur_ok) {
#pragma unroll
            for (int j = 0; j < LPER; j++) {
                const int l = l0 + j * (kTcThreads / N);
                a[cur_base | s_spread[l]] = *(const float2 *)&stage[nn * SROW + 2 * l];
            }
        }
        __syncthreads();   // staging (B region) free for the next gather
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)N));
}

// Host side: pads the block to 6 qubits (identity on the highest unused
// qubits, which keeps the low qubits outside the block so consecutive groups
// are consecutive amplitudes), orders the 6 block bits by qubit (U permuted
// to match: the block's low qubits are its low index bits, its high qubits
// the high ones), forms A = [[Re U, -Im U], [Im U, Re U]] interleaved, and
// splits it into parts in the kernel's byte layout: TF32 hi / lo (3XTF32),
// BF16 hi / lo (BF16X3), or three BF16 slices of the FP64 value (BF16X6).
//
// kb = 7 (the 7-qubit kernel, complex64 BF16X3): the block is padded to 7
// qubits the same way and packed as two BF16 levels (hi, then lo), each a
// 256 x 128 matrix in the same layout (K = input index l) whose rows are the
// 64-row blocks Re U[0..63], Im U[0..63], Re U[64..127], Im U[64..127]. The
// kernel forms the real and imaginary outputs from these and the signed
// parts of the amplitudes, so the real embedding's duplicated blocks are
// never stored.
static qsim_status tc_build7(int n, int k, const int *phys, const cd *u, qsim_prec prec,
                             std::vector<unsigned char> &A, TcSpec &ts)
{
    if (prec != QSIM_PREC_BF16X3) return fail(QSIM_E_UNSUPPORTED, "7-qubit tensor-core blocks take BF16X3");
    if (k > 7) return fail(QSIM_E_UNSUPPORTED, "tensor-core blocks take k <= 7");
    if (n < 14) return fail(QSIM_E_UNSUPPORTED, "7-qubit tensor-core blocks need n >= 14");
    int q0[7];
    uint64_t used = 0;
    for (int b = 0; b < k; b++) {
        q0[b] = phys[b];
        used |= bit(phys[b]);
    }
    int kk = k;
    for (int p = n - 1; p >= 0 && kk < 7; p--)
        if (!(used & bit(p))) {
            q0[kk++] = p;
            used |= bit(p);
        }
    int order[7], q[7];
    for (int b = 0; b < 7; b++) order[b] = b;
    std::sort(order, order + 7, [&](int x, int y) { return q0[x] < q0[y]; });
    for (int b = 0; b < 7; b++) q[b] = q0[order[b]];
    auto old_index = [&](int r) {
        int o = 0;
        for (int j = 0; j < 7; j++)
            if ((r >> j) & 1) o |= 1 << order[j];
        return o;
    };
    const int D = 1 << k;
    const size_t level = (size_t)2 * kTcRows * kTcRows * 2;   // 256 rows x 128 K of BF16
    A.assign(2 * level, 0);
    for (int r = 0; r < 128; r++)
        for (int c = 0; c < 128; c++) {
            const int ro = old_index(r), co = old_index(c);
            const cd v = ((ro >> k) == (co >> k)) ? u[(ro & (D - 1)) * D + (co & (D - 1))] : cd(0.0);
            const float x[2] = {(float)v.real(), (float)v.imag()};
            for (int ri = 0; ri < 2; ri++) {
                const uint32_t off = canon_off(128 * (r >> 6) + 64 * ri + (r & 63), c, 2);
                const __nv_bfloat16 h = __float2bfloat16_rn(x[ri]);
                const __nv_bfloat16 lo = __float2bfloat16_rn(x[ri] - __bfloat162float(h));
                memcpy(A.data() + off, &h, 2);
                memcpy(A.data() + level + off, &lo, 2);
            }
        }
    for (int b = 0; b < 7; b++) ts.q[b] = q[b];
    ts.kb = 7;
    ts.ins.npos = 7;
    for (int b = 0; b < 7; b++) ts.ins.pos[b] = q[b];
    ts.pd_off = nullptr;
    ts.pd_bit = nullptr;
    ts.pd_tw = nullptr;
    return QSIM_OK;
}

qsim_status tc_build(int n, int k, const int *phys, const cd *u, qsim_prec prec, std::vector<unsigned char> &A,
                     TcSpec &ts, int kb)
{
    if (kb == 7) return tc_build7(n, k, phys, u, prec, A, ts);
    if (k > 6) return fail(QSIM_E_UNSUPPORTED, "tensor-core blocks of 7 qubits take complex64 kets with BF16X3");
    if (n < 6) return fail(QSIM_E_UNSUPPORTED, "tensor-core blocks need n >= 6");
    int q0[6];
    uint64_t used = 0;
    for (int b = 0; b < k; b++) {
        q0[b] = phys[b];
        used |= bit(phys[b]);
    }
    int kk = k;
    for (int p = n - 1; p >= 0 && kk < 6; p--)
        if (!(used & bit(p))) {
            q0[kk++] = p;
            used |= bit(p);
        }
    // new bit b <-> old bit order[b], ascending qubits
    int order[6], q[6];
    for (int b = 0; b < 6; b++) order[b] = b;
    std::sort(order, order + 6, [&](int x, int y) { return q0[x] < q0[y]; });
    for (int b = 0; b < 6; b++) q[b] = q0[order[b]];
    auto old_index = [&](int r) {
        int o = 0;
        for (int j = 0; j < 6; j++)
            if ((r >> j) & 1) o |= 1 << order[j];
        return o;
    };
    const int D = 1 << k;
    const int es = prec == QSIM_PREC_3XTF32 ? 4 : 2;
    const int nparts = prec == QSIM_PREC_BF16X6 ? 3 : 2;
    const size_t abytes = (size_t)kTcRows * kTcRows * es;
    A.assign((size_t)nparts * abytes, 0);
    for (int r = 0; r < 64; r++)
        for (int c = 0; c < 64; c++) {
            // padded 64 x 64 block in the old bit order: identity on bits >= k
            const int ro = old_index(r), co = old_index(c);
            cd v = ((ro >> k) == (co >> k)) ? u[(ro & (D - 1)) * D + (co & (D - 1))] : cd(0.0);
            double e[2][2] = {{v.real(), -v.imag()}, {v.imag(), v.real()}};
            for (int ri = 0; ri < 2; ri++)
                for (int ci = 0; ci < 2; ci++) {
                    int row = 2 * r + ri, col = 2 * c + ci;
                    float x = (float)e[ri][ci];
                    uint32_t off = canon_off(row, col, es);
                    if (es == 4) {
                        // TF32 hi part: keep 10 mantissa bits, round half away from zero
                        uint32_t bits;
                        memcpy(&bits, &x, 4);
                        uint32_t h = (bits + 0x1000u) & 0xFFFFE000u;
                        float hf;
                        memcpy(&hf, &h, 4);
                        float lo = x - hf;
                        memcpy(A.data() + off, &h, 4);
                        memcpy(A.data() + abytes + off, &lo, 4);
                    } else if (nparts == 3) {
                        // slices of the FP64 value: each takes the remainder of the ones before
                        double rem = e[ri][ci];
                        for (int sl = 0; sl < 3; sl++) {
                            __nv_bfloat16 h = __float2bfloat16_rn((float)rem);
                            rem -= (double)__bfloat162float(h);
                            memcpy(A.data() + (size_t)sl * abytes + off, &h, 2);
                        }
                    } else {
                        __nv_bfloat16 h = __float2bfloat16_rn(x);
                        float hf = __bfloat162float(h);
                        __nv_bfloat16 lo = __float2bfloat16_rn(x - hf);
                        memcpy(A.data() + off, &h, 2);
                        memcpy(A.data() + abytes + off, &lo, 2);
                    }
                }
        }
    for (int b = 0; b < 6; b++) ts.q[b] = q[b];
    ts.kb = 6;
    ts.ins.npos = 6;
    for (int b = 0; b < 6; b++) ts.ins.pos[b] = q[b];
    ts.pd_off = nullptr;
    ts.pd_bit = nullptr;
    ts.pd_tw = nullptr;
    return QSIM_OK;
}

// Launches one block (stream-ordered; the kernel raises *derr if an MMA
// completion wait gave up).
cudaError_t tc_launch(qsim_state *s, const TcSpec &ts, const unsigned char *dA, qsim_prec prec, int *derr)
{
    const uint64_t ngroups = s->N() >> 6;
    if (prec == QSIM_PREC_3XTF32) {
        const int N = 64;
        size_t smem = 2 * (size_t)kTcRows * kTcRows * 4 +
                      std::max<size_t>(2 * (size_t)N * kTcRows * 4, (size_t)N * (kTcRows + 2) * 4);
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_tc_block<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            attr = true;
        }
        int grid = (int)std::min<uint64_t>((ngroups + N - 1) / N, (uint64_t)num_sms());
        k_tc_block<1><<<grid, kTcThreads, smem, s->stream>>>((float2 *)s->amps, ngroups, ts, dA, derr);
    } else {
        const int N = 64;
        size_t smem = 2 * (size_t)kTcRows * kTcRows * 2 +
                      std::max<size_t>(2 * (size_t)N * kTcRows * 2, (size_t)N * (kTcRows + 2) * 4);
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_tc_block<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            attr = true;
        }
        int occ = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_tc_block<2>, kTcThreads, smem);
        int grid = (int)std::min<uint64_t>((ngroups + N - 1) / N, (uint64_t)num_sms() * std::max(1, occ));
        k_tc_block<2><<<grid, kTcThreads, smem, s->stream>>>((float2 *)s->amps, ngroups, ts, dA, derr);
    }
    return cudaGetLastError();
}

qsim_status apply_fused_tc(qsim_state *s, int k, const int *phys, const cd *u, qsim_prec prec)
{
    if (s->dt == QSIM_C64 && prec == QSIM_PREC_BF16X6)
        return fail(QSIM_E_UNSUPPORTED, "BF16X6 blocks take complex128 kets");
    if (s->dt == QSIM_C128 && !tc_pipe_eligible(s->n, s->dt, prec))
        return fail(QSIM_E_UNSUPPORTED, "complex128 kets take BF16X6 tensor-core blocks with n >= 13");
    const int kb = k == 7 ? 7 : 6;
    if (kb == 7 && !tc_pipe_eligible(s->n, s->dt, prec, 7))
        return fail(QSIM_E_UNSUPPORTED, "7-qubit tensor-core blocks take complex64 kets, BF16X3 and n >= 14");
    std::vector<unsigned char> A;
    TcSpec ts;
    QS_TRY(tc_build(s->n, k, phys, u, prec, A, ts, kb));
    unsigned char *dA = nullptr;
    int *derr = nullptr;
    QS_CUDA(cudaMallocAsync((void **)&dA, A.size(), s->stream));
    QS_CUDA(cudaMallocAsync((void **)&derr, sizeof(int), s->stream));
    QS_CUDA(cudaMemsetAsync(derr, 0, sizeof(int), s->stream));
    QS_CUDA(cudaMemcpyAsync(dA, A.data(), A.size(), cudaMemcpyHostToDevice, s->stream));
    cudaError_t e;
    if (tc_pipe_eligible(s->n, s->dt, prec, kb)) {
        TcPipeHost H;
        qsim_status st = tc_pipe_prepare(s->n, ts, nullptr, H, tc_pipe_kind(s->dt, prec, kb));
        e = st == QSIM_OK ? tc_pipe_launch(s, H, dA, derr) : cudaErrorInvalidValue;
    } else {
        e = tc_launch(s, ts, dA, prec, derr);
    }
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    cudaFreeAsync(dA, s->stream);
    cudaFreeAsync(derr, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core block");
    if (herr) return fail(QSIM_E_TIMEOUT, "tensor-core block: MMA completion wait gave up");
    return QSIM_OK;
}

// One CTA waits on an mbarrier that no thread arrives at (its phase 0 never
// completes), through the same bounded wait as the block kernels; when the
// wait gives up it sets the error word.
__global__ void k_wait_selftest(int *err, unsigned long long limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_addr(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait(smem_addr(&bar), 0, limit_ns)) atomicExch(err, 1);
}

}  // namespace qs

using namespace qs;

extern "C" qsim_status qsim_selftest_wait_timeout(qsim_state *s, int64_t limit_ns)
{
    clear_error();
    if (!s) return fail(QSIM_E_INVAL, "NULL state");
    if (limit_ns < 1000 || limit_ns > 10000000000ll)
        return fail(QSIM_E_INVAL, "limit_ns=%lld outside [1e3, 1e10]", (long long)limit_ns);
    QS_TRY(err_ensure(s));
    k_wait_selftest<<<1, 32, 0, s->stream>>>(s->d_err, (unsigned long long)limit_ns);
    QS_CUDA(cudaGetLastError());
    return QSIM_OK;
}
