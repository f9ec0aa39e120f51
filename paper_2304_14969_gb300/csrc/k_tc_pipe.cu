// Pipelined tensor-core block (BF16x3 split, k <= 6 padded to 6), n >= 13.
//
// Same contraction as k_tc_block (Table I fused blocks, real embedding of
// U, three-product BF16 split with FP32 accumulation in TMEM), organised as
// a persistent, warp-specialised pipeline fed by TMA:
//
//   tile   = 128 groups x 64 block amplitudes = 8192 complex64 (64 KB): the
//            block's 6 qubits and the 7 lowest qubits outside it;
//   warp 0 = one thread issuing the TMA loads of the next tiles into two
//            64 KB shared-memory stages (up to four 5-D boxes per tile);
//   warp 1 = one thread issuing the MMAs: D[g][2l'+ri'] = sum_k S[g][k]
//            U[2l'+ri'][k], S the tile (M = 128 groups, K = 128) and U the
//            real-embedded block (N = 128), into one of two 128-column TMEM
//            accumulators;
//   warps 2..9 = convert (read the raw tile from its stage, apply the
//            deferred per-group phases, write its BF16 hi / lo split in
//            place as the MMA's A operand) and write back (each thread owns
//            one TMEM lane = one group and 32 of its amplitudes, stored to
//            HBM directly: lanes are consecutive groups, so stores are
//            coalesced when the low qubits are outside the block).
//
// Stage s is reloaded once the MMAs that read it have completed; TMEM
// accumulator b is reused once the write-back of the tile before has read
// it. Every wait is bounded; a wait that gives up sets the error word and
// every role leaves its loop (loads still in flight are waited for, with a
// bound, before the CTA exits).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "qsim_internal.h"
#include "tc_ptx.cuh"

namespace qs {

namespace {

constexpr int kPThreads = 320;
constexpr int kPConv = 256;                  // converter / write-back threads (warps 2..9)
constexpr uint32_t kPStage = 65536;          // one tile of complex64
constexpr uint32_t kPHalf = 32768;           // hi or lo BF16 operand of a tile (128 x 128)
constexpr uint32_t kPU = 65536;              // U hi + lo
constexpr size_t kPSmem = kPU + 2 * (size_t)kPStage + 1024;


__device__ __forceinline__ uint64_t tile_base(const TcPipeArgs &P, uint64_t t)
{
    uint64_t base = t;
#pragma unroll
    for (int j = 0; j < 13; j++) {
        const int p = P.tpos[j];
        base = ((base >> p) << (p + 1)) | (base & ((1ull << p) - 1));
    }
    return base;
}

__device__ __forceinline__ void turns_sincos(uint64_t tt, float &s, float &c)
{
    const float f = (float)(int64_t)tt * 5.42101086242752217e-20f;   // turns in [-0.5, 0.5)
    sincospif(2.0f * f, &s, &c);
}

__global__ void __launch_bounds__(kPThreads, 1)
    k_tc_pipe(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ TcPipeArgs P, float2 *__restrict__ a,
              const unsigned char *__restrict__ Ug, int *err)
{
    extern __shared__ unsigned char sm_dyn[];
    unsigned char *smb = (unsigned char *)(((uintptr_t)sm_dyn + 1023) & ~(uintptr_t)1023);
    unsigned char *Us = smb;                              // U operand (N x K): hi [0, 32K), lo [32K, 64K)
    unsigned char *St = smb + kPU;                        // raw stages 0 and 1
    __shared__ __align__(8) uint64_t bar_full[2], bar_sfree[2], bar_aready[2], bar_mma[2], bar_accf[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    __shared__ uint16_t s_posL[64];
    __shared__ uint64_t s_spL[64];
    __shared__ uint64_t s_bt[6];
    __shared__ uint64_t s_gturn[128 * 6];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool has_pd = P.pd_off != nullptr;
    for (int i = tid; i < 64; i += kPThreads) {
        s_posL[i] = P.posL[i];
        s_spL[i] = P.spL[i];
    }
    if (has_pd)
        for (int i = tid; i < 128 * 6; i += kPThreads) s_gturn[i] = P.gturn[i];
    {
        const int4 *src = (const int4 *)Ug;
        int4 *dst = (int4 *)Us;
        for (uint32_t i = tid; i < kPU / 16; i += kPThreads) dst[i] = src[i];
    }
    if (tid == 0) {
        s_abort = 0;
        for (int s = 0; s < 2; s++) {
            mbar_init(smem_addr(&bar_full[s]), 1);
            mbar_init(smem_addr(&bar_sfree[s]), kPConv);
            mbar_init(smem_addr(&bar_aready[s]), kPConv);
            mbar_init(smem_addr(&bar_mma[s]), 1);
            mbar_init(smem_addr(&bar_accf[s]), kPConv);
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                     "r"(512u));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    // TMEM columns: accumulators [0, 128) and [128, 256); A operands (hi, lo:
    // 64 + 64 columns, BF16 pairs) [256, 384) and [384, 512)
    const uint32_t tmem = s_tmem;
    volatile int *abort_flag = &s_abort;
    auto give_up = [&]() {
        *abort_flag = 1;
        atomicExch(err, 1);
    };
    // tiles of this CTA: blockIdx.x + j * gridDim.x, j < J
    const uint64_t J = P.ntiles > blockIdx.x ? (P.ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;

    if (warp == 0) {
        // ---------------- TMA producer: stage s is reloaded once the
        // converters have read the tile two before
        if (lane == 0) {
            uint64_t issued = 0;
            for (uint64_t j = 0; j < J && !*abort_flag; j++) {
                const int s = (int)(j & 1);
                if (j >= 2 &&
                    !mbar_wait_or_abort(smem_addr(&bar_sfree[s]), (uint32_t)(((j - 2) >> 1) & 1), abort_flag)) {
                    give_up();
                    break;
                }
                const uint64_t base = tile_base(P, blockIdx.x + j * gridDim.x);
                int c[5];
#pragma unroll
                for (int d = 0; d < 5; d++) c[d] = (int)((base >> P.dim_lo[d]) & ((1ull << P.dim_bits[d]) - 1));
                const uint32_t fb = smem_addr(&bar_full[s]);
                mbar_arrive_expect_tx(fb, P.box_bytes * (uint32_t)P.nload);
                const uint32_t dst = smem_addr(St + (size_t)s * kPStage);
                for (int v = 0; v < P.nload; v++)
                    tma_load_5d(dst + (uint32_t)v * P.box_bytes, &tmap, fb, c[0], c[1], c[2], c[3], c[4] + P.xoff[v]);
                issued = j + 1;
            }
            // loads still in flight (only after an abort) land before the CTA exits
            for (uint64_t j = issued >= 2 ? issued - 2 : 0; j < issued; j++)
                mbar_wait(smem_addr(&bar_full[j & 1]), (uint32_t)((j >> 1) & 1));
        }
    } else if (warp == 1) {
        // ---------------- MMA issue: D[g][n] = sum_k A[g][k] U[n][k], A in TMEM
        if (lane == 0) {
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(128 >> 3) << 17) |
                                   ((uint32_t)(128 >> 4) << 24);
            const uint32_t SBO = 2048u;
            uint64_t issued = 0;
            for (uint64_t j = 0; j < J && !*abort_flag; j++) {
                const int b = (int)(j & 1);
                if (!mbar_wait_or_abort(smem_addr(&bar_aready[b]), (uint32_t)((j >> 1) & 1), abort_flag)) {
                    give_up();
                    break;
                }
                if (j >= 2 &&
                    !mbar_wait_or_abort(smem_addr(&bar_accf[b]), (uint32_t)(((j - 2) >> 1) & 1), abort_flag)) {
                    give_up();
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t d = tmem + (uint32_t)b * 128u;
                const uint32_t ah = tmem + 256u + (uint32_t)b * 128u, al = ah + 64u;
                const uint32_t uh = smem_addr(Us), ul = uh + kPHalf;
                uint32_t accum = 0;
#pragma unroll 1
                for (int part = 0; part < 3; part++) {
                    const uint32_t abase = part == 2 ? al : ah, bbase = part == 1 ? ul : uh;
#pragma unroll
                    for (int kk = 0; kk < 8; kk++) {
                        // K step of 16 BF16 = 8 TMEM columns of A, two core matrices of U
                        mma_issue_tmem_a(d, abase + (uint32_t)kk * 8u, smem_desc(bbase + (uint32_t)kk * 256u, 128u, SBO),
                                         idesc, accum);
                        accum = 1;
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_addr(&bar_mma[b])));
                issued = j + 1;
            }
            if (issued) mbar_wait(smem_addr(&bar_mma[(issued - 1) & 1]), (uint32_t)(((issued - 1) >> 1) & 1));
        }
    } else {
        // ---------------- convert + write back (warps 2..9). A thread owns one
        // group (its TMEM lane) and half of its 64 amplitudes.
        const int ct = tid - 64, cw = ct >> 5;
        const int quarter = warp & 3, half = cw >> 2;
        const int g = 32 * quarter + lane;
        const uint32_t lane_off = (uint32_t)(32 * quarter) << 16;
        const uint32_t offG = 8u * P.posG[g];
        const uint64_t spG = P.spG[g];

        for (uint64_t j = 0; j <= J; j++) {
            if (j < J) {
                const int s = (int)(j & 1), b = (int)(j & 1);
                if (has_pd && ct < 6) {
                    // base turns of the deferred phases (published by the barrier below)
                    const uint64_t base = tile_base(P, blockIdx.x + j * gridDim.x);
                    uint64_t tt = 0;
                    for (int e = P.pd_off[ct]; e < P.pd_off[ct + 1]; e++)
                        if ((base >> P.pd_bit[e]) & 1) tt += P.pd_tw[e];
                    s_bt[ct] = tt;
                }
                const bool ok = mbar_wait_or_abort(smem_addr(&bar_full[s]), (uint32_t)((j >> 1) & 1), abort_flag);
                // one decision for all converter threads (none may be left at a barrier)
                if (named_bar_or(1, kPConv, !ok || *abort_flag)) {
                    give_up();
                    break;
                }
                const unsigned char *stage = St + (size_t)s * kPStage + offG;
                float2 v[32];
#pragma unroll
                for (int i = 0; i < 32; i++) v[i] = *(const float2 *)(stage + 8u * s_posL[32 * half + i]);
                mbar_arrive(smem_addr(&bar_sfree[s]));   // the stage may be reloaded
                if (has_pd) {
                    // factor of (g, l) = prod_b e_b(g)^(l_b), l = 32 half + i
                    float er[6], ei[6];
#pragma unroll
                    for (int bb = 0; bb < 6; bb++) turns_sincos(s_bt[bb] + s_gturn[g * 6 + bb], ei[bb], er[bb]);
                    float fr = half ? er[5] : 1.f, fi = half ? ei[5] : 0.f;
                    float tr[32], ti[32];
                    tr[0] = fr;
                    ti[0] = fi;
#pragma unroll
                    for (int i = 1; i < 32; i++) {
                        const int low = ctz_const(i), prev = i & (i - 1);
                        tr[i] = tr[prev] * er[low] - ti[prev] * ei[low];
                        ti[i] = tr[prev] * ei[low] + ti[prev] * er[low];
                    }
#pragma unroll
                    for (int i = 0; i < 32; i++) {
                        const float xr = v[i].x * tr[i] - v[i].y * ti[i];
                        v[i].y = v[i].x * ti[i] + v[i].y * tr[i];
                        v[i].x = xr;
                    }
                }
                // BF16 hi / lo split into the A operand of accumulator b (the MMAs
                // of tile j - 2, the last reader of these columns, completed
                // before this thread wrote that tile back)
                uint32_t hi[32], lo[32];
#pragma unroll
                for (int i = 0; i < 32; i++) {
                    const __nv_bfloat162 h = __floats2bfloat162_rn(v[i].x, v[i].y);
                    const float2 hf = __bfloat1622float2(h);
                    const __nv_bfloat162 l2 = __floats2bfloat162_rn(v[i].x - hf.x, v[i].y - hf.y);
                    hi[i] = *(const uint32_t *)&h;
                    lo[i] = *(const uint32_t *)&l2;
                }
                const uint32_t acol = tmem + lane_off + 256u + (uint32_t)b * 128u + (uint32_t)(32 * half);
                tmem_st32(acol, hi);
                tmem_st32(acol + 64u, lo);
                tmem_wait_st();
                asm volatile("tcgen05.fence::before_thread_sync;");
                mbar_arrive(smem_addr(&bar_aready[b]));
            }
            if (j >= 1) {
                // write back tile j - 1
                const uint64_t jj = j - 1;
                const int b = (int)(jj & 1);
                const bool ok = mbar_wait_or_abort(smem_addr(&bar_mma[b]), (uint32_t)((jj >> 1) & 1), abort_flag);
                if (named_bar_or(1, kPConv, !ok || *abort_flag)) {
                    give_up();
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint64_t base = tile_base(P, blockIdx.x + jj * gridDim.x);
                float2 *dstg = a + (base + spG);
#pragma unroll 1
                for (int c0 = 0; c0 < 64; c0 += 32) {
                    uint32_t r[32];
                    tmem_ld32(tmem + lane_off + (uint32_t)b * 128u + (uint32_t)(64 * half + c0), r);
                    tmem_wait_ld();
                    const int l0 = 32 * half + c0 / 2;
#pragma unroll
                    for (int i = 0; i < 16; i++)
                        dstg[s_spL[l0 + i]] = make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
                }
                asm volatile("tcgen05.fence::before_thread_sync;");
                mbar_arrive(smem_addr(&bar_accf[b]));
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u));
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, []() {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

}  // namespace

cudaError_t tc_pipe_launch(qsim_state *s, const TcPipeHost &H, const unsigned char *dU, int *derr)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    alignas(64) CUtensorMap tm;
    CUresult r = enc(&tm, CU_TENSOR_MAP_DATA_TYPE_INT64, (cuuint32_t)H.rank, s->amps, (const cuuint64_t *)H.gdim,
                     (const cuuint64_t *)H.gstr, (const cuuint32_t *)H.box, (const cuuint32_t *)H.estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_tc_pipe, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPSmem);
        attr = true;
    }
    const int grid = (int)std::min<uint64_t>(H.args.ntiles, (uint64_t)num_sms());
    k_tc_pipe<<<grid, kPThreads, kPSmem, s->stream>>>(tm, H.args, (float2 *)s->amps, dU, derr);
    return cudaGetLastError();
}

}  // namespace qs
