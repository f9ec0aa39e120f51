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
//   warps 2..17 = convert: read the raw tile from its stage (and release
//            the stage at once), apply the deferred per-group phases, write
//            the BF16 hi / lo split into TMEM as the MMA's A operand;
//   warps 18..21 = write back: each thread owns one TMEM lane = one group
//            and stores its 64 amplitudes to HBM directly (lanes are
//            consecutive groups, so stores are coalesced when the low
//            qubits are outside the block).
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

constexpr int kPConvWarps = 16;              // converter warps (2 .. 17)
constexpr int kPConv = 32 * kPConvWarps;
constexpr int kPEpiWarps = 4;                // write-back warps (18 .. 21), one per TMEM lane quarter
constexpr int kPEpi = 32 * kPEpiWarps;
constexpr int kPThreads = 64 + kPConv + kPEpi;
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

// G = false: one block over one ket, CTAs stride over its tiles (the
// tensor map, geometry, ket and U come as parameters). G = true: grouped
// (batched circuits): CTA i takes work entry i, a range of tiles of the
// block that descs[works[i].desc] describes, and stamps the circuit's first
// load and last store with %globaltimer.
template <bool G>
__global__ void __launch_bounds__(kPThreads, 1)
    k_tc_pipe(const __grid_constant__ CUtensorMap tmap_param, const __grid_constant__ TcPipeArgs P_param,
              float2 *__restrict__ a_param, const unsigned char *__restrict__ Ug_param, int *err,
              const TcBatchDesc *__restrict__ descs, const TcWork *__restrict__ works, unsigned long long *t0s,
              unsigned long long *t1s, double *norm_out)
{
    extern __shared__ unsigned char sm_dyn[];
    __shared__ __align__(16) TcPipeArgs s_P;
    const TcBatchDesc *desc = G ? &descs[works[blockIdx.x].desc] : nullptr;
    {
        const uint64_t *src = (const uint64_t *)(G ? &desc->args : &P_param);
        uint64_t *dst = (uint64_t *)&s_P;
        for (int i = threadIdx.x; i < (int)(sizeof(TcPipeArgs) / 8); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const TcPipeArgs &P = s_P;
    const void *tmap = G ? (const void *)desc->tmap : (const void *)&tmap_param;
    float2 *__restrict__ a = G ? desc->amps : a_param;
    const unsigned char *__restrict__ Ug = G ? desc->U : Ug_param;
    const uint64_t wtile0 = G ? works[blockIdx.x].tile0 : 0, wntiles = G ? works[blockIdx.x].ntiles : 0;
    // tile of this CTA's j-th iteration
    auto tile_of = [&](uint64_t j) -> uint64_t { return G ? wtile0 + j : blockIdx.x + j * gridDim.x; };
    unsigned char *smb = (unsigned char *)(((uintptr_t)sm_dyn + 1023) & ~(uintptr_t)1023);
    unsigned char *Us = smb;                              // U operand (N x K): hi [0, 32K), lo [32K, 64K)
    unsigned char *St = smb + kPU;                        // raw stages 0 and 1
    __shared__ __align__(8) uint64_t bar_full[2], bar_sfree[2], bar_aready[2], bar_mma[2], bar_accf[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    __shared__ uint16_t s_posL[64];
    __shared__ uint64_t s_spL[64];
    __shared__ uint64_t s_tturn[6 * 24];
    __shared__ float2 s_gfac[128 * 6];
    __shared__ float2 s_E[4][6];             // tile factors of the deferred phases (tile j in slot j & 3)

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool has_pd = P.gfac != nullptr;
    for (int i = tid; i < 64; i += kPThreads) {
        s_posL[i] = P.posL[i];
        s_spL[i] = P.spL[i];
    }
    if (has_pd) {
        for (int i = tid; i < 128 * 6; i += kPThreads) s_gfac[i] = P.gfac[i];
        for (int i = tid; i < 6 * 24; i += kPThreads) s_tturn[i] = P.tturn[i];
    }
    {
        const int4 *src = (const int4 *)Ug;
        int4 *dst = (int4 *)Us;
        for (uint32_t i = tid; i < kPU / 16; i += kPThreads) dst[i] = src[i];
    }
    if (tid == 0) {
        s_abort = 0;
        for (int s = 0; s < 2; s++) {
            // with deferred phases the producer arrives a second time once the
            // tile factors are written
            mbar_init(smem_addr(&bar_full[s]), has_pd ? 2 : 1);
            mbar_init(smem_addr(&bar_sfree[s]), kPConv);
            mbar_init(smem_addr(&bar_aready[s]), kPConv);
            mbar_init(smem_addr(&bar_mma[s]), 1);
            mbar_init(smem_addr(&bar_accf[s]), kPEpi);
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
    // number of tiles of this CTA
    const uint64_t J = G ? wntiles : (P.ntiles > blockIdx.x ? (P.ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0);
    if (G && tid == 0 && J > 0) atomicMin(&t0s[desc->circ], global_ns());

    if (warp == 0) {
        // ---------------- TMA producer (lane 0) and tile factors of the
        // deferred phases (lanes 0..5): stage s is reloaded once the
        // converters have read the tile two before
        uint64_t issued = 0;
        for (uint64_t j = 0; j < J; j++) {
            const int s = (int)(j & 1);
            int stop = 0;
            if (lane == 0) {
                const bool ok = j < 2 ||
                                mbar_wait_or_abort(smem_addr(&bar_sfree[s]), (uint32_t)(((j - 2) >> 1) & 1), abort_flag);
                if (!ok) give_up();
                stop = !ok || *abort_flag;
            }
            if (__shfl_sync(0xffffffffu, stop, 0)) break;
            const uint64_t t = tile_of(j);
            const uint32_t fb = smem_addr(&bar_full[s]);
            if (lane == 0) {
                const uint64_t base = tile_base(P, t);
                int c[5];
#pragma unroll
                for (int d = 0; d < 5; d++) c[d] = (int)((base >> P.dim_lo[d]) & ((1ull << P.dim_bits[d]) - 1));
                mbar_arrive_expect_tx(fb, P.box_bytes * (uint32_t)P.nload);
                const uint32_t dst = smem_addr(St + (size_t)s * kPStage);
                for (int v = 0; v < P.nload; v++)
                    tma_load_5d(dst + (uint32_t)v * P.box_bytes, tmap, fb, c[0], c[1], c[2], c[3], c[4] + P.xoff[v]);
            }
            if (has_pd) {
                if (lane < 6) {
                    uint64_t tt = 0;
                    for (int i = 0; i < P.ntb; i++)
                        if ((t >> i) & 1) tt += s_tturn[lane * 24 + i];
                    float sn, cs;
                    turns_sincos(tt, sn, cs);
                    s_E[j & 3][lane] = make_float2(cs, sn);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(fb);
            }
            issued = j + 1;
        }
        // loads still in flight (only after an abort) land before the CTA exits
        if (lane == 0)
            for (uint64_t j = issued >= 2 ? issued - 2 : 0; j < issued; j++)
                mbar_wait(smem_addr(&bar_full[j & 1]), (uint32_t)((j >> 1) & 1));
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
    } else if (warp < 2 + kPConvWarps) {
        // ---------------- convert (warps 2..17). A thread owns one group (its
        // TMEM lane) and 16 of its 64 amplitudes, l = 16 part + i. The stage
        // is released as soon as it has been read: with two stages, the time
        // a landed tile waits to be read is what bounds the load pipeline.
        const int ct = tid - 64, cw = ct >> 5;
        const int quarter = warp & 3, part = cw >> 2;
        const int g = 32 * quarter + lane;
        const uint32_t lane_off = (uint32_t)(32 * quarter) << 16;
        const uint32_t offG = 8u * P.posG[g];
        const int rot = P.rot_bits ? (lane >> (4 - P.rot_bits)) & ((1 << P.rot_bits) - 1) : 0;
        // in-stage byte offsets of this thread's reads (the same for every tile)
        uint32_t offL[16];
#pragma unroll
        for (int i = 0; i < 16; i++) offL[i] = offG + 8u * s_posL[16 * part + (i ^ rot)];

        for (uint64_t j = 0; j < J; j++) {
            const int s = (int)(j & 1), b = (int)(j & 1);
            const bool ok = mbar_wait_or_abort(smem_addr(&bar_full[s]), (uint32_t)((j >> 1) & 1), abort_flag);
            // one decision for all converter threads (none may be left at a barrier)
            if (named_bar_or(1, kPConv, !ok || *abort_flag)) {
                give_up();
                break;
            }
            const unsigned char *stage = St + (size_t)s * kPStage;
            float2 v[16];
            // Block qubits among qubits 0..3 (block bits 0..rot_bits-1) would put
            // the 16 lanes of a half-warp on one bank: each lane reads its
            // amplitudes in an order XOR-rotated by its own lane bits, so every
            // read instruction covers 16 distinct banks; v[] is put back in
            // order below.
#pragma unroll
            for (int i = 0; i < 16; i++) v[i] = *(const float2 *)(stage + offL[i]);
            mbar_arrive(smem_addr(&bar_sfree[s]));   // the stage may be reloaded
#pragma unroll
            for (int bb = 0; bb < 4; bb++) {
                if (bb < P.rot_bits) {
                    const bool sw = (rot >> bb) & 1;
#pragma unroll
                    for (int i = 0; i < 16; i++)
                        if (!(i & (1 << bb))) {
                            const float2 x = v[i], y = v[i | (1 << bb)];
                            v[i] = sw ? y : x;
                            v[i | (1 << bb)] = sw ? x : y;
                        }
                }
            }
            if (has_pd) {
                // factor of (g, l) = prod_b e_b(g)^(l_b), e_b(g) = E_b(tile) G_b(g);
                // bits 4, 5 of l from part, 0..3 from i
                float er[6], ei[6];
#pragma unroll
                for (int bb = 0; bb < 6; bb++) {
                    const float2 E = s_E[j & 3][bb], G = s_gfac[g * 6 + bb];
                    er[bb] = E.x * G.x - E.y * G.y;
                    ei[bb] = E.x * G.y + E.y * G.x;
                }
                float fr = 1.f, fi = 0.f;
                if (part & 1) {
                    fr = er[4];
                    fi = ei[4];
                }
                if (part & 2) {
                    const float xr = fr * er[5] - fi * ei[5];
                    fi = fr * ei[5] + fi * er[5];
                    fr = xr;
                }
                float tr[16], ti[16];
                tr[0] = fr;
                ti[0] = fi;
                // tr[m + 2^bb] = tr[m] e_bb (constant indices: the factors stay in registers)
#pragma unroll
                for (int bb = 0; bb < 4; bb++) {
#pragma unroll
                    for (int m = 0; m < (1 << bb); m++) {
                        tr[m + (1 << bb)] = tr[m] * er[bb] - ti[m] * ei[bb];
                        ti[m + (1 << bb)] = tr[m] * ei[bb] + ti[m] * er[bb];
                    }
                }
#pragma unroll
                for (int i = 0; i < 16; i++) {
                    const float xr = v[i].x * tr[i] - v[i].y * ti[i];
                    v[i].y = v[i].x * ti[i] + v[i].y * tr[i];
                    v[i].x = xr;
                }
            }
            // BF16 hi / lo split into A operand b (TMEM)
            uint32_t hi[16], lo[16];
#pragma unroll
            for (int i = 0; i < 16; i++) {
                const __nv_bfloat162 h = __floats2bfloat162_rn(v[i].x, v[i].y);
                const float2 hf = __bfloat1622float2(h);
                const __nv_bfloat162 l2 = __floats2bfloat162_rn(v[i].x - hf.x, v[i].y - hf.y);
                hi[i] = *(const uint32_t *)&h;
                lo[i] = *(const uint32_t *)&l2;
            }
            if (j >= 2) {
                // A operand b was last read by the MMAs of tile j - 2
                const bool ok2 =
                    mbar_wait_or_abort(smem_addr(&bar_mma[b]), (uint32_t)(((j - 2) >> 1) & 1), abort_flag);
                if (named_bar_or(1, kPConv, !ok2 || *abort_flag)) {
                    give_up();
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
            }
            const uint32_t acol = tmem + lane_off + 256u + (uint32_t)b * 128u + (uint32_t)(16 * part);
            tmem_st16(acol, hi);
            tmem_st16(acol + 64u, lo);
            tmem_wait_st();
            asm volatile("tcgen05.fence::before_thread_sync;");
            mbar_arrive(smem_addr(&bar_aready[b]));
        }
    } else {
        // ---------------- write back (warps 18..21): TMEM lane = group,
        // accumulator columns 2l + {re, im}; 32 amplitudes per pass
        const int quarter = warp & 3;
        const int g = 32 * quarter + lane;
        const uint32_t lane_off = (uint32_t)(32 * quarter) << 16;
        const uint64_t spG = P.spG[g];
        double nacc = 0;   // sum of |amplitude|^2 written (norm_out): FP32 runs of 16, FP64 across runs
        for (uint64_t j = 0; j < J; j++) {
            const int b = (int)(j & 1);
            const bool ok = mbar_wait_or_abort(smem_addr(&bar_mma[b]), (uint32_t)((j >> 1) & 1), abort_flag);
            if (named_bar_or(2, kPEpi, !ok || *abort_flag)) {
                give_up();
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint64_t base = tile_base(P, tile_of(j));
            float2 *dstg = a + (base + spG);
#pragma unroll 1
            for (int c0 = 0; c0 < 128; c0 += 32) {
                uint32_t r[32];
                tmem_ld32(tmem + lane_off + (uint32_t)b * 128u + (uint32_t)c0, r);
                tmem_wait_ld();
                if (norm_out) {
                    float run = 0.f;
#pragma unroll
                    for (int i = 0; i < 32; i++) run = fmaf(__uint_as_float(r[i]), __uint_as_float(r[i]), run);
                    nacc += (double)run;
                }
                const int l0 = c0 / 2;
                if (P.vec2) {
                    // amplitudes l, l + 1 adjacent: one 16-byte store per pair
#pragma unroll
                    for (int i = 0; i < 16; i += 2)
                        *(float4 *)(dstg + s_spL[l0 + i]) =
                            make_float4(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]),
                                        __uint_as_float(r[2 * i + 2]), __uint_as_float(r[2 * i + 3]));
                } else {
#pragma unroll
                    for (int i = 0; i < 16; i++)
                        dstg[s_spL[l0 + i]] = make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            mbar_arrive(smem_addr(&bar_accf[b]));
        }
        if (norm_out) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) nacc += __shfl_down_sync(0xffffffffu, nacc, o);
            if (lane == 0) atomicAdd(norm_out, nacc);
        }
        if (G) {
            named_bar_sync(2, kPEpi);
            if (warp == 2 + kPConvWarps && lane == 0 && J > 0) atomicMax(&t1s[desc->circ], global_ns());
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

qsim_status tc_pipe_encode(const TcPipeHost &H, void *amps, unsigned char tmap[128])
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) return fail(QSIM_E_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    alignas(64) CUtensorMap tm;
    CUresult r = enc(&tm, CU_TENSOR_MAP_DATA_TYPE_INT64, (cuuint32_t)H.rank, amps, (const cuuint64_t *)H.gdim,
                     (const cuuint64_t *)H.gstr, (const cuuint32_t *)H.box, (const cuuint32_t *)H.estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(QSIM_E_CUDA, "tensor map encoding failed (CUresult %d)", (int)r);
    static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
    memcpy(tmap, &tm, 128);
    return QSIM_OK;
}

static void tc_pipe_attrs()
{
    static std::once_flag once;
    std::call_once(once, []() {
        cudaFuncSetAttribute(k_tc_pipe<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPSmem);
        cudaFuncSetAttribute(k_tc_pipe<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPSmem);
    });
}

cudaError_t tc_pipe_launch(qsim_state *s, const TcPipeHost &H, const unsigned char *dU, int *derr, double *norm_out)
{
    alignas(64) CUtensorMap tm;
    if (tc_pipe_encode(H, s->amps, (unsigned char *)&tm) != QSIM_OK) return cudaErrorInvalidValue;
    tc_pipe_attrs();
    const int grid = (int)std::min<uint64_t>(H.args.ntiles, (uint64_t)num_sms());
    k_tc_pipe<false><<<grid, kPThreads, kPSmem, s->stream>>>(tm, H.args, (float2 *)s->amps, dU, derr, nullptr, nullptr,
                                                              nullptr, nullptr, norm_out);
    return cudaGetLastError();
}

cudaError_t tc_pipe_launch_grouped(const TcBatchDesc *descs, const TcWork *works, int nwork, unsigned long long *t0,
                                   unsigned long long *t1, int *err, cudaStream_t st)
{
    if (nwork <= 0) return cudaSuccess;
    tc_pipe_attrs();
    alignas(64) CUtensorMap tm;
    memset(&tm, 0, sizeof tm);
    TcPipeArgs none;
    memset(&none, 0, sizeof none);
    k_tc_pipe<true><<<nwork, kPThreads, kPSmem, st>>>(tm, none, nullptr, nullptr, err, descs, works, t0, t1, nullptr);
    return cudaGetLastError();
}

}  // namespace qs
