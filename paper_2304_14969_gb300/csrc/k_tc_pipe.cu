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
// Stage s is reloaded once the converters have read it; TMEM accumulator b
// is reused once the write-back of the tile before has read it. Every wait
// is bounded; a wait that gives up sets the error word and every role
// leaves its loop (loads still in flight are waited for, with a bound,
// before the CTA exits).
//
// Complex128 kets (W = true, BF16X6): the tile is the same 128 x 64
// amplitudes but 128 KB, so it is loaded as four 32 KB quarter tiles (one
// per value of the block's two highest qubits) into a ring of three stages;
// the four converter warps whose amplitudes lie in a quarter (one part, one
// warp per SM sub-partition) read it. A
// converter rounds each FP64 amplitude to FP32 (integer arithmetic on the
// IEEE encodings: FP64 instructions are scarce on this part), applies the
// phases in FP32 and writes three BF16 slices (24 bits) into the one TMEM
// A buffer (3 x 64 columns; two accumulators take the other 256). The MMA
// warp issues the six slice products a_i u_j with i + j <= 2, smallest
// first; the write-back widens FP32 to FP64 exactly and stores 16 bytes
// per amplitude. Shared memory: U slices 96 KB + 3 x 32 KB stages.
//
// Complex64 kets with 3xTF32 (KD = 2): TF32 parts take twice the bytes of
// BF16 ones, so U (hi, lo) fills 128 KB of shared memory and one A operand
// (hi, lo: 2 x 128 columns) sits in TMEM beside the two accumulators. The
// tile then comes as four 16 KB quarter tiles (the complex128 scheme: one
// per value of block bits 4, 5, read by the converter warps of one part)
// into a ring of five stages (eight full / free barrier pairs). A converter splits each amplitude x into
// hi = x rounded to TF32 and lo = x - hi (exact in FP32); the MMA warp issues
// a_hi u_hi, a_hi u_lo, a_lo u_hi as kind::tf32 (K = 8 per instruction).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "qsim_internal.h"
#include "tc_pipe_dev.cuh"
#include "tc_ptx.cuh"

namespace qs {

namespace {

constexpr int kPConvWarps = 16;              // converter warps (2 .. 17)
constexpr int kPConv = 32 * kPConvWarps;
constexpr int kPEpiWarps = 4;                // write-back warps (18 .. 21), one per TMEM lane quarter
constexpr int kPEpi = 32 * kPEpiWarps;
constexpr int kPThreads = 64 + kPConv + kPEpi;
constexpr uint32_t kPHalf = 32768;           // one BF16 operand part of 128 x 128
// per amplitude width: stage bytes, stages, U parts, loads per tile
// KD: 0 complex64 BF16x3 (whole tiles), 1 complex128 BF16X6 (quarter
// tiles), 2 complex64 3xTF32 (quarter tiles)
template <int KD> struct PipeCfg {
    static constexpr bool W = KD == 1, TF = KD == 2, QT = KD != 0;
    // a tile of complex64 / a quarter tile of complex128 / of complex64
    static constexpr uint32_t kStage = W ? 32768u : TF ? 16384u : 65536u;
    static constexpr int kNStage = W ? 3 : TF ? 5 : 2;
    static constexpr int kParts = W ? 3 : 2;                   // parts of U (and of A)
    static constexpr uint32_t kPart = TF ? 2 * kPHalf : kPHalf;   // bytes of one part of U
    static constexpr uint32_t kU = kParts * kPart;
    static constexpr int kQ = QT ? 4 : 1;                      // loads per tile
    // full / free barrier pairs: load m signals full[m % kNBar]. Quarter
    // tiles give each quarter its own pair (load m is quarter m % 4; with
    // five stages, two pairs per quarter by tile parity), so every waiter
    // sees a barrier's completions one by one in order: a barrier shared by
    // loads of different quarters would be waited on for its second
    // completion before its first (a parity wait cannot tell them apart),
    // and fewer pairs than stages let the producer's wait for a stage find
    // its barrier two completions on. With kNBar >= kNStage, issuing load
    // m + kNBar implies load m was read.
    static constexpr int kNBar = TF ? 8 : QT ? 4 : 2;
    static constexpr size_t kSmem = kU + (size_t)kNStage * kStage + 1024;
};

// IEEE binary64 -> binary32, round to nearest (ties away from zero), on the
// encodings, for magnitudes below 2^128 (amplitudes); magnitudes below
// 2^-126 become signed zero. Shifting the double's top 35 bits left by 3
// leaves its low 9 exponent bits above the 23 mantissa bits; the exponent
// bias differs by 896 = 384 (mod 512), so one subtraction rebiases them.
__device__ __forceinline__ float f64_to_f32_rn(double x)
{
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const uint32_t t = __funnelshift_l(lo, hi, 3) - (384u << 23) + ((lo >> 28) & 1u);
    const uint32_t f = (t & 0x7fffffffu) | (hi & 0x80000000u);
    return __uint_as_float(((hi >> 20) & 0x7ffu) > 896u ? f : (hi & 0x80000000u));
}

// IEEE binary32 -> binary64 (exact) on the encodings; binary32 subnormals
// (below 2^-126) become signed zero.
__device__ __forceinline__ double f32_to_f64(uint32_t f)
{
    const uint32_t hi = (((f & 0x7fffffffu) >> 3) + (896u << 20)) | (f & 0x80000000u);
    const bool nz = (f & 0x7f800000u) != 0u;
    return __hiloint2double((int)(nz ? hi : (f & 0x80000000u)), (int)(nz ? (f << 29) : 0u));
}


// TMEM column of the A part and index of the U part of product p: complex64
// a0 u0, a0 u1, a1 u0 (parts at +0, +64); complex128 a1 u1, a0 u2, a2 u0,
// a0 u1, a1 u0, a0 u0 (slices at +0, +64, +128; the smallest first)
template <bool W>
__device__ __forceinline__ uint32_t prod_a(int p)
{
    return W ? (p == 0 || p == 4 ? 64u : p == 2 ? 128u : 0u) : (p == 2 ? 64u : 0u);
}
template <bool W>
__device__ __forceinline__ uint32_t prod_u(int p)
{
    return W ? (p == 0 || p == 3 ? 1u : p == 1 ? 2u : 0u) : (p == 1 ? 1u : 0u);
}

// G = false: one block over one ket, CTAs stride over its tiles (the
// tensor map, geometry, ket and U come as parameters). G = true (complex64
// only): grouped (batched circuits): CTA i takes work entry i, a range of
// tiles of the block that descs[works[i].desc] describes, and stamps the
// circuit's first load and last store with %globaltimer. W: complex128 ket.
template <bool W> struct AmpOf { using T = float2; };
template <> struct AmpOf<true> { using T = double2; };

template <bool G, int KD>
__global__ void __launch_bounds__(kPThreads, 1)
    k_tc_pipe(const __grid_constant__ CUtensorMap tmap_param, const __grid_constant__ TcPipeArgs P_param,
              typename AmpOf<KD == 1>::T *__restrict__ a_param, const unsigned char *__restrict__ Ug_param, int *err,
              const TcBatchDesc *__restrict__ descs, const TcWork *__restrict__ works, unsigned long long *t0s,
              unsigned long long *t1s, double *norm_out)
{
    using Cfg = PipeCfg<KD>;
    constexpr bool W = Cfg::W, TF = Cfg::TF, QT = Cfg::QT;
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
    // the ket (typed and restrict-qualified: its stores may not alias the
    // shared-memory tables the write-back reads)
    typename AmpOf<W>::T *__restrict__ a = G ? (typename AmpOf<W>::T *)desc->amps : a_param;
    const unsigned char *__restrict__ Ug = G ? desc->U : Ug_param;
    const uint64_t wtile0 = G ? works[blockIdx.x].tile0 : 0, wntiles = G ? works[blockIdx.x].ntiles : 0;
    // tile of this CTA's j-th iteration
    auto tile_of = [&](uint64_t j) -> uint64_t { return G ? wtile0 + j : blockIdx.x + j * gridDim.x; };
    unsigned char *smb = (unsigned char *)(((uintptr_t)sm_dyn + 1023) & ~(uintptr_t)1023);
    unsigned char *Us = smb;                              // U operand (N x K): kParts parts of 32 KB
    unsigned char *St = smb + Cfg::kU;                    // raw stages
    __shared__ __align__(8) uint64_t bar_full[8], bar_sfree[8], bar_aready[2], bar_mma[2], bar_accf[2], bar_lofree,
        bar_loready, bar_fin;
    static_assert(Cfg::kNBar <= 8 && Cfg::kNBar >= Cfg::kNStage, "barrier pairs per stage ring");
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    __shared__ uint16_t s_posL[64];
    __shared__ uint64_t s_spL[64];
    __shared__ uint64_t s_tturn[6 * 24];
    __shared__ float2 s_gfac[6 * 128];       // [b][g]: a warp's lanes read consecutive entries
    __shared__ float2 s_E[4][6];             // tile factors of the deferred phases (tile j in slot j & 3)

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool has_pd = P.gfac != nullptr;
    for (int i = tid; i < 64; i += kPThreads) {
        s_posL[i] = P.posL[i];
        s_spL[i] = P.spL[i];
    }
    if (has_pd) {
        for (int i = tid; i < 128 * 6; i += kPThreads) s_gfac[(i % 6) * 128 + i / 6] = P.gfac[i];
        for (int i = tid; i < 6 * 24; i += kPThreads) s_tturn[i] = P.tturn[i];
    }
    {
        const int4 *src = (const int4 *)Ug;
        int4 *dst = (int4 *)Us;
        for (uint32_t i = tid; i < Cfg::kU / 16; i += kPThreads) dst[i] = src[i];
    }
    if (tid == 0) {
        s_abort = 0;
        for (int s = 0; s < Cfg::kNBar; s++) {
            // with deferred phases the producer arrives a second time once the
            // tile factors are written
            mbar_init(smem_addr(&bar_full[s]), has_pd ? 2 : 1);
            // a complex128 quarter tile is read by the four warps it belongs to
            mbar_init(smem_addr(&bar_sfree[s]), QT ? kPConv / 4 : kPConv);
        }
        // 3xTF32: the lo half of the one A operand has its own handshake
        // (lo free after the tile's first product, lo ready from the converters)
        mbar_init(smem_addr(&bar_lofree), 1);
        mbar_init(smem_addr(&bar_loready), kPConv);
        mbar_init(smem_addr(&bar_fin), 1);
        for (int b = 0; b < 2; b++) {
            mbar_init(smem_addr(&bar_aready[b]), kPConv);
            mbar_init(smem_addr(&bar_mma[b]), 1);
            mbar_init(smem_addr(&bar_accf[b]), kPEpi);
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
    // TMEM columns: accumulators [0, 128) and [128, 256); complex64: A
    // operands (hi, lo: 64 + 64 columns, BF16 pairs) [256, 384) and
    // [384, 512); complex128: one A operand (three slices) [256, 448)
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
        // deferred phases (lanes 0..5)
        if constexpr (!QT) {
            // whole tiles: tile j goes to stage j & 1 once the converters have
            // read tile j - 2
            uint64_t issued = 0;
            for (uint64_t j = 0; j < J; j++) {
                const int s = (int)(j & 1);
                int stop = 0;
                if (lane == 0) {
                    const bool ok = j < 2 || mbar_wait_or_abort(smem_addr(&bar_sfree[s]),
                                                                (uint32_t)(((j - 2) >> 1) & 1), abort_flag);
                    if (!ok) give_up();
                    stop = !ok || *abort_flag;
                }
                if (__shfl_sync(0xffffffffu, stop, 0)) break;
                const uint64_t t = tile_of(j);
                const uint32_t fb = smem_addr(&bar_full[s]);
                if (lane == 0) {
                    const uint64_t base = tile_base<13>(P, t);
                    int c[5];
#pragma unroll
                    for (int d = 0; d < 5; d++) c[d] = (int)((base >> P.dim_lo[d]) & ((1ull << P.dim_bits[d]) - 1));
                    mbar_arrive_expect_tx(fb, P.box_bytes * (uint32_t)P.nload);
                    const uint32_t dst = smem_addr(St + (size_t)s * Cfg::kStage);
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
        } else {
            // quarter tiles: load m (quarter m & 3 of tile m >> 2) goes to
            // stage m mod kNStage once the converters have read load
            // m - kNStage, and signals full[m mod kNBar]
            uint32_t m = 0;   // loads issued
            bool quit = false;
            for (uint64_t j = 0; j < J && !quit; j++) {
                const uint64_t t = tile_of(j);
                for (int q = 0; q < Cfg::kQ; q++, m++) {
                    const int s = (int)(m % Cfg::kNStage);
                    int stop = 0;
                    if (lane == 0) {
                        const uint32_t r = m - Cfg::kNStage;   // the load stage s held before
                        const bool ok = m < (uint32_t)Cfg::kNStage ||
                                        mbar_wait_or_abort(smem_addr(&bar_sfree[r % Cfg::kNBar]), (r / Cfg::kNBar) & 1u,
                                                           abort_flag);
                        if (!ok) give_up();
                        stop = !ok || *abort_flag;
                    }
                    quit = __shfl_sync(0xffffffffu, stop, 0) != 0;
                    if (quit) break;
                    const uint32_t fb = smem_addr(&bar_full[m % Cfg::kNBar]);
                    if (lane == 0) {
                        const uint64_t bq = tile_base<13>(P, t) | ((uint64_t)(q & 1) << P.qpos[0]) |
                                            ((uint64_t)(q >> 1) << P.qpos[1]);
                        int c[5];
#pragma unroll
                        for (int d = 0; d < 5; d++) c[d] = (int)((bq >> P.dim_lo[d]) & ((1ull << P.dim_bits[d]) - 1));
                        if (W) c[0] <<= 1;   // dimension 0 counts the 8-byte halves of an amplitude
                        mbar_arrive_expect_tx(fb, P.box_bytes * (uint32_t)P.nload);
                        const uint32_t dst = smem_addr(St + (size_t)s * Cfg::kStage);
                        for (int v = 0; v < P.nload; v++)
                            tma_load_5d(dst + (uint32_t)v * P.box_bytes, tmap, fb, c[0], c[1], c[2], c[3], c[4] + P.xoff[v]);
                    }
                    if (has_pd) {
                        if (q == 0) {
                            if (lane < 6) {
                                uint64_t tt = 0;
                                for (int i = 0; i < P.ntb; i++)
                                    if ((t >> i) & 1) tt += s_tturn[lane * 24 + i];
                                float sn, cs;
                                turns_sincos(tt, sn, cs);
                                s_E[j & 3][lane] = make_float2(cs, sn);
                            }
                            __syncwarp();
                        }
                        if (lane == 0) mbar_arrive(fb);
                    }
                }
            }
            // loads still in flight (only after an abort) land before the CTA
            // exits; the loads before them have been read, so these waits see
            // each barrier's completions in order
            if (lane == 0)
                for (uint32_t x = m >= (uint32_t)Cfg::kNStage ? m - Cfg::kNStage : 0; x < m; x++)
                    mbar_wait(smem_addr(&bar_full[x % Cfg::kNBar]), (x / Cfg::kNBar) & 1u);
        }
    } else if (warp == 1) {
        // ---------------- MMA issue: D[g][n] = sum_k A[g][k] U[n][k], A in TMEM
        if (lane == 0) {
            // instruction descriptor: FP32 accumulator, A and B BF16 (kind::f16)
            // or TF32 (kind::tf32), both K-major, N = 128, M = 128
            const uint32_t ab = TF ? 2u : 1u;
            const uint32_t idesc = (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(128 >> 3) << 17) |
                                   ((uint32_t)(128 >> 4) << 24);
            // U part: 8-row groups of core matrices SBO bytes apart (K = 128 elements per row)
            const uint32_t SBO = TF ? 4096u : 2048u;
            if constexpr (TF) {
                // a_lo u_hi first, then a commit that lets the converters write the
                // next tile's lo parts while a_hi u_hi and a_hi u_lo run; A hi at +0,
                // lo at +128 columns
                const uint32_t a0 = tmem + 256u, u0 = smem_addr(Us);
                bool any = false;
                for (uint64_t j = 0; j < J && !*abort_flag; j++) {
                    const int b = (int)(j & 1);
                    if (j >= 2 &&
                        !mbar_wait_or_abort(smem_addr(&bar_accf[b]), (uint32_t)(((j - 2) >> 1) & 1), abort_flag)) {
                        give_up();
                        break;
                    }
                    if (!mbar_wait_or_abort(smem_addr(&bar_loready), (uint32_t)(j & 1), abort_flag)) {
                        give_up();
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t d = tmem + (uint32_t)b * 128u;
#pragma unroll
                    for (int kk = 0; kk < 16; kk++)
                        mma_issue_tmem_a_tf32(d, a0 + 128u + (uint32_t)kk * 8u,
                                              smem_desc(u0 + (uint32_t)kk * 256u, 128u, SBO), idesc, kk ? 1u : 0u);
                    any = true;
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        smem_addr(&bar_lofree)));
                    if (!mbar_wait_or_abort(smem_addr(&bar_aready[0]), (uint32_t)(j & 1), abort_flag)) {
                        give_up();
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
                    for (int p = 0; p < 2; p++) {
#pragma unroll
                        for (int kk = 0; kk < 16; kk++)
                            mma_issue_tmem_a_tf32(d, a0 + (uint32_t)kk * 8u,
                                                  smem_desc(u0 + (uint32_t)p * Cfg::kPart + (uint32_t)kk * 256u, 128u,
                                                            SBO),
                                                  idesc, 1u);
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        smem_addr(&bar_mma[b])));
                }
                // every issued MMA completes before TMEM is released
                if (any) {
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        smem_addr(&bar_fin)));
                    mbar_wait(smem_addr(&bar_fin), 0u);
                }
            }
            uint64_t issued = 0;
            for (uint64_t j = 0; j < J && !*abort_flag && !TF; j++) {
                const int b = (int)(j & 1);
                // whole tiles: A operand b, its (j >> 1)-th fill; quarter tiles: the one A operand, its j-th
                if (!mbar_wait_or_abort(smem_addr(&bar_aready[QT ? 0 : b]),
                                        QT ? (uint32_t)(j & 1) : (uint32_t)((j >> 1) & 1), abort_flag)) {
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
                const uint32_t a0 = tmem + 256u + (QT ? 0u : (uint32_t)b * 128u);
                const uint32_t u0 = smem_addr(Us);
                uint32_t accum = 0;
#pragma unroll
                for (int p = 0; p < (W ? 6 : 3); p++) {
                    const uint32_t abase = a0 + prod_a<W>(p), bbase = u0 + prod_u<W>(p) * kPHalf;
#pragma unroll
                    for (int kk = 0; kk < 8; kk++) {
                        // K step of 16 BF16 = 8 TMEM columns of A, two core matrices of U
                        mma_issue_tmem_a(d, abase + (uint32_t)kk * 8u,
                                         smem_desc(bbase + (uint32_t)kk * 256u, 128u, SBO), idesc, accum);
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
        // is released as soon as it has been read: the time a landed tile
        // waits to be read is what bounds the load pipeline.
        const int ct = tid - 64, cw = ct >> 5;
        const int quarter = warp & 3, part = cw >> 2;
        const int g = 32 * quarter + lane;
        const uint32_t lane_off = (uint32_t)(32 * quarter) << 16;
        const int rot = P.rot_bits ? (lane >> (P.rot_shift - P.rot_bits)) & ((1 << P.rot_bits) - 1) : 0;
        // quarter tiles: this thread's amplitudes lie in quarter tile `part`
        // (block bits 4, 5); the part's warp of lane quarter 0 polls its barriers
        const int qi = QT ? part : 0;
        const bool qlead = !QT || quarter == 0;
        // in-stage byte offsets of this thread's reads (the same for every
        // tile): held in registers, except for TF32, whose split keeps 64
        // registers live and which reads them from shared memory instead
        constexpr uint32_t kEsz = W ? 16u : 8u;
        const uint32_t offG = kEsz * (uint32_t)P.posG[g];
        uint32_t offL[TF ? 1 : 16];
        if constexpr (!TF) {
#pragma unroll
            for (int i = 0; i < 16; i++) offL[i] = offG + kEsz * s_posL[16 * part + (i ^ rot)];
        }

        for (uint64_t j = 0; j < J; j++) {
            const int b = (int)(j & 1);
            const uint32_t m = QT ? (uint32_t)(4 * j + qi) : (uint32_t)j;   // the load this thread reads
            const int s = (int)(m % Cfg::kNStage), fbi = (int)(m % Cfg::kNBar);
            const uint32_t fbar = smem_addr(&bar_full[fbi]), fpar = (m / Cfg::kNBar) & 1u;
            const unsigned char *stage = St + (size_t)s * Cfg::kStage;
            float2 v[16];
            bool qbad = false;
            // Block qubits among the lowest rot_shift qubits (block bits
            // 0..rot_bits-1) would put the lanes sharing a shared-memory row
            // on one bank group: each lane reads its amplitudes in an order
            // XOR-rotated by its own lane bits, so every read instruction
            // covers distinct banks; v[] is put back in order below.
            if (!QT) {
                // one decision for all converter threads (none may be left at a barrier)
                const bool ok = mbar_wait_or_abort(fbar, fpar, abort_flag);
                if (named_bar_or(1, kPConv, !ok || *abort_flag)) {
                    give_up();
                    break;
                }
#pragma unroll
                for (int i = 0; i < 16; i++) v[i] = *(const float2 *)(stage + offL[i]);
                mbar_arrive(smem_addr(&bar_sfree[fbi]));   // the stage may be reloaded
            } else {
                // one decision per quarter tile (its four warps): the quarters
                // land one after another, and a quarter's stage must be released
                // before the next quarters can load
                const bool ok = !qlead || mbar_wait_or_abort(fbar, fpar, abort_flag);
                qbad = named_bar_or(3 + qi, kPConv / 4, !ok || *abort_flag);
                if (!qbad) {
                    (void)mbar_try_wait(fbar, fpar);
                    if constexpr (W) {
#pragma unroll
                        for (int i = 0; i < 16; i++) {
                            const double2 x = *(const double2 *)(stage + offL[i]);
                            v[i] = make_float2(f64_to_f32_rn(x.x), f64_to_f32_rn(x.y));
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < 16; i++)
                            v[i] = *(const float2 *)(stage + offG + kEsz * s_posL[16 * part + (i ^ rot)]);
                    }
                    mbar_arrive(smem_addr(&bar_sfree[fbi]));
            } else {
#pragma unroll
                    for (int i = 0; i < 16; i++) v[i] = make_float2(0.f, 0.f);
                }
            }
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
                    const float2 E = s_E[j & 3][bb], F = s_gfac[bb * 128 + g];
                    er[bb] = E.x * F.x - E.y * F.y;
                    ei[bb] = E.x * F.y + E.y * F.x;
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
                    for (int mm = 0; mm < (1 << bb); mm++) {
                        tr[mm + (1 << bb)] = tr[mm] * er[bb] - ti[mm] * ei[bb];
                        ti[mm + (1 << bb)] = tr[mm] * ei[bb] + ti[mm] * er[bb];
                    }
                }
#pragma unroll
                for (int i = 0; i < 16; i++) {
                    const float xr = v[i].x * tr[i] - v[i].y * ti[i];
                    v[i].y = v[i].x * ti[i] + v[i].y * tr[i];
                    v[i].x = xr;
                }
            }
            if constexpr (!QT) {
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
                    const uint32_t mb = smem_addr(&bar_mma[b]), mp = (uint32_t)(((j - 2) >> 1) & 1);
                    const bool ok2 = mbar_wait_or_abort(mb, mp, abort_flag);
                    if (named_bar_or(1, kPConv, !ok2 || *abort_flag)) {
                        give_up();
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                }
                const uint32_t acol = tmem + lane_off + 256u + (uint32_t)b * 128u + (uint32_t)(16 * part);
                tmem_st16(acol, hi);
                tmem_st16(acol + 64u, lo);
            } else {
                // TF32: split before waiting for the MMAs (the split overlaps
                // them; only the TMEM stores wait): hi = x rounded to TF32
                // (to nearest, ties away), lo = x - hi (exact in FP32), kept
                // in v; K index 2 l + ri of l = 16 part + i is column
                // 32 part + 2 i + ri of the part
                uint32_t hi0[16], hi1[16];
                if constexpr (TF) {
#pragma unroll
                    for (int i = 0; i < 8; i++) {
                        const uint32_t a0 = f32_to_tf32_rna(v[i].x), a1 = f32_to_tf32_rna(v[i].y);
                        const uint32_t b0 = f32_to_tf32_rna(v[8 + i].x), b1 = f32_to_tf32_rna(v[8 + i].y);
                        hi0[2 * i] = a0;
                        hi0[2 * i + 1] = a1;
                        hi1[2 * i] = b0;
                        hi1[2 * i + 1] = b1;
                        v[i] = make_float2(v[i].x - __uint_as_float(a0), v[i].y - __uint_as_float(a1));
                        v[8 + i] = make_float2(v[8 + i].x - __uint_as_float(b0), v[8 + i].y - __uint_as_float(b1));
                    }
                }
                if constexpr (TF) {
                    // lo parts first: their columns were last read by tile j - 1's
                    // first product (lo free); then the hi parts, once tile j - 1's
                    // MMAs are done (converter warp 0 polls)
                    const uint32_t acol = tmem + lane_off + 256u + (uint32_t)(32 * part);
                    uint32_t lo0[16], lo1[16];
#pragma unroll
                    for (int i = 0; i < 8; i++) {
                        lo0[2 * i] = __float_as_uint(v[i].x);
                        lo0[2 * i + 1] = __float_as_uint(v[i].y);
                        lo1[2 * i] = __float_as_uint(v[8 + i].x);
                        lo1[2 * i + 1] = __float_as_uint(v[8 + i].y);
                    }
                    const uint32_t lf = smem_addr(&bar_lofree), lp = (uint32_t)((j - 1) & 1);
                    const bool okl = !qbad && (j == 0 || cw != 0 || mbar_wait_or_abort(lf, lp, abort_flag));
                    if (named_bar_or(1, kPConv, !okl || *abort_flag)) {
                        give_up();
                        break;
                    }
                    if (j >= 1) (void)mbar_try_wait(lf, lp);
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    tmem_st16(acol + 128u, lo0);
                    tmem_st16(acol + 144u, lo1);
                    tmem_wait_st();
                    asm volatile("tcgen05.fence::before_thread_sync;");
                    mbar_arrive(smem_addr(&bar_loready));
                    const uint32_t hb = smem_addr(&bar_mma[(j - 1) & 1]), hp = (uint32_t)(((j - 1) >> 1) & 1);
                    const bool okh = j == 0 || cw != 0 || mbar_wait_or_abort(hb, hp, abort_flag);
                    if (named_bar_or(1, kPConv, !okh || *abort_flag)) {
                        give_up();
                        break;
                    }
                    if (j >= 1) (void)mbar_try_wait(hb, hp);
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    tmem_st16(acol, hi0);
                    tmem_st16(acol + 16u, hi1);
                    tmem_wait_st();
                    asm volatile("tcgen05.fence::before_thread_sync;");
                    mbar_arrive(smem_addr(&bar_aready[0]));
                    continue;
                }
                // the one A operand was last read by the MMAs of tile j - 1
                // (converter warp 0 polls)
                const uint32_t mb = smem_addr(&bar_mma[(j - 1) & 1]), mp = (uint32_t)(((j - 1) >> 1) & 1);
                const bool ok2 = !qbad && (j == 0 || cw != 0 || mbar_wait_or_abort(mb, mp, abort_flag));
                if (named_bar_or(1, kPConv, !ok2 || *abort_flag)) {
                    give_up();
                    break;
                }
                if (j >= 1) (void)mbar_try_wait(mb, mp);
                asm volatile("tcgen05.fence::after_thread_sync;");
                if constexpr (W) {
                    // three BF16 slices, each of the remainder of the ones before
                    const uint32_t acol = tmem + lane_off + 256u + (uint32_t)(16 * part);
#pragma unroll
                    for (int sl = 0; sl < 3; sl++) {
                        uint32_t pk[16];
#pragma unroll
                        for (int i = 0; i < 16; i++) {
                            const __nv_bfloat162 h = __floats2bfloat162_rn(v[i].x, v[i].y);
                            const float2 hf = __bfloat1622float2(h);
                            v[i].x -= hf.x;
                            v[i].y -= hf.y;
                            pk[i] = *(const uint32_t *)&h;
                        }
                        tmem_st16(acol + 64u * (uint32_t)sl, pk);
                    }
                }
            }
            tmem_wait_st();
            asm volatile("tcgen05.fence::before_thread_sync;");
            mbar_arrive(smem_addr(&bar_aready[QT ? 0 : b]));
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
            const uint32_t mb = smem_addr(&bar_mma[b]), mp = (uint32_t)((j >> 1) & 1);
            const bool ok = mbar_wait_or_abort(mb, mp, abort_flag);
            if (named_bar_or(2, kPEpi, !ok || *abort_flag)) {
                give_up();
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint64_t base = tile_base<13>(P, tile_of(j));
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
                auto *dstg = a + (base + spG);
                if constexpr (W) {
                    // (32-byte pair stores measured 0.4 % slower here)
#pragma unroll
                    for (int i = 0; i < 16; i++)
                        dstg[s_spL[l0 + i]] = make_double2(f32_to_f64(r[2 * i]), f32_to_f64(r[2 * i + 1]));
                } else {
                    if (P.vecw >= 2) {
                        // amplitudes l .. l + 3 adjacent: one 32-byte store per quad
#pragma unroll
                        for (int i = 0; i < 16; i += 4)
                            st_global_256(dstg + s_spL[l0 + i], r[2 * i], r[2 * i + 1], r[2 * i + 2], r[2 * i + 3],
                                          r[2 * i + 4], r[2 * i + 5], r[2 * i + 6], r[2 * i + 7]);
                    } else if (P.vecw == 1) {
                        // amplitudes l, l + 1 adjacent: one 16-byte store per pair
#pragma unroll
                        for (int i = 0; i < 16; i += 2)
                            *(float4 *)(dstg + s_spL[l0 + i]) =
                                make_float4(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]),
                                            __uint_as_float(r[2 * i + 2]), __uint_as_float(r[2 * i + 3]));
                    } else {
#pragma unroll
                        for (int i = 0; i < 16; i++)
                            dstg[s_spL[l0 + i]] =
                                make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
                    }
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
        cudaFuncSetAttribute(k_tc_pipe<false, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PipeCfg<0>::kSmem);
        cudaFuncSetAttribute(k_tc_pipe<false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PipeCfg<1>::kSmem);
        cudaFuncSetAttribute(k_tc_pipe<false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PipeCfg<2>::kSmem);
        cudaFuncSetAttribute(k_tc_pipe<true, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PipeCfg<0>::kSmem);
    });
}

cudaError_t tc_pipe_launch(qsim_state *s, const TcPipeHost &H, const unsigned char *dU, int *derr, double *norm_out)
{
    alignas(64) CUtensorMap tm;
    if (tc_pipe_encode(H, s->amps, (unsigned char *)&tm) != QSIM_OK) return cudaErrorInvalidValue;
    tc_pipe_attrs();
    const int grid = (int)std::min<uint64_t>(H.args.ntiles, (uint64_t)num_sms());
    const int kind = H.args.kind;
    if ((kind == 1) != (s->dt == QSIM_C128)) return cudaErrorInvalidValue;
    if (kind == 3) return tc_pipe7_launch(s, H, dU, derr, norm_out);
    if (kind == 1)
        k_tc_pipe<false, 1><<<grid, kPThreads, PipeCfg<1>::kSmem, s->stream>>>(
            tm, H.args, (double2 *)s->amps, dU, derr, nullptr, nullptr, nullptr, nullptr, norm_out);
    else if (kind == 2)
        k_tc_pipe<false, 2><<<grid, kPThreads, PipeCfg<2>::kSmem, s->stream>>>(
            tm, H.args, (float2 *)s->amps, dU, derr, nullptr, nullptr, nullptr, nullptr, norm_out);
    else
        k_tc_pipe<false, 0><<<grid, kPThreads, PipeCfg<0>::kSmem, s->stream>>>(
            tm, H.args, (float2 *)s->amps, dU, derr, nullptr, nullptr, nullptr, nullptr, norm_out);
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
    k_tc_pipe<true, 0><<<nwork, kPThreads, PipeCfg<0>::kSmem, st>>>(tm, none, nullptr, nullptr, err, descs, works, t0,
                                                                     t1, nullptr);
    return cudaGetLastError();
}

}  // namespace qs
