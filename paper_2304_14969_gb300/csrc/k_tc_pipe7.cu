// Pipelined tensor-core block of 7 qubits (complex64 ket, BF16x3 split),
// n >= 14: the Table I fused block at k = 7, M = 128 groups per tile.
//
// The real embedding of a 128 x 128 complex U is 256 x 256; its BF16 hi / lo
// parts (256 KB) do not fit one CTA's shared memory. Only two of its four
// blocks are distinct, so shared memory keeps Re U and Im U (hi and lo
// levels, 64 KB each) and the kernel forms, per output amplitude l' and
// group g,
//   D_re = sum_l a_re(g, l) Re U[l'][l] - a_im(g, l) Im U[l'][l]
//   D_im = sum_l a_re(g, l) Im U[l'][l] + a_im(g, l) Re U[l'][l]
// with the minus sign from the instruction descriptor's negate-A bit. Each
// product is split three ways (a_hi u_hi + a_hi u_lo + a_lo u_hi) with FP32
// accumulation in TMEM. A level stores U's rows as 64-row blocks Re 0..63,
// Im 0..63, Re 64..127, Im 64..127, so that the rows [Re_h; Im_h] of output
// half h are one 128-row operand.
//
//   tile   = 128 groups x 128 block amplitudes = 16384 complex64 (128 KB):
//            the block's 7 qubits and the 7 lowest qubits outside it,
//            loaded as eight 16 KB eighth tiles (one per value of block bits
//            4, 5, 6) into a ring of five stages (one full / free barrier
//            pair per eighth);
//   warp 0 = one thread issuing the TMA loads (and lanes 0..6 the tile
//            factors of the deferred phases);
//   warp 1 = one thread issuing the MMAs: output half h (l' = 64 h ..
//            64 h + 63) of tile j goes to TMEM slot h (D_re at +0, D_im at
//            +64 columns), K-step c = eighth c (16 amplitudes): per K-step
//            a_re [Re_h; Im_h] as one N = 128 MMA (an MMA takes as long at
//            N = 64 as at N = 128), - a_im Im_h and a_im Re_h as N = 64;
//   warps 2..17 = convert: part p (four warps, one per TMEM lane quarter)
//            reads eighths p and p + 4, applies the deferred phases and
//            writes the BF16 hi / lo parts of the real and imaginary parts
//            into A chunk c of TMEM (32 columns per eighth);
//   warps 18..21 = write back: TMEM lane = group, 64 amplitudes per half.
//
// TMEM: slots [0, 128) and [128, 256), A chunks [256, 512). Slot h of tile
// j + 1 is written once the write-back has read slot h of tile j, so one
// half's write-back overlaps the other half's MMAs; A chunk c of tile j + 1
// is written once the MMAs of tile j's second half have read chunk c. All
// waits are bounded; a wait that gives up sets the error word and every role
// leaves its loop (loads in flight land and issued MMAs complete before the
// CTA releases TMEM and exits).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "qsim_internal.h"
#include "tc_pipe_dev.cuh"
#include "tc_ptx.cuh"

namespace qs {

namespace {

constexpr int kConvWarps = 16;                 // converter warps (2 .. 17)
constexpr int kConv = 32 * kConvWarps;
constexpr int kEpiWarps = 4;                   // write-back warps (18 .. 21)
constexpr int kEpi = 32 * kEpiWarps;
constexpr int kThreads = 64 + kConv + kEpi;
constexpr uint32_t kULevel = 65536;            // one BF16 level of U: 256 rows (Re and Im) x 128 K
constexpr uint32_t kU = 2 * kULevel;           // hi, lo
constexpr uint32_t kStage = 16384;             // an eighth tile
constexpr int kNStage = 5;
constexpr int kNLoad = 8;                      // loads per tile: load m is eighth m % 8 and signals full[m % 8]
constexpr size_t kSmem = kU + (size_t)kNStage * kStage + 1024;
static_assert(kNLoad >= kNStage, "one barrier pair per eighth: issuing load m + 8 implies load m was read");

// 32 lanes x 8 consecutive 32-bit columns of tensor memory into r[].
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

__device__ __forceinline__ uint32_t bf16x2_bits(__nv_bfloat162 h) { return *(const uint32_t *)&h; }

__global__ void __launch_bounds__(kThreads, 1)
    k_tc_pipe7(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ TcPipeArgs P_param,
               float2 *__restrict__ a, const unsigned char *__restrict__ Ug, int *err, double *norm_out)
{
    extern __shared__ unsigned char sm_dyn[];
    __shared__ __align__(16) TcPipeArgs s_P;
    {
        const uint64_t *src = (const uint64_t *)&P_param;
        uint64_t *dst = (uint64_t *)&s_P;
        for (int i = threadIdx.x; i < (int)(sizeof(TcPipeArgs) / 8); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const TcPipeArgs &P = s_P;
    unsigned char *smb = (unsigned char *)(((uintptr_t)sm_dyn + 1023) & ~(uintptr_t)1023);
    unsigned char *Us = smb;            // U: hi, lo levels, each rows Re 0..63, Im 0..63, Re 64.., Im 64.. (K = l)
    unsigned char *St = smb + kU;       // raw stages
    __shared__ __align__(8) uint64_t bar_full[kNLoad], bar_sfree[kNLoad], bar_aready[8], bar_afree[8], bar_mma[2],
        bar_accf[2], bar_fin;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    __shared__ uint16_t s_posL[16];
    __shared__ uint64_t s_spL[128];
    __shared__ uint64_t s_tturn[7 * 24];
    __shared__ float2 s_gfac[7 * 128];       // [b][g]
    __shared__ float2 s_E[4][7];             // tile factors of the deferred phases (tile j in slot j & 3)

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool has_pd = P.gfac != nullptr;
    for (int i = tid; i < 16; i += kThreads) s_posL[i] = P.posL[i];
    for (int i = tid; i < 128; i += kThreads) s_spL[i] = P.spL[i];
    if (has_pd) {
        for (int i = tid; i < 128 * 7; i += kThreads) s_gfac[(i % 7) * 128 + i / 7] = P.gfac[i];
        for (int i = tid; i < 7 * 24; i += kThreads) s_tturn[i] = P.tturn[i];
    }
    {
        const int4 *src = (const int4 *)Ug;
        int4 *dst = (int4 *)Us;
        for (uint32_t i = tid; i < kU / 16; i += kThreads) dst[i] = src[i];
    }
    if (tid == 0) {
        s_abort = 0;
        for (int e = 0; e < kNLoad; e++) {
            // with deferred phases the producer arrives a second time once the
            // tile factors are written
            mbar_init(smem_addr(&bar_full[e]), has_pd ? 2 : 1);
            mbar_init(smem_addr(&bar_sfree[e]), kConv / 4);     // the four warps of one part
        }
        for (int c = 0; c < 8; c++) {
            mbar_init(smem_addr(&bar_aready[c]), kConv / 4);
            mbar_init(smem_addr(&bar_afree[c]), 1);
        }
        for (int h = 0; h < 2; h++) {
            mbar_init(smem_addr(&bar_mma[h]), 1);
            mbar_init(smem_addr(&bar_accf[h]), kEpi);
        }
        mbar_init(smem_addr(&bar_fin), 1);
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
    const uint32_t tmem = s_tmem;
    volatile int *abort_flag = &s_abort;
    auto give_up = [&]() {
        *abort_flag = 1;
        atomicExch(err, 1);
    };
    const uint64_t J = P.ntiles > blockIdx.x ? (P.ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    auto tile_of = [&](uint64_t j) -> uint64_t { return blockIdx.x + j * gridDim.x; };

    if (warp == 0) {
        // ---------------- TMA producer: load m = 8 j + e (eighth e of tile j)
        // goes to stage m mod 5 once the converters have read load m - 5
        uint32_t m = 0;
        bool quit = false;
        for (uint64_t j = 0; j < J && !quit; j++) {
            const uint64_t t = tile_of(j);
            for (int e = 0; e < kNLoad; e++, m++) {
                const int s = (int)(m % kNStage);
                int stop = 0;
                if (lane == 0) {
                    const uint32_t r = m - kNStage;
                    const bool ok = m < (uint32_t)kNStage ||
                                    mbar_wait_or_abort(smem_addr(&bar_sfree[r % kNLoad]), (r / kNLoad) & 1u, abort_flag);
                    if (!ok) give_up();
                    stop = !ok || *abort_flag;
                }
                quit = __shfl_sync(0xffffffffu, stop, 0) != 0;
                if (quit) break;
                const uint32_t fb = smem_addr(&bar_full[e]);
                if (lane == 0) {
                    const uint64_t bq = tile_base<14>(P, t) | ((uint64_t)(e & 1) << P.qpos[0]) |
                                        ((uint64_t)((e >> 1) & 1) << P.qpos[1]) | ((uint64_t)(e >> 2) << P.qpos[2]);
                    int c[5];
#pragma unroll
                    for (int d = 0; d < 5; d++) c[d] = (int)((bq >> P.dim_lo[d]) & ((1ull << P.dim_bits[d]) - 1));
                    mbar_arrive_expect_tx(fb, P.box_bytes * (uint32_t)P.nload);
                    const uint32_t dst = smem_addr(St + (size_t)s * kStage);
                    for (int v = 0; v < P.nload; v++)
                        tma_load_5d(dst + (uint32_t)v * P.box_bytes, &tmap, fb, c[0], c[1], c[2], c[3], c[4] + P.xoff[v]);
                }
                if (has_pd) {
                    if (e == 0) {
                        if (lane < 7) {
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
        // exits; the five most recent loads use five distinct barriers
        if (lane == 0)
            for (uint32_t x = m >= (uint32_t)kNStage ? m - kNStage : 0; x < m; x++)
                mbar_wait(smem_addr(&bar_full[x % kNLoad]), (x / kNLoad) & 1u);
    } else if (warp == 1) {
        // ---------------- MMA issue. An MMA costs the same time at N = 64 as
        // at N = 128, so the products of A_re take both parts of an output
        // half at once: U's rows are stored as 64-row blocks Re 0..63, Im
        // 0..63, Re 64..127, Im 64..127 (per BF16 level), so [Re_h; Im_h] is
        // one 128-row operand and slot h's D_re | D_im one N = 128
        // accumulator; the products of A_im (D_re -= a_im Im_h, D_im += a_im
        // Re_h, opposite signs) take one N = 64 MMA each.
        if (lane == 0) {
            // FP32 accumulator, A and B BF16 (kind::f16), both K-major, M = 128; bit 13 negates A
            const uint32_t id0 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(128 >> 4) << 24);
            const uint32_t id128 = id0 | ((uint32_t)(128 >> 3) << 17);
            const uint32_t id64 = id0 | ((uint32_t)(64 >> 3) << 17);
            const uint32_t id64n = id64 | (1u << 13);
            // 8-row groups 2048 bytes apart, K core matrices 128 bytes apart; the descriptor's
            // address field counts 16-byte units, so a byte offset o adds o >> 4
            const uint64_t db = smem_desc(smem_addr(Us), 128u, 2048u);
            constexpr uint32_t HI = 0, LO = kULevel >> 4, IMH = 16384u >> 4;
            bool any = false;
            for (uint64_t j = 0; j < J && !*abort_flag; j++) {
                bool bad = false;
                for (int h = 0; h < 2 && !bad; h++) {
                    if (j >= 1 && !mbar_wait_or_abort(smem_addr(&bar_accf[h]), (uint32_t)((j - 1) & 1), abort_flag)) {
                        bad = true;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t dsl = tmem + 128u * (uint32_t)h, dim = dsl + 64u;
                    const uint64_t dh = db + (uint64_t)((32768u * (uint32_t)h) >> 4);   // rows of [Re_h; Im_h]
                    for (int c = 0; c < 8; c++) {
                        if (h == 0) {
                            if (!mbar_wait_or_abort(smem_addr(&bar_aready[c]), (uint32_t)(j & 1), abort_flag)) {
                                bad = true;
                                break;
                            }
                            asm volatile("tcgen05.fence::after_thread_sync;");
                        }
                        // A chunk c: re hi +0, im hi +8, re lo +16, im lo +24 columns; K = 16 c ..
                        const uint32_t ac = tmem + 256u + 32u * (uint32_t)c;
                        const uint64_t bc = dh + (uint64_t)(16u * (uint32_t)c);
                        const uint32_t acc = c > 0 ? 1u : 0u;
                        // [D_re | D_im] += a_re [Re_h; Im_h]
                        mma_issue_tmem_a(dsl, ac + 0u, bc + HI, id128, acc);
                        mma_issue_tmem_a(dsl, ac + 0u, bc + LO, id128, 1u);
                        mma_issue_tmem_a(dsl, ac + 16u, bc + HI, id128, 1u);
                        // D_re -= a_im Im_h
                        mma_issue_tmem_a(dsl, ac + 8u, bc + HI + IMH, id64n, 1u);
                        mma_issue_tmem_a(dsl, ac + 8u, bc + LO + IMH, id64n, 1u);
                        mma_issue_tmem_a(dsl, ac + 24u, bc + HI + IMH, id64n, 1u);
                        // D_im += a_im Re_h
                        mma_issue_tmem_a(dim, ac + 8u, bc + HI, id64, 1u);
                        mma_issue_tmem_a(dim, ac + 8u, bc + LO, id64, 1u);
                        mma_issue_tmem_a(dim, ac + 24u, bc + HI, id64, 1u);
                        any = true;
                        if (h == 1)
                            asm volatile(
                                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                    smem_addr(&bar_afree[c])));
                    }
                    if (bad) break;
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        smem_addr(&bar_mma[h])));
                }
                if (bad) {
                    give_up();
                    break;
                }
            }
            // every issued MMA completes before TMEM is released
            if (any) {
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_addr(&bar_fin)));
                mbar_wait(smem_addr(&bar_fin), 0u);
            }
        }
    } else if (warp < 2 + kConvWarps) {
        // ---------------- convert (warps 2..17). A thread owns one group (its
        // TMEM lane) and, per eighth, its 16 amplitudes l = 16 c + i.
        const int cw = (tid - 64) >> 5;
        const int quarter = warp & 3, part = cw >> 2;
        const int g = 32 * quarter + lane;
        const uint32_t lane_off = (uint32_t)(32 * quarter) << 16;
        const int rot = P.rot_bits ? (lane >> (P.rot_shift - P.rot_bits)) & ((1 << P.rot_bits) - 1) : 0;
        const bool qlead = quarter == 0;   // the part's warp that polls its barriers
        const int nbar = 3 + part;         // the part's named barrier
        const uint32_t offG = 8u * (uint32_t)P.posG[g];
        uint32_t offL[16];
#pragma unroll
        for (int i = 0; i < 16; i++) offL[i] = offG + 8u * s_posL[i ^ rot];
        bool quit = false;
        for (uint64_t j = 0; j < J && !quit; j++) {
            for (int hh = 0; hh < 2; hh++) {
                const int c = part + 4 * hh;                 // eighth = A chunk
                const uint32_t m = 8u * (uint32_t)j + (uint32_t)c;
                const unsigned char *stage = St + (size_t)(m % kNStage) * kStage;
                const uint32_t fbar = smem_addr(&bar_full[c]), fpar = (uint32_t)(j & 1);
                // one decision per part (its four warps)
                const bool ok = !qlead || mbar_wait_or_abort(fbar, fpar, abort_flag);
                if (named_bar_or(nbar, kConv / 4, !ok || *abort_flag)) {
                    give_up();
                    quit = true;
                    break;
                }
                (void)mbar_try_wait(fbar, fpar);
                float2 v[16];
                // each lane reads in an order XOR-rotated by its own lane bits
                // (block qubits among the lowest four would otherwise put the
                // lanes of a shared-memory row on one bank group)
#pragma unroll
                for (int i = 0; i < 16; i++) v[i] = *(const float2 *)(stage + offL[i]);
                mbar_arrive(smem_addr(&bar_sfree[c]));   // the stage may be reloaded
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
                    // bits 4..6 of l from c, 0..3 from i
                    float er[7], ei[7];
#pragma unroll
                    for (int bb = 0; bb < 7; bb++) {
                        const float2 E = s_E[j & 3][bb], F = s_gfac[bb * 128 + g];
                        er[bb] = E.x * F.x - E.y * F.y;
                        ei[bb] = E.x * F.y + E.y * F.x;
                    }
                    float fr = 1.f, fi = 0.f;
#pragma unroll
                    for (int bb = 4; bb < 7; bb++)
                        if ((c >> (bb - 4)) & 1) {
                            const float xr = fr * er[bb] - fi * ei[bb];
                            fi = fr * ei[bb] + fi * er[bb];
                            fr = xr;
                        }
                    // factors of i = 0..7 (bits 0..2), then of i + 8 (times e_3)
                    float tr[8], ti[8];
                    tr[0] = fr;
                    ti[0] = fi;
#pragma unroll
                    for (int bb = 0; bb < 3; bb++) {
#pragma unroll
                        for (int mm = 0; mm < (1 << bb); mm++) {
                            tr[mm + (1 << bb)] = tr[mm] * er[bb] - ti[mm] * ei[bb];
                            ti[mm + (1 << bb)] = tr[mm] * ei[bb] + ti[mm] * er[bb];
                        }
                    }
#pragma unroll
                    for (int hi = 0; hi < 2; hi++) {
#pragma unroll
                        for (int i = 0; i < 8; i++) {
                            float2 &x = v[8 * hi + i];
                            const float xr = x.x * tr[i] - x.y * ti[i];
                            x.y = x.x * ti[i] + x.y * tr[i];
                            x.x = xr;
                        }
                        if (hi == 0) {
#pragma unroll
                            for (int i = 0; i < 8; i++) {
                                const float xr = tr[i] * er[3] - ti[i] * ei[3];
                                ti[i] = tr[i] * ei[3] + ti[i] * er[3];
                                tr[i] = xr;
                            }
                        }
                    }
                }
                // BF16 hi / lo of the real and imaginary parts, K pairs (2 i, 2 i + 1)
                // per TMEM column: re hi, im hi, re lo, im lo, 8 columns each
                uint32_t pk[32];
#pragma unroll
                for (int i = 0; i < 8; i++) {
                    const float2 x0 = v[2 * i], x1 = v[2 * i + 1];
                    const __nv_bfloat162 hr = __floats2bfloat162_rn(x0.x, x1.x);
                    const __nv_bfloat162 hm = __floats2bfloat162_rn(x0.y, x1.y);
                    const float2 fr = __bfloat1622float2(hr), fm = __bfloat1622float2(hm);
                    pk[i] = bf16x2_bits(hr);
                    pk[8 + i] = bf16x2_bits(hm);
                    pk[16 + i] = bf16x2_bits(__floats2bfloat162_rn(x0.x - fr.x, x1.x - fr.y));
                    pk[24 + i] = bf16x2_bits(__floats2bfloat162_rn(x0.y - fm.x, x1.y - fm.y));
                }
                // A chunk c was last read by the MMAs of tile j - 1's second half
                const uint32_t ab = smem_addr(&bar_afree[c]), apar = (uint32_t)((j - 1) & 1);
                const bool ok2 = j == 0 || !qlead || mbar_wait_or_abort(ab, apar, abort_flag);
                if (named_bar_or(nbar, kConv / 4, !ok2 || *abort_flag)) {
                    give_up();
                    quit = true;
                    break;
                }
                if (j >= 1) (void)mbar_try_wait(ab, apar);
                asm volatile("tcgen05.fence::after_thread_sync;");
                tmem_st32(tmem + lane_off + 256u + 32u * (uint32_t)c, pk);
                tmem_wait_st();
                asm volatile("tcgen05.fence::before_thread_sync;");
                mbar_arrive(smem_addr(&bar_aready[c]));
            }
        }
    } else {
        // ---------------- write back (warps 18..21): TMEM lane = group; slot
        // h holds outputs l = 64 h + l0: D_re at column l0, D_im at 64 + l0
        const int quarter = warp & 3;
        const int g = 32 * quarter + lane;
        const uint32_t lane_off = (uint32_t)(32 * quarter) << 16;
        const uint64_t spG = P.spG[g];
        double nacc = 0;   // sum of |amplitude|^2 written (norm_out): FP32 runs of 8, FP64 across runs
        bool quit = false;
        for (uint64_t j = 0; j < J && !quit; j++) {
            float2 *dstg = a + (tile_base<14>(P, tile_of(j)) + spG);
            for (int h = 0; h < 2; h++) {
                const uint32_t mb = smem_addr(&bar_mma[h]), mp = (uint32_t)(j & 1);
                const bool ok = mbar_wait_or_abort(mb, mp, abort_flag);
                if (named_bar_or(2, kEpi, !ok || *abort_flag)) {
                    give_up();
                    quit = true;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll 1
                for (int l0 = 0; l0 < 64; l0 += 8) {
                    uint32_t re[8], im[8];
                    const uint32_t col = tmem + lane_off + 128u * (uint32_t)h + (uint32_t)l0;
                    tmem_ld8(col, re);
                    tmem_ld8(col + 64u, im);
                    tmem_wait_ld();
                    if (norm_out) {
                        float run = 0.f;
                        for (int i = 0; i < 8; i++) {
                            run = fmaf(__uint_as_float(re[i]), __uint_as_float(re[i]), run);
                            run = fmaf(__uint_as_float(im[i]), __uint_as_float(im[i]), run);
                        }
                        nacc += (double)run;
                    }
                    const int lb = 64 * h + l0;
                    if (P.vecw >= 2) {
#pragma unroll
                        for (int i = 0; i < 8; i += 4)
                            st_global_256(dstg + s_spL[lb + i], re[i], im[i], re[i + 1], im[i + 1], re[i + 2],
                                          im[i + 2], re[i + 3], im[i + 3]);
                    } else if (P.vecw == 1) {
#pragma unroll
                        for (int i = 0; i < 8; i += 2)
                            *(float4 *)(dstg + s_spL[lb + i]) =
                                make_float4(__uint_as_float(re[i]), __uint_as_float(im[i]),
                                            __uint_as_float(re[i + 1]), __uint_as_float(im[i + 1]));
                    } else {
#pragma unroll
                        for (int i = 0; i < 8; i++)
                            dstg[s_spL[lb + i]] = make_float2(__uint_as_float(re[i]), __uint_as_float(im[i]));
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;");
                mbar_arrive(smem_addr(&bar_accf[h]));
            }
        }
        if (norm_out) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) nacc += __shfl_down_sync(0xffffffffu, nacc, o);
            if (lane == 0) atomicAdd(norm_out, nacc);
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

}  // namespace

cudaError_t tc_pipe7_launch(qsim_state *s, const TcPipeHost &H, const unsigned char *dU, int *derr, double *norm_out)
{
    if (s->dt != QSIM_C64 || H.args.kind != 3) return cudaErrorInvalidValue;
    alignas(64) CUtensorMap tm;
    if (tc_pipe_encode(H, s->amps, (unsigned char *)&tm) != QSIM_OK) return cudaErrorInvalidValue;
    static std::once_flag once;
    std::call_once(once, []() {
        cudaFuncSetAttribute(k_tc_pipe7, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    });
    const int grid = (int)std::min<uint64_t>(H.args.ntiles, (uint64_t)num_sms());
    k_tc_pipe7<<<grid, kThreads, kSmem, s->stream>>>(tm, H.args, (float2 *)s->amps, dU, derr, norm_out);
    return cudaGetLastError();
}

}  // namespace qs
