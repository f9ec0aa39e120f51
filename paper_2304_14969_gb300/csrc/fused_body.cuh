// Device code of a fused pass, shared by the per-pass kernel and the
// batched persistent kernel (see k_fused.cu for the design).
#pragma once

#include "plan.h"

namespace qs {

template <typename R> struct FV;
template <> struct FV<float> { using T = float2; };
template <> struct FV<double> { using T = double2; };

__device__ __forceinline__ uint32_t swz(uint32_t t, float2 *) { return t ^ (((t >> 4) ^ (t >> 8) ^ (t >> 12)) & 15u); }
__device__ __forceinline__ uint32_t swz(uint32_t t, double2 *)
{
    return t ^ (((t >> 3) ^ (t >> 6) ^ (t >> 9) ^ (t >> 12)) & 7u);
}

__device__ __forceinline__ void tsincos(uint64_t tt, float &s, float &c)
{
    float f = (float)(int64_t)tt * 5.42101086242752217e-20f;  // turns in [-0.5, 0.5)
    sincospif(2.0f * f, &s, &c);
}
__device__ __forceinline__ void tsincos(uint64_t tt, double &s, double &c)
{
    double f = (double)(int64_t)tt * 5.42101086242752217e-20;
    sincospi(2.0 * f, &s, &c);
}

template <typename V, typename R>
__device__ __forceinline__ V cmul(V a, R br, R bi)
{
    V o;
    o.x = a.x * br - a.y * bi;
    o.y = a.x * bi + a.y * br;
    return o;
}

// ---- register ops (J: register bit, compile time)

// Dense 2x2 on register bit J (form UF) after multiplying every amplitude
// with bit J set by its prefactor (PR: none, D[xr], or f * D[xr]; xr =
// register index without bit J). UF: U_NONE pure phase, U_REAL 4 reals,
// U_CPLX 4 complex, U_ANTI anti-diagonal (2 complex), U_HAD (p + q, p - q).
template <int J, int UF, int PR, int NR, typename V, typename R>
__device__ __forceinline__ void op_g1f(V (&v)[NR], const R *__restrict__ u, R fr, R fi, const R *__restrict__ D)
{
    if constexpr ((1 << J) < NR && !(UF == U_NONE && PR == PRE_NONE)) {
        R a0 = 0, a1 = 0, b0 = 0, b1 = 0, c0 = 0, c1 = 0, d0 = 0, d1 = 0;
        if constexpr (UF == U_REAL) {
            a0 = u[0]; b0 = u[1]; c0 = u[2]; d0 = u[3];
        } else if constexpr (UF == U_CPLX) {
            a0 = u[0]; a1 = u[1]; b0 = u[2]; b1 = u[3]; c0 = u[4]; c1 = u[5]; d0 = u[6]; d1 = u[7];
        } else if constexpr (UF == U_ANTI) {
            b0 = u[0]; b1 = u[1]; c0 = u[2]; c1 = u[3];
        }
#pragma unroll
        for (int x = 0; x < NR; x++) {
            if (x & (1 << J)) continue;
            const int xr = ((x >> (J + 1)) << J) | (x & ((1 << J) - 1));
            V p = v[x], q = v[x | (1 << J)];
            if constexpr (UF == U_HAD && PR != PRE_NONE) {
                // butterfly with the prefactor F folded in: o0 = p + F q in four
                // FMAs, o1 = p - F q = 2 p - o0 in two
                R Fr = D[2 * xr], Fi = D[2 * xr + 1];
                if constexpr (PR == PRE_FD) {
                    const R dr = Fr;
                    Fr = fr * dr - fi * Fi;
                    Fi = fr * Fi + fi * dr;
                }
                V o0, o1;
                o0.x = fma(Fr, q.x, fma(-Fi, q.y, p.x));
                o0.y = fma(Fr, q.y, fma(Fi, q.x, p.y));
                o1.x = fma((R)2, p.x, -o0.x);
                o1.y = fma((R)2, p.y, -o0.y);
                v[x] = o0;
                v[x | (1 << J)] = o1;
                continue;
            }
            if constexpr (PR == PRE_D) {
                q = cmul(q, D[2 * xr], D[2 * xr + 1]);
            } else if constexpr (PR == PRE_FD) {
                const R dr = D[2 * xr], di = D[2 * xr + 1];
                q = cmul(q, fr * dr - fi * di, fr * di + fi * dr);
            }
            if constexpr (UF == U_NONE) {
                v[x | (1 << J)] = q;
            } else if constexpr (UF == U_HAD) {
                V o0, o1;
                o0.x = p.x + q.x;
                o0.y = p.y + q.y;
                o1.x = p.x - q.x;
                o1.y = p.y - q.y;
                v[x] = o0;
                v[x | (1 << J)] = o1;
            } else if constexpr (UF == U_REAL) {
                V o0, o1;
                o0.x = a0 * p.x + b0 * q.x;
                o0.y = a0 * p.y + b0 * q.y;
                o1.x = c0 * p.x + d0 * q.x;
                o1.y = c0 * p.y + d0 * q.y;
                v[x] = o0;
                v[x | (1 << J)] = o1;
            } else if constexpr (UF == U_CPLX) {
                V o0, o1;
                o0.x = a0 * p.x - a1 * p.y + b0 * q.x - b1 * q.y;
                o0.y = a0 * p.y + a1 * p.x + b0 * q.y + b1 * q.x;
                o1.x = c0 * p.x - c1 * p.y + d0 * q.x - d1 * q.y;
                o1.y = c0 * p.y + c1 * p.x + d0 * q.y + d1 * q.x;
                v[x] = o0;
                v[x | (1 << J)] = o1;
            } else {
                v[x] = cmul(q, b0, b1);
                v[x | (1 << J)] = cmul(p, c0, c1);
            }
        }
    }
}

template <int J0, int J1, int NR, typename V, typename R>
__device__ __forceinline__ void op_g2(V (&v)[NR], const R *__restrict__ u)
{
    if constexpr ((1 << J0) < NR && (1 << J1) < NR && J0 != J1) {
#pragma unroll
        for (int x = 0; x < NR; x++) {
            if ((x & (1 << J0)) || (x & (1 << J1))) continue;
            const int id[4] = {x, x | (1 << J0), x | (1 << J1), x | (1 << J0) | (1 << J1)};
            V in[4];
#pragma unroll
            for (int k = 0; k < 4; k++) in[k] = v[id[k]];
#pragma unroll
            for (int r = 0; r < 4; r++) {
                // one matrix row at a time keeps the live coefficient set small
                asm volatile("" ::: "memory");
                R orr = 0, oi = 0;
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    R ur = u[2 * (r * 4 + k)], ui = u[2 * (r * 4 + k) + 1];
                    orr += ur * in[k].x - ui * in[k].y;
                    oi += ur * in[k].y + ui * in[k].x;
                }
                v[id[r]].x = orr;
                v[id[r]].y = oi;
            }
        }
    }
}

template <int J0, int J1, int NR, typename V, typename R>
__device__ __forceinline__ void op_g2m(V (&v)[NR], const R *__restrict__ u, int perm)
{
    if constexpr ((1 << J0) < NR && (1 << J1) < NR && J0 != J1) {
        int pr[4];
        R cr[4], ci[4];
#pragma unroll
        for (int r = 0; r < 4; r++) {
            pr[r] = (perm >> (2 * r)) & 3;
            cr[r] = u[2 * r];
            ci[r] = u[2 * r + 1];
        }
#pragma unroll
        for (int x = 0; x < NR; x++) {
            if ((x & (1 << J0)) || (x & (1 << J1))) continue;
            const int id[4] = {x, x | (1 << J0), x | (1 << J1), x | (1 << J0) | (1 << J1)};
            const V a0 = v[id[0]], a1 = v[id[1]], a2 = v[id[2]], a3 = v[id[3]];
#pragma unroll
            for (int r = 0; r < 4; r++) {
                V src = pr[r] == 0 ? a0 : pr[r] == 1 ? a1 : pr[r] == 2 ? a2 : a3;
                v[id[r]] = cmul(src, cr[r], ci[r]);
            }
        }
    }
}

#define QS_CASE1(J, CALL) \
    case J:               \
        CALL(J);          \
        break;
#define QS_SWITCH1(j, CALL) \
    switch (j) { QS_CASE1(0, CALL) QS_CASE1(1, CALL) QS_CASE1(2, CALL) QS_CASE1(3, CALL) QS_CASE1(4, CALL) }
#define QS_SWITCHG(j, CALL) \
    switch (j) { \
    case 0: CALL(0, 0, 0); break; \
    case 1: CALL(0, 0, 1); break; \
    case 2: CALL(0, 0, 2); break; \
    case 3: CALL(0, 1, 0); break; \
    case 4: CALL(0, 1, 1); break; \
    case 5: CALL(0, 1, 2); break; \
    case 6: CALL(0, 2, 0); break; \
    case 7: CALL(0, 2, 1); break; \
    case 8: CALL(0, 2, 2); break; \
    case 9: CALL(0, 3, 0); break; \
    case 10: CALL(0, 3, 1); break; \
    case 11: CALL(0, 3, 2); break; \
    case 12: CALL(0, 4, 0); break; \
    case 13: CALL(0, 4, 1); break; \
    case 14: CALL(0, 4, 2); break; \
    case 16: CALL(1, 0, 0); break; \
    case 17: CALL(1, 0, 1); break; \
    case 18: CALL(1, 0, 2); break; \
    case 19: CALL(1, 1, 0); break; \
    case 20: CALL(1, 1, 1); break; \
    case 21: CALL(1, 1, 2); break; \
    case 22: CALL(1, 2, 0); break; \
    case 23: CALL(1, 2, 1); break; \
    case 24: CALL(1, 2, 2); break; \
    case 25: CALL(1, 3, 0); break; \
    case 26: CALL(1, 3, 1); break; \
    case 27: CALL(1, 3, 2); break; \
    case 28: CALL(1, 4, 0); break; \
    case 29: CALL(1, 4, 1); break; \
    case 30: CALL(1, 4, 2); break; \
    case 32: CALL(2, 0, 0); break; \
    case 33: CALL(2, 0, 1); break; \
    case 34: CALL(2, 0, 2); break; \
    case 35: CALL(2, 1, 0); break; \
    case 36: CALL(2, 1, 1); break; \
    case 37: CALL(2, 1, 2); break; \
    case 38: CALL(2, 2, 0); break; \
    case 39: CALL(2, 2, 1); break; \
    case 40: CALL(2, 2, 2); break; \
    case 41: CALL(2, 3, 0); break; \
    case 42: CALL(2, 3, 1); break; \
    case 43: CALL(2, 3, 2); break; \
    case 44: CALL(2, 4, 0); break; \
    case 45: CALL(2, 4, 1); break; \
    case 46: CALL(2, 4, 2); break; \
    case 48: CALL(3, 0, 0); break; \
    case 49: CALL(3, 0, 1); break; \
    case 50: CALL(3, 0, 2); break; \
    case 51: CALL(3, 1, 0); break; \
    case 52: CALL(3, 1, 1); break; \
    case 53: CALL(3, 1, 2); break; \
    case 54: CALL(3, 2, 0); break; \
    case 55: CALL(3, 2, 1); break; \
    case 56: CALL(3, 2, 2); break; \
    case 57: CALL(3, 3, 0); break; \
    case 58: CALL(3, 3, 1); break; \
    case 59: CALL(3, 3, 2); break; \
    case 60: CALL(3, 4, 0); break; \
    case 61: CALL(3, 4, 1); break; \
    case 62: CALL(3, 4, 2); break; \
    case 64: CALL(4, 0, 0); break; \
    case 65: CALL(4, 0, 1); break; \
    case 66: CALL(4, 0, 2); break; \
    case 67: CALL(4, 1, 0); break; \
    case 68: CALL(4, 1, 1); break; \
    case 69: CALL(4, 1, 2); break; \
    case 70: CALL(4, 2, 0); break; \
    case 71: CALL(4, 2, 1); break; \
    case 72: CALL(4, 2, 2); break; \
    case 73: CALL(4, 3, 0); break; \
    case 74: CALL(4, 3, 1); break; \
    case 75: CALL(4, 3, 2); break; \
    case 76: CALL(4, 4, 0); break; \
    case 77: CALL(4, 4, 1); break; \
    case 78: CALL(4, 4, 2); break; \
    }
#define QS_CASE2(A, B, CALL) \
    case A * 8 + B:          \
        CALL(A, B);          \
        break;
#define QS_SWITCH2(j, CALL)                                                                                  \
    switch (j) {                                                                                             \
        QS_CASE2(0, 1, CALL) QS_CASE2(0, 2, CALL) QS_CASE2(0, 3, CALL) QS_CASE2(0, 4, CALL)                  \
        QS_CASE2(1, 0, CALL) QS_CASE2(1, 2, CALL) QS_CASE2(1, 3, CALL) QS_CASE2(1, 4, CALL)                  \
        QS_CASE2(2, 0, CALL) QS_CASE2(2, 1, CALL) QS_CASE2(2, 3, CALL) QS_CASE2(2, 4, CALL)                  \
        QS_CASE2(3, 0, CALL) QS_CASE2(3, 1, CALL) QS_CASE2(3, 2, CALL) QS_CASE2(3, 4, CALL)                  \
        QS_CASE2(4, 0, CALL) QS_CASE2(4, 1, CALL) QS_CASE2(4, 2, CALL) QS_CASE2(4, 3, CALL)                  \
    }


// One tile of a fused pass: load 2^t amplitudes (lanes on the low 5
// qubits), run the pass's ops on register bits, store. Every thread of the
// CTA calls it (it holds barriers); threads beyond 2^(t - RB) only take part
// in the barriers. `stg` is the pass's staged constant block.
template <typename R, int RB>
__device__ __forceinline__ void fused_tile(typename FV<R>::T *__restrict__ a, const FPassDev &P, uint64_t tile,
                                           unsigned char *smraw, R *E, const unsigned char *stg,
                                           const int *s_hq, const int *s_pos)
{
    using V = typename FV<R>::T;
    constexpr int NR = 1 << RB;
    V *sm = (V *)smraw;
    const R *cf = (const R *)(stg + P.off_cf);
    const FOp *ops = (const FOp *)(stg + P.off_ops);
    const FMap *maps = (const FMap *)(stg + P.off_maps);
    const int32_t *lin_off = (const int32_t *)(stg + P.off_lin);
    const int32_t *ext_bit = (const int32_t *)(stg + P.off_eb);
    const uint64_t *ext_tw = (const uint64_t *)(stg + P.off_et);
    const int c = P.c;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool active = tid < (1 << (P.t - P.RB));

        uint64_t base = tile << c;
        for (int j = 0; j < P.ins.npos; j++) {
            int p = s_pos[j];
            base = ((base >> p) << (p + 1)) | (base & ((1ull << p) - 1));
        }
        for (int l = tid; l < P.nlin; l += blockDim.x) {
            uint64_t sacc = 0;
            for (int e = lin_off[l]; e < lin_off[l + 1]; e++)
                if ((base >> ext_bit[e]) & 1) sacc += ext_tw[e];
            R sn, cs;
            tsincos(sacc, sn, cs);
            E[2 * l] = cs;
            E[2 * l + 1] = sn;
        }
        const FMap *mp = &maps[0];
        uint32_t tthr = 0;
        uint64_t pthr = 0;
        auto thread_bits = [&]() {
            tthr = 0;
            pthr = 0;
#pragma unroll
            for (int l = 0; l < 5; l++)
                if ((lane >> l) & 1) {
                    int tb = mp->lane[l];
                    tthr |= 1u << tb;
                    pthr |= 1ull << (tb < c ? tb : s_hq[tb - c]);
                }
            for (int w = 0; w < P.W; w++)
                if ((warp >> w) & 1) {
                    int tb = mp->warp[w];
                    tthr |= 1u << tb;
                    pthr |= 1ull << (tb < c ? tb : s_hq[tb - c]);
                }
        };
        thread_bits();
        V v[NR];
        if (active) {
            const V *src = a + (base | pthr);
#pragma unroll
            for (int x = 0; x < NR; x++) v[x] = src[mp->preg[x]];
        }
        __syncthreads();   // E ready

        for (int i = 0; i < P.nops; i++) {
            const FOp op = ops[i];
            const R *u = cf + op.coef;
            if (!active && op.kind != FO_XPOSE) continue;
            switch (op.kind) {
            case FO_G1F: {
                const int uf = op.j1 & 15, pr = op.j1 >> 4;
                R fr = 1, fi = 0;
                if (pr == PRE_FD) {
                    fr = cf[op.aux4];
                    fi = cf[op.aux4 + 1];
                    if (op.aux >= 0) {
                        const R tr = cf[op.aux + 2 * tid], ti = cf[op.aux + 2 * tid + 1];
                        const R xr = fr * tr - fi * ti;
                        fi = fr * ti + fi * tr;
                        fr = xr;
                    }
                    if (op.aux2 >= 0) {
                        const R er = E[2 * op.aux2], ei = E[2 * op.aux2 + 1];
                        const R xr = fr * er - fi * ei;
                        fi = fr * ei + fi * er;
                        fr = xr;
                    }
                }
                const R *D = cf + (op.aux3 >= 0 ? op.aux3 : 0);
#define QS_C(J, UF, PR) op_g1f<J, UF, PR>(v, u, fr, fi, D)
                QS_SWITCHG(op.j0 * 16 + uf * 3 + pr, QS_C)
#undef QS_C
                break;
            }
            case FO_RSCALE: {
                const R sc = u[0];
#pragma unroll
                for (int x = 0; x < NR; x++) {
                    v[x].x *= sc;
                    v[x].y *= sc;
                }
                break;
            }
            case FO_G2: {
                // dense 4x4 ops are planned only for kernels with <= 16 registers
                // of amplitudes per thread (register pressure)
                if constexpr (RB <= 4) {
#define QS_C(A, B) op_g2<A, B>(v, u)
                    QS_SWITCH2(op.j0 * 8 + op.j1, QS_C)
#undef QS_C
                }
                break;
            }
            case FO_G2M: {
#define QS_C(A, B) op_g2m<A, B>(v, u, op.aux)
                QS_SWITCH2(op.j0 * 8 + op.j1, QS_C)
#undef QS_C
                break;
            }
            case FO_SCALE: {
                const R cr = u[0], ci = u[1];
#pragma unroll
                for (int x = 0; x < NR; x++) v[x] = cmul(v[x], cr, ci);
                break;
            }
            case FO_XPOSE: {
                uint32_t sw = swz(tthr, (V *)nullptr);
                if (active) {
#pragma unroll
                    for (int x = 0; x < NR; x++) sm[sw ^ mp->tsw[x]] = v[x];
                }
                __syncthreads();
                mp = &maps[op.aux];
                thread_bits();
                sw = swz(tthr, (V *)nullptr);
                if (active) {
#pragma unroll
                    for (int x = 0; x < NR; x++) v[x] = sm[sw ^ mp->tsw[x]];
                }
                __syncthreads();
                break;
            }
            default:
                break;
            }
        }
        if (active) {
            V *dst = a + (base | pthr);
#pragma unroll
            for (int x = 0; x < NR; x++) dst[mp->preg[x]] = v[x];
        }
    }

}  // namespace qs
