// Fused pass kernel (SIMT, register-resident tiles) and plan execution.
//
// One CTA per tile of 2^t amplitudes. Each thread holds 2^RB amplitudes in
// registers; lanes and warps index the other tile bits according to the
// current phase map. The tile is read from HBM once (lanes on the 5 lowest
// physical qubits, so each warp load is a contiguous 32-amplitude run),
// every gate of the pass is applied to register bits, phases change by one
// transpose through swizzled shared memory, and the tile is written back
// once. Diagonal terms arrive as per-thread phase factors (LINR) built from
// fixed-point turns (exact modulo one turn), a per-thread table for the
// lane/warp partners and a per-CTA sum for partners outside the tile.
#include <algorithm>
#include <cstring>

#include "plan.h"

namespace qs {

qsim_status plan_build(const qsim_circuit *cir, qsim_dtype dt, const qsim_run_opts *opts, qsim_plan *P);
qsim_status validate_circuit(const qsim_circuit *c);
qsim_status apply_one_gate(qsim_state *s, const qsim_gate &g, const double *pool, int64_t pool_len, bool relabel);

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
template <int J, int NR, typename V, typename R>
__device__ __forceinline__ void op_g1(V (&v)[NR], const R *__restrict__ u)
{
    if constexpr ((1 << J) < NR) {
        const R a0 = u[0], a1 = u[1], b0 = u[2], b1 = u[3], c0 = u[4], c1 = u[5], d0 = u[6], d1 = u[7];
#pragma unroll
        for (int x = 0; x < NR; x++) {
            if (x & (1 << J)) continue;
            V p = v[x], q = v[x | (1 << J)], o0, o1;
            o0.x = a0 * p.x - a1 * p.y + b0 * q.x - b1 * q.y;
            o0.y = a0 * p.y + a1 * p.x + b0 * q.y + b1 * q.x;
            o1.x = c0 * p.x - c1 * p.y + d0 * q.x - d1 * q.y;
            o1.y = c0 * p.y + c1 * p.x + d0 * q.y + d1 * q.x;
            v[x] = o0;
            v[x | (1 << J)] = o1;
        }
    }
}

template <int J, int NR, typename V, typename R>
__device__ __forceinline__ void op_g1r(V (&v)[NR], const R *__restrict__ u)
{
    if constexpr ((1 << J) < NR) {
        const R a = u[0], b = u[1], c = u[2], d = u[3];
#pragma unroll
        for (int x = 0; x < NR; x++) {
            if (x & (1 << J)) continue;
            V p = v[x], q = v[x | (1 << J)], o0, o1;
            o0.x = a * p.x + b * q.x;
            o0.y = a * p.y + b * q.y;
            o1.x = c * p.x + d * q.x;
            o1.y = c * p.y + d * q.y;
            v[x] = o0;
            v[x | (1 << J)] = o1;
        }
    }
}

template <int J, int NR, typename V, typename R>
__device__ __forceinline__ void op_g1x(V (&v)[NR], const R *__restrict__ u)
{
    if constexpr ((1 << J) < NR) {
        const R b0 = u[0], b1 = u[1], c0 = u[2], c1 = u[3];
#pragma unroll
        for (int x = 0; x < NR; x++) {
            if (x & (1 << J)) continue;
            V p = v[x], q = v[x | (1 << J)];
            v[x] = cmul(q, b0, b1);
            v[x | (1 << J)] = cmul(p, c0, c1);
        }
    }
}

template <int J, int NR, typename V, typename R>
__device__ __forceinline__ void op_lin(V (&v)[NR], R c, R s)
{
    if constexpr ((1 << J) < NR) {
#pragma unroll
        for (int x = 0; x < NR; x++)
            if (x & (1 << J)) v[x] = cmul(v[x], c, s);
    }
}

template <int J0, int J1, int NR, typename V, typename R>
__device__ __forceinline__ void op_diagr(V (&v)[NR], R c, R s)
{
    if constexpr ((1 << J0) < NR && (1 << J1) < NR && J0 != J1) {
#pragma unroll
        for (int x = 0; x < NR; x++)
            if ((x & (1 << J0)) && (x & (1 << J1))) v[x] = cmul(v[x], c, s);
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


template <typename R, int RB, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_fused_pass(typename FV<R>::T *__restrict__ a, FPassDev P,
                                                         uint64_t ntiles)
{
    using V = typename FV<R>::T;
    constexpr int NR = 1 << RB;
    extern __shared__ __align__(16) unsigned char smraw[];
    V *sm = (V *)smraw;
    const size_t tile_bytes = (size_t)sizeof(V) << P.t;
    // per-CTA sums of the LINR ops' partners outside the tile
    uint64_t *E = (uint64_t *)(smraw + tile_bytes);
    // the pass's constant block (ops, coefficients, turns, maps, partners)
    unsigned char *stg = smraw + tile_bytes + (((size_t)P.nlin * 8 + 15) & ~(size_t)15);
    __shared__ int s_hq[kMaxTile], s_pos[12];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    {
        const int4 *src = (const int4 *)P.stage;
        int4 *dst = (int4 *)stg;
        for (int i = tid; i < P.stage_bytes / 16; i += blockDim.x) dst[i] = src[i];
        if (tid < kMaxTile) s_hq[tid] = P.hq[tid];
        if (tid < 12) s_pos[tid] = P.ins.pos[tid];
    }
    const uint64_t *tw = (const uint64_t *)(stg + P.off_tw);
    const R *cf = (const R *)(stg + P.off_cf);
    const FOp *ops = (const FOp *)(stg + P.off_ops);
    const FMap *maps = (const FMap *)(stg + P.off_maps);
    const int32_t *lin_off = (const int32_t *)(stg + P.off_lin);
    const int32_t *ext_bit = (const int32_t *)(stg + P.off_eb);
    const uint64_t *ext_tw = (const uint64_t *)(stg + P.off_et);
    const int c = P.c;

    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        __syncthreads();   // staging done / previous tile finished with E and sm
        uint64_t base = tile << c;
        for (int j = 0; j < P.ins.npos; j++) {
            int p = s_pos[j];
            base = ((base >> p) << (p + 1)) | (base & ((1ull << p) - 1));
        }
        for (int l = tid; l < P.nlin; l += blockDim.x) {
            uint64_t sacc = 0;
            for (int e = lin_off[l]; e < lin_off[l + 1]; e++)
                if ((base >> ext_bit[e]) & 1) sacc += ext_tw[e];
            E[l] = sacc;
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
        {
            const V *src = a + (base | pthr);
#pragma unroll
            for (int x = 0; x < NR; x++) v[x] = src[mp->preg[x]];
        }
        __syncthreads();   // E ready

        for (int i = 0; i < P.nops; i++) {
            const FOp op = ops[i];
            const R *u = cf + op.coef;
            switch (op.kind) {
            case FO_G1: {
#define QS_C(J) op_g1<J>(v, u)
                QS_SWITCH1(op.j0, QS_C)
#undef QS_C
                break;
            }
            case FO_G1R: {
#define QS_C(J) op_g1r<J>(v, u)
                QS_SWITCH1(op.j0, QS_C)
#undef QS_C
                break;
            }
            case FO_G1X: {
#define QS_C(J) op_g1x<J>(v, u)
                QS_SWITCH1(op.j0, QS_C)
#undef QS_C
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
            case FO_DIAGR: {
                const R cr = u[0], ci = u[1];
                int jj = op.j0 * 8 + op.j1;
#define QS_C(A, B) op_diagr<A, B>(v, cr, ci)
                QS_SWITCH2(jj, QS_C)
#undef QS_C
                break;
            }
            case FO_LINR: {
                uint64_t tt = tw[op.coef] + E[op.aux2];
                if (op.aux >= 0) tt += tw[op.aux + tid];
                R sn, cs;
                tsincos(tt, sn, cs);
#define QS_C(J) op_lin<J>(v, cs, sn)
                QS_SWITCH1(op.j0, QS_C)
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
#pragma unroll
                for (int x = 0; x < NR; x++) sm[sw ^ mp->tsw[x]] = v[x];
                __syncthreads();
                mp = &maps[op.aux];
                thread_bits();
                sw = swz(tthr, (V *)nullptr);
#pragma unroll
                for (int x = 0; x < NR; x++) v[x] = sm[sw ^ mp->tsw[x]];
                __syncthreads();
                break;
            }
            default:
                break;
            }
        }
        {
            V *dst = a + (base | pthr);
#pragma unroll
            for (int x = 0; x < NR; x++) dst[mp->preg[x]] = v[x];
        }
    }
}

// ------------------------------------------------------------- host

namespace {

template <typename T>
size_t push_bytes(std::vector<unsigned char> &buf, const std::vector<T> &v)
{
    size_t off = (buf.size() + 255) & ~(size_t)255;
    buf.resize(off + v.size() * sizeof(T));
    if (!v.empty()) memcpy(buf.data() + off, v.data(), v.size() * sizeof(T));
    return off;
}

qsim_status plan_upload(qsim_plan *P)
{
    std::vector<unsigned char> buf;
    std::vector<size_t> offs;
    for (PlanPass &ps : P->passes) {
        size_t off = (buf.size() + 255) & ~(size_t)255;
        buf.resize(off + ps.stage.size());
        if (!ps.stage.empty()) memcpy(buf.data() + off, ps.stage.data(), ps.stage.size());
        offs.push_back(off);
    }
    if (buf.empty()) buf.resize(256);
    QS_CUDA(cudaMalloc(&P->dmem, buf.size()));
    P->dbytes = buf.size();
    QS_CUDA(cudaMemcpy(P->dmem, buf.data(), buf.size(), cudaMemcpyHostToDevice));
    for (size_t i = 0; i < P->passes.size(); i++)
        P->passes[i].dev.stage = (const unsigned char *)P->dmem + offs[i];
    return QSIM_OK;
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

template <typename R, int RB, int NT, int MINB>
cudaError_t launch_pass_t(void *amps, const FPassDev &d, cudaStream_t st)
{
    using V = typename FV<R>::T;
    size_t smem = ((size_t)sizeof(V) << d.t) + (((size_t)d.nlin * 8 + 15) & ~(size_t)15) + d.stage_bytes;
    if (smem > 220 * 1024) return cudaErrorInvalidValue;
    auto kern = k_fused_pass<R, RB, NT, MINB>;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        attr = true;
    }
    uint64_t ntiles = 1ull << (d.n - d.t);
    int threads = 1 << (d.t - d.RB);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
    if (occ < 1) occ = 1;
    uint64_t grid = std::min<uint64_t>(ntiles, (uint64_t)num_sms() * occ);
    kern<<<(unsigned)grid, threads, smem, st>>>((V *)amps, d, ntiles);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fused_pass(qsim_state *s, const FPassDev &d)
{
    const int threads = 1 << (d.t - d.RB);
    if (s->dt == QSIM_C64) {
        if (d.RB == 5)
            return threads <= 256 ? launch_pass_t<float, 5, 256, 2>(s->amps, d, s->stream)
                                  : launch_pass_t<float, 5, 512, 1>(s->amps, d, s->stream);
        return threads <= 512 ? launch_pass_t<float, 4, 512, 1>(s->amps, d, s->stream)
                              : launch_pass_t<float, 4, 1024, 1>(s->amps, d, s->stream);
    }
    return threads <= 256 ? launch_pass_t<double, 4, 256, 1>(s->amps, d, s->stream)
                          : launch_pass_t<double, 4, 512, 1>(s->amps, d, s->stream);
}

}  // namespace qs

using namespace qs;

extern "C" {

qsim_status qsim_plan_create(const qsim_circuit *c, qsim_dtype dt, const qsim_run_opts *opts, qsim_plan **out)
{
    clear_error();
    if (!out) return fail(QSIM_E_INVAL, "out is NULL");
    *out = nullptr;
    QS_TRY(validate_circuit(c));
    if (dt != QSIM_C64 && dt != QSIM_C128) return fail(QSIM_E_INVAL, "unknown dtype");
    if (opts && opts->prec != QSIM_PREC_NATIVE)
        return fail(QSIM_E_UNSUPPORTED, "tensor-core fused plans are not available in this build");
    qsim_plan *P = new qsim_plan();
    qsim_status st = plan_build(c, dt, opts, P);
    if (st != QSIM_OK) {
        if (P->dmem) cudaFree(P->dmem);
        delete P;
        return st;
    }
    *out = P;
    return QSIM_OK;
}

qsim_status qsim_plan_destroy(qsim_plan *p)
{
    if (!p) return QSIM_OK;
    if (p->dmem) {
        cudaDeviceSynchronize();
        cudaFree(p->dmem);
    }
    delete p;
    return QSIM_OK;
}

qsim_status qsim_plan_info(const qsim_plan *p, int64_t info[8])
{
    clear_error();
    if (!p || !info) return fail(QSIM_E_INVAL, "NULL argument");
    info[0] = (int64_t)p->passes.size();
    info[1] = p->ngates;
    info[2] = p->ndense;
    info[3] = p->nswaps;
    info[4] = p->t;
    info[5] = p->c;
    info[6] = p->npergate;
    int64_t xp = 0;
    for (const FOp &o : p->ops) xp += (o.kind == FO_XPOSE);
    info[7] = xp;
    return QSIM_OK;
}

qsim_status qsim_plan_execute(qsim_state *s, const qsim_plan *p)
{
    clear_error();
    if (!s || !s->amps || !p) return fail(QSIM_E_INVAL, "NULL argument");
    if (p->n != s->n || p->dt != s->dt) return fail(QSIM_E_INVAL, "plan and state differ in n or dtype");
    if (!p->dmem && !p->passes.empty()) QS_TRY(plan_upload(const_cast<qsim_plan *>(p)));
    QS_TRY(qsim_materialize(s));
    for (const PlanStep &st : p->steps) {
        if (st.kind == 0) {
            QS_CUDA(launch_fused_pass(s, p->passes[st.pass].dev));
        } else if (st.kind == 1) {
            const qsim_gate &g = st.gate;
            if (g.kind == QSIM_G_CP) {
                QS_CUDA(launch_cphase(s, g.q0, g.q1, g.params[0]));
            } else {
                uint64_t cmask = 0, cval = 0;
                for (int j = 0; j < g.ncontrols; j++) {
                    cmask |= bit(g.controls[j]);
                    if ((g.control_values >> j) & 1) cval |= bit(g.controls[j]);
                }
                QS_CUDA(launch_gate1(s, st.mat.data(), g.q0, cmask, cval));
            }
        } else {
            cd m[4] = {st.phase, 0.0, 0.0, st.phase};
            QS_CUDA(launch_gate1(s, m, 0, 0, 0));
        }
    }
    s->l2p = p->final_l2p;
    return QSIM_OK;
}

}  // extern "C"
