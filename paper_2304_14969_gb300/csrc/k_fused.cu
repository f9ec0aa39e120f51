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

#include "fused_body.cuh"

namespace qs {

qsim_status plan_build(const qsim_circuit *cir, qsim_dtype dt, const qsim_run_opts *opts, const int *start_l2p,
                       qsim_plan *P);
qsim_status permute_state(qsim_state *s, const std::vector<int> &new_pos);
qsim_status plan_build_tc(const qsim_circuit *cir, const qsim_run_opts *opts, const int *start_l2p, qsim_plan *P);
qsim_status validate_circuit(const qsim_circuit *c);
qsim_status apply_one_gate(qsim_state *s, const qsim_gate &g, const double *pool, int64_t pool_len, bool relabel);

template <typename R, int RB, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_fused_pass(typename FV<R>::T *__restrict__ a, FPassDev P,
                                                         uint64_t ntiles)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const size_t tile_bytes = (size_t)sizeof(typename FV<R>::T) << P.t;
    // per-tile phase factors of the partners outside the tile (2 R each)
    R *E = (R *)(smraw + tile_bytes);
    // the pass's constant block (ops, coefficients, maps, partners)
    unsigned char *stg = smraw + tile_bytes + (((size_t)P.nlin * 16 + 15) & ~(size_t)15);
    __shared__ int s_hq[kMaxTile], s_pos[12];
    const int tid = threadIdx.x;
    {
        const int4 *src = (const int4 *)P.stage;
        int4 *dst = (int4 *)stg;
        for (int i = tid; i < P.stage_bytes / 16; i += blockDim.x) dst[i] = src[i];
        if (tid < kMaxTile) s_hq[tid] = P.hq[tid];
        if (tid < 12) s_pos[tid] = P.ins.pos[tid];
    }
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        __syncthreads();   // staging done / previous tile finished with E and the buffer
        fused_tile<R, RB>(a, P, tile, smraw, E, stg, s_hq, s_pos);
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
    P->tc_off.clear();
    for (auto &A : P->tc_A) {
        size_t off = (buf.size() + 255) & ~(size_t)255;
        buf.resize(off + A.size());
        memcpy(buf.data() + off, A.data(), A.size());
        P->tc_off.push_back(off);
    }
    // pre-diagonal partner lists of the tensor-core blocks
    std::vector<size_t> pd_o(P->tc_A.size(), 0), pd_b(P->tc_A.size(), 0), pd_t(P->tc_A.size(), 0);
    auto put = [&](const void *src, size_t bytes) {
        size_t off = (buf.size() + 15) & ~(size_t)15;
        buf.resize(off + std::max<size_t>(bytes, 16));
        if (bytes) memcpy(buf.data() + off, src, bytes);
        return off;
    };
    const int kb = P->tc_spec.empty() ? 6 : P->tc_spec[0].kb;   // every block of a plan has the same size
    const bool pipe = !P->tc_A.empty() && tc_pipe_eligible(P->n, P->dt, (qsim_prec)P->prec, kb);
    std::vector<size_t> gt(P->tc_A.size(), 0);
    for (size_t i = 0; i < P->tc_A.size(); i++) {
        if (P->tc_pd_off[i].empty()) continue;
        pd_o[i] = put(P->tc_pd_off[i].data(), 4 * P->tc_pd_off[i].size());
        pd_b[i] = put(P->tc_pd_bit[i].data(), 4 * P->tc_pd_bit[i].size());
        pd_t[i] = put(P->tc_pd_tw[i].data(), 8 * P->tc_pd_tw[i].size());
        if (pipe) {
            std::vector<unsigned char> tb;
            tc_pipe_tables(P->n, P->tc_spec[i], P->tc_pd_off[i], P->tc_pd_bit[i], P->tc_pd_tw[i], tb);
            gt[i] = put(tb.data(), tb.size());
        }
    }
    if (buf.empty()) buf.resize(256);
    QS_CUDA(cudaMalloc(&P->dmem, buf.size()));
    P->dbytes = buf.size();
    QS_CUDA(cudaMemcpy(P->dmem, buf.data(), buf.size(), cudaMemcpyHostToDevice));
    for (size_t i = 0; i < P->passes.size(); i++)
        P->passes[i].dev.stage = (const unsigned char *)P->dmem + offs[i];
    for (size_t i = 0; i < P->tc_A.size(); i++) {
        TcSpec &ts = P->tc_spec[i];
        if (P->tc_pd_off[i].empty()) {
            ts.pd_off = nullptr;
            ts.pd_bit = nullptr;
            ts.pd_tw = nullptr;
        } else {
            unsigned char *d = (unsigned char *)P->dmem;
            ts.pd_off = (const int32_t *)(d + pd_o[i]);
            ts.pd_bit = (const int32_t *)(d + pd_b[i]);
            ts.pd_tw = (const uint64_t *)(d + pd_t[i]);
        }
    }
    P->tc_pipe.clear();
    if (pipe) {
        P->tc_pipe.resize(P->tc_A.size());
        for (size_t i = 0; i < P->tc_A.size(); i++) {
            const void *g = P->tc_pd_off[i].empty() ? nullptr : (const void *)((unsigned char *)P->dmem + gt[i]);
            QS_TRY(tc_pipe_prepare(P->n, P->tc_spec[i], g, P->tc_pipe[i], tc_pipe_kind(P->dt, (qsim_prec)P->prec, kb)));
        }
    }
    return QSIM_OK;
}

template <typename R, int RB, int NT, int MINB>
cudaError_t launch_pass_t(void *amps, const FPassDev &d, cudaStream_t st)
{
    using V = typename FV<R>::T;
    const size_t smem = fused_pass_smem(d, sizeof(V) == 8 ? QSIM_C64 : QSIM_C128);
    if (smem > kFusedSmemCap) return cudaErrorInvalidValue;
    auto kern = k_fused_pass<R, RB, NT, MINB>;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedSmemCap);
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

qsim_status plan_upload_ext(qsim_plan *P)
{
    if (P->dmem || P->passes.empty()) return QSIM_OK;
    return plan_upload(P);
}

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

static qsim_status plan_create_impl(const qsim_circuit *c, qsim_dtype dt, const qsim_run_opts *opts,
                                    const int *start, qsim_plan **out)
{
    if (!out) return fail(QSIM_E_INVAL, "out is NULL");
    *out = nullptr;
    QS_TRY(validate_circuit(c));
    if (dt != QSIM_C64 && dt != QSIM_C128) return fail(QSIM_E_INVAL, "unknown dtype");
    qsim_plan *P = new qsim_plan();
    qsim_status st;
    if (opts && opts->prec != QSIM_PREC_NATIVE) {
        if (opts->prec != QSIM_PREC_3XTF32 && opts->prec != QSIM_PREC_BF16X3 && opts->prec != QSIM_PREC_BF16X6)
            st = fail(QSIM_E_INVAL, "unknown prec");
        else if (dt == QSIM_C64 && opts->prec == QSIM_PREC_BF16X6)
            st = fail(QSIM_E_UNSUPPORTED, "BF16X6 plans take complex128 kets");
        else if (dt == QSIM_C128 && !tc_pipe_eligible(c->n, dt, (qsim_prec)opts->prec))
            st = fail(QSIM_E_UNSUPPORTED, "complex128 tensor-core plans take BF16X6 and n >= 13");
        else if (opts->max_block == 7 && !tc_pipe_eligible(c->n, dt, (qsim_prec)opts->prec, 7))
            st = fail(QSIM_E_UNSUPPORTED, "7-qubit tensor-core plans take complex64 kets, BF16X3 and n >= 14");
        else {
            st = plan_build_tc(c, opts, start, P);
            P->dt = dt;
        }
    } else {
        st = plan_build(c, dt, opts, start, P);
    }
    if (st != QSIM_OK) {
        delete P;
        return st;
    }
    *out = P;
    return QSIM_OK;
}

qsim_status qsim_plan_create(const qsim_circuit *c, qsim_dtype dt, const qsim_run_opts *opts, qsim_plan **out)
{
    clear_error();
    return plan_create_impl(c, dt, opts, nullptr, out);
}

qsim_status qsim_plan_create_for_state(const qsim_circuit *c, const qsim_state *s, const qsim_run_opts *opts,
                                       qsim_plan **out)
{
    clear_error();
    if (!s) return fail(QSIM_E_INVAL, "state is NULL");
    if (c && c->n != s->n) return fail(QSIM_E_INVAL, "circuit has n=%d but the state n=%d", c->n, s->n);
    return plan_create_impl(c, s->dt, opts, s->l2p.data(), out);
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
    info[0] = (int64_t)(p->passes.size() + p->tc_spec.size());
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

// Executes p on s; when norm_dev is not NULL and the last step is a
// pipelined tensor-core block, that block adds the sum of |psi_i|^2 of its
// output to *norm_dev.
static qsim_status plan_execute_impl(qsim_state *s, const qsim_plan *p, double *norm_dev)
{
    if (!s || !s->amps || !p) return fail(QSIM_E_INVAL, "NULL argument");
    if (p->n != s->n || p->dt != s->dt) return fail(QSIM_E_INVAL, "plan and state differ in n or dtype");
    if (!p->dmem && (!p->passes.empty() || !p->tc_A.empty())) QS_TRY(plan_upload(const_cast<qsim_plan *>(p)));
    if (s->l2p != p->start_l2p) {
        // move logical qubit L from physical bit s->l2p[L] to p->start_l2p[L]
        std::vector<int> to(s->n);
        for (int L = 0; L < s->n; L++) to[s->l2p[L]] = p->start_l2p[L];
        QS_TRY(permute_state(s, to));
        s->l2p = p->start_l2p;
    }
    for (size_t k = 0; k < p->steps.size(); k++) {
        const PlanStep &st = p->steps[k];
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
        } else if (st.kind == 3) {
            const unsigned char *dU = (const unsigned char *)p->dmem + p->tc_off[st.pass];
            QS_TRY(err_ensure(s));
            if (!p->tc_pipe.empty())
                QS_CUDA(tc_pipe_launch(s, p->tc_pipe[st.pass], dU, s->d_err,
                                       k + 1 == p->steps.size() ? norm_dev : nullptr));
            else
                QS_CUDA(tc_launch(s, p->tc_spec[st.pass], dU, (qsim_prec)p->prec, s->d_err));
        } else {
            cd m[4] = {st.phase, 0.0, 0.0, st.phase};
            QS_CUDA(launch_gate1(s, m, 0, 0, 0));
        }
    }
    s->l2p = p->final_l2p;
    // tensor-core blocks report a bounded wait that gave up through the
    // state's error word, read at the next call that synchronises
    return QSIM_OK;
}

qsim_status qsim_plan_execute(qsim_state *s, const qsim_plan *p)
{
    clear_error();
    return plan_execute_impl(s, p, nullptr);
}

qsim_status qsim_plan_execute_norm(qsim_state *s, const qsim_plan *p, double *norm)
{
    clear_error();
    if (!norm) return fail(QSIM_E_INVAL, "norm is NULL");
    if (p && !p->dmem && (!p->passes.empty() || !p->tc_A.empty())) QS_TRY(plan_upload(const_cast<qsim_plan *>(p)));
    const bool fused = p && !p->steps.empty() && p->steps.back().kind == 3 && !p->tc_pipe.empty() && s;
    if (!fused) {
        QS_TRY(plan_execute_impl(s, p, nullptr));
        return qsim_norm(s, norm);
    }
    QS_TRY(ensure_scratch(s->red, 64));
    QS_CUDA(cudaMemsetAsync(s->red.d, 0, sizeof(double), s->stream));
    QS_TRY(plan_execute_impl(s, p, s->red.d));
    QS_CUDA(cudaMemcpyAsync(s->red.h, s->red.d, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    err_fetch(s);
    QS_CUDA(cudaStreamSynchronize(s->stream));
    QS_TRY(err_check(s));
    *norm = s->red.h[0];
    return QSIM_OK;
}

}  // extern "C"
