// Batched circuits in one persistent launch, and the fused-plan autotuner.
//
// Every circuit of the batch is planned into fused passes (the same plans
// and tile body as qsim_plan_execute). Work items are (circuit, pass, tile)
// triples ordered by pass round, so an item only ever depends on items
// that were handed out before it. Persistent CTAs take items from one
// atomic counter; before a tile of pass p they wait, with a bounded spin,
// until every tile of pass p - 1 of the same circuit is done (a per-pass
// completion counter). A wait that runs out sets an error word, every CTA
// stops at its next item, and the host reports QSIM_E_TIMEOUT. The launch
// (plus the counter resets) is captured once in a CUDA graph and replayed.
// Per-circuit latency comes from %globaltimer stamps of the first and last
// tile of each circuit.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>

#include "fused_body.cuh"

namespace qs {

qsim_status permute_state(qsim_state *s, const std::vector<int> &new_pos);
qsim_status plan_build(const qsim_circuit *cir, qsim_dtype dt, const qsim_run_opts *opts, const int *start_l2p,
                       qsim_plan *P);
qsim_status plan_build_tc(const qsim_circuit *cir, const qsim_run_opts *opts, const int *start_l2p, qsim_plan *P);
qsim_status validate_circuit(const qsim_circuit *c);
int num_sms();

struct BatchItem {
    int32_t circ, gp, prev, pad;
    uint64_t tile;
};

static const int kBatchThreads = 256;
static const int kChunk = 8;
static const size_t kBatchTile = (size_t)8 << 13;   // complex64 tile of 13 qubits

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void __launch_bounds__(kBatchThreads, 2)
    k_batch(float2 *__restrict__ arena, const FPassDev *__restrict__ passes, const uint64_t *__restrict__ amp_off,
            const BatchItem *__restrict__ items, int nitems, unsigned *__restrict__ head, unsigned *done,
            const unsigned *__restrict__ need, unsigned long long *t0, unsigned long long *t1, int *err,
            long long wait_limit_ns, int max_lin16, int stage_off)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ int s_item, s_bad;
    __shared__ FPassDev sP;
    __shared__ int s_hq[kMaxTile], s_pos[12];
    float *E = (float *)(smraw + kBatchTile);
    unsigned char *stg = smraw + stage_off;
    int cur = -1;
    (void)max_lin16;
    // items are taken in chunks of kChunk consecutive ones (consecutive
    // items mostly share a pass, so its constants are staged once per chunk)
    int chunk_at = 0, chunk_end = 0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            if (chunk_at >= chunk_end) {
                chunk_at = (int)atomicAdd(head, 1u) * kChunk;
                chunk_end = min(chunk_at + kChunk, nitems);
            }
            int it = chunk_at < nitems ? chunk_at++ : nitems;
            int bad = *(volatile int *)err;
            if (!bad && it < nitems) {
                BatchItem b = items[it];
                if (b.prev >= 0) {
                    const unsigned long long w0 = gtimer();
                    while (*(volatile unsigned *)&done[b.prev] < need[b.prev]) {
                        if (gtimer() - w0 > (unsigned long long)wait_limit_ns || *(volatile int *)err) {
                            atomicExch(err, 1);
                            bad = 1;
                            break;
                        }
                        __nanosleep(100);
                    }
                    __threadfence();
                }
                if (!bad) atomicMin(&t0[b.circ], gtimer());
            }
            s_item = it;
            s_bad = bad;
        }
        __syncthreads();
        const int it = s_item;
        if (it >= nitems || s_bad) break;
        const BatchItem b = items[it];
        if (b.gp != cur) {
            if (threadIdx.x == 0) sP = passes[b.gp];
            __syncthreads();
            const int4 *src = (const int4 *)sP.stage;
            int4 *dst = (int4 *)stg;
            for (int i = threadIdx.x; i < sP.stage_bytes / 16; i += blockDim.x) dst[i] = src[i];
            if (threadIdx.x < kMaxTile) s_hq[threadIdx.x] = sP.hq[threadIdx.x];
            if (threadIdx.x < 12) s_pos[threadIdx.x] = sP.ins.pos[threadIdx.x];
            __syncthreads();
            cur = b.gp;
        }
        fused_tile<float, 5>(arena + amp_off[b.circ], sP, b.tile, smraw, E, stg, s_hq, s_pos);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(&done[b.gp], 1u);
            atomicMax(&t1[b.circ], gtimer());
        }
    }
}

__global__ void k_batch_reset(float2 *__restrict__ arena, uint64_t total, const uint64_t *__restrict__ amp_off,
                              int count)
{
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride)
        arena[i] = make_float2(0.f, 0.f);
}

__global__ void k_batch_ones(float2 *__restrict__ arena, const uint64_t *__restrict__ amp_off, int count)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < count; c += gridDim.x * blockDim.x)
        arena[amp_off[c]] = make_float2(1.f, 0.f);
}

// ------------------------------------------------------------ autotuner

qsim_status plan_upload_ext(qsim_plan *P);
cudaError_t launch_fused_pass(qsim_state *s, const FPassDev &d);

// Tile choice per qubit count from the tuner's JSON-lines cache: the
// complex64 entry for that n with the lowest batch cost (sm_ms, else ms);
// 0 if none.
static int cached_tile(const char *path, int n)
{
    if (!path) return 0;
    std::ifstream f(path);
    if (!f) return 0;
    std::string line;
    double best = 1e300;
    int tile = 0;
    while (std::getline(f, line)) {
        int ln = -1, lt = 0, ldt = -1;
        double ms = 0;
        const char *s = line.c_str();
        const char *p;
        if ((p = strstr(s, "\"n\":"))) ln = atoi(p + 4);
        if ((p = strstr(s, "\"tile\":"))) lt = atoi(p + 7);
        if ((p = strstr(s, "\"dtype\":"))) ldt = atoi(p + 8);
        if ((p = strstr(s, "\"ms\":"))) ms = atof(p + 5);
        if ((p = strstr(s, "\"sm_ms\":"))) ms = atof(p + 8);   // batch cost when recorded
        if (ln == n && ldt == 0 && lt > 0 && ms < best) {
            best = ms;
            tile = lt;
        }
    }
    return tile;
}

// True if the complex64 tune-cache entry for n with the lowest batch cost
// (sm_ms, else ms) is a tensor-core plan ("path": "tc").
static bool cached_tc(const char *path, int n)
{
    if (!path) return false;
    std::ifstream f(path);
    if (!f) return false;
    std::string line;
    double best = 1e300;
    bool tc = false;
    while (std::getline(f, line)) {
        int ln = -1, ldt = -1;
        double ms = 0;
        const char *s = line.c_str();
        const char *p;
        if ((p = strstr(s, "\"n\":"))) ln = atoi(p + 4);
        if ((p = strstr(s, "\"dtype\":"))) ldt = atoi(p + 8);
        if ((p = strstr(s, "\"ms\":"))) ms = atof(p + 5);
        if ((p = strstr(s, "\"sm_ms\":"))) ms = atof(p + 8);
        if (ln == n && ldt == 0 && ms > 0 && ms < best) {
            best = ms;
            tc = strstr(s, "\"path\": \"tc\"") != nullptr;
        }
    }
    return tc;
}

}  // namespace qs

using namespace qs;

struct qsim_batch {
    int count = 0;
    std::vector<qsim_plan *> plans;
    std::vector<int> n;
    std::vector<uint64_t> amp_off;
    uint64_t total_amps = 0;
    float2 *arena = nullptr;
    void *dtab = nullptr;       // passes, items, amp_off, need
    unsigned *dcnt = nullptr;   // head + done[npasses]
    unsigned long long *dts = nullptr;  // t0[count], t1[count]
    int *derr = nullptr;
    int npasses = 0, nitems = 0;
    FPassDev *d_passes = nullptr;
    BatchItem *d_items = nullptr;
    uint64_t *d_off = nullptr;
    unsigned *d_need = nullptr;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
    bool use_graph = false;
    int grid = 0;
    size_t smem = 0;
    int stage_off = 0;
    bool dirty = false;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    // circuits on tensor-core blocks: descriptors, work entries per round
    int ntc = 0;
    void *tc_mem = nullptr;
    TcBatchDesc *d_desc = nullptr;
    TcWork *d_work = nullptr;
    std::vector<int> round_off, round_cnt;
    cudaStream_t st2 = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};

static void batch_free(qsim_batch *b)
{
    if (!b) return;
    if (b->st) cudaStreamSynchronize(b->st);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->st2) cudaStreamSynchronize(b->st2);
    for (void *p : {(void *)b->arena, b->dtab, (void *)b->dcnt, (void *)b->dts, (void *)b->derr, b->tc_mem})
        if (p) cudaFree(p);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->join) cudaEventDestroy(b->join);
    if (b->st2) cudaStreamDestroy(b->st2);
    for (qsim_plan *p : b->plans) qsim_plan_destroy(p);
    if (b->e0) cudaEventDestroy(b->e0);
    if (b->e1) cudaEventDestroy(b->e1);
    if (b->own_stream && b->st) cudaStreamDestroy(b->st);
    delete b;
}

static qsim_status batch_launch(qsim_batch *b)
{
    QS_CUDA(cudaMemsetAsync(b->dcnt, 0, sizeof(unsigned) * (1 + b->npasses), b->st));
    QS_CUDA(cudaMemsetAsync(b->dts, 0xff, sizeof(unsigned long long) * b->count, b->st));
    QS_CUDA(cudaMemsetAsync(b->dts + b->count, 0, sizeof(unsigned long long) * b->count, b->st));
    QS_CUDA(cudaMemsetAsync(b->derr, 0, sizeof(int), b->st));
    const long long wait_limit_ns = 2000000000;   // 2 s of device time per wait
    if (!b->round_cnt.empty()) {
        // tensor-core circuits: one grouped launch per block round on a second
        // stream, concurrent with the persistent SIMT launch
        QS_CUDA(cudaEventRecord(b->fork, b->st));
        QS_CUDA(cudaStreamWaitEvent(b->st2, b->fork, 0));
        for (size_t r = 0; r < b->round_cnt.size(); r++)
            QS_CUDA(tc_pipe_launch_grouped(b->d_desc, b->d_work + b->round_off[r], b->round_cnt[r], b->dts,
                                           b->dts + b->count, b->derr, b->st2));
        QS_CUDA(cudaEventRecord(b->join, b->st2));
    }
    if (b->nitems > 0) {
        k_batch<<<b->grid, kBatchThreads, b->smem, b->st>>>(b->arena, b->d_passes, b->d_off, b->d_items, b->nitems,
                                                           b->dcnt, b->dcnt + 1, b->d_need, b->dts, b->dts + b->count,
                                                           b->derr, wait_limit_ns, 0, b->stage_off);
        QS_CUDA(cudaGetLastError());
    }
    if (!b->round_cnt.empty()) QS_CUDA(cudaStreamWaitEvent(b->st, b->join, 0));
    return QSIM_OK;
}

extern "C" {

qsim_status qsim_batch_create(const qsim_circuit *const *cs, int count, const qsim_batch_opts *opts,
                              qsim_batch **out)
{
    clear_error();
    if (!out) return fail(QSIM_E_INVAL, "out is NULL");
    *out = nullptr;
    if (!cs || count < 1) return fail(QSIM_E_INVAL, "no circuits");
    qsim_batch_opts o{};
    if (opts) o = *opts;
    qsim_batch *b = new qsim_batch();
    b->count = count;
    b->use_graph = o.use_graph != 0;
    if (o.stream) b->st = (cudaStream_t)o.stream;
    else {
        cudaError_t e = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            batch_free(b);
            return cuda_fail(e, "stream");
        }
        b->own_stream = true;
    }
    // ---- plans
    std::vector<FPassDev> passes;
    std::vector<std::vector<int>> pass_of(count);
    size_t max_stage = 0;
    int max_lin = 0;
    for (int i = 0; i < count; i++) {
        const qsim_circuit *c = cs[i];
        qsim_status st = validate_circuit(c);
        if (st == QSIM_OK && (c->n < 10 || c->n > 34)) st = fail(QSIM_E_UNSUPPORTED, "batch circuits need 10 <= n <= 34");
        int t = o.tile_qubits ? o.tile_qubits : cached_tile(o.tune_cache, c ? c->n : 0);
        if (t == 0) t = 13;
        t = std::min(t, 13);
        qsim_run_opts ro{};
        ro.mode = QSIM_MODE_FUSED;
        ro.relabel_swaps = 1;
        ro.tile_qubits = t;
        qsim_plan *P = nullptr;
        // tensor-core blocks (BF16x3) when asked for or autotuned, if the plan
        // is blocks only; otherwise fused SIMT passes
        const bool want_tc = c && c->n >= 13 && (o.path == 2 || (o.path == 0 && cached_tc(o.tune_cache, c->n)));
        if (st == QSIM_OK && want_tc) {
            qsim_run_opts to{};
            to.mode = QSIM_MODE_FUSED;
            to.relabel_swaps = 1;
            to.prec = QSIM_PREC_BF16X3;
            P = new qsim_plan();
            bool ok = plan_build_tc(c, &to, nullptr, P) == QSIM_OK;
            for (const PlanStep &s2 : P->steps) ok = ok && s2.kind == 3;
            if (ok) {
                b->plans.push_back(P);
                b->n.push_back(c->n);
                b->ntc++;
                continue;
            }
            delete P;
            P = nullptr;
            clear_error();
        }
        if (st == QSIM_OK) {
            P = new qsim_plan();
            st = plan_build(c, QSIM_C64, &ro, nullptr, P);
            if (st != QSIM_OK) delete P;
        }
        if (st == QSIM_OK && P->RB != 5) {
            st = fail(QSIM_E_UNSUPPORTED, "circuit %d needs dense two-qubit blocks (not batched)", i);
            delete P;
        }
        if (st == QSIM_OK)
            for (const PlanStep &s : P->steps)
                if (s.kind != 0) {
                    st = fail(QSIM_E_UNSUPPORTED, "circuit %d has steps outside fused passes", i);
                    delete P;
                    break;
                }
        if (st != QSIM_OK) {
            batch_free(b);
            return st;
        }
        b->plans.push_back(P);
        b->n.push_back(c->n);
        for (PlanPass &ps : P->passes) {
            pass_of[i].push_back((int)passes.size());
            passes.push_back(ps.dev);
            max_stage = std::max(max_stage, ps.stage.size());
            max_lin = std::max(max_lin, ps.nlin);
        }
    }
    b->npasses = (int)passes.size();
    // ---- arena (largest kets first keeps every ket 2^n-aligned)
    std::vector<int> order(count);
    for (int i = 0; i < count; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->n[x] > b->n[y]; });
    b->amp_off.assign(count, 0);
    uint64_t off = 0;
    for (int i : order) {
        b->amp_off[i] = off;
        off += 1ull << b->n[i];
    }
    b->total_amps = off;
    cudaError_t e = cudaMalloc(&b->arena, off * sizeof(float2));
    if (e != cudaSuccess) {
        batch_free(b);
        return cuda_fail(e, "batch arena");
    }
    // ---- stage blocks of every pass
    std::vector<unsigned char> sbuf;
    std::vector<size_t> soff;
    for (int i = 0; i < count; i++)
        for (PlanPass &ps : b->plans[i]->passes) {
            size_t so = (sbuf.size() + 255) & ~(size_t)255;
            sbuf.resize(so + ps.stage.size());
            memcpy(sbuf.data() + so, ps.stage.data(), ps.stage.size());
            soff.push_back(so);
        }
    // ---- items, ordered by pass round
    std::vector<BatchItem> items;
    std::vector<unsigned> need(b->npasses);
    int rounds = 0;
    for (int i = 0; i < count; i++) rounds = std::max(rounds, (int)pass_of[i].size());
    for (int r = 0; r < rounds; r++)
        for (int i = 0; i < count; i++) {
            if (r >= (int)pass_of[i].size()) continue;
            int gp = pass_of[i][r];
            const FPassDev &d = passes[gp];
            uint64_t ntiles = 1ull << (d.n - d.t);
            need[gp] = (unsigned)ntiles;
            for (uint64_t tl = 0; tl < ntiles; tl++)
                items.push_back(BatchItem{i, gp, r ? pass_of[i][r - 1] : -1, 0, tl});
        }
    b->nitems = (int)items.size();
    // ---- device tables: stage blocks | passes | items | offsets | need
    size_t o_st = 0, o_pa = (sbuf.size() + 255) & ~(size_t)255;
    size_t o_it = (o_pa + passes.size() * sizeof(FPassDev) + 255) & ~(size_t)255;
    size_t o_of = (o_it + items.size() * sizeof(BatchItem) + 255) & ~(size_t)255;
    size_t o_ne = (o_of + count * sizeof(uint64_t) + 255) & ~(size_t)255;
    size_t tot = o_ne + need.size() * sizeof(unsigned) + 256;
    e = cudaMalloc(&b->dtab, tot);
    if (e != cudaSuccess) {
        batch_free(b);
        return cuda_fail(e, "batch tables");
    }
    unsigned char *d = (unsigned char *)b->dtab;
    for (size_t i = 0; i < passes.size(); i++) passes[i].stage = d + o_st + soff[i];
    std::vector<unsigned char> h(tot, 0);
    memcpy(h.data() + o_st, sbuf.data(), sbuf.size());
    memcpy(h.data() + o_pa, passes.data(), passes.size() * sizeof(FPassDev));
    memcpy(h.data() + o_it, items.data(), items.size() * sizeof(BatchItem));
    memcpy(h.data() + o_of, b->amp_off.data(), count * sizeof(uint64_t));
    memcpy(h.data() + o_ne, need.data(), need.size() * sizeof(unsigned));
    e = cudaMemcpy(b->dtab, h.data(), tot, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&b->dcnt, sizeof(unsigned) * (1 + b->npasses));
    if (e == cudaSuccess) e = cudaMalloc(&b->dts, sizeof(unsigned long long) * 2 * count);
    if (e == cudaSuccess) e = cudaMalloc(&b->derr, sizeof(int));
    if (e == cudaSuccess) e = cudaEventCreate(&b->e0);
    if (e == cudaSuccess) e = cudaEventCreate(&b->e1);
    if (e != cudaSuccess) {
        batch_free(b);
        return cuda_fail(e, "batch setup");
    }
    b->d_passes = (FPassDev *)(d + o_pa);
    b->d_items = (BatchItem *)(d + o_it);
    b->d_off = (uint64_t *)(d + o_of);
    b->d_need = (unsigned *)(d + o_ne);
    // ---- tensor-core circuits: per block a descriptor (tensor map over the
    // circuit's ket, geometry, U, deferred-phase tables); work entries of at
    // most kTcChunk tiles, grouped by block round
    if (b->ntc > 0) {
        const uint64_t kTcChunk = 16;
        std::vector<std::pair<int, int>> blocks;   // (circuit, block)
        int rounds_tc = 0;
        for (int i = 0; i < count; i++)
            if (b->plans[i]->passes.empty() && !b->plans[i]->tc_A.empty()) {
                for (int j = 0; j < (int)b->plans[i]->tc_A.size(); j++) blocks.push_back({i, j});
                rounds_tc = std::max(rounds_tc, (int)b->plans[i]->tc_A.size());
            }
        const size_t nb = blocks.size();
        const size_t o_desc = 0, o_u = (nb * sizeof(TcBatchDesc) + 255) & ~(size_t)255;
        size_t o_tab = o_u + nb * 65536, o_work;
        std::vector<size_t> tab_off(nb, 0);
        for (size_t k = 0; k < nb; k++) {
            const qsim_plan *Pk = b->plans[blocks[k].first];
            if (!Pk->tc_pd_off[blocks[k].second].empty()) {
                tab_off[k] = o_tab;
                o_tab += (kTcPipeTableBytes + 255) & ~(size_t)255;
            }
        }
        std::vector<std::vector<int>> desc_of(count);
        for (size_t k = 0; k < nb; k++) desc_of[blocks[k].first].push_back((int)k);
        std::vector<TcWork> works;
        for (int r = 0; r < rounds_tc; r++) {
            b->round_off.push_back((int)works.size());
            for (int i = 0; i < count; i++) {
                if (r >= (int)desc_of[i].size()) continue;
                const uint64_t ntiles = 1ull << (b->n[i] - 13);
                for (uint64_t t0 = 0; t0 < ntiles; t0 += kTcChunk)
                    works.push_back(TcWork{desc_of[i][r], 0, t0, std::min(kTcChunk, ntiles - t0)});
            }
            b->round_cnt.push_back((int)works.size() - b->round_off.back());
        }
        o_work = (o_tab + 255) & ~(size_t)255;
        const size_t tot_tc = o_work + works.size() * sizeof(TcWork) + 256;
        e = cudaMalloc(&b->tc_mem, tot_tc);
        if (e != cudaSuccess) {
            batch_free(b);
            return cuda_fail(e, "batch tensor-core tables");
        }
        unsigned char *dm = (unsigned char *)b->tc_mem;
        std::vector<unsigned char> hm(tot_tc, 0);
        std::vector<TcBatchDesc> descs(nb);
        for (size_t k = 0; k < nb; k++) {
            const int i = blocks[k].first, j = blocks[k].second;
            const qsim_plan *Pk = b->plans[i];
            if (Pk->tc_A[j].size() != 65536) {
                batch_free(b);
                return fail(QSIM_E_UNSUPPORTED, "unexpected tensor-core operand size");
            }
            memcpy(hm.data() + o_u + k * 65536, Pk->tc_A[j].data(), 65536);
            const void *tabs = nullptr;
            if (tab_off[k]) {
                std::vector<unsigned char> tb;
                tc_pipe_tables(b->n[i], Pk->tc_spec[j], Pk->tc_pd_off[j], Pk->tc_pd_bit[j], Pk->tc_pd_tw[j], tb);
                memcpy(hm.data() + tab_off[k], tb.data(), tb.size());
                tabs = dm + tab_off[k];
            }
            TcPipeHost H;
            qsim_status st = tc_pipe_prepare(b->n[i], Pk->tc_spec[j], tabs, H);
            if (st == QSIM_OK) st = tc_pipe_encode(H, b->arena + b->amp_off[i], descs[k].tmap);
            if (st != QSIM_OK) {
                batch_free(b);
                return st;
            }
            descs[k].args = H.args;
            descs[k].U = dm + o_u + k * 65536;
            descs[k].amps = b->arena + b->amp_off[i];
            descs[k].circ = i;
        }
        memcpy(hm.data() + o_desc, descs.data(), nb * sizeof(TcBatchDesc));
        memcpy(hm.data() + o_work, works.data(), works.size() * sizeof(TcWork));
        e = cudaMemcpy(b->tc_mem, hm.data(), tot_tc, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->st2, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            batch_free(b);
            return cuda_fail(e, "batch tensor-core setup");
        }
        b->d_desc = (TcBatchDesc *)(dm + o_desc);
        b->d_work = (TcWork *)(dm + o_work);
    }
    // ---- launch shape
    size_t lin_bytes = ((size_t)max_lin * 16 + 15) & ~(size_t)15;
    b->stage_off = (int)(kBatchTile + lin_bytes);
    b->smem = kBatchTile + lin_bytes + max_stage;
    if (b->smem > kFusedSmemCap) {
        batch_free(b);
        return fail(QSIM_E_UNSUPPORTED, "batch pass constants too large for shared memory");
    }
    cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedSmemCap);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch, kBatchThreads, b->smem);
    if (occ < 1) occ = 1;
    int ctas = num_sms() * occ;
    if (o.ctas > 0) ctas = std::min(ctas, o.ctas);
    b->grid = std::max(1, std::min(ctas, std::max(1, b->nitems)));
    // ---- kets at |0...0>
    k_batch_reset<<<num_sms() * 4, 256, 0, b->st>>>(b->arena, b->total_amps, b->d_off, count);
    k_batch_ones<<<(count + 255) / 256, 256, 0, b->st>>>(b->arena, b->d_off, count);
    e = cudaGetLastError();
    if (e == cudaSuccess && b->use_graph) {
        e = cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            qsim_status ls = batch_launch(b);
            cudaError_t e2 = cudaStreamEndCapture(b->st, &b->graph);
            if (ls != QSIM_OK) e = cudaErrorUnknown;
            else e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, b->graph, 0);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) {
        batch_free(b);
        return cuda_fail(e, "batch graph");
    }
    *out = b;
    return QSIM_OK;
}

qsim_status qsim_batch_destroy(qsim_batch *b)
{
    batch_free(b);
    return QSIM_OK;
}

qsim_status qsim_batch_upload(qsim_batch *b, int i, const void *host_amps)
{
    clear_error();
    if (!b || !host_amps || i < 0 || i >= b->count) return fail(QSIM_E_INVAL, "bad argument");
    QS_CUDA(cudaMemcpyAsync(b->arena + b->amp_off[i], host_amps, sizeof(float2) << b->n[i], cudaMemcpyHostToDevice,
                            b->st));
    QS_CUDA(cudaStreamSynchronize(b->st));
    b->dirty = false;
    return QSIM_OK;
}

qsim_status qsim_batch_reset(qsim_batch *b)
{
    clear_error();
    if (!b) return fail(QSIM_E_INVAL, "batch is NULL");
    k_batch_reset<<<num_sms() * 4, 256, 0, b->st>>>(b->arena, b->total_amps, b->d_off, b->count);
    k_batch_ones<<<(b->count + 255) / 256, 256, 0, b->st>>>(b->arena, b->d_off, b->count);
    QS_CUDA(cudaGetLastError());
    b->dirty = false;
    return QSIM_OK;
}

qsim_status qsim_batch_run(qsim_batch *b, double *seconds, double *latency_s)
{
    clear_error();
    if (!b) return fail(QSIM_E_INVAL, "batch is NULL");
    if (b->dirty) return fail(QSIM_E_INVAL, "kets were already run: reset or upload them first");
    QS_CUDA(cudaEventRecord(b->e0, b->st));
    if (b->gexec) QS_CUDA(cudaGraphLaunch(b->gexec, b->st));
    else QS_TRY(batch_launch(b));
    QS_CUDA(cudaEventRecord(b->e1, b->st));
    QS_CUDA(cudaStreamSynchronize(b->st));
    b->dirty = true;
    int err = 0;
    QS_CUDA(cudaMemcpy(&err, b->derr, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) return fail(QSIM_E_TIMEOUT, "a batch tile waited too long for its previous pass");
    if (seconds) {
        float ms = 0;
        QS_CUDA(cudaEventElapsedTime(&ms, b->e0, b->e1));
        *seconds = ms * 1e-3;
    }
    if (latency_s) {
        std::vector<unsigned long long> ts(2 * (size_t)b->count);
        QS_CUDA(cudaMemcpy(ts.data(), b->dts, ts.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
        for (int i = 0; i < b->count; i++)
            latency_s[i] = ts[b->count + i] >= ts[i] ? (double)(ts[b->count + i] - ts[i]) * 1e-9 : 0.0;
    }
    return QSIM_OK;
}

qsim_status qsim_batch_download(qsim_batch *b, int i, void *host_amps)
{
    clear_error();
    if (!b || !host_amps || i < 0 || i >= b->count) return fail(QSIM_E_INVAL, "bad argument");
    qsim_state v;
    v.n = b->n[i];
    v.dt = QSIM_C64;
    v.stream = b->st;
    v.amps = b->arena + b->amp_off[i];
    v.owned = false;
    v.l2p = b->dirty ? b->plans[i]->final_l2p : std::vector<int>();
    if (v.l2p.empty()) {
        v.l2p.resize(v.n);
        for (int q = 0; q < v.n; q++) v.l2p[q] = q;
    }
    qsim_status st = qsim_download(&v, host_amps);
    free_scratch(v.red);
    return st;
}

qsim_status qsim_batch_info(const qsim_batch *b, int64_t info[8])
{
    clear_error();
    if (!b || !info) return fail(QSIM_E_INVAL, "NULL argument");
    info[0] = b->count;
    info[1] = b->nitems;
    info[2] = b->grid;
    info[3] = (int64_t)(b->total_amps * sizeof(float2));
    info[4] = b->npasses;
    info[5] = (int64_t)b->smem;
    info[6] = b->gexec ? 1 : 0;
    info[7] = b->ntc;
    return QSIM_OK;
}

}  // extern "C"

// Batch cost of one setting: device time per circuit of a batch of R copies
// of c (R large enough to occupy every SM a few times over), run through
// the batch runner itself; negative if the setting cannot be batched.
static double batch_cost_ms(const qsim_circuit *c, int path, int tile)
{
    const int t = path == 2 ? 13 : tile;
    const uint64_t tiles = 1ull << std::max(0, c->n - t);
    uint64_t R = (4ull * (uint64_t)num_sms() * 2 + tiles - 1) / tiles;
    R = std::max<uint64_t>(1, std::min<uint64_t>(R, 512));
    while (R > 1 && (R << c->n) * 8 > (2ull << 30)) R--;
    std::vector<const qsim_circuit *> cs((size_t)R, c);
    qsim_batch_opts o{};
    o.use_graph = 1;
    o.path = path;
    o.tile_qubits = path == 2 ? 0 : tile;
    qsim_batch *b = nullptr;
    if (qsim_batch_create(cs.data(), (int)R, &o, &b) != QSIM_OK) {
        clear_error();
        return -1;
    }
    double sec = 0;
    bool ok = qsim_batch_run(b, nullptr, nullptr) == QSIM_OK && qsim_batch_reset(b) == QSIM_OK &&
              qsim_batch_run(b, &sec, nullptr) == QSIM_OK;
    qsim_batch_destroy(b);
    if (!ok) {
        clear_error();
        return -1;
    }
    return sec * 1e3 / (double)R;
}

extern "C" {

qsim_status qsim_autotune(const qsim_circuit *c, qsim_dtype dt, const char *tune_cache, qsim_run_opts *best_opts,
                          double *best_seconds)
{
    clear_error();
    QS_TRY(validate_circuit(c));
    if (dt != QSIM_C64 && dt != QSIM_C128) return fail(QSIM_E_INVAL, "unknown dtype");
    if (c->n < 10 || c->n > 30) return fail(QSIM_E_INVAL, "autotuning needs 10 <= n <= 30");
    qsim_state *s = nullptr;
    QS_TRY(qsim_create(c->n, dt, nullptr, &s));
    cudaEvent_t a, z;
    cudaEventCreate(&a);
    cudaEventCreate(&z);
    double best = 1e300;
    int best_t = 0;
    int tmax = dt == QSIM_C64 ? 14 : 13;
    qsim_status st = QSIM_OK;
    for (int t = 10; t <= std::min(tmax, c->n) && st == QSIM_OK; t++) {
        qsim_run_opts o{};
        o.mode = QSIM_MODE_FUSED;
        o.relabel_swaps = 1;
        o.tile_qubits = t;
        // one warm-up run, then three timed runs; every run is planned for
        // the ket's current layout (planning and upload are not timed)
        float tot = 0;
        bool ok = true;
        for (int r = 0; r < 4 && st == QSIM_OK; r++) {
            qsim_plan *p = nullptr;
            if (qsim_plan_create_for_state(c, s, &o, &p) != QSIM_OK) {
                ok = false;
                break;
            }
            st = plan_upload_ext(p);
            if (st == QSIM_OK) {
                cudaEventRecord(a, s->stream);
                st = qsim_plan_execute(s, p);
                cudaEventRecord(z, s->stream);
                cudaEventSynchronize(z);
                float ms = 0;
                cudaEventElapsedTime(&ms, a, z);
                if (r > 0) tot += ms;
            }
            qsim_plan_destroy(p);
        }
        if (!ok) {
            clear_error();
            continue;
        }
        if (st != QSIM_OK) break;
        double avg = tot / 3.0;
        if (tune_cache) {
            FILE *f = fopen(tune_cache, "a");
            if (f) {
                // sm_ms: device time per circuit when a batch of copies runs
                // side by side (complex64 tiles the batch runner takes)
                const double bc = dt == QSIM_C64 && t <= 13 ? batch_cost_ms(c, 1, t) : -1.0;
                if (bc > 0)
                    fprintf(f, "{\"n\": %d, \"dtype\": %d, \"gates\": %d, \"tile\": %d, \"ms\": %.6f, \"sm_ms\": %.6f}\n",
                            c->n, (int)dt, c->ngates, t, avg, bc);
                else
                    fprintf(f, "{\"n\": %d, \"dtype\": %d, \"gates\": %d, \"tile\": %d, \"ms\": %.6f}\n", c->n,
                            (int)dt, c->ngates, t, avg);
                fclose(f);
            }
        }
        if (avg < best) {
            best = avg;
            best_t = t;
        }
    }
    // complex64 with n >= 13: the same circuit as tensor-core blocks (BF16x3)
    bool best_tc = false;
    if (st == QSIM_OK && dt == QSIM_C64 && c->n >= 13) {
        qsim_run_opts o{};
        o.mode = QSIM_MODE_FUSED;
        o.relabel_swaps = 1;
        o.prec = QSIM_PREC_BF16X3;
        float tot = 0;
        bool ok = true;
        for (int r = 0; r < 4 && st == QSIM_OK; r++) {
            qsim_plan *p = nullptr;
            if (qsim_plan_create_for_state(c, s, &o, &p) != QSIM_OK) {
                ok = false;
                break;
            }
            cudaEventRecord(a, s->stream);
            st = qsim_plan_execute(s, p);
            cudaEventRecord(z, s->stream);
            cudaEventSynchronize(z);
            if (st == QSIM_OK) st = qsim_synchronize(s);
            float ms = 0;
            cudaEventElapsedTime(&ms, a, z);
            if (r > 0) tot += ms;
            qsim_plan_destroy(p);
        }
        if (!ok) {
            clear_error();
        } else if (st == QSIM_OK) {
            double avg = tot / 3.0;
            if (tune_cache) {
                FILE *f = fopen(tune_cache, "a");
                if (f) {
                    const double bc = batch_cost_ms(c, 2, 0);
                    if (bc > 0)
                        fprintf(f,
                                "{\"n\": %d, \"dtype\": %d, \"gates\": %d, \"tile\": 0, \"path\": \"tc\", \"ms\": %.6f, "
                                "\"sm_ms\": %.6f}\n",
                                c->n, (int)dt, c->ngates, avg, bc);
                    else
                        fprintf(f, "{\"n\": %d, \"dtype\": %d, \"gates\": %d, \"tile\": 0, \"path\": \"tc\", \"ms\": %.6f}\n",
                                c->n, (int)dt, c->ngates, avg);
                    fclose(f);
                }
            }
            if (avg < best) {
                best = avg;
                best_tc = true;
            }
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(z);
    qsim_destroy(s);
    if (st != QSIM_OK) return st;
    if (best_opts) {
        memset(best_opts, 0, sizeof *best_opts);
        best_opts->mode = QSIM_MODE_FUSED;
        best_opts->relabel_swaps = 1;
        best_opts->tile_qubits = best_tc ? 0 : best_t;
        best_opts->prec = best_tc ? QSIM_PREC_BF16X3 : QSIM_PREC_NATIVE;
    }
    if (best_seconds) *best_seconds = best * 1e-3;
    return QSIM_OK;
}

}  // extern "C"
