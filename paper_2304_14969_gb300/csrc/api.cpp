// C-ABI entry points: states, per-gate calls, reductions.
//
// Every argument is validated on the host before any launch. Logical
// qubits are translated to physical bits through the state's map, which
// changes only through SWAP relabels (Table I of arXiv 2304.14969: a SWAP
// is a constant-cost relabel) and is undone by qsim_materialize.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "qsim_internal.h"

using namespace qs;

namespace {

bool is_identity(const qsim_state *s)
{
    for (int q = 0; q < s->n; q++)
        if (s->l2p[q] != q) return false;
    return true;
}

qsim_status check_state(const qsim_state *s)
{
    if (!s) return fail(QSIM_E_INVAL, "state is NULL");
    if (!s->amps) return fail(QSIM_E_INVAL, "state has no amplitudes");
    return QSIM_OK;
}

qsim_status check_qubit(const qsim_state *s, int q, const char *what)
{
    if (q < 0 || q >= s->n) return fail(QSIM_E_INVAL, "%s %d out of range for n=%d", what, q, s->n);
    return QSIM_OK;
}

qsim_status make_state(int n, qsim_dtype dt, void *stream, qsim_state **out)
{
    if (!out) return fail(QSIM_E_INVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > 36) return fail(QSIM_E_INVAL, "n=%d outside [1, 36]", n);
    if (dt != QSIM_C64 && dt != QSIM_C128) return fail(QSIM_E_INVAL, "unknown dtype %d", (int)dt);
    qsim_state *s = new qsim_state();
    s->n = n;
    s->dt = dt;
    s->stream = (cudaStream_t)stream;
    s->l2p.resize(n);
    for (int q = 0; q < n; q++) s->l2p[q] = q;
    cudaGetDevice(&s->device);
    *out = s;
    return QSIM_OK;
}

}  // namespace

namespace qs {
// Kets up to this size keep their permutation buffer (a stream-ordered
// temporary taken from the shared pool per call would make a second state's
// stream wait for the first's frees, serialising pipelined kets).
static const size_t kPermKeepBytes = (size_t)8 << 30;

// A ket-sized device buffer for a permutation of s: the state's kept buffer,
// or (*temporary set) a stream-ordered temporary the caller frees after use.
static qsim_status perm_buffer(qsim_state *s, void **buf, bool *temporary)
{
    *temporary = false;
    if (s->perm) {
        *buf = s->perm;
        return QSIM_OK;
    }
    if (s->amp_bytes() <= kPermKeepBytes && cudaMalloc(&s->perm, s->amp_bytes()) == cudaSuccess) {
        *buf = s->perm;
        return QSIM_OK;
    }
    cudaGetLastError();   // a failed keep falls back to a temporary
    s->perm = nullptr;
    cudaError_t e = cudaMallocAsync(buf, s->amp_bytes(), s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (permutation buffer)");
    *temporary = true;
    return QSIM_OK;
}

// Moves the amplitudes so that physical bit p ends up at new_pos[p].
qsim_status permute_state(qsim_state *s, const std::vector<int> &new_pos)
{
    void *tmp = nullptr;
    bool temporary = false;
    QS_TRY(perm_buffer(s, &tmp, &temporary));
    cudaError_t e = launch_permute(s->amps, tmp, s->dt, s->n, new_pos.data(), s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->amps, tmp, s->amp_bytes(), cudaMemcpyDeviceToDevice, s->stream);
    if (temporary) cudaFreeAsync(tmp, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "permute");
    return QSIM_OK;
}
}  // namespace qs

namespace {
}  // namespace

extern "C" {

qsim_status qsim_create(int n, qsim_dtype dt, void *stream, qsim_state **out)
{
    clear_error();
    QS_TRY(make_state(n, dt, stream, out));
    qsim_state *s = *out;
    cudaError_t e = cudaMalloc(&s->amps, s->amp_bytes());
    if (e != cudaSuccess) {
        delete s;
        *out = nullptr;
        return cuda_fail(e, "cudaMalloc (ket)");
    }
    s->owned = true;
    e = launch_set_basis(s, 0);
    if (e != cudaSuccess) {
        cudaFree(s->amps);
        delete s;
        *out = nullptr;
        return cuda_fail(e, "set_basis");
    }
    return QSIM_OK;
}

qsim_status qsim_wrap(int n, qsim_dtype dt, void *dev_amps, void *stream, qsim_state **out)
{
    clear_error();
    if (!dev_amps) return fail(QSIM_E_INVAL, "dev_amps is NULL");
    if (((uintptr_t)dev_amps) & 15) return fail(QSIM_E_INVAL, "dev_amps is not 16-byte aligned");
    QS_TRY(make_state(n, dt, stream, out));
    (*out)->amps = dev_amps;
    (*out)->owned = false;
    return QSIM_OK;
}

qsim_status qsim_destroy(qsim_state *s)
{
    clear_error();
    if (!s) return QSIM_OK;
    if (s->stream) cudaStreamSynchronize(s->stream);
    else cudaDeviceSynchronize();
    if (s->owned && s->amps) cudaFree(s->amps);
    if (s->perm) cudaFree(s->perm);
    if (s->d_err) cudaFree(s->d_err);
    if (s->h_err) cudaFreeHost(s->h_err);
    free_scratch(s->red);
    delete s;
    return QSIM_OK;
}

qsim_status qsim_set_basis(qsim_state *s, uint64_t x)
{
    clear_error();
    QS_TRY(check_state(s));
    if (x >= s->N()) return fail(QSIM_E_INVAL, "basis index out of range");
    for (int q = 0; q < s->n; q++) s->l2p[q] = q;
    QS_CUDA(launch_set_basis(s, x));
    return QSIM_OK;
}

qsim_status qsim_upload(qsim_state *s, const void *host_amps)
{
    clear_error();
    QS_TRY(check_state(s));
    if (!host_amps) return fail(QSIM_E_INVAL, "host_amps is NULL");
    for (int q = 0; q < s->n; q++) s->l2p[q] = q;
    QS_CUDA(cudaMemcpyAsync(s->amps, host_amps, s->amp_bytes(), cudaMemcpyHostToDevice, s->stream));
    return QSIM_OK;
}

qsim_status qsim_download_async(qsim_state *s, void *host_amps)
{
    clear_error();
    QS_TRY(check_state(s));
    if (!host_amps) return fail(QSIM_E_INVAL, "host_amps is NULL");
    if (is_identity(s)) {
        QS_CUDA(cudaMemcpyAsync(host_amps, s->amps, s->amp_bytes(), cudaMemcpyDeviceToHost, s->stream));
        return QSIM_OK;
    }
    // physical bit p holds logical qubit L with l2p[L] = p; logical order puts it at bit L
    std::vector<int> to(s->n);
    for (int L = 0; L < s->n; L++) to[s->l2p[L]] = L;
    void *tmp = nullptr;
    bool temporary = false;
    QS_TRY(perm_buffer(s, &tmp, &temporary));
    cudaError_t e = launch_permute(s->amps, tmp, s->dt, s->n, to.data(), s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host_amps, tmp, s->amp_bytes(), cudaMemcpyDeviceToHost, s->stream);
    if (temporary) cudaFreeAsync(tmp, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "download");
    return QSIM_OK;
}

qsim_status qsim_download(qsim_state *s, void *host_amps)
{
    QS_TRY(qsim_download_async(s, host_amps));
    err_fetch(s);
    QS_CUDA(cudaStreamSynchronize(s->stream));
    return err_check(s);
}

qsim_status qsim_device_ptr(const qsim_state *s, void **dev_amps)
{
    clear_error();
    QS_TRY(check_state(s));
    if (!dev_amps) return fail(QSIM_E_INVAL, "dev_amps is NULL");
    *dev_amps = s->amps;
    return QSIM_OK;
}

qsim_status qsim_qubit_map(const qsim_state *s, int32_t *l2p)
{
    clear_error();
    QS_TRY(check_state(s));
    if (!l2p) return fail(QSIM_E_INVAL, "l2p is NULL");
    for (int q = 0; q < s->n; q++) l2p[q] = s->l2p[q];
    return QSIM_OK;
}

qsim_status qsim_materialize(qsim_state *s)
{
    clear_error();
    QS_TRY(check_state(s));
    if (is_identity(s)) return QSIM_OK;
    std::vector<int> to(s->n);
    for (int L = 0; L < s->n; L++) to[s->l2p[L]] = L;
    QS_TRY(permute_state(s, to));
    for (int q = 0; q < s->n; q++) s->l2p[q] = q;
    return QSIM_OK;
}

qsim_status qsim_synchronize(qsim_state *s)
{
    clear_error();
    QS_TRY(check_state(s));
    err_fetch(s);
    QS_CUDA(cudaStreamSynchronize(s->stream));
    return err_check(s);
}

// ------------------------------------------------------------ gates

qsim_status qsim_apply_gate(qsim_state *s, const double u[8], int target, const int *controls, int ncontrols,
                            uint64_t control_values)
{
    clear_error();
    QS_TRY(check_state(s));
    if (!u) return fail(QSIM_E_INVAL, "u is NULL");
    QS_TRY(check_qubit(s, target, "target"));
    if (ncontrols < 0 || ncontrols > QSIM_MAX_CONTROLS)
        return fail(QSIM_E_INVAL, "ncontrols %d outside [0, %d]", ncontrols, QSIM_MAX_CONTROLS);
    if (ncontrols > 0 && !controls) return fail(QSIM_E_INVAL, "controls is NULL");
    uint64_t cmask = 0, cval = 0;
    for (int j = 0; j < ncontrols; j++) {
        QS_TRY(check_qubit(s, controls[j], "control"));
        if (controls[j] == target) return fail(QSIM_E_INVAL, "control %d equals the target", target);
        uint64_t b = bit(s->l2p[controls[j]]);
        if (cmask & b) return fail(QSIM_E_INVAL, "duplicate control %d", controls[j]);
        cmask |= b;
        if ((control_values >> j) & 1) cval |= b;
    }
    cd m[4];
    for (int k = 0; k < 4; k++) m[k] = cd(u[2 * k], u[2 * k + 1]);
    QS_CUDA(launch_gate1(s, m, s->l2p[target], cmask, cval));
    return QSIM_OK;
}

qsim_status qsim_apply_cphase(qsim_state *s, int q0, int q1, double theta)
{
    clear_error();
    QS_TRY(check_state(s));
    QS_TRY(check_qubit(s, q0, "q0"));
    QS_TRY(check_qubit(s, q1, "q1"));
    if (q0 == q1) return fail(QSIM_E_INVAL, "cphase on duplicate qubit %d", q0);
    if (!std::isfinite(theta)) return fail(QSIM_E_INVAL, "theta is not finite");
    QS_CUDA(launch_cphase(s, s->l2p[q0], s->l2p[q1], theta));
    return QSIM_OK;
}

qsim_status qsim_apply_2q(qsim_state *s, const double u[32], int q0, int q1)
{
    clear_error();
    QS_TRY(check_state(s));
    if (!u) return fail(QSIM_E_INVAL, "u is NULL");
    QS_TRY(check_qubit(s, q0, "q0"));
    QS_TRY(check_qubit(s, q1, "q1"));
    if (q0 == q1) return fail(QSIM_E_INVAL, "two-qubit gate on duplicate qubit %d", q0);
    cd m[16];
    for (int k = 0; k < 16; k++) m[k] = cd(u[2 * k], u[2 * k + 1]);
    QS_CUDA(launch_gate2(s, m, s->l2p[q0], s->l2p[q1]));
    return QSIM_OK;
}

qsim_status qsim_apply_swap(qsim_state *s, int q0, int q1, int relabel)
{
    clear_error();
    QS_TRY(check_state(s));
    QS_TRY(check_qubit(s, q0, "q0"));
    QS_TRY(check_qubit(s, q1, "q1"));
    if (q0 == q1) return fail(QSIM_E_INVAL, "swap on duplicate qubit %d", q0);
    if (relabel) {
        std::swap(s->l2p[q0], s->l2p[q1]);
        return QSIM_OK;
    }
    QS_CUDA(launch_swap(s, s->l2p[q0], s->l2p[q1]));
    return QSIM_OK;
}

qsim_status qsim_apply_fused(qsim_state *s, int k, const int *qubits, const double *u, qsim_prec prec)
{
    clear_error();
    QS_TRY(check_state(s));
    if (!qubits || !u) return fail(QSIM_E_INVAL, "qubits or u is NULL");
    if (k < 1 || k > 7 || k > s->n) return fail(QSIM_E_INVAL, "k=%d outside [1, min(7, n)]", k);
    int phys[8];
    uint64_t seen = 0;
    for (int b = 0; b < k; b++) {
        QS_TRY(check_qubit(s, qubits[b], "block qubit"));
        phys[b] = s->l2p[qubits[b]];
        if (seen & bit(phys[b])) return fail(QSIM_E_INVAL, "duplicate block qubit %d", qubits[b]);
        seen |= bit(phys[b]);
    }
    size_t D = (size_t)1 << k;
    std::vector<cd> m(D * D);
    for (size_t i = 0; i < D * D; i++) m[i] = cd(u[2 * i], u[2 * i + 1]);
    if (prec == QSIM_PREC_NATIVE) {
        QS_CUDA(launch_fused_simt(s, k, phys, m.data()));
        return QSIM_OK;
    }
    if (prec != QSIM_PREC_3XTF32 && prec != QSIM_PREC_BF16X3 && prec != QSIM_PREC_BF16X6)
        return fail(QSIM_E_INVAL, "unknown prec %d", prec);
    return apply_fused_tc(s, k, phys, m.data(), prec);
}

// ------------------------------------------------------- reductions

qsim_status qsim_norm(qsim_state *s, double *out)
{
    clear_error();
    QS_TRY(check_state(s));
    if (!out) return fail(QSIM_E_INVAL, "out is NULL");
    return reduce_norm(s, out);
}

qsim_status qsim_renormalize(qsim_state *s)
{
    clear_error();
    QS_TRY(check_state(s));
    double nrm = 0;
    QS_TRY(reduce_norm(s, &nrm));
    if (!(nrm > 0) || !std::isfinite(nrm)) return fail(QSIM_E_INVAL, "cannot renormalise a ket of norm %g", nrm);
    QS_CUDA(launch_scale(s->amps, s->dt, s->N(), 1.0 / std::sqrt(nrm), s->stream));
    return QSIM_OK;
}

qsim_status qsim_measure_prob(qsim_state *s, int qubit, double *p1)
{
    clear_error();
    QS_TRY(check_state(s));
    QS_TRY(check_qubit(s, qubit, "qubit"));
    if (!p1) return fail(QSIM_E_INVAL, "p1 is NULL");
    double one = 0, all = 0;
    QS_TRY(reduce_prob1(s, s->l2p[qubit], &one, &all));
    if (!(all > 0)) return fail(QSIM_E_INVAL, "ket has zero norm");
    *p1 = one / all;
    return QSIM_OK;
}

qsim_status qsim_probs(qsim_state *s, double *host_out)
{
    clear_error();
    QS_TRY(check_state(s));
    if (!host_out) return fail(QSIM_E_INVAL, "host_out is NULL");
    size_t bytes = (size_t)8 << s->n;
    double *d = nullptr;
    QS_CUDA(cudaMallocAsync((void **)&d, bytes * (is_identity(s) ? 1 : 2), s->stream));
    qsim_status st = probs_to_device(s, d);
    double *src = d;
    if (st == QSIM_OK && !is_identity(s)) {
        std::vector<int> to(s->n);
        for (int L = 0; L < s->n; L++) to[s->l2p[L]] = L;
        // doubles are 8-byte elements like complex64 amplitudes
        cudaError_t e = launch_permute(d, d + s->N(), QSIM_C64, s->n, to.data(), s->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "permute probs");
        src = d + s->N();
    }
    if (st == QSIM_OK) {
        cudaError_t e = cudaMemcpyAsync(host_out, src, bytes, cudaMemcpyDeviceToHost, s->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "copy probs");
    }
    cudaFreeAsync(d, s->stream);
    if (st != QSIM_OK) return st;
    err_fetch(s);
    QS_CUDA(cudaStreamSynchronize(s->stream));
    return err_check(s);
}

qsim_status qsim_inner_product(qsim_state *a, qsim_state *b, double out[2])
{
    clear_error();
    QS_TRY(check_state(a));
    QS_TRY(check_state(b));
    if (!out) return fail(QSIM_E_INVAL, "out is NULL");
    if (a->n != b->n || a->dt != b->dt) return fail(QSIM_E_INVAL, "inner product of kets of different n or dtype");
    if (a->l2p != b->l2p) {
        QS_TRY(qsim_materialize(a));
        QS_TRY(qsim_materialize(b));
    }
    return reduce_inner(a, b, out);
}

qsim_status qsim_bloch(qsim_state *s, int qubit, double r[3])
{
    clear_error();
    QS_TRY(check_state(s));
    QS_TRY(check_qubit(s, qubit, "qubit"));
    if (!r) return fail(QSIM_E_INVAL, "r is NULL");
    double v[4];
    QS_TRY(reduce_bloch(s, s->l2p[qubit], v));
    double tr = v[0] + v[1];
    if (!(tr > 0)) return fail(QSIM_E_INVAL, "ket has zero norm");
    r[0] = 2.0 * v[2] / tr;
    r[1] = 2.0 * v[3] / tr;
    r[2] = (v[0] - v[1]) / tr;
    return QSIM_OK;
}

qsim_status qsim_bloch_all(qsim_state *s, double *r)
{
    clear_error();
    QS_TRY(check_state(s));
    if (!r) return fail(QSIM_E_INVAL, "r is NULL");
    std::vector<double> sums(4 * (size_t)s->n);
    QS_TRY(reduce_bloch_all(s, sums.data()));
    for (int L = 0; L < s->n; L++) {
        const double *v = &sums[4 * (size_t)s->l2p[L]];
        double tr = v[0] + v[1];
        if (!(tr > 0)) return fail(QSIM_E_INVAL, "ket has zero norm");
        r[3 * L + 0] = 2.0 * v[2] / tr;
        r[3 * L + 1] = 2.0 * v[3] / tr;
        r[3 * L + 2] = (v[0] - v[1]) / tr;
    }
    return QSIM_OK;
}

const char *qsim_version(void) { return "qsim-gb300 0.1 (sm_103a)"; }

}  // extern "C"

namespace qs {

qsim_status err_ensure(qsim_state *s)
{
    if (s->d_err) return QSIM_OK;
    QS_CUDA(cudaMalloc((void **)&s->d_err, sizeof(int)));
    QS_CUDA(cudaMallocHost((void **)&s->h_err, sizeof(int)));
    *s->h_err = 0;
    QS_CUDA(cudaMemsetAsync(s->d_err, 0, sizeof(int), s->stream));
    return QSIM_OK;
}

void err_fetch(qsim_state *s)
{
    if (s->d_err) cudaMemcpyAsync(s->h_err, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
}

qsim_status err_check(qsim_state *s)
{
    if (!s->h_err || !*s->h_err) return QSIM_OK;
    *s->h_err = 0;
    cudaMemsetAsync(s->d_err, 0, sizeof(int), s->stream);
    return fail(QSIM_E_TIMEOUT, "tensor-core block: a bounded wait in the MMA pipeline gave up (result invalid)");
}

}  // namespace qs
