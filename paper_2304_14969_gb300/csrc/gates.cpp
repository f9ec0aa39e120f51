// Host-side FP64 gate matrices and validation for the GPU library.
//
// Kernels only multiply and add: every matrix entry (and every phase) is
// formed here in double precision and passed to the device as constants.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "qsim_internal.h"

namespace qs {

static thread_local std::string g_err;

qsim_status fail(qsim_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

qsim_status cuda_fail(cudaError_t e, const char *what)
{
    cudaGetLastError();  // clear a sticky launch error where possible
    qsim_status st = (e == cudaErrorMemoryAllocation) ? QSIM_E_NOMEM : QSIM_E_CUDA;
    return fail(st, "%s: %s", what, cudaGetErrorString(e));
}

void clear_error() { g_err.clear(); }

const char *g_last_error_cstr() { return g_err.c_str(); }

bool gate_is_two_qubit_kind(int kind) { return kind >= 16; }

// Sec. III.C U(theta, phi, lambda); sqrt(P) = ((1+i) I + (1-i) P)/2 for the
// Paulis and W = (X + Y)/sqrt(2); fSim(theta, phi) on |00>,|01>,|10>,|11>.
int gate_matrix(const qsim_gate &g, const double *pool, int64_t pool_len, cd *m)
{
    const cd I(0.0, 1.0);
    const double h = 1.0 / std::sqrt(2.0);
    auto pauli_root = [&](const cd P[4]) {
        for (int k = 0; k < 4; k++) {
            cd id = (k == 0 || k == 3) ? cd(1.0) : cd(0.0);
            m[k] = (cd(1.0, 1.0) * id + cd(1.0, -1.0) * P[k]) * 0.5;
        }
    };
    switch (g.kind) {
    case QSIM_G_H: m[0] = h; m[1] = h; m[2] = h; m[3] = -h; return 2;
    case QSIM_G_X: m[0] = 0.0; m[1] = 1.0; m[2] = 1.0; m[3] = 0.0; return 2;
    case QSIM_G_Y: m[0] = 0.0; m[1] = -I; m[2] = I; m[3] = 0.0; return 2;
    case QSIM_G_Z: m[0] = 1.0; m[1] = 0.0; m[2] = 0.0; m[3] = -1.0; return 2;
    case QSIM_G_S: m[0] = 1.0; m[1] = 0.0; m[2] = 0.0; m[3] = I; return 2;
    case QSIM_G_T: m[0] = 1.0; m[1] = 0.0; m[2] = 0.0; m[3] = std::polar(1.0, M_PI / 4); return 2;
    case QSIM_G_SQRTX: { cd P[4] = {0.0, 1.0, 1.0, 0.0}; pauli_root(P); return 2; }
    case QSIM_G_SQRTY: { cd P[4] = {0.0, -I, I, 0.0}; pauli_root(P); return 2; }
    case QSIM_G_SQRTW: { cd P[4] = {0.0, cd(h, -h), cd(h, h), 0.0}; pauli_root(P); return 2; }
    case QSIM_G_U3: {
        double th = g.params[0], ph = g.params[1], la = g.params[2];
        m[0] = std::cos(th / 2);
        m[1] = -std::polar(1.0, la) * std::sin(th / 2);
        m[2] = std::polar(1.0, ph) * std::sin(th / 2);
        m[3] = std::polar(1.0, ph + la) * std::cos(th / 2);
        return 2;
    }
    case QSIM_G_PHASE: m[0] = 1.0; m[1] = 0.0; m[2] = 0.0; m[3] = std::polar(1.0, g.params[0]); return 2;
    case QSIM_G_RZ:
        m[0] = std::polar(1.0, -g.params[0] / 2); m[1] = 0.0; m[2] = 0.0;
        m[3] = std::polar(1.0, g.params[0] / 2);
        return 2;
    case QSIM_G_MAT1:
        if (!pool || g.matrix_offset < 0 || g.matrix_offset + 8 > pool_len) return 0;
        for (int k = 0; k < 4; k++) m[k] = cd(pool[g.matrix_offset + 2 * k], pool[g.matrix_offset + 2 * k + 1]);
        return 2;
    case QSIM_G_CP:
        for (int k = 0; k < 16; k++) m[k] = 0.0;
        m[0] = m[5] = m[10] = 1.0;
        m[15] = std::polar(1.0, g.params[0]);
        return 4;
    case QSIM_G_SWAP:
        for (int k = 0; k < 16; k++) m[k] = 0.0;
        m[0] = m[6] = m[9] = m[15] = 1.0;
        return 4;
    case QSIM_G_FSIM: {
        double th = g.params[0], ph = g.params[1];
        for (int k = 0; k < 16; k++) m[k] = 0.0;
        m[0] = 1.0;
        m[5] = std::cos(th); m[6] = -I * std::sin(th);
        m[9] = -I * std::sin(th); m[10] = std::cos(th);
        m[15] = std::polar(1.0, -ph);
        return 4;
    }
    case QSIM_G_MAT2:
        if (!pool || g.matrix_offset < 0 || g.matrix_offset + 32 > pool_len) return 0;
        for (int k = 0; k < 16; k++) m[k] = cd(pool[g.matrix_offset + 2 * k], pool[g.matrix_offset + 2 * k + 1]);
        return 4;
    default:
        return 0;
    }
}

bool gate_is_diagonal(const qsim_gate &g)
{
    switch (g.kind) {
    case QSIM_G_Z: case QSIM_G_S: case QSIM_G_T: case QSIM_G_PHASE: case QSIM_G_RZ: case QSIM_G_CP:
        return true;
    default:
        return false;
    }
}

qsim_status validate_gate(const qsim_gate &g, int n, const double *pool, int64_t pool_len)
{
    cd m[16];
    int d = gate_matrix(g, pool, pool_len, m);
    if (d == 0) return fail(QSIM_E_INVAL, "gate kind %d unknown or matrix_offset out of range", g.kind);
    if (g.q0 < 0 || g.q0 >= n) return fail(QSIM_E_INVAL, "qubit %d out of range for n=%d", g.q0, n);
    if (d == 4) {
        if (g.q1 < 0 || g.q1 >= n) return fail(QSIM_E_INVAL, "qubit %d out of range for n=%d", g.q1, n);
        if (g.q1 == g.q0) return fail(QSIM_E_INVAL, "two-qubit gate on duplicate qubit %d", g.q0);
        if (g.ncontrols != 0) return fail(QSIM_E_INVAL, "two-qubit kinds take no controls");
    } else {
        if (g.ncontrols < 0 || g.ncontrols > QSIM_MAX_CONTROLS)
            return fail(QSIM_E_INVAL, "ncontrols %d outside [0, %d]", g.ncontrols, QSIM_MAX_CONTROLS);
        for (int j = 0; j < g.ncontrols; j++) {
            int c = g.controls[j];
            if (c < 0 || c >= n) return fail(QSIM_E_INVAL, "control %d out of range for n=%d", c, n);
            if (c == g.q0) return fail(QSIM_E_INVAL, "control %d equals the target", c);
            for (int i = 0; i < j; i++)
                if (g.controls[i] == c) return fail(QSIM_E_INVAL, "duplicate control %d", c);
        }
    }
    return QSIM_OK;
}

}  // namespace qs

extern "C" const char *qsim_last_error(void) { return qs::g_last_error_cstr(); }
