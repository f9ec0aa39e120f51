// qsim_run_circuit: the per-gate path (one kernel per gate) and dispatch to
// fused plans.
#include <cmath>

#include "qsim_internal.h"
#include "plan.h"

using namespace qs;

namespace qs {

qsim_status validate_circuit(const qsim_circuit *c)
{
    if (!c) return fail(QSIM_E_INVAL, "circuit is NULL");
    if (c->n < 1 || c->n > 64) return fail(QSIM_E_INVAL, "circuit n=%d out of range", c->n);
    if (c->ngates < 0 || (c->ngates > 0 && !c->gates)) return fail(QSIM_E_INVAL, "circuit has no gate array");
    for (int k = 0; k < c->ngates; k++) {
        qsim_status st = validate_gate(c->gates[k], c->n, c->matrices, c->nmatrix_doubles);
        if (st != QSIM_OK) return fail(st, "gate %d: %s", k, g_last_error_cstr());
    }
    return QSIM_OK;
}

// One gate through the per-gate kernels (logical qubits -> physical bits).
qsim_status apply_one_gate(qsim_state *s, const qsim_gate &g, const double *pool, int64_t pool_len, bool relabel)
{
    cd m[16];
    int d = gate_matrix(g, pool, pool_len, m);
    if (d == 2) {
        uint64_t cmask = 0, cval = 0;
        for (int j = 0; j < g.ncontrols; j++) {
            uint64_t b = bit(s->l2p[g.controls[j]]);
            cmask |= b;
            if ((g.control_values >> j) & 1) cval |= b;
        }
        QS_CUDA(launch_gate1(s, m, s->l2p[g.q0], cmask, cval));
        return QSIM_OK;
    }
    int p0 = s->l2p[g.q0], p1 = s->l2p[g.q1];
    switch (g.kind) {
    case QSIM_G_CP:
        QS_CUDA(launch_cphase(s, p0, p1, g.params[0]));
        return QSIM_OK;
    case QSIM_G_SWAP:
        if (relabel) std::swap(s->l2p[g.q0], s->l2p[g.q1]);
        else QS_CUDA(launch_swap(s, p0, p1));
        return QSIM_OK;
    default:
        QS_CUDA(launch_gate2(s, m, p0, p1));
        return QSIM_OK;
    }
}

}  // namespace qs

extern "C" {

qsim_status qsim_run_circuit(qsim_state *s, const qsim_circuit *c, const qsim_run_opts *opts)
{
    clear_error();
    if (!s || !s->amps) return fail(QSIM_E_INVAL, "state is NULL");
    QS_TRY(validate_circuit(c));
    if (c->n != s->n) return fail(QSIM_E_INVAL, "circuit has n=%d but the state n=%d", c->n, s->n);
    qsim_run_opts o{};
    if (opts) o = *opts;
    if (o.mode == QSIM_MODE_PER_GATE) {
        for (int k = 0; k < c->ngates; k++)
            QS_TRY(apply_one_gate(s, c->gates[k], c->matrices, c->nmatrix_doubles, o.relabel_swaps != 0));
        return QSIM_OK;
    }
    if (o.mode != QSIM_MODE_FUSED) return fail(QSIM_E_INVAL, "unknown mode %d", o.mode);
    if (c->n < 9) {
        // tiles need at least 9 qubits; smaller kets run gate by gate
        for (int k = 0; k < c->ngates; k++)
            QS_TRY(apply_one_gate(s, c->gates[k], c->matrices, c->nmatrix_doubles, true));
        return QSIM_OK;
    }
    qsim_plan *p = nullptr;
    QS_TRY(qsim_plan_create_for_state(c, s, &o, &p));
    qsim_status st = qsim_plan_execute(s, p);
    qsim_plan_destroy(p);
    return st;
}

}  // extern "C"
