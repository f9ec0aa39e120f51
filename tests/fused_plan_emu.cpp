// Host-side check of the fused SIMT planner (test infrastructure).
//
// Links the library's host planner and applies a fused plan to a ket on the
// CPU with the semantics the fused-pass kernel gives the plan's staged
// constant block (the same bytes the kernel reads): per tile of 2^t
// amplitudes (tile bits: the c low qubits, then the pass's high qubits),
// the per-tile factors of the deferred phases, then the ops in order on
// register bits of the current map (a transpose only changes the map: the
// tile is kept as one array indexed by tile bits), then the store. Per-gate
// steps and the global phase are applied as plain matrix-vector updates.
// Arithmetic is FP64 on the staged coefficients (FP32 for complex64 plans).
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>

#include "plan.h"

namespace qs {
qsim_status plan_build(const qsim_circuit *, qsim_dtype, const qsim_run_opts *, const int *, qsim_plan *);
// the tensor-core planner is linked in but not used here
qsim_status tc_build(int, int, const int *, const cd *, qsim_prec, std::vector<unsigned char> &, TcSpec &, int)
{
    return QSIM_E_UNSUPPORTED;
}
}  // namespace qs

using namespace qs;

namespace {

struct Stage {
    const FPassDev *d;
    const unsigned char *b;
    bool wide;   // coefficients in FP64
    cd coef(int i) const
    {
        if (wide) {
            double re, im;
            memcpy(&re, b + d->off_cf + 8 * i, 8);
            memcpy(&im, b + d->off_cf + 8 * (i + 1), 8);
            return cd(re, im);
        }
        float re, im;
        memcpy(&re, b + d->off_cf + 4 * i, 4);
        memcpy(&im, b + d->off_cf + 4 * (i + 1), 4);
        return cd(re, im);
    }
    double real(int i) const
    {
        if (wide) {
            double v;
            memcpy(&v, b + d->off_cf + 8 * i, 8);
            return v;
        }
        float v;
        memcpy(&v, b + d->off_cf + 4 * i, 4);
        return v;
    }
    FOp op(int i) const
    {
        FOp o;
        memcpy(&o, b + d->off_ops + sizeof(FOp) * i, sizeof(FOp));
        return o;
    }
    FMap map(int i) const
    {
        FMap m;
        memcpy(&m, b + d->off_maps + sizeof(FMap) * i, sizeof(FMap));
        return m;
    }
    int32_t i32(int off, int i) const
    {
        int32_t v;
        memcpy(&v, b + off + 4 * i, 4);
        return v;
    }
    uint64_t u64(int off, int i) const
    {
        uint64_t v;
        memcpy(&v, b + off + 8 * i, 8);
        return v;
    }
};

cd turns_phase(uint64_t tt)
{
    const double ang = 2.0 * M_PI * ((double)(int64_t)tt / 18446744073709551616.0);
    return cd(std::cos(ang), std::sin(ang));
}

void run_pass(const PlanPass &ps, bool wide, std::vector<cd> &a)
{
    const FPassDev &d = ps.dev;
    Stage S{&d, ps.stage.data(), wide};
    const int t = d.t, c = d.c, RB = d.RB, W = d.W;
    const uint64_t T = 1ull << t;
    const uint64_t ntiles = 1ull << (d.n - t);
    // tile bit -> physical qubit
    std::vector<int> phys_bit(t);
    for (int b = 0; b < c; b++) phys_bit[b] = b;
    for (int j = 0; j < t - c; j++) phys_bit[c + j] = d.hq[j];
    std::vector<cd> tile(T), E(d.nlin > 0 ? d.nlin : 1);
    for (uint64_t tl = 0; tl < ntiles; tl++) {
        uint64_t base = tl << c;
        for (int j = 0; j < d.ins.npos; j++) {
            const int p = d.ins.pos[j];
            base = ((base >> p) << (p + 1)) | (base & ((1ull << p) - 1));
        }
        for (int l = 0; l < d.nlin; l++) {
            uint64_t sacc = 0;
            for (int e = S.i32(d.off_lin, l); e < S.i32(d.off_lin, l + 1); e++)
                if ((base >> S.i32(d.off_eb, e)) & 1) sacc += S.u64(d.off_et, e);
            E[l] = turns_phase(sacc);
        }
        auto phys = [&](uint64_t i) {
            uint64_t o = base;
            for (int b = 0; b < t; b++)
                if ((i >> b) & 1) o |= 1ull << phys_bit[b];
            return o;
        };
        for (uint64_t i = 0; i < T; i++) tile[i] = a[phys(i)];
        FMap mp = S.map(0);
        auto regidx = [&](uint64_t i) {
            int x = 0;
            for (int r = 0; r < RB; r++) x |= (int)((i >> mp.reg[r]) & 1) << r;
            return x;
        };
        auto tidx = [&](uint64_t i) {
            int ln = 0, wp = 0;
            for (int l = 0; l < 5; l++) ln |= (int)((i >> mp.lane[l]) & 1) << l;
            for (int w = 0; w < W; w++) wp |= (int)((i >> mp.warp[w]) & 1) << w;
            return ln + 32 * wp;
        };
        for (int k = 0; k < d.nops; k++) {
            const FOp op = S.op(k);
            switch (op.kind) {
            case FO_XPOSE:
                mp = S.map(op.aux);
                break;
            case FO_RSCALE: {
                const double sc = S.real(op.coef);
                for (auto &v : tile) v *= sc;
                break;
            }
            case FO_SCALE: {
                const cd sc = S.coef(op.coef);
                for (auto &v : tile) v *= sc;
                break;
            }
            case FO_G1F: {
                const int uf = op.j1 & 15, pr = op.j1 >> 4, J = op.j0;
                if (uf == U_NONE && pr == PRE_NONE) break;
                const uint64_t tb = 1ull << mp.reg[J];
                for (uint64_t i = 0; i < T; i++) {
                    if (i & tb) continue;
                    const int x = regidx(i);
                    const int xr = ((x >> (J + 1)) << J) | (x & ((1 << J) - 1));
                    cd p = tile[i], q = tile[i | tb];
                    if (pr == PRE_D || pr == PRE_FD) {
                        cd f = S.coef((op.aux3 >= 0 ? op.aux3 : 0) + 2 * xr);
                        if (pr == PRE_FD) {
                            cd g = S.coef(op.aux4);
                            if (op.aux >= 0) g *= S.coef(op.aux + 2 * tidx(i));
                            if (op.aux2 >= 0) g *= E[op.aux2];
                            f *= g;
                        }
                        q *= f;
                    }
                    cd o0, o1;
                    if (uf == U_NONE) {
                        o0 = p;
                        o1 = q;
                    } else if (uf == U_HAD) {
                        o0 = p + q;
                        o1 = p - q;
                    } else if (uf == U_REAL) {
                        o0 = S.real(op.coef) * p + S.real(op.coef + 1) * q;
                        o1 = S.real(op.coef + 2) * p + S.real(op.coef + 3) * q;
                    } else if (uf == U_CPLX) {
                        o0 = S.coef(op.coef) * p + S.coef(op.coef + 2) * q;
                        o1 = S.coef(op.coef + 4) * p + S.coef(op.coef + 6) * q;
                    } else {
                        o0 = S.coef(op.coef) * q;
                        o1 = S.coef(op.coef + 2) * p;
                    }
                    tile[i] = o0;
                    tile[i | tb] = o1;
                }
                break;
            }
            case FO_G2:
            case FO_G2M: {
                const uint64_t b0 = 1ull << mp.reg[op.j0], b1 = 1ull << mp.reg[op.j1];
                for (uint64_t i = 0; i < T; i++) {
                    if (i & (b0 | b1)) continue;
                    const uint64_t id[4] = {i, i | b0, i | b1, i | b0 | b1};
                    cd in[4];
                    for (int k2 = 0; k2 < 4; k2++) in[k2] = tile[id[k2]];
                    for (int r = 0; r < 4; r++) {
                        cd o = 0.0;
                        if (op.kind == FO_G2) {
                            for (int k2 = 0; k2 < 4; k2++) o += S.coef(op.coef + 2 * (r * 4 + k2)) * in[k2];
                        } else {
                            o = S.coef(op.coef + 2 * r) * in[(op.aux >> (2 * r)) & 3];
                        }
                        tile[id[r]] = o;
                    }
                }
                break;
            }
            default:
                break;
            }
        }
        for (uint64_t i = 0; i < T; i++) a[phys(i)] = tile[i];
    }
}

}  // namespace

// psi_io: 2^n interleaved complex doubles in logical order (in and out).
// dt: qsim_dtype of the plan (coefficient precision, tile size); tile: tile
// qubits (0: default); start_l2p: NULL = identity. info[0..3]: passes,
// per-gate steps, transposes, registers per thread (log2).
extern "C" int emu_fused_run(const qsim_circuit *c, int dt, int tile, const int *start_l2p, double *psi_io,
                             int64_t info[4])
{
    qsim_run_opts o;
    memset(&o, 0, sizeof o);
    o.mode = QSIM_MODE_FUSED;
    o.tile_qubits = tile;
    o.relabel_swaps = 1;
    qsim_plan P;
    qsim_status st = plan_build(c, (qsim_dtype)dt, &o, start_l2p, &P);
    if (st != QSIM_OK) return (int)st;
    const int n = c->n;
    const uint64_t N = 1ull << n;
    std::vector<cd> a(N), b(N);
    for (uint64_t i = 0; i < N; i++) {
        uint64_t j = 0;
        for (int q = 0; q < n; q++)
            if ((i >> q) & 1) j |= 1ull << P.start_l2p[q];
        a[j] = cd(psi_io[2 * i], psi_io[2 * i + 1]);
    }
    int64_t npergate = 0, nx = 0;
    for (const PlanStep &s : P.steps) {
        if (s.kind == 0) {
            const PlanPass &ps = P.passes[s.pass];
            run_pass(ps, dt == QSIM_C128, a);
            for (int k = 0; k < ps.dev.nops; k++) {
                FOp op;
                memcpy(&op, ps.stage.data() + ps.dev.off_ops + sizeof(FOp) * k, sizeof(FOp));
                nx += op.kind == FO_XPOSE;
            }
        } else if (s.kind == 1) {
            npergate++;
            const qsim_gate &g = s.gate;
            if (g.kind == QSIM_G_CP) {
                cd f = std::polar(1.0, g.params[0]);
                for (uint64_t i = 0; i < N; i++)
                    if (((i >> g.q0) & 1) && ((i >> g.q1) & 1)) a[i] *= f;
            } else {
                uint64_t cm = 0, cv = 0;
                for (int j = 0; j < g.ncontrols; j++) {
                    cm |= 1ull << g.controls[j];
                    if ((g.control_values >> j) & 1) cv |= 1ull << g.controls[j];
                }
                for (uint64_t i = 0; i < N; i++) {
                    if (((i >> g.q0) & 1) || (i & cm) != cv) continue;
                    uint64_t j = i | (1ull << g.q0);
                    cd x = a[i], y = a[j];
                    a[i] = s.mat[0] * x + s.mat[1] * y;
                    a[j] = s.mat[2] * x + s.mat[3] * y;
                }
            }
        } else if (s.kind == 2) {
            for (cd &x : a) x *= s.phase;
        } else {
            return 100 + s.kind;
        }
    }
    for (uint64_t i = 0; i < N; i++) {
        uint64_t j = 0;
        for (int q = 0; q < n; q++)
            if ((i >> q) & 1) j |= 1ull << P.final_l2p[q];
        b[i] = a[j];
    }
    for (uint64_t i = 0; i < N; i++) {
        psi_io[2 * i] = b[i].real();
        psi_io[2 * i + 1] = b[i].imag();
    }
    info[0] = (int64_t)P.passes.size();
    info[1] = npergate;
    info[2] = nx;
    info[3] = P.RB;
    return 0;
}
