// Fusion planner: turns a circuit into fused passes over the ket.
//
// Table I of arXiv 2304.14969 lists the ideas this planner builds on:
// gates "coalesced ... with a single traversal", SWAP as a constant-cost
// qubit relabel, and controlled-phase gates "buffered and commuted" rather
// than applied one by one. Concretely:
//
//  * Every gate is classified once (FP64 host matrices). Diagonal gates
//    (CP, phase, Z/S/T, RZ, controlled diagonals) never move data: they are
//    decomposed into a global phase, linear terms theta*b_q and pair terms
//    theta*b_q*b_r, and kept "pending". A pending term commutes with every
//    gate that does not densely act on its qubits, so it is flushed only
//    right before the next dense gate on one of its qubits, where it costs
//    one multiply per amplitude on chip.
//  * Dense gates (1 qubit, or 2 qubits incl. singly-controlled 1-qubit
//    gates) are grouped into passes by a commutation-aware sweep: a pass
//    owns a tile of t qubits (the c lowest physical qubits plus high qubits
//    added greedily in circuit order while room remains); a gate runs in
//    the pass when all its qubits are in the tile and no earlier unrun gate
//    shares a qubit with it.
//  * Inside a pass, gates act on RB register bits of each thread; a new
//    "phase" (one transpose through shared memory) brings the next gates'
//    qubits into registers.
//  * Gates with two or more controls, and pending terms left at the end,
//    run through the per-gate kernels.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>

#include "plan.h"

namespace qs {

qsim_status validate_circuit(const qsim_circuit *c);

namespace {

const double kTiny = 1e-14;

uint64_t to_turns(double theta)
{
    long double f = (long double)theta / (2.0L * 3.14159265358979323846264338327950288L);
    f -= std::floor(f);
    long double x = f * 18446744073709551616.0L;
    if (x >= 18446744073709551615.0L) return 0;
    return (uint64_t)x;
}

struct Term {
    int a, b;      // physical bits; b = -1 for a linear term
    double th;
};

struct Item {
    int kind = 0;            // 0 dense, 1 diagonal, 2 barrier
    int nq = 0;
    int q[2] = {0, 0};       // physical bits; dense: q[0] = matrix bit 0
    cd m[16];
    std::vector<Term> terms; // diagonal
    cd gphase = 1.0;         // diagonal
    qsim_gate gate{};        // barrier (physical qubits)
    std::vector<cd> bmat;
};

bool is_diag(const cd *m, int d)
{
    for (int r = 0; r < d; r++)
        for (int c = 0; c < d; c++)
            if (r != c && std::abs(m[r * d + c]) > kTiny) return false;
    for (int r = 0; r < d; r++)
        if (std::abs(std::abs(m[r * d + r]) - 1.0) > 1e-12) return false;
    return true;
}

void add_term(Item &it, int a, int b, double th)
{
    // terms that vanish modulo one turn are dropped
    if (std::fabs(std::remainder(th, 2.0 * M_PI)) < 1e-15) return;
    it.terms.push_back({a, b, th});
}

// Diagonal of phases alpha[idx] on qubits q (q[0] = bit 0) -> terms.
void diag_terms(const cd *m, int nq, const int *q, Item &it)
{
    if (nq == 1) {
        double a0 = std::arg(m[0]), a1 = std::arg(m[3]);
        it.gphase *= std::polar(1.0, a0);
        add_term(it, q[0], -1, a1 - a0);
    } else {
        double a[4];
        for (int k = 0; k < 4; k++) a[k] = std::arg(m[k * 4 + k]);
        it.gphase *= std::polar(1.0, a[0]);
        add_term(it, q[0], -1, a[1] - a[0]);
        add_term(it, q[1], -1, a[2] - a[0]);
        add_term(it, q[0], q[1], a[3] - a[1] - a[2] + a[0]);
    }
}

// Shared-memory slot of tile index t: the low bank bits are XORed with the
// higher bit groups (linear over XOR, so slot(a ^ b) = slot(a) ^ slot(b)).
uint32_t swz_host(uint32_t t, qsim_dtype dt)
{
    if (dt == QSIM_C64) return t ^ (((t >> 4) ^ (t >> 8) ^ (t >> 12)) & 15u);
    return t ^ (((t >> 3) ^ (t >> 6) ^ (t >> 9) ^ (t >> 12)) & 7u);
}

// ------------------------------------------------------------ pass builder

struct Builder {
    qsim_plan &P;
    qsim_dtype dt;
    int n, t, c, RB, W, NT;
    std::vector<Term> pending;
    cd gphase = 1.0;

    Builder(qsim_plan &p, qsim_dtype d, int n_, int t_, int c_, int rb) : P(p), dt(d), n(n_), t(t_), c(c_), RB(rb)
    {
        W = t - RB - 5;
        NT = 1 << (t - RB);
    }

    int add_coef(const cd *v, int count, bool realonly = false)
    {
        int off = (int)P.coef.size();
        for (int i = 0; i < count; i++) {
            P.coef.push_back(v[i].real());
            if (!realonly) P.coef.push_back(v[i].imag());
        }
        return off;
    }

    // -------- per-pass state
    std::vector<int> tq;         // tau bit -> physical
    std::vector<int> tau_of;     // physical -> tau bit or -1
    int reg[kMaxRB], lane[5], warp[kMaxW];
    int cur_map = -1;
    int lin_count = 0;
    double pass_scale = 1.0;
    PlanPass *pass = nullptr;

    int reg_of_tau(int tb) const
    {
        for (int r = 0; r < RB; r++)
            if (reg[r] == tb) return r;
        return -1;
    }

    int push_map()
    {
        FMap m;
        memset(&m, 0, sizeof m);
        for (int r = 0; r < RB; r++) m.reg[r] = (int8_t)reg[r];
        for (int l = 0; l < 5; l++) m.lane[l] = (int8_t)lane[l];
        for (int w = 0; w < W; w++) m.warp[w] = (int8_t)warp[w];
        for (int x = 0; x < (1 << RB); x++) {
            uint32_t tt = 0;
            uint64_t pp = 0;
            for (int r = 0; r < RB; r++)
                if ((x >> r) & 1) {
                    tt |= 1u << reg[r];
                    pp |= 1ull << tq[reg[r]];
                }
            m.treg[x] = tt;
            m.tsw[x] = swz_host(tt, dt);
            m.preg[x] = pp;
        }
        P.maps.push_back(m);
        return (int)P.maps.size() - 1 - pass->map_begin;
    }

    // Chooses lanes and warps for the tau bits not in registers. load_store:
    // lanes are the 5 lowest tau bits (coalesced HBM access).
    void assign_lanes(bool load_store)
    {
        std::vector<int> rest;
        for (int b = 0; b < t; b++)
            if (reg_of_tau(b) < 0) rest.push_back(b);
        std::vector<int> ln;
        bool low_free = true;
        for (int r = 0; r < RB; r++) low_free = low_free && reg[r] >= 5;
        if (load_store || low_free) {
            // lanes on the 5 lowest tile bits: coalesced HBM access, and a
            // phase that can store without another transpose
            for (int l = 0; l < 5; l++) ln.push_back(l);
        } else {
            // cover residues mod 4 (shared-memory swizzle folds bit groups of 4)
            for (int r = 0; r < 4 && (int)ln.size() < 5; r++)
                for (int b : rest)
                    if (b % 4 == r && std::find(ln.begin(), ln.end(), b) == ln.end()) {
                        ln.push_back(b);
                        break;
                    }
            for (int b : rest)
                if ((int)ln.size() < 5 && std::find(ln.begin(), ln.end(), b) == ln.end()) ln.push_back(b);
        }
        int w = 0;
        for (int l = 0; l < 5; l++) lane[l] = ln[l];
        for (int b : rest)
            if (std::find(ln.begin(), ln.end(), b) == ln.end()) warp[w++] = b;
    }

    void emit(int kind, int j0, int j1, int coef, int aux, int aux2)
    {
        P.ops.push_back(FOp{kind, j0, j1, coef, aux, aux2, 0, 0});
    }

    // Register set for a new phase starting at dense op i of `ops`.
    void choose_regs(const std::vector<std::vector<int>> &opt, size_t i, bool exclude_low)
    {
        std::vector<int> S;
        for (size_t j = i; j < opt.size(); j++) {
            std::vector<int> U = S;
            bool bad = false;
            for (int b : opt[j]) {
                if (exclude_low && b < 5) bad = true;
                if (std::find(U.begin(), U.end(), b) == U.end()) U.push_back(b);
            }
            if (bad || (int)U.size() > RB) break;
            S = U;
        }
        // pad: bits needed soonest by later ops, then the highest tau bits
        for (size_t j = i; j < opt.size() && (int)S.size() < RB; j++)
            for (int b : opt[j])
                if ((int)S.size() < RB && !(exclude_low && b < 5) && std::find(S.begin(), S.end(), b) == S.end())
                    S.push_back(b);
        for (int b = t - 1; b >= 0 && (int)S.size() < RB; b--)
            if (!(exclude_low && b < 5) && std::find(S.begin(), S.end(), b) == S.end()) S.push_back(b);
        for (int r = 0; r < RB; r++) reg[r] = S[r];
    }

    // Takes the pending terms touching any physical qubit of `phys` (all in
    // registers now) and returns, per register bit, the prefactor of the
    // amplitudes with that bit set: a constant angle, partners among the
    // other register bits, partners on lane/warp bits and partners outside
    // the tile. A pair term between two op qubits goes to the first one.
    struct Pre {
        double th0 = 0;
        std::map<int, double> regp;                  // other register bit -> angle
        std::vector<std::pair<int, double>> tile;    // tau bit (lane/warp) -> angle
        std::vector<std::pair<int, double>> ext;     // physical bit outside the tile -> angle
    };
    std::map<int, Pre> take_pending(const std::vector<int> &phys)
    {
        std::map<int, Pre> pre;
        std::vector<Term> keep;
        auto touches = [&](int q) { return std::find(phys.begin(), phys.end(), q) != phys.end(); };
        for (const Term &tm : pending) {
            if (!touches(tm.a) && !(tm.b >= 0 && touches(tm.b))) {
                keep.push_back(tm);
                continue;
            }
            int a = tm.a, b = tm.b;
            if (b >= 0 && !touches(a)) std::swap(a, b);  // a is an op qubit
            int ra = reg_of_tau(tau_of[a]);
            Pre &P0 = pre[ra];
            if (b < 0) {
                P0.th0 += tm.th;
                continue;
            }
            int tb = tau_of[b];
            int rb = tb >= 0 ? reg_of_tau(tb) : -1;
            if (rb >= 0) P0.regp[rb] += tm.th;
            else if (tb >= 0) P0.tile.push_back({tb, tm.th});
            else P0.ext.push_back({b, tm.th});
        }
        pending.swap(keep);
        return pre;
    }

    // Emits a FO_G1F op on register bit r with prefactor `pr` and matrix form
    // uform (U_NONE for a pure phase op), matrix coefficients at ucoef.
    void emit_g1f(int r, const Pre &pr, int uform, int ucoef)
    {
        const bool has_f = !pr.tile.empty() || !pr.ext.empty();
        const bool has_d = !pr.regp.empty();
        const cd c0 = std::polar(1.0, pr.th0);
        const bool has_c = std::abs(c0 - cd(1.0)) > 1e-15;
        int pre = !has_f && !has_d && !has_c ? PRE_NONE : (!has_f ? PRE_D : PRE_FD);
        if (uform == U_NONE && pre == PRE_NONE) return;   // nothing to do
        int oc0 = add_coef(&c0, 1);
        int taux = -1, laux = -1, daux = -1;
        if (!pr.tile.empty()) {
            std::vector<cd> tab(NT);
            for (int tid = 0; tid < NT; tid++) {
                int ln = tid & 31, wp = tid >> 5;
                uint32_t tt = 0;
                for (int l = 0; l < 5; l++)
                    if ((ln >> l) & 1) tt |= 1u << lane[l];
                for (int w = 0; w < W; w++)
                    if ((wp >> w) & 1) tt |= 1u << warp[w];
                double ang = 0;
                for (auto &pt : pr.tile)
                    if ((tt >> pt.first) & 1) ang += pt.second;
                tab[tid] = std::polar(1.0, ang);
            }
            taux = add_coef(tab.data(), NT);
        }
        if (!pr.ext.empty()) {
            laux = lin_count++;
            for (auto &pe : pr.ext) {
                P.ext_bit.push_back(pe.first);
                P.ext_tw.push_back(to_turns(pe.second));
            }
            P.lin_off.push_back((int32_t)P.ext_bit.size());
        }
        if (pre != PRE_NONE) {
            // register-partner table over x without bit r; PRE_D folds c0 in
            int half = 1 << (RB - 1);
            std::vector<cd> tab(half);
            for (int xr = 0; xr < half; xr++) {
                int x = ((xr >> r) << (r + 1)) | (xr & ((1 << r) - 1));
                double ang = pre == PRE_D ? pr.th0 : 0.0;
                for (auto &kv : pr.regp)
                    if ((x >> kv.first) & 1) ang += kv.second;
                tab[xr] = std::polar(1.0, ang);
            }
            daux = add_coef(tab.data(), half);
        }
        P.ops.push_back(FOp{FO_G1F, r, uform | (pre << 4), ucoef, taux, laux, daux, oc0});
    }

    void emit_dense(const Item &it)
    {
        std::vector<int> ph(it.q, it.q + it.nq);
        std::map<int, Pre> pre = take_pending(ph);
        if (it.nq == 1) {
            int r = reg_of_tau(tau_of[it.q[0]]);
            const cd *m = it.m;
            bool real = true;
            for (int k = 0; k < 4; k++) real = real && std::abs(m[k].imag()) < 1e-15;
            int uform, uc;
            if (real && std::abs(m[0] - m[1]) < 1e-15 && std::abs(m[0] - m[2]) < 1e-15 &&
                std::abs(m[0] + m[3]) < 1e-15 && std::abs(m[0]) > kTiny) {
                // a * [[1, 1], [1, -1]]: unnormalised butterfly, a applied once per pass
                uform = U_HAD;
                uc = 0;
                pass_scale *= m[0].real();
            } else if (std::abs(m[0]) < kTiny && std::abs(m[3]) < kTiny) {
                cd v[2] = {m[1], m[2]};
                uform = U_ANTI;
                uc = add_coef(v, 2);
            } else if (real) {
                uform = U_REAL;
                uc = add_coef(m, 4, true);
            } else {
                uform = U_CPLX;
                uc = add_coef(m, 4);
            }
            Pre none;
            auto f = pre.find(r);
            emit_g1f(r, f != pre.end() ? f->second : none, uform, uc);
            return;
        }
        int r0 = reg_of_tau(tau_of[it.q[0]]), r1 = reg_of_tau(tau_of[it.q[1]]);
        for (auto &kv : pre) emit_g1f(kv.first, kv.second, U_NONE, 0);
        // monomial?
        int perm[4];
        cd phv[4];
        bool mono = true;
        for (int r = 0; r < 4 && mono; r++) {
            int cnt = 0;
            for (int col = 0; col < 4; col++)
                if (std::abs(it.m[r * 4 + col]) > kTiny) {
                    cnt++;
                    perm[r] = col;
                    phv[r] = it.m[r * 4 + col];
                }
            mono = (cnt == 1);
        }
        if (mono) {
            int packed = perm[0] | (perm[1] << 2) | (perm[2] << 4) | (perm[3] << 6);
            P.ops.push_back(FOp{FO_G2M, r0, r1, add_coef(phv, 4), packed, 0, 0, 0});
        } else {
            P.ops.push_back(FOp{FO_G2, r0, r1, add_coef(it.m, 16), 0, 0, 0, 0});
        }
    }

    // Builds one fused pass over tile `tile_phys` (c low + high bits) from the
    // in-order list of executed items.
    void build_pass(const std::vector<int> &high, const std::vector<const Item *> &exec)
    {
        P.passes.emplace_back();
        pass = &P.passes.back();
        pass->op_begin = (int)P.ops.size();
        pass->map_begin = (int)P.maps.size();
        pass->lin_begin = (int)P.lin_off.size();
        pass_scale = 1.0;
        pass->coef_begin = (int)P.coef.size();
        pass->tw_begin = (int)P.tw.size();
        pass->ext_begin = (int)P.ext_bit.size();
        P.lin_off.push_back((int32_t)P.ext_bit.size());
        lin_count = 0;
        tq.assign(t, 0);
        tau_of.assign(n, -1);
        for (int b = 0; b < c; b++) tq[b] = b;
        for (int j = 0; j < t - c; j++) tq[c + j] = high[j];
        for (int b = 0; b < t; b++) tau_of[tq[b]] = b;

        std::vector<std::vector<int>> opt;  // tau bits of each dense op
        for (const Item *it : exec)
            if (it->kind == 0) {
                std::vector<int> v;
                for (int k = 0; k < it->nq; k++) v.push_back(tau_of[it->q[k]]);
                opt.push_back(v);
            }
        // phase 0 (load): lanes = tau 0..4, registers exclude them
        choose_regs(opt, 0, true);
        assign_lanes(true);
        push_map();   // map 0: the load map
        size_t di = 0;
        int ndense = 0;
        for (const Item *it : exec) {
            if (it->kind == 1) {
                for (const Term &tm : it->terms) pending.push_back(tm);
                gphase *= it->gphase;
                continue;
            }
            bool in_regs = true;
            for (int k = 0; k < it->nq; k++) in_regs = in_regs && reg_of_tau(tau_of[it->q[k]]) >= 0;
            if (!in_regs) {
                choose_regs(opt, di, false);
                assign_lanes(false);
                emit(FO_XPOSE, 0, 0, 0, push_map(), 0);
            }
            emit_dense(*it);
            di++;
            ndense++;
        }
        if (pass_scale != 1.0) {
            cd sc(pass_scale, 0.0);
            P.ops.push_back(FOp{FO_RSCALE, 0, 0, add_coef(&sc, 1, true), 0, 0, 0, 0});
        }
        // store: lanes = tau 0..4 and no register on them
        bool store_ok = true;
        for (int r = 0; r < RB; r++) store_ok = store_ok && reg[r] >= 5;
        for (int l = 0; l < 5; l++) store_ok = store_ok && lane[l] == l;
        if (!store_ok) {
            std::vector<std::vector<int>> none;
            choose_regs(none, 0, true);
            assign_lanes(true);
            emit(FO_XPOSE, 0, 0, 0, push_map(), 0);
        }
        pass->op_end = (int)P.ops.size();
        pass->map_end = (int)P.maps.size();
        pass->nlin = lin_count;
        pass->ndense = ndense;
        FPassDev &d = pass->dev;
        memset(&d, 0, sizeof d);
        d.n = n;
        d.t = t;
        d.c = c;
        d.RB = RB;
        d.W = W;
        for (int j = 0; j < t - c; j++) d.hq[j] = high[j];
        std::vector<int> s(high.begin(), high.end());
        std::sort(s.begin(), s.end());
        d.ins.npos = (int)s.size();
        for (size_t j = 0; j < s.size(); j++) d.ins.pos[j] = s[j];
    }

    // Host image of a pass's constant block (ops with offsets rebased to
    // the block, coefficients in the ket's precision, phase turns, maps and
    // partner lists), staged into shared memory by every CTA.
    void finalize(PlanPass &ps)
    {
        FPassDev &d = ps.dev;
        d.nops = ps.op_end - ps.op_begin;
        d.ncoef = ps.coef_end - ps.coef_begin;
        d.ntw = ps.tw_end - ps.tw_begin;
        d.nmaps = ps.map_end - ps.map_begin;
        d.nlin = ps.nlin;
        d.next = ps.ext_end - ps.ext_begin;
        const size_t rs = dt == QSIM_C64 ? 4 : 8;
        auto al = [](size_t x) { return (x + 15) & ~(size_t)15; };
        size_t o = 0;
        d.off_tw = (int)o; o = al(o + 8 * (size_t)d.ntw);
        d.off_cf = (int)o; o = al(o + rs * (size_t)d.ncoef);
        d.off_ops = (int)o; o = al(o + sizeof(FOp) * (size_t)d.nops);
        d.off_maps = (int)o; o = al(o + sizeof(FMap) * (size_t)d.nmaps);
        d.off_lin = (int)o; o = al(o + 4 * (size_t)(d.nlin + 1));
        d.off_eb = (int)o; o = al(o + 4 * (size_t)d.next);
        d.off_et = (int)o; o = al(o + 8 * (size_t)d.next);
        d.stage_bytes = (int)o;
        ps.stage.assign(o, 0);
        unsigned char *b = ps.stage.data();
        memcpy(b + d.off_tw, P.tw.data() + ps.tw_begin, 8 * (size_t)d.ntw);
        for (int i = 0; i < d.ncoef; i++) {
            double v = P.coef[ps.coef_begin + i];
            if (rs == 4) { float f = (float)v; memcpy(b + d.off_cf + 4 * i, &f, 4); }
            else memcpy(b + d.off_cf + 8 * i, &v, 8);
        }
        for (int i = 0; i < d.nops; i++) {
            FOp op = P.ops[ps.op_begin + i];
            if (op.kind == FO_G1F) {
                int uf = op.j1 & 15;
                if (uf != U_NONE && uf != U_HAD) op.coef -= ps.coef_begin;
                if (op.aux >= 0) op.aux -= ps.coef_begin;
                if (op.aux3 >= 0) op.aux3 -= ps.coef_begin;
                op.aux4 -= ps.coef_begin;
            } else if (op.kind != FO_XPOSE) {
                op.coef -= ps.coef_begin;
            }
            memcpy(b + d.off_ops + sizeof(FOp) * i, &op, sizeof(FOp));
        }
        memcpy(b + d.off_maps, P.maps.data() + ps.map_begin, sizeof(FMap) * (size_t)d.nmaps);
        for (int i = 0; i <= d.nlin; i++) {
            int32_t v = P.lin_off[ps.lin_begin + i] - ps.ext_begin;
            memcpy(b + d.off_lin + 4 * i, &v, 4);
        }
        memcpy(b + d.off_eb, P.ext_bit.data() + ps.ext_begin, 4 * (size_t)d.next);
        memcpy(b + d.off_et, P.ext_tw.data() + ps.ext_begin, 8 * (size_t)d.next);
    }
};

// Classifies every gate (FP64 host matrices, physical qubits after SWAP
// relabels): dense one/two-qubit items, diagonal items as phase terms, and
// barriers (gates with two or more controls).
void classify_gates(const qsim_circuit *cir, const int *start_l2p, bool relabel, std::vector<Item> &items,
                    std::vector<int> &final_l2p, int64_t &nswaps)
{
    const int n = cir->n;
    std::vector<int> l2p(n);
    for (int q = 0; q < n; q++) l2p[q] = start_l2p ? start_l2p[q] : q;
    items.clear();
    items.reserve(cir->ngates);
    for (int k = 0; k < cir->ngates; k++) {
        const qsim_gate &g = cir->gates[k];
        cd m[16];
        int d = gate_matrix(g, cir->matrices, cir->nmatrix_doubles, m);
        Item it;
        if (g.kind == QSIM_G_SWAP && relabel) {
            std::swap(l2p[g.q0], l2p[g.q1]);
            nswaps++;
            continue;
        }
        if (d == 2 && g.ncontrols >= 2) {
            it.kind = 2;
            it.gate = g;
            it.gate.q0 = l2p[g.q0];
            for (int j = 0; j < g.ncontrols; j++) it.gate.controls[j] = l2p[g.controls[j]];
            it.bmat.assign(m, m + 4);
            items.push_back(it);
            continue;
        }
        if (d == 2 && g.ncontrols == 1) {
            // 4x4 on (target = bit 0, control = bit 1)
            cd M[16];
            for (int z = 0; z < 16; z++) M[z] = 0.0;
            int cv = (int)(g.control_values & 1);
            for (int bc = 0; bc < 2; bc++)
                for (int r = 0; r < 2; r++)
                    for (int col = 0; col < 2; col++)
                        M[(r + 2 * bc) * 4 + (col + 2 * bc)] = (bc == cv) ? m[r * 2 + col] : cd(r == col ? 1.0 : 0.0);
            memcpy(m, M, sizeof M);
            d = 4;
            it.q[0] = l2p[g.q0];
            it.q[1] = l2p[g.controls[0]];
        } else if (d == 2) {
            it.q[0] = l2p[g.q0];
        } else {
            it.q[0] = l2p[g.q0];
            it.q[1] = l2p[g.q1];
        }
        it.nq = d == 2 ? 1 : 2;
        if (is_diag(m, d)) {
            it.kind = 1;
            diag_terms(m, it.nq, it.q, it);
        } else {
            it.kind = 0;
            for (int z = 0; z < d * d; z++) it.m[z] = m[z];
        }
        items.push_back(it);
    }
    final_l2p = l2p;
}

}  // namespace

qsim_status plan_build(const qsim_circuit *cir, qsim_dtype dt, const qsim_run_opts *opts, const int *start_l2p,
                       qsim_plan *P)
{
    const int n = cir->n;
    qsim_run_opts o{};
    if (opts) o = *opts;
    int t = o.tile_qubits ? o.tile_qubits : (dt == QSIM_C64 ? 13 : 12);
    if (dt == QSIM_C128 && t > 13) return fail(QSIM_E_INVAL, "complex128 tiles hold at most 13 qubits");
    if (t > 14) return fail(QSIM_E_INVAL, "tiles hold at most 14 qubits");
    int c = 5;
    if (o.low_qubits && o.low_qubits != 5) return fail(QSIM_E_UNSUPPORTED, "low_qubits must be 5 (warp lanes)");
    if (t > n) t = n;
    // registers per thread: 2^5 amplitudes for complex64, 2^4 for complex128
    int RB = std::min(dt == QSIM_C64 ? 5 : 4, t - 5);
    if (RB < 4) return fail(QSIM_E_UNSUPPORTED, "fused path needs n >= 9");
    if (t - RB - 5 > kMaxW || t > kMaxTile) return fail(QSIM_E_INVAL, "tile_qubits %d too large", t);
    if (t - c > 12) return fail(QSIM_E_INVAL, "tile_qubits %d too large", t);
    P->n = n;
    P->dt = dt;
    P->t = t;
    P->c = c;
    P->RB = RB;
    P->ngates = cir->ngates;
    bool relabel = opts ? (o.relabel_swaps != 0 || o.mode == QSIM_MODE_FUSED) : true;

    // ---- classify gates into items (physical bits after relabels)
    std::vector<Item> items;
    {
        std::vector<int> l2p(n);
        for (int q = 0; q < n; q++) l2p[q] = start_l2p ? start_l2p[q] : q;
        P->start_l2p = l2p;
    }
    classify_gates(cir, start_l2p, relabel, items, P->final_l2p, P->nswaps);

    // complex64 plans with a dense (non-monomial) two-qubit gate use 16
    // amplitude registers per thread: the 4x4 product needs the headroom
    if (RB == 5) {
        for (const Item &it : items) {
            if (it.kind != 0 || it.nq != 2) continue;
            bool mono = true;
            for (int r = 0; r < 4 && mono; r++) {
                int cnt = 0;
                for (int col = 0; col < 4; col++) cnt += std::abs(it.m[r * 4 + col]) > kTiny;
                mono = (cnt == 1);
            }
            if (!mono) {
                RB = 4;
                break;
            }
        }
        P->RB = RB;
    }

    // ---- passes
    Builder B(*P, dt, n, t, c, RB);
    std::vector<const Item *> rem;
    for (auto &it : items) rem.push_back(&it);
    auto item_qubits = [](const Item *it, std::vector<int> &v) {
        v.clear();
        if (it->kind == 2) {
            v.push_back(it->gate.q0);
            for (int j = 0; j < it->gate.ncontrols; j++) v.push_back(it->gate.controls[j]);
        } else if (it->kind == 1) {
            for (const Term &tm : it->terms) {
                if (std::find(v.begin(), v.end(), tm.a) == v.end()) v.push_back(tm.a);
                if (tm.b >= 0 && std::find(v.begin(), v.end(), tm.b) == v.end()) v.push_back(tm.b);
            }
        } else {
            for (int k = 0; k < it->nq; k++) v.push_back(it->q[k]);
        }
    };
    auto flush_all_pergate = [&]() {
        for (const Term &tm : B.pending) {
            PlanStep st;
            st.kind = 1;
            memset(&st.gate, 0, sizeof st.gate);
            if (tm.b < 0) {
                st.gate.kind = QSIM_G_PHASE;
                st.gate.q0 = tm.a;
                st.mat = {1.0, 0.0, 0.0, std::polar(1.0, tm.th)};
            } else {
                st.gate.kind = QSIM_G_CP;
                st.gate.q0 = tm.a;
                st.gate.q1 = tm.b;
                st.gate.params[0] = tm.th;
            }
            P->steps.push_back(st);
            P->npergate++;
        }
        B.pending.clear();
    };
    // One pass's sweep over rm: the tile's high qubits grow in circuit order
    // (allow != 0: only from allow), diagonal items run wherever they are not
    // blocked. Returns the dense items taken.
    auto pass_sweep = [&](const std::vector<const Item *> &rm, uint64_t allow, std::vector<int> &tile,
                          std::vector<const Item *> &exec, std::vector<const Item *> &left) {
        tile.clear();
        exec.clear();
        left.clear();
        std::vector<char> in_tile(n, 0), blocked(n, 0);
        for (int b = 0; b < c; b++) in_tile[b] = 1;
        int nd = 0;
        std::vector<int> qv;
        for (const Item *it : rm) {
            item_qubits(it, qv);
            bool blk = false;
            for (int q : qv) blk = blk || blocked[q];
            if (!blk && it->kind == 1) {
                exec.push_back(it);
                continue;
            }
            if (!blk && it->kind == 0) {
                int need = 0;
                bool ok = true;
                for (int q : qv)
                    if (!in_tile[q]) {
                        need++;
                        if (allow && !(allow & bit(q))) ok = false;
                    }
                if (ok && (int)tile.size() + need <= t - c) {
                    for (int q : qv)
                        if (!in_tile[q]) {
                            in_tile[q] = 1;
                            tile.push_back(q);
                        }
                    exec.push_back(it);
                    nd++;
                    continue;
                }
            }
            for (int q : qv) blocked[q] = 1;
            left.push_back(it);
        }
        return nd;
    };
    // Candidate high-qubit sets for the next pass (as for tensor-core blocks:
    // sets grown from each of the first dense items, by overlap in circuit
    // order and by interaction-graph weight to the set and the low qubits);
    // the candidate whose sweep takes the most dense items wins.
    auto pass_choose = [&](const std::vector<const Item *> &rm) -> uint64_t {
        const int kMaxSeeds = 48, kWindow = 400, hq = t - c;
        std::vector<int> w((size_t)n * n, 0);
        int cnt = 0;
        for (size_t i = 0; i < rm.size() && cnt < kWindow; i++) {
            const Item *it = rm[i];
            if (it->kind != 0 || it->nq != 2) continue;
            w[(size_t)it->q[0] * n + it->q[1]]++;
            w[(size_t)it->q[1] * n + it->q[0]]++;
            cnt++;
        }
        const uint64_t low = bit(c) - 1;
        std::vector<uint64_t> cands;
        auto add = [&](uint64_t m) {
            if (m && std::find(cands.begin(), cands.end(), m) == cands.end()) cands.push_back(m);
        };
        int seeds = 0;
        for (size_t s0 = 0; s0 < rm.size() && seeds < kMaxSeeds; s0++) {
            const Item *sd = rm[s0];
            if (sd->kind != 0) continue;
            seeds++;
            uint64_t m0 = 0;
            for (int k = 0; k < sd->nq; k++) m0 |= bit(sd->q[k]);
            m0 &= ~low;
            // (1) overlap growth in circuit order
            uint64_t m = m0;
            for (size_t i = 0; i < rm.size() && __builtin_popcountll(m) < hq; i++) {
                const Item *it = rm[i];
                if (it->kind != 0) continue;
                uint64_t mi = 0;
                for (int k = 0; k < it->nq; k++) mi |= bit(it->q[k]);
                if (!(mi & (m | low))) continue;
                if (__builtin_popcountll(m | (mi & ~low)) <= hq) m |= mi & ~low;
            }
            add(m);
            // (2) interaction-graph growth
            m = m0;
            while (__builtin_popcountll(m) < hq) {
                int best = -1, bw = 0;
                for (int q = c; q < n; q++) {
                    if (m & bit(q)) continue;
                    int ww = 0;
                    for (int x = 0; x < n; x++)
                        if ((m | low) & bit(x)) ww += w[(size_t)q * n + x];
                    if (ww > bw) {
                        bw = ww;
                        best = q;
                    }
                }
                if (best < 0) break;
                m |= bit(best);
            }
            add(m);
        }
        std::vector<int> tl;
        std::vector<const Item *> ex, lf;
        int best = pass_sweep(rm, 0, tl, ex, lf);
        uint64_t pick = 0;
        for (uint64_t m : cands) {
            const int nd = pass_sweep(rm, m, tl, ex, lf);
            if (nd > best) {
                best = nd;
                pick = m;
            }
        }
        return pick;
    };
    // passes of a whole sweep (choose: per-pass choice), without building
    // them; masks receives the high-qubit set chosen at each step of the
    // sweep, which the build loop below repeats step for step
    auto count_passes = [&](bool choose, std::vector<uint64_t> *masks) {
        std::vector<const Item *> rm = rem, ex, lf;
        std::vector<int> tl;
        int np = 0;
        while (!rm.empty()) {
            const uint64_t m = choose ? pass_choose(rm) : 0;
            if (masks) masks->push_back(m);
            const int nd = pass_sweep(rm, m, tl, ex, lf);
            if (nd == 0) {
                if (lf.empty()) break;
                lf.erase(lf.begin());
                rm = lf;
                continue;
            }
            np++;
            rm = lf;
        }
        return np;
    };
    std::vector<uint64_t> chosen;
    const bool choose = count_passes(true, &chosen) < count_passes(false, nullptr);
    size_t step_i = 0;
    while (!rem.empty()) {
        std::vector<int> tile;  // high qubits
        std::vector<const Item *> exec, left;
        const uint64_t mask = choose && step_i < chosen.size() ? chosen[step_i] : 0;
        step_i++;
        const int ndense = pass_sweep(rem, mask, tile, exec, left);
        std::vector<char> in_tile(n, 0);
        for (int b = 0; b < c; b++) in_tile[b] = 1;
        for (int q : tile) in_tile[q] = 1;
        if (ndense == 0) {
            // only diagonal items and barriers remain runnable: fold the
            // diagonal ones, then run the first barrier per gate
            for (const Item *it : exec) {
                for (const Term &tm : it->terms) B.pending.push_back(tm);
                B.gphase *= it->gphase;
            }
            if (left.empty()) {
                rem.clear();
                break;
            }
            const Item *bar = left.front();
            flush_all_pergate();
            PlanStep st;
            st.kind = 1;
            st.gate = bar->gate;
            st.mat = bar->bmat;
            P->steps.push_back(st);
            P->npergate++;
            left.erase(left.begin());
            rem = left;
            continue;
        }
        // fill the tile with unused high qubits
        for (int q = n - 1; q >= c && (int)tile.size() < t - c; q--)
            if (!in_tile[q]) {
                in_tile[q] = 1;
                tile.push_back(q);
            }
        std::sort(tile.begin(), tile.end());
        B.build_pass(tile, exec);
        PlanStep st;
        st.kind = 0;
        st.pass = (int)P->passes.size() - 1;
        P->steps.push_back(st);
        P->ndense += ndense;
        rem = left;
    }
    // global phase: into the last fused pass, else a per-gate step
    if (std::abs(B.gphase - cd(1.0)) > 1e-15) {
        if (!P->passes.empty() && P->steps.back().kind == 0) {
            PlanPass &ps = P->passes.back();
            cd g = B.gphase;
            P->ops.push_back(FOp{FO_SCALE, 0, 0, B.add_coef(&g, 1), 0, 0, 0, 0});
            ps.op_end = (int)P->ops.size();
        } else {
            PlanStep st;
            st.kind = 2;
            st.phase = B.gphase;
            P->steps.push_back(st);
        }
    }
    flush_all_pergate();
    for (size_t i = 0; i < P->passes.size(); i++) {
        // coefficient / turn / partner ranges end where the next pass begins
        PlanPass &ps = P->passes[i];
        bool last = (i + 1 == P->passes.size());
        ps.coef_end = last ? (int)P->coef.size() : P->passes[i + 1].coef_begin;
        ps.tw_end = last ? (int)P->tw.size() : P->passes[i + 1].tw_begin;
        ps.ext_end = last ? (int)P->ext_bit.size() : P->passes[i + 1].ext_begin;
        B.finalize(ps);
        // the pass kernel stages tile, per-tile partner factors and the
        // constant block in shared memory: refuse at plan time a pass that
        // could not launch
        const size_t need = fused_pass_smem(ps.dev, dt);
        if (need > kFusedSmemCap)
            return fail(QSIM_E_UNSUPPORTED,
                        "fused pass %zu needs %zu bytes of shared memory (at most %zu); plan with fewer tile qubits",
                        i, need, kFusedSmemCap);
    }
    return QSIM_OK;
}

}  // namespace qs

namespace qs {

// Tensor-core plans: dense gates are fused into blocks of at most 6 qubits
// (7 with the 7-qubit kernel) by the commutation-aware sweep of the fused passes (a gate joins the
// current block when its qubits fit and no earlier gate left for later
// shares a qubit with it). Diagonal gates never block: as in the fused
// passes they become pending phase terms and are applied right before the
// next dense gate on one of their qubits. There a term whose qubits are both
// in the block is folded into the block's FP64 unitary; a term pairing a
// block qubit q with an outside qubit o becomes part of the block's
// pre-diagonal (applied per group at gather time, o read from the group's
// index) when no earlier gate of the block acted on q (so the term may move
// to the block's start), and o is then kept out of the block. SWAPs are
// relabels. Every block is one pass of the tensor-core kernel.
//
// Which qubits a block gets: the first-fit sweep lets the earliest gates
// decide, which on 2-D circuits often closes a block after gates of one
// layer. The sweep can also be restricted to a candidate qubit set; the
// candidates are the sets grown from each of the first dense gates (the
// gate's qubits plus those of the following gates that overlap and fit).
// Per block the candidate taking the most dense gates wins (sweeps without
// matrices decide). The plan is built with per-block choice when a full
// matrix-free sweep shows it needs fewer blocks than first fit, else with
// first fit, so no circuit gets more blocks than before.
namespace {

struct TcSweep {
    int n;
    int kb = 6;                                                // block size limit (6, or 7 for the 7-qubit kernel)
    std::vector<Term> pending;
    cd gphase = 1.0;
    // one block's outcome
    std::vector<int> Q;                                        // block qubits, block bit b <-> Q[b]
    std::vector<cd> U;
    std::vector<char> outside;
    std::vector<std::pair<int, std::pair<int, double>>> pre;   // (block qubit, (outside qubit, angle))
    std::vector<const Item *> left;
    int ng = 0;
};

void item_qubits(const Item *it, std::vector<int> &v)
{
    v.clear();
    if (it->kind == 2) {
        v.push_back(it->gate.q0);
        for (int j = 0; j < it->gate.ncontrols; j++) v.push_back(it->gate.controls[j]);
    } else if (it->kind == 1) {
        for (const Term &tm : it->terms) {
            if (std::find(v.begin(), v.end(), tm.a) == v.end()) v.push_back(tm.a);
            if (tm.b >= 0 && std::find(v.begin(), v.end(), tm.b) == v.end()) v.push_back(tm.b);
        }
    } else {
        for (int k = 0; k < it->nq; k++) v.push_back(it->q[k]);
    }
}

// One block of the sweep over rem (state in S: pending terms, global phase;
// results in S.Q / U / pre / outside / left / ng). allow != 0 restricts the
// block to those qubits; dry skips the matrices.
void tc_sweep_block(TcSweep &S, const std::vector<const Item *> &rem, uint64_t allow, bool dry)
{
    const int n = S.n;
    S.Q.clear();
    S.U.assign(1, 1.0);
    S.outside.assign(n, 0);
    S.pre.clear();
    S.left.clear();
    S.ng = 0;
    std::vector<char> blocked(n, 0), touched(n, 0);
    std::vector<int> qv;
    std::vector<int> &Q = S.Q;
    std::vector<cd> &U = S.U;
    for (const Item *it : rem) {
        item_qubits(it, qv);
        bool blk = false;
        for (int q : qv) blk = blk || blocked[q];
        if (!blk && it->kind == 1) {
            for (const Term &tm : it->terms) S.pending.push_back(tm);
            S.gphase *= it->gphase;
            continue;
        }
        bool fits = !blk && it->kind == 0;
        std::vector<int> nq = Q;
        if (fits) {
            for (int q : qv) {
                if (S.outside[q]) fits = false;
                if (allow && !(allow & bit(q))) fits = false;
                if (std::find(nq.begin(), nq.end(), q) == nq.end()) nq.push_back(q);
            }
            if ((int)nq.size() > S.kb) fits = false;
        }
        // pending terms this gate must see first
        std::vector<Term> keep, fold, hoist;
        if (fits) {
            auto in_op = [&](int q) { return std::find(qv.begin(), qv.end(), q) != qv.end(); };
            auto in_blk = [&](int q) { return std::find(nq.begin(), nq.end(), q) != nq.end(); };
            for (const Term &tm : S.pending) {
                bool t = in_op(tm.a) || (tm.b >= 0 && in_op(tm.b));
                if (!t) {
                    keep.push_back(tm);
                    continue;
                }
                if (tm.b < 0 || (in_blk(tm.a) && in_blk(tm.b))) {
                    fold.push_back(tm);
                    continue;
                }
                int q = in_blk(tm.a) ? tm.a : tm.b;
                if (touched[q]) {
                    fits = false;
                    break;
                }
                hoist.push_back(tm);
            }
        }
        if (!fits) {
            for (int q : qv) blocked[q] = 1;
            S.left.push_back(it);
            continue;
        }
        S.pending.swap(keep);
        // extend U to nq (new qubits become higher block bits)
        int od = 1 << Q.size(), nd = 1 << nq.size();
        if (nd != od) {
            if (!dry) {
                std::vector<cd> V((size_t)nd * nd, 0.0);
                for (int r = 0; r < nd; r++)
                    for (int c = 0; c < nd; c++)
                        if ((r / od) == (c / od)) V[(size_t)r * nd + c] = U[(size_t)(r % od) * od + (c % od)];
                U.swap(V);
            }
            Q = nq;
        }
        auto bpos = [&](int q) { return (int)(std::find(Q.begin(), Q.end(), q) - Q.begin()); };
        // folded terms: a diagonal on the block, applied now
        if (!fold.empty() && !dry) {
            for (int r = 0; r < nd; r++) {
                double ang = 0;
                for (const Term &tm : fold) {
                    bool ba = (r >> bpos(tm.a)) & 1;
                    bool bb = tm.b < 0 ? true : (bool)((r >> bpos(tm.b)) & 1);
                    if (ba && bb) ang += tm.th;
                }
                cd f = std::polar(1.0, ang);
                for (int c = 0; c < nd; c++) U[(size_t)r * nd + c] *= f;
            }
        }
        for (const Term &tm : hoist) {
            int q = std::find(Q.begin(), Q.end(), tm.a) != Q.end() ? tm.a : tm.b;
            int o = q == tm.a ? tm.b : tm.a;
            S.pre.push_back({q, {o, tm.th}});
            S.outside[o] = 1;
        }
        // the gate
        if (!dry) {
            int gd = 1 << it->nq, gmask = 0;
            int pos[2];
            for (int k = 0; k < it->nq; k++) {
                pos[k] = bpos(it->q[k]);
                gmask |= 1 << pos[k];
            }
            auto loc = [&](int r) {
                int l = 0;
                for (int k = 0; k < it->nq; k++) l |= ((r >> pos[k]) & 1) << k;
                return l;
            };
            std::vector<cd> W((size_t)nd * nd, 0.0);
            for (int r = 0; r < nd; r++)
                for (int x = 0; x < nd; x++) {
                    if ((r & ~gmask) != (x & ~gmask)) continue;
                    cd a = it->m[loc(r) * gd + loc(x)];
                    if (a == cd(0.0)) continue;
                    for (int c = 0; c < nd; c++) W[(size_t)r * nd + c] += a * U[(size_t)x * nd + c];
                }
            U.swap(W);
        }
        for (int k = 0; k < it->nq; k++) touched[it->q[k]] = 1;
        S.ng++;
    }
}

// Candidate qubit sets for the next block, from each of the first
// kMaxSeeds dense items: (1) the item's qubits plus those of the following
// items that overlap and fit; (2) for a two-qubit item, its qubits grown one
// qubit at a time by the qubit with the most dense two-qubit gates to the
// set among the next kWindow ones (compact clusters of the interaction
// graph, e.g. patches of a 2-D grid).
std::vector<uint64_t> tc_candidates(const std::vector<const Item *> &rem, int n, int kb)
{
    const int kMaxSeeds = 48, kWindow = 400;
    std::vector<uint64_t> out;
    std::vector<int> w((size_t)n * n, 0);
    {
        int cnt = 0;
        for (size_t i = 0; i < rem.size() && cnt < kWindow; i++) {
            const Item *it = rem[i];
            if (it->kind != 0 || it->nq != 2) continue;
            w[(size_t)it->q[0] * n + it->q[1]]++;
            w[(size_t)it->q[1] * n + it->q[0]]++;
            cnt++;
        }
    }
    int gseeds = 0;
    for (size_t s = 0; s < rem.size() && gseeds < kMaxSeeds; s++) {
        if (rem[s]->kind != 0 || rem[s]->nq != 2) continue;
        gseeds++;
        uint64_t m = bit(rem[s]->q[0]) | bit(rem[s]->q[1]);
        for (int size = 2; size < kb; size++) {
            int best = -1, bw = 0;
            for (int q = 0; q < n; q++) {
                if (m & bit(q)) continue;
                int ww = 0;
                for (int x = 0; x < n; x++)
                    if (m & bit(x)) ww += w[(size_t)q * n + x];
                if (ww > bw) {
                    bw = ww;
                    best = q;
                }
            }
            if (best < 0) break;
            m |= bit(best);
        }
        if (std::find(out.begin(), out.end(), m) == out.end()) out.push_back(m);
    }
    int seeds = 0;
    for (size_t s = 0; s < rem.size() && seeds < kMaxSeeds; s++) {
        if (rem[s]->kind != 0) continue;
        seeds++;
        uint64_t m = 0;
        int cnt = 0;
        for (int k = 0; k < rem[s]->nq; k++)
            if (!(m & bit(rem[s]->q[k]))) {
                m |= bit(rem[s]->q[k]);
                cnt++;
            }
        for (size_t i = 0; i < rem.size() && cnt < kb; i++) {
            const Item *it = rem[i];
            if (it->kind != 0) continue;
            uint64_t mi = 0;
            int ci = 0;
            for (int k = 0; k < it->nq; k++)
                if (!(mi & bit(it->q[k]))) {
                    mi |= bit(it->q[k]);
                    ci++;
                }
            if (!(mi & m)) continue;
            int add = 0;
            for (int k = 0; k < it->nq; k++) add += !(m & bit(it->q[k])) && (mi & bit(it->q[k]));
            if (cnt + add > kb) continue;
            m |= mi;
            cnt += add;
        }
        if (std::find(out.begin(), out.end(), m) == out.end()) out.push_back(m);
    }
    return out;
}

// The restriction for the next block: 0 (first fit) unless a candidate set
// takes more dense items in a matrix-free sweep.
uint64_t tc_choose(const TcSweep &S0, const std::vector<const Item *> &rem)
{
    TcSweep T = S0;
    tc_sweep_block(T, rem, 0, true);
    int best = T.ng;
    uint64_t pick = 0;
    for (uint64_t m : tc_candidates(rem, S0.n, S0.kb)) {
        TcSweep C = S0;
        tc_sweep_block(C, rem, m, true);
        if (C.ng > best) {
            best = C.ng;
            pick = m;
        }
    }
    return pick;
}

// Blocks of a matrix-free sweep of the whole circuit (choose: per-block choice).
int tc_count_blocks(int n, int kb, const std::vector<Item> &items, bool choose)
{
    TcSweep S;
    S.n = n;
    S.kb = kb;
    std::vector<const Item *> rem;
    for (auto &it : items) rem.push_back(&it);
    int blocks = 0;
    while (!rem.empty()) {
        const uint64_t allow = choose ? tc_choose(S, rem) : 0;
        tc_sweep_block(S, rem, allow, true);
        if (S.ng == 0) {
            if (S.left.empty()) break;
            S.pending.clear();   // flushed per gate before the barrier
            S.left.erase(S.left.begin());
            rem = S.left;
            continue;
        }
        blocks++;
        rem = S.left;
    }
    return blocks;
}

}  // namespace

qsim_status plan_build_tc(const qsim_circuit *cir, const qsim_run_opts *opts, const int *start_l2p, qsim_plan *P)
{
    const int n = cir->n;
    if (n < 6) return fail(QSIM_E_UNSUPPORTED, "tensor-core plans need n >= 6");
    P->n = n;
    P->dt = QSIM_C64;
    P->prec = opts->prec;
    P->ngates = cir->ngates;
    {
        std::vector<int> l2p(n);
        for (int q = 0; q < n; q++) l2p[q] = start_l2p ? start_l2p[q] : q;
        P->start_l2p = l2p;
    }
    // block size: 6 (blocks of fewer qubits are padded to 6), or 7 when
    // max_block asks for it (the 7-qubit kernel: complex64, BF16X3, n >= 14)
    const int kb = opts->max_block == 7 ? 7 : 6;
    if (kb == 7 && (opts->prec != QSIM_PREC_BF16X3 || n < 14))
        return fail(QSIM_E_UNSUPPORTED, "7-qubit tensor-core blocks take BF16X3 and n >= 14");
    std::vector<Item> items;
    classify_gates(cir, start_l2p, true, items, P->final_l2p, P->nswaps);
    const bool choose = tc_count_blocks(n, kb, items, true) < tc_count_blocks(n, kb, items, false);
    TcSweep S;
    S.n = n;
    S.kb = kb;
    auto flush_pergate = [&]() {
        for (const Term &tm : S.pending) {
            PlanStep st;
            st.kind = 1;
            memset(&st.gate, 0, sizeof st.gate);
            if (tm.b < 0) {
                st.gate.kind = QSIM_G_PHASE;
                st.gate.q0 = tm.a;
                st.mat = {1.0, 0.0, 0.0, std::polar(1.0, tm.th)};
            } else {
                st.gate.kind = QSIM_G_CP;
                st.gate.q0 = tm.a;
                st.gate.q1 = tm.b;
                st.gate.params[0] = tm.th;
            }
            P->steps.push_back(st);
            P->npergate++;
        }
        S.pending.clear();
    };
    std::vector<const Item *> rem;
    for (auto &it : items) rem.push_back(&it);
    while (!rem.empty()) {
        const uint64_t allow = choose ? tc_choose(S, rem) : 0;
        tc_sweep_block(S, rem, allow, false);
        std::vector<int> &Q = S.Q;
        std::vector<cd> &U = S.U;
        auto &pre = S.pre;
        auto &outside = S.outside;
        std::vector<const Item *> left = S.left;
        const int ng = S.ng;
        if (ng == 0) {
            if (left.empty()) {
                rem.clear();
                break;
            }
            // a barrier heads the remaining gates: flush, then run it per gate
            const Item *bar = left.front();
            flush_pergate();
            PlanStep st;
            st.kind = 1;
            st.gate = bar->gate;
            st.mat = bar->bmat;
            P->steps.push_back(st);
            P->npergate++;
            left.erase(left.begin());
            rem = left;
            continue;
        }
        // the global phase gathered so far rides on this block
        if (std::abs(S.gphase - cd(1.0)) > 1e-15) {
            for (auto &x : U) x *= S.gphase;
            S.gphase = 1.0;
        }
        // pad the block to kb qubits here (the kernel reads a pre-diagonal
        // partner's bit from the group index, where padded bits are 0):
        // highest free qubits that are no partner first, then partners,
        // whose terms then act inside the block as a diagonal before U
        {
            std::vector<int> pad;
            for (int pass = 0; pass < 2; pass++)
                for (int p = n - 1; p >= 0 && (int)(Q.size() + pad.size()) < kb; p--)
                    if (std::find(Q.begin(), Q.end(), p) == Q.end() &&
                        std::find(pad.begin(), pad.end(), p) == pad.end() && (bool)outside[p] == (pass == 1))
                        pad.push_back(p);
            int od = 1 << Q.size();
            Q.insert(Q.end(), pad.begin(), pad.end());
            int nd = 1 << Q.size();
            if (nd != od) {
                std::vector<cd> V((size_t)nd * nd, 0.0);
                for (int r = 0; r < nd; r++)
                    for (int c = 0; c < nd; c++)
                        if ((r / od) == (c / od)) V[(size_t)r * nd + c] = U[(size_t)(r % od) * od + (c % od)];
                U.swap(V);
            }
            auto bpos = [&](int q) { return (int)(std::find(Q.begin(), Q.end(), q) - Q.begin()); };
            std::vector<std::pair<int, std::pair<int, double>>> rest;
            for (auto &x : pre) {
                int o = x.second.first;
                if (std::find(pad.begin(), pad.end(), o) == pad.end()) {
                    rest.push_back(x);
                    continue;
                }
                int ba = bpos(x.first), bb = bpos(o);
                cd f = std::polar(1.0, x.second.second);
                for (int c = 0; c < nd; c++)
                    if (((c >> ba) & 1) && ((c >> bb) & 1))
                        for (int r = 0; r < nd; r++) U[(size_t)r * nd + c] *= f;
            }
            pre.swap(rest);
        }
        TcSpec ts;
        std::vector<unsigned char> A;
        QS_TRY(tc_build(n, (int)Q.size(), Q.data(), U.data(), (qsim_prec)opts->prec, A, ts, kb));
        // pre-diagonal partner lists per block bit, in tc_build's bit order
        std::vector<int32_t> off(kb + 1, 0), pb;
        std::vector<uint64_t> ptw;
        for (int b = 0; b < kb; b++) {
            off[b] = (int32_t)pb.size();
            if (b < (int)Q.size())
                for (auto &x : pre)
                    if (x.first == ts.q[b]) {
                        pb.push_back(x.second.first);
                        ptw.push_back(to_turns(x.second.second));
                    }
        }
        off[kb] = (int32_t)pb.size();
        P->tc_spec.push_back(ts);
        P->tc_A.push_back(std::move(A));
        P->tc_pd_off.push_back(pre.empty() ? std::vector<int32_t>() : off);
        P->tc_pd_bit.push_back(pb);
        P->tc_pd_tw.push_back(ptw);
        PlanStep st;
        st.kind = 3;
        st.pass = (int)P->tc_spec.size() - 1;
        P->steps.push_back(st);
        P->ndense += ng;
        rem = left;
    }
    if (std::abs(S.gphase - cd(1.0)) > 1e-15) {
        PlanStep st;
        st.kind = 2;
        st.phase = S.gphase;
        P->steps.push_back(st);
    }
    flush_pergate();
    return QSIM_OK;
}

}  // namespace qs
