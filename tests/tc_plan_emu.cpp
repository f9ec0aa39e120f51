// Host-side check of the tensor-core block planner (test infrastructure).
//
// Links the library's host planner with a stand-in for tc_build that keeps
// each block's qubits and complex matrix instead of packing split operands
// for the MMA, then applies the plan's steps to a ket on the CPU with the
// semantics the block kernel has: per-group pre-diagonal phases read from
// the group base index (where the block's own bits, padding included, are
// 0), then the 2^k x 2^k matrix on the block qubits. Per-gate steps and the
// global phase are applied as plain matrix-vector updates.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "plan.h"

namespace qs {
qsim_status plan_build_tc(const qsim_circuit *, const qsim_run_opts *, const int *, qsim_plan *);

struct EmuBlock {
    int k, kb;
    int q[7];
    std::vector<cd> U;
};
static std::vector<EmuBlock> g_blocks;

qsim_status tc_build(int n, int k, const int *phys, const cd *u, qsim_prec, std::vector<unsigned char> &, TcSpec &ts,
                     int kb)
{
    EmuBlock b;
    b.k = k;
    b.kb = kb;
    uint64_t used = 0;
    for (int j = 0; j < k; j++) {
        b.q[j] = phys[j];
        used |= 1ull << phys[j];
    }
    int kk = k;
    for (int p = n - 1; p >= 0 && kk < kb; p--)
        if (!((used >> p) & 1)) {
            b.q[kk++] = p;
            used |= 1ull << p;
        }
    b.U.assign(u, u + (size_t)(1 << k) * (1 << k));
    for (int j = 0; j < kb; j++) ts.q[j] = b.q[j];
    ts.kb = kb;
    g_blocks.push_back(b);
    return QSIM_OK;
}
}  // namespace qs

using namespace qs;

// psi_io: 2^n interleaved complex doubles in logical order (in and out).
// start_l2p: logical -> physical map the plan starts from (NULL = identity).
// max_block: the plan option (7: 7-qubit blocks). info[0..2]: blocks,
// per-gate steps, qubits tc_build padded (0 when the planner pads every
// block itself).
extern "C" int emu_tc_run(const qsim_circuit *c, int prec, const int *start_l2p, int max_block, double *psi_io,
                          int64_t info[3])
{
    g_blocks.clear();
    qsim_run_opts o;
    memset(&o, 0, sizeof o);
    o.mode = QSIM_MODE_FUSED;
    o.prec = prec;
    o.max_block = max_block;
    o.relabel_swaps = 1;
    qsim_plan P;
    qsim_status st = plan_build_tc(c, &o, start_l2p, &P);
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
    int64_t npergate = 0, padded = 0;
    for (const PlanStep &s : P.steps) {
        if (s.kind == 3) {
            const EmuBlock &B = g_blocks[s.pass];
            const int kb = B.kb, KB = 1 << kb;
            padded += kb - B.k;
            uint64_t m6 = 0;
            for (int x = 0; x < kb; x++) m6 |= 1ull << B.q[x];
            const std::vector<int32_t> &off = P.tc_pd_off[s.pass];
            const std::vector<int32_t> &pb = P.tc_pd_bit[s.pass];
            const std::vector<uint64_t> &tw = P.tc_pd_tw[s.pass];
            const int D = 1 << B.k;
            std::vector<cd> v(D), w(D);
            for (uint64_t base = 0; base < N; base++) {
                if (base & m6) continue;
                for (int hi = 0; hi < KB / D; hi++) {
                    for (int l = 0; l < D; l++) {
                        int row = l | (hi * D);
                        uint64_t idx = base;
                        for (int x = 0; x < kb; x++)
                            if ((row >> x) & 1) idx |= 1ull << B.q[x];
                        cd f = a[idx];
                        if (!off.empty())
                            for (int bb = 0; bb < kb; bb++)
                                if ((row >> bb) & 1)
                                    for (int z = off[bb]; z < off[bb + 1]; z++)
                                        if ((base >> pb[z]) & 1)
                                            f *= std::polar(1.0, (double)tw[z] * (2.0 * M_PI / 18446744073709551616.0));
                        v[l] = f;
                    }
                    for (int r = 0; r < D; r++) {
                        w[r] = 0.0;
                        for (int cc = 0; cc < D; cc++) w[r] += B.U[(size_t)r * D + cc] * v[cc];
                    }
                    for (int l = 0; l < D; l++) {
                        int row = l | (hi * D);
                        uint64_t idx = base;
                        for (int x = 0; x < kb; x++)
                            if ((row >> x) & 1) idx |= 1ull << B.q[x];
                        a[idx] = w[l];
                    }
                }
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
    info[0] = (int64_t)g_blocks.size();
    info[1] = npergate;
    info[2] = padded;
    return 0;
}

// Tile geometry of the pipelined tensor-core kernel for block qubits qk (6,
// or 7 for kind 3):
// dims[0..4] lowest qubit, dims[5..9] coordinate bits, dims[10..14] box
// extents, dims[15..19] global extents, dims[20..23] byte strides of
// dimensions 1..4, dims[24] boxes per tile, dims[25..28] dimension-4
// offsets of the boxes, dims[29] box bytes, dims[30] rotated low block bits,
// dims[31] log2 of the write-back's store runs, dims[32] rotation shift, dims[33] wide,
// dims[34..35] quarter-tile qubits, dims[36] kernel variant, dims[37] the
// third load-select qubit (kind 3), dims[38] block bits; tpos[13 or 14]
// tile qubits; posL / spL 2^kb entries. qk ascending (as tc_build orders a
// block). kind: 0 complex64 whole tiles, 1 complex128 quarter tiles, 2
// complex64 quarter tiles (TF32), 3 complex64 7-qubit blocks (eighth tiles).
extern "C" int emu_tc_geometry(int n, const int *q6, int kind, int64_t *dims, int *tpos, int *posL, int *posG,
                               uint64_t *spL, uint64_t *spG)
{
    const int kb = kind == 3 ? 7 : 6;
    TcSpec ts;
    memset(&ts, 0, sizeof ts);
    for (int b = 0; b < kb; b++) ts.q[b] = q6[b];
    ts.kb = kb;
    TcPipeHost H;
    qsim_status st = tc_pipe_prepare(n, ts, nullptr, H, kind);
    if (st != QSIM_OK) return (int)st;
    const TcPipeArgs &A = H.args;
    for (int d = 0; d < 5; d++) {
        dims[d] = A.dim_lo[d];
        dims[5 + d] = A.dim_bits[d];
        dims[10 + d] = H.box[d];
        dims[15 + d] = (int64_t)H.gdim[d];
        if (d < 4) dims[20 + d] = (int64_t)H.gstr[d];
    }
    dims[24] = A.nload;
    for (int v = 0; v < 4; v++) dims[25 + v] = A.xoff[v];
    dims[29] = A.box_bytes;
    dims[30] = A.rot_bits;
    dims[31] = A.vecw;
    dims[32] = A.rot_shift;
    dims[33] = A.wide;
    dims[34] = A.qpos[0];
    dims[35] = A.qpos[1];
    dims[36] = A.kind;
    dims[37] = A.qpos[2];
    dims[38] = A.kb;
    for (int j = 0; j < kb + 7; j++) tpos[j] = A.tpos[j];
    for (int l = 0; l < (1 << kb); l++) {
        posL[l] = A.posL[l];
        spL[l] = A.spL[l];
    }
    for (int g = 0; g < 128; g++) {
        posG[g] = A.posG[g];
        spG[g] = A.spG[g];
    }
    return 0;
}

// Deferred-phase tables of the pipelined kernel for kb (6 or 7) block
// qubits q6 and partner lists (off[kb + 1], pbit, tw): out = tturn[kb][24]
// (uint64) followed by gfac[128][kb] (float2).
extern "C" int emu_tc_tables(int n, int kb, const int *q6, const int32_t *off, const int32_t *pbit,
                             const uint64_t *tw, unsigned char *out)
{
    TcSpec ts;
    memset(&ts, 0, sizeof ts);
    for (int b = 0; b < kb; b++) ts.q[b] = q6[b];
    ts.kb = kb;
    std::vector<int32_t> o(off, off + kb + 1), pb(pbit, pbit + off[kb]);
    std::vector<uint64_t> t(tw, tw + off[kb]);
    std::vector<unsigned char> blob;
    tc_pipe_tables(n, ts, o, pb, t, blob);
    memcpy(out, blob.data(), blob.size());
    return (int)blob.size();
}

// Builds the tensor-core plan of c (from start_l2p, NULL = identity) and
// writes each block's six physical qubits (as tc_build received them) to
// q_out[6 * b ..] and its number of deferred-phase partners to npd[b];
// returns the number of blocks (at most cap), or -status.
extern "C" int emu_tc_plan_blocks(const qsim_circuit *c, const int *start_l2p, int cap, int *q_out, int *npd)
{
    g_blocks.clear();
    qsim_run_opts o;
    memset(&o, 0, sizeof o);
    o.mode = QSIM_MODE_FUSED;
    o.prec = QSIM_PREC_BF16X3;
    o.relabel_swaps = 1;
    qsim_plan P;
    qsim_status st = plan_build_tc(c, &o, start_l2p, &P);
    if (st != QSIM_OK) return -(int)st;
    int nb = 0;
    for (const PlanStep &s : P.steps) {
        if (s.kind != 3 || nb >= cap) continue;
        const EmuBlock &B = g_blocks[s.pass];
        for (int x = 0; x < 6; x++) q_out[6 * nb + x] = B.q[x];
        npd[nb] = P.tc_pd_bit[s.pass].size();
        nb++;
    }
    return nb;
}
