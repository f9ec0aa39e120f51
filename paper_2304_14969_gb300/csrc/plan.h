// Fused execution plans: the host planner's output and the device-side
// descriptors of one fused pass.
//
// A pass streams the ket through the SMs once: each CTA owns a tile of 2^t
// amplitudes whose index bits are the c lowest physical qubits (contiguous
// runs in HBM) plus t - c chosen high qubits. The tile is spread over the
// CTA as 2^RB registers per thread x 32 lanes x 2^W warps; a "phase" assigns
// tile bits to register, lane and warp bits, and gates act on register bits
// only. Changing phase is one transpose through shared memory.
#pragma once

#include <vector>

#include "qsim_internal.h"

namespace qs {

enum FOpKind : int32_t {
    // FO_G1F: dense 2x2 on register bit j0, preceded by the phase prefactor
    // of the amplitudes with bit j0 set (deferred diagonal terms). j1 = matrix
    // form (0 none / pure phase, 1 real 2x2, 2 complex 2x2, 3 anti-diagonal).
    // The prefactor of register element x is
    //   cf[aux4] * (aux >= 0 ? cf[aux + 2 tid] : 1) * (aux2 >= 0 ? Ec[aux2] : 1) * cf[aux3 + 2 xr]
    // with xr = x without bit j0 (aux3 table of 2^(RB-1) complex entries for
    // partners among the other register bits) and Ec[l] a per-tile factor
    // from partners outside the tile.
    FO_G1F = 1,
    FO_G2 = 4,     // dense 4x4 on (j0 = bit 0, j1 = bit 1); cf[coef .. +32)
    FO_G2M = 5,    // monomial 4x4: out[r] = ph[r] * in[perm[r]]; aux = perm packed 2 bits each; cf: 8
    FO_XPOSE = 8,  // transpose through shared memory to map aux
    FO_SCALE = 9,  // every register amplitude *= cf[coef .. +2)
    FO_RSCALE = 10 // every register amplitude *= the real cf[coef]
};

// j1 of FO_G1F = uform | (pre << 4).
// uform: U_NONE pure phase, U_REAL 4 reals, U_CPLX 4 complex, U_ANTI
// anti-diagonal (2 complex), U_HAD unnormalised Hadamard butterfly
// (p + q, p - q); the pass's product of the dropped scales is applied once by
// a FO_RSCALE op. pre: PRE_NONE no prefactor, PRE_D prefactor D[xr] (a
// constant table), PRE_FD prefactor f * D[xr] (per-thread f).
enum { U_NONE = 0, U_REAL = 1, U_CPLX = 2, U_ANTI = 3, U_HAD = 4 };
enum { PRE_NONE = 0, PRE_D = 1, PRE_FD = 2 };

struct FOp {
    int32_t kind, j0, j1, coef, aux, aux2, aux3, aux4;
};

static const int kMaxRB = 5;
static const int kMaxW = 6;
static const int kMaxTile = 16;

// Phase map: tile bit of each register, lane and warp bit, plus the tile
// index and physical offset of each register element x (bit r of x is
// register bit r).
struct FMap {
    int8_t reg[kMaxRB];
    int8_t lane[5];
    int8_t warp[kMaxW];
    int8_t pad[16 - kMaxRB - 5 - kMaxW + 16];
    uint32_t treg[1 << kMaxRB];
    uint32_t tsw[1 << kMaxRB];   // swizzled shared-memory slot of treg[x] (linear over XOR)
    uint64_t preg[1 << kMaxRB];
};

struct FPassDev {
    int n, t, c, RB, W;
    // pass-local constant block staged into shared memory by every CTA:
    // counts and the byte offset of each array inside the block
    int nops, ncoef, ntw, nmaps, nlin, next;
    int off_tw, off_cf, off_ops, off_maps, off_lin, off_eb, off_et, stage_bytes;
    const unsigned char *stage;  // the block in global memory
    int hq[kMaxTile];        // physical bit of tile bit c + j
    InsSpec ins;             // sorted hq for tile-id expansion
};

// Dynamic shared memory of one fused-pass CTA: the tile, the per-tile
// factors of partners outside the tile, the pass's constant block; a pass
// needing more than kFusedSmemCap is refused when the plan is built.
constexpr size_t kFusedSmemCap = 220 * 1024;
inline size_t fused_pass_smem(const FPassDev &d, qsim_dtype dt)
{
    const size_t amp = dt == QSIM_C64 ? 8 : 16;
    return (amp << d.t) + (((size_t)d.nlin * 16 + 15) & ~(size_t)15) + (size_t)d.stage_bytes;
}

// Host-side plan
struct PlanPass {
    FPassDev dev;            // stage pointer filled at upload
    int op_begin, op_end;    // into ops
    int map_begin, map_end;  // into maps
    int lin_begin, nlin;     // into lin_off (nlin + 1 entries, rebased to ext_begin)
    int coef_begin, coef_end, tw_begin, tw_end, ext_begin, ext_end;
    int ndense;
    std::vector<unsigned char> stage;  // host image of the staged block
};

struct PlanStep {
    int kind;                // 0 fused pass, 1 per-gate gate (physical qubits), 2 global phase,
                             // 3 tensor-core block (pass = index into tc_spec)
    int pass;                // kind 0
    qsim_gate gate;          // kind 1 (physical qubits, matrix in mats)
    std::vector<cd> mat;     // kind 1: 2x2 or 4x4
    cd phase;                // kind 2
};

struct CircuitPlanner;

}  // namespace qs

struct qsim_plan {
    int n = 0;
    qsim_dtype dt = QSIM_C64;
    int t = 0, c = 0, RB = 0;
    std::vector<qs::PlanStep> steps;
    std::vector<qs::PlanPass> passes;
    std::vector<int> start_l2p, final_l2p;
    // host arrays
    std::vector<qs::FOp> ops;
    std::vector<double> coef;
    std::vector<uint64_t> tw;
    std::vector<qs::FMap> maps;
    std::vector<int32_t> lin_off, ext_bit;
    std::vector<uint64_t> ext_tw;
    // tensor-core blocks
    int prec = QSIM_PREC_NATIVE;
    std::vector<qs::TcSpec> tc_spec;
    std::vector<std::vector<unsigned char>> tc_A;
    std::vector<std::vector<int32_t>> tc_pd_off, tc_pd_bit;   // pre-diagonal partner lists per block
    std::vector<std::vector<uint64_t>> tc_pd_tw;
    std::vector<size_t> tc_off;
    std::vector<qs::TcPipeHost> tc_pipe;                       // pipelined kernel geometry (BF16x3, n >= 13)
    // device copies
    void *dmem = nullptr;
    size_t dbytes = 0;
    int64_t ngates = 0, ndense = 0, nswaps = 0, npergate = 0;
};
