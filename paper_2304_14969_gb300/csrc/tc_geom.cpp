// Host-side geometry of the pipelined tensor-core block kernel
// (k_tc_pipe.cu): which qubits form a tile, how a 5-D TMA tensor map
// covers it, and the index tables the kernel uses. Plain C++ so that the
// CPU tests can check it.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "qsim_internal.h"

namespace qs {

bool tc_pipe_eligible(int n, qsim_dtype dt, qsim_prec prec, int kb)
{
    if (kb == 7) return n >= 14 && dt == QSIM_C64 && prec == QSIM_PREC_BF16X3;
    return n >= 13 && ((dt == QSIM_C64 && (prec == QSIM_PREC_BF16X3 || prec == QSIM_PREC_3XTF32)) ||
                       (dt == QSIM_C128 && prec == QSIM_PREC_BF16X6));
}

int tc_pipe_kind(qsim_dtype dt, qsim_prec prec, int kb)
{
    if (kb == 7) return 3;
    return dt == QSIM_C128 ? 1 : prec == QSIM_PREC_3XTF32 ? 2 : 0;
}

// Tile geometry of a block: tile qubits T = the block's kb qubits (6, or 7
// for kind 3) and the 7 lowest qubits outside it; the tensor map views the
// ket as up to 5 dimensions, each a run of consecutive qubits of T (at most
// 8 per dimension) plus the non-tile qubits above it, so a box is exactly
// the tile's amplitudes with the tile base's bits as coordinates. Runs
// beyond the fifth become extra boxes along dimension 4.
//
// kind 1 (complex128, 16-byte amplitudes) and kind 2 (complex64 with TF32
// operands): the box is a quarter tile, the tile qubits other than the
// block's two highest (block bits 4, 5), which become coordinates. For
// complex128 dimension 0 counts 8-byte halves, so its run is at most 7
// qubits (a box dimension spans at most 256 elements). kind 3 (7-qubit
// blocks): the box is an eighth of the 14-qubit tile, block bits 4, 5, 6
// being coordinates; a box again covers 11 tile qubits (16 KB).
qsim_status tc_pipe_prepare(int n, const TcSpec &ts, const void *pd_tables_dev, TcPipeHost &H, int kind)
{
    if (kind < 0 || kind > 3) return fail(QSIM_E_INVAL, "unknown tensor-core kernel variant %d", kind);
    const bool wide = kind == 1;          // 16-byte amplitudes (halves along dimension 0)
    const bool split = kind != 0;         // quarter- or eighth-tile boxes
    const int kb = kind == 3 ? 7 : 6;     // block bits
    const int ntq = kb + 7;               // tile qubits
    if (n < ntq || n > 36)
        return fail(QSIM_E_UNSUPPORTED, "pipelined tensor-core blocks of %d qubits need %d <= n <= 36", kb, ntq);
    uint64_t blk = 0;
    for (int b = 0; b < kb; b++) blk |= bit(ts.q[b]);
    std::vector<int> freeq;
    for (int p = 0; p < n && (int)freeq.size() < 7; p++)
        if (!(blk & bit(p))) freeq.push_back(p);
    std::vector<int> T;
    for (int p = 0; p < n; p++)
        if ((blk & bit(p)) || std::find(freeq.begin(), freeq.end(), p) != freeq.end()) T.push_back(p);
    const int es = wide ? 16 : 8;                   // bytes per amplitude
    const int nbox = split ? 11 : 13;                // tile qubits a box covers
    auto is_sel = [&](int p) {                       // a qubit whose value selects the load
        for (int b = 4; b < kb; b++)
            if (p == ts.q[b]) return true;
        return false;
    };
    std::vector<int> Tb;                             // box qubits, ascending
    for (int p : T)
        if (!split || !is_sel(p)) Tb.push_back(p);
    // chunks of consecutive box qubits, at most 8 each (7 for dimension 0 when wide)
    std::vector<std::pair<int, int>> ch;   // (first qubit, length)
    for (int j = 0; j < nbox; j++) {
        const int p = Tb[j];
        const int cap = (wide && ch.size() == 1) ? 7 : 8;
        if (!ch.empty() && ch.back().first + ch.back().second == p && ch.back().second < cap)
            ch.back().second++;
        else
            ch.push_back({p, 1});
    }
    int nd = std::min<int>((int)ch.size(), 5);
    TcPipeArgs &A = H.args;
    memset(&A, 0, sizeof A);
    A.ntiles = 1ull << (n - ntq);
    for (int j = 0; j < ntq; j++) A.tpos[j] = T[j];
    uint64_t gdim[5], gstr[4];
    uint32_t box[5], estr[5] = {1, 1, 1, 1, 1};
    int boxbits = 0;
    for (int d = 0; d < 5; d++) {
        if (d < nd) {
            const int lo = ch[d].first;
            const int hi = (d + 1 < nd) ? ch[d + 1].first : n;
            A.dim_lo[d] = lo;
            A.dim_bits[d] = hi - lo;
            gdim[d] = (d == 0 && wide ? 2ull : 1ull) << (hi - lo);
            box[d] = (d == 0 && wide ? 2u : 1u) << ch[d].second;
            boxbits += ch[d].second;
        } else {
            A.dim_lo[d] = n;
            A.dim_bits[d] = 0;
            gdim[d] = 1;
            box[d] = 1;
        }
        if (d >= 1) gstr[d - 1] = (uint64_t)es << ((d < nd) ? A.dim_lo[d] : n);
    }
    // extra boxes enumerate the qubits of chunks 5.. (inside dimension 4)
    std::vector<int> xq;
    for (size_t c = 5; c < ch.size(); c++)
        for (int i = 0; i < ch[c].second; i++) xq.push_back(ch[c].first + i);
    if ((int)xq.size() > 2 || boxbits + (int)xq.size() != nbox)
        return fail(QSIM_E_UNSUPPORTED, "tensor-core tile geometry not covered (%d extra qubits)", (int)xq.size());
    A.nload = 1 << xq.size();
    for (int v = 0; v < A.nload; v++) {
        int off = 0;
        for (size_t i = 0; i < xq.size(); i++)
            if ((v >> i) & 1) off |= 1 << (xq[i] - A.dim_lo[4]);
        A.xoff[v] = off;
    }
    A.box_bytes = (uint32_t)es << boxbits;
    // in-stage element index: rank among the box qubits (the qubits that
    // select a split load add nothing)
    auto rank_bit = [&](int q) {
        const auto it = std::find(Tb.begin(), Tb.end(), q);
        return it == Tb.end() ? 0 : 1 << (int)(it - Tb.begin());
    };
    for (int l = 0; l < (1 << kb); l++) {
        int r = 0;
        uint64_t o = 0;
        for (int b = 0; b < kb; b++)
            if ((l >> b) & 1) {
                r |= rank_bit(ts.q[b]);
                o |= bit(ts.q[b]);
            }
        A.posL[l] = (uint16_t)r;
        A.spL[l] = o;
    }
    for (int g = 0; g < 128; g++) {
        int r = 0;
        uint64_t o = 0;
        for (int f = 0; f < 7; f++)
            if ((g >> f) & 1) {
                r |= rank_bit(freeq[f]);
                o |= bit(freeq[f]);
            }
        A.posG[g] = (uint16_t)r;
        A.spG[g] = o;
    }
    A.ntb = n - ntq;
    // tile qubits 0..rot_shift-1 are the in-stage bits 0..rot_shift-1 (the
    // tile holds the lowest qubits: each is a block qubit or one of the
    // lowest outside ones); one shared-memory row holds 2^rot_shift amplitudes
    A.rot_shift = wide ? 3 : 4;
    A.rot_bits = 0;
    for (int b = 0; b < kb; b++) A.rot_bits += ts.q[b] < A.rot_shift;
    for (int b = 1; b < kb; b++)
        if (ts.q[b] <= ts.q[b - 1])
            return fail(QSIM_E_UNSUPPORTED, "tensor-core block bits not in ascending qubit order");
    A.vecw = (wide || ts.q[0] != 0) ? 0 : ts.q[1] != 1 ? 1 : 2;   // complex64 only
    A.wide = wide;
    A.kind = kind;
    A.kb = kb;
    for (int i = 0; i < 3; i++) A.qpos[i] = (split && 4 + i < kb) ? ts.q[4 + i] : 0;
    A.tturn = pd_tables_dev ? (const uint64_t *)pd_tables_dev : nullptr;
    A.gfac = pd_tables_dev ? (const float2 *)((const unsigned char *)pd_tables_dev + (size_t)kb * 24 * 8) : nullptr;
    H.rank = 5;
    for (int d = 0; d < 5; d++) {
        H.gdim[d] = gdim[d];
        H.box[d] = box[d];
        H.estr[d] = estr[d];
        if (d < 4) H.gstr[d] = gstr[d];
    }
    for (int f = 0; f < 7; f++) H.freeq[f] = freeq[f];
    return QSIM_OK;
}

// Deferred-phase tables of a block: T_b(amplitude index) = sum of tw[e] over
// the partners pbit[e] of block bit b whose bit is set; the partners are
// outside the block, so each is either a tile-index bit or a group bit.
// tturn[b][i] sums the partners at the i-th non-tile qubit; gfac[g][b] =
// exp(2 pi i (sum of the partners among g's bits)), in double, rounded.
// Block bits kb = ts.kb (6 or 7); off has kb + 1 entries.
void tc_pipe_tables(int n, const TcSpec &ts, const std::vector<int32_t> &off, const std::vector<int32_t> &pbit,
                    const std::vector<uint64_t> &tw, std::vector<unsigned char> &out)
{
    const int kb = ts.kb == 7 ? 7 : 6;
    uint64_t blk = 0;
    for (int b = 0; b < kb; b++) blk |= bit(ts.q[b]);
    std::vector<int> freeq;
    for (int p = 0; p < n && (int)freeq.size() < 7; p++)
        if (!(blk & bit(p))) freeq.push_back(p);
    uint64_t tmask = blk;
    for (int f : freeq) tmask |= bit(f);
    std::vector<int> tbit;   // i-th tile-index bit -> qubit
    for (int p = 0; p < n; p++)
        if (!(tmask & bit(p))) tbit.push_back(p);
    std::vector<uint64_t> tturn((size_t)kb * 24, 0);
    std::vector<float> gfac((size_t)128 * kb * 2, 0.f);
    for (int b = 0; b < kb; b++) {
        for (size_t i = 0; i < tbit.size(); i++)
            for (int e = off[b]; e < off[b + 1]; e++)
                if (pbit[e] == tbit[i]) tturn[b * 24 + i] += tw[e];
        for (int g = 0; g < 128; g++) {
            uint64_t o = 0;
            for (int f = 0; f < 7; f++)
                if ((g >> f) & 1) o |= bit(freeq[f]);
            uint64_t t = 0;
            for (int e = off[b]; e < off[b + 1]; e++)
                if ((o >> pbit[e]) & 1) t += tw[e];
            const double ang = 2.0 * 3.14159265358979323846 * ((double)t / 18446744073709551616.0);
            gfac[(g * kb + b) * 2] = (float)std::cos(ang);
            gfac[(g * kb + b) * 2 + 1] = (float)std::sin(ang);
        }
    }
    out.resize(tc_pipe_table_bytes(kb));
    memcpy(out.data(), tturn.data(), (size_t)kb * 24 * 8);
    memcpy(out.data() + (size_t)kb * 24 * 8, gfac.data(), (size_t)128 * kb * 8);
}

}  // namespace qs
