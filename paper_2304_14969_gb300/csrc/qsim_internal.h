// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <complex>
#include <string>
#include <vector>

#include "../../include/qsim.h"

namespace qs {

// ------------------------------------------------------------ errors
qsim_status fail(qsim_status st, const char *fmt, ...);
qsim_status cuda_fail(cudaError_t e, const char *what);
void clear_error();
const char *g_last_error_cstr();

#define QS_CUDA(expr)                                              \
    do {                                                           \
        cudaError_t _e = (expr);                                   \
        if (_e != cudaSuccess) return ::qs::cuda_fail(_e, #expr);  \
    } while (0)

#define QS_TRY(expr)                                \
    do {                                            \
        qsim_status _s = (expr);                    \
        if (_s != QSIM_OK) return _s;               \
    } while (0)

// ------------------------------------------------------- host matrices
using cd = std::complex<double>;

// Matrix of a named gate kind in FP64 (2x2 or 4x4, row-major). Returns the
// dimension, 0 for an unknown kind. pool: matrix pool of the circuit.
int gate_matrix(const qsim_gate &g, const double *pool, int64_t pool_len, cd *m);
bool gate_is_two_qubit_kind(int kind);
// Validates a gate against n qubits; returns QSIM_OK or QSIM_E_INVAL (with
// the error message set).
qsim_status validate_gate(const qsim_gate &g, int n, const double *pool, int64_t pool_len);
// True when the gate's matrix is diagonal (phase-only) in its qubits.
bool gate_is_diagonal(const qsim_gate &g);

// ------------------------------------------------------- device state
struct Scratch {
    double *d = nullptr;     // device partials
    double *h = nullptr;     // pinned host results
    size_t cap = 0;          // doubles in d
};

}  // namespace qs

struct qsim_state {
    int n = 0;
    qsim_dtype dt = QSIM_C64;
    cudaStream_t stream = nullptr;
    void *amps = nullptr;
    bool owned = false;
    int device = 0;
    std::vector<int> l2p;    // logical qubit -> physical bit
    qs::Scratch red;
    // error word of kernels that report asynchronously (tensor-core blocks:
    // an MMA completion wait that gave up); device word + pinned host copy,
    // allocated on first use, read at the next call that synchronises
    int *d_err = nullptr;
    int *h_err = nullptr;
    // a second ket-sized buffer for permutations (downloads of a relabelled
    // ket, materialisation), allocated at the first permutation of a ket of
    // at most 8 GiB and kept until destroy; larger kets take a
    // stream-ordered temporary per permutation instead
    void *perm = nullptr;
    size_t amp_bytes() const { return (size_t)(dt == QSIM_C64 ? 8 : 16) << n; }
    uint64_t N() const { return (uint64_t)1 << n; }
};

namespace qs {

// Bit positions are physical unless stated otherwise.
struct InsSpec {
    int npos = 0;
    int pos[12] = {0};  // ascending
};

// Tensor-core block (k <= 6 padded to 6, or k = 7): physical bit of block
// bit b (ascending) and the sorted block qubits for group expansion.
struct TcSpec {
    int q[7];
    int kb = 6;              // block bits: 6, or 7 (complex64 BF16X3 blocks of the 7-qubit kernel)
    InsSpec ins;
    // optional pre-diagonal: the amplitude with block index l in the group
    // whose outside bits are G is multiplied by exp(2 pi i sum_b l_b T_b(G))
    // with T_b(G) = sum of pd_tw[e] over e in [pd_off[b], pd_off[b+1]) with
    // bit pd_bit[e] of G set (device arrays, NULL when there is none)
    const int32_t *pd_off;
    const int32_t *pd_bit;
    const uint64_t *pd_tw;
};
// kb = 7: the block is padded to seven qubits and packed for the 7-qubit
// kernel (complex64 BF16X3 only).
qsim_status tc_build(int n, int k, const int *phys, const cd *u, qsim_prec prec, std::vector<unsigned char> &A,
                     TcSpec &ts, int kb = 6);
cudaError_t tc_launch(qsim_state *s, const TcSpec &ts, const unsigned char *dA, qsim_prec prec, int *derr);

// Pipelined block kernel (BF16X3 on complex64, BF16X6 on complex128;
// n >= 13): tile geometry and tables, built on the host per block
// (k_tc_pipe.cu).
struct TcPipeArgs {
    uint64_t ntiles;
    int tpos[14];            // tile qubits, ascending (tile index bits go to the other positions)
    int dim_lo[5];           // lowest qubit of each tensor dimension
    int dim_bits[5];         // qubits covered by each tensor dimension (coordinate width)
    int nload;               // boxes per tile (per quarter tile when wide)
    int xoff[4];             // coordinate offset along dimension 4 of box v
    uint32_t box_bytes;
    uint16_t posL[128];      // in-stage element index of block index l (split loads: within its load)
    uint16_t posG[128];      // in-stage element index of group g
    uint64_t spL[128];       // amplitude offset of block index l
    uint64_t spG[128];       // amplitude offset of group g
    int ntb;                 // tile-index bits (n - 13, or n - 14 for 7-qubit blocks)
    int rot_bits;            // block qubits among qubits 0..3 (= block index bits 0..rot_bits-1)
    int vecw;                // complex64: the lowest qubits are block bits 0..vecw-1, so a thread's
                             // amplitudes come in runs of 2^vecw adjacent ones (stored 16 or 32 bytes at a time)
    int rot_shift;           // lanes sharing a shared-memory row: 2^rot_shift (4: 8-byte, 3: 16-byte amplitudes)
    // complex128 kets (wide = 1): a tile is loaded as four quarter tiles,
    // one per value of block bits 4, 5 (qubits qpos[0], qpos[1]), so that
    // each quarter is read by the converter warps of one part, one on each
    // SM sub-partition; posL / posG then rank the other 11 tile qubits
    int wide;
    int qpos[3];             // block qubits 4, 5 (and 6) whose values select a split load
    int kind;                // 0: complex64 BF16X3 whole tiles, 1: complex128 BF16X6, 2: complex64 3XTF32
                             // (quarter tiles of 8-byte amplitudes, TF32 operands), 3: complex64 BF16X3
                             // 7-qubit blocks (tiles of 14 qubits in eighths, one per value of block bits 4..6)
    int kb;                  // block bits (6, or 7 for kind 3)
    // deferred phases (NULL if none): exp(2 pi i T_b) of block bit b for a
    // group is the product of a tile factor, from the turns tturn[b][i] of
    // the tile-index bits i, and the group factor gfac[g][b]
    const uint64_t *tturn;   // [kb][24]
    const float2 *gfac;      // [128][kb]
};
struct TcPipeHost {
    TcPipeArgs args;
    int rank;
    uint64_t gdim[5], gstr[4];
    uint32_t box[5], estr[5];
    int freeq[7];
};
// complex64 with BF16X3 or 3XTF32, or complex128 with BF16X6; n >= 13
// (kb = 7: complex64 with BF16X3 and n >= 14)
bool tc_pipe_eligible(int n, qsim_dtype dt, qsim_prec prec, int kb = 6);
// kernel variant (TcPipeArgs::kind) of an eligible pairing
int tc_pipe_kind(qsim_dtype dt, qsim_prec prec, int kb = 6);
qsim_status tc_pipe_prepare(int n, const TcSpec &ts, const void *pd_tables_dev, TcPipeHost &H, int kind = 0);
// Deferred-phase tables of a block (tturn then gfac: tc_pipe_table_bytes(kb)
// bytes; kTcPipeTableBytes is the larger of the two sizes).
inline size_t tc_pipe_table_bytes(int kb) { return (size_t)kb * 24 * 8 + 128 * (size_t)kb * 8; }
const size_t kTcPipeTableBytes = 7 * 24 * 8 + 128 * 7 * 8;
void tc_pipe_tables(int n, const TcSpec &ts, const std::vector<int32_t> &off, const std::vector<int32_t> &pbit,
                    const std::vector<uint64_t> &tw, std::vector<unsigned char> &out);
// norm_out (device, optional): the kernel adds the sum of |amplitude|^2 of
// everything it writes (FP64 accumulation); the caller zeroes it first.
cudaError_t tc_pipe_launch(qsim_state *s, const TcPipeHost &H, const unsigned char *dU, int *derr,
                           double *norm_out = nullptr);
// The 7-qubit variant (kind 3, k_tc_pipe7.cu); tc_pipe_launch forwards to it.
cudaError_t tc_pipe7_launch(qsim_state *s, const TcPipeHost &H, const unsigned char *dU, int *derr,
                            double *norm_out);

// Grouped launches of the pipelined kernel (batched circuits): one CTA per
// work entry = a range of tiles of one block of one circuit.
struct alignas(64) TcBatchDesc {
    unsigned char tmap[128];     // tensor map of the block over the circuit's ket
    TcPipeArgs args;
    const unsigned char *U;      // BF16 hi / lo operand of the block (64 KB, device; complex64 kets only)
    float2 *amps;                // the circuit's ket (device)
    int circ;                    // circuit index (latency stamps)
};
struct TcWork {
    int32_t desc, pad;
    uint64_t tile0, ntiles;
};
qsim_status tc_pipe_encode(const TcPipeHost &H, void *amps, unsigned char tmap[128]);
cudaError_t tc_pipe_launch_grouped(const TcBatchDesc *descs, const TcWork *works, int nwork, unsigned long long *t0,
                                   unsigned long long *t1, int *err, cudaStream_t st);

// Asynchronous error word of a state (see qsim_state): ensure allocates it,
// fetch enqueues its copy to the host (before a synchronisation), check
// reports and clears it (after the synchronisation).
qsim_status err_ensure(qsim_state *s);
void err_fetch(qsim_state *s);
qsim_status err_check(qsim_state *s);

// ------------------------------------------------------ kernel launchers
// (all stream-ordered, no sync; return cuda errors)
cudaError_t launch_gate1(qsim_state *s, const cd u[4], int t, uint64_t cmask, uint64_t cval);
cudaError_t launch_gate2(qsim_state *s, const cd u[16], int q0, int q1);
cudaError_t launch_cphase(qsim_state *s, int q0, int q1, double theta);
cudaError_t launch_swap(qsim_state *s, int q0, int q1);
cudaError_t launch_fused_simt(qsim_state *s, int k, const int *phys, const cd *u);
qsim_status apply_fused_tc(qsim_state *s, int k, const int *phys, const cd *u, qsim_prec prec);
cudaError_t launch_set_basis(qsim_state *s, uint64_t x_phys);
cudaError_t launch_scale(void *amps, qsim_dtype dt, uint64_t N, double f, cudaStream_t st);
cudaError_t launch_permute(const void *src, void *dst, qsim_dtype dt, int n, const int *new_of_old,
                           cudaStream_t st);

// Reductions (write FP64 results into s->red.h after a stream sync).
qsim_status reduce_norm(qsim_state *s, double *out);
qsim_status reduce_prob1(qsim_state *s, int phys_q, double *p1, double *total);
qsim_status reduce_inner(qsim_state *a, qsim_state *b, double out[2]);
qsim_status reduce_bloch(qsim_state *s, int phys_q, double out4[4]);
qsim_status reduce_bloch_all(qsim_state *s, double *sums /* 4 per physical qubit */);
qsim_status probs_to_device(qsim_state *s, double *d_out);
// d_gate (device, optional): when it holds 0 the tiled passes return at once
// (a check round with no candidate: the sums are then not read).
qsim_status bloch_sums_device(const void *amps, qsim_dtype dt, int n, cudaStream_t stream, Scratch &sc,
                              const int *d_gate, double *d_out, int *passes);

// Generic device buffers ("raw" kets used by approx mode).
qsim_status ensure_scratch(Scratch &sc, size_t doubles);
void free_scratch(Scratch &sc);

// Helpers
inline uint64_t bit(int q) { return (uint64_t)1 << q; }
int default_grid(uint64_t work, int threads);
int num_sms();

}  // namespace qs
