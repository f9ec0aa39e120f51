/*
 * qsim.h -- C ABI of the GB300 state-vector library (libqsim.so).
 *
 * Method: arXiv 2304.14969, "Exact and approximate simulation of large
 * quantum circuits on a single GPU". The library implements its
 * data-parallel hot path: Schroedinger-picture application of gates to all
 * 2^n amplitudes of a ket (Sec. II), the FP64 norm / probability /
 * inner-product / Bloch-vector reductions, and the Schmidt decomposition
 * rounding (SDRP) approximate mode (Sec. III.A-B).
 *
 * Conventions for every call:
 *  - Amplitudes are interleaved complex numbers: QSIM_C64 = two float32
 *    (re, im), QSIM_C128 = two float64. Qubit q is bit q of the amplitude
 *    index (little-endian); amplitude index i holds basis state
 *    sum_q b_q 2^q.
 *  - Host pointers are plain CPU memory; device pointers are CUDA global
 *    memory on the current device. Every pointer argument says which.
 *  - Gate matrices are row-major complex, passed as re/im interleaved
 *    doubles. For a two-qubit matrix, q0 is bit 0 and q1 is bit 1 of the
 *    row/column index. They are copied before the call returns.
 *  - Gate calls are ordered on the state's CUDA stream and return before
 *    the work finishes. Reductions, downloads and run_* calls that return
 *    host values synchronise that stream.
 *  - Every call returns a qsim_status; nothing aborts the process. On an
 *    error, qsim_last_error() gives a one-line reason (thread-local).
 *    Argument errors (qubit >= n, duplicate qubits, a control equal to the
 *    target, k > n, NULL pointers) are found on the host before any launch
 *    and return QSIM_E_INVAL with the state unchanged.
 *  - A state's logical qubits may be stored permuted (SWAP folded into a
 *    relabel, Table I "SWAP gate is constant complexity"). Every call takes
 *    and returns logical qubit numbers and logical index order; the
 *    permutation is visible only through qsim_qubit_map/qsim_device_ptr.
 */
#ifndef QSIM_H
#define QSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qsim_state qsim_state;
typedef struct qsim_plan qsim_plan;
typedef struct qsim_batch qsim_batch;
typedef struct qsim_mlp qsim_mlp;

typedef enum { QSIM_C64 = 0, QSIM_C128 = 1 } qsim_dtype;

/* Arithmetic of fused blocks (qsim_apply_fused, fused plans).
 * NATIVE: SIMT FMA in the state's precision.
 * 3XTF32: tensor-core products a_hi*b_hi + a_hi*b_lo + a_lo*b_hi of TF32
 *         parts, FP32 accumulation (complex64 states only).
 * BF16X3: the same three-product split with BF16 parts (complex64 states).
 * BF16X6: complex128 states: amplitudes rounded to FP32, each operand split
 *         into three BF16 slices (x ~ x0 + x1 + x2, 24 bits), the six slice
 *         products x_i*y_j with i + j <= 2 accumulated in FP32, results
 *         widened to FP64 (exactly); n >= 13. Per-block error ~1e-7
 *         relative, against ~1e-5 for BF16X3. */
typedef enum {
    QSIM_PREC_NATIVE = 0,
    QSIM_PREC_3XTF32 = 1,
    QSIM_PREC_BF16X3 = 2,
    QSIM_PREC_BF16X6 = 3
} qsim_prec;

typedef enum {
    QSIM_OK = 0,
    QSIM_E_INVAL = 1,        /* bad argument, found before any launch */
    QSIM_E_NOMEM = 2,        /* device allocation failed */
    QSIM_E_CUDA = 3,         /* a CUDA call failed */
    QSIM_E_TIMEOUT = 4,      /* a bounded device-side wait gave up */
    QSIM_E_BUDGET = 5,       /* approximate mode exceeded its memory budget */
    QSIM_E_UNSUPPORTED = 6   /* valid request this build does not handle */
} qsim_status;

/* Gate kinds of qsim_gate (one-qubit kinds < 16, two-qubit kinds >= 16). */
typedef enum {
    QSIM_G_H = 0, QSIM_G_X = 1, QSIM_G_Y = 2, QSIM_G_Z = 3, QSIM_G_S = 4, QSIM_G_T = 5,
    QSIM_G_SQRTX = 6, QSIM_G_SQRTY = 7, QSIM_G_SQRTW = 8,
    QSIM_G_U3 = 9,     /* Sec. III.C U(theta=params[0], phi=params[1], lambda=params[2]) */
    QSIM_G_PHASE = 10, /* diag(1, e^{i params[0]}) */
    QSIM_G_RZ = 11,    /* diag(e^{-i params[0]/2}, e^{i params[0]/2}) */
    QSIM_G_MAT1 = 12,  /* explicit 2x2 from the circuit's matrix pool */
    QSIM_G_CP = 16,    /* diag(1,1,1,e^{i params[0]}), Sec. II.E controlled phase */
    QSIM_G_SWAP = 17,
    QSIM_G_FSIM = 18,  /* fSim(theta=params[0], phi=params[1]) */
    QSIM_G_MAT2 = 19   /* explicit 4x4 from the circuit's matrix pool */
} qsim_gate_kind;

#define QSIM_MAX_CONTROLS 4

/* One gate of a circuit (host memory). One-qubit kinds use q0 as target and
 * may carry up to QSIM_MAX_CONTROLS controls; bit j of control_values is
 * the value controls[j] must have (1: "C" control, 0: "A" control, Sec.
 * III.C). Two-qubit kinds use q0 (matrix bit 0) and q1 (bit 1) and take no
 * controls. matrix_offset indexes the circuit's matrix pool in doubles
 * (re/im interleaved), or is -1. */
typedef struct {
    int32_t kind;
    int32_t q0, q1;
    int32_t ncontrols;
    int32_t controls[QSIM_MAX_CONTROLS];
    uint32_t control_values;
    int32_t reserved;
    double params[4];
    int64_t matrix_offset;
} qsim_gate;

/* A circuit on n logical qubits (all host memory, read during the call). */
typedef struct {
    int32_t n;
    int32_t ngates;
    const qsim_gate *gates;
    const double *matrices;  /* may be NULL when no gate uses the pool */
    int64_t nmatrix_doubles;
} qsim_circuit;

typedef enum { QSIM_MODE_PER_GATE = 0, QSIM_MODE_FUSED = 1 } qsim_mode;

/* Options of qsim_run_circuit / qsim_plan_create. Zero means "default". */
typedef struct {
    int32_t mode;           /* qsim_mode */
    int32_t prec;           /* qsim_prec of fused blocks (fused mode) */
    int32_t tile_qubits;    /* fused: qubits per on-chip tile t (default 13/12 for c64/c128) */
    int32_t low_qubits;     /* fused: low physical qubits kept in every tile (default 5/4) */
    int32_t max_block;      /* tensor-core plans: 7 fuses blocks of up to 7 qubits (complex64,
                               BF16X3, n >= 14, else QSIM_E_UNSUPPORTED); any other value: 6 */
    int32_t relabel_swaps;  /* 1: SWAP changes the qubit map instead of moving data */
    int32_t reserved[6];
} qsim_run_opts;

/* ------------------------------------------------------------- states */

/* Allocates a ket of n qubits (1 <= n <= 36) on the current device, owned
 * by the library, initialised to |0...0> (Sec. II: |psi_0>). stream is a
 * cudaStream_t (NULL = the legacy default stream). */
qsim_status qsim_create(int n, qsim_dtype dt, void *stream, qsim_state **out);

/* Wraps an existing device buffer of 2^n amplitudes (for example a
 * PyTorch tensor). The library never frees it; the caller keeps it alive
 * and 16-byte aligned. The contents are taken as the state in identity
 * qubit order. */
qsim_status qsim_wrap(int n, qsim_dtype dt, void *dev_amps, void *stream, qsim_state **out);

qsim_status qsim_destroy(qsim_state *s);

/* Sets the state to the basis state |x> (x < 2^n) and the map to identity. */
qsim_status qsim_set_basis(qsim_state *s, uint64_t x);

/* Copies 2^n amplitudes of the state's dtype from host memory (logical
 * index order); the map becomes the identity. Stream-ordered: from
 * page-locked host memory the copy is asynchronous, and the buffer must not
 * change until the stream has passed it (e.g. qsim_synchronize); from
 * pageable memory the call returns once the data has been staged. */
qsim_status qsim_upload(qsim_state *s, const void *host_amps);

/* Copies the state to host memory in logical index order (synchronises). */
qsim_status qsim_download(qsim_state *s, void *host_amps);

/* Stream-ordered form of qsim_download: queues the copy (and the permutation
 * into logical order when the map is not the identity) and returns.
 * host_amps should be page-locked; it holds the result once the stream has
 * passed the copy (qsim_synchronize). Lets a caller overlap one ket's
 * download with another's upload and gates. The permutation goes through a
 * second ket-sized device buffer that a state of at most 8 GiB allocates at
 * its first permutation and keeps until qsim_destroy (so kets pipelined on
 * different streams never wait for one another's temporaries); larger kets
 * take a stream-ordered temporary per call. */
qsim_status qsim_download_async(qsim_state *s, void *host_amps);

/* Device address of the amplitudes (physical order) and the current map:
 * l2p[q] = physical bit holding logical qubit q (host array of n). */
qsim_status qsim_device_ptr(const qsim_state *s, void **dev_amps);
qsim_status qsim_qubit_map(const qsim_state *s, int32_t *l2p);

/* Moves the amplitudes so that the map becomes the identity (one
 * read+write pass per permutation cycle group; no-op if already identity). */
qsim_status qsim_materialize(qsim_state *s);

/* Waits for all work queued on the state's stream. Kernels that report
 * errors asynchronously (a bounded wait inside a tensor-core block that
 * gave up) are reported here, and by every other call that synchronises
 * the stream (reductions, downloads), as QSIM_E_TIMEOUT; the report clears
 * the error and the state stays usable (its amplitudes are then invalid). */
qsim_status qsim_synchronize(qsim_state *s);

/* Self-test of that failure path (the paper has no counterpart): queues on
 * s's stream one CTA that waits on an mbarrier no thread ever arrives at,
 * with the bounded wait the tensor-core kernels use but a limit of limit_ns
 * nanoseconds of device time (1e3 .. 1e10). The wait gives up and sets s's
 * asynchronous error word; nothing else is touched (s's amplitudes stay
 * valid). Returns QSIM_E_INVAL for a limit outside the range. */
qsim_status qsim_selftest_wait_timeout(qsim_state *s, int64_t limit_ns);

/* --------------------------------------------------- per-gate path */

/* Sec. II, one-qubit gate: (a, b) <- (u00 a + u01 b, u10 a + u11 b) on every
 * index pair that differs in bit `target`, restricted to indices where
 * controls[j] has value bit j of control_values. u: 8 doubles (2x2 complex,
 * row-major, re/im). controls: host array of ncontrols (<= 4), may be NULL
 * when ncontrols = 0. */
qsim_status qsim_apply_gate(qsim_state *s, const double u[8], int target,
                            const int *controls, int ncontrols, uint64_t control_values);

/* Sec. II.E controlled phase: psi_i <- e^{i theta} psi_i where bits q0 and q1
 * are both 1 (touches a quarter of the amplitudes). */
qsim_status qsim_apply_cphase(qsim_state *s, int q0, int q1, double theta);

/* Dense two-qubit gate: u is 32 doubles (4x4 complex), q0 = row bit 0. */
qsim_status qsim_apply_2q(qsim_state *s, const double u[32], int q0, int q1);

/* Table I SWAP. relabel = 1 swaps the two entries of the qubit map (no data
 * moves); relabel = 0 exchanges the amplitudes. */
qsim_status qsim_apply_swap(qsim_state *s, int q0, int q1, int relabel);

/* Fused block: U of size 2^k x 2^k (k <= 7; host, 2*4^k doubles, re/im,
 * row-major) applied on qubits[0..k-1], where qubits[b] is bit b of U's
 * row/column index (Table I "coalesced gates with a single traversal").
 * prec selects SIMT (NATIVE, k <= 7) or the tensor-core split precisions;
 * the tensor-core forms take k <= 6 (smaller blocks are padded with
 * identity qubits) and a complex64 state with n >= 6 (3XTF32, BF16X3) or a
 * complex128 state with n >= 13 (BF16X6), or k = 7 with BF16X3 on a
 * complex64 state with n >= 14; other pairings return QSIM_E_UNSUPPORTED. */
qsim_status qsim_apply_fused(qsim_state *s, int k, const int *qubits, const double *u,
                             qsim_prec prec);

/* ------------------------------------------------ circuits and plans */

/* Runs a whole circuit on s (circuit n must equal the state's n). Per-gate
 * mode issues one kernel per gate; fused mode builds a plan (below) and
 * executes it. opts may be NULL (per-gate, no relabel). */
qsim_status qsim_run_circuit(qsim_state *s, const qsim_circuit *c, const qsim_run_opts *opts);

/* Plans the fused execution of a circuit once: gates are grouped into
 * passes, each one read+write of the ket in HBM with all of the pass's
 * gates applied to 2^t-amplitude tiles on chip. */
qsim_status qsim_plan_create(const qsim_circuit *c, qsim_dtype dt, const qsim_run_opts *opts,
                             qsim_plan **out);
/* As qsim_plan_create, for the dtype of s and starting from s's current
 * qubit map, so that a ket left permuted by earlier SWAP relabels is used
 * in place (no data movement before the first pass). */
qsim_status qsim_plan_create_for_state(const qsim_circuit *c, const qsim_state *s, const qsim_run_opts *opts,
                                       qsim_plan **out);
qsim_status qsim_plan_destroy(qsim_plan *p);
/* info[0] passes, info[1] gates, info[2] dense blocks, info[3] swaps
 * folded into the map, info[4] tile qubits, info[5] low qubits. */
qsim_status qsim_plan_info(const qsim_plan *p, int64_t info[8]);
/* Executes the plan on s (stream-ordered, no host sync). If s's qubit map is
 * not the plan's starting map, the amplitudes are first permuted to it (one
 * extra read+write of the ket). */
qsim_status qsim_plan_execute(qsim_state *s, const qsim_plan *p);
/* Executes the plan and returns the FP64 sum of |psi_i|^2 of the result in
 * *norm (synchronises), as qsim_plan_execute then qsim_norm. When the plan
 * ends with a tensor-core block the sum is taken by that block's write-back
 * (FP32 runs of 16 squares, FP64 accumulation) instead of a separate read
 * of the ket. */
qsim_status qsim_plan_execute_norm(qsim_state *s, const qsim_plan *p, double *norm);

/* ------------------------------------------------------ reductions */

/* FP64 sum of |psi_i|^2 (synchronises). */
qsim_status qsim_norm(qsim_state *s, double *out);

/* psi <- psi / sqrt(sum |psi_i|^2) with the sum in FP64 (Sec. III.A step 3,
 * "normalized state"). */
qsim_status qsim_renormalize(qsim_state *s);

/* P(qubit = 1) = sum_{bit q = 1} |psi_i|^2 / sum |psi_i|^2, FP64. */
qsim_status qsim_measure_prob(qsim_state *s, int qubit, double *p1);

/* p_i = |psi_i|^2 in FP64 for all i, written to host memory in logical
 * index order (2^n doubles). */
qsim_status qsim_probs(qsim_state *s, double *host_out);

/* <a|b> = sum_i conj(a_i) b_i in FP64 (Eq. fid_exact uses |<a|b>|^2).
 * a and b must have the same n and dtype; maps may differ. out[0] = re,
 * out[1] = im. */
qsim_status qsim_inner_product(qsim_state *a, qsim_state *b, double out[2]);

/* <a|b> = sum_i conj(a_i) b_i in FP64 for callers that cannot let the library
 * allocate device memory (the paper has no counterpart: this is a service
 * variant of qsim_inner_product). a_dev and b_dev are device arrays of 2^n
 * interleaved complex numbers of dt in the same qubit order, 1 <= n <= 36;
 * out is host memory (out[0] = re, out[1] = im). Partial sums live in one
 * fixed 16.4 KB __device__ array of the library, so the call performs no
 * cudaMalloc, cudaFree or other allocation; it synchronises `stream`
 * (cudaStream_t, NULL = legacy default). The first call on a device looks up
 * that array's address (cudaGetSymbolAddress) with the device current; make
 * that first call before any stream capture. All calls share the array:
 * calls whose kernels overlap on the GPU race. n outside [1, 36] returns
 * QSIM_E_INVAL. */
qsim_status qsim_inner_product_noalloc(const void *a_dev, const void *b_dev, int n, qsim_dtype dt, void *stream,
                                       double out[2]);

/* Sec. III.A step 1: Bloch vector r = (<X_q>, <Y_q>, <Z_q>) of the reduced
 * state of `qubit`, normalised by the state's norm, FP64. */
qsim_status qsim_bloch(qsim_state *s, int qubit, double r[3]);

/* Bloch vectors of all n qubits (3n doubles, host), computed with tiled
 * passes that each cover several qubits. */
qsim_status qsim_bloch_all(qsim_state *s, double *r);

/* ------------------------------------------------- approximate mode */

/* One SDRP decision (Sec. III.A step 2). action: 0 kept, 1 rounded
 * (eps <= p/2), 2 exact separation (eps <= tau). reserved: 0 for a
 * one-qubit check; 1 + the second qubit for a two-qubit check (opts->pairs). */
typedef struct {
    int32_t gate;
    int32_t qubit;
    int32_t action;
    int32_t reserved;
    double eps;
    double r[3];
} qsim_decision;

typedef enum {
    QSIM_SCHED_EXHAUSTIVE = 0,  /* check every qubit of the touched subsystem */
    QSIM_SCHED_MLP = 1,         /* check the MLP's top_m candidates first */
    QSIM_SCHED_FORCED = 2       /* check exactly the (gate, qubit) list `force` */
} qsim_schedule;

typedef struct {
    double budget_bytes;        /* cap on the bytes of all subsystem kets (0: 64 GiB) */
    double tau;                 /* exact-separation threshold (0: 1e-6 c64, 1e-13 c128) */
    int32_t dtype;              /* qsim_dtype of the subsystem kets */
    int32_t schedule;           /* qsim_schedule */
    int32_t top_m;              /* MLP schedule: candidates per gate */
    int32_t fallback_every;     /* MLP schedule: exhaustive check every this many
                                   two-qubit gates (0: never) */
    int32_t exhaustive_from;    /* MLP schedule: a subsystem of at least this many
                                   qubits is checked exhaustively (memory is what a
                                   missed rounding costs; 0: never) */
    const qsim_mlp *mlp;        /* MLP schedule */
    const int32_t *force;       /* forced schedule: nforce (gate, qubit) pairs, host */
    int32_t nforce;
    int32_t log_cap;            /* capacity of log (entries) */
    qsim_decision *log;         /* host, optional */
    void *state_out;            /* host, optional: the expanded 2^n state (n <= 30),
                                   logical order, in dtype */
    float *trace_features;      /* host, optional: MLP features of each check */
    int32_t *trace_labels;      /* host, optional: 1 if that check rounded */
    int64_t trace_cap;
    void *stream;               /* cudaStream_t to run on (NULL: default) */
    int32_t unobservable;       /* 1: Sec. II.B unobservable optimisation (Table I, "eliminates
                                   Z-basis eigenstate controls"): before a controlled one-qubit
                                   gate or a controlled phase, a control (either qubit of a CP)
                                   that is a one-qubit subsystem whose probability of the other
                                   value is at most tau is projected onto that Z eigenstate (as
                                   an exact separation: F unchanged); a control holding the
                                   value the gate waits for is dropped, one holding the other
                                   value removes the gate. A gate left acting on one qubit is
                                   applied locally: nothing is composed and no check runs.
                                   0: off */
    int32_t pairs;              /* 1: two-qubit-subsystem SDRP (Sec. III.A, the rounding generalised
                                   to a subsystem of two qubits): after the one-qubit checks of a
                                   gate coupling exactly two qubits (a, b) still in one subsystem of
                                   three or more qubits, the pair's reduced density matrix rho_ab
                                   (FP64) gives eps = 1 - (its largest eigenvalue); eps <= p/2
                                   rounds (F <- F (1 - eps)) and eps <= tau separates exactly,
                                   projecting onto the top eigenvector, which becomes a two-qubit
                                   subsystem. Its log entry: qubit a, reserved 1 + b, r the three
                                   largest eigenvalues. 0: off */
} qsim_approx_opts;

typedef struct {
    double fidelity_model;      /* Eq. (fid_model): prod_j (1 - eps_j) */
    double seconds;             /* wall time of the run */
    int64_t n_rounds;           /* SDRP roundings */
    int64_t n_exact;            /* exact separations */
    int64_t n_checks;           /* qubits checked */
    int64_t n_bloch_passes;     /* reduction kernels over subsystem kets */
    int64_t peak_bytes;         /* peak bytes of subsystem kets */
    int64_t n_log;              /* decisions produced (may exceed log_cap) */
    int64_t n_trace;            /* trace rows produced (may exceed trace_cap) */
    int32_t max_subsystem_qubits;
    int32_t budget_gate;        /* gate index where the budget was hit, or -1 */
    int64_t n_unobservable;     /* gates removed or reduced by the unobservable optimisation */
} qsim_approx_result;

/* Runs circuit c from |0...0> with SDRP rounding at threshold p in [0, 1]
 * (Eq. sdrp: round when eps <= p/2; p = 0 rounds nothing, only exact
 * separations with eps <= tau happen) on a factorised ket: a list of
 * subsystem kets, composed when a two-qubit gate spans two of them
 * (Sec. II.A) and split when a check rounds or separates a qubit. Returns
 * QSIM_E_BUDGET (with result filled up to that gate) when the kets would
 * exceed budget_bytes. */
qsim_status qsim_approx_run(const qsim_circuit *c, double p, const qsim_approx_opts *opts,
                            qsim_approx_result *result);

/* ---------------------------------------------------------- batches */

typedef struct {
    int32_t tile_qubits;        /* 0: autotuned */
    int32_t low_qubits;         /* 0: autotuned */
    int32_t ctas;               /* persistent CTAs (0: one per SM x occupancy) */
    int32_t use_graph;          /* 1: launch through a captured CUDA graph */
    int32_t path;               /* per circuit: 0 autotuned (tensor-core blocks for a qubit count
                                   whose fastest tune-cache entry is a tensor-core plan, else
                                   fused SIMT passes), 1 fused SIMT passes only, 2 tensor-core
                                   blocks (BF16x3) for every circuit with n >= 13 */
    const char *tune_cache;     /* JSON file of autotuner results, may be NULL */
    void *stream;
} qsim_batch_opts;

/* Plans count circuits (complex64), allocates one device arena holding all
 * their kets, each initialised to |0...0>, and prepares the launch (captured
 * in a CUDA graph when use_graph = 1): one persistent launch runs every
 * circuit planned as fused SIMT passes; circuits planned as tensor-core
 * blocks (see path) run as one grouped launch per block round, each CTA a
 * range of tiles of one block, concurrently with it on a second stream. */
qsim_status qsim_batch_create(const qsim_circuit *const *cs, int count, const qsim_batch_opts *opts,
                              qsim_batch **out);
qsim_status qsim_batch_destroy(qsim_batch *b);
/* Uploads circuit i's initial state (host, 2^n complex64). */
qsim_status qsim_batch_upload(qsim_batch *b, int i, const void *host_amps);
/* Resets every ket to |0...0>. */
qsim_status qsim_batch_reset(qsim_batch *b);
/* Runs all circuits in one persistent launch. latency_s (host, count
 * doubles, optional) receives each circuit's device time from its first to
 * its last tile (globaltimer stamps); *seconds the launch's device time. */
qsim_status qsim_batch_run(qsim_batch *b, double *seconds, double *latency_s);
/* Downloads circuit i's final state (host, 2^n complex64, logical order). */
qsim_status qsim_batch_download(qsim_batch *b, int i, void *host_amps);
/* info[0] circuits, info[1] work items, info[2] ctas, info[3] arena bytes. */
qsim_status qsim_batch_info(const qsim_batch *b, int64_t info[8]);

/* Autotuner: times the circuit on a scratch state of its size as fused SIMT
 * passes with every tile width (10 .. 14 qubits) and, for complex64 with
 * n >= 13, as tensor-core blocks (BF16x3); returns the fastest in best_opts
 * (prec QSIM_PREC_BF16X3 for the tensor-core plan) and appends one JSON
 * line per candidate to tune_cache if not NULL: its time alone ("ms") and,
 * for complex64, its batch cost ("sm_ms": device time per circuit of a
 * batch of copies of the circuit that fills the GPU, run through the batch
 * runner); "path": "tc" marks the tensor-core plan. qsim_batch_create
 * ranks a qubit count's candidates by batch cost. */
qsim_status qsim_autotune(const qsim_circuit *c, qsim_dtype dt, const char *tune_cache,
                          qsim_run_opts *best_opts, double *best_seconds);

/* ------------------------------------------------ proposal network */

/* Two-hidden-layer MLP (nfeat -> hidden -> hidden -> 1 logit, ReLU) that
 * scores which qubits to check in the approximate mode. FP32 master
 * weights, BF16 copies for inference, FP32 accumulation. */
qsim_status qsim_mlp_create(int nfeat, int hidden, uint64_t seed, qsim_mlp **out);
qsim_status qsim_mlp_destroy(qsim_mlp *m);
/* Parameter vector layout: W1[hidden][nfeat], b1[hidden], W2[hidden][hidden],
 * b2[hidden], W3[hidden], b3[1] (host FP32). */
qsim_status qsim_mlp_num_params(const qsim_mlp *m, int64_t *count);
qsim_status qsim_mlp_get_params(const qsim_mlp *m, float *host);
qsim_status qsim_mlp_set_params(qsim_mlp *m, const float *host);
/* Logits of `rows` feature rows (host FP32 [rows][nfeat]) with the BF16
 * weights (bf16 = 1) or the FP32 master weights (bf16 = 0). */
qsim_status qsim_mlp_infer(qsim_mlp *m, const float *host_x, int rows, int bf16, float *host_logits);
/* Mean binary cross-entropy loss and its gradient with respect to every
 * parameter (host FP32, same layout as the parameter vector). */
qsim_status qsim_mlp_loss_grad(qsim_mlp *m, const float *host_x, const float *host_y, int rows,
                               float *loss, float *host_grad);
/* One Adam step on the device (forward, BCE loss, backward, update). */
qsim_status qsim_mlp_train_step(qsim_mlp *m, const float *host_x, const float *host_y, int rows,
                                float lr, float *loss);

/* ----------------------------------------------------------- misc */

/* Reason for the last error on this thread ("" if none). */
const char *qsim_last_error(void);

/* Library version string. */
const char *qsim_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QSIM_H */
