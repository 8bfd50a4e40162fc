/*
 * qc.h -- C ABI of a single-GPU (GB300, sm_103a) state-vector simulator for the
 * computation defined in QCLAB (Keip, Camps, Van Beeumen, "QCLAB: A Matlab Toolbox
 * for Quantum Computing", arXiv:2503.03016, 2025).
 *
 * Conventions used by every call (QCLAB Sec. 3.1, Sec. 3.2, Sec. 5.1):
 *   - A state on n qubits is 2^n complex amplitudes, interleaved (re, im), either
 *     complex64 (2 x float) or complex128 (2 x double), contiguous, in device memory.
 *   - Qubit 0 is the leftmost Kronecker factor: amplitude index
 *     i = sum_q b_q * 2^(n-1-q).  A bitstring's character j is qubit j, so '01' is
 *     index 1 (Sec. 3.1: simulate('00') equals simulate([1;0;0;0])).
 *   - A k-qubit gate U' on qubits (q_0, ..., q_{k-1}) acts as I_l (x) U' (x) I_r
 *     (Sec. 3.2); the row/column index of U' has q_0 as its most significant bit.
 *   - Gate matrices are passed from the host in FP64, row-major, as (re, im) pairs;
 *     complex64 states round them to FP32.
 *   - Complex128 arithmetic: the per-gate sweeps (qc_apply_1q, qc_apply_2q,
 *     qc_apply_ctrl and circuits run per gate), the fused circuit passes
 *     (QC_RUN_FUSED) and the adjoint gradient's forward and reverse passes on states
 *     of 2^14 amplitudes or more compute in double-float arithmetic: each binary64 value taken as a pair of
 *     binary32 numbers (48-bit significand) and every product and sum formed with
 *     error-free transformations on the FP32 pipe, about 2^-47 relative error per
 *     gate.  Magnitudes below 2^-74 keep 24 bits, below 2^-126 fewer (binary32
 *     subnormals) and below 2^-149 become zero; magnitudes of 2^128 or more (never
 *     those of a normalised state) overflow to infinity.  The adjoint's H psi and the
 *     per-thread sums of Z-string expectations use the same arithmetic (block and
 *     cross-block sums in FP64).  Smaller states, the other readouts (probabilities,
 *     sampling, X/Y-string expectations, collapse), the adjoint's energy and every
 *     other kernel compute in FP64.
 *
 * Errors: every call returns a qc_status.  Argument errors are reported before
 * anything is launched and leave the state untouched.  CUDA errors surface as
 * QC_ERR_CUDA at the call that observes them (asynchronous calls report launch
 * errors; synchronising calls also report execution errors).  qc_last_error()
 * returns a thread-local, human-readable message for the last failure of the
 * calling thread.  No C++ exception and no process exit ever crosses this ABI.
 *
 * Streams: each state carries a CUDA stream (default: the legacy default stream).
 * Calls are asynchronous on that stream unless documented as synchronising.
 *
 * Ownership: pointers passed in stay owned by the caller; the library owns only
 * what qc_state_alloc allocates (amplitudes) and the per-state scratch it creates
 * lazily, all released by qc_state_free.
 */
#ifndef QC_H_
#define QC_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QC_OK = 0,
  QC_ERR_INVALID_ARG = 1, /* bad qubit index, size, pointer, dtype, ...        */
  QC_ERR_OOM = 2,         /* device allocation failed                            */
  QC_ERR_CUDA = 3,        /* a CUDA runtime error (message in qc_last_error)     */
  QC_ERR_UNSUPPORTED = 4, /* valid request this build does not implement         */
  QC_ERR_ZERO_PROB = 5,   /* collapse onto an outcome of (numerically) zero prob.*/
  QC_ERR_TIMEOUT = 6      /* a bounded device wait ran out                       */
} qc_status;

typedef enum { QC_C64 = 0, QC_C128 = 1 } qc_dtype;

/* Arithmetic of fused k-qubit blocks (qc_apply_fused_k, qc_run_circuit). */
typedef enum {
  QC_PREC_NATIVE = 0, /* FMA in the state's own precision on the CUDA cores        */
  QC_PREC_TF32X3 = 1, /* complex64 only: tensor cores (tcgen05, kind::tf32), each
                         product split as a_hi*b_hi + a_hi*b_lo + a_lo*b_hi with
                         FP32 accumulation                                          */
  QC_PREC_BF16X3 = 2, /* the same split in BF16 (8-bit significands): rejected with
                         QC_ERR_UNSUPPORTED -- its products keep about 16 bits, too
                         few for 1e-5 relative L2 over a circuit's stages            */
  QC_PREC_AUTO = 3    /* qc_run_circuit, QC_RUN_FUSED: the faster of QC_PREC_NATIVE's
                         CUDA-core tile passes and QC_PREC_TF32X3's tensor-core stage
                         passes for the circuit's structure (complex64, n >= 12;
                         otherwise QC_PREC_NATIVE), chosen by timing both once      */
} qc_prec;

typedef struct qc_state qc_state; /* opaque */

/* Message describing the calling thread's last error ("" if none). */
const char* qc_last_error(void);
/* ABI version (incremented on incompatible changes). */
int qc_abi_version(void);
/* The status the tensor-core entry points (QC_PREC_TF32X3 blocks and passes) return for
 * the status word their kernels write: 0 -> QC_OK; 1 (a bounded wait for a copy or for
 * the products ran out: the kernel set the word, waited (bounded) for its copies and
 * products in flight, released its tensor memory and returned early) -> QC_ERR_TIMEOUT,
 * after which the state's amplitudes are undefined; anything else -> QC_ERR_CUDA.  Host
 * only; the message is set as by those entry points. */
qc_status qc_status_of_device_word(int word);
/* Number of CUDA kernels this library has launched in this process (all threads);
 * a diagnostic for benchmarks. */
uint64_t qc_launch_count(void);
/* Number of tile passes the planner used for the most recent QC_RUN_FUSED circuit or
 * fused adjoint reverse sweep (of the calling thread; a diagnostic for benchmarks). */
int qc_last_pass_count(void);
/* How the calling thread's most recent QC_RUN_FUSED circuit ran (a diagnostic): 0 one
 * sweep per gate (fewer than 10 qubits), 1 tile passes on the CUDA cores, 2 tile passes
 * whose stages ran as 32 x 32 blocks on the tensor cores (QC_PREC_TF32X3). */
int qc_last_fused_path(void);
/* Register stages (CUDA-core passes) or 32 x 32 stage blocks (tensor-core passes) of
 * the calling thread's most recent QC_RUN_FUSED circuit (a diagnostic). */
int qc_last_stage_count(void);
/* Plans circuit `c` as QC_RUN_FUSED would for a state of `dtype` and reports the number
 * of tile passes, register stages and tile ops; host only (no device work, no GPU
 * needed).  Circuits on fewer than 10 qubits report 0 (they run per gate). */
struct qc_circuit;
qc_status qc_plan_info(const struct qc_circuit* c, const double* params, qc_dtype dtype, int* passes,
                       int* stages, int* ops);
/* The box plan the tensor-core tile passes use to move a tile of 12 index bits
 * (`tile_bits`: 12 distinct bits below n, index bits 0..3 among them, any order) by
 * cp.async.bulk.tensor; host only.  Outputs (caller-owned): local_bits[12] = the tile's
 * bits in the local order of its boxes; dims[15] = per box dimension d = 0..4 its first
 * index bit, its number of bits and 1 if it is copied whole (0: one element at a time);
 * coords[5] = the number c of tile bits taken as box coordinates (the tile is 2^c boxes)
 * and for each its dimension and its bit within that dimension (-1 if unused).
 * QC_ERR_UNSUPPORTED: no plan with at most 2 coordinate bits (such a pass copies per
 * amplitude). */
qc_status qc_tc_box_plan(int n, const int* tile_bits, int* local_bits, int* dims, int* coords);
/* The tile and box plan of a dense block of k <= 5 qubits run as a one-stage
 * tensor-core tile pass (qc_apply_fused_k with QC_PREC_TF32X3): outputs as for
 * qc_tc_box_plan; QC_ERR_UNSUPPORTED: no tile of the block has a box plan (the block
 * then runs in the gathering block kernel).  Host only. */
qc_status qc_tc_block_plan(int n, const int* qubits, int k, int* local_bits, int* dims, int* coords);
/* Applies circuit `c` (12 <= c->n <= 26) to `state` (host, 2^n interleaved complex128
 * values, modified in place) the way the tensor-core tile passes would -- the same
 * passes, stage blocks (their FP64 products, not the TF32 split), deferred phase factors
 * (the FP32 tables the kernel reads), relabelings and copy passes -- on the host: a
 * check of the plan's logic, not of the arithmetic.  QC_ERR_UNSUPPORTED: the circuit does
 * not fit the tensor-core stages (QC_RUN_FUSED would take the CUDA-core passes). */
qc_status qc_tc_emulate(const struct qc_circuit* c, const double* params, double* state);
/* Applies circuit `c` (10 <= c->n <= 24) to `state` (host, 2^n interleaved complex128
 * values, modified in place) through the CUDA-core tile-pass plan QC_RUN_FUSED builds for
 * a state of `dtype` -- its passes, register stages, tile ops with their conditions,
 * matrices, phase tables, CZ code words and relabeled SWAPs -- interpreted on the host in
 * FP64 in the kernel's order: a check of the planner's logic.  Host only. */
qc_status qc_tile_emulate(const struct qc_circuit* c, const double* params, qc_dtype dtype, double* state);
/* The fused adjoint reverse sweep's plan for circuit `c` (12 <= c->n <= 24; its RX, RY,
 * RZ with a parameter are the recorded rotations) applied on the host in FP64 to `psi`
 * (the circuit's output state) and `lam` (H psi) -- both host, 2^n interleaved complex128,
 * modified in place -- with the sweep's record of each rotation, Im <lambda|G|psi> just
 * before it is undone, written to records[0 .. rotations) in circuit order: the plan the
 * gradient launches for a state of `dtype`, a check of its logic.  Host only. */
qc_status qc_adjoint_emulate(const struct qc_circuit* c, const double* params, qc_dtype dtype, double* psi,
                             double* lam, double* records, int nrec);
/* The tensor-core plan of circuit `c` (12 <= c->n <= 34): passes, stage blocks, deferred
 * phase factors and passes that are only a relabeling (copied by the CUDA-core pass);
 * host only.  QC_ERR_UNSUPPORTED: the circuit does not fit the tensor-core stages. */
qc_status qc_tc_plan_info(const struct qc_circuit* c, const double* params, int* passes, int* stages, int* factors,
                          int* copy_passes);

/* ---------------------------------------------------------------------------
 * State handles (QCLAB Sec. 3.1 "Initialization")
 * ------------------------------------------------------------------------- */

/* Allocates a 2^n-amplitude state on the current device; 1 <= n <= 34.  `stream`
 * is a cudaStream_t (NULL = legacy default stream).  The amplitudes are left
 * uninitialised; call one of the qc_state_init_* functions. */
qc_status qc_state_alloc(int n, qc_dtype dtype, void* stream, qc_state** out);

/* Wraps caller-owned device memory (e.g. a torch tensor) of 2^n amplitudes, at
 * least 16-byte aligned.  qc_state_free will not free it. */
qc_status qc_state_wrap(int n, qc_dtype dtype, void* dev_amps, void* stream, qc_state** out);

/* Releases the handle, its scratch and (if library-owned) its amplitudes.  NULL is
 * accepted.  Synchronises the state's stream first. */
qc_status qc_state_free(qc_state* s);

/* n, dtype and the device address of the amplitudes. */
qc_status qc_state_info(const qc_state* s, int* n, qc_dtype* dtype, void** dev_amps);

/* Replaces the stream subsequent calls on `s` use. */
qc_status qc_state_set_stream(qc_state* s, void* stream);

/* Basis state |index>, index per the convention above (Sec. 3.1: bitstring start). */
qc_status qc_state_init_basis(qc_state* s, uint64_t index);

/* Copies 2^n amplitudes of dtype `src_dtype` from `amps` (device memory, or host
 * memory if `src_on_host` is nonzero) into the state, converting precision
 * (Sec. 3.1: vector start).  The vector is not normalised. */
qc_status qc_state_init_vector(qc_state* s, const void* amps, qc_dtype src_dtype, int src_on_host);

/* Normalised complex Gaussian state generated on the device: amplitude j uses the
 * counter-based SplitMix64 stream (Steele, Lea, Flood, OOPSLA 2014) with uniforms
 * u1 = U(2j), u2 = U(2j+1), U(c) = (mix(seed + (c+1)*0x9E3779B97F4A7C15) >> 11) * 2^-53,
 * and the Box-Muller transform r = sqrt(-2 ln(1-u1)), (re, im) = r (cos, sin)(2 pi u2).
 * The norm is accumulated in FP64.  Complex128: transform and division by the norm in
 * FP64.  Complex64: transform in FP32 with 1-u1 formed exactly from the integer draw,
 * then multiplied by the FP64 reciprocal of the norm rounded once to FP32 (amplitudes
 * within ~1e-7 relative of the FP64 construction).  Synchronising. */
qc_status qc_state_init_gaussian(qc_state* s, uint64_t seed);

/* dst <- src (same n and dtype); used to branch on measurement outcomes. */
qc_status qc_state_copy(qc_state* dst, const qc_state* src);

/* Copies the amplitudes to host memory `host_dst` (2^n amplitudes of the state's
 * dtype).  Synchronising. */
qc_status qc_state_download(const qc_state* s, void* host_dst);

/* ---------------------------------------------------------------------------
 * Gate application (QCLAB Sec. 3.2: U = I_l (x) U' (x) I_r applied to the state)
 * ------------------------------------------------------------------------- */

/* U' = U (2x2, 8 doubles) on qubit q. */
qc_status qc_apply_1q(qc_state* s, int q, const double U[8]);

/* U' = U (4x4, 32 doubles) on (qa, qb), row index 2*b_qa + b_qb; qa != qb, either
 * order. */
qc_status qc_apply_2q(qc_state* s, int qa, int qb, const double U[32]);

/* U (2x2) on `target`, applied only where control j reads ctrl_states[j] (0 or 1;
 * NULL = all 1).  Covers CNOT/CZ (Sec. 2, Sec. 5.3) and MCX with open controls
 * (Sec. 5.4).  0 <= nctrl <= 6; all qubits distinct. */
qc_status qc_apply_ctrl(qc_state* s, const int* ctrls, const int* ctrl_states, int nctrl, int target,
                        const double U[8]);

/* A dense 2^k x 2^k block on qubits[0..k-1] (qubits[0] = MSB of the block index),
 * 1 <= k <= 7 (QC_PREC_TF32X3: 2 <= k <= 6, complex64, n >= k_eff + 7 where k_eff = 5
 * for k <= 5 (padded with identity qubits) and 6 for k = 6; a block of k <= 5 runs as a
 * one-stage tensor-core tile pass where its tile moves as at most four boxes, else as a
 * gathering block kernel).  The product of consecutive gates that act on at most k
 * qubits (gate fusion). */
qc_status qc_apply_fused_k(qc_state* s, const int* qubits, int k, const double* U, qc_prec prec);

/* ---------------------------------------------------------------------------
 * Measurement, probabilities, sampling (QCLAB Sec. 3.3)
 * ------------------------------------------------------------------------- */

/* Measures qubit q in the Z basis: P(o) = sum over indices whose bit for q is o of
 * |psi_i|^2, summed in FP64 (complex64: each |psi_i|^2 formed in FP32).  With
 * T = P(0) + P(1), the outcome is 1 iff u*T >= P(0) (u in [0,1), supplied by the
 * caller).  The state is collapsed onto the outcome and renormalised: the kept
 * amplitudes are multiplied by 1/sqrt(P(outcome)), formed once in FP64 (complex64:
 * rounded once to FP32), which is within one rounding of dividing by sqrt(P(outcome));
 * the others are set to zero.  Returns the outcome and P(outcome)/T.  Synchronising. */
qc_status qc_measure(qc_state* s, int q, double u, int* outcome, double* prob);

/* Forced branch: collapses onto `outcome` and renormalises, returning its
 * probability P(outcome)/T; QC_ERR_ZERO_PROB (state untouched) if that probability
 * is <= 1e-12 (complex128) or <= 1e-6 (complex64).  Synchronising. */
qc_status qc_collapse(qc_state* s, int q, int outcome, double* prob);

/* Collapse with a caller-supplied normaliser, for a register split into shards over
 * several processes (each process holds one shard as a state; the outcome probability
 * of Sec. 3.3 is then the sum of the shards' sums): keeps the amplitudes whose qubit q
 * reads `outcome` (q = -1: every amplitude) and multiplies them by 1/sqrt(p), formed
 * once in FP64 as in qc_collapse; the others are set to zero; p = 0 sets the whole
 * state to zero.  n >= 1.  Asynchronous. */
qc_status qc_collapse_norm(qc_state* s, int q, int outcome, double p);

/* <a|b> = sum_i conj(a_i) b_i (same n and dtype; both on a's stream): host_out[0] =
 * real part, host_out[1] = imaginary part; each product at the states' precision, the
 * sums in FP64 (fixed order).  The inner product Sec. 5.2's expectations reduce to.
 * Synchronising. */
qc_status qc_inner(const qc_state* a, const qc_state* b, double* host_out);

/* P(outcome) for qubit q without collapsing (host scalar, synchronising). */
qc_status qc_outcome_prob(const qc_state* s, int q, int outcome, double* prob);

/* dev_out[i] = re_i*re_i + im_i*im_i in FP64 (two rounded products, one rounded
 * sum; complex64 amplitudes are widened exactly first).  2^n doubles. */
qc_status qc_probs(const qc_state* s, double* dev_out);

/* Draws `shots` outcomes: with cdf_k the FP64 number nearest the exact prefix sum of
 * the p_i above and T = cdf_{N-1}, dev_out[s] = min{k : dev_u[s]*T < cdf_k} for
 * caller-supplied uniforms dev_u in [0,1) (device memory).  Bit-exact given the
 * same p_i and uniforms. */
qc_status qc_sample(const qc_state* s, const double* dev_u, int64_t shots, uint64_t* dev_out);

/* The same rule as qc_sample applied to a caller-supplied probability vector dev_p
 * (device, 2^n nonnegative doubles, 16-byte aligned, sum below 2^10), e.g. a marginal
 * distribution.  `s` supplies the stream and scratch; its amplitudes are not read. */
qc_status qc_sample_probs(qc_state* s, const double* dev_p, int n, const double* dev_u, int64_t shots,
                          uint64_t* dev_out);

/* QCLAB's reducedStatevector (Sec. 5.1): the 2^(n-m) amplitudes whose `known` qubits
 * (m distinct qubits) carry `bits` (0/1 each), in the order of the remaining qubits
 * (the last remaining qubit is the least significant).  dev_out: device memory of the
 * state's dtype, 16-byte aligned.  A gather, not renormalised.  0 <= m < n. */
qc_status qc_reduced_state(const qc_state* s, const int* known, const int* bits, int m, void* dev_out);

/* Marginal outcome distribution of measuring `qubits` (1 <= m <= 12, distinct):
 * dev_out[x] = sum of p_i over indices whose measured qubits read x, with qubits[0] the
 * most significant bit of x (Sec. 3.3's P(o) generalised to m qubits; with
 * qc_sample_probs it gives counts(shots) of Sec. 5.2 for partial measurements).
 * FP64; block partial histograms use FP64 shared-memory atomics, so the last bits
 * may vary between runs. */
qc_status qc_marginal_probs(const qc_state* s, const int* qubits, int m, double* dev_out);

/* host_out[t] = coeffs[t] * <psi| P_t |psi> for Pauli strings P_t of n characters
 * in {I,X,Y,Z}, character j acting on qubit j (coeffs NULL = all 1).  Reductions in
 * FP64.  Synchronising.  (Sec. 5.2 builds a density-matrix estimate from such
 * expectations.) */
qc_status qc_expect_pauli(const qc_state* s, const char* const* strings, const double* coeffs, int nterms,
                          double* host_out);

/* Allocation-free form of qc_expect_pauli (the paper has no counterpart: it is an
 * interface for callers that cannot allocate device memory while they run, e.g. a
 * process whose device memory is wholly reserved by another allocator, or a service
 * that must not meet an allocation failure or the synchronisation cudaMalloc/cudaFree
 * can cause).  Same arguments and results as qc_expect_pauli, but every intermediate
 * lives in one fixed array in the library's device image: 157,696 bytes (1216 blocks
 * x 16 partial sums + 256 term values), held on every device that loads the library
 * until the process exits.  Limits: at most 256 terms per call (more is rejected with
 * QC_ERR_INVALID_ARG and a message); the reduction grid is capped at 1216 blocks
 * (608 blocks x 32 partial sums for the Z-only strings, in the same array).
 * Every call looks up the array's device address (cudaGetSymbolAddress, which
 * allocates nothing) with the state's device current, so the address stays valid
 * after a device reset; the first call on a device may load the library's device
 * code there, so make that first call before any stream capture.  All calls share
 * the array and it keeps the last call's contents:
 * calls whose work overlaps on the GPU (other threads, other streams) race and must
 * be serialised by the caller.  Calls no cudaMalloc/cudaFree.  Synchronising. */
qc_status qc_expect_pauli_noalloc(const qc_state* s, const char* const* strings, const double* coeffs, int nterms,
                                  double* host_out);

/* ---------------------------------------------------------------------------
 * Circuits (QCLAB Sec. 2: QCircuit / push_back; nested circuits are flattened by
 * the caller)
 * ------------------------------------------------------------------------- */

#define QC_MAX_OP_QUBITS 8

typedef enum {
  QC_GATE_MATRIX1 = 0,      /* dense 2x2 at pool[matrix], qubits[0]                  */
  QC_GATE_MATRIX2 = 1,      /* dense 4x4 at pool[matrix], (qubits[0], qubits[1])      */
  QC_GATE_H = 2,
  QC_GATE_X = 3,
  QC_GATE_Y = 4,
  QC_GATE_Z = 5,
  QC_GATE_S = 6,
  QC_GATE_SDG = 7,
  QC_GATE_T = 8,
  QC_GATE_TDG = 9,
  QC_GATE_RX = 10,          /* exp(-i t X/2)                                          */
  QC_GATE_RY = 11,          /* exp(-i t Y/2)                                          */
  QC_GATE_RZ = 12,          /* exp(-i t Z/2) = diag(e^{-it/2}, e^{it/2})              */
  QC_GATE_U3 = 13,          /* OpenQASM U3(theta, phi, lambda)                        */
  QC_GATE_CNOT = 14,        /* qubits = (control, target)                             */
  QC_GATE_CZ = 15,          /* qubits = (a, b)                                        */
  QC_GATE_CP = 16,          /* diag(1,1,1,e^{i phi}) on (a, b)                        */
  QC_GATE_SWAP = 17,
  QC_GATE_MCX = 18,         /* qubits = (controls..., target), ctrl_states            */
  QC_GATE_CTRL_MATRIX1 = 19 /* controlled dense 2x2 at pool[matrix]                   */
} qc_gate_kind;

typedef struct qc_op {
  int32_t kind;                        /* qc_gate_kind                                  */
  int32_t nq;                          /* entries used in qubits[]                      */
  int32_t qubits[QC_MAX_OP_QUBITS];    /* controlled kinds: controls first, target last */
  uint32_t ctrl_states;                /* bit j = required value of control j (MCX,
                                          CTRL_MATRIX1); CNOT/CZ/CP use 1              */
  int32_t param;                       /* >= 0: angles from params[param ...]; -1: angle[] */
  int32_t adjoint;                     /* nonzero: apply U^dagger                        */
  int32_t reserved;
  double angle[3];
  int64_t matrix;                      /* offset in doubles into pool, or -1             */
} qc_op;

typedef struct qc_circuit {
  int32_t n;
  int32_t nops;
  const qc_op* ops;   /* host memory */
  const double* pool; /* host FP64 (re,im) row-major matrices referenced by ops */
  int64_t pool_len;   /* doubles in pool */
} qc_circuit;

typedef enum {
  QC_RUN_PER_GATE = 0, /* one full sweep per gate: the paper's plain method (Sec. 3.2) */
  QC_RUN_FUSED = 1     /* planner: gates grouped into shared-memory tile passes and
                          fused k-qubit blocks; same result up to rounding            */
} qc_run_mode;

/* Applies every op of `c` (c->n must equal the state's n) in order.  `params`
 * (host, may be NULL if no op uses it) supplies angles for ops with param >= 0.
 * `prec` selects the arithmetic of fused blocks in QC_RUN_FUSED: with QC_PREC_TF32X3 and a
 * complex64 state of n >= 12 qubits, the tile passes (2^12 amplitudes) run each stage --
 * the ops on 5 of the tile's bits, controls and phase bits included -- as one 32 x 32
 * block on the tensor cores (host FP64 product of the stage's gates; TF32 split with
 * round-to-nearest, the large and the small products in two FP32 accumulators added on
 * the CUDA cores; synchronising: a bounded-wait timeout returns QC_ERR_TIMEOUT, after
 * which the state's amplitudes are undefined).  Every control of an op is a slot of its
 * stage; a phase op conditioned on at most one qubit may have phase bits elsewhere (that
 * part is applied per output after the stage's product), and exact SWAPs may be taken as
 * a relabeling of the tile.  A circuit that does not fit these stages runs on the
 * CUDA-core passes.  With QC_PREC_AUTO the first run of a
 * circuit structure (gate kinds, qubits and controls; not the angles or matrices) on a
 * device times both kinds of pass on a scratch state of the same size (allocated and
 * freed by the call; if that allocation fails, the tensor-core passes are taken) and
 * keeps the faster for later runs; with the environment variable QC_AUTOTUNE_CACHE
 * naming a file, choices are appended to it and read back by later processes.  Host
 * planning: the tensor-core plan of the last circuit run is kept (with its device copy,
 * library-owned) and reused while the circuit and its values are unchanged; the stage
 * cuts and plan variants found for a circuit structure are kept process-wide (the 512
 * most recent of each, under a lock), so the same structure with new values re-plans in
 * milliseconds; the plan is built in memory the calling thread keeps for its next plan. */
qc_status qc_run_circuit(qc_state* s, const qc_circuit* c, const double* params, qc_run_mode mode,
                         qc_prec prec);

/* ---------------------------------------------------------------------------
 * Batched circuits and adjoint gradients (parameterised ansatz circuits)
 * ------------------------------------------------------------------------- */

/* One term coeff * P of a Pauli sum on the index bits: bit b of xmask / zmask acts on
 * qubit n-1-b as X (xmask only), Z (zmask only) or Y (both), i.e.
 * P = i^{|xmask & zmask|} X^xmask Z^zmask and P|j> = i^{|x & z|} (-1)^{|j & z|} |j ^ x>
 * (the Pauli decomposition behind Sec. 5.2's density-matrix estimate). */
typedef struct qc_pauli_term {
  uint64_t xmask;
  uint64_t zmask;
  double coeff;
} qc_pauli_term;

/* H = sum_t terms[t] (host memory). */
typedef struct qc_hamiltonian {
  int32_t nterms;
  int32_t reserved;
  const qc_pauli_term* terms;
} qc_hamiltonian;

/* Adjoint (reverse-sweep) gradient of E(theta) = <psi(theta)| H |psi(theta)>,
 * psi(theta) = U_L ... U_1 |0...0>, H = sum_t coeffs[t] P_t (Pauli strings as in
 * qc_expect_pauli).  Parameterised ops must be RX/RY/RZ with param >= 0 (each
 * U = exp(-i t G/2)); dE/dt_l = Im <lambda_l| G_l |psi_l> summed over the ops that use
 * parameter l, with psi_l the state after op l and lambda_l = U_{l+1}^dag ... U_L^dag H psi.
 * `params` (host, nparams doubles).  Writes *host_energy and host_grad[nparams].
 * Uses two state buffers of c->n qubits in `dtype` (library workspace, kept between
 * calls).  With n >= 12 (both dtypes): the reverse sweep runs as tile passes over psi and
 * lambda together (a recorded rotation's share is added before it is undone);
 * otherwise one kernel per rotation.  Sums in FP64, fixed order (bitwise repeatable).
 * The two state buffers, the reduction partials and the plan buffers are one
 * process-wide workspace owned by the library (grown when a larger register needs it,
 * kept until the process exits); calls are serialised by the library, and a call on
 * another stream waits (on the device) for the previous call's kernels.
 * Synchronising. */
qc_status qc_adjoint_grad(const qc_circuit* c, const double* params, int nparams, const char* const* strings,
                          const double* coeffs, int nterms, qc_dtype dtype, void* stream, double* host_energy,
                          double* host_grad);

/* Device-pointer form of qc_adjoint_grad for training loops on one stream: the angles
 * in device memory (`dev_params`, nparams FP64), H as mask terms (qc_hamiltonian, host),
 * the energy (one FP64) and the gradient (nparams FP64) written to device memory on
 * `stream`.  The gate plan is built on the host from the angle values, so the call
 * copies dev_params to the host on `stream` and waits for that copy; every step after
 * it, the outputs included, is queued on `stream` without a host round trip (the
 * outputs are valid once `stream` reaches them).  Same workspace, serialisation and
 * arithmetic as qc_adjoint_grad. */
qc_status qc_adjoint_grad_dev(const qc_circuit* c, const double* dev_params, int nparams, const qc_hamiltonian* H,
                              qc_dtype dtype, void* stream, double* dev_energy, double* dev_grad);

/* A batch of independent circuits of uneven qubit counts (QCLAB Sec. 2 circuits,
 * Sec. 3.2 applied to each one's own register from |0...0>), evaluated in one
 * persistent launch, complex64 state, FP32 gate arithmetic.
 *   circuits[b]     : any gate kinds, 1 <= n <= 20 qubits, host memory.
 *   dev_params      : device FP64 angles; an op of circuit b with param p >= 0 (RX, RY,
 *                     RZ, CP: one angle; U3: three) reads dev_params[param_offset[b] + p
 *                     ...]; its matrix is formed on the device in FP64 and rounded to
 *                     FP32.  NULL if no op is parameterised.  param_offset NULL = 0.
 *   observables     : host; one qc_hamiltonian per circuit, or one for all when
 *                     shared_observable is nonzero; dev_out[b] = <psi_b| H_b |psi_b>
 *                     (per-amplitude products in FP32, sums in FP64 over groups of 16
 *                     amplitudes).  NULL: no values (dev_out may be NULL).
 *   dev_states      : host array of `count` device pointers, each to 2^n[b] complex64
 *                     amplitudes (16-byte aligned) that receive circuit b's final state;
 *                     NULL entries or a NULL array: not stored.
 * Circuits of at most 13 qubits live in shared memory for their whole run; larger ones
 * in a device workspace (or in their dev_states buffer), one sweep per gate by one
 * block.  When every circuit is the layered RY.RZ + CZ-chain ansatz (parameter index
 * layer*2n + 2q + {0: RY, 1: RZ}, n >= 6) and every observable is sum_i Z_i Z_{i+1} of
 * the chain with unit coefficients, the batch runs on the ansatz kernel below instead
 * (angles rounded to FP32 first).  Asynchronous on `stream`; the tables are uploaded
 * from host memory during the call.  Calls are serialised by the library (one
 * process-wide workspace). */
typedef struct qc_batch {
  int32_t count;
  int32_t shared_observable;
  const qc_circuit* circuits;
  const int64_t* param_offset;
  const double* dev_params;
  int64_t nparams;
  const qc_hamiltonian* observables;
  void* const* dev_states;
} qc_batch;

qc_status qc_run_batch(const qc_batch* b, void* stream, double* dev_out);
/* Which kernel the calling thread's most recent qc_run_batch used (a diagnostic):
 * 0 the general batch kernel, 1 the ansatz kernel. */
int qc_last_batch_path(void);

/* The layered ansatz as its own batch entry point (the fast path qc_run_batch picks):
 * circuit b has n[b] qubits (6 <= n <= 20) and runs `layers` layers of [RY(t) then
 * RZ(t) on every qubit, then CZ(i, i+1), i = 0..n-2], parameter index
 * layer*2n + 2q + {0: RY, 1: RZ}, from |0...0>, reading FP32 angles from
 * dev_params + param_offset[b] (device memory).  dev_out[b] =
 * <psi_b| sum_{i<n-1} Z_i Z_{i+1} |psi_b>, accumulated in FP64.  One persistent launch,
 * recorded once in a CUDA graph and replayed; its launch shape is chosen by timing. */
typedef struct qc_ansatz_batch {
  int32_t count;                /* number of circuits                                */
  int32_t layers;
  const int32_t* n;             /* host: qubit count per circuit                     */
  const int64_t* param_offset;  /* host: offset of circuit b's parameters            */
  const float* dev_params;      /* device: all parameters (FP32 angles)              */
  int64_t nparams;              /* total number of parameters                        */
} qc_ansatz_batch;

qc_status qc_run_ansatz_batch(const qc_ansatz_batch* b, void* stream, double* dev_out);
/* Fusion width (register-stage bits, 4 or 5) the autotuner chose for the most recent
 * ansatz batch (diagnostic). */
int qc_batch_fusion_width(void);

#ifdef __cplusplus
}
#endif

#endif /* QC_H_ */
