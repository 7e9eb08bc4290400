/*
 * soft.h -- C ABI of the GB300 generalized-stabilizer (GS) shot simulator.
 *
 * The library runs many independent noisy shots of one Clifford+T circuit.
 * Every shot keeps a GS state |phi> = sum_a v_a d_a |psi_S> (arxiv
 * 2512.23037, Sec. II-C, Definition "Generalized stabilizer representation"):
 * a stabilizer/destabilizer tableau plus a sparse map of complex
 * coefficients v. Clifford gates conjugate the tableau (Theorem 1 (1));
 * T / T^dagger / Rz act as a I + b Z_q on the map through the Pauli-on-basis
 * identity (Eq. T_gate, Eq. pauli_on_basis, Theorem 1 (3)); Z measurements
 * filter or pair the map and replace tableau rows (Theorem 1 (2)); noise is
 * sampled Paulis applied through the same identity (Sec. II-C, "Pure-state
 * simulation model"; uniform depolarizing model of Sec. III). The shot-parallel
 * device design replaces the staged per-op kernel pipeline of Sec. IV-B with
 * one persistent kernel per launch.
 *
 * Conventions shared by every call:
 *   - Return value: SOFT_OK (0) or a negative SOFT_E_* code. On error,
 *     soft_last_error() returns a message for the calling thread.
 *   - All host pointers are owned by the caller and only read/written during
 *     the call (soft_run_shots may read `ops` nowhere: it uses the compiled
 *     circuit). Device pointers passed in soft_run_opts stay owned by the
 *     caller and must outlive the run's stream work.
 *   - Handles are owned by the library; free them with the matching *_free.
 *     One handle must not be used from two threads at once.
 *   - Results depend only on (circuit, noise, seed, shot index): splitting a
 *     shot range over calls or GPUs does not change them.
 */
#ifndef SOFT_ABI_H_
#define SOFT_ABI_H_
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
enum {
  SOFT_OK = 0,
  SOFT_E_ARG = -1,             /* bad argument (null pointer, size, noise value, cap) */
  SOFT_E_QUBIT_RANGE = -2,     /* qubit index >= n_qubits, equal qubits of a 2-qubit gate, n_qubits > 128 */
  SOFT_E_RECORD_REF = -3,      /* record index not yet measured */
  SOFT_E_UNSUPPORTED_OP = -4,  /* unknown op code or unsupported noise (p_idle != 0) */
  SOFT_E_OOM = -5,             /* host or device allocation failed */
  SOFT_E_CUDA = -6,            /* a CUDA runtime call failed */
  SOFT_E_DEVICE_TIMEOUT = -7   /* reserved: a device-side bound was hit (never traps) */
};

/* Per-shot status byte. */
enum { SOFT_SHOT_KEPT = 0, SOFT_SHOT_DISCARDED = 1, SOFT_SHOT_OVERFLOW = 2, SOFT_SHOT_ERROR = 3 };

/* ---------------------------------------------------------------- circuit format */
/* Op codes. Clifford gates (Sec. II-A generating set plus CZ, S^dag, Paulis),
 * T / T^dag (Eq. T_gate / T_dagger, with the global phase kept so that
 * T = diag(1, e^{i pi/4}) exactly), RZ(angle) = cos(angle/2) I - i sin(angle/2) Z,
 * Z-basis M / R (measure, then X if -1) / MR, CPAULI (Pauli flags&3 = 1 X,
 * 2 Y, 3 Z on q0 applied when the parity of rec[0], rec[1] is 1),
 * DETECTOR (parity of rec[] xor INVERT = 1 => shot discarded, the early
 * discard of Sec. V-C), OBSERVABLE (parity = 1 => logical error flag),
 * NOISELESS_BEGIN/END (ops in between carry no noise), MPP (a factor pair of
 * a Pauli-product measurement, the general Pauli measurement of Theorem 1 (2);
 * see SOFT_MPP_MORE). */
enum {
  SOFT_H = 0, SOFT_S = 1, SOFT_S_DAG = 2, SOFT_X = 3, SOFT_Y = 4, SOFT_Z = 5, SOFT_CX = 6, SOFT_CZ = 7,
  SOFT_T = 8, SOFT_T_DAG = 9, SOFT_RZ = 10, SOFT_M = 11, SOFT_R = 12, SOFT_MR = 13, SOFT_CPAULI = 14,
  SOFT_DETECTOR = 15, SOFT_OBSERVABLE = 16, SOFT_NOISELESS_BEGIN = 17, SOFT_NOISELESS_END = 18, SOFT_MPP = 19
};
/* DETECTOR / OBSERVABLE flags: INVERT xors 1 into the parity; CHAIN carries
 * the parity into the next DETECTOR / OBSERVABLE instead of testing it. */
enum { SOFT_FLAG_INVERT = 1, SOFT_FLAG_CHAIN = 2 };
/* MPP flags: bits 0-1 = Pauli on q0 (1 X, 2 Y, 3 Z, never 0), bits 2-3 =
 * Pauli on q1 (0: no second factor), SOFT_MPP_MORE = the product continues in
 * the next op, which must be an MPP. The chain's last op measures the product
 * of all its factors (distinct qubits) and appends one record. With p_meas > 0
 * a flip precedes the chain: the Pauli on its first qubit that anticommutes
 * with the first factor (Z for X; X for Y and Z). Before M/MR the flip is X,
 * and after R/MR an X with p_reset. */
enum { SOFT_MPP_MORE = 16 };

/* 32-byte op record. q1 only for CX (control q0, target q1) and CZ. rec[] are
 * absolute record indices (0 = first M/MR of the circuit), -1 = unused. */
typedef struct {
  uint16_t op;
  uint16_t flags;
  uint32_t q0, q1;
  uint32_t pad;
  double angle;
  int32_t rec[2];
} soft_op;

/* Uniform depolarizing noise (Sec. III): DEPOL1(p1) after every 1-qubit gate
 * (T, T^dag, RZ included), DEPOL2(p2) after every CX/CZ (one of the 15
 * non-identity two-qubit Paulis), X flip with p_meas before every M/MR and
 * with p_reset after every R/MR. p_idle must be 0 (no idle layers). */
typedef struct {
  double p1, p2, p_meas, p_reset, p_idle;
} soft_noise;

typedef struct soft_circuit soft_circuit;
typedef struct soft_run soft_run;

typedef struct {
  uint32_t n_qubits;
  uint32_t n_records;     /* M and MR ops */
  uint32_t record_words;  /* ceil(n_records / 64), at least 1 */
  uint32_t n_sites;       /* noise sites after expansion */
  uint32_t n_events;      /* per-shot device program length */
  uint32_t coeff_cap;
  uint64_t program_bytes; /* device bytes of the compiled program */
} soft_circuit_info_t;

/* Validate the op list, expand the noise model into numbered noise sites,
 * evolve the shot-invariant X/Z part of the tableau once on the host and
 * upload the per-shot device program to the current CUDA device.
 *   ops: n_ops records (host); n_qubits in 1..128; noise: host struct;
 *   coeff_cap: largest |v| a shot may hold (power of two not required,
 *   1..65536); a shot whose |v| exceeds it after pruning ends as OVERFLOW
 *   (the overflow mark of Sec. IV-B, "Memory layout").
 *   out: receives a handle freed with soft_circuit_free.
 * Errors: SOFT_E_ARG, SOFT_E_QUBIT_RANGE, SOFT_E_RECORD_REF,
 * SOFT_E_UNSUPPORTED_OP, SOFT_E_OOM, SOFT_E_CUDA; *out is NULL then. */
int soft_compile_circuit(const soft_op *ops, size_t n_ops, uint32_t n_qubits, const soft_noise *noise,
                         uint32_t coeff_cap, soft_circuit **out);

int soft_circuit_info(const soft_circuit *c, soft_circuit_info_t *out);

/* Final X/Z words of the shot-invariant tableau (rows d_0..d_{n-1} then
 * s_0..s_{n-1}, 2 words per row each; host buffers of 4*n words). With the
 * per-shot sign words of soft_get_state this gives the full tableau. */
int soft_circuit_tableau(const soft_circuit *c, uint64_t *rows_x, uint64_t *rows_z);

void soft_circuit_free(soft_circuit *c);

/* ---------------------------------------------------------------- runs */
enum { SOFT_FP64 = 0, SOFT_FP32 = 1 };
enum { SOFT_REC_NONE = 0, SOFT_REC_FIRST_K = 1, SOFT_REC_ALL = 2 };

typedef struct {
  int32_t precision;     /* SOFT_FP64 (coefficients complex128) or SOFT_FP32 (complex64;
                            probabilities and tallies stay FP64) */
  int32_t record_mode;   /* which shots' records and status bytes are kept */
  uint64_t record_k;     /* K for SOFT_REC_FIRST_K */
  void *stream;          /* cudaStream_t to launch on; NULL = legacy default stream */
  uint32_t group_size;   /* lanes per shot: 0 = 32, else 16 (two shots per warp) or 32 */
  uint32_t blocks_per_sm;/* 0 = as many as fit */
  uint64_t chunk_shots;  /* shots per launch; 0 = auto */
  uint32_t first_cap;    /* capacity of the first pass (0 = auto); shots that exceed
                            it and not coeff_cap are rerun at coeff_cap */
  uint32_t capture_k;    /* keep the final GS state of the first capture_k shots */
  uint64_t *d_records;   /* optional caller device buffer, record_words per kept shot */
  uint8_t *d_status;     /* optional caller device buffer, one byte per kept shot */
  uint32_t groups_per_block; /* shots resident per 128-thread block: 0 = 128 / group lanes,
                                else 1..that number */
  uint32_t flags;        /* SOFT_RUN_GRAPH: capture one chunk (counter reset, both passes,
                            device-side advance of the chunk base) in a CUDA graph and
                            replay it for every full chunk; needs a non-NULL stream */
} soft_run_opts;
/* SOFT_RUN_FIDELITY: every measurement whose record an OBSERVABLE reads is
 * projected onto +1 instead of sampled, and each kept shot adds F, the
 * product of those measurements' conditional probabilities of +1, to the
 * tally's sum_fidelity (F = |<0..0|phi>|^2 on the observed qubits, the exact
 * fidelity of the final chain of Sec. V; E[1 - F | kept] is the sampled
 * logical-error rate, estimated with lower variance). A shot for which +1 is
 * impossible ends there, kept, with F = 0. Observed records then read 0.
 * Needs every DETECTOR before the first observed measurement (SOFT_E_ARG
 * otherwise). */
/* SOFT_RUN_NO_PREFIX: run every shot from the first event. By default a shot
 * starts at the event that applies its first error (or at the end of the
 * circuit's decided noiseless prefix, if earlier), from the state the noiseless
 * run reached there: soft_compile_circuit records that run once per precision
 * (the state at the top of each event, while every outcome is decided and the
 * map has at most 64 entries; with SOFT_RUN_FIDELITY, only up to the first
 * observed measurement). Both give the same results; the flag is for
 * comparison. */
/* Lane-per-shot scheduling (the default where it applies): one shot per lane,
 * 32 shots per warp. Shots are bucketed by the event they start at, and each
 * warp executes one event at a time for all its lanes, each lane updating its
 * own shot's map (up to 16 entries, whose keys a lane keeps as an affine space
 * of at most 4 directions). A shot whose map outgrows its lane is
 * handed over at that event (its whole state in a spill record): to the wide
 * round's lanes (see below), or to a warp with a register map of up to
 * first_cap entries (default 64); shots beyond that rerun from their start at
 * the circuit's cap. A warp left with few active lanes moves their shots to a
 * second round that packs them into full warps again. In a
 * batch each circuit has its own buckets, and a warp serves one circuit at a
 * time. It applies to runs without a forced group size (state capture
 * included: a captured shot's state is written wherever it ends), to
 * the circuits whose noiseless run's maps fit a lane, when those circuits hold
 * at most 50 000 events (plus one per circuit) together; otherwise a warp
 * (group) runs each shot. A circuit whose noiseless maps need more than 16
 * entries or 4 directions gets lanes of 32 entries (5 directions) or, with
 * SOFT_FP32 coefficients, of 64 (6 directions): these neither hand over nor
 * evict, and a shot that outgrows one reruns from its start in a warp. The
 * shots of a batch's other circuits go straight to the warp pass.
 * SOFT_RUN_NO_LANES always uses the warp per shot. Same results either way,
 * another order. */
/* SOFT_RUN_TIME_PASSES records CUDA events between the passes of every chunk
 * (ignored with SOFT_RUN_GRAPH), read back by soft_run_pass_timing. */
/* The wide round (single-circuit runs; batches never use it): shots whose map
 * outgrows a lane continue in lanes of twice the map before any warp. By
 * default it runs for chunks of at least 2^23 shots; SOFT_RUN_WIDE_LANES runs
 * it for any chunk, SOFT_RUN_NO_WIDE_LANES never.
 * Same results either way. */
enum { SOFT_RUN_GRAPH = 1, SOFT_RUN_FIDELITY = 2, SOFT_RUN_NO_PREFIX = 4, SOFT_RUN_NO_LANES = 8,
       SOFT_RUN_TIME_PASSES = 16, SOFT_RUN_NO_WIDE_LANES = 32, SOFT_RUN_WIDE_LANES = 64 };

/* Launch shots [first_shot, first_shot + n_shots) of a compiled circuit,
 * asynchronously on opts->stream: the paper's shot-parallel simulation
 * (Sec. IV-B: many independent noisy shots, each evolved in the GS
 * representation of Sec. II-C by the update rules of Theorem 1, with
 * overflow marked when |v| exceeds the cap). Philox4x32-10 keyed by `seed` drives all
 * randomness: noise gaps on counter (shot, 0, k), measurement uniforms on
 * counter (shot, 1, ordinal).
 *   opts may be NULL (FP64, no records, auto tuning, default stream).
 *   out: receives a run handle (freed with soft_run_free) that owns the
 *   device tallies and, unless caller buffers are given, the record/status
 *   buffers. All device buffers a run owns sit in one workspace, borrowed from
 *   the device's cached workspace when that is idle and large enough; at
 *   soft_run_free it goes back to the cache (the larger one is kept), so
 *   repeated runs allocate no device memory. soft_release_workspace frees the
 *   cache.
 * Errors: SOFT_E_ARG, SOFT_E_OOM, SOFT_E_CUDA. */
int soft_run_shots(soft_circuit *c, uint64_t n_shots, uint64_t first_shot, uint64_t seed, const soft_run_opts *opts,
                   soft_run **out);

typedef struct {
  uint64_t shots, discarded, overflow, kept, logical_errors;
  double sum_fidelity, sum_weight; /* SOFT_RUN_FIDELITY: sum of F over kept shots, and kept; else 0 */
} soft_tally_t;

/* Batched form of soft_run_shots (Sec. IV-B's shot-parallel execution, over
 * several circuits at once; Sec. V-C measures throughput against the batch
 * size). One persistent launch sequence over up to 64 compiled circuits (shots and
 * circuits whose coefficient caps differ share the kernel; a shot's overflow
 * threshold is its own circuit's cap). Circuit i runs shots
 * [first_shots[i], first_shots[i] + n_shots[i]). All circuits must be on one
 * device and all have n <= 64 qubits or all n > 64. Records and state capture
 * are not available for batches (record_mode must be NONE, capture_k 0).
 * Results per shot are identical to soft_run_shots of that circuit alone.
 * Errors: SOFT_E_ARG, SOFT_E_OOM, SOFT_E_CUDA. */
int soft_run_batch(soft_circuit *const *circs, const uint64_t *n_shots, const uint64_t *first_shots, uint32_t n_circ,
                   uint64_t seed, const soft_run_opts *opts, soft_run **out);

/* Wait for the run's stream work and copy its tallies (Sec. V-A fields:
 * total, discarded, kept shots and detected logical errors), summed over
 * the circuits of a batch. */
int soft_tally(soft_run *r, soft_tally_t *out);

/* Tally of circuit `index` of a batch run (index 0 for soft_run_shots). */
int soft_tally_batch(soft_run *r, uint32_t index, soft_tally_t *out);

/* The measurement record of each shot (the outcomes the post-selection and
 * logical-error statistics of Sec. V-A are computed from; Sec. IV-B keeps it
 * per shot). Wait, then copy records (shot-major, record_words per shot, bit j = 1 when
 * record j measured -1; bits after a discard are 0) and status bytes of the
 * kept shots (the first K, or all). n_words / n_status give the host buffer
 * sizes; either pointer may be NULL. */
int soft_get_records(soft_run *r, uint64_t *host_words, size_t n_words, uint8_t *host_status, size_t n_status);

/* Wait, then copy the final GS state of shot `shot_offset` (< capture_k):
 * sign words (4: destabilizer signs w0,w1 then stabilizer signs w0,w1),
 * keys (2 words each) and values (re, im as double) of up to `cap` entries;
 * *nnz receives the entry count. */
int soft_get_state(soft_run *r, uint64_t shot_offset, uint64_t *signs, uint64_t *keys, double *vals, size_t cap,
                   size_t *nnz);

/* Wait, then report the run's in-kernel bounds checks: out[0] = number of
 * failed checks (each ends its shot with SOFT_SHOT_ERROR, which the tally
 * counts as shots - discarded - overflow - kept), and for the first failure
 * out[1] = check code << 32 | event index, out[2] = shot index,
 * out[3] = the offending value. All zero when every check passed. */
int soft_run_diagnostics(soft_run *r, uint64_t out[4]);

/* Device time of the run's kernels in milliseconds (CUDA events on the run's
 * stream), and how many kernels were launched. Waits for the run. */
int soft_run_timing(soft_run *r, double *ms, uint32_t *n_launches);

/* Device time of each pass, summed over the run's chunks, in milliseconds:
 * ms[0] the lane-per-shot bucketing pre-pass (0 for warp-per-shot runs),
 * ms[1] the first pass (the shot kernel of the chosen scheduling), ms[2] the
 * rerun pass of shots whose maps outgrew the first pass (0 without one).
 * n_chunks (may be NULL) receives the number of chunks, n_rerun (may be NULL)
 * the number of shots the rerun pass finished. Waits for the run.
 * SOFT_E_ARG unless the run was launched with SOFT_RUN_TIME_PASSES and
 * without SOFT_RUN_GRAPH. */
int soft_run_pass_timing(soft_run *r, double ms[3], uint32_t *n_chunks, uint64_t *n_rerun);

/* Waits for the run, then hands its workspace back to the device's cache (or
 * frees it) and releases the handle. */
void soft_run_free(soft_run *r);

/* Frees the cached run workspace of every device (one per device, the largest
 * a freed run used). Runs still alive keep theirs until soft_run_free. */
int soft_release_workspace(void);

/* Run entry point that allocates no device memory. The paper has no
 * counterpart: this exists for callers that cannot call cudaMalloc, such as
 * code whose device memory is owned by another allocator (a framework's
 * caching allocator or a fixed arena) and latency-critical loops that cannot
 * take cudaMalloc's implicit device synchronisation.
 *   Same shots, same results as soft_run_shots with default tuning, FP64 or
 *   FP32 (`precision`), launched asynchronously on `stream`. It runs a warp
 *   per shot from the first event (no lane-per-shot scheduling, no shared
 *   noiseless prefix), so its throughput is below soft_run_shots'. The map at
 *   the circuit's cap must fit one block's shared memory (the device's opt-in
 *   limit; w42's cap 2^8 does, w97's 2^12 does not): larger caps, which
 *   soft_run_shots moves to a global-memory slab, are rejected with
 *   SOFT_E_ARG.
 *   d_tally: caller device buffer of 5 uint64 counters (shots, discarded,
 *   overflow, kept, logical errors); the call zeroes it, then accumulates.
 *   d_status / d_records: optional caller device buffers of n_shots bytes /
 *   n_shots * record_words words (NULL = not written).
 *   Scratch (work counters and the rerun list) lives in one static device
 *   array of about 4 MiB, sized for at most 1048576 shots per call; every GPU
 *   that loads the library keeps it until the process exits. Larger n_shots
 *   is rejected with SOFT_E_ARG. Each call looks up that array's device
 *   address (cudaGetSymbolAddress, which allocates nothing) with the
 *   circuit's device current. All calls share the array: calls that overlap
 *   on the GPU (different streams, no ordering) race on it and give wrong
 *   results; calls ordered on one stream are safe.
 * Errors: SOFT_E_ARG, SOFT_E_CUDA. No cudaMalloc, cudaFree or other
 * allocating routine is called. */
int soft_run_shots_noalloc(soft_circuit *c, uint64_t n_shots, uint64_t first_shot, uint64_t seed, int32_t precision,
                           void *stream, unsigned long long *d_tally, uint8_t *d_status, uint64_t *d_records);

/* Post-selected output fidelity and its gradient for fixed error patterns
 * (differentiation of Rz angles; the paper's T gates, Eq. T_gate, with the
 * angle made a parameter). A pattern is the noise draw of one shot index of
 * the circuit's noise model (same Philox stream as soft_run_shots). Every
 * measurement whose record a single-record DETECTOR reads is projected onto
 * its passing outcome (post-selection as projection, not sampling), every
 * measurement an OBSERVABLE reads is projected onto 0, resets must be
 * decided, nothing is renormalised; with phi_pre the state before the first
 * observable-read measurement and phi_end the final state,
 *   N_acc = |phi_pre|^2 (the acceptance probability), F = |phi_end|^2 / N_acc.
 * dF/dtheta_k comes from one forward pass and two reverse (adjoint) sweeps
 * in the GS basis, one warp per pattern.
 *   theta: host array of n_params angles; a parameterised RZ (op.pad = k+1,
 *   flags bit 0 = negated) uses +-theta_k. n_params must cover every k.
 *   Patterns [first_pattern, first_pattern + n_patterns), key `seed`.
 *   Caller device buffers: d_fid, d_pacc (n_patterns doubles), d_grad
 *   (n_patterns x n_params doubles, row-major), d_status (n_patterns bytes:
 *   0 ok, 1 zero acceptance (skipped, F = 0), 2 unsupported (a map above 256
 *   entries, an undecided reset, a multi-record detector), 3 error). Maps of
 *   up to 32 entries stay in registers; patterns that need more are rerun by a
 *   second launch inside the call with maps in shared memory.
 *   d_sums (may be NULL): 3 doubles, zeroed by the call, receiving the sums
 *   over ok patterns of N_acc and of N_fid = N_acc F, and their count; the
 *   ratio estimator of the post-selected fidelity is d_sums[1] / d_sums[0].
 * Synchronous: returns after the work on `stream` finished. The scratch
 * (per-warp tapes: forward coefficient maps after every rotation, sign words
 * per event) is allocated by the first call on a handle, grown when a later
 * call needs more and kept until soft_circuit_free.
 * Errors: SOFT_E_ARG, SOFT_E_OOM, SOFT_E_CUDA. */
int soft_fidelity_grad(soft_circuit *c, const double *theta, uint32_t n_params, uint64_t n_patterns,
                       uint64_t first_pattern, uint64_t seed, int32_t precision, void *stream, double *d_fid,
                       double *d_pacc, double *d_grad, uint8_t *d_status, double *d_sums);

const char *soft_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
