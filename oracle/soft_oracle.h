/*
 * soft_oracle.h -- declarations of the FP64 CPU oracle (test infrastructure).
 *
 * The op record below is the circuit interchange format. Its layout and op
 * numbering are the same as the public library's (a data format both sides
 * must read identically); the oracle declares its own copy and includes no
 * header of the CUDA path.
 */
#ifndef SOFT_ORACLE_H
#define SOFT_ORACLE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  OR_H = 0, OR_S = 1, OR_SDAG = 2, OR_X = 3, OR_Y = 4, OR_Z = 5, OR_CX = 6, OR_CZ = 7,
  OR_T = 8, OR_TDAG = 9, OR_RZ = 10, OR_M = 11, OR_R = 12, OR_MR = 13, OR_CPAULI = 14,
  OR_DETECTOR = 15, OR_OBSERVABLE = 16, OR_NOISELESS_BEGIN = 17, OR_NOISELESS_END = 18, OR_MPP = 19
};
enum { OR_FLAG_INVERT = 1, OR_FLAG_CHAIN = 2 };
/* MPP (Pauli-product measurement): flags bits 0-1 = Pauli on q0 (1 X, 2 Y,
 * 3 Z), bits 2-3 = Pauli on q1 (0: no second factor), OR_MPP_MORE = the
 * product continues in the next op, which must be an MPP. The chain's last
 * op measures the product and appends one record. */
enum { OR_MPP_MORE = 16 };
/* or_run_ex flags: OR_RUN_FIDELITY projects every measurement whose record an
 * OBSERVABLE reads onto outcome +1 and accumulates the product of their
 * conditional probabilities. */
enum { OR_RUN_FIDELITY = 1 };

/* 32-byte op: rec[] are absolute record indices (-1 = unused). */
typedef struct {
  uint16_t op;
  uint16_t flags;
  uint32_t q0, q1;
  uint32_t pad;
  double angle;
  int32_t rec[2];
} or_op;

typedef struct {
  double p1, p2, p_meas, p_reset, p_idle;
} or_noise;

enum { OR_OK = 0, OR_E_ARG = -1, OR_E_QUBIT_RANGE = -2, OR_E_RECORD_REF = -3, OR_E_UNSUPPORTED_OP = -4, OR_E_OOM = -5 };
enum { OR_ST_OK = 0, OR_ST_DISCARDED = 1, OR_ST_OVERFLOW = 2, OR_ST_ERROR = 3 };
enum { OR_EV_ERROR = 1, OR_EV_ROT = 2, OR_EV_MEAS = 3 };

typedef struct {
  int32_t kind;     /* OR_EV_* */
  int32_t op_index; /* index of the op in the circuit */
  int32_t a;        /* ERROR: site; ROT: qubit; MEAS: measurement ordinal */
  int32_t b;        /* ERROR: Pauli code (1..3 single, 1..15 two-qubit); MEAS: record index or -1 */
  double p_plus;    /* MEAS: probability of outcome +1 */
  double u;         /* MEAS: the uniform drawn for this measurement */
  int32_t outcome;  /* MEAS: +1 / -1 */
  int32_t det;      /* MEAS: 1 if decided by the integer test */
  int32_t caseb;    /* MEAS: 1 if beta(P) != 0 */
  int32_t nnz_before, nnz_after;
  int32_t pad;
  double norm;      /* sum |v|^2 after the op */
} or_event;

typedef struct {
  uint64_t shots;
  uint64_t t_out_entries;  /* output entries of T/Rz with beta != 0 */
  uint64_t t_diag_entries; /* entries of T/Rz with beta = 0 */
  uint64_t meas_entries;   /* entries visited by measurements */
  uint64_t noise_entries;  /* entries touched by applied Paulis */
  uint64_t errors;         /* sampled errors applied */
  /* The same four counts restricted to the part of each shot that differs from
   * the circuit's noiseless run: from the earliest of the first applied error,
   * the first outcome with 0 < p_+ < 1, the first map above 64 entries and, in
   * fidelity mode, the first measurement an OBSERVABLE reads, to the end of the
   * shot. */
  uint64_t post_t_out, post_t_diag, post_meas, post_noise;
} or_counts;

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double or_uniform53(uint64_t seed, uint64_t shot, uint32_t j);
uint64_t or_gap_threshold(double p, uint64_t g);

int or_run(const or_op *ops, size_t n_ops, uint32_t n_qubits, const or_noise *noise, uint32_t cap, uint64_t seed,
           uint64_t first_shot, uint64_t n_shots, int n_threads, uint8_t *status, uint64_t *records, uint32_t rw,
           uint64_t tally[5], or_counts *counts);

/* or_run with run flags. fsum (may be NULL) receives {sum of F over kept
 * shots, number of kept shots}; fid (may be NULL, one per shot) receives each
 * shot's F (0 for shots that are not kept). */
int or_run_ex(const or_op *ops, size_t n_ops, uint32_t n_qubits, const or_noise *noise, uint32_t cap, uint64_t seed,
              uint64_t first_shot, uint64_t n_shots, int n_threads, int flags, uint8_t *status, uint64_t *records,
              uint32_t rw, uint64_t tally[5], double fsum[2], double *fid, or_counts *counts);

int or_trace(const or_op *ops, size_t n_ops, uint32_t n_qubits, const or_noise *noise, uint32_t cap, uint64_t seed,
             uint64_t shot, size_t stop_after, or_event *events, size_t events_cap, size_t *n_events,
             uint64_t *rows_x, uint64_t *rows_z, uint8_t *rows_r, uint64_t *keys, double *vals, size_t keys_cap,
             size_t *n_keys, uint64_t *records, uint32_t rw, int *status_out, int *logical_out);

/* Projection run of the error pattern of shot `pattern` (see soft_oracle.c).
 * Returns 0 ok, 2 overflow, 3 unsupported/error, 4 zero acceptance. */
int or_project(const or_op *ops, size_t n_ops, uint32_t n_qubits, const or_noise *noise, uint32_t cap, uint64_t seed,
               uint64_t pattern, const double *theta, uint32_t n_theta, int64_t shift_op, double shift, double *n_acc,
               double *n_fid);

/* Error sites and Pauli codes of shot `pattern`; returns the count. */
int or_errors(const or_op *ops, size_t n_ops, uint32_t n_qubits, const or_noise *noise, uint64_t seed,
              uint64_t pattern, uint32_t *sites, uint32_t *codes, uint32_t max_out);

uint32_t or_count_sites(const or_op *ops, size_t n_ops, uint32_t n_qubits, const or_noise *noise, uint32_t *n_records);

#ifdef __cplusplus
}
#endif
#endif
