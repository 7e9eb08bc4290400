// program.h -- compiled per-shot device program (internal to libsoft).
//
// Across shots the X/Z words of the tableau evolve identically: Clifford
// conjugation, the case split of a measurement (beta(P) = 0 or not), its
// pivot and row operations depend only on X/Z bits, while noise and
// outcomes only touch sign bits and coefficients. The host therefore evolves
// X/Z once and the device keeps per shot only the 2n sign bits, the
// coefficient map and the record. Every sign update is affine over GF(2):
// a run of Clifford gates is one XOR mask (dsd/dss), and the phase c of
// Q = c d_beta s_gamma (Eq. pauli_on_basis) is
//   c = i^e0 * (-1)^{popc(sd & beta) + popc(ss & gamma)}
// with e0 computed at zero signs, sd the destabilizer signs and ss the
// stabilizer signs.
#pragma once
#include <cstdint>

namespace soft {

enum EvType : uint32_t {
  EV_ROT = 1,       // a I + b Z_q with beta(Z_q) != 0 (Theorem 1 (3))
  EV_ROT_DIAG = 2,  // a I + b Z_q with beta(Z_q) == 0 (no branching)
  EV_MEAS_A = 3,    // Z_q measurement, beta = 0: filter by eigenvalue
  EV_MEAS_B = 4,    // Z_q measurement, beta != 0: pivot, relabel, pair, replace
  EV_PAULI = 5,     // conditional Pauli (reset correction, classical feedback)
  EV_PARITY = 6,    // DETECTOR / OBSERVABLE
  EV_END = 7
};

enum : uint32_t {
  F_RECORD = 1,      // MEAS: append the outcome to the record
  F_DETECTOR = 4,    // PARITY
  F_OBSERVABLE = 8,  // PARITY
  F_CHAIN = 16,      // PARITY: carry into the next parity op
  F_INVERT = 32,     // PARITY
  F_COND_LAST = 64,  // PAULI: apply if the last measurement gave -1
  F_COND_REC = 128   // PAULI: apply if parity of records r0, r1 is 1
};

struct alignas(16) EvRec {
  uint32_t type, flags, site_begin, e0;  // site_begin: sites numbered before this event
  uint32_t ord, rec;                      // MEAS: RNG ordinal, record index
  int32_t r0, r1;                         // record references
  uint64_t dsd[2], dss[2];                // sign XOR masks applied before the event
  uint64_t beta[2], gamma[2];
  double a_re, a_im, b_re, b_im;          // ROT: a, b
  uint32_t lowbit, caseb, pad0, pad1;     // ROT: lowest set bit of beta; MEAS_B: CaseB index
};

// Constants of a case-B measurement of P (pivot p, J = other rows whose
// stabilizer anticommutes with P). See EV_MEAS_B in kernels.cu.
struct alignas(16) CaseB {
  uint64_t J[2];       // rows j with s_j <- s_j s_p
  uint64_t Hs[2];      // sign bit of s_j s_p at zero signs
  uint64_t G[2];       // rows j != p with d_j <- d_j s_p (P anticommutes with d_j)
  uint64_t Hd[2];      // sign bit of d_j s_p at zero signs
  uint64_t gamma2[2];  // gamma(P) after the row operations
  uint32_t p, hdp, e0b, rP;  // hdp: sign bit of d_p prod d_j; e0b: phase exponent of P; rP: sign of P
};

// One noise site. X_q / Z_q of the site's qubits (index 0 = q0, 1 = q1)
// carry beta/gamma words; c0 holds 2 bits per Pauli code (code 1..15).
struct alignas(16) Site {
  uint64_t dsd[2], dss[2];  // sign XOR since the previous event
  uint64_t bx[2][2], gx[2][2], bz[2][2], gz[2][2];
  uint32_t two, thin, always, c0;
};

}  // namespace soft
