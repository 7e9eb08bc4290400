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

#ifdef __CUDACC__
#define SOFT_HD __host__ __device__
#else
#define SOFT_HD
#endif

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
  F_FIDELITY = 2,    // MEAS: an OBSERVABLE reads this record (projected onto 0 in gradient runs)
  F_DETECTOR = 4,    // PARITY
  F_OBSERVABLE = 8,  // PARITY
  F_CHAIN = 16,      // PARITY: carry into the next parity op
  F_INVERT = 32,     // PARITY
  F_COND_LAST = 64,  // PAULI: apply if the last measurement gave -1
  F_COND_REC = 128   // PAULI: apply if parity of records a, b is 1
};

// Header word 0: type (bits 0-3) | flags (4-11) | e0 (12-13) | lowbit (16-23) | xe0 (24-25).
// The gap search's index: bucket b of the top kThrTabBits bits of U holds the
// first gap g with U < thr[g] for the bucket's lowest U (bucket 2^bits: n_sites).
constexpr uint32_t kThrTabBits = 12;

SOFT_HD inline uint32_t ev_type(uint32_t w0) { return w0 & 15u; }
SOFT_HD inline uint32_t ev_flags(uint32_t w0) { return (w0 >> 4) & 255u; }
SOFT_HD inline uint32_t ev_e0(uint32_t w0) { return (w0 >> 12) & 3u; }
SOFT_HD inline uint32_t ev_lowbit(uint32_t w0) { return (w0 >> 16) & 255u; }
SOFT_HD inline uint32_t ev_xe0(uint32_t w0) { return (w0 >> 24) & 3u; }
inline uint32_t ev_pack(uint32_t type, uint32_t flags, uint32_t e0, uint32_t lowbit) {
  return (type & 15u) | ((flags & 255u) << 4) | ((e0 & 3u) << 12) | ((lowbit & 255u) << 16);
}

// Fused actions of a MEAS event (set by the compiler's peephole pass when the
// op right after the measurement touches nothing else):
//   F_COND_LAST: the reset correction X_q (xbeta/xgamma/xe0) when m = -1;
//   F_DETECTOR (+ F_INVERT): a detector on this measurement's record alone.

// One event; W = 64-bit words per n-bit vector (1 for n <= 64, else 2).
//   ROT/ROT_DIAG: a = coefficient index, b = parameter << 1 | negated (kNoRec: fixed angle),
//                 beta/gamma of Z_q
//   MEAS_A:       a = RNG ordinal, b = record index, gamma of Z_q
//   MEAS_B:       a = RNG ordinal, b = record index, beta[0] = CaseB index
//   PAULI:        a, b = record refs (F_COND_REC), beta/gamma of the Pauli
//   PARITY:       a, b = record refs (0xFFFFFFFF = none)
template <int W>
struct alignas(16) Ev {
  uint32_t w0, site_begin, a, b;
  uint64_t dsd[W], dss[W];    // sign XOR masks applied before the event
  uint64_t beta[W], gamma[W];
  uint64_t xbeta[W], xgamma[W];  // MEAS with F_COND_LAST: X_q after the measurement
};

// a I + b Z_q coefficients, FP64 and the FP32 copies the FP32 kernel uses.
struct alignas(16) Coef {
  double a_re, a_im, b_re, b_im;
  float fa_re, fa_im, fb_re, fb_im;
};

// Constants of a case-B measurement of P (pivot p, J = other rows whose
// stabilizer anticommutes with P). See meas_b in kernels.cu.
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
// kind: bits 0-1 = SITE_DEPOL1 (X, Y, Z uniform), SITE_DEPOL2 (15 Paulis
// uniform) or SITE_FLIP (the one-qubit Pauli code in bits 2-3).
enum : uint32_t { SITE_DEPOL1 = 0, SITE_DEPOL2 = 1, SITE_FLIP = 2 };
struct alignas(16) Site {
  uint64_t dsd[2], dss[2];  // sign XOR since the previous event
  uint64_t bx[2][2], gx[2][2], bz[2][2], gz[2][2];
  uint32_t kind, thin, always, c0;
};

constexpr uint32_t kNoRec = 0xFFFFFFFFu;

}  // namespace soft
