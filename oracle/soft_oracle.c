/*
 * soft_oracle.c -- plain, slow, FP64 CPU oracle of the generalized-stabilizer
 * (GS) shot simulator.
 *
 * TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library. It shares
 * no code, header, table or constant generator with the CUDA path.
 *
 * What it computes (arxiv 2512.23037):
 *   - A pure state |phi> = sum_alpha v_alpha d_alpha |psi_S>  (Sec. II-C,
 *     Definition "Generalized stabilizer representation", Eq. gsf_pure).
 *   - The tableau (S, D) with signs on stabilizers AND destabilizers
 *     (Sec. II-B); rows are Hermitian Paulis (x, z, r) meaning
 *     (-1)^r prod_k i^{x_k z_k} X^{x_k} Z^{z_k}.
 *   - Pauli-on-basis identity Q|b_a> = xi_a(Q)|b_{a^beta(Q)}> (Eq.
 *     pauli_on_basis): beta_i = [Q anticommutes with s_i],
 *     gamma_i = [Q anticommutes with d_i], Q = c * d_beta * s_gamma, and
 *     xi_a(Q) = c * (-1)^{gamma . a}.
 *   - Clifford gates: conjugate every row; v unchanged (Theorem 1 (1)).
 *   - T/T^dagger/Rz = a I + b Z_q (Eq. T_gate / T_dagger): every entry feeds
 *     keys a and a^beta(Z_q) (Theorem 1 (3)).
 *   - Pauli measurement (Theorem 1 (2)): case A (beta(P) = 0) filters the
 *     entries by their eigenvalue; case B pivots the tableau, relabels the
 *     keys, pairs entries a0/a0^e_p, renormalises and replaces the pivot rows.
 *   - Monte Carlo noise: sampled Paulis applied through the same identity
 *     (Sec. II-C "Pure-state simulation model"; uniform depolarizing model,
 *     Sec. III).
 *
 * Parity status of each function is stated in the test files that pin it
 * (dense statevector replay, Aaronson-Gottesman sampler, closed forms,
 * invariants, Philox known-answer vectors).
 *
 * Implementation style: obviously-correct loops; the coefficient map is an
 * array kept sorted by key with qsort after every update; no blocking, no
 * fusion.
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "soft_oracle.h"

#define MW 2           /* words per n-bit vector: n <= 128 */
#define MAXQ 128
static const double kPi = 3.14159265358979323846264338327950288;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as    */
/* easy as 1, 2, 3", SC'11), written from the published round function.      */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c[3] ^ k1;
    uint32_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
  }
  out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

static void draw(uint64_t seed, uint64_t shot, uint32_t stream, uint32_t index, uint32_t w[4]) {
  uint32_t ctr[4] = {(uint32_t)shot, (uint32_t)(shot >> 32), stream, index};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  or_philox4x32_10(ctr, key, w);
}

/* Measurement uniform: 53 bits from words 0 and 1 of block (shot, 1, j). */
double or_uniform53(uint64_t seed, uint64_t shot, uint32_t j) {
  uint32_t w[4];
  draw(seed, shot, 1u, j, w);
  uint64_t m = (((uint64_t)w[0]) << 21) ^ (uint64_t)(w[1] >> 11);
  return ldexp((double)m, -53);
}

/* Gap threshold: floor(2^64 * (1 - (1-p)^(g+1))), the CDF of the geometric
 * gap between errors at uniform site probability p. */
uint64_t or_gap_threshold(double p, uint64_t g) {
  double q = -expm1((double)(g + 1) * log1p(-p));
  if (!(q > 0.0)) return 0;
  if (q >= 1.0) return UINT64_MAX;
  double t = ldexp(q, 64);
  if (t >= 18446744073709551615.0) return UINT64_MAX;
  return (uint64_t)t;
}

/* ------------------------------------------------------------------------ */
/* Bit vectors and Paulis                                                   */
/* ------------------------------------------------------------------------ */
static inline int getbit(const uint64_t *v, int i) { return (int)((v[i >> 6] >> (i & 63)) & 1u); }
static inline void flipbit(uint64_t *v, int i) { v[i >> 6] ^= (uint64_t)1 << (i & 63); }
static inline void setbitv(uint64_t *v, int i, int b) {
  if (getbit(v, i) != (b & 1)) flipbit(v, i);
}
static inline int popc2(const uint64_t *a) {
  return __builtin_popcountll(a[0]) + __builtin_popcountll(a[1]);
}

/* General Pauli i^e X^x Z^z (X factor written before Z on every qubit). */
typedef struct {
  uint64_t x[MW], z[MW];
  int e;
} pauli;

/* Hermitian tableau row (-1)^r prod i^{x z} X^x Z^z. */
typedef struct {
  uint64_t x[MW], z[MW];
  int r;
} row;

static pauli row_to_pauli(const row *a) {
  pauli p;
  uint64_t xz[MW];
  for (int w = 0; w < MW; ++w) {
    p.x[w] = a->x[w];
    p.z[w] = a->z[w];
    xz[w] = a->x[w] & a->z[w];
  }
  p.e = (2 * a->r + popc2(xz)) & 3;
  return p;
}

/* Returns 0 on success, -1 if p is not Hermitian. */
static int pauli_to_row(const pauli *p, row *out) {
  uint64_t xz[MW];
  for (int w = 0; w < MW; ++w) {
    out->x[w] = p->x[w];
    out->z[w] = p->z[w];
    xz[w] = p->x[w] & p->z[w];
  }
  int d = (p->e - popc2(xz)) & 3;
  if (d & 1) return -1;
  out->r = d >> 1;
  return 0;
}

/* (i^e1 X^x1 Z^z1)(i^e2 X^x2 Z^z2) = i^(e1+e2) (-1)^{z1.x2} X^(x1^x2) Z^(z1^z2) */
static pauli pauli_mul(const pauli *a, const pauli *b) {
  pauli o;
  uint64_t zx[MW];
  for (int w = 0; w < MW; ++w) {
    o.x[w] = a->x[w] ^ b->x[w];
    o.z[w] = a->z[w] ^ b->z[w];
    zx[w] = a->z[w] & b->x[w];
  }
  o.e = (a->e + b->e + 2 * popc2(zx)) & 3;
  return o;
}

static int anticommute(const uint64_t *ax, const uint64_t *az, const uint64_t *bx, const uint64_t *bz) {
  uint64_t t[MW];
  for (int w = 0; w < MW; ++w) t[w] = (ax[w] & bz[w]) ^ (az[w] & bx[w]);
  return popc2(t) & 1;
}

/* Single-qubit Pauli code: 0 I, 1 X, 2 Y, 3 Z. */
static pauli pauli_single(int code, int q) {
  pauli p;
  memset(&p, 0, sizeof p);
  if (code == 1 || code == 2) flipbit(p.x, q);
  if (code == 3 || code == 2) flipbit(p.z, q);
  p.e = (code == 2) ? 1 : 0; /* Y = i X Z */
  return p;
}

/* ------------------------------------------------------------------------ */
/* Per-shot GS state                                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
  uint64_t k[MW];
  double complex v;
} entry;

typedef struct {
  int n;
  row d[MAXQ], s[MAXQ];
  entry *e;
  size_t ne, alloc;
} gs_state;

static int ensure(gs_state *st, size_t need) {
  if (need <= st->alloc) return 0;
  size_t na = st->alloc ? st->alloc : 16;
  while (na < need) na *= 2;
  entry *ne = (entry *)realloc(st->e, na * sizeof(entry));
  if (!ne) return -1;
  st->e = ne;
  st->alloc = na;
  return 0;
}

static int cmp_entry(const void *pa, const void *pb) {
  const entry *a = (const entry *)pa, *b = (const entry *)pb;
  for (int w = MW - 1; w >= 0; --w) {
    if (a->k[w] < b->k[w]) return -1;
    if (a->k[w] > b->k[w]) return 1;
  }
  return 0;
}

/* Sort by key, add up equal keys, drop |v|^2 < tau. */
static void normalize_map(gs_state *st, double tau) {
  if (st->ne == 0) return;
  qsort(st->e, st->ne, sizeof(entry), cmp_entry);
  size_t o = 0;
  for (size_t i = 0; i < st->ne; ++i) {
    if (o > 0 && cmp_entry(&st->e[o - 1], &st->e[i]) == 0) {
      st->e[o - 1].v += st->e[i].v;
    } else {
      st->e[o++] = st->e[i];
    }
  }
  size_t m = 0;
  for (size_t i = 0; i < o; ++i) {
    double a2 = creal(st->e[i].v) * creal(st->e[i].v) + cimag(st->e[i].v) * cimag(st->e[i].v);
    if (a2 >= tau) st->e[m++] = st->e[i];
  }
  st->ne = m;
}

static void init_state(gs_state *st, int n) {
  st->n = n;
  memset(st->d, 0, sizeof st->d);
  memset(st->s, 0, sizeof st->s);
  for (int i = 0; i < n; ++i) {
    flipbit(st->d[i].x, i); /* d_i = +X_i */
    flipbit(st->s[i].z, i); /* s_i = +Z_i */
  }
  ensure(st, 16);
  memset(&st->e[0], 0, sizeof(entry));
  st->e[0].v = 1.0;
  st->ne = 1;
}

/* Q = i^c * d_beta * s_gamma (d factors first, ascending; then s factors,
 * ascending).  Returns 0, or -1 if the tableau does not span Q. */
static int decompose(const gs_state *st, const pauli *q, uint64_t beta[MW], uint64_t gamma[MW], int *c) {
  int n = st->n;
  memset(beta, 0, MW * sizeof(uint64_t));
  memset(gamma, 0, MW * sizeof(uint64_t));
  pauli acc;
  memset(&acc, 0, sizeof acc);
  for (int i = 0; i < n; ++i) {
    if (anticommute(q->x, q->z, st->s[i].x, st->s[i].z)) flipbit(beta, i);
    if (anticommute(q->x, q->z, st->d[i].x, st->d[i].z)) flipbit(gamma, i);
  }
  for (int i = 0; i < n; ++i)
    if (getbit(beta, i)) {
      pauli r = row_to_pauli(&st->d[i]);
      acc = pauli_mul(&acc, &r);
    }
  for (int i = 0; i < n; ++i)
    if (getbit(gamma, i)) {
      pauli r = row_to_pauli(&st->s[i]);
      acc = pauli_mul(&acc, &r);
    }
  for (int w = 0; w < MW; ++w)
    if (acc.x[w] != q->x[w] || acc.z[w] != q->z[w]) return -1;
  *c = (q->e - acc.e) & 3;
  return 0;
}

static double complex ipow(int e) {
  switch (e & 3) {
    case 0: return 1.0;
    case 1: return I;
    case 2: return -1.0;
    default: return -I;
  }
}

/* xi_alpha = i^c (-1)^{gamma . alpha} */
static double complex xi_of(int c, const uint64_t gamma[MW], const uint64_t alpha[MW]) {
  uint64_t t[MW];
  for (int w = 0; w < MW; ++w) t[w] = gamma[w] & alpha[w];
  return ipow(c + 2 * (popc2(t) & 1));
}

/* Apply a Pauli Q to the state: v'_{a^beta} = xi_a(Q) v_a. */
static int apply_pauli(gs_state *st, const pauli *q, or_counts *cnt) {
  uint64_t beta[MW], gamma[MW];
  int c;
  if (decompose(st, q, beta, gamma, &c)) return -1;
  for (size_t i = 0; i < st->ne; ++i) {
    double complex xi = xi_of(c, gamma, st->e[i].k);
    st->e[i].v *= xi;
    for (int w = 0; w < MW; ++w) st->e[i].k[w] ^= beta[w];
  }
  if (cnt) cnt->noise_entries += st->ne;
  qsort(st->e, st->ne, sizeof(entry), cmp_entry);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Clifford conjugation of one row (standard binary-symplectic rules).       */
/* ------------------------------------------------------------------------ */
static void conj_row(row *t, int op, int a, int b) {
  int xa = getbit(t->x, a), za = getbit(t->z, a);
  switch (op) {
    case OR_H:
      t->r ^= xa & za;
      setbitv(t->x, a, za);
      setbitv(t->z, a, xa);
      break;
    case OR_S:
      t->r ^= xa & za;
      setbitv(t->z, a, za ^ xa);
      break;
    case OR_SDAG:
      t->r ^= xa & (za ^ 1);
      setbitv(t->z, a, za ^ xa);
      break;
    case OR_X: t->r ^= za; break;
    case OR_Y: t->r ^= xa ^ za; break;
    case OR_Z: t->r ^= xa; break;
    case OR_CX: {
      int xb = getbit(t->x, b), zb = getbit(t->z, b);
      t->r ^= xa & zb & (xb ^ za ^ 1);
      setbitv(t->x, b, xb ^ xa);
      setbitv(t->z, a, za ^ zb);
      break;
    }
    case OR_CZ: {
      int xb = getbit(t->x, b), zb = getbit(t->z, b);
      t->r ^= xa & xb & (za ^ zb);
      setbitv(t->z, a, za ^ xb);
      setbitv(t->z, b, zb ^ xa);
      break;
    }
    default: break;
  }
}

static void apply_clifford(gs_state *st, int op, int a, int b) {
  for (int i = 0; i < st->n; ++i) {
    conj_row(&st->d[i], op, a, b);
    conj_row(&st->s[i], op, a, b);
  }
}

/* ------------------------------------------------------------------------ */
/* Circuit preprocessing: noise sites                                        */
/* ------------------------------------------------------------------------ */
typedef struct {
  const or_op *ops;
  size_t n_ops;
  int n;
  or_noise noise;
  uint32_t cap;
  double tau;
  double pmax;
  uint32_t n_sites;
  int32_t *pre_site;  /* per op: site index of the flip before a measurement, or -1 */
  int32_t *post_site; /* per op: site index after the op, or -1 */
  double *site_p;
  uint8_t *site_kind; /* SITE_DEPOL1, SITE_DEPOL2 or SITE_FLIP */
  uint8_t *site_code; /* SITE_FLIP: the Pauli code it applies */
  uint64_t *thr;      /* gap thresholds, n_sites entries */
  uint32_t n_records;
  uint8_t *observed;  /* per record: 1 if an OBSERVABLE reads it */
  int fid_ok;         /* no DETECTOR at or after the first observed measurement */
} circ;

/* Noise site kinds: one-qubit depolarizing (X, Y, Z uniform), two-qubit
 * depolarizing (15 Paulis uniform), and a flip (one fixed Pauli). */
enum { SITE_DEPOL1 = 0, SITE_DEPOL2 = 1, SITE_FLIP = 2 };

/* Pauli code that anticommutes with the single-qubit Pauli `code`: X for Z
 * and Y, Z for X. Applied before a measurement it flips the outcome. */
static int flip_code_for(int code) { return code == 1 ? 3 : 1; }

/* MPP chains: first op of the chain that ends at op i. */
static size_t mpp_chain_start(const or_op *ops, size_t i) {
  size_t j = i;
  while (j > 0 && ops[j - 1].op == OR_MPP && (ops[j - 1].flags & OR_MPP_MORE)) --j;
  return j;
}

static int is_1q_gate(int op) {
  return op == OR_H || op == OR_S || op == OR_SDAG || op == OR_X || op == OR_Y || op == OR_Z || op == OR_T ||
         op == OR_TDAG || op == OR_RZ;
}
static int is_2q_gate(int op) { return op == OR_CX || op == OR_CZ; }

static void circ_free(circ *c) {
  free(c->pre_site);
  free(c->post_site);
  free(c->site_p);
  free(c->site_kind);
  free(c->site_code);
  free(c->thr);
  free(c->observed);
}

/* Product of the Pauli factors of the MPP chain ops[first..last]. */
static pauli mpp_product(const or_op *ops, size_t first, size_t last) {
  pauli P;
  memset(&P, 0, sizeof P);
  for (size_t j = first; j <= last; ++j) {
    pauli a = pauli_single(ops[j].flags & 3, (int)ops[j].q0);
    P = pauli_mul(&P, &a);
    if ((ops[j].flags >> 2) & 3) {
      pauli b = pauli_single((ops[j].flags >> 2) & 3, (int)ops[j].q1);
      P = pauli_mul(&P, &b);
    }
  }
  return P;
}

/* True for an op that measures and appends a record: M, MR, or the last op of an MPP chain. */
static int records_outcome(const or_op *o) {
  return o->op == OR_M || o->op == OR_MR || (o->op == OR_MPP && !(o->flags & OR_MPP_MORE));
}

static int circ_build(circ *c, const or_op *ops, size_t n_ops, uint32_t n, const or_noise *noise, uint32_t cap) {
  memset(c, 0, sizeof *c);
  if (n == 0 || n > MAXQ) return OR_E_ARG;
  c->ops = ops;
  c->n_ops = n_ops;
  c->n = (int)n;
  c->noise = *noise;
  c->cap = cap;
  c->tau = 1e-20;
  c->pmax = fmax(fmax(noise->p1, noise->p2), fmax(noise->p_meas, noise->p_reset));
  c->pre_site = (int32_t *)malloc((n_ops + 1) * sizeof(int32_t));
  c->post_site = (int32_t *)malloc((n_ops + 1) * sizeof(int32_t));
  c->site_p = (double *)malloc((2 * n_ops + 1) * sizeof(double));
  c->site_kind = (uint8_t *)malloc(2 * n_ops + 1);
  c->site_code = (uint8_t *)malloc(2 * n_ops + 1);
  if (!c->pre_site || !c->post_site || !c->site_p || !c->site_kind || !c->site_code) return OR_E_OOM;
  int noiseless = 0;
  uint32_t ns = 0, nrec = 0;
  uint64_t mpp_q[MW] = {0, 0}; /* qubits already in the open MPP chain */
  for (size_t i = 0; i < n_ops; ++i) {
    const or_op *o = &ops[i];
    c->pre_site[i] = -1;
    c->post_site[i] = -1;
    int op = o->op;
    if (op > OR_MPP) return OR_E_UNSUPPORTED_OP;
    if (i > 0 && ops[i - 1].op == OR_MPP && (ops[i - 1].flags & OR_MPP_MORE) && op != OR_MPP) return OR_E_ARG;
    if (is_1q_gate(op) || is_2q_gate(op) || op == OR_M || op == OR_R || op == OR_MR || op == OR_CPAULI ||
        op == OR_MPP) {
      if (o->q0 >= n) return OR_E_QUBIT_RANGE;
    }
    if (op == OR_MPP) {
      int pa = o->flags & 3, pb = (o->flags >> 2) & 3;
      if (pa == 0 || (o->flags & ~(uint32_t)(15 | OR_MPP_MORE))) return OR_E_ARG;
      if (pb && (o->q1 >= n || o->q1 == o->q0)) return OR_E_QUBIT_RANGE;
      if (getbit(mpp_q, (int)o->q0) || (pb && getbit(mpp_q, (int)o->q1))) return OR_E_ARG; /* repeated qubit */
      flipbit(mpp_q, (int)o->q0);
      if (pb) flipbit(mpp_q, (int)o->q1);
      if (!(o->flags & OR_MPP_MORE)) mpp_q[0] = mpp_q[1] = 0;
      else if (i + 1 == n_ops) return OR_E_ARG; /* open chain at the end */
    }
    if (is_2q_gate(op) && (o->q1 >= n || o->q1 == o->q0)) return OR_E_QUBIT_RANGE;
    if (op == OR_DETECTOR || op == OR_OBSERVABLE || op == OR_CPAULI) {
      for (int r = 0; r < 2; ++r)
        if (o->rec[r] >= 0 && (uint32_t)o->rec[r] >= nrec) return OR_E_RECORD_REF;
    }
    if (op == OR_NOISELESS_BEGIN) noiseless = 1;
    if (op == OR_NOISELESS_END) noiseless = 0;
    if (!noiseless) {
      /* measurement flip: X before M/MR; before an MPP chain, the Pauli on its
       * first qubit that anticommutes with the chain's first factor */
      int first_mpp = op == OR_MPP && mpp_chain_start(ops, i) == i;
      if ((op == OR_M || op == OR_MR || first_mpp) && noise->p_meas > 0) {
        c->site_p[ns] = noise->p_meas;
        c->site_kind[ns] = SITE_FLIP;
        c->site_code[ns] = (uint8_t)(op == OR_MPP ? flip_code_for(o->flags & 3) : 1);
        c->pre_site[i] = (int32_t)ns++;
      }
      if (is_1q_gate(op) && noise->p1 > 0) {
        c->site_p[ns] = noise->p1;
        c->site_kind[ns] = SITE_DEPOL1;
        c->site_code[ns] = 0;
        c->post_site[i] = (int32_t)ns++;
      } else if (is_2q_gate(op) && noise->p2 > 0) {
        c->site_p[ns] = noise->p2;
        c->site_kind[ns] = SITE_DEPOL2;
        c->site_code[ns] = 0;
        c->post_site[i] = (int32_t)ns++;
      } else if ((op == OR_R || op == OR_MR) && noise->p_reset > 0) {
        c->site_p[ns] = noise->p_reset;
        c->site_kind[ns] = SITE_FLIP;
        c->site_code[ns] = 1;
        c->post_site[i] = (int32_t)ns++;
      }
    }
    if (records_outcome(o)) nrec++;
  }
  c->n_sites = ns;
  c->n_records = nrec;
  /* records read by OBSERVABLE ops, and whether a DETECTOR follows the first of their measurements */
  c->observed = (uint8_t *)calloc(nrec + 1, 1);
  if (!c->observed) return OR_E_OOM;
  for (size_t i = 0; i < n_ops; ++i)
    if (ops[i].op == OR_OBSERVABLE)
      for (int r = 0; r < 2; ++r)
        if (ops[i].rec[r] >= 0 && (uint32_t)ops[i].rec[r] < nrec) c->observed[ops[i].rec[r]] = 1;
  c->fid_ok = 1;
  {
    uint32_t rcount = 0;
    int seen = 0;
    for (size_t i = 0; i < n_ops; ++i) {
      if (records_outcome(&ops[i])) {
        if (c->observed[rcount]) seen = 1;
        rcount++;
      }
      if (ops[i].op == OR_DETECTOR && seen) c->fid_ok = 0;
    }
  }
  c->thr = (uint64_t *)malloc((ns + 1) * sizeof(uint64_t));
  if (!c->thr) return OR_E_OOM;
  for (uint32_t g = 0; g < ns; ++g) c->thr[g] = or_gap_threshold(c->pmax, g);
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Noise stream: next accepted error at or after site `cur`.                  */
/* ------------------------------------------------------------------------ */
typedef struct {
  uint32_t cur;   /* first site not yet decided */
  uint32_t k;     /* next block index of stream 0 */
  uint32_t site;  /* site of the pending error, UINT32_MAX if none */
  uint32_t word2; /* Pauli choice word of the pending error */
} noise_stream;

static void next_error(const circ *c, uint64_t seed, uint64_t shot, noise_stream *ns) {
  for (;;) {
    if (ns->cur >= c->n_sites) {
      ns->site = UINT32_MAX;
      return;
    }
    uint32_t w[4];
    draw(seed, shot, 0u, ns->k, w);
    ns->k++;
    uint64_t u = (uint64_t)w[0] | ((uint64_t)w[1] << 32);
    uint32_t remaining = c->n_sites - ns->cur;
    uint32_t g = UINT32_MAX;
    for (uint32_t t = 0; t < remaining; ++t)
      if (u < c->thr[t]) {
        g = t;
        break;
      }
    if (g == UINT32_MAX) {
      ns->cur = c->n_sites;
      ns->site = UINT32_MAX;
      return;
    }
    uint32_t s = ns->cur + g;
    ns->cur = s + 1;
    double ps = c->site_p[s];
    if (ps < c->pmax) {
      uint32_t thr = (uint32_t)floor(ldexp(ps / c->pmax, 32));
      if (!(w[3] < thr)) continue; /* thinned out */
    }
    ns->site = s;
    ns->word2 = w[2];
    return;
  }
}

/* Pauli code of an error at `site` with choice word `word2`: a depolarizing
 * site picks idx = floor(word2 K / 2^32) with K = 3 (X, Y, Z) or K = 15
 * ((P_a, P_b) with 4 P_a + P_b = idx + 1, code 0 I, 1 X, 2 Y, 3 Z); a flip
 * site applies its fixed code. */
static int error_code(const circ *c, uint32_t site, uint32_t word2) {
  if (c->site_kind[site] == SITE_FLIP) return c->site_code[site];
  if (c->site_kind[site] == SITE_DEPOL2) return (int)(((uint64_t)word2 * 15u) >> 32) + 1;
  return (int)(((uint64_t)word2 * 3u) >> 32) + 1;
}

static pauli error_pauli(const circ *c, uint32_t site, uint32_t word2, const or_op *o, int *code_out) {
  if (c->site_kind[site] == SITE_FLIP) {
    *code_out = c->site_code[site];
    return pauli_single(c->site_code[site], (int)o->q0);
  }
  if (c->site_kind[site] == SITE_DEPOL2) {
    uint32_t idx = (uint32_t)(((uint64_t)word2 * 15u) >> 32);
    int pa = (int)((idx + 1) >> 2), pb = (int)((idx + 1) & 3);
    pauli A = pauli_single(pa, (int)o->q0), B = pauli_single(pb, (int)o->q1);
    *code_out = (int)(idx + 1);
    return pauli_mul(&A, &B);
  }
  uint32_t idx = (uint32_t)(((uint64_t)word2 * 3u) >> 32);
  *code_out = (int)(idx + 1);
  return pauli_single((int)(idx + 1), (int)o->q0);
}

/* ------------------------------------------------------------------------ */
/* Non-Clifford and measurement updates                                       */
/* ------------------------------------------------------------------------ */

/* a I + b Z_q (Theorem 1 (3)). Returns status. */
static int apply_rot_tau(gs_state *st, const circ *c, int q, double complex a, double complex b, double tau,
                         or_counts *cnt);
static int apply_rot(gs_state *st, const circ *c, int q, double complex a, double complex b, or_counts *cnt) {
  return apply_rot_tau(st, c, q, a, b, c->tau, cnt);
}
static int apply_rot_tau(gs_state *st, const circ *c, int q, double complex a, double complex b, double tau,
                         or_counts *cnt) {
  pauli Z = pauli_single(3, q);
  uint64_t beta[MW], gamma[MW];
  int ce;
  if (decompose(st, &Z, beta, gamma, &ce)) return OR_ST_ERROR;
  size_t n0 = st->ne;
  if (ensure(st, 2 * n0 + 1)) return OR_ST_ERROR;
  for (size_t i = 0; i < n0; ++i) {
    entry src = st->e[i];
    double complex xi = xi_of(ce, gamma, src.k);
    st->e[i].v = a * src.v;
    entry t;
    for (int w = 0; w < MW; ++w) t.k[w] = src.k[w] ^ beta[w];
    t.v = b * xi * src.v;
    st->e[n0 + i] = t;
  }
  st->ne = 2 * n0;
  normalize_map(st, tau);
  if (cnt) {
    if ((beta[0] | beta[1]) == 0) cnt->t_diag_entries += n0;
    else cnt->t_out_entries += st->ne;
  }
  if (st->ne > c->cap) return OR_ST_OVERFLOW;
  return OR_ST_OK;
}

typedef struct {
  double p_plus, u;
  int m;    /* +1 or -1 */
  int det;  /* 1 if deterministic (integer test), else 0 */
  int caseb;
} meas_info;

static double snap(double p) {
  if (p < 1e-12) return 0.0;
  if (p > 1.0 - 1e-12) return 1.0;
  return p;
}

/* Measure the Hermitian Pauli P (Theorem 1 (2), Eq. Pi_pm). */
/* With `force` set the outcome is +1 whenever p_+ > 0 (a projection onto +1,
 * renormalised), and -1 only when +1 is impossible. */
static int measure(gs_state *st, const circ *c, const pauli *P, uint64_t seed, uint64_t shot, uint32_t ordinal,
                   int force, meas_info *mi, or_counts *cnt) {
  uint64_t beta[MW], gamma[MW];
  int ce;
  if (decompose(st, P, beta, gamma, &ce)) return OR_ST_ERROR;
  mi->u = or_uniform53(seed, shot, ordinal);
  if ((beta[0] | beta[1]) == 0) {
    /* Case A: P = i^ce s_gamma with i^ce = +-1. */
    mi->caseb = 0;
    if (ce & 1) return OR_ST_ERROR;
    int sgn = (ce == 2); /* 1 if c = -1 */
    int first = -1, same = 1;
    double sp = 0.0, sm = 0.0;
    for (size_t i = 0; i < st->ne; ++i) {
      uint64_t t[MW];
      for (int w = 0; w < MW; ++w) t[w] = gamma[w] & st->e[i].k[w];
      int lam_neg = (popc2(t) & 1) ^ sgn; /* 1 if lambda = -1 */
      if (first < 0) first = lam_neg;
      else if (first != lam_neg) same = 0;
      double a2 = creal(st->e[i].v) * creal(st->e[i].v) + cimag(st->e[i].v) * cimag(st->e[i].v);
      if (lam_neg) sm += a2;
      else sp += a2;
    }
    if (cnt) cnt->meas_entries += st->ne;
    if (same) {
      mi->det = 1;
      mi->m = first ? -1 : +1;
      mi->p_plus = first ? 0.0 : 1.0;
      return OR_ST_OK;
    }
    mi->det = 0;
    double pp = snap(sp / (sp + sm));
    mi->p_plus = pp;
    mi->m = force ? (pp > 0.0 ? +1 : -1) : ((mi->u < pp) ? +1 : -1);
    double keep = (mi->m == 1) ? sp : sm;
    double scale = 1.0 / sqrt(keep);
    size_t o = 0;
    for (size_t i = 0; i < st->ne; ++i) {
      uint64_t t[MW];
      for (int w = 0; w < MW; ++w) t[w] = gamma[w] & st->e[i].k[w];
      int lam_neg = (popc2(t) & 1) ^ sgn;
      if ((lam_neg ? -1 : +1) == mi->m) {
        st->e[o] = st->e[i];
        st->e[o].v *= scale;
        o++;
      }
    }
    st->ne = o;
    normalize_map(st, c->tau);
    return OR_ST_OK;
  }

  /* Case B. Pivot p = lowest i with beta_i = 1; J = the other such i. */
  mi->caseb = 1;
  mi->det = 0;
  int n = st->n, p = -1;
  for (int i = 0; i < n; ++i)
    if (getbit(beta, i)) {
      p = i;
      break;
    }
  uint64_t J[MW] = {beta[0], beta[1]};
  flipbit(J, p);
  /* Row operations: s_j <- s_j s_p (j in J); d_p <- d_p prod_{j in J} d_j. */
  pauli sp_ = row_to_pauli(&st->s[p]);
  for (int j = 0; j < n; ++j)
    if (getbit(J, j)) {
      pauli sj = row_to_pauli(&st->s[j]);
      pauli prod = pauli_mul(&sj, &sp_);
      if (pauli_to_row(&prod, &st->s[j])) return OR_ST_ERROR;
    }
  pauli dp = row_to_pauli(&st->d[p]);
  for (int j = 0; j < n; ++j)
    if (getbit(J, j)) {
      pauli dj = row_to_pauli(&st->d[j]);
      dp = pauli_mul(&dp, &dj);
    }
  if (pauli_to_row(&dp, &st->d[p])) return OR_ST_ERROR;
  /* Relabel keys: alpha_j ^= alpha_p for j in J. */
  for (size_t i = 0; i < st->ne; ++i)
    if (getbit(st->e[i].k, p))
      for (int w = 0; w < MW; ++w) st->e[i].k[w] ^= J[w];
  qsort(st->e, st->ne, sizeof(entry), cmp_entry);
  /* Now P = i^ce2 d_p s_gamma2. */
  uint64_t beta2[MW], gamma2[MW];
  int ce2;
  if (decompose(st, P, beta2, gamma2, &ce2)) return OR_ST_ERROR;
  {
    uint64_t ep[MW] = {0, 0};
    flipbit(ep, p);
    if (beta2[0] != ep[0] || beta2[1] != ep[1]) return OR_ST_ERROR;
  }
  /* Pair a0 (bit p clear) with a1 = a0 ^ e_p. Build the list of a0 keys with
   * (v0, v1); entries are sorted so a plain search is enough. */
  size_t n0 = st->ne;
  entry *pairs_k = (entry *)malloc((n0 + 1) * sizeof(entry)); /* key a0, v unused */
  double complex *v0 = (double complex *)malloc((n0 + 1) * sizeof(double complex));
  double complex *v1 = (double complex *)malloc((n0 + 1) * sizeof(double complex));
  if (!pairs_k || !v0 || !v1) {
    free(pairs_k); free(v0); free(v1);
    return OR_ST_ERROR;
  }
  size_t np = 0;
  for (size_t i = 0; i < n0; ++i) {
    entry a0 = st->e[i];
    int hi = getbit(a0.k, p);
    if (hi) flipbit(a0.k, p);
    size_t f = np;
    for (size_t t = 0; t < np; ++t)
      if (cmp_entry(&pairs_k[t], &a0) == 0) {
        f = t;
        break;
      }
    if (f == np) {
      pairs_k[np] = a0;
      v0[np] = 0.0;
      v1[np] = 0.0;
      np++;
    }
    if (hi) v1[f] = st->e[i].v;
    else v0[f] = st->e[i].v;
  }
  double s_plus = 0.0, s_minus = 0.0;
  for (size_t t = 0; t < np; ++t) {
    uint64_t a1[MW] = {pairs_k[t].k[0], pairs_k[t].k[1]};
    flipbit(a1, p);
    double complex x1 = xi_of(ce2, gamma2, a1) * v1[t];
    double complex wp = v0[t] + x1, wm = v0[t] - x1;
    s_plus += 0.5 * (creal(wp) * creal(wp) + cimag(wp) * cimag(wp));
    s_minus += 0.5 * (creal(wm) * creal(wm) + cimag(wm) * cimag(wm));
  }
  if (cnt) cnt->meas_entries += n0;
  double pp = snap(s_plus / (s_plus + s_minus));
  mi->p_plus = pp;
  mi->m = force ? (pp > 0.0 ? +1 : -1) : ((mi->u < pp) ? +1 : -1);
  double sm_ = (mi->m == 1) ? s_plus : s_minus;
  double scale = 1.0 / sqrt(2.0 * sm_);
  st->ne = 0;
  for (size_t t = 0; t < np; ++t) {
    uint64_t a1[MW] = {pairs_k[t].k[0], pairs_k[t].k[1]};
    flipbit(a1, p);
    double complex x1 = xi_of(ce2, gamma2, a1) * v1[t];
    entry ne_;
    ne_.k[0] = pairs_k[t].k[0];
    ne_.k[1] = pairs_k[t].k[1];
    ne_.v = (v0[t] + (double)mi->m * x1) * scale;
    st->e[st->ne++] = ne_;
  }
  free(pairs_k); free(v0); free(v1);
  /* Tableau replacement: d_j <- d_j * old s_p for j != p with gamma2_j = 1;
   * d_p <- old s_p; s_p <- m P. */
  row old_sp = st->s[p];
  pauli osp = row_to_pauli(&old_sp);
  for (int j = 0; j < n; ++j)
    if (j != p && getbit(gamma2, j)) {
      pauli dj = row_to_pauli(&st->d[j]);
      pauli prod = pauli_mul(&dj, &osp);
      if (pauli_to_row(&prod, &st->d[j])) return OR_ST_ERROR;
    }
  st->d[p] = old_sp;
  row newsp;
  if (pauli_to_row(P, &newsp)) return OR_ST_ERROR;
  if (mi->m == -1) newsp.r ^= 1;
  st->s[p] = newsp;
  normalize_map(st, c->tau);
  return OR_ST_OK;
}

/* ------------------------------------------------------------------------ */
/* One shot                                                                   */
/* ------------------------------------------------------------------------ */
typedef struct {
  or_event *ev;
  size_t n_ev, cap_ev;
} trace_buf;

static void push_ev(trace_buf *tb, const or_event *e) {
  if (!tb || !tb->ev) return;
  if (tb->n_ev < tb->cap_ev) tb->ev[tb->n_ev] = *e;
  tb->n_ev++;
}

static double map_norm(const gs_state *st) {
  double s = 0.0;
  for (size_t i = 0; i < st->ne; ++i)
    s += creal(st->e[i].v) * creal(st->e[i].v) + cimag(st->e[i].v) * cimag(st->e[i].v);
  return s;
}

static int apply_error_if_due(gs_state *st, const circ *c, uint64_t seed, uint64_t shot, noise_stream *ns,
                              int32_t site, size_t op_index, trace_buf *tb, or_counts *cnt) {
  if (site < 0 || (uint32_t)site != ns->site) return OR_ST_OK;
  int code = 0;
  pauli q = error_pauli(c, (uint32_t)site, ns->word2, &c->ops[op_index], &code);
  if (apply_pauli(st, &q, cnt)) return OR_ST_ERROR;
  if (cnt) cnt->errors++;
  or_event e;
  memset(&e, 0, sizeof e);
  e.kind = OR_EV_ERROR;
  e.op_index = (int32_t)op_index;
  e.a = site;
  e.b = code;
  e.nnz_before = e.nnz_after = (int32_t)st->ne;
  e.norm = map_norm(st);
  push_ev(tb, &e);
  next_error(c, seed, shot, ns);
  return OR_ST_OK;
}

/* Adds the work counted since `c0` to the post-prefix counters. */
static void add_post(or_counts *cnt, const or_counts *c0) {
  cnt->post_t_out += cnt->t_out_entries - c0->t_out_entries;
  cnt->post_t_diag += cnt->t_diag_entries - c0->t_diag_entries;
  cnt->post_meas += cnt->meas_entries - c0->meas_entries;
  cnt->post_noise += cnt->noise_entries - c0->noise_entries;
}

/* One shot. In fidelity mode (fid != NULL) every measurement whose record an
 * OBSERVABLE reads is projected onto +1 and *fid accumulates the product of
 * their conditional probabilities p_+; when +1 is impossible *fid = 0 and the
 * shot ends there (kept). */
static int run_shot(const circ *c, gs_state *st, uint64_t seed, uint64_t shot, uint64_t *rec, uint32_t rw,
                    int *logical, size_t stop_after, trace_buf *tb, or_counts *cnt, double *fid) {
  init_state(st, c->n);
  if (fid) *fid = 1.0;
  if (rec) memset(rec, 0, rw * sizeof(uint64_t));
  noise_stream ns = {0, 0, UINT32_MAX, 0};
  next_error(c, seed, shot, &ns);
  uint32_t ordinal = 0, nrec = 0;
  int chain = 0;
  *logical = 0;
  uint64_t recbits_local[64];
  uint64_t *rb = rec;
  if (!rb) {
    if (c->n_records > 64 * 64) return OR_ST_ERROR;
    memset(recbits_local, 0, sizeof recbits_local);
    rb = recbits_local;
  }
  size_t lim = stop_after < c->n_ops ? stop_after : c->n_ops;
  int live = 0; /* past the noiseless-run prefix (see or_counts) */
  or_counts c0;
  memset(&c0, 0, sizeof c0);
  for (size_t i = 0; i < lim; ++i) {
    const or_op *o = &c->ops[i];
    int op = o->op;
    if (cnt) c0 = *cnt;
    int stt = apply_error_if_due(st, c, seed, shot, &ns, c->pre_site[i], i, tb, cnt);
    if (stt) return stt;
    if (cnt) {
      if (cnt->errors != c0.errors) live = 1;
      if (live) add_post(cnt, &c0);
      c0 = *cnt;
    }
    size_t nb = st->ne;
    switch (op) {
      case OR_H: case OR_S: case OR_SDAG: case OR_X: case OR_Y: case OR_Z: case OR_CX: case OR_CZ:
        apply_clifford(st, op, (int)o->q0, (int)o->q1);
        break;
      case OR_T: case OR_TDAG: case OR_RZ: {
        double complex a, b;
        if (op == OR_T) {
          double complex w = cexp(I * kPi / 4.0);
          a = (1.0 + w) / 2.0;
          b = (1.0 - w) / 2.0;
        } else if (op == OR_TDAG) {
          double complex w = cexp(-I * kPi / 4.0);
          a = (1.0 + w) / 2.0;
          b = (1.0 - w) / 2.0;
        } else {
          a = cos(o->angle / 2.0);
          b = -I * sin(o->angle / 2.0);
        }
        int r = apply_rot(st, c, (int)o->q0, a, b, cnt);
        or_event e;
        memset(&e, 0, sizeof e);
        e.kind = OR_EV_ROT;
        e.op_index = (int32_t)i;
        e.a = (int32_t)o->q0;
        e.nnz_before = (int32_t)nb;
        e.nnz_after = (int32_t)st->ne;
        e.norm = map_norm(st);
        push_ev(tb, &e);
        if (r) return r;
        break;
      }
      case OR_M: case OR_R: case OR_MR: case OR_MPP: {
        if (op == OR_MPP && (o->flags & OR_MPP_MORE)) break; /* the chain's last op measures */
        pauli P = (op == OR_MPP) ? mpp_product(c->ops, mpp_chain_start(c->ops, i), i) : pauli_single(3, (int)o->q0);
        const int force = fid && op != OR_R && c->observed[nrec];
        if (fid && op != OR_R && c->observed[nrec]) live = 1;
        meas_info mi;
        int r = measure(st, c, &P, seed, shot, ordinal, force, &mi, cnt);
        if (r) return r;
        if (mi.p_plus > 0.0 && mi.p_plus < 1.0) live = 1;
        or_event e;
        memset(&e, 0, sizeof e);
        e.kind = OR_EV_MEAS;
        e.op_index = (int32_t)i;
        e.a = (int32_t)ordinal;
        e.b = (op == OR_R) ? -1 : (int32_t)nrec;
        e.p_plus = mi.p_plus;
        e.u = mi.u;
        e.outcome = mi.m;
        e.det = mi.det;
        e.caseb = mi.caseb;
        e.nnz_before = (int32_t)nb;
        e.nnz_after = (int32_t)st->ne;
        e.norm = map_norm(st);
        push_ev(tb, &e);
        ordinal++;
        if (force) {
          if (mi.m == -1) {
            *fid = 0.0;
            return OR_ST_OK;
          }
          *fid *= mi.p_plus;
        }
        if (op != OR_R) {
          if (mi.m == -1) flipbit(rb, (int)nrec);
          nrec++;
        }
        if ((op == OR_R || op == OR_MR) && mi.m == -1) {
          pauli X = pauli_single(1, (int)o->q0);
          if (apply_pauli(st, &X, cnt)) return OR_ST_ERROR;
        }
        break;
      }
      case OR_CPAULI: {
        int par = 0;
        for (int r = 0; r < 2; ++r)
          if (o->rec[r] >= 0) par ^= getbit(rb, o->rec[r]);
        if (par) {
          pauli q = pauli_single(o->flags & 3, (int)o->q0);
          if ((o->flags & 3) && apply_pauli(st, &q, cnt)) return OR_ST_ERROR;
        }
        break;
      }
      case OR_DETECTOR: case OR_OBSERVABLE: {
        int par = chain;
        for (int r = 0; r < 2; ++r)
          if (o->rec[r] >= 0) par ^= getbit(rb, o->rec[r]);
        par ^= (o->flags & OR_FLAG_INVERT) ? 1 : 0;
        if (o->flags & OR_FLAG_CHAIN) {
          chain = par;
          break;
        }
        chain = 0;
        if (op == OR_DETECTOR && par) return OR_ST_DISCARDED;
        if (op == OR_OBSERVABLE && par) *logical = 1;
        break;
      }
      default:
        break;
    }
    if (cnt) {
      if (st->ne > 64) live = 1;
      if (live) add_post(cnt, &c0);
      c0 = *cnt;
    }
    stt = apply_error_if_due(st, c, seed, shot, &ns, c->post_site[i], i, tb, cnt);
    if (stt) return stt;
    if (cnt) {
      if (cnt->errors != c0.errors) live = 1;
      if (live) add_post(cnt, &c0);
    }
  }
  return OR_ST_OK;
}

/* ------------------------------------------------------------------------ */
/* Public entry points                                                        */
/* ------------------------------------------------------------------------ */
typedef struct {
  const circ *c;
  uint64_t seed, first, count, shot0;
  uint8_t *status;
  uint64_t *records;
  uint32_t rw;
  uint64_t tally[5];
  double fsum[2];
  double *fid;
  int fid_mode;
  or_counts cnt;
  int err;
} worker_arg;

static void *worker(void *p) {
  worker_arg *a = (worker_arg *)p;
  gs_state *st = (gs_state *)calloc(1, sizeof(gs_state));
  if (!st) {
    a->err = OR_E_OOM;
    return NULL;
  }
  memset(a->tally, 0, sizeof a->tally);
  a->fsum[0] = a->fsum[1] = 0.0;
  for (uint64_t t = 0; t < a->count; ++t) {
    uint64_t shot = a->first + t;
    int logical = 0;
    uint64_t *rec = a->records ? a->records + (shot - a->shot0) * a->rw : NULL;
    double f = 0.0;
    int s = run_shot(a->c, st, a->seed, shot, rec, a->rw, &logical, (size_t)-1, NULL, &a->cnt,
                     a->fid_mode ? &f : NULL);
    if (a->status) a->status[shot - a->shot0] = (uint8_t)s;
    a->tally[0]++;
    if (s == OR_ST_DISCARDED) a->tally[1]++;
    else if (s == OR_ST_OVERFLOW) a->tally[2]++;
    else if (s == OR_ST_OK) {
      a->tally[3]++;
      if (logical) a->tally[4]++;
      if (a->fid_mode) {
        a->fsum[0] += f;
        a->fsum[1] += 1.0;
      }
    }
    if (a->fid) a->fid[shot - a->shot0] = (s == OR_ST_OK) ? f : 0.0;
    a->cnt.shots++;
  }
  free(st->e);
  free(st);
  return NULL;
}

int or_run(const or_op *ops, size_t n_ops, uint32_t n_qubits, const or_noise *noise, uint32_t cap, uint64_t seed,
           uint64_t first_shot, uint64_t n_shots, int n_threads, uint8_t *status, uint64_t *records, uint32_t rw,
           uint64_t tally[5], or_counts *counts) {
  return or_run_ex(ops, n_ops, n_qubits, noise, cap, seed, first_shot, n_shots, n_threads, 0, status, records, rw,
                   tally, NULL, NULL, counts);
}

int or_run_ex(const or_op *ops, size_t n_ops, uint32_t n_qubits, const or_noise *noise, uint32_t cap, uint64_t seed,
              uint64_t first_shot, uint64_t n_shots, int n_threads, int flags, uint8_t *status, uint64_t *records,
              uint32_t rw, uint64_t tally[5], double fsum[2], double *fid, or_counts *counts) {
  circ c;
  int rc = circ_build(&c, ops, n_ops, n_qubits, noise, cap);
  if (rc) {
    circ_free(&c);
    return rc;
  }
  const int fid_mode = (flags & OR_RUN_FIDELITY) != 0;
  if (fid_mode && !c.fid_ok) {
    circ_free(&c);
    return OR_E_ARG;
  }
  if (records && rw * 64u < c.n_records) {
    circ_free(&c);
    return OR_E_ARG;
  }
  if (n_threads < 1) n_threads = 1;
  if ((uint64_t)n_threads > n_shots && n_shots > 0) n_threads = (int)n_shots;
  worker_arg *args = (worker_arg *)calloc((size_t)n_threads, sizeof(worker_arg));
  pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
  if (!args || !th) {
    free(args); free(th); circ_free(&c);
    return OR_E_OOM;
  }
  uint64_t per = n_shots / (uint64_t)n_threads, extra = n_shots % (uint64_t)n_threads, at = first_shot;
  for (int t = 0; t < n_threads; ++t) {
    args[t].c = &c;
    args[t].seed = seed;
    args[t].first = at;
    args[t].count = per + ((uint64_t)t < extra ? 1 : 0);
    args[t].shot0 = first_shot;
    args[t].status = status;
    args[t].records = records;
    args[t].rw = rw;
    args[t].fid_mode = fid_mode;
    args[t].fid = fid;
    at += args[t].count;
  }
  if (n_threads == 1) worker(&args[0]);
  else {
    for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, worker, &args[t]);
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
  }
  memset(tally, 0, 5 * sizeof(uint64_t));
  if (counts) memset(counts, 0, sizeof *counts);
  if (fsum) fsum[0] = fsum[1] = 0.0;
  rc = OR_OK;
  for (int t = 0; t < n_threads; ++t) {
    if (args[t].err) rc = args[t].err;
    for (int k = 0; k < 5; ++k) tally[k] += args[t].tally[k];
    if (fsum) {
      fsum[0] += args[t].fsum[0];
      fsum[1] += args[t].fsum[1];
    }
    if (counts) {
      counts->shots += args[t].cnt.shots;
      counts->t_out_entries += args[t].cnt.t_out_entries;
      counts->t_diag_entries += args[t].cnt.t_diag_entries;
      counts->meas_entries += args[t].cnt.meas_entries;
      counts->noise_entries += args[t].cnt.noise_entries;
      counts->errors += args[t].cnt.errors;
      counts->post_t_out += args[t].cnt.post_t_out;
      counts->post_t_diag += args[t].cnt.post_t_diag;
      counts->post_meas += args[t].cnt.post_meas;
      counts->post_noise += args[t].cnt.post_noise;
    }
  }
  free(args); free(th); circ_free(&c);
  return rc;
}

int or_trace(const or_op *ops, size_t n_ops, uint32_t n_qubits, const or_noise *noise, uint32_t cap, uint64_t seed,
             uint64_t shot, size_t stop_after, or_event *events, size_t events_cap, size_t *n_events,
             uint64_t *rows_x, uint64_t *rows_z, uint8_t *rows_r, uint64_t *keys, double *vals, size_t keys_cap,
             size_t *n_keys, uint64_t *records, uint32_t rw, int *status_out, int *logical_out) {
  circ c;
  int rc = circ_build(&c, ops, n_ops, n_qubits, noise, cap);
  if (rc) {
    circ_free(&c);
    return rc;
  }
  gs_state *st = (gs_state *)calloc(1, sizeof(gs_state));
  if (!st) {
    circ_free(&c);
    return OR_E_OOM;
  }
  trace_buf tb = {events, 0, events_cap};
  int logical = 0;
  if (records && rw * 64u < c.n_records) {
    free(st);
    circ_free(&c);
    return OR_E_ARG;
  }
  int s = run_shot(&c, st, seed, shot, records, rw, &logical, stop_after, &tb, NULL, NULL);
  *status_out = s;
  *logical_out = logical;
  *n_events = tb.n_ev;
  int n = (int)n_qubits;
  /* rows: 2n rows, d_0..d_{n-1} then s_0..s_{n-1}; 2 words each. */
  for (int i = 0; i < n; ++i) {
    for (int w = 0; w < MW; ++w) {
      if (rows_x) rows_x[i * MW + w] = st->d[i].x[w];
      if (rows_z) rows_z[i * MW + w] = st->d[i].z[w];
      if (rows_x) rows_x[(n + i) * MW + w] = st->s[i].x[w];
      if (rows_z) rows_z[(n + i) * MW + w] = st->s[i].z[w];
    }
    if (rows_r) {
      rows_r[i] = (uint8_t)st->d[i].r;
      rows_r[n + i] = (uint8_t)st->s[i].r;
    }
  }
  *n_keys = st->ne;
  for (size_t i = 0; i < st->ne && i < keys_cap; ++i) {
    if (keys) {
      keys[i * MW] = st->e[i].k[0];
      keys[i * MW + 1] = st->e[i].k[1];
    }
    if (vals) {
      vals[2 * i] = creal(st->e[i].v);
      vals[2 * i + 1] = cimag(st->e[i].v);
    }
  }
  free(st->e);
  free(st);
  circ_free(&c);
  return OR_OK;
}

uint32_t or_count_sites(const or_op *ops, size_t n_ops, uint32_t n_qubits, const or_noise *noise, uint32_t *n_records) {
  circ c;
  int rc = circ_build(&c, ops, n_ops, n_qubits, noise, 1);
  uint32_t ns = rc ? 0 : c.n_sites;
  if (n_records) *n_records = rc ? 0 : c.n_records;
  circ_free(&c);
  return ns;
}

/* ------------------------------------------------------------------------ */
/* Projection mode: one fixed error pattern, outcomes forced, unnormalised.   */
/* ------------------------------------------------------------------------ */
static double sq_norm(const gs_state *st) { return map_norm(st); }

/* Project onto the eigenvalue m of the Hermitian Pauli P without
 * renormalising: Pi_m = (I + m P)/2 (Eq. Pi_pm). Case B leaves the pairs'
 * combination (v_a0 + m xi_a1 v_a1)/sqrt(2) in the replaced tableau's basis,
 * which is Pi_m |phi> expressed there. Returns status. */
static int project(gs_state *st, const pauli *P, int m, double tau_rel) {
  uint64_t beta[MW], gamma[MW];
  int ce;
  if (decompose(st, P, beta, gamma, &ce)) return OR_ST_ERROR;
  if ((beta[0] | beta[1]) == 0) {
    if (ce & 1) return OR_ST_ERROR;
    int sgn = (ce == 2);
    size_t o = 0;
    for (size_t i = 0; i < st->ne; ++i) {
      uint64_t t[MW];
      for (int w = 0; w < MW; ++w) t[w] = gamma[w] & st->e[i].k[w];
      int lam_neg = (popc2(t) & 1) ^ sgn;
      if ((lam_neg ? -1 : +1) == m) st->e[o++] = st->e[i];
    }
    st->ne = o;
    normalize_map(st, tau_rel * sq_norm(st));
    return OR_ST_OK;
  }
  int n = st->n, p = -1;
  for (int i = 0; i < n; ++i)
    if (getbit(beta, i)) {
      p = i;
      break;
    }
  uint64_t J[MW] = {beta[0], beta[1]};
  flipbit(J, p);
  pauli sp_ = row_to_pauli(&st->s[p]);
  for (int j = 0; j < n; ++j)
    if (getbit(J, j)) {
      pauli sj = row_to_pauli(&st->s[j]);
      pauli prod = pauli_mul(&sj, &sp_);
      if (pauli_to_row(&prod, &st->s[j])) return OR_ST_ERROR;
    }
  pauli dp = row_to_pauli(&st->d[p]);
  for (int j = 0; j < n; ++j)
    if (getbit(J, j)) {
      pauli dj = row_to_pauli(&st->d[j]);
      dp = pauli_mul(&dp, &dj);
    }
  if (pauli_to_row(&dp, &st->d[p])) return OR_ST_ERROR;
  for (size_t i = 0; i < st->ne; ++i)
    if (getbit(st->e[i].k, p))
      for (int w = 0; w < MW; ++w) st->e[i].k[w] ^= J[w];
  qsort(st->e, st->ne, sizeof(entry), cmp_entry);
  uint64_t beta2[MW], gamma2[MW];
  int ce2;
  if (decompose(st, P, beta2, gamma2, &ce2)) return OR_ST_ERROR;
  /* combine each a0 with a1 = a0 ^ e_p: new value (v0 + m xi_a1 v1)/sqrt(2) at a0 */
  size_t n0 = st->ne;
  entry *out = (entry *)malloc((n0 + 1) * sizeof(entry));
  if (!out) return OR_ST_ERROR;
  size_t no = 0;
  for (size_t i = 0; i < n0; ++i) {
    entry a0 = st->e[i];
    int hi = getbit(a0.k, p);
    if (hi) flipbit(a0.k, p);
    uint64_t a1k[MW] = {a0.k[0], a0.k[1]};
    flipbit(a1k, p);
    double complex add = hi ? (double)m * xi_of(ce2, gamma2, a1k) * st->e[i].v : st->e[i].v;
    size_t f = no;
    for (size_t t = 0; t < no; ++t)
      if (cmp_entry(&out[t], &a0) == 0) {
        f = t;
        break;
      }
    if (f == no) {
      out[no] = a0;
      out[no].v = 0.0;
      no++;
    }
    out[f].v += add / sqrt(2.0);
  }
  memcpy(st->e, out, no * sizeof(entry));
  st->ne = no;
  free(out);
  row old_sp = st->s[p];
  pauli osp = row_to_pauli(&old_sp);
  for (int j = 0; j < n; ++j)
    if (j != p && getbit(gamma2, j)) {
      pauli dj = row_to_pauli(&st->d[j]);
      pauli prod = pauli_mul(&dj, &osp);
      if (pauli_to_row(&prod, &st->d[j])) return OR_ST_ERROR;
    }
  st->d[p] = old_sp;
  row newsp;
  if (pauli_to_row(P, &newsp)) return OR_ST_ERROR;
  if (m == -1) newsp.r ^= 1;
  st->s[p] = newsp;
  normalize_map(st, tau_rel * sq_norm(st));
  return OR_ST_OK;
}

/* Outcome of a measurement of P that must be deterministic: +1 / -1, or 0 if
 * the state is not an eigenstate (case B, or eigenvalues that disagree). */
static int deterministic_outcome(const gs_state *st, const pauli *P) {
  uint64_t beta[MW], gamma[MW];
  int ce;
  if (decompose(st, P, beta, gamma, &ce)) return 0;
  if ((beta[0] | beta[1]) != 0 || (ce & 1)) return 0;
  int sgn = (ce == 2), first = -1;
  for (size_t i = 0; i < st->ne; ++i) {
    uint64_t t[MW];
    for (int w = 0; w < MW; ++w) t[w] = gamma[w] & st->e[i].k[w];
    int lam_neg = (popc2(t) & 1) ^ sgn;
    if (first < 0) first = lam_neg;
    else if (first != lam_neg) return 0;
  }
  return first ? -1 : +1;
}

int or_project(const or_op *ops, size_t n_ops, uint32_t n_qubits, const or_noise *noise, uint32_t cap, uint64_t seed,
               uint64_t pattern, const double *theta, uint32_t n_theta, int64_t shift_op, double shift, double *n_acc,
               double *n_fid) {
  circ c;
  int rc = circ_build(&c, ops, n_ops, n_qubits, noise, cap);
  if (rc) {
    circ_free(&c);
    return OR_ST_ERROR;
  }
  /* record roles: 1 post-selected (single-record detector), 2 fidelity (observable), 3 unsupported */
  uint8_t *role = (uint8_t *)calloc(c.n_records + 1, 1);
  uint8_t *target = (uint8_t *)calloc(c.n_records + 1, 1);
  gs_state *st = (gs_state *)calloc(1, sizeof(gs_state));
  if (!role || !target || !st) {
    free(role); free(target); free(st); circ_free(&c);
    return OR_ST_ERROR;
  }
  int chain = 0;
  for (size_t i = 0; i < n_ops; ++i) {
    const or_op *o = &ops[i];
    if (o->op == OR_DETECTOR) {
      int single = o->rec[0] >= 0 && o->rec[1] < 0 && !(o->flags & OR_FLAG_CHAIN) && !chain;
      for (int r = 0; r < 2; ++r)
        if (o->rec[r] >= 0) {
          if (single) {
            role[o->rec[r]] = 1;
            target[o->rec[r]] = (o->flags & OR_FLAG_INVERT) ? 1 : 0;
          } else {
            role[o->rec[r]] = 3;
          }
        }
      chain = (o->flags & OR_FLAG_CHAIN) != 0;
    } else if (o->op == OR_OBSERVABLE) {
      for (int r = 0; r < 2; ++r)
        if (o->rec[r] >= 0 && role[o->rec[r]] == 0) role[o->rec[r]] = 2;
      chain = (o->flags & OR_FLAG_CHAIN) != 0;
    }
  }
  const double tau_rel = 1e-20;
  init_state(st, c.n);
  noise_stream ns = {0, 0, UINT32_MAX, 0};
  next_error(&c, seed, pattern, &ns);
  uint64_t rb[64];
  memset(rb, 0, sizeof rb);
  uint32_t nrec = 0;
  int status = OR_ST_OK, seen_fid = 0;
  *n_acc = *n_fid = 0.0;
  for (size_t i = 0; i < n_ops && status == OR_ST_OK; ++i) {
    const or_op *o = &ops[i];
    int op = o->op;
    status = apply_error_if_due(st, &c, seed, pattern, &ns, c.pre_site[i], i, NULL, NULL);
    if (status) break;
    switch (op) {
      case OR_H: case OR_S: case OR_SDAG: case OR_X: case OR_Y: case OR_Z: case OR_CX: case OR_CZ:
        apply_clifford(st, op, (int)o->q0, (int)o->q1);
        break;
      case OR_T: case OR_TDAG: case OR_RZ: {
        double complex a, b;
        double ang = 0.0;
        if (op == OR_RZ) {
          ang = o->angle;
          if (theta && o->pad > 0 && o->pad <= n_theta) ang = ((o->flags & 1) ? -1.0 : 1.0) * theta[o->pad - 1];
        } else {
          ang = (op == OR_T) ? kPi / 4.0 : -kPi / 4.0;
        }
        if (op == OR_RZ) {
          if ((int64_t)i == shift_op) ang += shift;
          a = cos(ang / 2.0);
          b = -I * sin(ang / 2.0);
        } else {
          double complex w = cexp(I * ((op == OR_T) ? kPi : -kPi) / 4.0);
          a = (1.0 + w) / 2.0;
          b = (1.0 - w) / 2.0;
        }
        int r = apply_rot_tau(st, &c, (int)o->q0, a, b, tau_rel * sq_norm(st), NULL);
        if (r) status = r;
        break;
      }
      case OR_M: case OR_R: case OR_MR: case OR_MPP: {
        if (op == OR_MPP && (o->flags & OR_MPP_MORE)) break;
        pauli Z = (op == OR_MPP) ? mpp_product(ops, mpp_chain_start(ops, i), i) : pauli_single(3, (int)o->q0);
        int m;
        if (op == OR_R) {
          m = deterministic_outcome(st, &Z);
          if (m == 0) {
            status = OR_ST_ERROR;
            break;
          }
        } else {
          int rl = role[nrec];
          if (rl == 1) m = target[nrec] ? -1 : +1;
          else if (rl == 2) {
            if (!seen_fid) {
              *n_acc = sq_norm(st);
              seen_fid = 1;
            }
            m = +1;
          } else {
            status = OR_ST_ERROR;
            break;
          }
          int r = project(st, &Z, m, tau_rel);
          if (r) {
            status = r;
            break;
          }
          if (m == -1) flipbit(rb, (int)nrec);
          nrec++;
        }
        if ((op == OR_R || op == OR_MR) && m == -1) {
          pauli X = pauli_single(1, (int)o->q0);
          if (apply_pauli(st, &X, NULL)) status = OR_ST_ERROR;
        }
        break;
      }
      case OR_CPAULI: {
        int par = 0;
        for (int r = 0; r < 2; ++r)
          if (o->rec[r] >= 0) par ^= getbit(rb, o->rec[r]);
        if (par && (o->flags & 3)) {
          pauli q = pauli_single(o->flags & 3, (int)o->q0);
          if (apply_pauli(st, &q, NULL)) status = OR_ST_ERROR;
        }
        break;
      }
      default:
        break;
    }
    if (status) break;
    if (st->ne > c.cap) {
      status = OR_ST_OVERFLOW;
      break;
    }
    status = apply_error_if_due(st, &c, seed, pattern, &ns, c.post_site[i], i, NULL, NULL);
  }
  if (status == OR_ST_OK) {
    *n_fid = sq_norm(st);
    if (!seen_fid) *n_acc = *n_fid;
    if (!(*n_acc > 0.0)) status = 4; /* zero acceptance */
  }
  free(role); free(target); free(st->e); free(st); circ_free(&c);
  return status;
}

/* The error pattern of shot `pattern`: every accepted error site and its
 * Pauli code, in site order, from the same noise stream as or_run. */
int or_errors(const or_op *ops, size_t n_ops, uint32_t n_qubits, const or_noise *noise, uint64_t seed,
              uint64_t pattern, uint32_t *sites, uint32_t *codes, uint32_t max_out) {
  circ c;
  int rc = circ_build(&c, ops, n_ops, n_qubits, noise, 1);
  if (rc) {
    circ_free(&c);
    return -1;
  }
  noise_stream ns = {0, 0, UINT32_MAX, 0};
  next_error(&c, seed, pattern, &ns);
  uint32_t k = 0;
  while (ns.site != UINT32_MAX) {
    uint32_t code = (uint32_t)error_code(&c, ns.site, ns.word2);
    if (k < max_out) {
      sites[k] = ns.site;
      codes[k] = code;
    }
    k++;
    next_error(&c, seed, pattern, &ns);
  }
  circ_free(&c);
  return (int)k;
}
