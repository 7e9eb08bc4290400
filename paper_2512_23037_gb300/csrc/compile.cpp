// compile.cpp -- host compiler: op list + noise model -> per-shot device program.
//
// One pass over the circuit evolves the X/Z words of the tableau (the part
// that is the same in every shot), accumulates each Clifford gate's sign
// flips into XOR masks, numbers the noise sites of the uniform depolarizing
// model (Sec. III of arxiv 2512.23037) and emits one event per non-Clifford
// step: T/T^dag/Rz (Eq. T_gate), Z measurement (Theorem 1 (2)), conditional
// Paulis, parity checks.
//
// Clifford conjugation is derived from each gate's images of X and Z on its
// qubits (U X U^dag, U Z U^dag); the image of any row follows by Pauli
// multiplication, and its sign bit at zero input sign is the XOR mask entry.
#include "compile.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace soft {
namespace {

inline int pc(uint64_t v) { return __builtin_popcountll(v); }

// i^e X^x Z^z on n <= 128 qubits.
struct Pz {
  uint64_t x[2] = {0, 0}, z[2] = {0, 0};
  int e = 0;
};
struct Row {
  uint64_t x[2] = {0, 0}, z[2] = {0, 0};
};

Pz pmul(const Pz &a, const Pz &b) {
  Pz o;
  int t = 0;
  for (int w = 0; w < 2; ++w) {
    o.x[w] = a.x[w] ^ b.x[w];
    o.z[w] = a.z[w] ^ b.z[w];
    t += pc(a.z[w] & b.x[w]);
  }
  o.e = (a.e + b.e + 2 * t) & 3;
  return o;
}

// The Hermitian Pauli of a row with sign bit 0.
Pz herm(const Row &r) {
  Pz p;
  for (int w = 0; w < 2; ++w) {
    p.x[w] = r.x[w];
    p.z[w] = r.z[w];
  }
  p.e = (pc(r.x[0] & r.z[0]) + pc(r.x[1] & r.z[1])) & 3;
  return p;
}

// Sign bit of a Hermitian Pauli written i^e X^x Z^z; -1 if not Hermitian.
int sign_bit(const Pz &p) {
  int d = (p.e - pc(p.x[0] & p.z[0]) - pc(p.x[1] & p.z[1])) & 3;
  return (d & 1) ? -1 : (d >> 1);
}

Row row_of(const Pz &p) {
  Row r;
  for (int w = 0; w < 2; ++w) {
    r.x[w] = p.x[w];
    r.z[w] = p.z[w];
  }
  return r;
}

inline int bit(const uint64_t *v, uint32_t i) { return (int)((v[i >> 6] >> (i & 63)) & 1u); }
inline void flip(uint64_t *v, uint32_t i) { v[i >> 6] ^= 1ull << (i & 63); }

// Local two-qubit Pauli i^e X^x Z^z (bit 0 = first qubit, bit 1 = second).
struct L2 {
  uint32_t x, z;
  int e;
};
L2 l2mul(L2 a, L2 b) { return {a.x ^ b.x, a.z ^ b.z, (a.e + b.e + 2 * pc(a.z & b.x)) & 3}; }

// Row update table: input nibble (xa, za, xb, zb) -> output nibble, sign flip.
struct GateTab {
  uint8_t out[16];
  uint8_t flipb[16];
};

GateTab make_tab(L2 iXa, L2 iZa, L2 iXb, L2 iZb) {
  GateTab t{};
  for (uint32_t in = 0; in < 16; ++in) {
    uint32_t xa = in & 1, za = (in >> 1) & 1, xb = (in >> 2) & 1, zb = (in >> 3) & 1;
    L2 acc{0, 0, (int)((xa & za) + (xb & zb))};
    if (xa) acc = l2mul(acc, iXa);
    if (za) acc = l2mul(acc, iZa);
    if (xb) acc = l2mul(acc, iXb);
    if (zb) acc = l2mul(acc, iZb);
    int d = (acc.e - pc(acc.x & acc.z)) & 3;
    t.out[in] = (uint8_t)((acc.x & 1) | ((acc.z & 1) << 1) | (((acc.x >> 1) & 1) << 2) | (((acc.z >> 1) & 1) << 3));
    t.flipb[in] = (uint8_t)((d >> 1) | ((d & 1) << 7));  // bit 7 marks an impossible odd phase
  }
  return t;
}

struct Tabs {
  GateTab g[8];
  Tabs() {
    const L2 Xa{1, 0, 0}, Za{0, 1, 0}, Xb{2, 0, 0}, Zb{0, 2, 0};
    g[SOFT_H] = make_tab(Za, Xa, Xb, Zb);
    g[SOFT_S] = make_tab(L2{1, 1, 1}, Za, Xb, Zb);       // X -> Y
    g[SOFT_S_DAG] = make_tab(L2{1, 1, 3}, Za, Xb, Zb);   // X -> -Y
    g[SOFT_X] = make_tab(Xa, L2{0, 1, 2}, Xb, Zb);       // Z -> -Z
    g[SOFT_Y] = make_tab(L2{1, 0, 2}, L2{0, 1, 2}, Xb, Zb);
    g[SOFT_Z] = make_tab(L2{1, 0, 2}, Za, Xb, Zb);       // X -> -X
    g[SOFT_CX] = make_tab(L2{3, 0, 0}, Za, Xb, L2{0, 3, 0});        // Xa -> XaXb, Zb -> ZaZb
    g[SOFT_CZ] = make_tab(L2{1, 2, 0}, Za, L2{2, 1, 0}, Zb);        // Xa -> XaZb, Xb -> ZaXb
  }
};
const Tabs &tabs() {
  static Tabs t;
  return t;
}

struct Tableau {
  uint32_t n = 0;
  std::vector<Row> d, s;
  uint64_t pend_d[2] = {0, 0}, pend_s[2] = {0, 0};  // sign XOR since the last event

  void init(uint32_t nq) {
    n = nq;
    d.assign(n, Row{});
    s.assign(n, Row{});
    for (uint32_t i = 0; i < n; ++i) {
      flip(d[i].x, i);
      flip(s[i].z, i);
    }
  }

  // (bits replaced and sign flips applied without data-dependent branches)
  static int apply_row(const GateTab &t, Row &r, uint32_t a, uint32_t b, bool two) {
    const uint32_t wa = a >> 6, sa = a & 63, wb = b >> 6, sb = b & 63;
    uint32_t in = (uint32_t)((r.x[wa] >> sa) & 1u) | ((uint32_t)((r.z[wa] >> sa) & 1u) << 1);
    if (two) in |= ((uint32_t)((r.x[wb] >> sb) & 1u) << 2) | ((uint32_t)((r.z[wb] >> sb) & 1u) << 3);
    const uint64_t o = t.out[in];
    r.x[wa] = (r.x[wa] & ~(1ull << sa)) | ((o & 1u) << sa);
    r.z[wa] = (r.z[wa] & ~(1ull << sa)) | (((o >> 1) & 1u) << sa);
    if (two) {
      r.x[wb] = (r.x[wb] & ~(1ull << sb)) | (((o >> 2) & 1u) << sb);
      r.z[wb] = (r.z[wb] & ~(1ull << sb)) | (((o >> 3) & 1u) << sb);
    }
    return t.flipb[in];
  }

  // false if a row met an odd phase (impossible for a valid tableau; the compile stops)
  bool gate(int op, uint32_t a, uint32_t b) {
    const GateTab &t = tabs().g[op];
    const bool two = (op == SOFT_CX || op == SOFT_CZ);
    int bad = 0;
    for (uint32_t i = 0; i < n; ++i) {
      const int fd = apply_row(t, d[i], a, b, two);
      const int fs = apply_row(t, s[i], a, b, two);
      bad |= fd | fs;
      pend_d[i >> 6] ^= (uint64_t)(fd & 1) << (i & 63);
      pend_s[i >> 6] ^= (uint64_t)(fs & 1) << (i & 63);
    }
    return !(bad & 0x80);
  }

  // Q = i^e0 d_beta s_gamma at zero signs. NW: the 64-bit words in use. Bits are set
  // without branches and the product runs over the set bits in increasing order,
  // accumulating X, Z and the phase in place (the data-dependent branches and the
  // second word were most of the compile time).
  template <int NW>
  bool decompose_w(const Pz &q, uint64_t beta[2], uint64_t gamma[2], uint32_t *e0) const {
    beta[0] = beta[1] = gamma[0] = gamma[1] = 0;
    for (uint32_t i = 0; i < n; ++i) {
      int ts = 0, td = 0;
      for (int w = 0; w < NW; ++w) {
        ts += pc((q.x[w] & s[i].z[w]) ^ (q.z[w] & s[i].x[w]));
        td += pc((q.x[w] & d[i].z[w]) ^ (q.z[w] & d[i].x[w]));
      }
      beta[i >> 6] |= (uint64_t)(ts & 1) << (i & 63);
      gamma[i >> 6] |= (uint64_t)(td & 1) << (i & 63);
    }
    // acc <- acc * herm(r): phase + herm's own (popc(x & z)) + 2 popc(acc.z & r.x)
    uint64_t ax[2] = {0, 0}, az[2] = {0, 0};
    int ae = 0;
    auto mul = [&](const Row &r) {
      for (int w = 0; w < NW; ++w) {
        ae += pc(r.x[w] & r.z[w]) + 2 * pc(az[w] & r.x[w]);
        ax[w] ^= r.x[w];
        az[w] ^= r.z[w];
      }
    };
    for (int w = 0; w < NW; ++w)
      for (uint64_t m = beta[w]; m; m &= m - 1) mul(d[64 * w + __builtin_ctzll(m)]);
    for (int w = 0; w < NW; ++w)
      for (uint64_t m = gamma[w]; m; m &= m - 1) mul(s[64 * w + __builtin_ctzll(m)]);
    for (int w = 0; w < 2; ++w)
      if (ax[w] != q.x[w] || az[w] != q.z[w]) return false;
    *e0 = (uint32_t)((q.e - ae) & 3);
    return true;
  }
  bool decompose(const Pz &q, uint64_t beta[2], uint64_t gamma[2], uint32_t *e0) const {
    return n <= 64 ? decompose_w<1>(q, beta, gamma, e0) : decompose_w<2>(q, beta, gamma, e0);
  }
};

Pz single(int code, uint32_t q) {
  Pz p;
  if (code == 1 || code == 2) flip(p.x, q);
  if (code == 3 || code == 2) flip(p.z, q);
  p.e = (code == 2) ? 1 : 0;
  return p;
}

bool is1q(int op) {
  return op == SOFT_H || op == SOFT_S || op == SOFT_S_DAG || op == SOFT_X || op == SOFT_Y || op == SOFT_Z ||
         op == SOFT_T || op == SOFT_T_DAG || op == SOFT_RZ;
}
bool is2q(int op) { return op == SOFT_CX || op == SOFT_CZ; }
bool isclifford(int op) { return op <= SOFT_CZ; }

uint64_t gap_thr(double p, uint64_t g) {
  double q = -std::expm1((double)(g + 1) * std::log1p(-p));
  if (!(q > 0.0)) return 0;
  if (q >= 1.0) return UINT64_MAX;
  double t = std::ldexp(q, 64);
  if (t >= 18446744073709551615.0) return UINT64_MAX;
  return (uint64_t)t;
}

// Peephole pass: fold a reset's conditional X and a single-record detector
// into the measurement event right before them. Folding is exact when the
// folded event adds no noise sites and no Clifford sign masks in between and
// no parity chain is pending.
void fuse_events(std::vector<Ev<2>> &ev) {
  std::vector<Ev<2>> out;
  out.reserve(ev.size());
  bool chain_pending = false;
  auto quiet = [](const Ev<2> &e, const Ev<2> &prev) {
    return e.site_begin == prev.site_begin && !(e.dsd[0] | e.dsd[1] | e.dss[0] | e.dss[1]);
  };
  for (const Ev<2> &e : ev) {
    const uint32_t type = ev_type(e.w0), fl = ev_flags(e.w0);
    if (!out.empty()) {
      Ev<2> &m = out.back();
      const uint32_t mt = ev_type(m.w0), mf = ev_flags(m.w0);
      const bool is_meas = (mt == EV_MEAS_A || mt == EV_MEAS_B);
      if (is_meas && type == EV_PAULI && (fl & F_COND_LAST) && !(mf & (F_COND_LAST | F_DETECTOR)) && quiet(e, m)) {
        m.w0 |= (F_COND_LAST << 4) | (ev_e0(e.w0) << 24);
        m.xbeta[0] = e.beta[0];
        m.xbeta[1] = e.beta[1];
        m.xgamma[0] = e.gamma[0];
        m.xgamma[1] = e.gamma[1];
        continue;
      }
      if (is_meas && type == EV_PARITY && (fl & F_DETECTOR) && !(fl & F_CHAIN) && !chain_pending &&
          (mf & F_RECORD) && !(mf & F_DETECTOR) && e.a == m.b && e.b == kNoRec && quiet(e, m)) {
        m.w0 |= (F_DETECTOR << 4) | ((fl & F_INVERT) ? (F_INVERT << 4) : 0u);
        continue;
      }
    }
    if (type == EV_PARITY) chain_pending = (fl & F_CHAIN) != 0;
    out.push_back(e);
  }
  ev.swap(out);
}

}  // namespace

int compile_program(const soft_op *ops, size_t n_ops, uint32_t n, const soft_noise *noise, uint32_t cap,
                    HostProgram &P, std::string &err) {
  if (!noise || (!ops && n_ops)) {
    err = "null argument";
    return SOFT_E_ARG;
  }
  if (n == 0 || n > 128) {
    err = "n_qubits must be in 1..128";
    return SOFT_E_QUBIT_RANGE;
  }
  if (cap == 0 || cap > 65536) {
    err = "coeff_cap must be in 1..65536";
    return SOFT_E_ARG;
  }
  const double ps[4] = {noise->p1, noise->p2, noise->p_meas, noise->p_reset};
  for (double p : ps)
    if (!(p >= 0.0 && p < 1.0)) {
      err = "noise probabilities must be in [0, 1)";
      return SOFT_E_ARG;
    }
  if (noise->p_idle != 0.0) {
    err = "idle noise is not supported (p_idle must be 0)";
    return SOFT_E_UNSUPPORTED_OP;
  }
  P = HostProgram{};
  P.n = n;
  P.W = n <= 64 ? 1 : 2;
  P.cap = cap;
  P.pmax = std::fmax(std::fmax(noise->p1, noise->p2), std::fmax(noise->p_meas, noise->p_reset));
  Tableau tb;
  tb.init(n);
  bool noiseless = false;
  uint32_t nrec = 0, ord = 0;

  // kind: SITE_DEPOL1, SITE_DEPOL2, or SITE_FLIP | code << 2
  auto add_site = [&](uint32_t q0, uint32_t q1, uint32_t kind, double p) -> bool {
    const bool two = (kind & 3u) == SITE_DEPOL2;
    Site s{};
    s.dsd[0] = tb.pend_d[0];
    s.dsd[1] = tb.pend_d[1];
    s.dss[0] = tb.pend_s[0];
    s.dss[1] = tb.pend_s[1];
    s.kind = kind;
    // X_q and Z_q of each site qubit: Q = i^e d_beta s_gamma at zero signs
    uint32_t ex[2] = {0, 0}, ez[2] = {0, 0};
    for (int k = 0; k < (two ? 2 : 1); ++k) {
      uint32_t q = k == 0 ? q0 : q1;
      if (!tb.decompose(single(1, q), s.bx[k], s.gx[k], &ex[k])) return false;
      if (!tb.decompose(single(3, q), s.bz[k], s.gz[k], &ez[k])) return false;
    }
    // Phases of the other Paulis by composition. With P = i^a d_b s_c and
    // Q = i^a' d_b' s_c', PQ = i^(a + a' + 2 |c & b'|) d_(b^b') s_(c^c'): s_j
    // anticommutes with d_j only, and the d's (and the s's) commute and square to I.
    auto comp = [&](uint32_t a, const uint64_t *c, const uint64_t *b2, uint32_t a2) {
      return (a + a2 + 2u * (uint32_t)(pc(c[0] & b2[0]) + pc(c[1] & b2[1]))) & 3u;
    };
    struct One {
      uint64_t b[2], g[2];
      uint32_t e;
    };
    auto one = [&](int code, int k) -> One {  // 1 X, 2 Y = i X Z, 3 Z on site qubit k
      One o{};
      if (code == 1) o = One{{s.bx[k][0], s.bx[k][1]}, {s.gx[k][0], s.gx[k][1]}, ex[k]};
      else if (code == 3) o = One{{s.bz[k][0], s.bz[k][1]}, {s.gz[k][0], s.gz[k][1]}, ez[k]};
      else if (code == 2) {
        for (int w = 0; w < 2; ++w) {
          o.b[w] = s.bx[k][w] ^ s.bz[k][w];
          o.g[w] = s.gx[k][w] ^ s.gz[k][w];
        }
        o.e = comp(1u + ex[k], s.gx[k], s.bz[k], ez[k]);
      }
      return o;
    };
    uint32_t c0 = 0;
    for (int code = 1; code <= (two ? 15 : 3); ++code) {
      uint32_t e;
      if (!two) {
        e = one(code, 0).e;
      } else {
        const int pa = code >> 2, pb = code & 3;
        if (!pa) e = one(pb, 1).e;
        else if (!pb) e = one(pa, 0).e;
        else {
          const One A = one(pa, 0), B = one(pb, 1);
          e = comp(A.e, A.g, B.b, B.e);
        }
      }
      c0 |= (e & 3u) << (2 * code);
    }
    s.c0 = c0;
    if (p >= P.pmax) {
      s.always = 1;
      s.thin = 0xFFFFFFFFu;
    } else {
      s.always = 0;
      s.thin = (uint32_t)std::floor(std::ldexp(p / P.pmax, 32));
    }
    P.sites.push_back(s);
    return true;
  };

  auto new_event = [&](uint32_t type, uint32_t flags, uint32_t e0, uint32_t lowbit) -> Ev<2> & {
    Ev<2> e{};
    e.w0 = ev_pack(type, flags, e0, lowbit);
    e.site_begin = (uint32_t)P.sites.size();
    e.dsd[0] = tb.pend_d[0];
    e.dsd[1] = tb.pend_d[1];
    e.dss[0] = tb.pend_s[0];
    e.dss[1] = tb.pend_s[1];
    tb.pend_d[0] = tb.pend_d[1] = tb.pend_s[0] = tb.pend_s[1] = 0;
    e.a = e.b = kNoRec;
    P.ev.push_back(e);
    return P.ev.back();
  };

  auto pauli_event = [&](const Pz &Q, uint32_t flags, int32_t r0, int32_t r1) -> bool {
    uint64_t beta[2], gamma[2];
    uint32_t e0;
    if (!tb.decompose(Q, beta, gamma, &e0)) return false;
    Ev<2> &e = new_event(EV_PAULI, flags, e0, 0);
    e.a = (uint32_t)r0;
    e.b = (uint32_t)r1;
    std::memcpy(e.beta, beta, sizeof beta);
    std::memcpy(e.gamma, gamma, sizeof gamma);
    return true;
  };

  // fixed angles share entries by value; a parameterised angle gets one entry per (parameter, sign)
  auto coef_index = [&](double ar, double ai, double br, double bi, int32_t param) -> uint32_t {
    for (size_t k = 0; k < P.coefs.size(); ++k) {
      const Coef &c = P.coefs[k];
      if (param >= 0 ? P.coef_param[k] == param
                     : (P.coef_param[k] < 0 && c.a_re == ar && c.a_im == ai && c.b_re == br && c.b_im == bi))
        return (uint32_t)k;
    }
    Coef c{ar, ai, br, bi, (float)ar, (float)ai, (float)br, (float)bi};
    P.coefs.push_back(c);
    P.coef_param.push_back(param);
    return (uint32_t)(P.coefs.size() - 1);
  };
  // records read by OBSERVABLE ops (fidelity measurements of gradient runs)
  std::vector<uint8_t> observed;
  {
    uint32_t nr = 0;
    for (size_t i = 0; i < n_ops; ++i) {
      int op = ops[i].op;
      if (op == SOFT_M || op == SOFT_MR || (op == SOFT_MPP && !(ops[i].flags & SOFT_MPP_MORE))) nr++;
      if (op == SOFT_OBSERVABLE)
        for (int k = 0; k < 2; ++k)
          if (ops[i].rec[k] >= 0 && (uint32_t)ops[i].rec[k] < nr) {
            if (observed.size() <= (size_t)ops[i].rec[k]) observed.resize(ops[i].rec[k] + 1, 0);
            observed[ops[i].rec[k]] = 1;
          }
    }
  }

  // One Pauli measurement of P (Theorem 1 (2)): case A when P commutes with
  // every stabilizer row, else case B with its row operations and
  // replacement constants. Returns false on an internal inconsistency.
  auto meas_event = [&](const Pz &Pm, bool recd) -> bool {
    uint64_t beta[2], gamma[2];
    uint32_t e0;
    if (!tb.decompose(Pm, beta, gamma, &e0)) return false;
    const uint32_t fidf = (recd && nrec < observed.size() && observed[nrec]) ? F_FIDELITY : 0u;
    if ((beta[0] | beta[1]) == 0) {
      Ev<2> &e = new_event(EV_MEAS_A, (recd ? F_RECORD : 0) | fidf, e0, 0);
      std::memcpy(e.gamma, gamma, sizeof gamma);
      e.a = ord;
      e.b = recd ? nrec : 0;
      return true;
    }
    CaseB cb{};
    uint32_t p = beta[0] ? (uint32_t)__builtin_ctzll(beta[0]) : 64u + (uint32_t)__builtin_ctzll(beta[1]);
    cb.p = p;
    cb.J[0] = beta[0];
    cb.J[1] = beta[1];
    flip(cb.J, p);
    // s_j <- s_j s_p
    for (uint32_t j = 0; j < n; ++j)
      if (bit(cb.J, j)) {
        Pz prod = pmul(herm(tb.s[j]), herm(tb.s[p]));
        int sb = sign_bit(prod);
        if (sb < 0) return false;
        if (sb) flip(cb.Hs, j);
        tb.s[j] = row_of(prod);
      }
    // d_p <- d_p prod_{j in J} d_j
    {
      Pz acc = herm(tb.d[p]);
      for (uint32_t j = 0; j < n; ++j)
        if (bit(cb.J, j)) acc = pmul(acc, herm(tb.d[j]));
      int sb = sign_bit(acc);
      if (sb < 0) return false;
      cb.hdp = (uint32_t)sb;
      tb.d[p] = row_of(acc);
    }
    uint64_t b2[2];
    if (!tb.decompose(Pm, b2, cb.gamma2, &cb.e0b)) return false;
    if (b2[0] != (p < 64 ? (1ull << p) : 0) || b2[1] != (p >= 64 ? (1ull << (p - 64)) : 0)) return false;
    Row old_sp = tb.s[p];
    for (uint32_t j = 0; j < n; ++j)
      if (j != p && bit(cb.gamma2, j)) {
        flip(cb.G, j);
        Pz prod = pmul(herm(tb.d[j]), herm(old_sp));
        int sb = sign_bit(prod);
        if (sb < 0) return false;
        if (sb) flip(cb.Hd, j);
        tb.d[j] = row_of(prod);
      }
    tb.d[p] = old_sp;
    // s_p <- m P: the row of P with P's own sign bit, flipped on the device when m = -1
    const int rp = sign_bit(Pm);
    if (rp < 0) return false;
    tb.s[p] = row_of(Pm);
    cb.rP = (uint32_t)rp;
    Ev<2> &e = new_event(EV_MEAS_B, (recd ? F_RECORD : 0) | fidf, 0, 0);
    e.a = ord;
    e.b = recd ? nrec : 0;
    e.beta[0] = P.cb.size();
    P.cb.push_back(cb);
    return true;
  };

  Pz mpp_acc;                     // product of the open MPP chain's factors
  uint64_t mpp_q[2] = {0, 0};     // its qubits
  bool mpp_open = false, seen_observed = false;
  for (size_t i = 0; i < n_ops; ++i) {
    const soft_op &o = ops[i];
    int op = o.op;
    if (op > SOFT_MPP) {
      err = "unknown op code at op " + std::to_string(i);
      return SOFT_E_UNSUPPORTED_OP;
    }
    if (mpp_open && op != SOFT_MPP) {
      err = "an MPP chain is continued by a non-MPP op at op " + std::to_string(i);
      return SOFT_E_ARG;
    }
    bool needs_q = is1q(op) || is2q(op) || op == SOFT_M || op == SOFT_R || op == SOFT_MR || op == SOFT_CPAULI ||
                   op == SOFT_MPP;
    if (needs_q && o.q0 >= n) {
      err = "qubit out of range at op " + std::to_string(i);
      return SOFT_E_QUBIT_RANGE;
    }
    if (is2q(op) && (o.q1 >= n || o.q1 == o.q0)) {
      err = "bad second qubit at op " + std::to_string(i);
      return SOFT_E_QUBIT_RANGE;
    }
    const bool mpp_first = op == SOFT_MPP && !mpp_open;
    if (op == SOFT_MPP) {
      const int pa = o.flags & 3, pb = (o.flags >> 2) & 3;
      if (pa == 0 || (o.flags & ~(uint32_t)(15 | SOFT_MPP_MORE))) {
        err = "bad MPP flags at op " + std::to_string(i);
        return SOFT_E_ARG;
      }
      if (pb && (o.q1 >= n || o.q1 == o.q0)) {
        err = "bad second MPP qubit at op " + std::to_string(i);
        return SOFT_E_QUBIT_RANGE;
      }
      if (bit(mpp_q, o.q0) || (pb && bit(mpp_q, o.q1))) {
        err = "MPP chain repeats a qubit at op " + std::to_string(i);
        return SOFT_E_ARG;
      }
      if ((o.flags & SOFT_MPP_MORE) && i + 1 == n_ops) {
        err = "MPP chain left open at the end of the circuit";
        return SOFT_E_ARG;
      }
    }
    if (op == SOFT_DETECTOR && seen_observed) P.fid_ok = false;
    if (op == SOFT_DETECTOR || op == SOFT_OBSERVABLE || op == SOFT_CPAULI) {
      for (int k = 0; k < 2; ++k)
        if (o.rec[k] >= 0 && (uint32_t)o.rec[k] >= nrec) {
          err = "record reference to a future measurement at op " + std::to_string(i);
          return SOFT_E_RECORD_REF;
        }
    }
    if (op == SOFT_NOISELESS_BEGIN) noiseless = true;
    if (op == SOFT_NOISELESS_END) noiseless = false;

    if (!noiseless && noise->p_meas > 0) {
      if (op == SOFT_M || op == SOFT_MR) {
        if (!add_site(o.q0, 0, SITE_FLIP | (1u << 2), noise->p_meas)) goto internal;
      } else if (mpp_first) {
        const uint32_t fc = (o.flags & 3) == 1 ? 3u : 1u;  // anticommutes with the first factor
        if (!add_site(o.q0, 0, SITE_FLIP | (fc << 2), noise->p_meas)) goto internal;
      }
    }

    if (isclifford(op)) {
      if (!tb.gate(op, o.q0, o.q1)) goto internal;
    } else if (op == SOFT_T || op == SOFT_T_DAG || op == SOFT_RZ) {
      uint64_t beta[2], gamma[2];
      uint32_t e0;
      if (!tb.decompose(single(3, o.q0), beta, gamma, &e0)) goto internal;
      bool diag = (beta[0] | beta[1]) == 0;
      double ar, ai, br, bi;
      if (op == SOFT_RZ) {
        ar = std::cos(0.5 * o.angle);
        ai = 0.0;
        br = 0.0;
        bi = -std::sin(0.5 * o.angle);
      } else {
        // diag(1, e^{+-i pi/4}) = (1 + w)/2 I + (1 - w)/2 Z with w = e^{+-i pi/4}
        double c = std::cos(0.25 * M_PI), sn = (op == SOFT_T ? 1.0 : -1.0) * std::sin(0.25 * M_PI);
        ar = 0.5 * (1.0 + c);
        ai = 0.5 * sn;
        br = 0.5 * (1.0 - c);
        bi = -0.5 * sn;
      }
      uint32_t lowbit = 0;
      if (!diag) lowbit = beta[0] ? (uint32_t)__builtin_ctzll(beta[0]) : 64u + (uint32_t)__builtin_ctzll(beta[1]);
      int32_t param = -1;
      if (op == SOFT_RZ && o.pad > 0) {
        param = (int32_t)(((o.pad - 1) << 1) | (o.flags & 1));
        P.n_params = std::max<uint32_t>(P.n_params, o.pad);
      }
      uint32_t ci = coef_index(ar, ai, br, bi, param);
      Ev<2> &e = new_event(diag ? EV_ROT_DIAG : EV_ROT, 0, e0, lowbit);
      e.a = ci;
      e.b = param >= 0 ? (uint32_t)param : kNoRec;
      P.n_rot++;
      std::memcpy(e.beta, beta, sizeof beta);
      std::memcpy(e.gamma, gamma, sizeof gamma);
    } else if (op == SOFT_M || op == SOFT_R || op == SOFT_MR) {
      bool recd = (op != SOFT_R);
      if (recd && nrec < observed.size() && observed[nrec]) seen_observed = true;
      if (!meas_event(single(3, o.q0), recd)) goto internal;
      ord++;
      if (recd) nrec++;
      if (op == SOFT_R || op == SOFT_MR)
        if (!pauli_event(single(1, o.q0), F_COND_LAST, -1, -1)) goto internal;
    } else if (op == SOFT_MPP) {
      if (!mpp_open) mpp_acc = Pz{};
      mpp_acc = pmul(mpp_acc, single(o.flags & 3, o.q0));
      flip(mpp_q, o.q0);
      if ((o.flags >> 2) & 3) {
        mpp_acc = pmul(mpp_acc, single((o.flags >> 2) & 3, o.q1));
        flip(mpp_q, o.q1);
      }
      mpp_open = (o.flags & SOFT_MPP_MORE) != 0;
      if (!mpp_open) {
        mpp_q[0] = mpp_q[1] = 0;
        if (nrec < observed.size() && observed[nrec]) seen_observed = true;
        if (!meas_event(mpp_acc, true)) goto internal;
        ord++;
        nrec++;
      }
    } else if (op == SOFT_CPAULI) {
      int code = o.flags & 3;
      if (code) {
        if (!pauli_event(single(code, o.q0), F_COND_REC, o.rec[0], o.rec[1])) goto internal;
      }
    } else if (op == SOFT_DETECTOR || op == SOFT_OBSERVABLE) {
      uint32_t fl = (op == SOFT_DETECTOR ? F_DETECTOR : F_OBSERVABLE) | ((o.flags & SOFT_FLAG_CHAIN) ? F_CHAIN : 0) |
                    ((o.flags & SOFT_FLAG_INVERT) ? F_INVERT : 0);
      Ev<2> &e = new_event(EV_PARITY, fl, 0, 0);
      e.a = (uint32_t)o.rec[0];
      e.b = (uint32_t)o.rec[1];
    }

    if (!noiseless) {
      if (is1q(op) && noise->p1 > 0) {
        if (!add_site(o.q0, 0, SITE_DEPOL1, noise->p1)) goto internal;
      } else if (is2q(op) && noise->p2 > 0) {
        if (!add_site(o.q0, o.q1, SITE_DEPOL2, noise->p2)) goto internal;
      } else if ((op == SOFT_R || op == SOFT_MR) && noise->p_reset > 0) {
        if (!add_site(o.q0, 0, SITE_FLIP | (1u << 2), noise->p_reset)) goto internal;
      }
    }
  }
  new_event(EV_END, 0, 0, 0);
  fuse_events(P.ev);
  P.n_records = nrec;
  P.rw = nrec ? (nrec + 63) / 64 : 1;
  if (P.rw > 16) {
    err = "at most 1024 recorded measurements are supported";
    return SOFT_E_ARG;
  }
  P.n_sites = (uint32_t)P.sites.size();
  P.thr.resize(P.n_sites ? P.n_sites : 1);
  for (uint32_t g = 0; g < P.n_sites; ++g) P.thr[g] = gap_thr(P.pmax, g);
  // thr increases with g, so the first g with U < thr[g] for every U of a bucket of the top
  // bits lies between the bucket's entry and the next one's
  P.thr_tab.assign((1u << kThrTabBits) + 1u, P.n_sites);
  for (uint32_t b = 0; b < (1u << kThrTabBits); ++b) {
    const uint64_t U = (uint64_t)b << (64 - kThrTabBits);
    P.thr_tab[b] = (uint32_t)(std::upper_bound(P.thr.begin(), P.thr.begin() + P.n_sites, U) - P.thr.begin());
  }
  P.site_ev.assign(P.thr.size(), (uint32_t)P.ev.size());
  {
    uint32_t e = 0;
    for (uint32_t s = 0; s < P.n_sites; ++s) {
      while (e < P.ev.size() && P.ev[e].site_begin <= s) ++e;
      P.site_ev[s] = e;
    }
  }
  P.fin_x.assign(4 * (size_t)n, 0);
  P.fin_z.assign(4 * (size_t)n, 0);
  for (uint32_t i = 0; i < n; ++i)
    for (int w = 0; w < 2; ++w) {
      P.fin_x[2 * i + w] = tb.d[i].x[w];
      P.fin_z[2 * i + w] = tb.d[i].z[w];
      P.fin_x[2 * (n + i) + w] = tb.s[i].x[w];
      P.fin_z[2 * (n + i) + w] = tb.s[i].z[w];
    }
  return SOFT_OK;
internal:
  err = "internal tableau inconsistency";
  return SOFT_E_ARG;
}

}  // namespace soft
