// adjoint.cu -- post-selected output fidelity of fixed error patterns and its
// gradient with respect to the Rz angles, by a forward projection pass and an
// adjoint (reverse) sweep, one warp per pattern.
//
// A pattern is the noise draws of one shot index. Its circuit is run with
// every detector measurement projected onto the passing outcome and every
// fidelity measurement (a record read by an OBSERVABLE) onto 0, without
// renormalising (Pi_m = (I + m P)/2, Eq. Pi_pm). With phi_pre the state just
// before the first fidelity measurement and phi_end the final state,
//   N_acc = |phi_pre|^2,  N_fid = |phi_end|^2,  F = N_fid / N_acc.
// Each Rz(s theta_k) = cos(s theta_k / 2) I - i sin(s theta_k / 2) Z_q
// (Eq. T_gate with a general angle) has d/dtheta_k = s (-i/2) Z_q Rz, so for
// N = |A psi|^2
//   dN/dtheta_k = sum over its gates of s Im <lambda| Z_q |phi>,
// with phi the state right after the gate and lambda the adjoint state there
// (lambda = A_after^dagger phi_out, swept backwards from the end). Both
// vectors live in the same GS basis at every step (Sec. II-C): the basis is
// orthonormal, so adjoints are conjugate transposes of the coefficient maps.
//
// The maps live in registers (lane i holds entry i) while they have at most
// 32 entries. A pattern that needs more is listed and rerun by a second launch
// whose maps live in shared memory (up to kWideCap entries); beyond that it
// ends UNSUPPORTED.
#include <cooperative_groups.h>

#include <type_traits>

#include "adjoint.cuh"
#include "device_common.cuh"

namespace cg = cooperative_groups;

namespace soft {
namespace {

using namespace dev;

enum : uint8_t { G_OK = 0, G_ZERO = 1, G_UNSUPPORTED = 2, G_ERROR = 3, G_WIDE = 4 /* rerun wide */ };
constexpr uint32_t kWideCap = 256;  // entries of a shared-memory map

// shared memory per warp: 64 staging keys and values, the record words
__host__ __device__ inline size_t smem_per_warp(int fp32, uint32_t W, uint32_t rw) {
  const size_t v = fp32 ? 8 : 16;
  return ((64 * v + 64 * (size_t)W * 8 + (size_t)rw * 8) + 15) & ~(size_t)15;
}
constexpr uint32_t kMaxErr = 256;

template <int W>
struct ErrRec {
  uint32_t ev, site, code, pad;
  uint64_t sd[W], ss[W];
};

// Per-warp tape: the map after every rotation (`slot` entries each), the sign
// words after every event's Clifford XOR, outcome bits, the applied errors.
template <typename R, int W>
struct TapeLayout {
  size_t keys, vals, nnz, signs, bits, errs, total;
  uint32_t slot;
  __host__ __device__ TapeLayout(uint32_t n_rot, uint32_t n_events, uint32_t slot_entries = 32) {
    slot = slot_entries;
    size_t o = 0;
    keys = o;
    o += (size_t)n_rot * slot * W * 8;
    vals = o;
    o += (size_t)n_rot * slot * sizeof(Cx<R>);
    nnz = o;
    o += ((size_t)n_rot * 4 + 15) & ~(size_t)15;
    signs = o;
    o += (size_t)n_events * 2 * W * 8;
    bits = o;
    o += ((size_t)(n_events + 63) / 64) * 8;
    errs = o;
    o += (size_t)kMaxErr * sizeof(ErrRec<W>);
    total = (o + 255) & ~(size_t)255;
  }
};

template <typename R, int W>
struct RMap {
  Key<W> k;
  Cx<R> v;
  uint32_t n;
};
// A map in shared memory: n entries, key i at k[i * W ...], value v[i].
template <typename R, int W>
struct SMap {
  uint64_t *k;
  Cx<R> *v;
  uint32_t n;
};
// Wide mode shared memory per warp: four maps (phi, pre, lambda, a tape read),
// 2 kWideCap staging entries, the record words.
__host__ __device__ inline size_t wide_entry_bytes(int fp32, uint32_t W) { return (size_t)W * 8 + (fp32 ? 8 : 16); }
__host__ __device__ inline size_t wide_smem_per_warp(int fp32, uint32_t W, uint32_t rw) {
  return ((6 * (size_t)kWideCap * wide_entry_bytes(fp32, W) + (size_t)rw * 8) + 15) & ~(size_t)15;
}

template <typename R, int W, bool Wide = false>
struct GradWarp {
  using Tile = cg::thread_block_tile<32>;
  using Map = typename std::conditional<Wide, SMap<R, W>, RMap<R, W>>::type;
  // a capacity failure: listed for the wide rerun, or final in wide mode
  static constexpr uint8_t kCapFail = Wide ? G_UNSUPPORTED : G_WIDE;
  const Tile &t;
  const GradParams &P;
  const uint32_t lane;
  uint64_t *skeys;  // staging: 64 (wide: 2 kWideCap) keys x W words (shared)
  Cx<R> *svals;     // staging values (shared)
  uint64_t *rec;    // record bits (shared)
  unsigned char *tape;
  TapeLayout<R, W> L;   // this warp's tape
  TapeLayout<R, W> PL;  // the shared noiseless prefix tape (32-entry slots)
  uint64_t shot;
  uint64_t sd[W], ss[W];
  uint32_t nxt, cur, kblk, w2, n_err;
  uint8_t status;
  // forward projection run
  Map phi, pre;
  Map lam_store, phk_store;  // wide mode: the sweep's adjoint map and tape reads
  uint32_t r, ev_f, rot_before_f;
  bool seen_f, done_empty;
  double n_acc;
  int lastm;
  uint32_t ev0 = 0, r0 = 0;  // first event / rotation this pattern computes itself

  __device__ GradWarp(const Tile &tile, const GradParams &p, unsigned char *smem_base, unsigned char *tape_base)
      : t(tile), P(p), lane(tile.thread_rank()), L(p.n_rot, p.n_events, Wide ? kWideCap : 32u),
        PL(p.n_rot, p.n_events, 32u) {
    if constexpr (Wide) {
      const size_t kb = (size_t)kWideCap * W * 8, vb = (size_t)kWideCap * sizeof(Cx<R>);
      unsigned char *b = smem_base;
      Map *maps[4] = {&phi, &pre, &lam_store, &phk_store};
      for (int m = 0; m < 4; ++m) {
        maps[m]->k = reinterpret_cast<uint64_t *>(b);
        maps[m]->v = reinterpret_cast<Cx<R> *>(b + kb);
        maps[m]->n = 0;
        b += kb + vb;
      }
      skeys = reinterpret_cast<uint64_t *>(b);
      svals = reinterpret_cast<Cx<R> *>(b + 2 * kb);
      rec = reinterpret_cast<uint64_t *>(b + 2 * kb + 2 * vb);
    } else {
      svals = reinterpret_cast<Cx<R> *>(smem_base);
      skeys = reinterpret_cast<uint64_t *>(smem_base + 64 * sizeof(Cx<R>));
      rec = reinterpret_cast<uint64_t *>(smem_base + 64 * sizeof(Cx<R>) + 64 * W * 8);
    }
    tape = tape_base;
  }

  // ------------------------------------------------------------- shared-memory maps (wide mode)
  // Every lane walks entries lane, lane + 32, ...; lookups scan the map.
  __device__ __forceinline__ Key<W> smk(const SMap<R, W> &m, uint32_t i) const {
    Key<W> k;
#pragma unroll
    for (int w = 0; w < W; ++w) k.w[w] = m.k[(size_t)i * W + w];
    return k;
  }
  __device__ __forceinline__ void smk_set(SMap<R, W> &m, uint32_t i, const Key<W> &k) {
#pragma unroll
    for (int w = 0; w < W; ++w) m.k[(size_t)i * W + w] = k.w[w];
  }
  __device__ int sfind(const SMap<R, W> &m, const Key<W> &k) const {
    for (uint32_t j = 0; j < m.n; ++j)
      if (keq(smk(m, j), k)) return (int)j;
    return -1;
  }
  __device__ void copy_map(SMap<R, W> &d, const SMap<R, W> &s_) {
    for (uint32_t i = lane; i < s_.n; i += 32) {
      smk_set(d, i, smk(s_, i));
      d.v[i] = s_.v[i];
    }
    d.n = s_.n;
    t.sync();
  }
  __device__ void copy_map(RMap<R, W> &d, const RMap<R, W> &s_) { d = s_; }
  __device__ double norm2_map(const SMap<R, W> &m) const {
    double a = 0.0;
    for (uint32_t i = lane; i < m.n; i += 32) a += norm2d(m.v[i]);
    return wsum(a);
  }
  // stable compaction of the staged entries [0, n) with keep(i) into map m
  template <typename Keep>
  __device__ void sm_from_stage(SMap<R, W> &m, uint32_t n, Keep keep) {
    uint32_t out = 0;
    for (uint32_t base = 0; base < n; base += 32) {
      const uint32_t i = base + lane;
      const bool kp = i < n && keep(i);
      const uint32_t b = t.ballot(kp);
      if (kp) {
        const uint32_t d = out + lanes_below(b);
        smk_set(m, d, skey2(i));
        m.v[d] = svals[i];
      }
      out += __popc(b);
    }
    m.n = out;
    t.sync();
  }
  __device__ __forceinline__ void skey2_set(uint32_t i, const Key<W> &k) {
#pragma unroll
    for (int w = 0; w < W; ++w) skeys[(size_t)w * 2 * kWideCap + i] = k.w[w];
  }
  __device__ __forceinline__ Key<W> skey2(uint32_t i) const {
    Key<W> r_;
#pragma unroll
    for (int w = 0; w < W; ++w) r_.w[w] = skeys[(size_t)w * 2 * kWideCap + i];
    return r_;
  }
  // map -> stage (all entries), then back with the relative prune
  __device__ void prune_rel(SMap<R, W> &m) {
    const double thr = P.tau_rel * norm2_map(m);
    for (uint32_t i = lane; i < m.n; i += 32) {
      skey2_set(i, smk(m, i));
      svals[i] = m.v[i];
    }
    t.sync();
    sm_from_stage(m, m.n, [&](uint32_t i) { return norm2d(svals[i]) >= thr; });
  }
  __device__ void pauli(SMap<R, W> &m, const uint64_t *beta, const uint64_t *gamma, uint32_t e) {
    for (uint32_t i = lane; i < m.n; i += 32) {
      const Key<W> k = smk(m, i);
      m.v[i] = ipow(m.v[i], e + 2u * kpar(k, gamma));
      smk_set(m, i, kxor(k, beta));
    }
    t.sync();
  }
  __device__ void pauli_adj(SMap<R, W> &m, const uint64_t *beta, const uint64_t *gamma, uint32_t e) {
    for (uint32_t i = lane; i < m.n; i += 32) {
      const Key<W> a = kxor(smk(m, i), beta);
      m.v[i] = ipow(m.v[i], (4u - (e & 3u)) + 2u * kpar(a, gamma));
      smk_set(m, i, a);
    }
    t.sync();
  }
  // a I + b Z_q (beta != 0): stage [0, n) the updated old entries, [n, n + nA) the new ones
  __device__ bool rot(SMap<R, W> &m, uint32_t e, uint32_t lowbit, Cx<R> a, Cx<R> b, const uint64_t *beta,
                      const uint64_t *gamma) {
    (void)lowbit;
    const uint32_t n = m.n;
    uint32_t nA = 0;
    for (uint32_t base = 0; base < n; base += 32) {
      const uint32_t i = base + lane;
      bool app = false;
      Key<W> pk;
      Cx<R> tb{0, 0};
      if (i < n) {
        const Key<W> k = smk(m, i);
        pk = kxor(k, beta);
        const int j = sfind(m, pk);
        Cx<R> nv = cmul(a, m.v[i]);
        if (j >= 0) nv = cadd(nv, cmul(b, ipow(m.v[j], e + 2u * kpar(pk, gamma))));
        else {
          tb = cmul(b, ipow(m.v[i], e + 2u * kpar(k, gamma)));
          app = true;
        }
        skey2_set(i, k);
        svals[i] = nv;
      }
      const uint32_t bal = t.ballot(app);
      if (app) {
        const uint32_t d = n + nA + lanes_below(bal);
        if (d < 2 * kWideCap) {
          skey2_set(d, pk);
          svals[d] = tb;
        }
      }
      nA += __popc(bal);
    }
    t.sync();
    if (n + nA > kWideCap) return false;
    double tot = 0.0;
    for (uint32_t i = lane; i < n + nA; i += 32) tot += norm2d(svals[i]);
    const double thr = P.tau_rel * wsum(tot);
    sm_from_stage(m, n + nA, [&](uint32_t i) { return norm2d(svals[i]) >= thr; });
    return true;
  }
  __device__ void rot_diag(SMap<R, W> &m, uint32_t e, Cx<R> a, Cx<R> b, const uint64_t *gamma) {
    for (uint32_t i = lane; i < m.n; i += 32)
      m.v[i] = cadd(cmul(a, m.v[i]), cmul(b, ipow(m.v[i], e + 2u * kpar(smk(m, i), gamma))));
    t.sync();
    prune_rel(m);
  }
  __device__ void project_a(SMap<R, W> &m, const uint64_t *gamma, uint32_t sgn, int mm) {
    for (uint32_t i = lane; i < m.n; i += 32) {
      skey2_set(i, smk(m, i));
      svals[i] = m.v[i];
    }
    t.sync();
    sm_from_stage(m, m.n, [&](uint32_t i) { return ((kpar(skey2(i), gamma) ^ sgn) != 0u) == (mm == -1); });
    prune_rel(m);
  }
  // relabel a_j ^= a_p (j in J), then v''_{a0} = (v_{a0} + m xi_{a1} v_{a1}) / sqrt(2)
  __device__ void project_b(SMap<R, W> &m, uint32_t p, const uint64_t *J, const uint64_t *ep, const uint64_t *g2,
                            uint32_t e2, int mm) {
    for (uint32_t i = lane; i < m.n; i += 32) {
      const Key<W> k = smk(m, i);
      if (kbit(k, p)) smk_set(m, i, kxor(k, J));
    }
    t.sync();
    const R rs = (R)0.70710678118654752440;
    uint32_t out = 0;
    for (uint32_t base = 0; base < m.n; base += 32) {
      const uint32_t i = base + lane;
      bool own = false;
      Key<W> a0;
      Cx<R> nv{0, 0};
      if (i < m.n) {
        const Key<W> k = smk(m, i);
        const uint32_t hi = kbit(k, p);
        a0 = hi ? kxor(k, ep) : k;
        const int j = sfind(m, hi ? a0 : kxor(k, ep));
        Cx<R> v0{0, 0}, v1{0, 0};
        if (hi) {
          v1 = m.v[i];
          own = j < 0;  // else the a0 entry combines the pair
        } else {
          v0 = m.v[i];
          if (j >= 0) v1 = m.v[j];
          own = true;
        }
        const Cx<R> x1 = ipow(v1, e2 + 2u * kpar(kxor(a0, ep), g2));
        nv = cscale(mm == 1 ? cadd(v0, x1) : csub(v0, x1), rs);
      }
      const uint32_t b = t.ballot(own);
      if (own) {
        const uint32_t d = out + lanes_below(b);
        skey2_set(d, a0);
        svals[d] = nv;
      }
      out += __popc(b);
    }
    t.sync();
    sm_from_stage(m, out, [&](uint32_t) { return true; });
    prune_rel(m);
  }
  // adjoint of project_b: drop keys with bit p set, split each into (a0, a1), undo the relabel
  __device__ bool project_b_adj(SMap<R, W> &m, uint32_t p, const uint64_t *J, const uint64_t *ep,
                                const uint64_t *g2, uint32_t e2, int mm) {
    for (uint32_t i = lane; i < m.n; i += 32) {
      skey2_set(i, smk(m, i));
      svals[i] = m.v[i];
    }
    t.sync();
    sm_from_stage(m, m.n, [&](uint32_t i) { return !kbit(skey2(i), p); });
    if (2 * m.n > 2 * kWideCap) return false;
    const R rs = (R)0.70710678118654752440;
    const uint32_t n = m.n;
    for (uint32_t i = lane; i < n; i += 32) {
      Key<W> k0 = smk(m, i), k1 = kxor(k0, ep);
      const Cx<R> u0 = cscale(m.v[i], rs);
      const Cx<R> u1 = ipow(u0, (4u - (e2 & 3u)) + 2u * kpar(k1, g2) + (mm == -1 ? 2u : 0u));
      if (kbit(k1, p)) k1 = kxor(k1, J);
      if (kbit(k0, p)) k0 = kxor(k0, J);
      skey2_set(i, k0);
      svals[i] = u0;
      skey2_set(n + i, k1);
      svals[n + i] = u1;
    }
    t.sync();
    double tot = 0.0;
    for (uint32_t i = lane; i < 2 * n; i += 32) tot += norm2d(svals[i]);
    const double thr = P.tau_rel * wsum(tot);
    uint32_t keep_n = 0;
    for (uint32_t base = 0; base < 2 * n; base += 32) {
      const uint32_t i = base + lane;
      keep_n += __popc(t.ballot(i < 2 * n && norm2d(svals[i]) >= thr && norm2d(svals[i]) > 0.0));
    }
    if (keep_n > kWideCap) return false;
    sm_from_stage(m, 2 * n, [&](uint32_t i) { return norm2d(svals[i]) >= thr && norm2d(svals[i]) > 0.0; });
    return true;
  }
  // <lambda| Z_q |phi> = sum_a conj(lambda_{a^beta}) xi_a phi_a
  __device__ void zexp(const SMap<R, W> &lam, const SMap<R, W> &ph, const uint64_t *beta, const uint64_t *gamma,
                       uint32_t e, double *re, double *im) {
    double cr = 0.0, ci = 0.0;
    for (uint32_t i = lane; i < ph.n; i += 32) {
      const Key<W> k = smk(ph, i);
      const int j = sfind(lam, kxor(k, beta));
      if (j < 0) continue;
      const Cx<R> xp = ipow(ph.v[i], e + 2u * kpar(k, gamma));
      const Cx<R> l = lam.v[j];
      cr += (double)l.x * (double)xp.x + (double)l.y * (double)xp.y;
      ci += (double)l.x * (double)xp.y - (double)l.y * (double)xp.x;
    }
    *re = wsum(cr);
    *im = wsum(ci);
  }
  __device__ void reset_sides(const SMap<R, W> &m, const uint64_t *gamma, uint32_t sgn, bool &h0, bool &h1) {
    bool a0 = false, a1 = false;
    for (uint32_t i = lane; i < m.n; i += 32) {
      if (kpar(smk(m, i), gamma) ^ sgn) a1 = true;
      else a0 = true;
    }
    h0 = t.any(a0);
    h1 = t.any(a1);
  }
  __device__ void reset_sides(const RMap<R, W> &m, const uint64_t *gamma, uint32_t sgn, bool &h0, bool &h1) {
    const bool neg = (kpar(m.k, gamma) ^ sgn) != 0u;
    h1 = t.any(lane < m.n && neg);
    h0 = t.any(lane < m.n && !neg);
  }
  __device__ void map_init_one(SMap<R, W> &m) {
    if (lane == 0) {
      Key<W> z;
#pragma unroll
      for (int w = 0; w < W; ++w) z.w[w] = 0ull;
      smk_set(m, 0, z);
      m.v[0] = Cx<R>{(R)1, (R)0};
    }
    m.n = 1;
    t.sync();
  }
  __device__ void map_init_one(RMap<R, W> &m) {
    for (int w = 0; w < W; ++w) m.k.w[w] = 0ull;
    m.v = Cx<R>{(R)(lane == 0 ? 1 : 0), (R)0};
    m.n = 1;
  }

  // ------------------------------------------------------------- helpers
  __device__ __forceinline__ uint32_t vmask(uint32_t n) const { return n >= 32u ? 0xFFFFFFFFu : ((1u << n) - 1u); }
  __device__ __forceinline__ uint32_t lanes_below(uint32_t b) const { return __popc(b & ((1u << lane) - 1u)); }
  __device__ double wsum(double v) const {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += t.shfl_xor(v, off);
    return v;
  }
  __device__ __forceinline__ uint32_t match_key(const Key<W> &k) const {
    uint32_t m = __match_any_sync(0xFFFFFFFFu, (unsigned long long)k.w[0]);
    if (W == 2) m &= __match_any_sync(0xFFFFFFFFu, (unsigned long long)k.w[W - 1]);
    return m;
  }
  __device__ __forceinline__ Cx<R> shfl_c(Cx<R> v, uint32_t src) const {
    return Cx<R>{t.shfl(v.x, src), t.shfl(v.y, src)};
  }
  __device__ __forceinline__ void skey_set(uint32_t i, const Key<W> &k) {
#pragma unroll
    for (int w = 0; w < W; ++w) skeys[w * 64 + i] = k.w[w];
  }
  __device__ __forceinline__ Key<W> skey(uint32_t i) const {
    Key<W> r;
#pragma unroll
    for (int w = 0; w < W; ++w) r.w[w] = skeys[w * 64 + i];
    return r;
  }
  __device__ double norm2_map(const RMap<R, W> &m) const { return wsum(lane < m.n ? norm2d(m.v) : 0.0); }

  // keep the entries whose lane sets `keep`, in lane order
  __device__ void compact(RMap<R, W> &m, bool keep) {
    const uint32_t b = t.ballot(keep);
    if (b == vmask(m.n)) return;
    if (keep) {
      const uint32_t d = lanes_below(b);
      skey_set(d, m.k);
      svals[d] = m.v;
    }
    t.sync();
    m.n = __popc(b);
    if (lane < m.n) {
      m.k = skey(lane);
      m.v = svals[lane];
    }
    t.sync();
  }
  // drop |v|^2 < tau_rel |map|^2
  __device__ void prune_rel(RMap<R, W> &m) {
    const double thr = P.tau_rel * norm2_map(m);
    const bool keep = lane < m.n && norm2d(m.v) >= thr;
    compact(m, keep);
  }

  // Q: v'_{a^beta} = i^{e + 2 gamma.a} v_a
  __device__ void pauli(RMap<R, W> &m, const uint64_t *beta, const uint64_t *gamma, uint32_t e) {
    if (lane < m.n) {
      m.v = ipow(m.v, e + 2u * kpar(m.k, gamma));
      m.k = kxor(m.k, beta);
    }
  }
  // Q^dagger (the adjoint of the map above): lambda_a = i^{-e} (-1)^{gamma.a} lambda'_{a^beta}
  __device__ void pauli_adj(RMap<R, W> &m, const uint64_t *beta, const uint64_t *gamma, uint32_t e) {
    if (lane < m.n) {
      const Key<W> a = kxor(m.k, beta);
      m.v = ipow(m.v, (4u - (e & 3u)) + 2u * kpar(a, gamma));
      m.k = a;
    }
  }

  // a I + b Z_q (beta != 0); false if the result needs more than 32 entries
  __device__ bool rot(RMap<R, W> &m, uint32_t e, uint32_t lowbit, Cx<R> a, Cx<R> b, const uint64_t *beta,
                      const uint64_t *gamma) {
    const bool valid = lane < m.n;
    const Key<W> pk = kxor(m.k, beta);
    const Key<W> canon = kbit(m.k, lowbit) ? pk : m.k;
    const uint32_t partner = match_key(canon) & vmask(m.n) & ~(1u << lane);
    const uint32_t pl = partner ? (uint32_t)(__ffs(partner) - 1) : lane;
    const Cx<R> vj = shfl_c(m.v, pl);
    const bool has = valid && partner != 0u;
    const bool app = valid && !has;
    const Cx<R> src = has ? vj : m.v;
    const Cx<R> tb = cmul(b, ipow(src, e + 2u * kpar(has ? pk : m.k, gamma)));
    Cx<R> nv = cmul(a, m.v);
    if (has) nv = cadd(nv, tb);
    const uint32_t ab = t.ballot(app);
    const uint32_t nA = __popc(ab);
    if (m.n + nA > 32u) return false;
    if (app) {
      const uint32_t d = lanes_below(ab);
      skey_set(d, pk);
      svals[d] = tb;
    }
    t.sync();
    if (valid) m.v = nv;
    else if (lane < m.n + nA) {
      m.k = skey(lane - m.n);
      m.v = svals[lane - m.n];
    }
    t.sync();
    m.n += nA;
    prune_rel(m);
    return true;
  }
  __device__ void rot_diag(RMap<R, W> &m, uint32_t e, Cx<R> a, Cx<R> b, const uint64_t *gamma) {
    if (lane < m.n) m.v = cadd(cmul(a, m.v), cmul(b, ipow(m.v, e + 2u * kpar(m.k, gamma))));
    prune_rel(m);
  }

  // case A: Pi_m keeps entries with eigenvalue m of c s_gamma (c = (-1)^sgn)
  __device__ void project_a(RMap<R, W> &m, const uint64_t *gamma, uint32_t sgn, int mm) {
    const bool neg = (kpar(m.k, gamma) ^ sgn) != 0u;
    compact(m, lane < m.n && (neg == (mm == -1)));
    prune_rel(m);
  }
  // case B after the row operations: relabel a_j ^= a_p (j in J), then
  // v''_{a0} = (v_{a0} + m xi_{a1} v_{a1}) / sqrt(2), a1 = a0 ^ e_p
  __device__ void project_b(RMap<R, W> &m, uint32_t p, const uint64_t *J, const uint64_t *ep, const uint64_t *g2,
                            uint32_t e2, int mm) {
    const bool valid = lane < m.n;
    if (valid && kbit(m.k, p)) m.k = kxor(m.k, J);
    const uint32_t hi = kbit(m.k, p);
    const Key<W> a0 = hi ? kxor(m.k, ep) : m.k;
    const uint32_t partner = match_key(a0) & vmask(m.n) & ~(1u << lane);
    const uint32_t pl = partner ? (uint32_t)(__ffs(partner) - 1) : lane;
    const Cx<R> vj = shfl_c(m.v, pl);
    const bool owner = valid && (!hi || partner == 0u);
    Cx<R> v0{0, 0}, v1{0, 0};
    if (hi) v1 = m.v;
    else {
      v0 = m.v;
      if (partner) v1 = vj;
    }
    const Cx<R> x1 = ipow(v1, e2 + 2u * kpar(kxor(a0, ep), g2));
    const R rs = (R)0.70710678118654752440;
    if (owner) {
      m.v = cscale(mm == 1 ? cadd(v0, x1) : csub(v0, x1), rs);
      m.k = a0;
    }
    compact(m, owner);
    prune_rel(m);
  }
  // adjoint of project_b: lambda_{a0} = l/sqrt2, lambda_{a1} = m conj(xi_{a1}) l/sqrt2, then undo the relabel.
  // Components of lambda'' on keys with bit p set are orthogonal to the projected subspace and drop out.
  __device__ bool project_b_adj(RMap<R, W> &m, uint32_t p, const uint64_t *J, const uint64_t *ep, const uint64_t *g2,
                                uint32_t e2, int mm) {
    compact(m, lane < m.n && !kbit(m.k, p));
    const bool valid = lane < m.n;
    const R rs = (R)0.70710678118654752440;
    Key<W> k0 = m.k, k1 = kxor(m.k, ep);
    Cx<R> u0 = cscale(m.v, rs);
    // conj(xi_{a1}) = i^{-e2} (-1)^{g2.a1}
    Cx<R> u1 = ipow(u0, (4u - (e2 & 3u)) + 2u * kpar(k1, g2) + (mm == -1 ? 2u : 0u));
    if (kbit(k1, p)) k1 = kxor(k1, J);  // inverse relabel (an involution)
    if (kbit(k0, p)) k0 = kxor(k0, J);
    const uint32_t n2 = 2u * m.n;
    if (n2 > 64u) return false;
    if (valid) {
      skey_set(lane, k0);
      svals[lane] = u0;
      skey_set(m.n + lane, k1);
      svals[m.n + lane] = u1;
    }
    t.sync();
    // gather both halves, drop zeros, keep at most 32
    Key<W> ka = skey(lane), kb = skey(lane + 32 < 64 ? lane + 32 : 63);
    Cx<R> va = svals[lane], vb = svals[lane + 32 < 64 ? lane + 32 : 63];
    t.sync();
    const bool inA = lane < n2, inB = lane + 32u < n2;
    double tot = wsum((inA ? norm2d(va) : 0.0) + (inB ? norm2d(vb) : 0.0));
    const double thr = P.tau_rel * tot;
    const bool ka_keep = inA && norm2d(va) >= thr && norm2d(va) > 0.0;
    const bool kb_keep = inB && norm2d(vb) >= thr && norm2d(vb) > 0.0;
    const uint32_t ba = t.ballot(ka_keep), bb = t.ballot(kb_keep);
    const uint32_t cnt = __popc(ba) + __popc(bb);
    if (cnt > 32u) return false;
    if (ka_keep) {
      const uint32_t d = lanes_below(ba);
      skey_set(d, ka);
      svals[d] = va;
    }
    if (kb_keep) {
      const uint32_t d = __popc(ba) + lanes_below(bb);
      skey_set(d, kb);
      svals[d] = vb;
    }
    t.sync();
    m.n = cnt;
    if (lane < m.n) {
      m.k = skey(lane);
      m.v = svals[lane];
    }
    t.sync();
    return true;
  }

  // case-B sign updates: row operations (returns e2 of P = i^e2 d_p s_gamma2), then the
  // replacement with outcome mm (if mm != 0)
  __device__ uint32_t caseb_signs(const CaseB *B, int mm) {
    const uint32_t p = __ldg(&B->p);
    uint64_t J[W], g2[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
      J[w] = __ldg(&B->J[w]);
      g2[w] = __ldg(&B->gamma2[w]);
    }
    const uint32_t ssp = wbit<W>(ss, p);
    const uint32_t sdJ = wpar<W>(sd, J);
#pragma unroll
    for (int w = 0; w < W; ++w) ss[w] ^= (ssp ? J[w] : 0ull) ^ __ldg(&B->Hs[w]);
    if (sdJ ^ __ldg(&B->hdp)) wflip<W>(sd, p);
    const uint32_t e2 = (__ldg(&B->e0b) + 2u * (wbit<W>(sd, p) + wpar<W>(ss, g2))) & 3u;
    if (mm != 0) {
#pragma unroll
      for (int w = 0; w < W; ++w) sd[w] ^= (ssp ? __ldg(&B->G[w]) : 0ull) ^ __ldg(&B->Hd[w]);
      if (wbit<W>(sd, p) != ssp) wflip<W>(sd, p);
      const uint32_t newsp = (mm == -1 ? 1u : 0u) ^ __ldg(&B->rP);
      if (wbit<W>(ss, p) != newsp) wflip<W>(ss, p);
    }
    return e2;
  }

  __device__ __forceinline__ uint32_t pe(const uint64_t *beta, const uint64_t *gamma) const {
    uint32_t s = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) s += __popcll(sd[w] & beta[w]) + __popcll(ss[w] & gamma[w]);
    return s;
  }

  // ------------------------------------------------------------- noise
  __device__ void draw_next() {
    for (uint32_t guard = 0; guard <= P.n_sites; ++guard) {
      if (cur >= P.n_sites) {
        nxt = 0xFFFFFFFFu;
        return;
      }
      uint4 w = philox(P.seed, shot, 0u, kblk++);
      uint64_t U = (uint64_t)w.x | ((uint64_t)w.y << 32);
      uint32_t rem = P.n_sites - cur, lo = 0, hi = rem;
      if (P.thr_tab) {  // U's bucket bounds the answer
        const uint32_t b = (uint32_t)(U >> (64 - kThrTabBits));
        const uint32_t t0 = __ldg(&P.thr_tab[b]), t1 = __ldg(&P.thr_tab[b + 1]);
        lo = t0 < rem ? t0 : rem;
        hi = t1 < rem ? t1 : rem;
      }
      while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (U < __ldg(&P.thr[mid])) hi = mid;
        else lo = mid + 1u;
      }
      if (lo == rem) {
        cur = P.n_sites;
        nxt = 0xFFFFFFFFu;
        return;
      }
      uint32_t s = cur + lo;
      cur = s + 1u;
      const Site *st = P.sites + s;
      if (!__ldg(&st->always) && !(w.w < __ldg(&st->thin))) continue;
      nxt = s;
      w2 = w.z;
      return;
    }
    nxt = 0xFFFFFFFFu;
  }
  // beta/gamma/e of the error at site s with Pauli code `code`, signs (esd, ess) at the site
  __device__ void error_pauli(uint32_t s, uint32_t code, const uint64_t *esd, const uint64_t *ess, uint64_t *beta,
                              uint64_t *gamma, uint32_t *e) const {
    const Site *S = P.sites + s;
    const uint32_t two = (__ldg(&S->kind) & 3u) == SITE_DEPOL2;
    const uint32_t pa = two ? (code >> 2) : code, pb = two ? (code & 3u) : 0u;
    uint32_t q = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      uint64_t b = 0, g = 0;
      if (pa == 1u || pa == 2u) { b ^= __ldg(&S->bx[0][w]); g ^= __ldg(&S->gx[0][w]); }
      if (pa == 3u || pa == 2u) { b ^= __ldg(&S->bz[0][w]); g ^= __ldg(&S->gz[0][w]); }
      if (pb == 1u || pb == 2u) { b ^= __ldg(&S->bx[1][w]); g ^= __ldg(&S->gx[1][w]); }
      if (pb == 3u || pb == 2u) { b ^= __ldg(&S->bz[1][w]); g ^= __ldg(&S->gz[1][w]); }
      beta[w] = b;
      gamma[w] = g;
      q += __popcll(esd[w] & b) + __popcll(ess[w] & g);
    }
    *e = ((__ldg(&S->c0) >> (2u * code)) + 2u * q) & 3u;
  }

  // ------------------------------------------------------------- tape access
  __device__ void tape_store_phi(uint32_t r, const RMap<R, W> &m) {
    uint64_t *tk = reinterpret_cast<uint64_t *>(tape + L.keys);
    Cx<R> *tv = reinterpret_cast<Cx<R> *>(tape + L.vals);
    if (lane < m.n) {
#pragma unroll
      for (int w = 0; w < W; ++w) tk[((size_t)r * L.slot + lane) * W + w] = m.k.w[w];
      tv[(size_t)r * L.slot + lane] = m.v;
    }
    if (lane == 0) reinterpret_cast<uint32_t *>(tape + L.nnz)[r] = m.n;
  }
  __device__ void tape_store_phi(uint32_t r, const SMap<R, W> &m) {
    uint64_t *tk = reinterpret_cast<uint64_t *>(tape + L.keys);
    Cx<R> *tv = reinterpret_cast<Cx<R> *>(tape + L.vals);
    for (uint32_t i = lane; i < m.n; i += 32) {
#pragma unroll
      for (int w = 0; w < W; ++w) tk[((size_t)r * L.slot + i) * W + w] = m.k[(size_t)i * W + w];
      tv[(size_t)r * L.slot + i] = m.v[i];
    }
    if (lane == 0) reinterpret_cast<uint32_t *>(tape + L.nnz)[r] = m.n;
  }
  // the shared noiseless tape (32-entry slots) holds what precedes this pattern's first error
  __device__ __forceinline__ const unsigned char *tape_for_rot(uint32_t rr) const {
    return rr < r0 ? P.ptape : tape;
  }
  __device__ __forceinline__ const TapeLayout<R, W> &lay_for_rot(uint32_t rr) const { return rr < r0 ? PL : L; }
  __device__ __forceinline__ const unsigned char *tape_for_ev(uint32_t ev) const {
    return ev < ev0 ? P.ptape : tape;
  }
  __device__ __forceinline__ const TapeLayout<R, W> &lay_for_ev(uint32_t ev) const { return ev < ev0 ? PL : L; }
  __device__ void tape_load_phi(uint32_t r, RMap<R, W> &m) const {
    const unsigned char *tp = tape_for_rot(r);
    const TapeLayout<R, W> &ly = lay_for_rot(r);
    const uint64_t *tk = reinterpret_cast<const uint64_t *>(tp + ly.keys);
    const Cx<R> *tv = reinterpret_cast<const Cx<R> *>(tp + ly.vals);
    m.n = reinterpret_cast<const uint32_t *>(tp + ly.nnz)[r];
    if (lane < m.n) {
#pragma unroll
      for (int w = 0; w < W; ++w) m.k.w[w] = tk[((size_t)r * ly.slot + lane) * W + w];
      m.v = tv[(size_t)r * ly.slot + lane];
    }
  }
  __device__ void tape_load_phi(uint32_t r, SMap<R, W> &m) {
    const unsigned char *tp = tape_for_rot(r);
    const TapeLayout<R, W> &ly = lay_for_rot(r);
    const uint64_t *tk = reinterpret_cast<const uint64_t *>(tp + ly.keys);
    const Cx<R> *tv = reinterpret_cast<const Cx<R> *>(tp + ly.vals);
    m.n = reinterpret_cast<const uint32_t *>(tp + ly.nnz)[r];
    for (uint32_t i = lane; i < m.n; i += 32) {
#pragma unroll
      for (int w = 0; w < W; ++w) m.k[(size_t)i * W + w] = tk[((size_t)r * ly.slot + i) * W + w];
      m.v[i] = tv[(size_t)r * ly.slot + i];
    }
    t.sync();
  }
  __device__ void tape_signs_store(uint32_t ev) {
    if (lane == 0) {
      uint64_t *ts = reinterpret_cast<uint64_t *>(tape + L.signs) + (size_t)ev * 2 * W;
#pragma unroll
      for (int w = 0; w < W; ++w) {
        ts[w] = sd[w];
        ts[W + w] = ss[w];
      }
    }
  }
  __device__ void tape_signs_load(uint32_t ev) {
    const uint64_t *ts =
        reinterpret_cast<const uint64_t *>(tape_for_ev(ev) + lay_for_ev(ev).signs) + (size_t)ev * 2 * W;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      sd[w] = ts[w];
      ss[w] = ts[W + w];
    }
  }
  __device__ void tape_bit_set(uint32_t ev) {
    if (lane == 0) reinterpret_cast<uint64_t *>(tape + L.bits)[ev >> 6] |= 1ull << (ev & 63);
  }
  __device__ bool tape_bit(uint32_t ev) const {
    return (reinterpret_cast<const uint64_t *>(tape_for_ev(ev) + lay_for_ev(ev).bits)[ev >> 6] >> (ev & 63)) &
           1ull;
  }
  __device__ ErrRec<W> *errs() const { return reinterpret_cast<ErrRec<W> *>(tape + L.errs); }

  // <lambda| Z_q |phi> for the ROT event (beta, gamma, e): sum_a conj(lambda_{a^beta}) xi_a phi_a
  __device__ void zexp(const RMap<R, W> &lam, const RMap<R, W> &phi, const uint64_t *beta, const uint64_t *gamma,
                       uint32_t e, double *re, double *im) {
    if (lane < lam.n) {
      skey_set(lane, lam.k);
      svals[lane] = lam.v;
    }
    t.sync();
    double cr = 0.0, ci = 0.0;
    if (lane < phi.n) {
      const Key<W> target = kxor(phi.k, beta);
      const Cx<R> xp = ipow(phi.v, e + 2u * kpar(phi.k, gamma));  // xi_a phi_a
      for (uint32_t j = 0; j < lam.n; ++j) {
        if (keq(skey(j), target)) {
          const Cx<R> l = svals[j];
          // conj(l) * xp
          cr = (double)l.x * (double)xp.x + (double)l.y * (double)xp.y;
          ci = (double)l.x * (double)xp.y - (double)l.y * (double)xp.x;
          break;
        }
      }
    }
    t.sync();
    *re = wsum(cr);
    *im = wsum(ci);
  }

  // ------------------------------------------------------------- one pattern
  __device__ void run(uint64_t pattern, uint64_t off) {
    shot = pattern;
    status = G_OK;
    n_err = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) sd[w] = ss[w] = 0ull;
    for (uint32_t w = lane; w < P.rw; w += 32) rec[w] = 0ull;
    {
      uint64_t *bits = reinterpret_cast<uint64_t *>(tape + L.bits);
      for (uint32_t w = lane; w < (P.n_events + 63) / 64; w += 32) bits[w] = 0ull;
    }
    double *grad = P.grad + off * P.n_params;
    for (uint32_t k = lane; k < P.n_params; k += 32) grad[k] = 0.0;
    t.sync();
    fwd_init();
    cur = 0;
    kblk = 0;
    draw_next();
    if (P.psnap) load_prefix();  // every event before the first error is the noiseless run's
    for (uint32_t ev = ev0; ev < P.n_events && status == G_OK && !done_empty; ++ev) fwd_step(ev);
    double n_fid = 0.0, F = 0.0;
    if (status == G_OK) {
      n_fid = norm2_map(phi);
      if (!seen_f) {
        n_acc = n_fid;
        copy_map(pre, phi);
        ev_f = P.n_events;
        rot_before_f = r;
      }
      if (!(n_acc > 0.0)) status = G_ZERO;
      else F = n_fid / n_acc;
    }
    if (status == G_OK && n_fid > 0.0) {  // N_fid = 0: F = 0 and dF/dtheta = 0 exactly
      // sweep 1: N_fid from the end; sweep 2: N_acc from just before the first fidelity measurement
      if (!sweep(phi, P.n_events, r, grad, 1.0)) status = kCapFail;
      if (status == G_OK && !sweep(pre, ev_f, rot_before_f, grad, -F)) status = kCapFail;
      t.sync();
      for (uint32_t k = lane; k < P.n_params; k += 32) grad[k] /= n_acc;
    }
    if (status == G_WIDE) {  // rerun by the shared-memory pass; UNSUPPORTED unless it succeeds
      if (lane == 0) {
        const unsigned long long i = atomicAdd(P.wide_n, 1ull);
        if (i < P.wide_cap) P.wide_list[i] = (uint32_t)off;
      }
      status = G_UNSUPPORTED;
    }
    if (lane == 0) {
      P.status[off] = status;
      P.fid[off] = status == G_OK ? F : 0.0;
      P.pacc[off] = status == G_OK ? n_acc : 0.0;
      if (P.sums && status == G_OK) {  // ratio estimator sum N_fid / sum N_acc = sum p_acc F / sum p_acc
        atomicAdd(&P.sums[0], n_acc);
        atomicAdd(&P.sums[1], n_fid);
        atomicAdd(&P.sums[2], 1.0);
      }
    }
    if (status != G_OK)
      for (uint32_t k = lane; k < P.n_params; k += 32) grad[k] = 0.0;
    t.sync();
  }

  // One forward event of the projection run: its due errors, then the event.
  __device__ void fwd_step(uint32_t ev) {
    const Ev<W> *evs = reinterpret_cast<const Ev<W> *>(P.ev);
    {
      const Ev<W> *E = evs + ev;
      const uint4 hdr = __ldg(reinterpret_cast<const uint4 *>(E));
      uint64_t body[4 * W];
      const ulonglong2 *bp = reinterpret_cast<const ulonglong2 *>(&E->dsd[0]);
#pragma unroll
      for (int k = 0; k < 2 * W; ++k) {
        ulonglong2 v = __ldg(bp + k);
        body[2 * k] = v.x;
        body[2 * k + 1] = v.y;
      }
      const uint64_t *dsd = body, *dss = body + W, *beta = body + 2 * W, *gamma = body + 3 * W;
      while (nxt < hdr.y && status == G_OK) {
        const Site *S = P.sites + nxt;
        uint64_t esd[W], ess[W], b[W], g[W];
#pragma unroll
        for (int w = 0; w < W; ++w) {
          esd[w] = sd[w] ^ __ldg(&S->dsd[w]);
          ess[w] = ss[w] ^ __ldg(&S->dss[w]);
        }
        const uint32_t kind = __ldg(&S->kind);
        const uint32_t code = (kind & 3u) == SITE_DEPOL2 ? (uint32_t)(((uint64_t)w2 * 15u) >> 32) + 1u
                              : (kind & 3u) == SITE_FLIP ? (kind >> 2) & 3u
                                                         : (uint32_t)(((uint64_t)w2 * 3u) >> 32) + 1u;
        uint32_t e;
        error_pauli(nxt, code, esd, ess, b, g, &e);
        pauli(phi, b, g, e);
        if (n_err >= kMaxErr) {
          status = G_UNSUPPORTED;
          break;
        }
        if (lane == 0) {
          ErrRec<W> &er = errs()[n_err];
          er.ev = ev;
          er.site = nxt;
          er.code = code;
#pragma unroll
          for (int w = 0; w < W; ++w) {
            er.sd[w] = esd[w];
            er.ss[w] = ess[w];
          }
        }
        n_err++;
        draw_next();
      }
      if (status != G_OK) return;
#pragma unroll
      for (int w = 0; w < W; ++w) {
        sd[w] ^= dsd[w];
        ss[w] ^= dss[w];
      }
      tape_signs_store(ev);
      const uint32_t w0 = hdr.x, type = ev_type(w0), flags = ev_flags(w0);
      switch (type) {
        case EV_ROT:
        case EV_ROT_DIAG: {
          const uint32_t e = (ev_e0(w0) + 2u * pe(beta, gamma)) & 3u;
          const Coef *C = P.coef + hdr.z;
          Cx<R> a, b;
          if (sizeof(R) == 4) {
            a = Cx<R>{(R)__ldg(&C->fa_re), (R)__ldg(&C->fa_im)};
            b = Cx<R>{(R)__ldg(&C->fb_re), (R)__ldg(&C->fb_im)};
          } else {
            a = Cx<R>{(R)__ldg(&C->a_re), (R)__ldg(&C->a_im)};
            b = Cx<R>{(R)__ldg(&C->b_re), (R)__ldg(&C->b_im)};
          }
          if (type == EV_ROT) {
            if (!rot(phi, e, ev_lowbit(w0), a, b, beta, gamma)) status = kCapFail;
          } else {
            rot_diag(phi, e, a, b, gamma);
          }
          tape_store_phi(r, phi);
          r++;
          break;
        }
        case EV_MEAS_A:
        case EV_MEAS_B: {
          int mm = 0;
          if (flags & F_FIDELITY) {
            if (!seen_f) {
              seen_f = true;
              n_acc = norm2_map(phi);
              copy_map(pre, phi);
              ev_f = ev;
              rot_before_f = r;
            }
            mm = 1;
          } else if (flags & F_DETECTOR) {
            mm = (flags & F_INVERT) ? -1 : 1;
          } else if (!(flags & F_RECORD) && type == EV_MEAS_A) {
            // a reset: its outcome must be decided by the integer test
            const uint32_t sgn = ((ev_e0(w0) + 2u * pe(beta, gamma)) >> 1) & 1u;
            bool h0, h1;
            reset_sides(phi, gamma, sgn, h0, h1);
            if (h0 && h1) status = G_UNSUPPORTED;
            mm = h1 ? -1 : 1;
          } else {
            status = G_UNSUPPORTED;
          }
          if (status != G_OK) break;
          if (type == EV_MEAS_A) {
            const uint32_t e = (ev_e0(w0) + 2u * pe(beta, gamma)) & 3u;
            if (e & 1u) {
              status = G_ERROR;
              break;
            }
            project_a(phi, gamma, e >> 1, mm);
          } else {
            const CaseB *B = P.cb + (uint32_t)beta[0];
            const uint32_t p = __ldg(&B->p);
            uint64_t J[W], g2[W], ep[W];
#pragma unroll
            for (int w = 0; w < W; ++w) {
              J[w] = __ldg(&B->J[w]);
              g2[w] = __ldg(&B->gamma2[w]);
              ep[w] = ((int)(p >> 6) == w) ? (1ull << (p & 63)) : 0ull;
            }
            uint64_t sd0[W], ss0[W];
#pragma unroll
            for (int w = 0; w < W; ++w) {
              sd0[w] = sd[w];
              ss0[w] = ss[w];
            }
            const uint32_t e2 = caseb_signs(B, 0);
#pragma unroll
            for (int w = 0; w < W; ++w) {
              sd[w] = sd0[w];
              ss[w] = ss0[w];
            }
            project_b(phi, p, J, ep, g2, e2, mm);
            caseb_signs(B, mm);
          }
          lastm = mm;
          if (phi.n == 0u) {
            // the projection annihilated the state: N_acc = 0 (before the first fidelity
            // measurement) or N_fid = 0 (after it); nothing later changes either
            done_empty = true;
            break;
          }
          if ((flags & F_RECORD) && mm < 0 && lane == 0) rec[hdr.w >> 6] |= 1ull << (hdr.w & 63);
          if (mm == -1) tape_bit_set(ev);  // the outcome, for the reverse sweep
          t.sync();
          if ((flags & F_COND_LAST) && mm == -1) {
            uint64_t xb[W], xg[W];
#pragma unroll
            for (int w = 0; w < W; ++w) {
              xb[w] = __ldg(&E->xbeta[w]);
              xg[w] = __ldg(&E->xgamma[w]);
            }
            pauli(phi, xb, xg, (ev_xe0(w0) + 2u * pe(xb, xg)) & 3u);
          }
          break;
        }
        case EV_PAULI: {
          uint32_t cond;
          if (flags & F_COND_LAST) cond = (lastm == -1);
          else {
            const int32_t r0 = (int32_t)hdr.z, r1 = (int32_t)hdr.w;
            cond = (r0 >= 0 ? (uint32_t)((rec[r0 >> 6] >> (r0 & 63)) & 1ull) : 0u) ^
                   (r1 >= 0 ? (uint32_t)((rec[r1 >> 6] >> (r1 & 63)) & 1ull) : 0u);
          }
          if (cond) {
            pauli(phi, beta, gamma, (ev_e0(w0) + 2u * pe(beta, gamma)) & 3u);
            tape_bit_set(ev);
          }
          break;
        }
        case EV_PARITY:
          if (flags & F_DETECTOR) status = G_UNSUPPORTED;  // only single-record detectors fused into M
          break;
        default:
          break;
      }
    }
  }

  __device__ void fwd_init() {
#pragma unroll
    for (int w = 0; w < W; ++w) sd[w] = ss[w] = 0ull;
    for (uint32_t w = lane; w < P.rw; w += 32) rec[w] = 0ull;
    map_init_one(phi);
    copy_map(pre, phi);
    r = 0;
    ev_f = 0xFFFFFFFFu;
    rot_before_f = 0;
    seen_f = done_empty = false;
    n_acc = 0.0;
    lastm = 1;
    ev0 = r0 = 0;
    t.sync();
  }

  // --------------------------------------------------------- shared noiseless prefix
  // Until its first error a pattern's projection run is the pattern-independent
  // noiseless one (projections included). A tracing warp records it once per call:
  // its tape (maps after each rotation, signs, outcome bits) and, per event, the
  // state at the top of the event. Patterns start at the event that applies their
  // first error and read the shared tape below it in the reverse sweeps.
  struct SnapHdr {
    uint32_t nnz, r, lastm, pad;
    uint64_t sd[2], ss[2];
  };
  __host__ __device__ static constexpr size_t snap_stride(uint32_t rw) {
    return (sizeof(SnapHdr) + (size_t)rw * 8 + 32 * (size_t)W * 8 + 32 * sizeof(Cx<R>) + 15) & ~(size_t)15;
  }
  __device__ void save_snapshot(unsigned char *out) {
    SnapHdr *h = reinterpret_cast<SnapHdr *>(out);
    uint64_t *r_out = reinterpret_cast<uint64_t *>(out + sizeof(SnapHdr));
    uint64_t *k_out = r_out + P.rw;
    Cx<R> *v_out = reinterpret_cast<Cx<R> *>(k_out + 32 * W);
    if (lane == 0) {
      h->nnz = phi.n;
      h->r = r;
      h->lastm = (uint32_t)lastm;
#pragma unroll
      for (int w = 0; w < 2; ++w) {
        h->sd[w] = w < W ? sd[w < W ? w : 0] : 0ull;
        h->ss[w] = w < W ? ss[w < W ? w : 0] : 0ull;
      }
    }
    for (uint32_t w = lane; w < P.rw; w += 32) r_out[w] = rec[w];
    if (lane < phi.n) {
#pragma unroll
      for (int w = 0; w < W; ++w) k_out[lane * W + w] = phi.k.w[w];
      v_out[lane] = phi.v;
    }
  }
  __device__ void load_prefix() {
    const uint32_t stop = *P.pstop;
    ev0 = stop;
    if (nxt < P.n_sites) {
      const uint32_t e = __ldg(&P.site_ev[nxt]);
      ev0 = e < stop ? e : stop;
    }
    const unsigned char *in = P.psnap + (size_t)ev0 * P.psnap_stride;
    const SnapHdr *h = reinterpret_cast<const SnapHdr *>(in);
    const uint64_t *r_in = reinterpret_cast<const uint64_t *>(in + sizeof(SnapHdr));
    const uint64_t *k_in = r_in + P.rw;
    const Cx<R> *v_in = reinterpret_cast<const Cx<R> *>(k_in + 32 * W);
    phi.n = h->nnz;
    r0 = r = h->r;
    lastm = (int)h->lastm;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      sd[w] = h->sd[w];
      ss[w] = h->ss[w];
    }
    for (uint32_t w = lane; w < P.rw; w += 32) rec[w] = r_in[w];
    if constexpr (Wide) {
      for (uint32_t i = lane; i < phi.n; i += 32) {
#pragma unroll
        for (int w = 0; w < W; ++w) phi.k[(size_t)i * W + w] = k_in[i * W + w];
        phi.v[i] = v_in[i];
      }
    } else {
      if (lane < phi.n) {
#pragma unroll
        for (int w = 0; w < W; ++w) phi.k.w[w] = k_in[lane * W + w];
        phi.v = v_in[lane];
      }
    }
    t.sync();
    copy_map(pre, phi);
  }
  // The noiseless projection run from event 0, into this warp's tape (the shared
  // tape) and `snaps`; returns the last event a pattern may start at.
  __device__ uint32_t trace_prefix(unsigned char *snaps, size_t stride) {
    shot = 0;
    status = G_OK;
    n_err = 0;
    {
      uint64_t *bits = reinterpret_cast<uint64_t *>(tape + L.bits);
      for (uint32_t w = lane; w < (P.n_events + 63) / 64; w += 32) bits[w] = 0ull;
    }
    fwd_init();
    cur = P.n_sites;
    nxt = 0xFFFFFFFFu;
    const Ev<W> *evs = reinterpret_cast<const Ev<W> *>(P.ev);
    uint32_t ev = 0;
    for (; ev <= P.n_events; ++ev) {
      save_snapshot(snaps + (size_t)ev * stride);
      if (ev == P.n_events) break;
      const uint32_t w0 = __ldg(&evs[ev].w0), type = ev_type(w0);
      if ((type == EV_MEAS_A || type == EV_MEAS_B) && (ev_flags(w0) & F_FIDELITY)) break;
      fwd_step(ev);
      if (status != G_OK || done_empty) break;
    }
    t.sync();
    return ev;
  }

  // Reverse sweep from just before event `ev_end` (its errors included): the
  // adjoint starts as `lam` (the state there) and every parameterised rotation
  // adds weight * s * Im <lambda| Z_q |phi> to grad[k].
  __device__ bool sweep(const Map &src, uint32_t ev_end, uint32_t r_end, double *grad, double weight) {
    Map lam_local{};
    Map &lam = Wide ? lam_store : lam_local;  // registers, or the warp's shared-memory map
    copy_map(lam, src);
    const Ev<W> *evs = reinterpret_cast<const Ev<W> *>(P.ev);
    int64_t ei = (int64_t)n_err - 1;
    while (ei >= 0 && errs()[ei].ev > ev_end) --ei;  // errors after the sweep's start point
    uint32_t r = r_end;
    for (int64_t evi = (int64_t)(ev_end < P.n_events ? ev_end : P.n_events - 1); evi >= 0; --evi) {
      const uint32_t ev = (uint32_t)evi;
      if (ev < ev_end) {
        const Ev<W> *E = evs + ev;
        const uint4 hdr = __ldg(reinterpret_cast<const uint4 *>(E));
        uint64_t body[4 * W];
        const ulonglong2 *bp = reinterpret_cast<const ulonglong2 *>(&E->dsd[0]);
#pragma unroll
        for (int k = 0; k < 2 * W; ++k) {
          ulonglong2 v = __ldg(bp + k);
          body[2 * k] = v.x;
          body[2 * k + 1] = v.y;
        }
        const uint64_t *beta = body + 2 * W, *gamma = body + 3 * W;
        tape_signs_load(ev);
        const uint32_t w0 = hdr.x, type = ev_type(w0), flags = ev_flags(w0);
        if (type == EV_ROT || type == EV_ROT_DIAG) {
          --r;
          const uint32_t e = (ev_e0(w0) + 2u * pe(beta, gamma)) & 3u;
          if (hdr.w != kNoRec) {
            Map phk_local{};
            Map &phk = Wide ? phk_store : phk_local;
            tape_load_phi(r, phk);
            double zr, zi;
            zexp(lam, phk, beta, gamma, e, &zr, &zi);
            const double s = (hdr.w & 1u) ? -1.0 : 1.0;
            if (lane == 0) grad[hdr.w >> 1] += weight * s * zi;
          }
          const Coef *C = P.coef + hdr.z;
          Cx<R> a, b;
          if (sizeof(R) == 4) {
            a = Cx<R>{(R)__ldg(&C->fa_re), -(R)__ldg(&C->fa_im)};
            b = Cx<R>{(R)__ldg(&C->fb_re), -(R)__ldg(&C->fb_im)};
          } else {
            a = Cx<R>{(R)__ldg(&C->a_re), -(R)__ldg(&C->a_im)};
            b = Cx<R>{(R)__ldg(&C->b_re), -(R)__ldg(&C->b_im)};
          }
          if (type == EV_ROT) {
            if (!rot(lam, e, ev_lowbit(w0), a, b, beta, gamma)) return false;
          } else {
            rot_diag(lam, e, a, b, gamma);
          }
        } else if (type == EV_MEAS_A || type == EV_MEAS_B) {
          int mm;
          if (flags & F_FIDELITY) mm = 1;
          else if (flags & F_DETECTOR) mm = (flags & F_INVERT) ? -1 : 1;
          else mm = tape_bit(ev) ? -1 : 1;  // a reset: its decided outcome, from the tape
          if (type == EV_MEAS_A) {
            const uint32_t e = (ev_e0(w0) + 2u * pe(beta, gamma)) & 3u;
            if ((flags & F_COND_LAST) && mm == -1) {
              uint64_t xb[W], xg[W];
#pragma unroll
              for (int w = 0; w < W; ++w) {
                xb[w] = __ldg(&E->xbeta[w]);
                xg[w] = __ldg(&E->xgamma[w]);
              }
              pauli_adj(lam, xb, xg, (ev_xe0(w0) + 2u * pe(xb, xg)) & 3u);
            }
            project_a(lam, gamma, (e >> 1) & 1u, mm);
          } else {
            const CaseB *B = P.cb + (uint32_t)beta[0];
            const uint32_t p = __ldg(&B->p);
            uint64_t J[W], g2[W], ep[W];
#pragma unroll
            for (int w = 0; w < W; ++w) {
              J[w] = __ldg(&B->J[w]);
              g2[w] = __ldg(&B->gamma2[w]);
              ep[w] = ((int)(p >> 6) == w) ? (1ull << (p & 63)) : 0ull;
            }
            if ((flags & F_COND_LAST) && mm == -1) {
              // the correction ran with the replaced signs
              caseb_signs(B, mm);
              uint64_t xb[W], xg[W];
#pragma unroll
              for (int w = 0; w < W; ++w) {
                xb[w] = __ldg(&E->xbeta[w]);
                xg[w] = __ldg(&E->xgamma[w]);
              }
              pauli_adj(lam, xb, xg, (ev_xe0(w0) + 2u * pe(xb, xg)) & 3u);
              tape_signs_load(ev);
            }
            const uint32_t e2 = caseb_signs(B, 0);
            if (!project_b_adj(lam, p, J, ep, g2, e2, mm)) return false;
          }
        } else if (type == EV_PAULI) {
          if (tape_bit(ev)) pauli_adj(lam, beta, gamma, (ev_e0(w0) + 2u * pe(beta, gamma)) & 3u);
        }
      }
      // errors applied before this event, newest first
      while (ei >= 0 && errs()[ei].ev == ev) {
        const ErrRec<W> &er = errs()[ei];
        uint64_t esd[W], ess[W], b[W], g[W];
#pragma unroll
        for (int w = 0; w < W; ++w) {
          esd[w] = er.sd[w];
          ess[w] = er.ss[w];
        }
        uint32_t e;
        error_pauli(er.site, er.code, esd, ess, b, g, &e);
        pauli_adj(lam, b, g, e);
        --ei;
      }
    }
    return true;
  }
};

constexpr int kGradBlock = 128;

#ifndef SOFT_GRAD_MIN_BLOCKS
#define SOFT_GRAD_MIN_BLOCKS 4
#endif
template <typename R, int W>
__global__ void __launch_bounds__(kGradBlock, SOFT_GRAD_MIN_BLOCKS) grad_kernel(const __grid_constant__ GradParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  auto block = cg::this_thread_block();
  auto tile = cg::tiled_partition<32>(block);
  const uint32_t wid = threadIdx.x / 32;
  const size_t per = smem_per_warp(sizeof(R) == 4, W, P.rw);
  const uint32_t slot = blockIdx.x * (blockDim.x / 32) + wid;
  GradWarp<R, W> g(tile, P, smem + wid * per, P.tape + (size_t)slot * P.tape_stride);
  for (;;) {
    unsigned long long item = 0;
    if (tile.thread_rank() == 0) item = atomicAdd(P.next, 1ull);
    item = tile.shfl(item, 0);
    if (item >= P.n_patterns) break;
    g.run(P.first_pattern + item, item);
  }
}

// The patterns the register pass listed, with shared-memory maps (one warp per block).
template <typename R, int W>
__global__ void __launch_bounds__(32) grad_wide_kernel(const __grid_constant__ GradParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  auto tile = cg::tiled_partition<32>(cg::this_thread_block());
  GradWarp<R, W, true> g(tile, P, smem, P.wide_tape + (size_t)blockIdx.x * P.wide_tape_stride);
  const unsigned long long n = *P.wide_n < P.wide_cap ? *P.wide_n : P.wide_cap;
  for (;;) {
    unsigned long long i = 0;
    if (tile.thread_rank() == 0) i = atomicAdd(P.wide_next, 1ull);
    i = tile.shfl(i, 0);
    if (i >= n) break;
    const uint32_t off = P.wide_list[i];
    if (off >= P.n_patterns) break;
    g.run(P.first_pattern + off, off);
  }
}

template <typename R, int W>
__global__ void __launch_bounds__(32) grad_prefix_kernel(const __grid_constant__ GradParams P, unsigned char *tape,
                                                         unsigned char *snaps, uint32_t *stop) {
  extern __shared__ __align__(16) unsigned char smem[];
  auto tile = cg::tiled_partition<32>(cg::this_thread_block());
  GradWarp<R, W> g(tile, P, smem, tape);
  const uint32_t ev = g.trace_prefix(snaps, GradWarp<R, W>::snap_stride(P.rw));
  if (tile.thread_rank() == 0) *stop = ev;
}

template <typename R, int W>
cudaError_t launch_grad_prefix_t(const GradParams &p, unsigned char *tape, unsigned char *snaps, uint32_t *stop,
                                 cudaStream_t st) {
  GradParams q = p;
  q.psnap = nullptr;  // the tracer itself starts at event 0
  q.ptape = nullptr;
  const size_t smem = smem_per_warp(sizeof(R) == 4, W, p.rw);
  grad_prefix_kernel<R, W><<<1, 32, smem, st>>>(q, tape, snaps, stop);
  return cudaGetLastError();
}

template <typename R, int W>
cudaError_t launch_grad_t(const GradParams &p, cudaStream_t st) {
  const size_t smem = (kGradBlock / 32) * smem_per_warp(sizeof(R) == 4, W, p.rw);
  grad_kernel<R, W><<<p.blocks, kGradBlock, smem, st>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !p.wide_list || !p.wide_blocks) return e;
  const size_t wsmem = wide_smem_per_warp(sizeof(R) == 4, W, p.rw);
  e = cudaFuncSetAttribute(grad_wide_kernel<R, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsmem);
  if (e != cudaSuccess) return e;
  grad_wide_kernel<R, W><<<p.wide_blocks, 32, wsmem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace

size_t grad_smem_per_warp(int fp32, uint32_t W, uint32_t rw) { return smem_per_warp(fp32, W, rw); }

size_t grad_tape_bytes(int fp32, uint32_t W, uint32_t n_rot, uint32_t n_events) {
  if (fp32) return W == 1 ? TapeLayout<float, 1>(n_rot, n_events).total : TapeLayout<float, 2>(n_rot, n_events).total;
  return W == 1 ? TapeLayout<double, 1>(n_rot, n_events).total : TapeLayout<double, 2>(n_rot, n_events).total;
}

uint32_t grad_warps_per_block() { return kGradBlock / 32; }
uint32_t grad_blocks_per_sm() { return SOFT_GRAD_MIN_BLOCKS; }

size_t grad_wide_tape_bytes(int fp32, uint32_t W, uint32_t n_rot, uint32_t n_events) {
  if (fp32)
    return W == 1 ? TapeLayout<float, 1>(n_rot, n_events, kWideCap).total
                  : TapeLayout<float, 2>(n_rot, n_events, kWideCap).total;
  return W == 1 ? TapeLayout<double, 1>(n_rot, n_events, kWideCap).total
                : TapeLayout<double, 2>(n_rot, n_events, kWideCap).total;
}

size_t grad_prefix_stride(int fp32, uint32_t W, uint32_t rw) {
  if (fp32) return W == 1 ? GradWarp<float, 1>::snap_stride(rw) : GradWarp<float, 2>::snap_stride(rw);
  return W == 1 ? GradWarp<double, 1>::snap_stride(rw) : GradWarp<double, 2>::snap_stride(rw);
}

cudaError_t launch_grad_prefix(const GradParams &p, int fp32, uint32_t W, unsigned char *tape, unsigned char *snaps,
                               uint32_t *stop, cudaStream_t st) {
  if (fp32)
    return W == 1 ? launch_grad_prefix_t<float, 1>(p, tape, snaps, stop, st)
                  : launch_grad_prefix_t<float, 2>(p, tape, snaps, stop, st);
  return W == 1 ? launch_grad_prefix_t<double, 1>(p, tape, snaps, stop, st)
                : launch_grad_prefix_t<double, 2>(p, tape, snaps, stop, st);
}

cudaError_t launch_grad(const GradParams &p, int fp32, uint32_t W, cudaStream_t st) {
  if (fp32) return W == 1 ? launch_grad_t<float, 1>(p, st) : launch_grad_t<float, 2>(p, st);
  return W == 1 ? launch_grad_t<double, 1>(p, st) : launch_grad_t<double, 2>(p, st);
}

}  // namespace soft
