// kernels.cu -- persistent shot kernel for sm_103a.
//
// One tile of G lanes (G = 16 or 32) owns one shot at a time and walks the
// compiled event list of program.h. Per shot it holds, on chip:
//   - the 2n tableau sign bits (registers; the X/Z words are shot-invariant
//     and folded into the program),
//   - the sparse coefficient map v (shared memory): up to 2*cap keys and
//     complex values (FP64 or FP32) plus an open-addressing hash index,
//   - the measurement record bits (shared memory).
// Work items (shots) are handed out by an atomic counter, so shots that end
// early (a failed detector, Sec. V-C) free their tile at once.
//
// Arithmetic (arxiv 2512.23037):
//   T/Tdag/Rz: v'_a = A v_a + B xi_{a^beta} v_{a^beta}    (Eq. T_gate, Theorem 1 (3))
//   Pauli Q:   v'_{a^beta} = xi_a(Q) v_a, xi_a = c (-1)^{gamma.a}  (Eq. pauli_on_basis)
//   Z meas.:   filter (beta = 0) or pivot + pair (beta != 0), renormalise
//              (Eq. Pi_pm, Theorem 1 (2)); probabilities in FP64.
#include <cooperative_groups.h>

#include "device_common.cuh"
#include "shot_common.cuh"
#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace soft {
namespace {

using namespace dev;

enum : int { ST_RUN = -1, ST_KEPT = 0, ST_DISC = 1, ST_OVF = 2, ST_ERR = 3, ST_RERUN = 4 };

__host__ __device__ inline uint32_t pow2_at_least(uint32_t v) {
  uint32_t p = 1;
  while (p < v) p <<= 1;
  return p;
}
// Hash slots for a group of capacity `cap`: a power of two >= 4 cap (load <= 1/4).
__host__ __device__ inline uint32_t hash_slots(uint32_t cap) { return pow2_at_least(4u * cap < 16u ? 16u : 4u * cap); }

template <typename R, int W>
__host__ __device__ inline size_t group_bytes(uint32_t cap, uint32_t rw) {
  size_t slots = 2 * (size_t)cap;
  size_t b = slots * sizeof(Cx<R>) + (size_t)W * slots * 8 + 4 * (size_t)hash_slots(cap) + (size_t)rw * 8;
  return (b + 15) & ~(size_t)15;
}

// 1/sqrt(x) in the coefficient type: FP64 maps compute it in FP64, FP32 maps
// with the FP32 reciprocal square root (the scale is rounded to FP32 anyway).
template <typename R>
__device__ __forceinline__ R inv_sqrt_as(double x) {
  return (R)rsqrt(x);
}
template <>
__device__ __forceinline__ float inv_sqrt_as<float>(double x) {
  return rsqrtf((float)x);
}

template <typename R, int W, int G>
struct Shot {
  using Tile = cg::thread_block_tile<G>;
  const Tile &t;
  const ShotParams &P;
  Cx<R> *vals;
  uint64_t *keys;
  uint32_t *ht;
  uint64_t *rec;
  uint32_t slots, hsmask, hsmax, cap, lane;
  const CircDev *C = nullptr;  // the circuit of the current shot
  uint32_t ecap = 0;           // min(circuit cap, on-chip cap): |v| above it ends or reruns the shot
  mutable uint32_t bad_slot = 0;  // set by lookup() when the hash index holds an impossible slot
  uint64_t shot;
  uint32_t nnz;
  uint64_t sd[W], ss[W];
  uint32_t nxt, cur, kblk, w2;
  int status, chain, logical, lastm;
  bool force = false;  // fidelity mode: this measurement projects onto +1
  bool undecided = false;  // set when an outcome depended on the uniform (0 < p_+ < 1)
  double fid = 1.0;    // fidelity mode: product of the projected measurements' p_+
  // register mode: while |v| <= G, lane i < nnz holds entry i
  static constexpr bool kRegCapable = (G == 32 || G == 16);
  static constexpr uint32_t kTileFull = G == 32 ? 0xFFFFFFFFu : ((1u << G) - 1u);
  bool reg;
  Key<W> rk;
  Cx<R> rv;

  // The phase xi = i^e (-1)^{gamma.key} of a rotation: i^e folded into b once per event
  // (b xi is then b i^e or its negation, exact) takes instructions off the narrow FP64 pipe.
  // FP32 with two key words applies it per entry instead: there the folded constants stay
  // live across the entry loops of a kernel already at its register limit (80), and the
  // 97-qubit workload ran 27.1 M shots/s that way against 24.3 M folded. With one key word
  // (w42's warp passes) folding measured faster (1.26 against 1.50 ms per 2^24-shot step).
  static constexpr bool kFoldPhase = sizeof(R) == 8 || W == 1;
  PruneTest<R> pt;  // |v|^2 < tau (thresholds computed once per thread)

  __device__ Shot(const Tile &tile, const ShotParams &p, unsigned char *base) : t(tile), P(p), pt(p.tau) {
    cap = P.cap;
    slots = 2 * cap;
    hsmax = P.hs_max;
    hsmask = 15u;
    lane = t.thread_rank();
    vals = reinterpret_cast<Cx<R> *>(base);
    keys = reinterpret_cast<uint64_t *>(base + slots * sizeof(Cx<R>));
    ht = reinterpret_cast<uint32_t *>(base + slots * sizeof(Cx<R>) + (size_t)W * slots * 8);
    rec = reinterpret_cast<uint64_t *>(base + slots * sizeof(Cx<R>) + (size_t)W * slots * 8 + 4 * (size_t)hsmax);
    (void)P.rw_max;
  }
  // hash size for n live entries: power of two >= 4 n, at least 16, at most hsmax
  __device__ __forceinline__ uint32_t hs_for(uint32_t n) const {
    uint32_t want = 4u * n < 16u ? 16u : 4u * n;
    uint32_t p = 1u << (32 - __clz(want - 1u));
    return p < hsmax ? p : hsmax;
  }

  __device__ __forceinline__ Key<W> key(uint32_t e) const {
    Key<W> r;
#pragma unroll
    for (int w = 0; w < W; ++w) r.w[w] = keys[w * slots + e];
    return r;
  }
  __device__ __forceinline__ void set_key(uint32_t e, const Key<W> &k) {
#pragma unroll
    for (int w = 0; w < W; ++w) keys[w * slots + e] = k.w[w];
  }
  __device__ int lookup(const Key<W> &k) const {
    uint32_t h = khash(k) & hsmask;
    for (uint32_t probe = 0; probe <= hsmask; ++probe) {
      uint32_t v = ht[h];
      if (v == 0u) return -1;
      if (v - 1u >= slots) {
        bad_slot = v;
        return -1;
      }
      if (keq(key(v - 1u), k)) return (int)(v - 1u);
      h = (h + 1u) & hsmask;
    }
    return -1;
  }
  __device__ void insert(uint32_t s, const Key<W> &k) {
    uint32_t h = khash(k) & hsmask;
    for (uint32_t probe = 0; probe <= hsmask; ++probe) {
      if (atomicCAS(&ht[h], 0u, s + 1u) == 0u) return;
      h = (h + 1u) & hsmask;
    }
  }
  __device__ void rebuild() {
    hsmask = hs_for(nnz) - 1u;
    uint4 *h4 = reinterpret_cast<uint4 *>(ht);
    for (uint32_t i = lane; i <= (hsmask >> 2); i += G) h4[i] = make_uint4(0u, 0u, 0u, 0u);
    t.sync();
    for (uint32_t e = lane; e < nnz; e += G) insert(e, key(e));
    t.sync();
  }
  __device__ __forceinline__ uint32_t lanes_below(uint32_t ballot) const {
    return __popc(ballot & ((1u << lane) - 1u));
  }
  __device__ double tile_sum(double v) const {
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) v += t.shfl_xor(v, off);
    return v;
  }
  // Stable in-place compaction of entries [src, src + n) into [0, out).
  template <typename Keep>
  __device__ uint32_t compact(uint32_t src, uint32_t n, Keep keep) {
    uint32_t out = 0;
    for (uint32_t base = 0; base < n; base += G) {
      uint32_t e = base + lane;
      Key<W> k;
      Cx<R> v;
      bool kp = false;
      if (e < n) {
        k = key(src + e);
        v = vals[src + e];
        kp = keep(k, v);
      }
      uint32_t b = t.ballot(kp);
      t.sync();
      if (kp) {
        uint32_t d = out + lanes_below(b);
        set_key(d, k);
        vals[d] = v;
      }
      out += __popc(b);
      t.sync();
    }
    return out;
  }
  __device__ double uniform(uint32_t ord) const {
    uint4 w = philox(P.seed, shot, 1u, ord);
    uint64_t m = ((uint64_t)w.x << 21) ^ (uint64_t)(w.y >> 11);
    return (double)m * 0x1p-53;
  }

  // ---- noise: next accepted error site (geometric gaps, then thinning)
  __device__ void draw_next() {
    if (!next_site(C, P.seed, shot, cur, kblk, nxt, w2)) status = ST_ERR;
  }

  // v'_{a^beta} = i^{e + 2 gamma.a} v_a
  __device__ void apply_pauli(const uint64_t *beta, const uint64_t *gamma, uint32_t e) {
    if (kRegCapable && reg) {
      reg_pauli(beta, gamma, e);
      return;
    }
    bool moves = false;
#pragma unroll
    for (int w = 0; w < W; ++w) moves = moves || beta[w];
    for (uint32_t i = lane; i < nnz; i += G) {
      Key<W> k = key(i);
      vals[i] = ipow(vals[i], e + 2u * kpar(k, gamma));
      if (moves) set_key(i, kxor(k, beta));
    }
    t.sync();
    if (moves) rebuild();
  }

  __device__ void apply_error(uint32_t s) {
    if (s >= C->n_sites) {
      fail_check(CHK_SITE, s);
      return;
    }
    const Site *S = C->sites + s;
    const uint32_t kind = __ldg(&S->kind);
    uint32_t code, pa, pb;
    if ((kind & 3u) == SITE_DEPOL2) {
      code = (uint32_t)(((uint64_t)w2 * 15u) >> 32) + 1u;
      pa = code >> 2;
      pb = code & 3u;
    } else if ((kind & 3u) == SITE_FLIP) {
      code = (kind >> 2) & 3u;
      pa = code;
      pb = 0;
    } else {
      code = (uint32_t)(((uint64_t)w2 * 3u) >> 32) + 1u;
      pa = code;
      pb = 0;
    }
    uint64_t beta[W], gamma[W];
    uint32_t pe = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      uint64_t b = 0, g = 0;
      if (pa == 1u || pa == 2u) { b ^= __ldg(&S->bx[0][w]); g ^= __ldg(&S->gx[0][w]); }
      if (pa == 3u || pa == 2u) { b ^= __ldg(&S->bz[0][w]); g ^= __ldg(&S->gz[0][w]); }
      if (pb == 1u || pb == 2u) { b ^= __ldg(&S->bx[1][w]); g ^= __ldg(&S->gx[1][w]); }
      if (pb == 3u || pb == 2u) { b ^= __ldg(&S->bz[1][w]); g ^= __ldg(&S->gz[1][w]); }
      beta[w] = b;
      gamma[w] = g;
      pe += __popcll((sd[w] ^ __ldg(&S->dsd[w])) & b) + __popcll((ss[w] ^ __ldg(&S->dss[w])) & g);
    }
    uint32_t e = ((__ldg(&S->c0) >> (2u * code)) + 2u * pe) & 3u;
    apply_pauli(beta, gamma, e);
  }

  __device__ void fail_capacity() { status = (P.small_pass && C->cap > cap) ? ST_RERUN : ST_OVF; }

  // Record the first failed bounds check of the launch and end the shot as ERROR.
  uint32_t cur_ev = 0;
  __device__ void fail_check(uint32_t code, uint64_t value) {
    status = ST_ERR;
    if (lane == 0 && P.diag) {
      if (atomicAdd(&P.diag[0], 1ull) == 0ull) {
        P.diag[1] = ((unsigned long long)code << 32) | cur_ev;
        P.diag[2] = shot;
        P.diag[3] = value;
      }
    }
  }

  // ---------------------------------------------------------------- register mode
  // masks below are tile-relative: bit i = lane i of this G-lane tile
  __device__ __forceinline__ uint32_t vmask() const { return nnz >= (uint32_t)G ? kTileFull : ((1u << nnz) - 1u); }
  __device__ __forceinline__ uint32_t match_key(const Key<W> &k) const {
    uint32_t m = t.match_any((unsigned long long)k.w[0]);
    if (W == 2) m &= t.match_any((unsigned long long)k.w[W - 1]);
    return m;
  }
  __device__ __forceinline__ Cx<R> shfl_c(Cx<R> v, uint32_t src) const {
    return Cx<R>{t.shfl(v.x, src), t.shfl(v.y, src)};
  }
  // registers -> slots [0, nnz) (used before the shared-memory path takes over)
  __device__ void reg_spill() {
    if (lane < nnz) {
      set_key(lane, rk);
      vals[lane] = rv;
    }
    t.sync();
    reg = false;
  }
  // slots [0, nnz) -> registers (nnz <= 32)
  __device__ void reg_load() {
    if (lane < nnz) {
      rk = key(lane);
      rv = vals[lane];
    }
    t.sync();
    reg = true;
  }
  // keep the entries whose lane has `keep` set, in lane order (staged through shared memory)
  __device__ void reg_compact(bool keep) {
    const uint32_t b = t.ballot(keep);
    if (b == vmask()) return;
    if (keep) {
      const uint32_t d = lanes_below(b);
      set_key(d, rk);
      vals[d] = rv;
    }
    t.sync();
    nnz = __popc(b);
    if (lane < nnz) {
      rk = key(lane);
      rv = vals[lane];
    }
    t.sync();
  }

  __device__ void reg_pauli(const uint64_t *beta, const uint64_t *gamma, uint32_t e) {
    if (lane < nnz) {
      rv = ipow(rv, e + 2u * kpar(rk, gamma));
      rk = kxor(rk, beta);
    }
  }

  __device__ void reg_rot(uint32_t e, uint32_t lowbit, Cx<R> a, Cx<R> b, const uint64_t *beta,
                          const uint64_t *gamma) {
    const bool valid = lane < nnz;
    const Key<W> pk = kxor(rk, beta);
    const Key<W> canon = kbit(rk, lowbit) ? pk : rk;  // the pair's member with bit lowbit clear
    const uint32_t partner = match_key(canon) & vmask() & ~(1u << lane);
    const uint32_t pl = partner ? (uint32_t)(__ffs(partner) - 1) : lane;
    const Cx<R> vj = shfl_c(rv, pl);
    const bool has = valid && partner != 0u;
    const bool app = valid && !has;
    // one product serves both cases: b xi_{pk} v_partner (paired) or b xi_k v_k (new entry at pk)
    const Cx<R> src = has ? vj : rv;
    const uint32_t par = kpar(has ? pk : rk, gamma);
    Cx<R> tb;  // b xi v (the phase folded into b in FP64, exact; see kFoldPhase)
    if (kFoldPhase) {
      const Cx<R> bq = ipow(b, e);
      tb = cmul(par ? Cx<R>{negr(bq.x), negr(bq.y)} : bq, src);
    } else {
      tb = cmul(b, ipow(src, e + 2u * par));
    }
    Cx<R> nv = cmul(a, rv);
    if (has) nv = cadd(nv, tb);
    const Cx<R> av = tb;
    if (!valid) nv = Cx<R>{0, 0};
    const uint32_t ab = t.ballot(app);
    const uint32_t nA = __popc(ab);
    const bool small = (valid && pt.small(nv)) || (app && pt.small(av));
    const bool prune = t.any(small);
    if (nnz + nA > slots) {  // cannot happen while nnz <= cap before the gate
      fail_check(CHK_STAGE, nnz + nA);
      return;
    }
    if (nnz + nA <= (uint32_t)G) {
      if (nA) {
        if (app) {
          const uint32_t d = lanes_below(ab);
          set_key(d, pk);
          vals[d] = av;
        }
        t.sync();
        if (valid) rv = nv;
        else if (lane < nnz + nA) {
          rk = key(lane - nnz);
          rv = vals[lane - nnz];
        }
        t.sync();
        nnz += nA;
      } else if (valid) {
        rv = nv;
      }
      if (prune) reg_compact(lane < nnz && !pt.small(rv));
      if (nnz > ecap) fail_capacity();
      return;
    }
    // more than G entries: continue in shared memory with the hash index
    if (valid) {
      set_key(lane, rk);
      vals[lane] = nv;
    }
    if (app) {
      const uint32_t d = nnz + lanes_below(ab);
      set_key(d, pk);
      vals[d] = av;
    }
    t.sync();
    reg = false;
    nnz += nA;
    if (prune) nnz = compact(0, nnz, [&](Key<W> &, Cx<R> &v) { return !pt.small(v); });
    if (nnz > ecap) {
      fail_capacity();
      return;
    }
    rebuild();
  }

  __device__ void reg_rot_diag(uint32_t e, Cx<R> a, Cx<R> b, const uint64_t *gamma) {
    const bool valid = lane < nnz;
    if (kFoldPhase) {
      const Cx<R> bq = ipow(b, e);  // v' = (a + b xi) v, with a + b xi one of two constants
      if (valid) rv = cmul(kpar(rk, gamma) ? csub(a, bq) : cadd(a, bq), rv);
    } else if (valid) {
      rv = cadd(cmul(a, rv), cmul(b, ipow(rv, e + 2u * kpar(rk, gamma))));
    }
    if (t.any(valid && pt.small(rv))) reg_compact(valid && !pt.small(rv));
  }

  // Outcome of a non-deterministic measurement with p_+ = pp: sampled from the
  // stream, or in fidelity mode +1 (weight pp) unless +1 is impossible.
  // Outcome +1 iff u < p, with p = sp / (sp + sm) snapped to 0 or 1 within 1e-12:
  // decided as u (sp + sm) < sp, so that only the fidelity mode divides.
  __device__ __forceinline__ int pick(uint32_t ord, double sp, double sm) {
    const double tot = sp + sm;
    if (!(tot > 0.0)) return -1;
    const bool zero = sp < 1e-12 * tot, one = sp > (1.0 - 1e-12) * tot;
    if (!zero && !one) undecided = true;
    if (force) {
      if (zero) return -1;
      fid *= one ? 1.0 : sp / tot;
      return 1;
    }
    if (zero) return -1;
    if (one) return 1;
    return uniform(ord) * tot < sp ? 1 : -1;
  }

  __device__ int reg_meas_a(uint32_t sgn, uint32_t ord, const uint64_t *gamma) {
    const bool valid = lane < nnz;
    const bool neg = valid && (kpar(rk, gamma) ^ sgn);
    const bool h1 = t.any(neg), h0 = t.any(valid && !neg);
    if (!(h0 && h1)) return h1 ? -1 : 1;
    const double a2 = valid ? pnorm(rv) : 0.0;
    const double sp = tile_sum(neg ? 0.0 : a2), sm = tile_sum(neg ? a2 : 0.0);
    const int m = pick(ord, sp, sm);
    const R sc = inv_sqrt_as<R>(m == 1 ? sp : sm);
    bool keep = valid && (neg == (m == -1));
    if (keep) rv = cscale(rv, sc);
    reg_compact(keep && norm2(rv) >= (R)P.tau);
    return m;
  }

  __device__ int reg_meas_b(uint32_t p, const uint64_t *J, const uint64_t *g2, const uint64_t *ep, uint32_t e2,
                            uint32_t ord) {
    const bool valid = lane < nnz;
    if (valid && kbit(rk, p)) rk = kxor(rk, J);  // relabel a_j ^= a_p
    const uint32_t hi = kbit(rk, p);
    const Key<W> a0 = hi ? kxor(rk, ep) : rk;
    const uint32_t partner = match_key(a0) & vmask() & ~(1u << lane);
    const uint32_t pl = partner ? (uint32_t)(__ffs(partner) - 1) : lane;
    const Cx<R> vj = shfl_c(rv, pl);
    const bool owner = valid && (!hi || partner == 0u);
    Cx<R> v0{0, 0}, v1{0, 0};
    if (hi) v1 = rv;
    else {
      v0 = rv;
      if (partner) v1 = vj;
    }
    const Cx<R> x1 = ipow(v1, e2 + 2u * kpar(kxor(a0, ep), g2));
    const double sp = tile_sum(owner ? 0.5 * pnorm(cadd(v0, x1)) : 0.0);
    const double sm = tile_sum(owner ? 0.5 * pnorm(csub(v0, x1)) : 0.0);
    const int m = pick(ord, sp, sm);
    const R sc = inv_sqrt_as<R>(2.0 * (m == 1 ? sp : sm));
    if (owner) {
      rv = cscale(m == 1 ? cadd(v0, x1) : csub(v0, x1), sc);
      rk = a0;
    }
    reg_compact(owner && norm2(rv) >= (R)P.tau);
    return m;
  }

  __device__ void set_record(uint32_t r, int m) {
    if (r >= 64u * C->rw) {
      fail_check(CHK_RECORD, r);
      return;
    }
    if (lane == 0 && m < 0) rec[r >> 6] |= 1ull << (r & 63);
    t.sync();
  }

  // ---- a I + b Z_q, beta != 0
  __device__ __forceinline__ void coef(uint32_t ci, Cx<R> &a, Cx<R> &b) const {
    const Coef *cf = C->coef + (ci < C->n_coef ? ci : 0u);
    if (sizeof(R) == 4) {
      float4 f = __ldg(reinterpret_cast<const float4 *>(&cf->fa_re));
      a = Cx<R>{(R)f.x, (R)f.y};
      b = Cx<R>{(R)f.z, (R)f.w};
    } else {
      double2 d0 = __ldg(reinterpret_cast<const double2 *>(&cf->a_re));
      double2 d1 = __ldg(reinterpret_cast<const double2 *>(&cf->b_re));
      a = Cx<R>{(R)d0.x, (R)d0.y};
      b = Cx<R>{(R)d1.x, (R)d1.y};
    }
  }

  __device__ void rot(uint32_t w0, uint32_t ci, const uint64_t *beta, const uint64_t *gamma) {
    uint32_t pe = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) pe += __popcll(sd[w] & beta[w]) + __popcll(ss[w] & gamma[w]);
    const uint32_t e = (ev_e0(w0) + 2u * pe) & 3u;
    const uint32_t lowbit = ev_lowbit(w0);
    if (ci >= C->n_coef) {
      fail_check(CHK_COEF, ci);
      return;
    }
    Cx<R> a, b;
    coef(ci, a, b);
    if (kRegCapable && reg) {
      reg_rot(e, lowbit, a, b, beta, gamma);
      return;
    }
    const Cx<R> bq = ipow(b, e), bn = Cx<R>{negr(bq.x), negr(bq.y)};  // b xi: the phase folded into b
    uint32_t nA = 0;
    bool prune = false;
    const uint32_t n0 = nnz;
    for (uint32_t base = 0; base < n0; base += G) {
      uint32_t i = base + lane;
      bool app = false;
      Key<W> pk;
      Cx<R> nv{0, 0};
      if (i < n0) {
        Key<W> k = key(i);
        Cx<R> v = vals[i];
        pk = kxor(k, beta);
        int j = lookup(pk);
        if (j >= 0) {
          if (!kbit(k, lowbit)) {
            Cx<R> vj = vals[j];
            Cx<R> ni, nj;
            if (kFoldPhase) {
              ni = cadd(cmul(a, v), cmul(kpar(pk, gamma) ? bn : bq, vj));
              nj = cadd(cmul(a, vj), cmul(kpar(k, gamma) ? bn : bq, v));
            } else {
              ni = cadd(cmul(a, v), cmul(b, ipow(vj, e + 2u * kpar(pk, gamma))));
              nj = cadd(cmul(a, vj), cmul(b, ipow(v, e + 2u * kpar(k, gamma))));
            }
            vals[i] = ni;
            vals[j] = nj;
            prune = prune || pt.small(ni) || pt.small(nj);
          }
        } else {
          Cx<R> ni = cmul(a, v);
          vals[i] = ni;
          nv = kFoldPhase ? cmul(kpar(k, gamma) ? bn : bq, v) : cmul(b, ipow(v, e + 2u * kpar(k, gamma)));
          app = true;
          prune = prune || pt.small(ni) || pt.small(nv);
        }
      }
      uint32_t bal = t.ballot(app);
      if (app) {
        uint32_t slot = n0 + nA + lanes_below(bal);
        if (slot < slots) {
          set_key(slot, pk);
          vals[slot] = nv;
        } else {
          bad_slot = slot + 1u;
        }
      }
      nA += __popc(bal);
    }
    t.sync();
    nnz = n0 + nA;
    if (t.any(bad_slot != 0u)) {
      uint32_t worst = bad_slot;
#pragma unroll
      for (int off = G / 2; off > 0; off >>= 1) worst = max(worst, t.shfl_xor(worst, off));
      fail_check(CHK_HASH_SLOT, worst);
      return;
    }
    bool pruned = t.any(prune);
    if (pruned) nnz = compact(0, nnz, [&](Key<W> &, Cx<R> &v) { return !pt.small(v); });
    if (nnz > ecap) {
      fail_capacity();
      return;
    }
    if (pruned || hs_for(nnz) - 1u > hsmask) {
      rebuild();
    } else if (nA) {
      for (uint32_t i = n0 + lane; i < nnz; i += G) insert(i, key(i));
      t.sync();
    }
  }

  // ---- a I + b Z_q, beta == 0: v_a *= a + b xi_a
  __device__ void rot_diag(uint32_t w0, uint32_t ci, const uint64_t *gamma) {
    uint32_t pe = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) pe += __popcll(ss[w] & gamma[w]);
    const uint32_t e = (ev_e0(w0) + 2u * pe) & 3u;
    Cx<R> a, b;
    coef(ci, a, b);
    if (kRegCapable && reg) {
      reg_rot_diag(e, a, b, gamma);
      return;
    }
    const Cx<R> bq = ipow(b, e), c0 = cadd(a, bq), c1 = csub(a, bq);  // v' = (a + b xi) v
    bool prune = false;
    for (uint32_t i = lane; i < nnz; i += G) {
      Key<W> k = key(i);
      Cx<R> nv = kFoldPhase ? cmul(kpar(k, gamma) ? c1 : c0, vals[i])
                            : cadd(cmul(a, vals[i]), cmul(b, ipow(vals[i], e + 2u * kpar(k, gamma))));
      vals[i] = nv;
      prune = prune || pt.small(nv);
    }
    t.sync();
    if (t.any(prune)) {
      nnz = compact(0, nnz, [&](Key<W> &, Cx<R> &v) { return !pt.small(v); });
      rebuild();
    }
  }

  // ---- Z measurement, beta = 0: lambda_a = c (-1)^{gamma.a}
  __device__ int meas_a(uint32_t w0, uint32_t ord, const uint64_t *gamma) {
    uint32_t pe = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) pe += __popcll(ss[w] & gamma[w]);
    const uint32_t e = (ev_e0(w0) + 2u * pe) & 3u;
    if (e & 1u) {
      fail_check(CHK_PHASE, e);
      return 1;
    }
    const uint32_t sgn = e >> 1;
    if (kRegCapable && reg) return reg_meas_a(sgn, ord, gamma);
    // integer test first: the outcome is decided when every lambda_a agrees
    bool h0 = false, h1 = false;
    for (uint32_t i = lane; i < nnz; i += G) {
      if (kpar(key(i), gamma) ^ sgn) h1 = true;
      else h0 = true;
    }
    h0 = t.any(h0);
    h1 = t.any(h1);
    if (!(h0 && h1)) return h1 ? -1 : 1;
    double sp = 0.0, sm = 0.0;
    for (uint32_t i = lane; i < nnz; i += G) {
      double a2 = pnorm(vals[i]);
      if (kpar(key(i), gamma) ^ sgn) sm += a2;
      else sp += a2;
    }
    sp = tile_sum(sp);
    sm = tile_sum(sm);
    const int m = pick(ord, sp, sm);
    const R sc = inv_sqrt_as<R>(m == 1 ? sp : sm);
    const uint32_t want = (m == 1) ? 0u : 1u;
    const R tau = (R)P.tau;
    t.sync();
    nnz = compact(0, nnz, [&](Key<W> &k, Cx<R> &v) {
      if ((kpar(k, gamma) ^ sgn) != want) return false;
      v = cscale(v, sc);
      return norm2(v) >= tau;
    });
    rebuild();
    return m;
  }

  // ---- Z measurement, beta != 0 (case B)
  __device__ int meas_b(uint32_t ord, uint32_t cbi) {
    if (cbi >= C->n_cb) {
      fail_check(CHK_CASEB, cbi);
      return 1;
    }
    const CaseB *B = C->cb + cbi;
    const uint32_t p = __ldg(&B->p);
    uint64_t J[W], g2[W], ep[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
      J[w] = __ldg(&B->J[w]);
      g2[w] = __ldg(&B->gamma2[w]);
      ep[w] = ((int)(p >> 6) == w) ? (1ull << (p & 63)) : 0ull;
    }
    // row operations on the sign bits: s_j <- s_j s_p (j in J), d_p <- d_p prod d_j
    const uint32_t ssp = wbit<W>(ss, p);
    const uint32_t sdJ = wpar<W>(sd, J);
#pragma unroll
    for (int w = 0; w < W; ++w) ss[w] ^= (ssp ? J[w] : 0ull) ^ __ldg(&B->Hs[w]);
    if (sdJ ^ __ldg(&B->hdp)) wflip<W>(sd, p);
    // P = i^e2 d_p s_gamma2 in the new tableau
    const uint32_t e2 = (__ldg(&B->e0b) + 2u * (wbit<W>(sd, p) + wpar<W>(ss, g2))) & 3u;
    int m;
    if (kRegCapable && reg) {
      m = reg_meas_b(p, J, g2, ep, e2, ord);
    } else {
      m = smem_meas_b(p, J, g2, ep, e2, ord);
    }
    // replacement: d_j <- d_j s_p (j in G), d_p <- old s_p, s_p <- m P
#pragma unroll
    for (int w = 0; w < W; ++w) sd[w] ^= (ssp ? __ldg(&B->G[w]) : 0ull) ^ __ldg(&B->Hd[w]);
    if (wbit<W>(sd, p) != ssp) wflip<W>(sd, p);
    const uint32_t newsp = (m == -1 ? 1u : 0u) ^ __ldg(&B->rP);
    if (wbit<W>(ss, p) != newsp) wflip<W>(ss, p);
    return m;
  }

  __device__ int smem_meas_b(uint32_t p, const uint64_t *J, const uint64_t *g2, const uint64_t *ep, uint32_t e2,
                             uint32_t ord) {
    if (nnz > cap) {  // the staging half [cap, 2 cap) must hold every entry
      fail_check(CHK_NNZ, nnz);
      return 1;
    }
    // relabel keys: a_j ^= a_p for j in J
    for (uint32_t i = lane; i < nnz; i += G) {
      Key<W> k = key(i);
      if (kbit(k, p)) set_key(i, kxor(k, J));
    }
    t.sync();
    rebuild();
    double sp = 0.0, sm = 0.0;
    for (uint32_t i = lane; i < nnz; i += G) {
      Key<W> k = key(i);
      const uint32_t hi = kbit(k, p);
      const int j = lookup(kxor(k, ep));
      if (hi && j >= 0) continue;
      Cx<R> v0{0, 0}, v1{0, 0};
      if (hi) v1 = vals[i];
      else {
        v0 = vals[i];
        if (j >= 0) v1 = vals[j];
      }
      Key<W> a1 = hi ? k : kxor(k, ep);
      Cx<R> x1 = ipow(v1, e2 + 2u * kpar(a1, g2));
      sp += 0.5 * pnorm(cadd(v0, x1));
      sm += 0.5 * pnorm(csub(v0, x1));
    }
    sp = tile_sum(sp);
    sm = tile_sum(sm);
    if (t.any(bad_slot != 0u)) {
      fail_check(CHK_HASH_SLOT, bad_slot);
      return 1;
    }
    const int m = pick(ord, sp, sm);
    const R sc = inv_sqrt_as<R>(2.0 * (m == 1 ? sp : sm));
    // stage the paired values in slots [cap, cap + nnz)
    for (uint32_t i = lane; i < nnz; i += G) {
      Key<W> k = key(i);
      const uint32_t hi = kbit(k, p);
      const int j = lookup(kxor(k, ep));
      Cx<R> nv{0, 0};
      Key<W> a0 = hi ? kxor(k, ep) : k;
      if (!(hi && j >= 0)) {
        Cx<R> v0{0, 0}, v1{0, 0};
        if (hi) v1 = vals[i];
        else {
          v0 = vals[i];
          if (j >= 0) v1 = vals[j];
        }
        Key<W> a1 = kxor(a0, ep);
        Cx<R> x1 = ipow(v1, e2 + 2u * kpar(a1, g2));
        nv = cscale(m == 1 ? cadd(v0, x1) : csub(v0, x1), sc);
      }
      set_key(cap + i, a0);
      vals[cap + i] = nv;
    }
    t.sync();
    const R tau = (R)P.tau;
    nnz = compact(cap, nnz, [&](Key<W> &, Cx<R> &v) { return norm2(v) >= tau; });
    rebuild();
    return m;
  }

  __device__ uint32_t rec_bit(int32_t r) const {
    return (r < 0 || (uint32_t)r >= 64u * C->rw) ? 0u : (uint32_t)((rec[r >> 6] >> (r & 63)) & 1ull);
  }

  // Shot state at the top of event `ev` of the circuit's noiseless run, when that
  // run has one (traj_stop > ev): written by trace_prefix, read by load_prefix.
  __host__ __device__ static constexpr size_t snap_stride(uint32_t rw) { return dev::snap_stride<R, W>(rw); }
  __device__ void save_snapshot(unsigned char *out) {
    SnapHdr *h = reinterpret_cast<SnapHdr *>(out);
    uint64_t *rw_out = reinterpret_cast<uint64_t *>(out + sizeof(SnapHdr));
    uint64_t *k_out = rw_out + C->rw;
    Cx<R> *v_out = reinterpret_cast<Cx<R> *>(k_out + kSnapMax * W);
    if (lane == 0) {
      h->nnz = nnz;
      h->chain = (uint32_t)chain;
      h->logical = (uint32_t)logical;
      h->lastm = (uint32_t)lastm;
      h->fid = fid;
#pragma unroll
      for (int w = 0; w < 2; ++w) {
        h->sd[w] = w < W ? sd[w < W ? w : 0] : 0ull;
        h->ss[w] = w < W ? ss[w < W ? w : 0] : 0ull;
      }
    }
    for (uint32_t w = lane; w < C->rw; w += G) rw_out[w] = rec[w];
    if (reg) {
      if (lane < nnz) {
#pragma unroll
        for (int w = 0; w < W; ++w) k_out[lane * W + w] = rk.w[w];
        v_out[lane] = rv;
      }
    } else {
      for (uint32_t i = lane; i < nnz && i < kSnapMax; i += G) {
        const Key<W> k = key(i);
#pragma unroll
        for (int w = 0; w < W; ++w) k_out[i * W + w] = k.w[w];
        v_out[i] = vals[i];
      }
    }
  }
  // First event whose errors the shot must apply itself: the event that applies
  // its first error (the first with site_begin > nxt), capped at the end of the
  // noiseless run's valid prefix. Loads the snapshot there and returns it.
  __device__ uint32_t load_prefix() {
    const uint32_t lo = first_event(C, P.fid_mode, nxt);
    const unsigned char *in = C->traj + (size_t)lo * C->traj_stride;
    const SnapHdr *h = reinterpret_cast<const SnapHdr *>(in);
    const uint64_t *r_in = reinterpret_cast<const uint64_t *>(in + sizeof(SnapHdr));
    const uint64_t *k_in = r_in + C->rw;
    const Cx<R> *v_in = reinterpret_cast<const Cx<R> *>(k_in + kSnapMax * W);
    nnz = __ldg(&h->nnz);
    chain = (int)__ldg(&h->chain);
    logical = (int)__ldg(&h->logical);
    lastm = (int)__ldg(&h->lastm);
    fid = __ldg(&h->fid);
#pragma unroll
    for (int w = 0; w < W; ++w) {
      sd[w] = __ldg(&h->sd[w]);
      ss[w] = __ldg(&h->ss[w]);
    }
    for (uint32_t w = lane; w < C->rw; w += G) rec[w] = __ldg(&r_in[w]);
    if (nnz > kSnapMax) {  // a snapshot never holds more than kSnapMax entries
      fail_check(CHK_NNZ, nnz);
      return lo;
    }
    if (nnz > ecap) {  // the uninterrupted run would have outgrown this pass's capacity too
      fail_capacity();
      return lo;
    }
    if (kRegCapable && nnz <= (uint32_t)G) {
      reg = true;
      if (lane < nnz) {
#pragma unroll
        for (int w = 0; w < W; ++w) rk.w[w] = __ldg(&k_in[lane * W + w]);
        rv = v_in[lane];
      }
      t.sync();
    } else {
      for (uint32_t i = lane; i < nnz; i += G) {
        Key<W> k;
#pragma unroll
        for (int w = 0; w < W; ++w) k.w[w] = __ldg(&k_in[i * W + w]);
        set_key(i, k);
        vals[i] = v_in[i];
      }
      t.sync();
      reg = false;
      rebuild();
    }
    return lo;
  }

  __device__ void init_shot(uint64_t s) {
    shot = s;
    status = ST_RUN;
    bad_slot = 0;
    chain = 0;
    logical = 0;
    lastm = 1;
#pragma unroll
    for (int w = 0; w < W; ++w) sd[w] = ss[w] = 0ull;
    nnz = 1;
    Key<W> z;
#pragma unroll
    for (int w = 0; w < W; ++w) z.w[w] = 0ull;
    ecap = C->cap < cap ? C->cap : cap;
    for (uint32_t w = lane; w < C->rw; w += G) rec[w] = 0ull;
    if (kRegCapable) {
      reg = true;
      rk = z;
      rv = Cx<R>{(R)(lane == 0 ? 1 : 0), (R)0};
      t.sync();
    } else {
      reg = false;
      if (lane == 0) {
        set_key(0, z);
        vals[0] = Cx<R>{(R)1, (R)0};
      }
      t.sync();
      rebuild();
    }
    cur = 0;
    kblk = 0;
    fid = 1.0;
    force = false;
  }

  // A shot handed over by a lane: its whole state at the top of its resume event,
  // which is returned.
  __device__ uint32_t load_spill(uint32_t r) {
    const Spill<R, W> S(P.sp, P.sp_cap, P.rw_max);
    const size_t c = S.cap;
    const uint4 a = S.ha[r], b = S.hb[r];
    nnz = a.z;
    chain = (int)(a.w & 1u);
    logical = (int)((a.w >> 1) & 1u);
    lastm = (int)(int8_t)((a.w >> 8) & 255u);
    nxt = b.x;
    cur = b.y;
    kblk = b.z;
    w2 = b.w;
    fid = S.fid[r];
#pragma unroll
    for (int w = 0; w < W; ++w) {
      sd[w] = S.sd[w * c + r];
      ss[w] = S.ss[w * c + r];
    }
    for (uint32_t w = lane; w < C->rw; w += G) rec[w] = S.rec[w * c + r];
    if (nnz > kLaneCap || a.y >= C->n_events) {  // a record never holds more, nor resumes past the end
      fail_check(CHK_NNZ, nnz);
      return C->n_events;
    }
    if (nnz > ecap) {
      fail_capacity();
      return a.y;
    }
    if (kRegCapable && nnz <= (uint32_t)G) {
      reg = true;
      if (lane < nnz) {
#pragma unroll
        for (int w = 0; w < W; ++w) rk.w[w] = S.keys[((size_t)lane * W + w) * c + r];
        rv = S.vals[(size_t)lane * c + r];
      }
      t.sync();
    } else {
      for (uint32_t i = lane; i < nnz; i += G) {
        Key<W> k;
#pragma unroll
        for (int w = 0; w < W; ++w) k.w[w] = S.keys[((size_t)i * W + w) * c + r];
        set_key(i, k);
        vals[i] = S.vals[(size_t)i * c + r];
      }
      t.sync();
      reg = false;
      rebuild();
    }
    return a.y;
  }

  // rec: a spill record to resume from, or kNoRecord
  __device__ void run(uint64_t s, uint32_t r = kNoRecord) {
    init_shot(s);
    uint32_t ev0 = 0;
    if (r != kNoRecord) {
      ev0 = load_spill(r);
    } else {
      draw_next();
      if (C->traj) ev0 = load_prefix();  // every event before the first error is the noiseless run's
    }
    const uint32_t n_events = C->n_events;
    for (uint32_t ev = ev0; ev < n_events && status == ST_RUN; ++ev) step(ev);
    if (status == ST_RUN) status = ST_KEPT;
  }

  // The circuit's noiseless run (sampling semantics), recording the state at the
  // top of every event until an outcome is not decided (it would depend on the
  // shot's uniform), a map above kSnapMax entries, or the end. Event `stop` is the
  // last valid snapshot: shots resume there at the latest. *fid_stop receives the
  // first fidelity measurement's event (fidelity-mode shots resume there at the
  // latest), or the number of events.
  __device__ uint32_t trace_prefix(unsigned char *out, size_t stride, uint32_t *fid_stop, uint32_t *max_n) {
    init_shot(0);
    cur = C->n_sites;
    nxt = 0xFFFFFFFFu;
    const Ev<W> *evs = reinterpret_cast<const Ev<W> *>(C->ev);
    const uint32_t n_events = C->n_events;
    uint32_t ev = 0, fs = n_events, mx = 0;
    for (; ev <= n_events; ++ev) {
      save_snapshot(out + (size_t)ev * stride);
      mx = nnz > mx ? nnz : mx;
      if (ev == n_events) break;
      const uint32_t w0 = __ldg(&evs[ev].w0), type = ev_type(w0);
      if ((type == EV_MEAS_A || type == EV_MEAS_B) && (ev_flags(w0) & F_FIDELITY) && fs == n_events) fs = ev;
      undecided = false;
      step(ev);
      if (status != ST_RUN || undecided || nnz > kSnapMax) break;
    }
    t.sync();
    *fid_stop = fs;
    *max_n = mx;
    return ev;
  }

  __device__ __forceinline__ void step(uint32_t ev) {
    const Ev<W> *evs = reinterpret_cast<const Ev<W> *>(C->ev);
    {
      cur_ev = ev;
      const Ev<W> *E = evs + ev;
      const uint4 hdr = __ldg(reinterpret_cast<const uint4 *>(E));
      // dsd, dss, beta, gamma: 4 W words after the header
      uint64_t body[4 * W];
      const ulonglong2 *bp = reinterpret_cast<const ulonglong2 *>(&E->dsd[0]);
#pragma unroll
      for (int k = 0; k < 2 * W; ++k) {
        ulonglong2 v = __ldg(bp + k);
        body[2 * k] = v.x;
        body[2 * k + 1] = v.y;
      }
      const uint64_t *dsd = body, *dss = body + W, *beta = body + 2 * W, *gamma = body + 3 * W;
      if (kRegCapable && !reg && nnz <= (uint32_t)G) reg_load();
      while (nxt < hdr.y && status == ST_RUN) {
        apply_error(nxt);
        draw_next();
      }
      if (status != ST_RUN) return;
#pragma unroll
      for (int w = 0; w < W; ++w) {
        sd[w] ^= dsd[w];
        ss[w] ^= dss[w];
      }
      const uint32_t w0 = hdr.x, type = ev_type(w0), flags = ev_flags(w0);
      switch (type) {
        case EV_ROT: rot(w0, hdr.z, beta, gamma); break;
        case EV_ROT_DIAG: rot_diag(w0, hdr.z, gamma); break;
        case EV_MEAS_A:
        case EV_MEAS_B: {
          force = P.fid_mode && (flags & F_FIDELITY);
          int m = (type == EV_MEAS_A) ? meas_a(w0, hdr.z, gamma) : meas_b(hdr.z, (uint32_t)beta[0]);
          if (force && m == -1 && status == ST_RUN) {  // +1 impossible: F = 0, the shot ends kept
            fid = 0.0;
            status = ST_KEPT;
            break;
          }
          lastm = m;
          if (flags & F_RECORD) set_record(hdr.w, m);
          if ((flags & F_COND_LAST) && m == -1 && status == ST_RUN) {  // fused reset correction
            uint64_t xb[W], xg[W];
            uint32_t pe = 0;
#pragma unroll
            for (int w = 0; w < W; ++w) {
              xb[w] = __ldg(&E->xbeta[w]);
              xg[w] = __ldg(&E->xgamma[w]);
              pe += __popcll(sd[w] & xb[w]) + __popcll(ss[w] & xg[w]);
            }
            apply_pauli(xb, xg, (ev_xe0(w0) + 2u * pe) & 3u);
          }
          if ((flags & F_DETECTOR) && ((m == -1 ? 1u : 0u) ^ ((flags & F_INVERT) ? 1u : 0u)))
            status = ST_DISC;  // fused detector on this record
          break;
        }
        case EV_PAULI: {
          uint32_t cond = 0;
          if (flags & F_COND_LAST) cond = (lastm == -1);
          else cond = rec_bit((int32_t)hdr.z) ^ rec_bit((int32_t)hdr.w);
          if (cond) {
            uint32_t pe = 0;
#pragma unroll
            for (int w = 0; w < W; ++w) pe += __popcll(sd[w] & beta[w]) + __popcll(ss[w] & gamma[w]);
            apply_pauli(beta, gamma, (ev_e0(w0) + 2u * pe) & 3u);
          }
          break;
        }
        case EV_PARITY: {
          int par = chain ^ (int)rec_bit((int32_t)hdr.z) ^ (int)rec_bit((int32_t)hdr.w) ^
                    ((flags & F_INVERT) ? 1 : 0);
          if (flags & F_CHAIN) {
            chain = par;
          } else {
            chain = 0;
            if ((flags & F_DETECTOR) && par) status = ST_DISC;
            if ((flags & F_OBSERVABLE) && par) logical = 1;
          }
          break;
        }
        default: break;
      }
    }
  }

  __device__ void finish(uint64_t local, uint64_t off, uint32_t ci, unsigned long long (*btally)[5]) {
    if (status == ST_RERUN) {
      if (lane == 0) {
        unsigned long long i = atomicAdd(P.n_rerun, 1ull);
        if (i < P.rerun_cap) P.rerun[i] = (uint32_t)local;
        if (P.n_rerun_total) atomicAdd(P.n_rerun_total, 1ull);
      }
      t.sync();
      return;
    }
    if (lane == 0) {
      atomicAdd(&btally[ci][0], 1ull);
      if (status == ST_DISC) atomicAdd(&btally[ci][1], 1ull);
      else if (status == ST_OVF) atomicAdd(&btally[ci][2], 1ull);
      else if (status == ST_KEPT) {
        atomicAdd(&btally[ci][3], 1ull);
        if (logical) atomicAdd(&btally[ci][4], 1ull);
        if (P.fid_mode && C->fsum) atomicAdd(C->fsum, fid);
      }
      if (off < C->out_limit && C->status) C->status[off] = (uint8_t)status;
    }
    if (off < C->out_limit && C->records)
      for (uint32_t w = lane; w < C->rw; w += G) C->records[off * C->rw + w] = rec[w];
    if (ci == 0 && off < P.st_limit) {
      if (kRegCapable && reg) reg_spill();
      if (lane == 0) {
        P.st_nnz[off] = nnz;
        P.st_signs[off * 4 + 0] = sd[0];
        P.st_signs[off * 4 + 1] = (W == 2) ? sd[W - 1] : 0ull;
        P.st_signs[off * 4 + 2] = ss[0];
        P.st_signs[off * 4 + 3] = (W == 2) ? ss[W - 1] : 0ull;
      }
      for (uint32_t i = lane; i < nnz && i < P.st_stride; i += G) {
        Key<W> k = key(i);
        size_t o = (size_t)off * P.st_stride + i;
        P.st_keys[2 * o] = k.w[0];
        P.st_keys[2 * o + 1] = (W == 2) ? k.w[W - 1] : 0ull;
        P.st_vals[2 * o] = (double)vals[i].x;
        P.st_vals[2 * o + 1] = (double)vals[i].y;
      }
    }
    t.sync();
  }
};

constexpr int kBlock = 128;
// Register budget: resident 128-thread blocks per SM the compiler must allow
// (FP32: 6 -> 80 registers, FP64: 5 -> 96 registers), tuned on GB300.
#ifndef SOFT_MIN_BLOCKS_F32
#define SOFT_MIN_BLOCKS_F32 6
#endif
#ifndef SOFT_MIN_BLOCKS_F64
#define SOFT_MIN_BLOCKS_F64 5
#endif

template <typename R, int W, int G>
__global__ void __launch_bounds__(kBlock, sizeof(R) == 4 ? SOFT_MIN_BLOCKS_F32 : SOFT_MIN_BLOCKS_F64) shot_kernel(
    const __grid_constant__ ShotParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long btally[kMaxCirc][5];
  auto block = cg::this_thread_block();
  auto tile = cg::tiled_partition<G>(block);
  const uint32_t n_circ = P.n_circ < (uint32_t)kMaxCirc ? P.n_circ : (uint32_t)kMaxCirc;
  for (uint32_t i = threadIdx.x; i < 5 * n_circ; i += blockDim.x) btally[i / 5][i % 5] = 0ull;
  __syncthreads();
  const uint32_t gid = threadIdx.x / G;  // blockDim.x is a multiple of G
  const size_t gbytes = group_bytes<R, W>(P.cap, P.rw_max);
  unsigned char *base = P.gslab ? P.gslab + ((size_t)blockIdx.x * (blockDim.x / G) + gid) * gbytes
                                : smem + (size_t)gid * gbytes;
  Shot<R, W, G> s(tile, P, base);
  const unsigned long long n_items = P.n_items_dev ? *P.n_items_dev : P.n_items;
  const unsigned long long item_base = P.item_base_dev ? *P.item_base_dev : P.item_base;
  for (;;) {
    unsigned long long item = 0;
    if (tile.thread_rank() == 0) item = atomicAdd(P.next_item, 1ull);
    item = tile.shfl(item, 0);
    if (item >= n_items) break;
    if (P.list && item >= P.rerun_cap) break;  // a list never holds more than its capacity
    uint64_t local = P.list ? (uint64_t)P.list[item] : (uint64_t)item;
    uint32_t rec = kNoRecord;  // an entry naming a spill record resumes the shot a lane handed over
    if (P.list && (local & kSpillRef) && P.sp) {
      rec = (uint32_t)local & ~kSpillRef;
      if (rec >= P.sp_cap) break;  // never: records are taken below the pool's capacity
      local = Spill<R, W>(P.sp, P.sp_cap, P.rw_max).ha[rec].x;
    }
    const uint64_t g = item_base + local;
    // circuit of item g: the last one whose item range starts at or before g
    uint32_t lo = 0, hi = n_circ;
    while (hi - lo > 1u) {
      const uint32_t mid = (lo + hi) >> 1;
      if (P.circ[mid].item_begin <= g) lo = mid;
      else hi = mid;
    }
    s.C = &P.circ[lo];
    const uint64_t off = g - s.C->item_begin;
    s.run(s.C->first_shot + off, rec);
    s.finish(local, off, lo, btally);
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < 5 * n_circ; i += blockDim.x)
    if (btally[i / 5][i % 5]) atomicAdd(&P.circ[i / 5].tally[i % 5], btally[i / 5][i % 5]);
}

__global__ void advance_kernel(unsigned long long *item_base, unsigned long long step) { *item_base += step; }

// One warp records the noiseless run of circuit 0 (see Shot::trace_prefix).
template <typename R, int W>
__global__ void __launch_bounds__(32) prefix_kernel(const __grid_constant__ ShotParams P, unsigned char *out,
                                                    size_t stride, uint32_t *stop) {
  extern __shared__ __align__(16) unsigned char smem[];
  auto tile = cg::tiled_partition<32>(cg::this_thread_block());
  Shot<R, W, 32> s(tile, P, smem);
  s.C = &P.circ[0];
  uint32_t fs = 0, mx = 0;
  const uint32_t ev = s.trace_prefix(out, stride, &fs, &mx);
  if (tile.thread_rank() == 0) {
    stop[0] = ev;
    stop[1] = fs;
    stop[2] = mx;
  }
}

template <typename R, int W>
cudaError_t prefix_t(const ShotParams &p, unsigned char *out, uint32_t *stop, cudaStream_t st) {
  const size_t gb = group_bytes<R, W>(p.cap, p.rw_max);
  auto kern = prefix_kernel<R, W>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gb);
  if (e != cudaSuccess) return e;
  kern<<<1, 32, gb, st>>>(p, out, Shot<R, W, 32>::snap_stride(p.circ[0].rw), stop);
  return cudaGetLastError();
}

template <typename R, int W, int G>
cudaError_t prepare_t(const ShotParams &p, int blocks_per_sm, LaunchCfg *cfg) {
  auto kern = shot_kernel<R, W, G>;
  const size_t gb = group_bytes<R, W>(p.cap, p.rw_max);
  const size_t limit = 227 * 1024 - sizeof(unsigned long long) * 5 * kMaxCirc;
  size_t gpb = kBlock / G;
  if (p.groups_per_block && p.groups_per_block < gpb) gpb = p.groups_per_block;
  cfg->kern = reinterpret_cast<const void *>(kern);
  if (p.gslab) {
    if (!p.gslab_blocks) return cudaErrorInvalidValue;
    cfg->grid = p.gslab_blocks;
    cfg->block = (unsigned)(gpb * G);
    cfg->smem = 0;
    return cudaSuccess;
  }
  while (gpb > 1 && gpb * gb > limit) gpb >>= 1;
  if (gpb * gb > limit) return cudaErrorInvalidConfiguration;
  const int block = (int)(gpb * G);
  const size_t smem = gpb * gb;
  static int configured_smem = -1;
  if (configured_smem < (int)smem) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured_smem = (int)smem;
  }
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, block, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  if (blocks_per_sm > 0 && blocks_per_sm < occ) occ = blocks_per_sm;
  long long grid = (long long)occ * sms;
  const long long groups = (long long)gpb;
  if (!p.n_items_dev) {
    long long need = ((long long)p.n_items + groups - 1) / groups;
    if (need < grid) grid = need > 0 ? need : 1;
  }
  cfg->grid = (unsigned)grid;
  cfg->block = (unsigned)block;
  cfg->smem = smem;
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_advance(unsigned long long *item_base, unsigned long long step, cudaStream_t stream) {
  advance_kernel<<<1, 1, 0, stream>>>(item_base, step);
  return cudaGetLastError();
}

size_t global_slab_bytes(int fp32, uint32_t W, uint32_t cap, uint32_t rw, uint32_t blocks) {
  return group_smem_bytes(fp32, W, cap, rw) * (size_t)(kBlock / 32) * blocks;
}

size_t group_smem_bytes(int fp32, uint32_t W, uint32_t cap, uint32_t rw) {
  if (fp32) return W == 1 ? group_bytes<float, 1>(cap, rw) : group_bytes<float, 2>(cap, rw);
  return W == 1 ? group_bytes<double, 1>(cap, rw) : group_bytes<double, 2>(cap, rw);
}

cudaError_t prepare_shots(const ShotParams &p, int fp32, uint32_t W, uint32_t group, int blocks_per_sm,
                          LaunchCfg *cfg) {
#define SOFT_DISPATCH(R, WW, GG) return prepare_t<R, WW, GG>(p, blocks_per_sm, cfg)
  if (fp32) {
    if (W == 1) {
      if (group == 16) SOFT_DISPATCH(float, 1, 16);
      SOFT_DISPATCH(float, 1, 32);
    }
    if (group == 16) SOFT_DISPATCH(float, 2, 16);
    SOFT_DISPATCH(float, 2, 32);
  }
  if (W == 1) {
    if (group == 16) SOFT_DISPATCH(double, 1, 16);
    SOFT_DISPATCH(double, 1, 32);
  }
  if (group == 16) SOFT_DISPATCH(double, 2, 16);
  SOFT_DISPATCH(double, 2, 32);
#undef SOFT_DISPATCH
}

cudaError_t launch_prepared(const LaunchCfg &cfg, const ShotParams &p, cudaStream_t stream) {
  void *args[] = {const_cast<ShotParams *>(&p)};
  return cudaLaunchKernel(cfg.kern, dim3(cfg.grid), dim3(cfg.block), args, cfg.smem, stream);
}

cudaError_t launch_shots(const ShotParams &p, int fp32, uint32_t W, uint32_t group, int blocks_per_sm,
                         cudaStream_t stream, int *grid_out) {
  LaunchCfg cfg{};
  ShotParams q = p;
  q.hs_max = hash_slots(q.cap);
  cudaError_t e = prepare_shots(q, fp32, W, group, blocks_per_sm, &cfg);
  if (e != cudaSuccess) return e;
  if (grid_out) *grid_out = (int)cfg.grid;
  return launch_prepared(cfg, q, stream);
}

uint32_t hash_slots_for(uint32_t cap) { return hash_slots(cap); }

size_t prefix_stride(int fp32, uint32_t W, uint32_t rw) {
  if (fp32) return W == 1 ? Shot<float, 1, 32>::snap_stride(rw) : Shot<float, 2, 32>::snap_stride(rw);
  return W == 1 ? Shot<double, 1, 32>::snap_stride(rw) : Shot<double, 2, 32>::snap_stride(rw);
}

cudaError_t launch_prefix(const ShotParams &p, int fp32, uint32_t W, unsigned char *out, uint32_t *stop,
                          cudaStream_t st) {
  ShotParams q = p;
  q.hs_max = hash_slots(q.cap);
  if (fp32) return W == 1 ? prefix_t<float, 1>(q, out, stop, st) : prefix_t<float, 2>(q, out, stop, st);
  return W == 1 ? prefix_t<double, 1>(q, out, stop, st) : prefix_t<double, 2>(q, out, stop, st);
}

}  // namespace soft
