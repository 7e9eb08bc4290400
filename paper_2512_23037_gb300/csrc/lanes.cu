// lanes.cu -- shot kernel with one shot per lane, 32 shots per warp, all at the
// same event.
//
// Shots are first bucketed by the event they start at (the event that applies
// their first error, capped at the end of the circuit's recorded noiseless run).
// Every warp then walks the events in order. Its idle lanes claim shots from the
// bucket of the event it is at, load the noiseless run's state there, and the
// warp executes each event once for all its lanes: the event is decoded once,
// and every lane updates its own shot's coefficient map, kept in shared memory
// (entry i of lane l at row i, column l). A rotation whose map would outgrow
// kLaneCap entries hands the shot over: its state at the top of that event goes
// to a spill record, which the warp-per-shot kernel's next pass resumes. The
// per-shot arithmetic is that of the warp-per-shot kernel (the same formulas,
// pruning thresholds and outcome rule), entry by entry. In a batch, each circuit
// has its own range of buckets and a warp serves one circuit at a time; the shots
// of circuits whose maps outgrow a lane go straight to the warp pass.
//
// Most shots end at the first detector after their first error, but a few run to
// the end of the circuit, and they would hold a warp with a few active lanes. So a
// warp left with at most kEvictBelow active lanes writes their shots' state to a
// spill pool and moves on to fresh shots. The next round (another launch) buckets
// the evicted shots by the event they resume at, and packs them into warps again.
// The last round evicts nothing. Which lane runs a shot does not change its
// arithmetic, so the results are those of a single round.
#include <cooperative_groups.h>

#include "device_common.cuh"
#include "kernels.cuh"
#include "shot_common.cuh"

namespace soft {
namespace {

using namespace dev;
namespace cg = cooperative_groups;

enum : int { LS_RUN = -1, LS_KEPT = 0, LS_DISC = 1, LS_OVF = 2, LS_ERR = 3, LS_RERUN = 4, LS_HAND = 5 };
constexpr int kLaneBlock = 128;
constexpr uint32_t kLaneMaxBuckets = 50000;  // the pre-pass histogram of all buckets: 200 KB of shared memory
#ifndef SOFT_LANE_EVICT
#define SOFT_LANE_EVICT 8
#endif
constexpr uint32_t kEvictBelow = SOFT_LANE_EVICT;  // a warp with this many active lanes or fewer evicts them
#ifndef SOFT_LANE_ROUNDS
#define SOFT_LANE_ROUNDS 2
#endif
constexpr uint32_t kLaneRounds = SOFT_LANE_ROUNDS;  // rounds per chunk, the last without eviction
static_assert(kLaneRounds >= 1 && kLaneRounds <= 8, "lane rounds");


// The wide round's lanes: shots handed over by the first rounds continue in lanes
// of twice the map.
constexpr uint32_t kWideCap = 2 * kLaneCap;

template <typename R, int W, uint32_t Cap>
__host__ __device__ inline size_t lane_warp_bytes(uint32_t rw) {
  // map keys and values; record words
  return (size_t)Cap * W * 8 * 32 + (size_t)Cap * sizeof(Cx<R>) * 32 + (size_t)rw * 8 * 32;
}

// Partner indices, 5 bits per entry for maps of up to 32 entries: nibbles of
// entries 0-15 and 16-31, and a mask of the indices' fifth bit.
template <uint32_t Cap>
struct PartIdx {
  uint64_t lo = 0, hi = 0;
  uint32_t b4 = 0;
  __device__ __forceinline__ void set(uint32_t i, uint32_t j) {
    const uint64_t v = (uint64_t)(j & 15u) << (4 * (i & 15u));
    if (Cap <= 16 || i < 16) lo |= v;
    else hi |= v;
    if (Cap > 16) b4 |= ((j >> 4) & 1u) << i;
  }
  __device__ __forceinline__ uint32_t get(uint32_t i) const {
    const uint64_t w = (Cap <= 16 || i < 16) ? lo : hi;
    const uint32_t j = (uint32_t)(w >> (4 * (i & 15u))) & 15u;
    return Cap > 16 ? j | (((b4 >> i) & 1u) << 4) : j;
  }
};

template <typename R, int W, uint32_t Cap>
struct LaneShot {
  static_assert(Cap <= 32, "lane map masks are 32-bit");
  const ShotParams &P;
  const CircDev *C;
  uint32_t lane;
  uint64_t *keys;  // [i][w][lane]
  Cx<R> *vals;     // [i][lane]
  uint64_t *rec;           // [w][lane]
  // per-lane shot state
  uint64_t shot;
  uint32_t n;
  uint64_t sd[W], ss[W];
  uint32_t nxt, cur, kblk, w2;
  int status, chain, logical, lastm;
  double fid;
  bool force;

  // FP64 prune test (see is_small): high words of sqrt(tau/2) (1 - 2^-18) and sqrt(tau) (1 + 2^-18)
  uint32_t hs_lo = 0, hs_hi = 0;

  __device__ LaneShot(const ShotParams &p, unsigned char *base) : P(p), C(&p.circ[0]) {
    lane = threadIdx.x & 31u;
    if (sizeof(R) == 8) {
      hs_lo = (uint32_t)((unsigned long long)__double_as_longlong(sqrt(0.5 * p.tau) * (1.0 - 0x1p-18)) >> 32);
      hs_hi = (uint32_t)((unsigned long long)__double_as_longlong(sqrt(p.tau) * (1.0 + 0x1p-18)) >> 32);
    }
    const size_t kb = (size_t)Cap * W * 8 * 32, vb = (size_t)Cap * sizeof(Cx<R>) * 32;
    keys = reinterpret_cast<uint64_t *>(base);
    vals = reinterpret_cast<Cx<R> *>(base + kb);
    rec = reinterpret_cast<uint64_t *>(base + kb + vb);
  }

  __device__ __forceinline__ Key<W> key(uint32_t i) const {
    Key<W> k;
#pragma unroll
    for (int w = 0; w < W; ++w) k.w[w] = keys[((size_t)i * W + w) * 32 + lane];
    return k;
  }
  __device__ __forceinline__ void set_key(uint32_t i, const Key<W> &k) {
#pragma unroll
    for (int w = 0; w < W; ++w) keys[((size_t)i * W + w) * 32 + lane] = k.w[w];
  }
  __device__ __forceinline__ Cx<R> val(uint32_t i) const { return vals[(size_t)i * 32 + lane]; }
  __device__ __forceinline__ void set_val(uint32_t i, Cx<R> v) { vals[(size_t)i * 32 + lane] = v; }
  // Partners (a, a ^ x) differ in bit `bit`, set in x. Each entry with the bit clear
  // looks for its partner among the entries with it set (mask `him`). Out: `paired`,
  // the entries with the bit set that have a partner; `has`, those with it clear that
  // have one; part, the partner's index.
  __device__ void partners(uint32_t n0, uint32_t bit, const uint64_t *x, uint32_t &paired, uint32_t &has,
                           PartIdx<Cap> &part) const {
    uint32_t him = 0;
#pragma unroll 1
    for (uint32_t i = 0; i < n0; ++i) him |= kbit(key(i), bit) << i;
    paired = has = 0;
    part = PartIdx<Cap>{};
    const uint32_t all = n0 >= 32u ? 0xFFFFFFFFu : (1u << n0) - 1u;
#pragma unroll 1
    for (uint32_t lo = ~him & all; lo; lo &= lo - 1u) {
      const uint32_t i = __ffs(lo) - 1;
      const Key<W> pk = kxor(key(i), x);
#pragma unroll 1
      for (uint32_t m = him & ~paired; m; m &= m - 1u) {
        const uint32_t j = __ffs(m) - 1;
        if (keq(key(j), pk)) {
          paired |= 1u << j;
          has |= 1u << i;
          part.set(i, j);
          break;
        }
      }
    }
  }
  // The map would outgrow the lane before pruning. Overflow is decided after pruning
  // (|v| > the circuit's cap), so the warp pass at the circuit's cap, which stages the
  // whole update before it prunes, reruns the shot (every lane run has that pass).
  __device__ void fail_capacity() { status = P.small_pass ? LS_RERUN : LS_OVF; }
  __device__ void fail_check(uint32_t code, uint64_t value) {
    status = LS_ERR;
    if (P.diag && atomicAdd(&P.diag[0], 1ull) == 0ull) {
      P.diag[1] = ((unsigned long long)code << 32);
      P.diag[2] = shot;
      P.diag[3] = value;
    }
  }
  // |v|^2 < tau, the pruning test, decided exactly as the norm computed in R decides it.
  // FP64: when both |re| and |im| lie below sqrt(tau/2) (1 - 2^-18), or either lies above
  // sqrt(tau) (1 + 2^-18), integer compares of their high words settle it (the computed
  // norm's rounding cannot cross tau there); only values in that narrow band compute
  // the norm on the FP64 pipe, GB300's narrowest.
  __device__ __forceinline__ bool is_small(Cx<R> v, R tau) const {
    if (sizeof(R) == 4) return norm2(v) < tau;
    const uint32_t hx = (uint32_t)((unsigned long long)__double_as_longlong((double)v.x) >> 32) & 0x7FFFFFFFu;
    const uint32_t hy = (uint32_t)((unsigned long long)__double_as_longlong((double)v.y) >> 32) & 0x7FFFFFFFu;
    if (hx > hs_hi || hy > hs_hi) return false;
    if (hx < hs_lo && hy < hs_lo) return true;
    return norm2(v) < tau;
  }
  // keep the entries with |v|^2 >= tau, in order
  __device__ void prune() {
    const R tau = (R)P.tau;
    uint32_t o = 0;
#pragma unroll 1
    for (uint32_t i = 0; i < n; ++i) {
      const Cx<R> v = val(i);
      if (!is_small(v, tau)) {
        if (o != i) {
          set_key(o, key(i));
          set_val(o, v);
        }
        ++o;
      }
    }
    n = o;
  }

  __device__ double uniform(uint32_t ord) const {
    uint4 w = philox(P.seed, shot, 1u, ord);
    uint64_t m = ((uint64_t)w.x << 21) ^ (uint64_t)(w.y >> 11);
    return (double)m * 0x1p-53;
  }
  // Outcome +1 iff u < p, with p = sp / (sp + sm) snapped to 0 or 1 within 1e-12:
  // decided as u (sp + sm) < sp, so that only the fidelity mode divides.
  __device__ __forceinline__ int pick(uint32_t ord, double sp, double sm) {
    const double tot = sp + sm;
    if (!(tot > 0.0)) return -1;
    const bool zero = sp < 1e-12 * tot, one = sp > (1.0 - 1e-12) * tot;
    if (force) {
      if (zero) return -1;
      fid *= one ? 1.0 : sp / tot;
      return 1;
    }
    if (zero) return -1;
    if (one) return 1;
    return uniform(ord) * tot < sp ? 1 : -1;
  }
  __device__ __forceinline__ R inv_sqrt(double x) const {
    if (sizeof(R) == 4) return (R)rsqrtf((float)x);
    return (R)rsqrt(x);
  }

  // ---- start: shot s at event e of the noiseless run
  // (the pre-pass drew the shot's first error: its noise cursor comes with the item)
  __device__ void begin(uint64_t s, uint32_t e, uint4 cursor) {
    shot = s;
    status = LS_RUN;
    force = false;
    nxt = cursor.x;
    cur = cursor.y;
    kblk = cursor.z;
    w2 = cursor.w;
    if (kblk == 0xFFFFFFFFu) {
      status = LS_ERR;
      return;
    }
    const unsigned char *in = C->traj + (size_t)e * C->traj_stride;
    const SnapHdr *h = reinterpret_cast<const SnapHdr *>(in);
    const uint64_t *r_in = reinterpret_cast<const uint64_t *>(in + sizeof(SnapHdr));
    const uint64_t *k_in = r_in + C->rw;
    const Cx<R> *v_in = reinterpret_cast<const Cx<R> *>(k_in + kSnapMax * W);
    n = __ldg(&h->nnz);
    chain = (int)__ldg(&h->chain);
    logical = (int)__ldg(&h->logical);
    lastm = (int)__ldg(&h->lastm);
    fid = __ldg(&h->fid);
#pragma unroll
    for (int w = 0; w < W; ++w) {
      sd[w] = __ldg(&h->sd[w]);
      ss[w] = __ldg(&h->ss[w]);
    }
#pragma unroll 1
    for (uint32_t w = 0; w < C->rw; ++w) rec[(size_t)w * 32 + lane] = __ldg(&r_in[w]);
    if (n > Cap) {
      fail_capacity();
      return;
    }
#pragma unroll 1
    for (uint32_t i = 0; i < n; ++i) {
      Key<W> k;
#pragma unroll
      for (int w = 0; w < W; ++w) k.w[w] = __ldg(&k_in[i * W + w]);
      set_key(i, k);
      set_val(i, v_in[i]);
    }
  }

  // ---- eviction: the shot's whole state into record r, to resume at event ev
  __device__ void evict(const Spill<R, W> &S, uint32_t r, uint32_t item, uint32_t ev) const {
    const size_t c = S.cap;
    S.ha[r] = make_uint4(item, ev, n, (uint32_t)(chain & 1) | ((uint32_t)(logical & 1) << 1) |
                                          (((uint32_t)lastm & 255u) << 8));
    S.hb[r] = make_uint4(nxt, cur, kblk, w2);
    S.fid[r] = fid;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      S.sd[w * c + r] = sd[w];
      S.ss[w * c + r] = ss[w];
    }
#pragma unroll 1
    for (uint32_t w = 0; w < C->rw; ++w) S.rec[w * c + r] = rec[(size_t)w * 32 + lane];
#pragma unroll 1
    for (uint32_t i = 0; i < n; ++i) {
      const Key<W> k = key(i);
#pragma unroll
      for (int w = 0; w < W; ++w) S.keys[((size_t)i * W + w) * c + r] = k.w[w];
      S.vals[(size_t)i * c + r] = val(i);
    }
  }
  // ---- resumption from record r; returns the shot's item (chunk-local index)
  __device__ uint32_t resume(const Spill<R, W> &S, uint32_t r, uint64_t first) {
    const size_t c = S.cap;
    const uint4 a = S.ha[r], b = S.hb[r];
    shot = first + a.x;
    status = LS_RUN;
    force = false;
    n = a.z;
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
#pragma unroll 1
    for (uint32_t w = 0; w < C->rw; ++w) rec[(size_t)w * 32 + lane] = S.rec[w * c + r];
    if (n > kLaneCap) {  // a record never holds more; checked so that a bad record cannot index past the map
      fail_check(CHK_NNZ, n);
      n = 0;
      return a.x;
    }
#pragma unroll 1
    for (uint32_t i = 0; i < n; ++i) {
      Key<W> k;
#pragma unroll
      for (int w = 0; w < W; ++w) k.w[w] = S.keys[((size_t)i * W + w) * c + r];
      set_key(i, k);
      set_val(i, S.vals[(size_t)i * c + r]);
    }
    return a.x;
  }

  // ---- the shot's final state (signs, keys, values) for state capture at offset off
  __device__ void capture(uint64_t off) const {
    P.st_nnz[off] = n;
    P.st_signs[off * 4 + 0] = sd[0];
    P.st_signs[off * 4 + 1] = (W == 2) ? sd[W - 1] : 0ull;
    P.st_signs[off * 4 + 2] = ss[0];
    P.st_signs[off * 4 + 3] = (W == 2) ? ss[W - 1] : 0ull;
#pragma unroll 1
    for (uint32_t i = 0; i < n && i < P.st_stride; ++i) {
      const Key<W> k = key(i);
      const Cx<R> v = val(i);
      const size_t o = (size_t)off * P.st_stride + i;
      P.st_keys[2 * o] = k.w[0];
      P.st_keys[2 * o + 1] = (W == 2) ? k.w[W - 1] : 0ull;
      P.st_vals[2 * o] = (double)v.x;
      P.st_vals[2 * o + 1] = (double)v.y;
    }
  }

  // ---- Paulis: v'_{a^beta} = i^{e + 2 gamma.a} v_a
  __device__ void apply_pauli(const uint64_t *beta, const uint64_t *gamma, uint32_t e) {
#pragma unroll 1
    for (uint32_t i = 0; i < n; ++i) {
      const Key<W> k = key(i);
      set_val(i, ipow(val(i), e + 2u * kpar(k, gamma)));
      set_key(i, kxor(k, beta));
    }
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
    apply_pauli(beta, gamma, ((__ldg(&S->c0) >> (2u * code)) + 2u * pe) & 3u);
  }

  // ---- a I + b Z_q: paired entries (a, a^beta) mix, an unpaired entry gains its partner
  __device__ void rot(uint32_t w0, uint32_t ci, const uint64_t *beta, const uint64_t *gamma, bool diag) {
    uint32_t pe = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) pe += diag ? __popcll(ss[w] & gamma[w]) : __popcll(sd[w] & beta[w]) + __popcll(ss[w] & gamma[w]);
    const uint32_t e = (ev_e0(w0) + 2u * pe) & 3u;
    if (ci >= C->n_coef) {
      fail_check(CHK_COEF, ci);
      return;
    }
    const Coef *cf = C->coef + ci;
    Cx<R> a, b;
    if (sizeof(R) == 4) {
      const float4 f = __ldg(reinterpret_cast<const float4 *>(&cf->fa_re));
      a = Cx<R>{(R)f.x, (R)f.y};
      b = Cx<R>{(R)f.z, (R)f.w};
    } else {
      const double2 d0 = __ldg(reinterpret_cast<const double2 *>(&cf->a_re));
      const double2 d1 = __ldg(reinterpret_cast<const double2 *>(&cf->b_re));
      a = Cx<R>{(R)d0.x, (R)d0.y};
      b = Cx<R>{(R)d1.x, (R)d1.y};
    }
    const R tau = (R)P.tau;
    bool small = false;
    // the phase xi = i^e (-1)^{gamma.key} folded into b once per event: b_s = (-1)^s b i^e
    // (exact: a multiplication by i^e swaps and negates), so that an entry only selects one
    const Cx<R> bq = ipow(b, e), bn = Cx<R>{negr(bq.x), negr(bq.y)};
    if (diag) {
      // v' = (a + b xi) v: one complex product per entry
      const Cx<R> c0 = cadd(a, bq), c1 = cadd(a, bn);
#pragma unroll 1
      for (uint32_t i = 0; i < n; ++i) {
        const Cx<R> nv = cmul(kpar(key(i), gamma) ? c1 : c0, val(i));
        set_val(i, nv);
        small = small || is_small(nv, tau);
      }
      if (small) prune();
      return;
    }
    const uint32_t n0 = n;
    uint32_t paired, has;
    PartIdx<Cap> part;
    partners(n0, ev_lowbit(w0), beta, paired, has, part);
    // every entry without a partner gains one: if that outgrows the lane, nothing has
    // been written yet, and the shot can be taken over at the top of this event (by the
    // wide round's lanes, or a warp); otherwise (the wide round) it reruns in a warp
    if (n0 + (n0 - 2u * (uint32_t)__popc(has)) > Cap) {
      if (P.lane_hand && P.sp && P.small_pass && C->cap > Cap) status = LS_HAND;
      else fail_capacity();
      return;
    }
    uint32_t na = 0;
#pragma unroll 1
    for (uint32_t i = 0; i < n0; ++i) {
      if ((paired >> i) & 1u) continue;  // the pair's member with bit lowbit clear updates both
      const Key<W> k = key(i);
      const Key<W> pk = kxor(k, beta);
      const Cx<R> v = val(i);
      if ((has >> i) & 1u) {
        const uint32_t j = part.get(i);
        const Cx<R> vj = val(j);
        const Cx<R> ni = cadd(cmul(a, v), cmul(kpar(pk, gamma) ? bn : bq, vj));
        const Cx<R> nj = cadd(cmul(a, vj), cmul(kpar(k, gamma) ? bn : bq, v));
        set_val(i, ni);
        set_val((uint32_t)j, nj);
        small = small || is_small(ni, tau) || is_small(nj, tau);
      } else {
        const Cx<R> ni = cmul(a, v);
        const Cx<R> av = cmul(kpar(k, gamma) ? bn : bq, v);
        set_val(i, ni);
        if (n0 + na >= Cap) {
          fail_capacity();
          return;
        }
        set_key(n0 + na, pk);
        set_val(n0 + na, av);
        ++na;
        small = small || is_small(ni, tau) || is_small(av, tau);
      }
    }
    n = n0 + na;
    if (small) prune();
    if (n > C->cap) status = LS_OVF;  // the overflow rule, for circuits whose cap is below the lane's
  }

  // ---- measurement of P, beta = 0: lambda_a = c (-1)^{gamma.a}
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
    bool h0 = false, h1 = false;
#pragma unroll 1
    for (uint32_t i = 0; i < n; ++i) {
      if (kpar(key(i), gamma) ^ sgn) h1 = true;
      else h0 = true;
    }
    if (!(h0 && h1)) return h1 ? -1 : 1;
    double sp = 0.0, sm = 0.0;
#pragma unroll 1
    for (uint32_t i = 0; i < n; ++i) {
      const double a2 = norm2d(val(i));
      if (kpar(key(i), gamma) ^ sgn) sm += a2;
      else sp += a2;
    }
    const int m = pick(ord, sp, sm);
    const R sc = inv_sqrt(m == 1 ? sp : sm);
    const uint32_t want = (m == 1) ? 0u : 1u;
    const R tau = (R)P.tau;
    uint32_t o = 0;
#pragma unroll 1
    for (uint32_t i = 0; i < n; ++i) {
      const Key<W> k = key(i);
      if ((kpar(k, gamma) ^ sgn) != want) continue;
      const Cx<R> v = cscale(val(i), sc);
      if (is_small(v, tau)) continue;
      set_key(o, k);
      set_val(o, v);
      ++o;
    }
    n = o;
    return m;
  }

  // Entry i's pair after the relabel (entry i is not a paired a1): a0, v0 = v_{a0} and
  // x1 = xi_{a1} v_{a1} (zero when absent); j, the a1 partner that i consumes (-1 if none).
  __device__ void pair_at(uint32_t i, uint32_t p, const uint64_t *ep, const uint64_t *g2, uint32_t e2, uint32_t has,
                          const PartIdx<Cap> &part, Key<W> &a0, Cx<R> &v0, Cx<R> &x1, int &j) const {
    const Key<W> k = key(i);
    const bool hi = kbit(k, p);
    j = ((has >> i) & 1u) ? (int)part.get(i) : -1;
    Cx<R> v1{0, 0};
    v0 = Cx<R>{0, 0};
    if (hi) v1 = val(i);
    else {
      v0 = val(i);
      if (j >= 0) v1 = val((uint32_t)j);
    }
    a0 = hi ? kxor(k, ep) : k;
    x1 = ipow(v1, e2 + 2u * kpar(kxor(a0, ep), g2));
  }

  // ---- measurement of P, beta != 0 (case B): row operations on the signs, relabel,
  // pairing, replacement
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
    const uint32_t ssp = wbit<W>(ss, p);
    const uint32_t sdJ = wpar<W>(sd, J);
#pragma unroll
    for (int w = 0; w < W; ++w) ss[w] ^= (ssp ? J[w] : 0ull) ^ __ldg(&B->Hs[w]);
    if (sdJ ^ __ldg(&B->hdp)) wflip<W>(sd, p);
    const uint32_t e2 = (__ldg(&B->e0b) + 2u * (wbit<W>(sd, p) + wpar<W>(ss, g2))) & 3u;
    // relabel a_j ^= a_p (j in J)
#pragma unroll 1
    for (uint32_t i = 0; i < n; ++i) {
      const Key<W> k = key(i);
      if (kbit(k, p)) set_key(i, kxor(k, J));
    }
    // pair a0 (bit p clear) with a1 = a0 ^ e_p: first the outcome probabilities, then
    // the combined values (v0 + m x1) / sqrt(2 p_m)
    uint32_t paired, has;
    PartIdx<Cap> part;
    partners(n, p, ep, paired, has, part);
    double sp = 0.0, sm = 0.0;
#pragma unroll 1
    for (uint32_t i = 0; i < n; ++i) {
      if ((paired >> i) & 1u) continue;  // a paired a1 only feeds its a0's pair
      Key<W> a0;
      Cx<R> v0, x1;
      int j;
      pair_at(i, p, ep, g2, e2, has, part, a0, v0, x1, j);
      sp += 0.5 * norm2d(cadd(v0, x1));
      sm += 0.5 * norm2d(csub(v0, x1));
    }
    const int m = pick(ord, sp, sm);
    const R sc = inv_sqrt(2.0 * (m == 1 ? sp : sm));
    // In place: a pair's result goes to the slot of the entry that forms it (the a0
    // member, or a lone a1), and the consumed a1 partner's value is zeroed (the partners
    // were found before any write); the prune then drops the zeroed and the negligible
    // entries, keeping slot order.
#pragma unroll 1
    for (uint32_t i = 0; i < n; ++i) {
      if ((paired >> i) & 1u) continue;
      Key<W> a0;
      Cx<R> v0, x1;
      int j;
      pair_at(i, p, ep, g2, e2, has, part, a0, v0, x1, j);
      set_key(i, a0);
      set_val(i, cscale(m == 1 ? cadd(v0, x1) : csub(v0, x1), sc));
      if (j >= 0) set_val((uint32_t)j, Cx<R>{0, 0});  // only an a0 entry has a partner here
    }
    prune();
    // replacement: d_j <- d_j s_p (j in G), d_p <- old s_p, s_p <- m P
#pragma unroll
    for (int w = 0; w < W; ++w) sd[w] ^= (ssp ? __ldg(&B->G[w]) : 0ull) ^ __ldg(&B->Hd[w]);
    if (wbit<W>(sd, p) != ssp) wflip<W>(sd, p);
    const uint32_t newsp = (m == -1 ? 1u : 0u) ^ __ldg(&B->rP);
    if (wbit<W>(ss, p) != newsp) wflip<W>(ss, p);
    return m;
  }

  __device__ uint32_t rec_bit(int32_t r) const {
    return (r < 0 || (uint32_t)r >= 64u * C->rw) ? 0u : (uint32_t)((rec[(size_t)(r >> 6) * 32 + lane] >> (r & 63)) & 1ull);
  }

  // one event for this lane's shot
  __device__ void step(uint32_t ev, const uint4 &hdr, const uint64_t *body, const Ev<W> *E) {
    while (nxt < hdr.y && status == LS_RUN) {
      apply_error(nxt);
      if (!next_site(C, P.seed, shot, cur, kblk, nxt, w2)) status = LS_ERR;
    }
    if (status != LS_RUN) return;
    const uint64_t *dsd = body, *dss = body + W, *beta = body + 2 * W, *gamma = body + 3 * W;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      sd[w] ^= dsd[w];
      ss[w] ^= dss[w];
    }
    const uint32_t w0 = hdr.x, type = ev_type(w0), flags = ev_flags(w0);
    switch (type) {
      case EV_ROT: rot(w0, hdr.z, beta, gamma, false); break;
      case EV_ROT_DIAG: rot(w0, hdr.z, beta, gamma, true); break;
      case EV_MEAS_A:
      case EV_MEAS_B: {
        force = P.fid_mode && (flags & F_FIDELITY);
        const int m = (type == EV_MEAS_A) ? meas_a(w0, hdr.z, gamma) : meas_b(hdr.z, (uint32_t)beta[0]);
        if (status != LS_RUN) break;
        if (force && m == -1) {
          fid = 0.0;
          status = LS_KEPT;
          break;
        }
        lastm = m;
        if (flags & F_RECORD) {
          const uint32_t r = hdr.w;
          if (r >= 64u * C->rw) {
            fail_check(CHK_RECORD, r);
            break;
          }
          if (m < 0) rec[(size_t)(r >> 6) * 32 + lane] |= 1ull << (r & 63);
        }
        if ((flags & F_COND_LAST) && m == -1) {
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
        if ((flags & F_DETECTOR) && ((m == -1 ? 1u : 0u) ^ ((flags & F_INVERT) ? 1u : 0u))) status = LS_DISC;
        break;
      }
      case EV_PAULI: {
        uint32_t cond;
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
        const int par = chain ^ (int)rec_bit((int32_t)hdr.z) ^ (int)rec_bit((int32_t)hdr.w) ^
                        ((flags & F_INVERT) ? 1 : 0);
        if (flags & F_CHAIN) {
          chain = par;
        } else {
          chain = 0;
          if ((flags & F_DETECTOR) && par) status = LS_DISC;
          if ((flags & F_OBSERVABLE) && par) logical = 1;
        }
        break;
      }
      default: break;
    }
    if (status == LS_HAND) {  // back to the top of the event: the signs as before its XOR
#pragma unroll
      for (int w = 0; w < W; ++w) {
        sd[w] ^= dsd[w];
        ss[w] ^= dss[w];
      }
    }
    (void)ev;
  }
};

// ---- bucketing pre-pass. Buckets: per circuit of the run, one per event plus one
// (shots that start past the end), circuit after circuit from circuit.bucket0.
// The circuit of item g: the last one whose item range starts at or before g.
__device__ __forceinline__ uint32_t circ_of_item(const ShotParams &P, uint64_t g) {
  uint32_t lo = 0, hi = P.n_circ;
  while (hi - lo > 1u) {
    const uint32_t mid = (lo + hi) >> 1;
    if (P.circ[mid].item_begin <= g) lo = mid;
    else hi = mid;
  }
  return lo;
}
// The circuit of bucket g: the last one whose first bucket is at or before g.
__device__ __forceinline__ uint32_t circ_of_bucket(const ShotParams &P, uint32_t g) {
  uint32_t lo = 0, hi = P.n_circ;
  while (hi - lo > 1u) {
    const uint32_t mid = (lo + hi) >> 1;
    if (P.circ[mid].bucket0 <= g) lo = mid;
    else hi = mid;
  }
  return lo;
}
__global__ void lane_scan_kernel(const __grid_constant__ ShotParams P) {
  __shared__ uint32_t part[1024];
  const uint32_t nb = P.al_nb, tid = threadIdx.x, nt = blockDim.x;
  const uint32_t per = (nb + nt - 1) / nt, lo = tid * per < nb ? tid * per : nb, hi = lo + per < nb ? lo + per : nb;
  uint32_t sum = 0;
  for (uint32_t k = lo; k < hi; ++k) sum += P.al_count[k];
  part[tid] = sum;
  __syncthreads();
  if (tid == 0) {
    uint32_t run = 0;
    for (uint32_t k = 0; k < nt; ++k) {
      const uint32_t v = part[k];
      part[k] = run;
      run += v;
    }
    P.al_start[nb] = run;
  }
  __syncthreads();
  uint32_t run = part[tid];
  for (uint32_t k = lo; k < hi; ++k) {
    P.al_start[k] = run;
    run += P.al_count[k];
  }
}
// ---- round r >= 1: its records are those taken since round r - 1 began (the pool's
// count, capped at its capacity: reservations past it were not written)
__global__ void lane_round_setup_kernel(const __grid_constant__ ShotParams P) {
  const uint32_t r = P.lane_round;
  if (P.lane_wide_round) {  // the wide round: the handed-over shots' records
    const unsigned long long cap = P.sp_cap - P.sp_evict_cap;
    P.lr[2 + 2 * r] = P.sp_evict_cap;
    P.lr[3 + 2 * r] = P.lr[1] < cap ? P.lr[1] : cap;
    return;
  }
  const unsigned long long used = P.lr[0] < P.sp_evict_cap ? P.lr[0] : P.sp_evict_cap;
  const unsigned long long first = r == 1 ? 0ull : P.lr[2 + 2 * (r - 1)] + P.lr[3 + 2 * (r - 1)];
  P.lr[2 + 2 * r] = first;
  P.lr[3 + 2 * r] = used > first ? used - first : 0ull;
}
// ---- block-binned pre-pass: each block ranks its contiguous range of items per
// bucket with shared-memory atomics, then takes one global atomic per non-empty
// bucket for its base. The first errors cluster in a few buckets, and global
// atomics on one address serialise.
// Items of circuits whose maps outgrow a lane go to the warp pass's list instead: the
// block ranks them too and reserves their slots with one global atomic.
template <bool Resume, typename R, int W>
__global__ void __launch_bounds__(256) lane_bin_kernel(const __grid_constant__ ShotParams P) {
  extern __shared__ uint32_t hist[];  // nb buckets, then the block's count of warp-pass items
  const uint32_t nb = P.al_nb;
  for (uint32_t k = threadIdx.x; k <= nb; k += blockDim.x) hist[k] = 0u;
  __syncthreads();
  const unsigned long long n_items =
      Resume ? P.lr[3 + 2 * P.lane_round] : (P.n_items_dev ? *P.n_items_dev : P.n_items);
  const unsigned long long per = (n_items + gridDim.x - 1) / gridDim.x;
  const unsigned long long i0 = blockIdx.x * per, i1 = i0 + per < n_items ? i0 + per : n_items;
  const unsigned long long base = P.item_base_dev ? *P.item_base_dev : P.item_base;
  for (unsigned long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    uint32_t e;
    const CircDev *C;
    if (Resume) {
      const Spill<R, W> S(P.sp, P.sp_cap, P.rw_max);
      const uint4 a = S.ha[P.lr[2 + 2 * P.lane_round] + i];
      C = &P.circ[circ_of_item(P, base + a.x)];
      e = a.y < C->n_events ? a.y : C->n_events;  // a record always resumes at an event of its circuit
    } else {
      C = &P.circ[circ_of_item(P, base + i)];
      if (C->lanes_off) {
        reinterpret_cast<uint2 *>(P.al_ev)[i] = make_uint2(kNoRecord, atomicAdd(&hist[nb], 1u));
        continue;
      }
      uint32_t cur = 0, kblk = 0, nxt = 0, w2 = 0;
      if (!next_site(C, P.seed, C->first_shot + (base + i - C->item_begin), cur, kblk, nxt, w2))
        kblk = 0xFFFFFFFFu;  // a failure
      e = first_event(C, P.fid_mode, nxt);
      reinterpret_cast<uint4 *>(P.al_cursor)[i] = make_uint4(nxt, cur, kblk, w2);
    }
    e += C->bucket0;
    reinterpret_cast<uint2 *>(P.al_ev)[i] = make_uint2(e, atomicAdd(&hist[e], 1u));
  }
  __syncthreads();
  for (uint32_t k = threadIdx.x; k < nb; k += blockDim.x) {
    const uint32_t c = hist[k];
    P.al_base[(size_t)blockIdx.x * (nb + 1) + k] = c ? atomicAdd(&P.al_count[k], c) : 0u;
  }
  if (threadIdx.x == 0)
    P.al_base[(size_t)blockIdx.x * (nb + 1) + nb] = hist[nb] ? (uint32_t)atomicAdd(P.n_rerun, (unsigned long long)hist[nb]) : 0u;
}
// (same grid as lane_bin_kernel: it fixes each item's block)
template <bool Resume>
__global__ void __launch_bounds__(256) lane_bin_scatter_kernel(const __grid_constant__ ShotParams P) {
  const uint32_t nb = P.al_nb;
  const unsigned long long n_items =
      Resume ? P.lr[3 + 2 * P.lane_round] : (P.n_items_dev ? *P.n_items_dev : P.n_items);
  const unsigned long long per = (n_items + gridDim.x - 1) / gridDim.x;
  const unsigned long long i0 = blockIdx.x * per, i1 = i0 + per < n_items ? i0 + per : n_items;
  for (unsigned long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const uint2 er = reinterpret_cast<const uint2 *>(P.al_ev)[i];
    if (er.x == kNoRecord) {  // a shot of a circuit without lanes: the warp pass's list
      const unsigned long long slot = P.al_base[(size_t)blockIdx.x * (nb + 1) + nb] + er.y;
      if (slot < P.rerun_cap) P.rerun[slot] = (uint32_t)i;
      continue;
    }
    P.al_order[P.al_start[er.x] + P.al_base[(size_t)blockIdx.x * (nb + 1) + er.x] + er.y] = (uint32_t)i;
  }
}

// Blocks per SM each variant's shared memory allows (w42: FP32 16-entry lanes 6, FP64 4,
// the wide round's 32-entry lanes 3): the register budget is set not to lower it.
template <typename R, uint32_t Cap>
constexpr int kLaneMinBlocks() {
  return sizeof(R) == 4 ? (Cap <= 16 ? 6 : 3) : 4;
}

// Multi: the run holds several circuits (a warp serves one at a time); the single-
// circuit instantiation keeps circuit 0 and bucket offset 0 as constants. Cap: map
// entries per lane (kLaneCap in the first rounds, kWideCap in the wide round).
template <typename R, int W, bool Multi, uint32_t Cap>
__global__ void __launch_bounds__(kLaneBlock, kLaneMinBlocks<R, Cap>()) lane_kernel(const __grid_constant__ ShotParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  // per warp: tallies of its current circuit, added to the circuit's when the warp moves
  // to another circuit and at the end
  __shared__ unsigned long long wt[kLaneBlock / 32][5];
  const uint32_t warp = threadIdx.x / 32, lane = threadIdx.x & 31u;
  if (lane < 5) wt[warp][lane] = 0ull;
  __syncwarp();
  LaneShot<R, W, Cap> s(P, smem + (size_t)warp * lane_warp_bytes<R, W, Cap>(P.rw_max));
  const unsigned long long base = P.item_base_dev ? *P.item_base_dev : P.item_base;
  const unsigned long long n_items =
      P.lane_round ? P.lr[3 + 2 * P.lane_round] : (P.n_items_dev ? *P.n_items_dev : P.n_items);
  const unsigned long long rec0 = P.lane_round ? P.lr[2 + 2 * P.lane_round] : 0ull;
  const Spill<R, W> S(P.sp, P.sp_cap, P.rw_max);
  const uint32_t nb = P.al_nb;
  // warps start spread evenly over all buckets, so that they meet buckets that still hold shots
  const unsigned long long gw = (unsigned long long)blockIdx.x * (blockDim.x / 32) + warp;
  const unsigned long long nw = (unsigned long long)gridDim.x * (blockDim.x / 32);
  uint32_t g = (uint32_t)((gw * (unsigned long long)nb) / nw);
  uint32_t ci = Multi ? circ_of_bucket(P, g) : 0u;
  const CircDev *C = &P.circ[ci];
  uint32_t n_ev = C->n_events, e = Multi ? g - C->bucket0 : g;
  const Ev<W> *evs = reinterpret_cast<const Ev<W> *>(C->ev);
  s.C = C;
  auto flush = [&]() {  // the warp's tallies into its current circuit's
    __syncwarp();
    if (lane < 5 && wt[warp][lane]) {
      atomicAdd(&C->tally[lane], wt[warp][lane]);
      wt[warp][lane] = 0ull;
    }
    __syncwarp();
  };
  bool active = false;
  uint32_t item = 0;
  const unsigned long long limit = (n_items + 2ull) * (nb + 2ull) + 64ull;
  for (unsigned long long guard = 0; guard < limit; ++guard) {
    g = Multi ? C->bucket0 + e : e;
    // idle lanes claim shots that start at event e of circuit ci (one atomic per warp)
    const uint32_t idle = __ballot_sync(0xFFFFFFFFu, !active);
    if (idle) {
      const uint32_t b0 = __ldg(&P.al_start[g]), sz = __ldg(&P.al_start[g + 1]) - b0;
      uint32_t got0 = 0;
      const uint32_t leader = __ffs(idle) - 1;
      if (lane == leader) got0 = *(volatile unsigned int *)&P.al_next[g] < sz ? atomicAdd(&P.al_next[g], __popc(idle)) : sz;
      got0 = __shfl_sync(0xFFFFFFFFu, got0, leader);
      if (!active) {
        const uint32_t k = got0 + __popc(idle & ((1u << lane) - 1u));
        if (k < sz) {
          item = __ldg(&P.al_order[b0 + k]);
          if (item < n_items) {
            active = true;
            const uint64_t first = C->first_shot + base - (Multi ? C->item_begin : 0ull);  // shot of item i: first + i
            if (P.lane_round) item = s.resume(S, (uint32_t)(rec0 + item), first);
            else s.begin(first + item, e, reinterpret_cast<const uint4 *>(P.al_cursor)[item]);
          }
        }
      }
    }
    if (e < n_ev && __any_sync(0xFFFFFFFFu, active && s.status == LS_RUN)) {
      const Ev<W> *E = evs + e;
      const uint4 hdr = __ldg(reinterpret_cast<const uint4 *>(E));
      uint64_t body[4 * W];
      const ulonglong2 *bp = reinterpret_cast<const ulonglong2 *>(&E->dsd[0]);
#pragma unroll
      for (int k = 0; k < 2 * W; ++k) {
        const ulonglong2 v = __ldg(bp + k);
        body[2 * k] = v.x;
        body[2 * k + 1] = v.y;
      }
      if (active && s.status == LS_RUN) s.step(e, hdr, body, E);
    }
    // finish: ended, or past the last event
    if (active && (s.status != LS_RUN || e + 1u >= n_ev)) {
      if (s.status == LS_RUN) s.status = LS_KEPT;
      const uint64_t off = base + item - (Multi ? C->item_begin : 0ull);  // the shot's offset within its circuit
      uint32_t entry = item;  // a rerun starts the shot again from its start
      bool listed = true;
      if (s.status == LS_HAND) {  // or it resumes from its state at the top of event e
        const unsigned long long h = atomicAdd(&P.lr[1], 1ull);
        if (h < (unsigned long long)(P.sp_cap - P.sp_evict_cap)) {
          const uint32_t r = P.sp_evict_cap + (uint32_t)h;
          s.evict(S, r, item, e);
          entry = kSpillRef | r;    // in a warp, from the rerun list,
          listed = !P.lane_wide;    // or in the wide round, which takes every such record
        }
        s.status = LS_RERUN;
      }
      if (s.status == LS_RERUN) {
        if (listed) {
          const unsigned long long i = atomicAdd(P.n_rerun, 1ull);
          if (i < P.rerun_cap) P.rerun[i] = entry;
        }
        if (P.n_rerun_total) atomicAdd(P.n_rerun_total, 1ull);
      } else {
        atomicAdd(&wt[warp][0], 1ull);
        if (s.status == LS_DISC) atomicAdd(&wt[warp][1], 1ull);
        else if (s.status == LS_OVF) atomicAdd(&wt[warp][2], 1ull);
        else if (s.status == LS_KEPT) {
          atomicAdd(&wt[warp][3], 1ull);
          if (s.logical) atomicAdd(&wt[warp][4], 1ull);
          if (P.fid_mode && C->fsum) atomicAdd(C->fsum, s.fid);
        }
        if (!Multi && off < P.st_limit) s.capture(off);
        if (off < C->out_limit) {
          if (C->status) C->status[off] = (uint8_t)s.status;
          if (C->records)
#pragma unroll 1
            for (uint32_t w = 0; w < C->rw; ++w) C->records[off * C->rw + w] = s.rec[(size_t)w * 32 + lane];
        }
      }
      active = false;
    }
    // few active lanes: their shots go to the spill pool (when it has room), to resume in
    // the next round packed with others, and the warp moves on to fresh shots
    if (P.lane_evict) {
      const uint32_t am = __ballot_sync(0xFFFFFFFFu, active);
      if (am && (uint32_t)__popc(am) <= kEvictBelow && e + 1u < n_ev) {
        const uint32_t leader = __ffs(am) - 1;
        unsigned long long r0 = 0;
        if (lane == leader) r0 = atomicAdd(&P.lr[0], (unsigned long long)__popc(am));
        r0 = __shfl_sync(0xFFFFFFFFu, r0, leader);
        if (active) {
          const unsigned long long r = r0 + __popc(am & ((1u << lane) - 1u));
          if (r < P.sp_evict_cap) {
            s.evict(S, (uint32_t)r, item, e + 1u);
            active = false;
          }
        }
      }
    }
    uint32_t en = e + 1u > n_ev ? 0u : e + 1u;  // (within the circuit, cyclically)
    if (!__any_sync(0xFFFFFFFFu, active)) {
      // all lanes idle: the next bucket of any circuit (cyclically) that still has shots, or stop
      uint32_t found = 0xFFFFFFFFu;
      if (lane == 0) {
        const uint32_t g1 = (Multi ? C->bucket0 : 0u) + en;
        for (uint32_t k = 0; k < nb; ++k) {
          const uint32_t c = (g1 + k) % nb;
          if (*(volatile unsigned int *)&P.al_next[c] < __ldg(&P.al_start[c + 1]) - __ldg(&P.al_start[c])) {
            found = c;
            break;
          }
        }
      }
      found = __shfl_sync(0xFFFFFFFFu, found, 0);
      if (found == 0xFFFFFFFFu) break;
      if (Multi) {
        const uint32_t cn = circ_of_bucket(P, found);
        if (cn != ci) {
          flush();
          ci = cn;
          C = &P.circ[ci];
          n_ev = C->n_events;
          evs = reinterpret_cast<const Ev<W> *>(C->ev);
          s.C = C;
        }
        en = found - C->bucket0;
      } else {
        en = found;
      }
    }
    e = en;
  }
  flush();
}

}  // namespace

size_t lane_smem_bytes(int fp32, uint32_t W, uint32_t rw, bool wide) {
  size_t per;
  if (wide)
    per = W == 1 ? lane_warp_bytes<float, 1, kWideCap>(rw) : lane_warp_bytes<float, 2, kWideCap>(rw);
  else
    per = fp32 ? (W == 1 ? lane_warp_bytes<float, 1, kLaneCap>(rw) : lane_warp_bytes<float, 2, kLaneCap>(rw))
               : (W == 1 ? lane_warp_bytes<double, 1, kLaneCap>(rw) : lane_warp_bytes<double, 2, kLaneCap>(rw));
  return per * (kLaneBlock / 32);
}

uint32_t lane_map_cap() { return kLaneCap; }
uint32_t lane_rounds() { return kLaneRounds; }
uint32_t lane_max_buckets() { return kLaneMaxBuckets; }
uint32_t lane_prepass_grid() {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return (uint32_t)(sms > 0 ? sms : 1) * 8u;
}

size_t lane_spill_bytes(int fp32, uint32_t W, uint32_t rw, uint32_t cap) {
  return fp32 ? (W == 1 ? Spill<float, 1>::bytes(cap, rw) : Spill<float, 2>::bytes(cap, rw))
              : (W == 1 ? Spill<double, 1>::bytes(cap, rw) : Spill<double, 2>::bytes(cap, rw));
}

// the histogram of all buckets in shared memory (above 48 KB by the opt-in attribute)
template <bool Resume, typename R, int W>
static cudaError_t launch_bin(const ShotParams &p, cudaStream_t st) {
  const size_t sh = ((size_t)p.al_nb + 1) * sizeof(uint32_t);
  if (sh > 48 * 1024) {
    const cudaError_t e =
        cudaFuncSetAttribute(lane_bin_kernel<Resume, R, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
    if (e != cudaSuccess) return e;
  }
  lane_bin_kernel<Resume, R, W><<<p.al_grid, 256, sh, st>>>(p);
  lane_scan_kernel<<<1, 1024, 0, st>>>(p);
  lane_bin_scatter_kernel<Resume><<<p.al_grid, 256, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_lane_resume_prepass(const ShotParams &p, int fp32, uint32_t W, cudaStream_t st) {
  lane_round_setup_kernel<<<1, 1, 0, st>>>(p);
  if (fp32) return W == 1 ? launch_bin<true, float, 1>(p, st) : launch_bin<true, float, 2>(p, st);
  return W == 1 ? launch_bin<true, double, 1>(p, st) : launch_bin<true, double, 2>(p, st);
}

cudaError_t launch_lane_prepass(const ShotParams &p, cudaStream_t st) { return launch_bin<false, float, 1>(p, st); }

cudaError_t prepare_lanes(const ShotParams &p, int fp32, uint32_t W, int blocks_per_sm, LaunchCfg *cfg, bool wide) {
  const bool multi = p.n_circ > 1;
  constexpr uint32_t C1 = kLaneCap, C2 = kWideCap;
  const void *kern;
  if (wide) {  // FP32 single-circuit runs only
    if (!fp32 || multi) return cudaErrorInvalidConfiguration;
    kern = W == 1 ? reinterpret_cast<const void *>(lane_kernel<float, 1, false, C2>)
                  : reinterpret_cast<const void *>(lane_kernel<float, 2, false, C2>);
  } else
    kern = fp32 ? (W == 1 ? (multi ? reinterpret_cast<const void *>(lane_kernel<float, 1, true, C1>)
                                   : reinterpret_cast<const void *>(lane_kernel<float, 1, false, C1>))
                          : (multi ? reinterpret_cast<const void *>(lane_kernel<float, 2, true, C1>)
                                   : reinterpret_cast<const void *>(lane_kernel<float, 2, false, C1>)))
                : (W == 1 ? (multi ? reinterpret_cast<const void *>(lane_kernel<double, 1, true, C1>)
                                   : reinterpret_cast<const void *>(lane_kernel<double, 1, false, C1>))
                          : (multi ? reinterpret_cast<const void *>(lane_kernel<double, 2, true, C1>)
                                   : reinterpret_cast<const void *>(lane_kernel<double, 2, false, C1>)));
  const size_t smem = lane_smem_bytes(fp32, W, p.rw_max, wide);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kLaneBlock, smem)) != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  if (blocks_per_sm > 0 && blocks_per_sm < occ) occ = blocks_per_sm;
  cfg->kern = kern;
  cfg->grid = (unsigned)(occ * sms);
  cfg->block = kLaneBlock;
  cfg->smem = smem;
  return cudaSuccess;
}

}  // namespace soft
