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
// has its own range of buckets and a warp serves one circuit at a time. Circuits
// whose noiseless maps outgrow kLaneCap get lanes of 32 or (FP32) 64 entries, one
// launch per size over that size's buckets; the shots of circuits beyond those go
// straight to the warp pass.
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
// threads per block of a lane launch: 2 warps for 32-entry lanes (their shared memory per
// warp fits more warps per SM in small blocks: FP64 10 against 8, FP32 18 against 16; w42
// FP64 406.5 -> 421.0 M shots/s, FP32 713 -> 720 M through the wide round), 4 otherwise
template <uint32_t Cap>
__host__ __device__ constexpr int lane_block() { return Cap == 32u ? 64 : kLaneBlock; }
constexpr uint32_t kLaneMaxBuckets = 50000;  // the pre-pass histogram of all buckets: 200 KB of shared memory
#ifndef SOFT_LANE_EVICT
#define SOFT_LANE_EVICT 10
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
// First-pass lanes for circuits whose noiseless maps outgrow kLaneCap: 32 entries (kWideCap)
// or, with FP32 coefficients, 64 entries. These never evict or hand over: a shot whose map
// outgrows them runs again from its start in a warp.
constexpr uint32_t kLaneBigCap = 4 * kLaneCap;

// Lane map in affine form. The keys of a shot's coefficient map lie in an affine
// space alpha0 ^ span(B[0..d)) of dimension d <= kDim (Sec. II-C: the support of v
// grows by one direction per rotation whose beta is new, Theorem 1 (3), and shrinks
// with measurements and cancellations). Slot s (s < 2^d) holds the entry of key
//   key(s) = alpha0 ^ XOR over the set bits k of s of B[k],
// with its value in row s of the lane's value column, and `live` marks the slots that
// hold entries (values elsewhere are never read). Dual[k] (Dual[k] . B[j] = 1 iff
// k = j, over GF(2)) gives the coordinates of a vector x of the span: x = XOR over
// the k with Dual[k] . x = 1 of B[k]. So the partner key(s) ^ beta of a rotation is
// slot s ^ c (c: beta's coordinates), a parity gamma . key(s) is g0 ^ parity(s & gl)
// (g0 = gamma . alpha0, bit k of gl = gamma . B[k]), and a Pauli error moves alpha0
// only: per entry only values are read and written, and no key is stored. The live
// slots are the paper's sparse map: updates, pruning at tau and the overflow rule
// apply to them exactly as to a sparse map.
__host__ __device__ constexpr uint32_t lane_dim(uint32_t cap) { return cap <= 16u ? 4u : cap <= 32u ? 5u : 6u; }
// A set of slots: one bit per slot of the lane's cube (32 bits up to 32 slots, 64 for 64).
template <uint32_t Cap>
struct SlotSet {
  using T = uint32_t;
};
template <>
struct SlotSet<64> {
  using T = unsigned long long;
};
__device__ __forceinline__ uint32_t mffs(uint32_t m) { return (uint32_t)__ffs(m); }
__device__ __forceinline__ uint32_t mffs(unsigned long long m) { return (uint32_t)__ffsll((long long)m); }
__device__ __forceinline__ uint32_t mpopc(uint32_t m) { return (uint32_t)__popc(m); }
__device__ __forceinline__ uint32_t mpopc(unsigned long long m) { return (uint32_t)__popcll(m); }

template <typename R, int W, uint32_t Cap>
__host__ __device__ inline size_t lane_warp_bytes(uint32_t rw) {
  // values of Cap slots; alpha0, kDim basis and kDim dual vectors (W words each); record words
  return (size_t)Cap * sizeof(Cx<R>) * 32 + (size_t)(1 + 2 * lane_dim(Cap)) * W * 8 * 32 + (size_t)rw * 8 * 32;
}

// Slot masks over a cube of up to 32 (M = uint32_t) or 64 slots: the slots whose index has
// bit k set.
template <typename M>
__device__ __forceinline__ M slot_bit_mask(uint32_t k) {
  if (sizeof(M) == 4)
    return (M)(k == 0u ? 0xAAAAAAAAu : k == 1u ? 0xCCCCCCCCu : k == 2u ? 0xF0F0F0F0u : k == 3u ? 0xFF00FF00u : 0xFFFF0000u);
  return (M)(k == 0u   ? 0xAAAAAAAAAAAAAAAAull
             : k == 1u ? 0xCCCCCCCCCCCCCCCCull
             : k == 2u ? 0xF0F0F0F0F0F0F0F0ull
             : k == 3u ? 0xFF00FF00FF00FF00ull
             : k == 4u ? 0xFFFF0000FFFF0000ull
                       : 0xFFFFFFFF00000000ull);
}
// The slots s with parity(s & g) = 1.
template <typename M>
__device__ __forceinline__ M slot_par_mask(uint32_t g) {
  M m = 0;
#pragma unroll
  for (uint32_t k = 0; k < (sizeof(M) == 4 ? 5u : 6u); ++k)
    if ((g >> k) & 1u) m ^= slot_bit_mask<M>(k);
  return m;
}
// A slot set moved by s -> s ^ c.
template <typename M>
__device__ __forceinline__ M slot_xor_perm(M L, uint32_t c) {
#pragma unroll
  for (uint32_t k = 0; k < (sizeof(M) == 4 ? 5u : 6u); ++k)
    if ((c >> k) & 1u) {
      const M B = slot_bit_mask<M>(k);
      const uint32_t sh = 1u << k;
      L = ((L & B) >> sh) | ((L & ~B) << sh);
    }
  return L;
}
__device__ __forceinline__ uint32_t spar(uint32_t s, uint32_t g) { return (uint32_t)__popc(s & g) & 1u; }
template <int W>
__device__ __forceinline__ bool wnonzero(const uint64_t *x) {
  uint64_t o = 0;
#pragma unroll
  for (int w = 0; w < W; ++w) o |= x[w];
  return o != 0ull;
}
// The lowest set bit of a nonzero W-word vector.
template <int W>
__device__ __forceinline__ uint32_t wlow(const uint64_t *x) {
  return x[0] ? (uint32_t)(__ffsll((long long)x[0]) - 1) : 64u + (uint32_t)(__ffsll((long long)x[W - 1]) - 1);
}

template <typename R, int W, uint32_t Cap>
struct LaneShot {
  static constexpr uint32_t kDim = lane_dim(Cap);
  static_assert(Cap == (1u << kDim), "a lane holds a cube of slots");
  static constexpr uint32_t kRowB = 1, kRowD = 1 + kDim;  // rows: alpha0, B[0..kDim), Dual[0..kDim)
  using Mask = typename SlotSet<Cap>::T;  // a set of the cube's slots
  const ShotParams &P;
  const CircDev *C;
  uint32_t lane;
  Cx<R> *vals;     // [slot][lane]
  uint64_t *rows;  // [row][w][lane]
  uint64_t *rec;   // [w][lane]
  // per-lane shot state
  uint64_t shot;
  uint32_t d;
  Mask live;
  uint64_t sd[W], ss[W];
  uint32_t nxt, cur, kblk, w2;
  int status, chain, logical, lastm;
  double fid;
  bool force;

  PruneTest<R> pt;  // |v|^2 < tau

  __device__ LaneShot(const ShotParams &p, unsigned char *base) : P(p), C(&p.circ[0]), pt(p.tau) {
    lane = threadIdx.x & 31u;
    const size_t vb = (size_t)Cap * sizeof(Cx<R>) * 32, rb = (size_t)(1 + 2 * kDim) * W * 8 * 32;
    vals = reinterpret_cast<Cx<R> *>(base);
    rows = reinterpret_cast<uint64_t *>(base + vb);
    rec = reinterpret_cast<uint64_t *>(base + vb + rb);
  }

  __device__ __forceinline__ Cx<R> val(uint32_t s) const { return vals[(size_t)s * 32 + lane]; }
  __device__ __forceinline__ void set_val(uint32_t s, Cx<R> v) { vals[(size_t)s * 32 + lane] = v; }
  __device__ __forceinline__ uint64_t row(uint32_t r, int w) const { return rows[((size_t)r * W + w) * 32 + lane]; }
  __device__ __forceinline__ void set_row(uint32_t r, int w, uint64_t x) { rows[((size_t)r * W + w) * 32 + lane] = x; }
  __device__ __forceinline__ void get_row(uint32_t r, uint64_t *x) const {
#pragma unroll
    for (int w = 0; w < W; ++w) x[w] = row(r, w);
  }
  __device__ __forceinline__ void put_row(uint32_t r, const uint64_t *x) {
#pragma unroll
    for (int w = 0; w < W; ++w) set_row(r, w, x[w]);
  }
  __device__ __forceinline__ void xor_row(uint32_t r, const uint64_t *x) {
#pragma unroll
    for (int w = 0; w < W; ++w) set_row(r, w, row(r, w) ^ x[w]);
  }
  __device__ __forceinline__ uint32_t row_par(uint32_t r, const uint64_t *g) const {
    uint32_t t = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) t += __popcll(row(r, w) & g[w]);
    return t & 1u;
  }
  __device__ __forceinline__ uint32_t row_bit(uint32_t r, uint32_t p) const {
    return (uint32_t)((row(r, (W == 2 && p >= 64u) ? W - 1 : 0) >> (p & 63u)) & 1ull);
  }
  __device__ __forceinline__ Mask cube() const {
    if (sizeof(Mask) == 4) return (Mask)(d >= 5u ? 0xFFFFFFFFu : (1u << (1u << d)) - 1u);
    return (Mask)(d >= 6u ? ~0ull : (1ull << (1u << d)) - 1ull);
  }
  __device__ __forceinline__ uint32_t nnz() const { return mpopc(live); }

  // g . alpha0 into g0; bit k of the result: g . B[k]
  __device__ uint32_t parities(const uint64_t *g, uint32_t &g0) const {
    g0 = row_par(0, g);
    uint32_t m = 0;
#pragma unroll 1
    for (uint32_t k = 0; k < d; ++k) m |= row_par(kRowB + k, g) << k;
    return m;
  }
  // coordinates c of x (bit k: Dual[k] . x) and the residual r = x ^ XOR_{k in c} B[k],
  // zero iff x lies in the span (otherwise Dual[k] . r = 0 for every k)
  __device__ uint32_t coords(const uint64_t *x, uint64_t *r) const {
    uint32_t c = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) r[w] = x[w];
#pragma unroll 1
    for (uint32_t k = 0; k < d; ++k)
      if (row_par(kRowD + k, x)) {
        c |= 1u << k;
#pragma unroll
        for (int w = 0; w < W; ++w) r[w] ^= row(kRowB + k, w);
      }
    return c;
  }
  // B[d] = r (nonzero, Dual[k] . r = 0 for k < d); its dual e_p ^ XOR_k B[k][p] Dual[k] for
  // the lowest set bit p of r is orthogonal to every B[k] and has Dual . r = 1, and the
  // old duals stay dual (Dual[k] . r = 0)
  __device__ void add_dim(const uint64_t *r) {
    const uint32_t p = wlow<W>(r);
    uint64_t z[W];
#pragma unroll
    for (int w = 0; w < W; ++w) z[w] = ((int)(p >> 6) == w) ? (1ull << (p & 63u)) : 0ull;
#pragma unroll 1
    for (uint32_t k = 0; k < d; ++k)
      if (row_bit(kRowB + k, p)) {
#pragma unroll
        for (int w = 0; w < W; ++w) z[w] ^= row(kRowD + k, w);
      }
    put_row(kRowB + d, r);
    put_row(kRowD + d, z);
    ++d;
  }
  // The duals of the current basis, built one vector at a time (the same construction as
  // add_dim, on each vector's residual against the ones before it).
  __device__ void rebuild_duals() {
#pragma unroll 1
    for (uint32_t k = 0; k < d; ++k) {
      uint64_t r[W];
      get_row(kRowB + k, r);
      uint32_t cm = 0;  // Dual[j] . B[k] for j < k
#pragma unroll 1
      for (uint32_t j = 0; j < k; ++j)
        if (row_par(kRowD + j, r)) cm |= 1u << j;
#pragma unroll 1
      for (uint32_t j = 0; j < k; ++j)
        if ((cm >> j) & 1u) {
#pragma unroll
          for (int w = 0; w < W; ++w) r[w] ^= row(kRowB + j, w);
        }
      const uint32_t p = wlow<W>(r);
      uint64_t z[W];
#pragma unroll
      for (int w = 0; w < W; ++w) z[w] = ((int)(p >> 6) == w) ? (1ull << (p & 63u)) : 0ull;
#pragma unroll 1
      for (uint32_t j = 0; j < k; ++j)
        if (row_bit(kRowB + j, p)) {
#pragma unroll
          for (int w = 0; w < W; ++w) z[w] ^= row(kRowD + j, w);
        }
#pragma unroll 1
      for (uint32_t j = 0; j < k; ++j)
        if ((cm >> j) & 1u) xor_row(kRowD + j, z);
      put_row(kRowD + k, z);
    }
  }
  // Every live slot s has parity(s & g) = t, and g has bit q set (q < d): bit q of a live
  // slot follows from the others, so the map needs one coordinate less. alpha0 ^= t B[q],
  // B[k] ^= B[q] for the other k of g; B[q] and Dual[q] go (the other duals stay dual);
  // each live slot drops bit q of its index.
  __device__ void remove_dim(uint32_t q, uint32_t g, uint32_t t) {
    remove_rows(q, g, t);
    const uint32_t lo = (1u << q) - 1u;
    Mask nl = 0;
#pragma unroll 1
    for (Mask m = live; m; m &= m - (Mask)1) {  // ascending: a slot moves down onto a vacated one
      const uint32_t s = mffs(m) - 1, s2 = (s & lo) | ((s >> (q + 1u)) << q);
      if (s2 != s) set_val(s2, val(s));
      nl |= (Mask)1 << s2;
    }
    live = nl;
  }
  // the rows' part of remove_dim (d decreases); the caller moves the slots
  __device__ void remove_rows(uint32_t q, uint32_t g, uint32_t t) {
    uint64_t bq[W];
    get_row(kRowB + q, bq);
    if (t) xor_row(0, bq);
#pragma unroll 1
    for (uint32_t k = 0; k < d; ++k)
      if (k != q && ((g >> k) & 1u)) xor_row(kRowB + k, bq);
#pragma unroll 1
    for (uint32_t k = q; k + 1u < d; ++k) {
      uint64_t x[W];
      get_row(kRowB + k + 1u, x);
      put_row(kRowB + k, x);
      get_row(kRowD + k + 1u, x);
      put_row(kRowD + k, x);
    }
    --d;
  }
  // after a measurement: all live slots share parity(s & g); drop a coordinate if g != 0
  __device__ __forceinline__ void restrict_to(uint32_t g) {
    g &= (d >= 32u) ? 0xFFFFFFFFu : ((1u << d) - 1u);
    if (!g || !live) return;
    const uint32_t t = spar(mffs(live) - 1, g);
    remove_dim(31u - __clz(g), g, t);
  }
  // drop the coordinates no live slot uses
  __device__ void compact_dead(uint32_t &gl) {
#pragma unroll 1
    for (uint32_t k = d; k-- > 0;)
      if (!(live & slot_bit_mask<Mask>(k))) {
        remove_dim(k, 1u << k, 0);
        gl = (gl & ((1u << k) - 1u)) | ((gl >> (k + 1u)) << k);  // the parities follow the coordinates
      }
  }
  // key of slot s
  __device__ Key<W> key_of(uint32_t s) const {
    Key<W> k;
#pragma unroll
    for (int w = 0; w < W; ++w) k.w[w] = row(0, w);
#pragma unroll 1
    for (uint32_t j = 0; j < d; ++j)
      if ((s >> j) & 1u) {
#pragma unroll
        for (int w = 0; w < W; ++w) k.w[w] ^= row(kRowB + j, w);
      }
    return k;
  }
  // The map from explicit entries (a spill record): alpha0 = the first key, each further
  // key's residual a new direction. False if it needs more than kDim directions.
  template <typename KeyAt, typename ValAt>
  __device__ bool load_entries(uint32_t n, KeyAt key_at, ValAt val_at) {
    d = 0;
    live = 0;
    if (n == 0) {
#pragma unroll
      for (int w = 0; w < W; ++w) set_row(0, w, 0ull);
      return true;
    }
    const Key<W> k0 = key_at(0);
    put_row(0, k0.w);
#pragma unroll 1
    for (uint32_t i = 0; i < n; ++i) {
      const Key<W> k = key_at(i);
      const Key<W> x = kxor(k, k0.w);
      uint64_t r[W];
      uint32_t c = coords(x.w, r);
      if (wnonzero<W>(r)) {
        if (d == kDim) return false;
        add_dim(r);
        c |= 1u << (d - 1u);
      }
      set_val(c, val_at(i));
      live |= (Mask)1 << c;
    }
    return true;
  }

  __device__ void fail_capacity() { status = P.small_pass ? LS_RERUN : LS_OVF; }
  __device__ void fail_check(uint32_t code, uint64_t value) {
    status = LS_ERR;
    if (P.diag && atomicAdd(&P.diag[0], 1ull) == 0ull) {
      P.diag[1] = ((unsigned long long)code << 32);
      P.diag[2] = shot;
      P.diag[3] = value;
    }
  }

  __device__ double uniform(uint32_t ord) const {
    uint4 w = philox<true>(P.seed, shot, 1u, ord);
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

  // ---- start: shot s at event e of the noiseless run (its map in affine form, computed
  // once per snapshot when the circuit was compiled); the pre-pass drew the shot's first
  // error: its noise cursor comes with the item
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
    const SnapAffine<R, W> *a = reinterpret_cast<const SnapAffine<R, W> *>(in + snap_affine_off<R, W>(C->rw));
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
    const uint2 dl = __ldg(reinterpret_cast<const uint2 *>(&a->d));  // d and the low word of live
    d = 0;
    live = 0;
    if (dl.x > kDim) {
      fail_capacity();
      return;
    }
    d = dl.x;
    live = (Mask)dl.y;  // (no slot at or above 2^kDim is live)
    if (sizeof(Mask) == 8) live |= (Mask)__ldg(&a->live_hi) << 16 << 16;
#pragma unroll
    for (int w = 0; w < W; ++w) set_row(0, w, __ldg(&a->rows[0][w]));
#pragma unroll 1
    for (uint32_t k = 0; k < d; ++k)
#pragma unroll
      for (int w = 0; w < W; ++w) {
        set_row(kRowB + k, w, __ldg(&a->rows[1 + k][w]));
        set_row(kRowD + k, w, __ldg(&a->rows[1 + kSnapDim + k][w]));
      }
#pragma unroll 1
    for (Mask m = live; m; m &= m - (Mask)1) {
      const uint32_t j = mffs(m) - 1;
      set_val(j, a->v[j]);
    }
  }

  // ---- eviction: the shot's whole state into record r, to resume at event ev (entries
  // in slot order, at most kLaneCap of them: a first-round lane holds no more)
  __device__ void evict(const Spill<R, W> &S, uint32_t r, uint32_t item, uint32_t ev) const {
    const size_t c = S.cap;
    S.ha[r] = make_uint4(item, ev, nnz(), (uint32_t)(chain & 1) | ((uint32_t)(logical & 1) << 1) |
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
    uint32_t i = 0;
#pragma unroll 1
    for (Mask m = live; m && i < kLaneCap; m &= m - (Mask)1, ++i) {
      const uint32_t s = mffs(m) - 1;
      const Key<W> k = key_of(s);
#pragma unroll
      for (int w = 0; w < W; ++w) S.keys[((size_t)i * W + w) * c + r] = k.w[w];
      S.vals[(size_t)i * c + r] = val(s);
    }
  }
  // ---- resumption from record r; returns the shot's item (chunk-local index)
  __device__ uint32_t resume(const Spill<R, W> &S, uint32_t r, uint64_t first) {
    const size_t c = S.cap;
    const uint4 a = S.ha[r], b = S.hb[r];
    shot = first + a.x;
    status = LS_RUN;
    force = false;
    const uint32_t n = a.z;
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
    d = 0;
    live = 0;
    if (n > kLaneCap) {  // a record never holds more; checked so that a bad record cannot index past the map
      fail_check(CHK_NNZ, n);
      return a.x;
    }
    const bool ok = load_entries(
        n,
        [&](uint32_t i) {
          Key<W> k;
#pragma unroll
          for (int w = 0; w < W; ++w) k.w[w] = S.keys[((size_t)i * W + w) * c + r];
          return k;
        },
        [&](uint32_t i) { return S.vals[(size_t)i * c + r]; });
    if (!ok) fail_capacity();  // (records come from lanes of at most kDim directions)
    return a.x;
  }
  // ---- the shot's final state (signs, keys, values) for state capture at offset off
  __device__ void capture(uint64_t off) const {
    P.st_nnz[off] = nnz();
    P.st_signs[off * 4 + 0] = sd[0];
    P.st_signs[off * 4 + 1] = (W == 2) ? sd[W - 1] : 0ull;
    P.st_signs[off * 4 + 2] = ss[0];
    P.st_signs[off * 4 + 3] = (W == 2) ? ss[W - 1] : 0ull;
    uint32_t i = 0;
#pragma unroll 1
    for (Mask m = live; m && i < P.st_stride; m &= m - (Mask)1, ++i) {
      const uint32_t s = mffs(m) - 1;
      const Key<W> k = key_of(s);
      const Cx<R> v = val(s);
      const size_t o = (size_t)off * P.st_stride + i;
      P.st_keys[2 * o] = k.w[0];
      P.st_keys[2 * o + 1] = (W == 2) ? k.w[W - 1] : 0ull;
      P.st_vals[2 * o] = (double)v.x;
      P.st_vals[2 * o + 1] = (double)v.y;
    }
  }

  // ---- Paulis: v'_{a^beta} = i^{e + 2 gamma.a} v_a: phases per entry, then alpha0 moves
  __device__ void apply_pauli(const uint64_t *beta, const uint64_t *gamma, uint32_t e) {
    uint32_t g0;
    const uint32_t gl = parities(gamma, g0);
#pragma unroll 1
    for (Mask m = live; m; m &= m - (Mask)1) {
      const uint32_t s = mffs(m) - 1;
      set_val(s, ipow(val(s), e + 2u * (g0 ^ spar(s, gl))));
    }
    xor_row(0, beta);
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

  // ---- a I + b Z_q: v'_a = a v_a + b xi_{a^beta} v_{a^beta}; xi = i^e (-1)^{gamma.key}
  // folded into b (b or -b per entry, exact), and a diagonal rotation (beta = 0) is one
  // product (a + b xi) v per entry. gl, g0: gamma's parities with the basis and alpha0 on
  // entry (they follow the basis through the changes made here).
  __device__ void rot(uint32_t w0, uint32_t ci, const uint64_t *beta, const uint64_t *gamma, bool diag, uint32_t gl,
                      const uint32_t g0) {
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
    const Cx<R> bq = ipow(b, e), bn = Cx<R>{negr(bq.x), negr(bq.y)};
    Mask drop = 0;
    if (diag) {
      const Cx<R> c0 = cadd(a, bq), c1 = cadd(a, bn);
#pragma unroll 1
      for (Mask m = live; m; m &= m - (Mask)1) {
        const uint32_t s = mffs(m) - 1;
        const Cx<R> nv = cmul((g0 ^ spar(s, gl)) ? c1 : c0, val(s));
        const bool sm = pt.small(nv);
        if (!sm) set_val(s, nv);
        drop |= (Mask)sm << s;
      }
      live &= ~drop;
      return;
    }
    uint64_t r[W];
    uint32_t c;
    bool fresh;
#pragma unroll 1
    for (uint32_t pass = 0;; ++pass) {
      c = coords(beta, r);
      fresh = wnonzero<W>(r);  // beta outside the span: every entry gains a partner
      if (!fresh || d < kDim) break;
      if (pass) {
        // the map would outgrow the lane: nothing has been written yet, so the shot can be
        // taken over at the top of this event (by the wide round's lanes, or a warp);
        // otherwise (the wide round) it reruns in a warp
        if (P.lane_hand && P.sp && P.small_pass && C->cap > Cap) status = LS_HAND;
        else fail_capacity();
        return;
      }
      compact_dead(gl);
    }
    if (fresh) {
      add_dim(r);
      c |= 1u << (d - 1u);
      gl |= row_par(kRowB + d - 1u, gamma) << (d - 1u);
    }
    const Mask spread = live | slot_xor_perm<Mask>(live, c);
    const Mask lead = spread & ~slot_bit_mask<Mask>(__ffs(c) - 1) & cube();  // one member of each pair
#pragma unroll 1
    for (Mask m = lead; m; m &= m - (Mask)1) {
      const uint32_t s = mffs(m) - 1, t = s ^ c;
      const uint32_t ls = (uint32_t)(live >> s) & 1u, lt = (uint32_t)(live >> t) & 1u;
      const Cx<R> vs = ls ? val(s) : Cx<R>{0, 0}, vt = lt ? val(t) : Cx<R>{0, 0};
      const Cx<R> bs = (g0 ^ spar(s, gl)) ? bn : bq, bt = (g0 ^ spar(t, gl)) ? bn : bq;
      Cx<R> ns, nt;
      if (ls && lt) {  // one fused chain per component
        ns = cmad2(a, vs, bt, vt);
        nt = cmad2(a, vt, bs, vs);
      } else if (ls) {  // an entry without a partner gains one
        ns = cmul(a, vs);
        nt = cmul(bs, vs);
      } else {
        ns = cmul(bt, vt);
        nt = cmul(a, vt);
      }
      const bool ss_ = pt.small(ns), st_ = pt.small(nt);
      if (!ss_) set_val(s, ns);
      if (!st_) set_val(t, nt);
      drop |= ((Mask)ss_ << s) | ((Mask)st_ << t);
    }
    live = spread & ~drop;
    if (nnz() > C->cap) status = LS_OVF;  // the overflow rule, for circuits whose cap is below the lane's
  }

  // ---- measurement of P, beta = 0: lambda_a = c (-1)^{gamma.a}; gl, g0: gamma's parities
  // with the basis and alpha0
  __device__ int meas_a(uint32_t w0, uint32_t ord, const uint64_t *gamma, const uint32_t gl, const uint32_t g0) {
    uint32_t pe = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) pe += __popcll(ss[w] & gamma[w]);
    const uint32_t e = (ev_e0(w0) + 2u * pe) & 3u;
    if (e & 1u) {
      fail_check(CHK_PHASE, e);
      return 1;
    }
    const uint32_t sgn = e >> 1;
    const Mask pm = slot_par_mask<Mask>(gl) & cube();
    const Mask neg = live & (((sgn ^ g0) & 1u) ? ~pm : pm);  // slots with eigenvalue -1
    const Mask pos = live & ~neg;
    int m;
    R sc = (R)1;
    Mask keep;
    if (!neg || !pos) {  // decided (all eigenvalues equal): integer test only, no scaling
      m = neg ? -1 : 1;
      keep = live;
      if (!gl || !live) return m;
    } else {
      double sp = 0.0, sm = 0.0;
#pragma unroll 1
      for (Mask mm = live; mm; mm &= mm - (Mask)1) {
        const uint32_t s = mffs(mm) - 1;
        const double a2 = pnorm(val(s));
        if ((neg >> s) & 1u) sm += a2;
        else sp += a2;
      }
      m = pick(ord, sp, sm);
      sc = inv_sqrt(m == 1 ? sp : sm);
      keep = (m == 1) ? pos : neg;
    }
    // the kept slots share parity(s & gl) = t, so bit q of their index is redundant; each is
    // scaled straight into its slot of the restricted map. A decided outcome goes through
    // the same loop with the scale 1 (exact; no kept value is below tau), so that the
    // restriction is inlined once (w42 FP32: 676 -> 708 M shots/s)
    const uint32_t q = 31u - __clz(gl), lo = (1u << q) - 1u, t = spar(mffs(keep) - 1, gl);
    Mask nl = 0;
#pragma unroll 1
    for (Mask mm = keep; mm; mm &= mm - (Mask)1) {  // ascending: a write lands on a slot already read
      const uint32_t s = mffs(mm) - 1, s2 = (s & lo) | ((s >> (q + 1u)) << q);
      const Cx<R> v = cscale(val(s), sc);
      if (!pt.small(v)) {
        set_val(s2, v);
        nl |= (Mask)1 << s2;
      }
    }
    if (nl) remove_rows(q, gl, t);
    live = nl;
    return m;
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
    // relabel a_j ^= a_p (j in J), a linear map L of the keys: alpha0 and every B[k] go
    // through it, and the duals through its transpose (D ^= (D . J) e_p; L is its own inverse)
#pragma unroll 1
    for (uint32_t k = 0; k <= d; ++k) {
      const uint32_t rr = k == 0 ? 0u : kRowB + k - 1u;
      if (row_bit(rr, p)) xor_row(rr, J);
    }
#pragma unroll 1
    for (uint32_t k = 0; k < d; ++k)
      if (row_par(kRowD + k, J)) xor_row(kRowD + k, ep);
    // pair a0 (key bit p clear) with a1 = a0 ^ e_p: first the outcome probabilities, then
    // the combined values (v0 + m x1) / sqrt(2 p_m), x1 = xi_{a1} v_{a1}
    uint32_t g20;
    const uint32_t gl2 = parities(g2, g20);
    uint32_t bp = 0;  // bit k: B[k][p]
#pragma unroll 1
    for (uint32_t k = 0; k < d; ++k) bp |= row_bit(kRowB + k, p) << k;
    const Mask cb = cube();
    const Mask kb = (row_bit(0, p) ? ~slot_par_mask<Mask>(bp) : slot_par_mask<Mask>(bp)) & cb;  // slots whose key has bit p
    uint64_t rr[W];
    const uint32_t c = coords(ep, rr);
    const bool lone = wnonzero<W>(rr);  // e_p outside the span: no entry has a partner
    const Mask spread = lone ? live : (live | slot_xor_perm<Mask>(live, c));
    const Mask lead = lone ? live : (spread & ~kb);  // a0 members (lone: every entry)
    double sp = 0.0, sm = 0.0;
#pragma unroll 1
    for (Mask m = lead; m; m &= m - (Mask)1) {
      const uint32_t s = mffs(m) - 1;
      Cx<R> v0{0, 0}, x1{0, 0};
      if (lone) {
        if ((kb >> s) & 1u) x1 = ipow(val(s), e2 + 2u * (g20 ^ spar(s, gl2)));
        else v0 = val(s);
      } else {
        const uint32_t t = s ^ c;
        if ((live >> s) & 1u) v0 = val(s);
        if ((live >> t) & 1u) x1 = ipow(val(t), e2 + 2u * (g20 ^ spar(t, gl2)));
      }
      sp += 0.5 * pnorm(cadd(v0, x1));
      sm += 0.5 * pnorm(csub(v0, x1));
    }
    const int m = pick(ord, sp, sm);
    const R sc = inv_sqrt(2.0 * (m == 1 ? sp : sm));
    Mask nl = 0;
#pragma unroll 1
    for (Mask mm = lead; mm; mm &= mm - (Mask)1) {
      const uint32_t s = mffs(mm) - 1;
      Cx<R> v0{0, 0}, x1{0, 0};
      if (lone) {
        if ((kb >> s) & 1u) x1 = ipow(val(s), e2 + 2u * (g20 ^ spar(s, gl2)));
        else v0 = val(s);
      } else {
        const uint32_t t = s ^ c;
        if ((live >> s) & 1u) v0 = val(s);
        if ((live >> t) & 1u) x1 = ipow(val(t), e2 + 2u * (g20 ^ spar(t, gl2)));
      }
      const Cx<R> nv = cscale(m == 1 ? cadd(v0, x1) : csub(v0, x1), sc);
      if (!pt.small(nv)) {
        set_val(s, nv);
        nl |= (Mask)1 << s;
      }
    }
    live = nl;
    if (lone) {
      // every key loses bit p (a1 keys become a1 ^ e_p); injective on the space since e_p is
      // not in the span, so the slots stay, and the basis is rebuilt with new duals
#pragma unroll 1
      for (uint32_t k = 0; k <= d; ++k) {
        const uint32_t r2 = k == 0 ? 0u : kRowB + k - 1u;
        if (row_bit(r2, p)) xor_row(r2, ep);
      }
      rebuild_duals();
    } else {
      restrict_to(bp);  // the kept keys have bit p clear: parity(s & bp) = alpha0[p]
    }
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
      if (!next_site<true>(C, P.seed, shot, cur, kblk, nxt, w2)) status = LS_ERR;
    }
    if (status != LS_RUN) return;
    const uint64_t *dsd = body, *dss = body + W, *beta = body + 2 * W, *gamma = body + 3 * W;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      sd[w] ^= dsd[w];
      ss[w] ^= dss[w];
    }
    const uint32_t w0 = hdr.x, type = ev_type(w0), flags = ev_flags(w0);
    // gamma's parities with alpha0 and the basis, once for the event types that use them.
    // This kernel is bound by instruction fetch, so each helper is inlined at as few sites as
    // possible: one parity computation here instead of one per handler, one rotation handler
    // for both kinds, and the handlers in a chain of tests in order of frequency (a `break`
    // leaves the chain) rather than a jump table (w42: FP32 660 -> 675 M shots/s, FP64
    // 352 -> 382 M).
    uint32_t g0 = 0, gl = 0;
    if (type == EV_ROT || type == EV_ROT_DIAG || type == EV_MEAS_A) gl = parities(gamma, g0);
    do {
      if (type == EV_MEAS_A || type == EV_MEAS_B) {
        force = P.fid_mode && (flags & F_FIDELITY);
        const int m = (type == EV_MEAS_A) ? meas_a(w0, hdr.z, gamma, gl, g0) : meas_b(hdr.z, (uint32_t)beta[0]);
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
      if (type == EV_ROT || type == EV_ROT_DIAG) {
        rot(w0, hdr.z, beta, gamma, type == EV_ROT_DIAG, gl, g0);
        break;
      }
      if (type == EV_PAULI) {
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
      if (type == EV_PARITY) {
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
    } while (false);
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

// ---- the affine form (SnapAffine) of every valid snapshot of a noiseless run (events
// [0, stop[0]]), one thread per snapshot, once per compiled circuit and precision; the
// largest dimension goes to stop[3] (0xFF where a map needs more than kSnapDim)
template <typename R, int W>
__global__ void snap_affine_kernel(unsigned char *traj, uint32_t n_snap, uint32_t stride, uint32_t rw,
                                   uint32_t *stop) {
  const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_snap || e > stop[0]) return;
  unsigned char *in = traj + (size_t)e * stride;
  const SnapHdr *h = reinterpret_cast<const SnapHdr *>(in);
  const uint64_t *k_in = reinterpret_cast<const uint64_t *>(in + sizeof(SnapHdr)) + rw;
  const Cx<R> *v_in = reinterpret_cast<const Cx<R> *>(k_in + kSnapMax * W);
  SnapAffine<R, W> *out = reinterpret_cast<SnapAffine<R, W> *>(in + snap_affine_off<R, W>(rw));
  const uint32_t n = h->nnz < kSnapMax ? h->nnz : kSnapMax;
  constexpr uint32_t kB = 1, kD = 1 + kSnapDim;
  uint64_t rw_[1 + 2 * kSnapDim][W];
  for (uint32_t r = 0; r < 1 + 2 * kSnapDim; ++r)
    for (int w = 0; w < W; ++w) rw_[r][w] = 0ull;
  for (uint32_t j = 0; j < (1u << kSnapDim); ++j) out->v[j] = Cx<R>{0, 0};
  uint32_t d = 0;
  unsigned long long live = 0;
  bool ok = true;
  if (n) {
    for (int w = 0; w < W; ++w) rw_[0][w] = k_in[w];
  }
  for (uint32_t i = 0; i < n && ok; ++i) {
    uint64_t x[W], r[W];
    for (int w = 0; w < W; ++w) r[w] = x[w] = k_in[i * W + w] ^ rw_[0][w];
    uint32_t c = 0;
    for (uint32_t k = 0; k < d; ++k)
      if (wpar<W>(rw_[kD + k], x)) {
        c |= 1u << k;
        for (int w = 0; w < W; ++w) r[w] ^= rw_[kB + k][w];
      }
    if (wnonzero<W>(r)) {
      if (d == kSnapDim) {
        ok = false;
        break;
      }
      const uint32_t p = wlow<W>(r);  // the new direction's dual (as in LaneShot::add_dim)
      uint64_t z[W];
      for (int w = 0; w < W; ++w) z[w] = ((int)(p >> 6) == w) ? (1ull << (p & 63u)) : 0ull;
      for (uint32_t k = 0; k < d; ++k)
        if (wbit<W>(rw_[kB + k], p))
          for (int w = 0; w < W; ++w) z[w] ^= rw_[kD + k][w];
      for (int w = 0; w < W; ++w) {
        rw_[kB + d][w] = r[w];
        rw_[kD + d][w] = z[w];
      }
      c |= 1u << d;
      ++d;
    }
    out->v[c] = v_in[i];
    live |= 1ull << c;
  }
  for (uint32_t r = 0; r < 1 + 2 * kSnapDim; ++r)
    for (int w = 0; w < W; ++w) out->rows[r][w] = rw_[r][w];
  out->d = ok ? d : 0xFFFFFFFFu;
  out->live_lo = (uint32_t)live;
  out->live_hi = (uint32_t)(live >> 32);
  atomicMax(&stop[3], ok ? d : 0xFFu);
}

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

// Register budget: resident blocks per SM the compiler must allow. FP32 16-slot lanes: 8
// (64 registers; the shared memory allows 8 on w42; measured 617 M shots/s against 604 M
// at 6 blocks and 76 registers); 32-slot lanes (blocks of 2 warps): 8 in FP32, 4 in FP64,
// which leave the registers they use (shared memory allows 9 and 5); 64-slot lanes: 2;
// FP64 16-slot lanes: 5 (its shared memory allows 5; 272.8 M against 266.7 M at 4).
template <typename R, uint32_t Cap>
constexpr int kLaneMinBlocks() {
  return sizeof(R) == 4 ? (Cap <= 16 ? 8 : Cap <= 32 ? 8 : 2) : (Cap == 32 ? 4 : 5);
}

// Multi: the run holds several circuits (a warp serves one at a time); the single-
// circuit instantiation keeps circuit 0 and bucket offset 0 as constants. Cap: map
// entries per lane (kLaneCap in the first rounds, kWideCap in the wide round, or
// kWideCap / kLaneBigCap as the first pass of circuits with larger noiseless maps).
template <typename R, int W, bool Multi, uint32_t Cap>
__global__ void __launch_bounds__(lane_block<Cap>(), kLaneMinBlocks<R, Cap>()) lane_kernel(const __grid_constant__ ShotParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  // per warp: tallies of its current circuit, added to the circuit's when the warp moves
  // to another circuit and at the end
  __shared__ unsigned long long wt[lane_block<Cap>() / 32][5];
  const uint32_t warp = threadIdx.x / 32, lane = threadIdx.x & 31u;
  if (lane < 5) wt[warp][lane] = 0ull;
  __syncwarp();
  LaneShot<R, W, Cap> s(P, smem + (size_t)warp * lane_warp_bytes<R, W, Cap>(P.rw_max));
  const unsigned long long base = P.item_base_dev ? *P.item_base_dev : P.item_base;
  const unsigned long long n_items =
      P.lane_round ? P.lr[3 + 2 * P.lane_round] : (P.n_items_dev ? *P.n_items_dev : P.n_items);
  const unsigned long long rec0 = P.lane_round ? P.lr[2 + 2 * P.lane_round] : 0ull;
  const Spill<R, W> S(P.sp, P.sp_cap, P.rw_max);
  // a batch's launch serves the buckets [P.al_lo, P.al_hi) of its lane map size's circuits
  // (read from the launch parameters where used, so that no register holds them through the
  // loop); a single circuit's, all of them
  if (Multi && P.al_hi <= P.al_lo) return;
  // warps start spread evenly over the buckets, so that they meet buckets that still hold shots
  const unsigned long long gw = (unsigned long long)blockIdx.x * (blockDim.x / 32) + warp;
  const unsigned long long nw = (unsigned long long)gridDim.x * (blockDim.x / 32);
  uint32_t g = (Multi ? P.al_lo : 0u) + (uint32_t)((gw * (unsigned long long)(Multi ? P.al_hi - P.al_lo : P.al_nb)) / nw);
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
  const unsigned long long limit = (n_items + 2ull) * ((Multi ? P.al_hi - P.al_lo : P.al_nb) + 2ull) + 64ull;
  for (unsigned long long guard = 0; guard < limit; ++guard) {
    g = Multi ? C->bucket0 + e : e;
    // idle lanes claim shots that start at event e of circuit ci (one atomic per warp)
    // the event's header and body, loaded before the claims so that their latency overlaps
    // the claims' (w42 FP32: 710.8 -> 715.0 M shots/s)
    const Ev<W> *E = evs + e;
    uint4 hdr = make_uint4(0u, 0u, 0u, 0u);
    uint64_t body[4 * W];
#pragma unroll
    for (int k = 0; k < 4 * W; ++k) body[k] = 0ull;
    if (e < n_ev) {  // (no event past the last)
      hdr = __ldg(reinterpret_cast<const uint4 *>(E));
      const ulonglong2 *bp = reinterpret_cast<const ulonglong2 *>(&E->dsd[0]);
#pragma unroll
      for (int k = 0; k < 2 * W; ++k) {
        const ulonglong2 v = __ldg(bp + k);
        body[2 * k] = v.x;
        body[2 * k + 1] = v.y;
      }
    }
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
      if (active && s.status == LS_RUN) s.step(e, hdr, body, E);
    }
    // a spill record to write (a hand-over or an eviction), written once below
    uint32_t ev_r = 0xFFFFFFFFu, ev_e = 0;
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
          ev_r = r;
          ev_e = e;
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
            ev_r = (uint32_t)r;
            ev_e = e + 1u;
            active = false;
          }
        }
      }
    }
    if (ev_r != 0xFFFFFFFFu) s.evict(S, ev_r, item, ev_e);
    uint32_t en = e + 1u > n_ev ? 0u : e + 1u;  // (within the circuit, cyclically)
    if (!__any_sync(0xFFFFFFFFu, active)) {
      // all lanes idle: the next bucket of any circuit (cyclically) that still has shots, or stop
      uint32_t found = 0xFFFFFFFFu;
      if (lane == 0) {
        const uint32_t b_lo = Multi ? P.al_lo : 0u, nb = Multi ? P.al_hi - P.al_lo : P.al_nb;
        const uint32_t g1 = (Multi ? C->bucket0 : 0u) + en - b_lo;
        for (uint32_t k = 0; k < nb; ++k) {
          const uint32_t c = b_lo + (g1 + k) % nb;
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

template <uint32_t Cap>
static size_t lane_smem_bytes_t(int fp32, uint32_t W, uint32_t rw) {
  const size_t per = fp32 ? (W == 1 ? lane_warp_bytes<float, 1, Cap>(rw) : lane_warp_bytes<float, 2, Cap>(rw))
                          : (W == 1 ? lane_warp_bytes<double, 1, Cap>(rw) : lane_warp_bytes<double, 2, Cap>(rw));
  return per * (lane_block<Cap>() / 32);
}
size_t lane_smem_bytes(int fp32, uint32_t W, uint32_t rw, uint32_t cap) {
  return cap == kLaneBigCap ? lane_smem_bytes_t<kLaneBigCap>(fp32, W, rw)
         : cap == kWideCap  ? lane_smem_bytes_t<kWideCap>(fp32, W, rw)
                            : lane_smem_bytes_t<kLaneCap>(fp32, W, rw);
}

uint32_t lane_map_cap() { return kLaneCap; }
uint32_t lane_map_dim() { return lane_dim(kLaneCap); }
uint32_t lane_first_cap(uint32_t max_n, uint32_t max_d, int fp32) {
  if (max_n <= kLaneCap && max_d <= lane_dim(kLaneCap)) return kLaneCap;
  if (max_n <= kWideCap && max_d <= lane_dim(kWideCap)) return kWideCap;
  if (fp32 && max_n <= kLaneBigCap && max_d <= lane_dim(kLaneBigCap)) return kLaneBigCap;
  return 0;
}

cudaError_t launch_snap_affine(unsigned char *traj, uint32_t n_snap, uint32_t rw, int fp32, uint32_t W,
                               uint32_t *stop, cudaStream_t st) {
  const unsigned grid = (n_snap + 127) / 128;
  if (fp32) {
    if (W == 1) snap_affine_kernel<float, 1><<<grid, 128, 0, st>>>(traj, n_snap, (uint32_t)snap_stride<float, 1>(rw), rw, stop);
    else snap_affine_kernel<float, 2><<<grid, 128, 0, st>>>(traj, n_snap, (uint32_t)snap_stride<float, 2>(rw), rw, stop);
  } else {
    if (W == 1) snap_affine_kernel<double, 1><<<grid, 128, 0, st>>>(traj, n_snap, (uint32_t)snap_stride<double, 1>(rw), rw, stop);
    else snap_affine_kernel<double, 2><<<grid, 128, 0, st>>>(traj, n_snap, (uint32_t)snap_stride<double, 2>(rw), rw, stop);
  }
  return cudaGetLastError();
}
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

template <uint32_t Cap>
static const void *lane_kernel_for(int fp32, uint32_t W, bool multi) {
  if (fp32)
    return W == 1 ? (multi ? reinterpret_cast<const void *>(lane_kernel<float, 1, true, Cap>)
                           : reinterpret_cast<const void *>(lane_kernel<float, 1, false, Cap>))
                  : (multi ? reinterpret_cast<const void *>(lane_kernel<float, 2, true, Cap>)
                           : reinterpret_cast<const void *>(lane_kernel<float, 2, false, Cap>));
  if constexpr (Cap == kLaneBigCap) {
    return nullptr;  // 64-entry lanes: FP32 only (an FP64 warp's map would not leave room for two blocks)
  } else {
    return W == 1 ? (multi ? reinterpret_cast<const void *>(lane_kernel<double, 1, true, Cap>)
                           : reinterpret_cast<const void *>(lane_kernel<double, 1, false, Cap>))
                  : (multi ? reinterpret_cast<const void *>(lane_kernel<double, 2, true, Cap>)
                           : reinterpret_cast<const void *>(lane_kernel<double, 2, false, Cap>));
  }
}

cudaError_t prepare_lanes(const ShotParams &p, int fp32, uint32_t W, int blocks_per_sm, LaunchCfg *cfg, uint32_t cap) {
  const bool multi = p.n_circ > 1;
  const void *kern = cap == kLaneBigCap ? lane_kernel_for<kLaneBigCap>(fp32, W, multi)
                     : cap == kWideCap  ? lane_kernel_for<kWideCap>(fp32, W, multi)
                                        : lane_kernel_for<kLaneCap>(fp32, W, multi);
  if (!kern) return cudaErrorInvalidConfiguration;
  const size_t smem = lane_smem_bytes(fp32, W, p.rw_max, cap);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int block = cap == kWideCap ? lane_block<kWideCap>() : kLaneBlock;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, block, smem)) != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  if (blocks_per_sm > 0 && blocks_per_sm < occ) occ = blocks_per_sm;
  cfg->kern = kern;
  cfg->grid = (unsigned)(occ * sms);
  cfg->block = (unsigned)block;
  cfg->smem = smem;
  return cudaSuccess;
}

}  // namespace soft
