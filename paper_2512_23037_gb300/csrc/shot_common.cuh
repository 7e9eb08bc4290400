// shot_common.cuh -- per-shot device pieces shared by the shot kernels: the
// noise stream's next accepted site, the event a shot starts at, the layout of
// the noiseless run's snapshots, and the spill records through which a shot
// moves between lanes of later rounds, or from a lane to a warp.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "device_common.cuh"
#include "kernels.cuh"

namespace soft {
namespace dev {

// The next accepted error site at or after `cur` of shot `shot`: geometric gaps
// of the noise stream against the thresholds thr (the smallest gap g with
// U < thr[g]), then thinning. nxt = the site (0xFFFFFFFF if none), w2 = its
// Pauli choice word. False if the guard ran out (impossible for valid tables).
template <bool Rolled = false>
__device__ __forceinline__ bool next_site(const CircDev *C, uint64_t seed, uint64_t shot, uint32_t &cur,
                                          uint32_t &kblk, uint32_t &nxt, uint32_t &w2) {
  const uint32_t n_sites = C->n_sites;
  const uint64_t *thr = C->thr;
  for (uint32_t guard = 0; guard <= n_sites; ++guard) {
    if (cur >= n_sites) {
      nxt = 0xFFFFFFFFu;
      return true;
    }
    uint4 w = philox<Rolled>(seed, shot, 0u, kblk++);
    uint64_t U = (uint64_t)w.x | ((uint64_t)w.y << 32);
    const uint32_t rem = n_sites - cur;
    uint32_t lo = 0, hi = rem;
    if (C->thr_tab) {  // U's bucket bounds the answer: search between its entry and the next
      const uint32_t b = (uint32_t)(U >> (64 - kThrTabBits));
      const uint32_t t0 = __ldg(&C->thr_tab[b]), t1 = __ldg(&C->thr_tab[b + 1]);
      lo = t0 < rem ? t0 : rem;
      hi = t1 < rem ? t1 : rem;
    }
    while (lo < hi) {
      uint32_t mid = (lo + hi) >> 1;
      if (U < __ldg(&thr[mid])) hi = mid;
      else lo = mid + 1u;
    }
    if (lo == rem) {
      cur = n_sites;
      nxt = 0xFFFFFFFFu;
      return true;
    }
    uint32_t s = cur + lo;
    cur = s + 1u;
    const Site *st = C->sites + s;
    if (!__ldg(&st->always) && !(w.w < __ldg(&st->thin))) continue;
    nxt = s;
    w2 = w.z;
    return true;
  }
  nxt = 0xFFFFFFFFu;
  return false;
}

// The event a shot whose first error is at site nxt starts at: the event that
// applies that error, capped at the last valid event of the noiseless run
// (fidelity mode: of its part before the first observed measurement).
__device__ __forceinline__ uint32_t first_event(const CircDev *C, int fid_mode, uint32_t nxt) {
  const uint32_t stop = fid_mode && C->traj_fid_stop < C->traj_stop ? C->traj_fid_stop : C->traj_stop;
  if (nxt < C->n_sites) {
    const uint32_t e = __ldg(&C->site_ev[nxt]);
    return e < stop ? e : stop;
  }
  return stop;
}

// Snapshot of the noiseless run at the top of an event: header, rw record words,
// kSnapMax keys (W words each), kSnapMax values.
struct SnapHdr {
  uint32_t nnz, chain, logical, lastm;
  double fid;
  uint64_t sd[2], ss[2];
  uint64_t pad[2];
};
constexpr uint32_t kSnapMax = 64;

// The snapshot's map in the affine form of the lane kernels (lanes.cu): d directions
// (0xFFFFFFFF: more than kSnapDim), the live slots (bit s: slot s), rows alpha0,
// B[0..kSnapDim), Dual[0..kSnapDim), and the values of 2^kSnapDim slots (zero where not
// live). Computed once per circuit and precision, after the noiseless run.
constexpr uint32_t kSnapDim = 6;
template <typename R, int W>
struct SnapAffine {
  uint32_t d, live_lo, live_hi, pad;  // live: the slot set, in two words
  uint64_t rows[1 + 2 * kSnapDim][W];
  Cx<R> v[1u << kSnapDim];
};
template <typename R, int W>
__host__ __device__ constexpr size_t snap_affine_off(uint32_t rw) {
  return (sizeof(SnapHdr) + (size_t)rw * 8 + kSnapMax * (size_t)W * 8 + kSnapMax * sizeof(Cx<R>) + 15) &
         ~(size_t)15;
}
template <typename R, int W>
__host__ __device__ constexpr size_t snap_stride(uint32_t rw) {
  return (snap_affine_off<R, W>(rw) + sizeof(SnapAffine<R, W>) + 15) & ~(size_t)15;
}

#ifndef SOFT_LANE_CAP
#define SOFT_LANE_CAP 16
#endif
constexpr uint32_t kLaneCap = SOFT_LANE_CAP;  // map entries per lane
static_assert(kLaneCap >= 2 && kLaneCap <= 16, "lane map capacity (partner indices are 4-bit)");

// A rerun-list entry with this bit names a spill record (a shot handed from its
// lane to a warp) instead of an item.
constexpr uint32_t kSpillRef = 0x80000000u;
constexpr uint32_t kNoRecord = 0xFFFFFFFFu;

// A spill record holds one shot's whole state at the top of an event: item,
// resume event, n and flags (chain, logical, last outcome); the noise cursor
// (nxt, cur, kblk, w2); F; the signs; the record words; up to kLaneCap entries.
// Structure of arrays over `cap` records.
template <typename R, int W>
struct Spill {
  uint4 *ha, *hb;
  double *fid;
  uint64_t *sd, *ss, *rec, *keys;
  Cx<R> *vals;
  uint32_t cap;
  __host__ __device__ static size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }
  __host__ __device__ static size_t bytes(uint32_t cap, uint32_t rw) {
    const size_t c = cap;
    return 2 * al16(c * 16) + al16(c * 8) + 2 * al16(c * 8 * W) + al16(c * 8 * rw) + al16(c * 8 * W * kLaneCap) +
           al16(c * sizeof(Cx<R>) * kLaneCap);
  }
  __device__ Spill(unsigned char *b, uint32_t cap_, uint32_t rw) : cap(cap_) {
    const size_t c = cap;
    ha = reinterpret_cast<uint4 *>(b);
    b += al16(c * 16);
    hb = reinterpret_cast<uint4 *>(b);
    b += al16(c * 16);
    fid = reinterpret_cast<double *>(b);
    b += al16(c * 8);
    sd = reinterpret_cast<uint64_t *>(b);
    b += al16(c * 8 * W);
    ss = reinterpret_cast<uint64_t *>(b);
    b += al16(c * 8 * W);
    rec = reinterpret_cast<uint64_t *>(b);
    b += al16(c * 8 * rw);
    keys = reinterpret_cast<uint64_t *>(b);
    b += al16(c * 8 * W * kLaneCap);
    vals = reinterpret_cast<Cx<R> *>(b);
  }
};

}  // namespace dev
}  // namespace soft
