// api.cu -- the C ABI of include/soft.h: circuit handles, runs, tallies.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/soft.h"
#include "compile.h"
#include "handles.h"
#include "kernels.cuh"

namespace {
thread_local std::string g_err;

int fail(int code, const std::string &msg) {
  g_err = msg;
  return code;
}
int cuda_fail(cudaError_t e, const char *what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return SOFT_E_CUDA;
}

constexpr uint64_t kDefaultChunk = 1ull << 24;
using soft::kDefaultFirstCap;
using soft::kTauFp32;
using soft::kTauFp64;
}  // namespace

namespace soft {
int set_error(int code, const char *msg) { return fail(code, msg); }
}  // namespace soft

struct soft_run {
  cudaStream_t stream = nullptr;
  uint32_t n_circ = 0;
  std::vector<soft_circuit *> circs;       // borrowed: must outlive the run's stream work
  std::vector<uint64_t> n_shots;
  unsigned long long *d_tally = nullptr;   // 5 counters per circuit
  double *d_fsum = nullptr;                // fidelity mode: sum of F per circuit
  uint32_t *d_al = nullptr;                // lane-per-shot bucketing buffers
  unsigned char *d_sp = nullptr;           // lane-per-shot spill pool (shots evicted between rounds)
  unsigned long long *d_lr = nullptr;      // its record count and each round's record range
  bool fid_mode = false;
  unsigned long long *d_work = nullptr;    // next1, next2, n_rerun, item_base, diag[4], reruns of all chunks,
                                           // middle pass: next, n_rerun
  uint32_t *d_rerun = nullptr;
  unsigned char *d_slab = nullptr;         // global-memory state for large-cap reruns
  uint8_t *d_status = nullptr;             // circuit 0 only
  uint64_t *d_records = nullptr;
  uint64_t out_limit = 0;
  uint64_t *d_st_signs = nullptr, *d_st_keys = nullptr;
  double *d_st_vals = nullptr;
  uint32_t *d_st_nnz = nullptr;
  uint64_t st_limit = 0;
  uint32_t st_stride = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<cudaEvent_t> pass_ev;        // SOFT_RUN_TIME_PASSES: 4 per chunk around pre-pass, first, rerun
  uint32_t launches = 0;
  // every device buffer above that the run owns lives in one arena, borrowed from
  // the device's cached workspace when it fits
  void *arena = nullptr;
  size_t arena_bytes = 0;
  int device = 0;
};

namespace {
// Per device: the cached run workspace (one arena), lent to a run that fits in it
// and handed back at soft_run_free; freed by soft_release_workspace.
struct WsCache {
  std::mutex mu;
  void *p = nullptr;
  size_t bytes = 0;
};
constexpr int kMaxDevices = 64;
WsCache g_ws[kMaxDevices];
}  // namespace

// Records both precisions' noiseless runs of a freshly uploaded circuit (the
// prefix every shot shares until its first error). Synchronous, but on streams
// of its own: it waits for no other work on the device.
static cudaError_t build_prefixes(soft_circuit *c, cudaStream_t us) {
  const auto &hp = c->hp;
  const size_t n_snap = hp.ev.size() + 1;
  uint32_t *d_stop = nullptr;  // per precision: last valid event, first fidelity event, largest map, largest dimension
  cudaError_t e = cudaMalloc(&d_stop, 8 * sizeof(uint32_t));
  if (e != cudaSuccess) return e;
  c->d_stop = d_stop;
  if ((e = cudaMemsetAsync(d_stop, 0, 8 * sizeof(uint32_t), us)) != cudaSuccess ||
      (e = cudaStreamSynchronize(us)) != cudaSuccess)
    return e;
  // the two precisions' runs are one warp each: they run side by side on two streams
  cudaStream_t ps[2] = {nullptr, nullptr};
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaStreamCreateWithFlags(&ps[k], cudaStreamNonBlocking);
  for (int fp32 = 0; fp32 < 2 && e == cudaSuccess; ++fp32) {  // (allocations first: they may synchronise)
    const size_t stride = soft::prefix_stride(fp32, hp.W, hp.rw);
    if ((e = cudaMalloc(&c->d_traj[fp32], n_snap * stride)) != cudaSuccess) break;
    c->traj_stride[fp32] = (uint32_t)stride;
  }
  for (int fp32 = 0; fp32 < 2 && e == cudaSuccess; ++fp32) {
    soft::ShotParams p{};
    p.n_circ = 1;
    soft::CircDev &d = p.circ[0];
    d.ev = c->d_ev;
    d.coef = c->d_coef;
    d.cb = c->d_cb;
    d.sites = c->d_sites;
    d.thr = c->d_thr;
    d.n_events = (uint32_t)hp.ev.size();
    d.n_sites = hp.n_sites;
    d.rw = hp.rw;
    d.cap = hp.cap;
    d.n_coef = (uint32_t)hp.coefs.size();
    d.n_cb = (uint32_t)hp.cb.size();
    p.cap = std::min(hp.cap, soft::kDefaultFirstCap);
    p.rw_max = hp.rw;
    p.tau = fp32 ? kTauFp32 : kTauFp64;
    e = soft::launch_prefix(p, fp32, hp.W, c->d_traj[fp32], d_stop + 4 * fp32, ps[fp32]);
    if (e == cudaSuccess)
      e = soft::launch_snap_affine(c->d_traj[fp32], (uint32_t)n_snap, hp.rw, fp32, hp.W, d_stop + 4 * fp32, ps[fp32]);
  }
  for (int k = 0; k < 2; ++k)
    if (ps[k]) {
      const cudaError_t es = cudaStreamSynchronize(ps[k]);
      if (e == cudaSuccess) e = es;
      cudaStreamDestroy(ps[k]);
    }
  uint32_t stop[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (e == cudaSuccess && (e = cudaMemcpyAsync(stop, d_stop, sizeof stop, cudaMemcpyDeviceToHost, us)) == cudaSuccess)
    e = cudaStreamSynchronize(us);
  if (e != cudaSuccess) return e;
  for (int k = 0; k < 2; ++k) {
    c->traj_stop[k] = std::min<uint32_t>(stop[4 * k], (uint32_t)hp.ev.size());
    c->traj_fid_stop[k] = std::min<uint32_t>(stop[4 * k + 1], (uint32_t)hp.ev.size());
    c->traj_max_n[k] = stop[4 * k + 2];
    c->traj_max_d[k] = stop[4 * k + 3];
  }
  return cudaSuccess;
}

extern "C" {

const char *soft_last_error(void) { return g_err.c_str(); }

int soft_compile_circuit(const soft_op *ops, size_t n_ops, uint32_t n_qubits, const soft_noise *noise,
                         uint32_t coeff_cap, soft_circuit **out) {
  if (!out) return fail(SOFT_E_ARG, "out is NULL");
  *out = nullptr;
  soft_circuit *c = new (std::nothrow) soft_circuit();
  if (!c) return fail(SOFT_E_OOM, "host allocation failed");
  std::string err;
  int rc = soft::compile_program(ops, n_ops, n_qubits, noise, coeff_cap, c->hp, err);
  if (rc != SOFT_OK) {
    delete c;
    return fail(rc, err);
  }
  cudaGetDevice(&c->device);
  const auto &hp = c->hp;
  // narrow the events to the one-word layout when n <= 64
  std::vector<soft::Ev<1>> ev1;
  const void *ev_src = hp.ev.data();
  size_t b_ev = hp.ev.size() * sizeof(soft::Ev<2>);
  if (hp.W == 1) {
    ev1.resize(hp.ev.size());
    for (size_t i = 0; i < hp.ev.size(); ++i) {
      const auto &s = hp.ev[i];
      ev1[i] = soft::Ev<1>{s.w0, s.site_begin, s.a, s.b, {s.dsd[0]}, {s.dss[0]},
                           {s.beta[0]}, {s.gamma[0]}, {s.xbeta[0]}, {s.xgamma[0]}};
    }
    ev_src = ev1.data();
    b_ev = ev1.size() * sizeof(soft::Ev<1>);
  }
  size_t b_cf = std::max<size_t>(1, hp.coefs.size()) * sizeof(soft::Coef),
         b_cb = std::max<size_t>(1, hp.cb.size()) * sizeof(soft::CaseB),
         b_st = std::max<size_t>(1, hp.sites.size()) * sizeof(soft::Site),
         b_thr0 = hp.thr.size() * sizeof(uint64_t), b_thr1 = b_thr0 + hp.site_ev.size() * sizeof(uint32_t),
         b_thr = b_thr1 + hp.thr_tab.size() * sizeof(uint32_t);
  cudaError_t e;
  if ((e = cudaMalloc(&c->d_ev, b_ev)) != cudaSuccess || (e = cudaMalloc(&c->d_coef, b_cf)) != cudaSuccess ||
      (e = cudaMalloc(&c->d_cb, b_cb)) != cudaSuccess || (e = cudaMalloc(&c->d_sites, b_st)) != cudaSuccess ||
      (e = cudaMalloc(&c->d_thr, b_thr)) != cudaSuccess) {
    soft_circuit_free(c);
    return e == cudaErrorMemoryAllocation ? fail(SOFT_E_OOM, "device allocation failed") : cuda_fail(e, "cudaMalloc");
  }
  // uploads on a stream of the compile's own (a non-blocking one), so that compiling
  // waits for no other work on the device, a running batch of shots included
  cudaStream_t us = nullptr;
  if ((e = cudaStreamCreateWithFlags(&us, cudaStreamNonBlocking)) != cudaSuccess) {
    soft_circuit_free(c);
    return cuda_fail(e, "cudaStreamCreateWithFlags");
  }
  auto up = [&](void *dst, const void *src, size_t bytes) {
    return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, us) : cudaSuccess;
  };
  unsigned char *thr_b = reinterpret_cast<unsigned char *>(c->d_thr);
  if ((e = up(c->d_ev, ev_src, b_ev)) != cudaSuccess ||
      (e = up(c->d_coef, hp.coefs.data(), hp.coefs.size() * sizeof(soft::Coef))) != cudaSuccess ||
      (e = up(c->d_cb, hp.cb.data(), hp.cb.size() * sizeof(soft::CaseB))) != cudaSuccess ||
      (e = up(c->d_sites, hp.sites.data(), hp.sites.size() * sizeof(soft::Site))) != cudaSuccess ||
      (e = up(c->d_thr, hp.thr.data(), b_thr0)) != cudaSuccess ||
      (e = up(thr_b + b_thr0, hp.site_ev.data(), hp.site_ev.size() * sizeof(uint32_t))) != cudaSuccess ||
      (e = up(thr_b + b_thr1, hp.thr_tab.data(), hp.thr_tab.size() * sizeof(uint32_t))) != cudaSuccess ||
      (e = cudaStreamSynchronize(us)) != cudaSuccess) {
    cudaStreamDestroy(us);
    soft_circuit_free(c);
    return cuda_fail(e, "program upload");
  }
  c->bytes = b_ev + b_cf + b_cb + b_st + b_thr;
  e = build_prefixes(c, us);
  cudaStreamDestroy(us);
  if (e != cudaSuccess) {
    soft_circuit_free(c);
    return e == cudaErrorMemoryAllocation ? fail(SOFT_E_OOM, "device allocation failed")
                                          : cuda_fail(e, "noiseless prefix run");
  }
  *out = c;
  return SOFT_OK;
}

int soft_circuit_info(const soft_circuit *c, soft_circuit_info_t *out) {
  if (!c || !out) return fail(SOFT_E_ARG, "null argument");
  out->n_qubits = c->hp.n;
  out->n_records = c->hp.n_records;
  out->record_words = c->hp.rw;
  out->n_sites = c->hp.n_sites;
  out->n_events = (uint32_t)c->hp.ev.size();
  out->coeff_cap = c->hp.cap;
  out->program_bytes = c->bytes;
  return SOFT_OK;
}

int soft_circuit_tableau(const soft_circuit *c, uint64_t *rows_x, uint64_t *rows_z) {
  if (!c || !rows_x || !rows_z) return fail(SOFT_E_ARG, "null argument");
  std::memcpy(rows_x, c->hp.fin_x.data(), c->hp.fin_x.size() * sizeof(uint64_t));
  std::memcpy(rows_z, c->hp.fin_z.data(), c->hp.fin_z.size() * sizeof(uint64_t));
  return SOFT_OK;
}

void soft_circuit_free(soft_circuit *c) {
  if (!c) return;
  cudaFree(c->d_ev);
  cudaFree(c->d_coef);
  cudaFree(c->d_cb);
  cudaFree(c->d_sites);
  cudaFree(c->d_thr);
  cudaFree(c->d_traj[0]);
  cudaFree(c->d_traj[1]);
  cudaFree(c->d_stop);
  cudaFree(c->d_gcoef);
  cudaFree(c->d_gnext);
  cudaFree(c->d_gtape);
  cudaFree(c->d_gprefix);
  cudaFree(c->d_gwide);
  delete c;
}

void soft_run_free(soft_run *r) {
  if (!r) return;
  if (r->stream) cudaStreamSynchronize(r->stream);
  else cudaDeviceSynchronize();
  // the arena goes back to the circuit's slot (unless the circuit is gone, or keeps a
  // larger one), else it is freed
  if (r->arena) {
    bool kept = false;
    if (r->device >= 0 && r->device < kMaxDevices) {
      WsCache &w = g_ws[r->device];
      std::lock_guard<std::mutex> lk(w.mu);
      if (!w.p || w.bytes < r->arena_bytes) {
        cudaFree(w.p);
        w.p = r->arena;
        w.bytes = r->arena_bytes;
        kept = true;
      }
    }
    if (!kept) cudaFree(r->arena);
  }
  if (r->graph_exec) cudaGraphExecDestroy(r->graph_exec);
  if (r->graph) cudaGraphDestroy(r->graph);
  if (r->ev0) cudaEventDestroy(r->ev0);
  if (r->ev1) cudaEventDestroy(r->ev1);
  for (size_t k = 0; k < r->pass_ev.size(); ++k)
    if (k == 0 || r->pass_ev[k] != r->pass_ev[k - 1]) cudaEventDestroy(r->pass_ev[k]);
  delete r;
}

}  // extern "C"

namespace soft {

CircDev circ_desc(const soft_circuit *c, int fp32, bool prefix) {
  soft::CircDev d{};
  d.site_ev = reinterpret_cast<const uint32_t *>(c->d_thr + c->hp.thr.size());
  d.thr_tab = d.site_ev + c->hp.site_ev.size();
  if (prefix && c->d_traj[fp32]) {
    d.traj = c->d_traj[fp32];
    d.traj_stop = c->traj_stop[fp32];
    d.traj_fid_stop = c->traj_fid_stop[fp32];
    d.traj_stride = c->traj_stride[fp32];
  }
  d.ev = c->d_ev;
  d.coef = c->d_coef;
  d.cb = c->d_cb;
  d.sites = c->d_sites;
  d.thr = c->d_thr;
  d.n_events = (uint32_t)c->hp.ev.size();
  d.n_sites = c->hp.n_sites;
  d.rw = c->hp.rw;
  d.cap = c->hp.cap;
  d.n_coef = (uint32_t)c->hp.coefs.size();
  d.n_cb = (uint32_t)c->hp.cb.size();
  return d;
}

}  // namespace soft

namespace {

using soft::circ_desc;

// Shared launcher of soft_run_shots and soft_run_batch.
int run_many(soft_circuit *const *circs, const uint64_t *n_shots, const uint64_t *first_shots, uint32_t n_circ,
             uint64_t seed, const soft_run_opts *opts, soft_run **out) {
  if (!circs || !n_shots || !first_shots || !out || n_circ == 0) return fail(SOFT_E_ARG, "null argument or empty batch");
  *out = nullptr;
  if (n_circ > (uint32_t)soft::kMaxCirc) return fail(SOFT_E_ARG, "at most 64 circuits per batch");
  soft_run_opts o{};
  if (opts) o = *opts;
  if (o.precision != SOFT_FP64 && o.precision != SOFT_FP32) return fail(SOFT_E_ARG, "bad precision");
  if (o.record_mode < SOFT_REC_NONE || o.record_mode > SOFT_REC_ALL) return fail(SOFT_E_ARG, "bad record mode");
  if (o.group_size != 0 && o.group_size != 16 && o.group_size != 32)
    return fail(SOFT_E_ARG, "group_size must be 0, 16 or 32");
  if (o.groups_per_block > 128u / (o.group_size ? o.group_size : 32u))
    return fail(SOFT_E_ARG, "groups_per_block must be 0..128/group_size");
  if (n_circ > 1 && (o.record_mode != SOFT_REC_NONE || o.capture_k))
    return fail(SOFT_E_ARG, "records and state capture are per single-circuit run");
  const bool use_graph = (o.flags & SOFT_RUN_GRAPH) != 0;
  const bool fid_mode = (o.flags & SOFT_RUN_FIDELITY) != 0;
  if (o.flags & ~(uint32_t)(SOFT_RUN_GRAPH | SOFT_RUN_FIDELITY | SOFT_RUN_NO_PREFIX | SOFT_RUN_NO_LANES |
                          SOFT_RUN_TIME_PASSES | SOFT_RUN_NO_WIDE_LANES | SOFT_RUN_WIDE_LANES))
    return fail(SOFT_E_ARG, "unknown run flags");
  if (use_graph && !o.stream) return fail(SOFT_E_ARG, "graph replay needs a non-default stream");
  const int fp32 = o.precision == SOFT_FP32;
  uint32_t W = 0, cap_max = 0, rw_max = 1;
  uint64_t total = 0;
  for (uint32_t i = 0; i < n_circ; ++i) {
    if (!circs[i]) return fail(SOFT_E_ARG, "null circuit");
    if (W && circs[i]->hp.W != W) return fail(SOFT_E_ARG, "all circuits of a batch need n <= 64 or all n > 64");
    if (circs[i]->device != circs[0]->device) return fail(SOFT_E_ARG, "all circuits of a batch must be on one device");
    if (fid_mode && !circs[i]->hp.fid_ok)
      return fail(SOFT_E_ARG, "fidelity mode needs every DETECTOR before the first observed measurement");
    W = circs[i]->hp.W;
    cap_max = std::max(cap_max, circs[i]->hp.cap);
    rw_max = std::max(rw_max, circs[i]->hp.rw);
    total += n_shots[i];
  }
  const uint32_t cap1 = o.first_cap ? std::min(o.first_cap, cap_max) : std::min(kDefaultFirstCap, cap_max);
  // lane-per-shot scheduling: the noiseless prefix, group size not forced, a circuit whose
  // noiseless run's maps fit a lane's map (16 entries; else 32; else, FP32, 64), and at most
  // lane_max_buckets buckets (one per event, plus one, per such circuit). The shots of the
  // other circuits of a batch go straight to the warp pass that follows the lanes.
  const int pk = o.precision == SOFT_FP32 ? 1 : 0;
  const uint32_t lc16 = soft::lane_map_cap();
  std::vector<uint32_t> lcap(n_circ);  // each circuit's lane map (0: none)
  uint64_t nbc[3] = {0, 0, 0};         // buckets of the circuits of 16-, 32- and 64-entry lanes
  auto lane_class = [&](uint32_t c) { return c == lc16 ? 0 : c == 2 * lc16 ? 1 : c == 4 * lc16 ? 2 : 3; };
  for (uint32_t i = 0; i < n_circ; ++i) {
    lcap[i] = circs[i]->d_traj[pk] ? soft::lane_first_cap(circs[i]->traj_max_n[pk], circs[i]->traj_max_d[pk], fp32) : 0u;
    if (lcap[i]) nbc[lane_class(lcap[i])] += circs[i]->hp.ev.size() + 1;
  }
  const uint64_t n_buckets = nbc[0] + nbc[1] + nbc[2];
  const bool lanes = !(o.flags & SOFT_RUN_NO_LANES) && !(o.flags & SOFT_RUN_NO_PREFIX) && o.group_size == 0 &&
                     n_buckets > 0 && n_buckets <= soft::lane_max_buckets();
  const uint32_t nb = lanes ? (uint32_t)n_buckets : 0u;
  const bool lanes16 = lanes && nbc[0] > 0;  // the lanes that evict, hand over and feed the wide round
  // a rerun pass finishes the shots whose maps outgrow the first pass (cap1). After lanes it
  // always runs: a lane decides overflow only after pruning, and a map that outgrows the lane
  // before pruning is staged whole by the warp pass, even when the circuit's cap is the lane's.
  const bool lane_grow = lanes16 && lc16 < cap_max;  // maps may outgrow a 16-entry lane
  const bool two_pass = lanes || cap1 < cap_max;
  // after lanes, a middle pass (a warp per shot, map up to cap1 entries) takes the shots whose
  // maps outgrew a lane, and only those that outgrow cap1 go on to the pass at the circuit's
  // cap. Not when every lane of the run holds 64 entries already: then a shot that outgrew one
  // goes straight to the circuit's cap (w97 FP32: 44.7 M shots/s against 44.5 M through a
  // middle pass at 64, and 27.0 M through one at 256, whose larger maps cut its residency).
  // With smaller lanes in the run it stays for all (many maps that outgrow a 64-entry lane's
  // six directions still fit 64 entries: batch64 FP32 113 M shots/s when they skipped it)
  const bool mid_pass = lanes && lc16 < cap1 && cap1 < cap_max && (nbc[0] > 0 || nbc[1] > 0);
  const uint32_t g1 = o.group_size ? o.group_size : 32u;
  const uint32_t g2 = 32;
  const size_t smem_limit = 227 * 1024 - 5 * sizeof(unsigned long long) * soft::kMaxCirc;
  if (soft::group_smem_bytes(fp32, W, cap1, rw_max) > smem_limit)
    return fail(SOFT_E_ARG, "first_cap too large for the on-chip coefficient map");
  const bool global_rerun = two_pass && soft::group_smem_bytes(fp32, W, cap_max, rw_max) > smem_limit;
  const int dev = circs[0]->device;
  cudaError_t e = cudaSetDevice(dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");

  soft_run *r = new (std::nothrow) soft_run();
  if (!r) return fail(SOFT_E_OOM, "host allocation failed");
  r->stream = (cudaStream_t)o.stream;
  r->n_circ = n_circ;
  r->circs.assign(circs, circs + n_circ);
  r->n_shots.assign(n_shots, n_shots + n_circ);
  const uint64_t chunk = o.chunk_shots ? o.chunk_shots : std::min<uint64_t>(kDefaultChunk, std::max<uint64_t>(total, 1));
  if (chunk > 0xFFFFFFFFull) {
    soft_run_free(r);
    return fail(SOFT_E_ARG, "chunk_shots must be < 2^32");
  }
  const uint64_t n0 = n_shots[0];
  r->out_limit = o.record_mode == SOFT_REC_ALL ? n0 : (o.record_mode == SOFT_REC_FIRST_K ? std::min(o.record_k, n0) : 0);
  r->st_limit = std::min<uint64_t>(o.capture_k, n0);
  r->st_stride = circs[0]->hp.cap;
  cudaStream_t st = r->stream;
  // every buffer the run owns is carved from one arena (256-byte aligned pieces)
  struct Piece {
    void **ptr;
    size_t bytes;
  };
  std::vector<Piece> pieces;
  size_t arena_bytes = 0;
  auto need = [&](auto **ptr, size_t bytes) {
    pieces.push_back(Piece{reinterpret_cast<void **>(ptr), bytes});
    arena_bytes += (bytes + 255) & ~(size_t)255;
  };
  need(&r->d_tally, 5 * n_circ * sizeof(unsigned long long));
  // lanes: cursors (4 words per item, first: 16-byte aligned), (start event, rank) pairs, order,
  // bucket starts, counters
  // then the per-block bucket bases of the block-binned pre-pass
  const uint32_t al_grid = lanes ? soft::lane_prepass_grid() : 0u;
  if (lanes)
    need(&r->d_al, (7 * chunk + (nb + 1) + 2 * (size_t)nb + (size_t)al_grid * (nb + 1)) * sizeof(uint32_t));
  // spill pool: records for the shots a sparse warp evicts (a quarter of the chunk; when it is
  // full, warps keep their shots), then records for shots a lane hands to a warp (an eighth;
  // when full, the warp reruns them from their start). Entries of the rerun list name a record
  // with their top bit, so a chunk stays below 2^31 items for it.
  const uint32_t rounds = lanes ? soft::lane_rounds() : 1u;
  const bool spill = lanes16 && (rounds > 1 || lane_grow) && chunk < (1ull << 31);
  const uint32_t sp_evict = rounds > 1 ? (uint32_t)std::max<uint64_t>(std::min<uint64_t>(chunk, 1024), chunk / 4) : 0u;
  const uint32_t sp_hand = lane_grow ? (uint32_t)std::max<uint64_t>(std::min<uint64_t>(chunk, 1024), chunk / 8) : 0u;
  // the wide round: the handed-over shots continue in lanes of twice the map (their records
  // are its input), and only those that outgrow it rerun in a warp. Single-circuit runs only
  // (batches measured slower: 125.5 M against 130.3 M shots/s on batch64, before the affine
  // lanes). By default only for chunks of at least 2^23 shots: its pre-pass and launch cost
  // more than it saves in small runs (w42 at 2^21 shots: 389.0 M against 412.5 M). w42 at 2^24:
  // FP32 550.0 M against 533.0 M (sparse lanes); FP64 348.2 M against 344.5 M (affine lanes).
  const bool wide_ok = spill && lane_grow && n_circ == 1 && !(o.flags & SOFT_RUN_NO_WIDE_LANES);
  const bool wide = wide_ok && ((o.flags & SOFT_RUN_WIDE_LANES) || std::min(chunk, total) >= (1ull << 23));
  const size_t n_lr = 4 + 2 * ((size_t)rounds + 1);
  if (spill) {
    need(&r->d_sp, soft::lane_spill_bytes(fp32, W, rw_max, sp_evict + sp_hand));
    need(&r->d_lr, n_lr * sizeof(unsigned long long));
  }
  r->fid_mode = fid_mode;
  if (fid_mode) need(&r->d_fsum, n_circ * sizeof(double));
  need(&r->d_work, 11 * sizeof(unsigned long long));
  if (two_pass) need(&r->d_rerun, (mid_pass ? 2 : 1) * chunk * sizeof(uint32_t));
  uint32_t slab_blocks = 0;
  if (global_rerun) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // 4 blocks of 4 groups per SM: the rerun pass is latency-bound, so residency pays for the slab
    // memory (1 block/SM: w97 24.5 M shots/s, 4: 26.3 M, 6: 26.4 M)
    slab_blocks = (uint32_t)(sms > 0 ? sms : 1) * 4u;
    need(&r->d_slab, soft::global_slab_bytes(fp32, W, cap_max, rw_max, slab_blocks));
  }
  if (r->out_limit) {
    if (o.d_status) r->d_status = o.d_status;
    else need(&r->d_status, r->out_limit);
    if (o.d_records) r->d_records = o.d_records;
    else need(&r->d_records, r->out_limit * circs[0]->hp.rw * sizeof(uint64_t));
  }
  if (r->st_limit) {
    need(&r->d_st_signs, r->st_limit * 4 * sizeof(uint64_t));
    need(&r->d_st_keys, r->st_limit * r->st_stride * 2 * sizeof(uint64_t));
    need(&r->d_st_vals, r->st_limit * r->st_stride * 2 * sizeof(double));
    need(&r->d_st_nnz, r->st_limit * sizeof(uint32_t));
  }
  // borrow the device's cached arena when it is free and large enough
  r->device = dev;
  if (dev >= 0 && dev < kMaxDevices) {
    WsCache &w = g_ws[dev];
    std::lock_guard<std::mutex> lk(w.mu);
    if (w.p && w.bytes >= arena_bytes) {
      r->arena = w.p;
      r->arena_bytes = w.bytes;
      w.p = nullptr;
      w.bytes = 0;
    }
  }
  if (!r->arena) {
    if ((e = cudaMalloc(&r->arena, arena_bytes)) != cudaSuccess) {
      r->arena = nullptr;
      soft_run_free(r);
      return e == cudaErrorMemoryAllocation ? fail(SOFT_E_OOM, "device allocation failed") : cuda_fail(e, "cudaMalloc");
    }
    r->arena_bytes = arena_bytes;
  }
  {
    unsigned char *at = static_cast<unsigned char *>(r->arena);
    for (const Piece &pc : pieces) {
      *pc.ptr = at;
      at += (pc.bytes + 255) & ~(size_t)255;
    }
  }
  if ((e = cudaEventCreate(&r->ev0)) != cudaSuccess || (e = cudaEventCreate(&r->ev1)) != cudaSuccess) {
    soft_run_free(r);
    return cuda_fail(e, "cudaEventCreate");
  }
  if ((e = cudaMemsetAsync(r->d_tally, 0, 5 * n_circ * sizeof(unsigned long long), st)) != cudaSuccess ||
      (e = cudaMemsetAsync(r->d_work, 0, 11 * sizeof(unsigned long long), st)) != cudaSuccess ||
      (fid_mode && (e = cudaMemsetAsync(r->d_fsum, 0, n_circ * sizeof(double), st)) != cudaSuccess)) {
    soft_run_free(r);
    return cuda_fail(e, "cudaMemsetAsync");
  }
  // launch parameters: one descriptor per circuit, items laid out circuit after circuit. With
  // lanes the descriptors go in order of lane map (16, 32, 64 entries, none), so that each
  // map size's circuits hold a contiguous range of buckets for its own lane launch; each
  // descriptor keeps its circuit's tally (a batch has no records or captured states).
  std::vector<uint32_t> ord(n_circ);
  for (uint32_t i = 0; i < n_circ; ++i) ord[i] = i;
  if (lanes)
    std::stable_sort(ord.begin(), ord.end(), [&](uint32_t x, uint32_t y) {
      return (lcap[x] ? lane_class(lcap[x]) : 3) < (lcap[y] ? lane_class(lcap[y]) : 3);
    });
  soft::ShotParams p{};
  p.n_circ = n_circ;
  uint64_t begin = 0;
  for (uint32_t k = 0; k < n_circ; ++k) {
    const uint32_t i = ord[k];
    p.circ[k] = circ_desc(circs[i], fp32, !(o.flags & SOFT_RUN_NO_PREFIX));
    p.circ[k].item_begin = begin;
    p.circ[k].n_shots = n_shots[i];
    p.circ[k].first_shot = first_shots[i];
    p.circ[k].tally = r->d_tally + 5 * i;
    p.circ[k].fsum = fid_mode ? r->d_fsum + i : nullptr;
    begin += n_shots[i];
  }
  for (uint32_t k = 0, b = 0; lanes && k < n_circ; ++k) {  // each circuit's buckets, circuit after circuit
    const uint32_t i = ord[k];
    p.circ[k].bucket0 = b;
    p.circ[k].lanes_off = lcap[i] ? 0u : 1u;
    if (lcap[i]) b += p.circ[k].n_events + 1;
  }
  p.circ[0].status = r->d_status;
  p.circ[0].records = r->d_records;
  p.circ[0].out_limit = r->out_limit;
  p.rw_max = rw_max;
  p.tau = fp32 ? kTauFp32 : kTauFp64;
  p.seed = seed;
  p.next_item = r->d_work;
  p.rerun = r->d_rerun;
  p.rerun_cap = two_pass ? (uint32_t)chunk : 0u;
  p.n_rerun = r->d_work + 2;
  p.diag = r->d_work + 4;
  p.n_rerun_total = r->d_work + 8;
  p.groups_per_block = o.groups_per_block;
  p.fid_mode = fid_mode ? 1 : 0;
  if (r->st_limit) {
    p.st_limit = r->st_limit;
    p.st_signs = r->d_st_signs;
    p.st_keys = r->d_st_keys;
    p.st_vals = r->d_st_vals;
    p.st_nnz = r->d_st_nnz;
    p.st_stride = r->st_stride;
  }
  p.cap = cap1;
  p.hs_max = soft::hash_slots_for(cap1);
  p.small_pass = two_pass ? 1 : 0;
  soft::ShotParams q = p;
  q.cap = cap_max;
  q.hs_max = soft::hash_slots_for(cap_max);
  q.small_pass = 0;
  q.list = r->d_rerun;
  q.n_items_dev = r->d_work + 2;
  q.next_item = r->d_work + 1;
  q.n_rerun_total = nullptr;
  soft::ShotParams m = q;  // middle pass: first list in, second list out
  if (mid_pass) {
    m.cap = cap1;
    m.hs_max = soft::hash_slots_for(cap1);
    m.small_pass = 1;
    m.next_item = r->d_work + 9;
    m.rerun = r->d_rerun + chunk;
    m.n_rerun = r->d_work + 10;
    q.list = m.rerun;
    q.n_items_dev = m.n_rerun;
  }
  if (global_rerun) {
    q.gslab = r->d_slab;
    q.gslab_blocks = slab_blocks;
  }
  if (lanes) {  // start events, order, bucket starts, then the two counter arrays (zeroed per chunk)
    p.al_cursor = r->d_al;
    p.al_ev = r->d_al + 4 * chunk;
    p.al_order = r->d_al + 6 * chunk;
    p.al_start = r->d_al + 7 * chunk;
    p.al_count = r->d_al + 7 * chunk + (nb + 1);
    p.al_next = p.al_count + nb;
    p.al_base = p.al_next + nb;
    p.al_nb = nb;
    p.al_lo = 0;  // the 16-entry lanes' buckets; the larger lanes' launches set their own
    p.al_hi = (uint32_t)nbc[0];
    p.al_grid = al_grid;
    p.lane_round = 0;
    p.lane_evict = spill && rounds > 1 ? 1u : 0u;
    p.lane_hand = spill ? 1u : 0u;
    p.lane_wide = wide ? 1u : 0u;
    p.lane_wide_round = 0;
    p.sp = spill ? r->d_sp : nullptr;
    p.sp_cap = spill ? sp_evict + sp_hand : 0u;
    p.sp_evict_cap = spill ? sp_evict : 0u;
    p.lr = spill ? r->d_lr : nullptr;
    // the middle pass (or, without one, the pass at the circuit's cap) resumes handed-over shots
    soft::ShotParams &h = mid_pass ? m : q;
    h.sp = p.sp;
    h.sp_cap = p.sp_cap;
    h.sp_evict_cap = p.sp_evict_cap;
  }
  soft::LaunchCfg c1{}, c2{}, cm{}, cw{}, cb[2]{};
  p.n_items = std::min(chunk, total);
  // the larger lanes (32 and 64 entries): one launch each over their circuits' buckets, after
  // the 16-entry lanes' first round; they never evict or hand over
  soft::ShotParams pb[2] = {p, p};
  for (int k = 0; k < 2; ++k) {
    pb[k].al_lo = (uint32_t)(nbc[0] + (k ? nbc[1] : 0));
    pb[k].al_hi = pb[k].al_lo + (uint32_t)nbc[1 + k];
    pb[k].lane_evict = pb[k].lane_hand = pb[k].lane_wide = 0;
    pb[k].sp = nullptr;
    pb[k].sp_cap = pb[k].sp_evict_cap = 0;
    pb[k].lr = nullptr;
  }
  if ((e = !lanes ? soft::prepare_shots(p, fp32, W, g1, (int)o.blocks_per_sm, &c1)
                  : lanes16 ? soft::prepare_lanes(p, fp32, W, (int)o.blocks_per_sm, &c1, lc16) : cudaSuccess) !=
          cudaSuccess ||
      (lanes && nbc[1] && (e = soft::prepare_lanes(pb[0], fp32, W, 0, &cb[0], 2 * lc16)) != cudaSuccess) ||
      (lanes && nbc[2] && (e = soft::prepare_lanes(pb[1], fp32, W, 0, &cb[1], 4 * lc16)) != cudaSuccess) ||
      (wide && (e = soft::prepare_lanes(p, fp32, W, 0, &cw, 2 * lc16)) != cudaSuccess) ||
      (two_pass && (e = soft::prepare_shots(q, fp32, W, g2, (int)o.blocks_per_sm, &c2)) != cudaSuccess) ||
      (mid_pass && (e = soft::prepare_shots(m, fp32, W, g2, (int)o.blocks_per_sm, &cm)) != cudaSuccess)) {
    soft_run_free(r);
    return cuda_fail(e, "shot kernel configuration");
  }
  cudaEventRecord(r->ev0, st);
  // one chunk of items [base, base + cnt): clear counters, first pass, rerun pass
  const bool time_passes = (o.flags & SOFT_RUN_TIME_PASSES) && !use_graph;
  // marks the boundary between passes of a chunk when the caller asked for per-pass times
  // (a pass that does not run repeats the previous event: it reports exactly 0)
  auto mark = [&](bool ran = true) -> cudaError_t {
    if (!time_passes) return cudaSuccess;
    if (!ran && !r->pass_ev.empty()) {
      r->pass_ev.push_back(r->pass_ev.back());
      return cudaSuccess;
    }
    cudaEvent_t ev;
    cudaError_t err = cudaEventCreate(&ev);
    if (err != cudaSuccess) return err;
    r->pass_ev.push_back(ev);
    return cudaEventRecord(ev, st);
  };
  auto enqueue_chunk = [&](uint64_t base, uint64_t cnt, bool dev_base) -> cudaError_t {
    cudaError_t err;
    if ((err = cudaMemsetAsync(r->d_work, 0, 3 * sizeof(unsigned long long), st)) != cudaSuccess) return err;
    if (mid_pass && (err = cudaMemsetAsync(r->d_work + 9, 0, 2 * sizeof(unsigned long long), st)) != cudaSuccess)
      return err;
    soft::ShotParams a = p, b = q, c = m;
    a.n_items = b.n_items = c.n_items = cnt;
    a.item_base = b.item_base = c.item_base = base;
    if (dev_base) a.item_base_dev = b.item_base_dev = c.item_base_dev = r->d_work + 3;
    if ((err = mark()) != cudaSuccess) return err;
    if (lanes) {
      if ((err = cudaMemsetAsync(a.al_count, 0, 2 * (size_t)nb * sizeof(uint32_t), st)) != cudaSuccess ||
          (err = soft::launch_lane_prepass(a, st)) != cudaSuccess)
        return err;
      r->launches += 3;
    }
    if ((err = mark(lanes)) != cudaSuccess) return err;
    if (spill && (err = cudaMemsetAsync(r->d_lr, 0, n_lr * sizeof(unsigned long long), st)) != cudaSuccess)
      return err;
    if (!lanes || lanes16) {
      if ((err = soft::launch_prepared(c1, a, st)) != cudaSuccess) return err;
      r->launches++;
    }
    // the larger lanes, before any later round re-buckets (it clears every bucket's counters)
    for (int k = 0; lanes && k < 2; ++k)
      if (nbc[1 + k]) {
        soft::ShotParams ab = pb[k];
        ab.n_items = cnt;
        ab.item_base = base;
        if (dev_base) ab.item_base_dev = r->d_work + 3;
        if ((err = soft::launch_prepared(cb[k], ab, st)) != cudaSuccess) return err;
        r->launches++;
      }
    // later rounds: the evicted shots, bucketed by the event they resume at
    for (uint32_t rd = 1; spill && rd < rounds; ++rd) {
      soft::ShotParams ar = a;
      ar.lane_round = rd;
      ar.lane_evict = rd + 1 < rounds ? 1u : 0u;
      ar.n_items_dev = r->d_lr + 3 + 2 * rd;
      if ((err = cudaMemsetAsync(ar.al_count, 0, 2 * (size_t)nb * sizeof(uint32_t), st)) != cudaSuccess ||
          (err = soft::launch_lane_resume_prepass(ar, fp32, W, st)) != cudaSuccess ||
          (err = soft::launch_prepared(c1, ar, st)) != cudaSuccess)
        return err;
      r->launches += 5;
    }
    if (wide) {  // the handed-over shots, bucketed by the event they resume at
      soft::ShotParams aw = a;
      aw.lane_round = rounds;
      aw.lane_wide_round = 1;
      aw.lane_evict = 0;
      aw.lane_hand = 0;
      aw.n_rerun_total = nullptr;  // (counted when they left the first rounds)
      aw.n_items_dev = r->d_lr + 3 + 2 * rounds;
      if ((err = cudaMemsetAsync(aw.al_count, 0, 2 * (size_t)nb * sizeof(uint32_t), st)) != cudaSuccess ||
          (err = soft::launch_lane_resume_prepass(aw, fp32, W, st)) != cudaSuccess ||
          (err = soft::launch_prepared(cw, aw, st)) != cudaSuccess)
        return err;
      r->launches += 5;
    }
    if ((err = mark()) != cudaSuccess) return err;
    if (mid_pass) {
      if ((err = soft::launch_prepared(cm, c, st)) != cudaSuccess) return err;
      r->launches++;
    }
    if (two_pass) {
      if ((err = soft::launch_prepared(c2, b, st)) != cudaSuccess) return err;
      r->launches++;
    }
    return mark(two_pass);
  };
  uint64_t s0 = 0;
  const uint64_t n_full = total / chunk;
  if (use_graph && n_full >= 2) {
    // capture one full chunk plus the device-side advance of the item base, replay it
    unsigned long long zero = 0;
    if ((e = cudaMemcpyAsync(r->d_work + 3, &zero, sizeof zero, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess) {
      soft_run_free(r);
      return cuda_fail(e, "graph set-up");
    }
    const uint32_t launches_before = r->launches;
    if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
      soft_run_free(r);
      return cuda_fail(e, "cudaStreamBeginCapture");
    }
    cudaError_t ce = enqueue_chunk(0, chunk, true);
    if (ce == cudaSuccess) ce = soft::launch_advance(r->d_work + 3, chunk, st);
    e = cudaStreamEndCapture(st, &r->graph);
    if (ce != cudaSuccess || e != cudaSuccess) {
      soft_run_free(r);
      return cuda_fail(ce != cudaSuccess ? ce : e, "graph capture");
    }
    if ((e = cudaGraphInstantiate(&r->graph_exec, r->graph, 0)) != cudaSuccess) {
      soft_run_free(r);
      return cuda_fail(e, "cudaGraphInstantiate");
    }
    const uint32_t per_chunk = r->launches - launches_before + 1;  // + the advance kernel
    r->launches = launches_before;
    for (uint64_t k = 0; k < n_full; ++k) {
      if ((e = cudaGraphLaunch(r->graph_exec, st)) != cudaSuccess) {
        soft_run_free(r);
        return cuda_fail(e, "cudaGraphLaunch");
      }
      r->launches += per_chunk;
    }
    s0 = n_full * chunk;
  }
  for (; s0 < total; s0 += chunk) {
    const uint64_t cnt = std::min(chunk, total - s0);
    if ((e = enqueue_chunk(s0, cnt, false)) != cudaSuccess) {
      soft_run_free(r);
      return cuda_fail(e, "shot kernel launch");
    }
  }
  cudaEventRecord(r->ev1, st);
  *out = r;
  return SOFT_OK;
}

}  // namespace

extern "C" {

int soft_run_shots(soft_circuit *c, uint64_t n_shots, uint64_t first_shot, uint64_t seed, const soft_run_opts *opts,
                   soft_run **out) {
  if (!c || !out) return fail(SOFT_E_ARG, "null argument");
  return run_many(&c, &n_shots, &first_shot, 1, seed, opts, out);
}

int soft_run_batch(soft_circuit *const *circs, const uint64_t *n_shots, const uint64_t *first_shots, uint32_t n_circ,
                   uint64_t seed, const soft_run_opts *opts, soft_run **out) {
  return run_many(circs, n_shots, first_shots, n_circ, seed, opts, out);
}

int soft_tally_batch(soft_run *r, uint32_t index, soft_tally_t *out) {
  if (!r || !out || index >= r->n_circ) return fail(SOFT_E_ARG, "bad argument");
  unsigned long long t[5];
  cudaError_t e = cudaMemcpyAsync(t, r->d_tally + 5 * index, sizeof t, cudaMemcpyDeviceToHost, r->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
  if (e != cudaSuccess) return cuda_fail(e, "tally copy");
  double f = 0.0;
  if (r->fid_mode) {
    e = cudaMemcpyAsync(&f, r->d_fsum + index, sizeof f, cudaMemcpyDeviceToHost, r->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
    if (e != cudaSuccess) return cuda_fail(e, "fidelity sum copy");
  }
  out->shots = t[0];
  out->discarded = t[1];
  out->overflow = t[2];
  out->kept = t[3];
  out->logical_errors = t[4];
  out->sum_fidelity = f;
  out->sum_weight = r->fid_mode ? (double)t[3] : 0.0;
  return SOFT_OK;
}

int soft_tally(soft_run *r, soft_tally_t *out) {
  if (!r || !out) return fail(SOFT_E_ARG, "null argument");
  std::vector<unsigned long long> t(5 * (size_t)r->n_circ);
  cudaError_t e = cudaMemcpyAsync(t.data(), r->d_tally, t.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                  r->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
  if (e != cudaSuccess) return cuda_fail(e, "tally copy");
  uint64_t s[5] = {0, 0, 0, 0, 0};
  for (size_t i = 0; i < t.size(); ++i) s[i % 5] += t[i];
  double f = 0.0;
  if (r->fid_mode) {
    std::vector<double> fs(r->n_circ);
    e = cudaMemcpyAsync(fs.data(), r->d_fsum, fs.size() * sizeof(double), cudaMemcpyDeviceToHost, r->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
    if (e != cudaSuccess) return cuda_fail(e, "fidelity sum copy");
    for (double v : fs) f += v;
  }
  out->shots = s[0];
  out->discarded = s[1];
  out->overflow = s[2];
  out->kept = s[3];
  out->logical_errors = s[4];
  out->sum_fidelity = f;
  out->sum_weight = r->fid_mode ? (double)s[3] : 0.0;
  return SOFT_OK;
}

int soft_get_records(soft_run *r, uint64_t *host_words, size_t n_words, uint8_t *host_status, size_t n_status) {
  if (!r) return fail(SOFT_E_ARG, "null argument");
  cudaError_t e = cudaStreamSynchronize(r->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  const size_t rw = r->circs[0]->hp.rw;
  if (host_words) {
    size_t n = std::min<size_t>(n_words, r->out_limit * rw);
    if (n && (e = cudaMemcpy(host_words, r->d_records, n * sizeof(uint64_t), cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_fail(e, "records copy");
  }
  if (host_status) {
    size_t n = std::min<size_t>(n_status, r->out_limit);
    if (n && (e = cudaMemcpy(host_status, r->d_status, n, cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_fail(e, "status copy");
  }
  return SOFT_OK;
}

int soft_get_state(soft_run *r, uint64_t off, uint64_t *signs, uint64_t *keys, double *vals, size_t cap, size_t *nnz) {
  if (!r || !nnz) return fail(SOFT_E_ARG, "null argument");
  if (off >= r->st_limit) return fail(SOFT_E_ARG, "shot offset was not captured");
  cudaError_t e = cudaStreamSynchronize(r->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  uint32_t n = 0;
  if ((e = cudaMemcpy(&n, r->d_st_nnz + off, sizeof n, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "state copy");
  *nnz = n;
  if (signs && (e = cudaMemcpy(signs, r->d_st_signs + off * 4, 4 * sizeof(uint64_t), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "state copy");
  size_t m = std::min<size_t>({(size_t)n, cap, (size_t)r->st_stride});
  if (keys && m &&
      (e = cudaMemcpy(keys, r->d_st_keys + off * r->st_stride * 2, m * 2 * sizeof(uint64_t), cudaMemcpyDeviceToHost)) !=
          cudaSuccess)
    return cuda_fail(e, "state copy");
  if (vals && m &&
      (e = cudaMemcpy(vals, r->d_st_vals + off * r->st_stride * 2, m * 2 * sizeof(double), cudaMemcpyDeviceToHost)) !=
          cudaSuccess)
    return cuda_fail(e, "state copy");
  return SOFT_OK;
}

int soft_run_diagnostics(soft_run *r, uint64_t out[4]) {
  if (!r || !out) return fail(SOFT_E_ARG, "null argument");
  unsigned long long d[4];
  cudaError_t e = cudaMemcpyAsync(d, r->d_work + 4, sizeof d, cudaMemcpyDeviceToHost, r->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
  if (e != cudaSuccess) return cuda_fail(e, "diagnostics copy");
  for (int i = 0; i < 4; ++i) out[i] = d[i];
  return SOFT_OK;
}

int soft_release_workspace(void) {
  int prev = 0;
  cudaGetDevice(&prev);
  for (int d = 0; d < kMaxDevices; ++d) {
    std::lock_guard<std::mutex> lk(g_ws[d].mu);
    if (!g_ws[d].p) continue;
    cudaSetDevice(d);
    cudaFree(g_ws[d].p);
    g_ws[d].p = nullptr;
    g_ws[d].bytes = 0;
  }
  cudaSetDevice(prev);
  return SOFT_OK;
}

int soft_run_timing(soft_run *r, double *ms, uint32_t *n_launches) {
  if (!r) return fail(SOFT_E_ARG, "null argument");
  cudaError_t e = cudaEventSynchronize(r->ev1);
  if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
  float f = 0.f;
  if ((e = cudaEventElapsedTime(&f, r->ev0, r->ev1)) != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
  if (ms) *ms = (double)f;
  if (n_launches) *n_launches = r->launches;
  return SOFT_OK;
}

int soft_run_pass_timing(soft_run *r, double ms[3], uint32_t *n_chunks, uint64_t *n_rerun) {
  if (!r || !ms) return fail(SOFT_E_ARG, "null argument");
  if (r->pass_ev.empty()) return fail(SOFT_E_ARG, "run was not launched with SOFT_RUN_TIME_PASSES (or used a graph)");
  cudaError_t e = cudaEventSynchronize(r->ev1);
  if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
  ms[0] = ms[1] = ms[2] = 0.0;
  for (size_t k = 0; k + 3 < r->pass_ev.size(); k += 4)
    for (int j = 0; j < 3; ++j) {
      float f = 0.f;
      if ((e = cudaEventElapsedTime(&f, r->pass_ev[k + j], r->pass_ev[k + j + 1])) != cudaSuccess)
        return cuda_fail(e, "cudaEventElapsedTime");
      ms[j] += (double)f;
    }
  if (n_chunks) *n_chunks = (uint32_t)(r->pass_ev.size() / 4);
  if (n_rerun) {
    unsigned long long t = 0;
    if ((e = cudaMemcpy(&t, r->d_work + 8, sizeof t, cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_fail(e, "rerun count copy");
    *n_rerun = t;
  }
  return SOFT_OK;
}

}  // extern "C"
