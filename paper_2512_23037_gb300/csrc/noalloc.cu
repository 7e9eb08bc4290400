// noalloc.cu -- soft_run_shots_noalloc: the run entry point for callers that
// must not allocate device memory.
//
// The regular soft_run_shots carves its scratch (work counters, rerun list,
// lane-per-shot buffers) from a per-device cached workspace, which it
// allocates with cudaMalloc the first time, and again whenever a run needs a
// larger one. This variant keeps its scratch in one file-scope __device__
// array instead, sized for kNoallocMaxShots shots per call, so a call never
// allocates: the caller passes the compiled circuit and its own output
// buffers, and the library only clears the counters (cudaMemsetAsync) and
// launches the warp-per-shot kernel, every shot from the first event (no
// lane-per-shot scheduling and no shared noiseless prefix, whose buffers
// scale with the shot count; same results, lower throughput).
#include <cuda_runtime.h>

#include "../../include/soft.h"
#include "handles.h"
#include "kernels.cuh"

namespace {

constexpr uint64_t kNoallocMaxShots = 1ull << 20;
constexpr size_t kCounterBytes = 256;  // work counter, rerun counter, rerun count (padded)
constexpr size_t kScratchBytes = kCounterBytes + kNoallocMaxShots * sizeof(uint32_t);

// The scratch itself. In host code `g_noalloc_scratch` is only a host-side
// stand-in for the symbol, never a device address: the address comes from
// cudaGetSymbolAddress in the current context, taken on every call (it
// allocates nothing, and no cached address can outlive a context reset).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

int scratch_address(unsigned char **out) {
  void *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) return soft::set_error(SOFT_E_CUDA, "cudaGetSymbolAddress of the no-alloc scratch failed");
  *out = static_cast<unsigned char *>(p);
  return SOFT_OK;
}

}  // namespace

extern "C" int soft_run_shots_noalloc(soft_circuit *c, uint64_t n_shots, uint64_t first_shot, uint64_t seed,
                                      int32_t precision, void *stream, unsigned long long *d_tally, uint8_t *d_status,
                                      uint64_t *d_records) {
  if (!c || !d_tally) return soft::set_error(SOFT_E_ARG, "circuit and d_tally must not be NULL");
  if (precision != SOFT_FP64 && precision != SOFT_FP32) return soft::set_error(SOFT_E_ARG, "bad precision");
  if (n_shots > kNoallocMaxShots)
    return soft::set_error(SOFT_E_ARG, "n_shots exceeds the no-alloc limit of 1048576 shots per call");
  const auto &hp = c->hp;
  const int fp32 = precision == SOFT_FP32;
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return soft::set_error(SOFT_E_CUDA, "cudaSetDevice failed");
  // the whole map at the circuit's cap lives in one block's shared memory (the regular
  // entry point moves larger caps to a global-memory slab, which this one cannot allocate)
  int smem_optin = 0;
  if ((e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device)) != cudaSuccess)
    return soft::set_error(SOFT_E_CUDA, "cudaDeviceGetAttribute failed");
  if (soft::group_smem_bytes(fp32, hp.W, hp.cap, hp.rw) > (size_t)smem_optin - 5 * 8 * soft::kMaxCirc)
    return soft::set_error(SOFT_E_ARG, "coeff_cap too large for this entry point's shared-memory coefficient map");
  unsigned char *scratch = nullptr;
  int rc = scratch_address(&scratch);  // with the circuit's device current
  if (rc != SOFT_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned long long *work = reinterpret_cast<unsigned long long *>(scratch);
  uint32_t *rerun = reinterpret_cast<uint32_t *>(scratch + kCounterBytes);
  if ((e = cudaMemsetAsync(d_tally, 0, 5 * sizeof(unsigned long long), st)) != cudaSuccess ||
      (e = cudaMemsetAsync(work, 0, 8 * sizeof(unsigned long long), st)) != cudaSuccess)
    return soft::set_error(SOFT_E_CUDA, "cudaMemsetAsync failed");
  if (n_shots == 0) return SOFT_OK;
  const uint32_t cap = hp.cap, cap1 = cap < soft::kDefaultFirstCap ? cap : soft::kDefaultFirstCap;
  const bool two_pass = cap1 < cap;
  soft::ShotParams p{};
  p.n_circ = 1;
  soft::CircDev &d = p.circ[0];
  d = soft::circ_desc(c, fp32, false);  // the program and the gap-search index, no prefix
  d.item_begin = 0;
  d.n_shots = n_shots;
  d.first_shot = first_shot;
  d.tally = d_tally;
  d.status = d_status;
  d.records = d_records;
  d.out_limit = (d_status || d_records) ? n_shots : 0;
  p.rw_max = hp.rw;
  p.tau = fp32 ? soft::kTauFp32 : soft::kTauFp64;
  p.seed = seed;
  p.n_items = n_shots;
  p.next_item = work;
  p.rerun = rerun;
  p.rerun_cap = (uint32_t)kNoallocMaxShots;
  p.n_rerun = work + 2;
  p.diag = work + 4;
  p.cap = cap1;
  p.small_pass = two_pass ? 1 : 0;
  if ((e = soft::launch_shots(p, fp32, hp.W, 32u, 0, st, nullptr)) != cudaSuccess)
    return soft::set_error(SOFT_E_CUDA, "shot kernel launch failed");
  if (two_pass) {
    soft::ShotParams q = p;
    q.cap = cap;
    q.small_pass = 0;
    q.list = rerun;
    q.n_items_dev = work + 2;
    q.next_item = work + 1;
    if ((e = soft::launch_shots(q, fp32, hp.W, 32u, 0, st, nullptr)) != cudaSuccess)
      return soft::set_error(SOFT_E_CUDA, "rerun kernel launch failed");
  }
  return SOFT_OK;
}
