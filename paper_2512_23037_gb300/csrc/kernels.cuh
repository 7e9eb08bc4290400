// kernels.cuh -- launch interface of the shot kernel (internal to libsoft).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "program.h"

namespace soft {

struct ShotParams {
  // compiled program (device)
  const void *ev;  // Ev<W>
  const Coef *coef;
  const CaseB *cb;
  const Site *sites;
  const uint64_t *thr;
  uint32_t n_events, n_sites, rw, cap;
  uint32_t hs_max;  // hash slots per group: power of two >= 4 * cap
  double tau;
  // work
  uint64_t seed, first_shot, n_items;  // shots first_shot + [0, n_items) or the list below
  const unsigned long long *n_items_dev;  // optional: item count read on the device
  const uint32_t *list;                // optional: shot offsets (relative to first_shot)
  unsigned long long *next_item;       // work counter (zeroed before launch)
  int small_pass;                      // 1: |v| > cap marks the shot for a rerun
  uint32_t *rerun;                     // rerun list (capacity n_items)
  unsigned long long *n_rerun;
  // outputs
  unsigned long long *tally;           // [5]: shots, discarded, overflow, kept, logical
  uint8_t *status;                     // per shot offset < out_limit
  uint64_t *records;                   // rw words per shot offset < out_limit
  uint64_t out_limit;
  uint64_t *st_signs;                  // 4 words per shot offset < st_limit
  uint64_t *st_keys;                   // st_stride entries x 2 words
  double *st_vals;                     // st_stride entries x (re, im)
  uint32_t *st_nnz;
  uint64_t st_limit;
  uint32_t st_stride;
  // global-memory mode (caps whose state does not fit in shared memory):
  // group g of block b uses gslab + (b * groups_per_block + g) * group_bytes
  unsigned char *gslab;
  uint32_t gslab_blocks;
  // bounds of the program arrays and of the rerun list, for the in-kernel checks
  uint32_t n_coef, n_cb, rerun_cap;
  // first failed in-kernel check: [0] count, [1] code << 32 | event, [2] shot, [3] value
  unsigned long long *diag;
};

// In-kernel check codes (a failed check ends the shot with SOFT_SHOT_ERROR
// and skips the access).
enum : uint32_t {
  CHK_HASH_SLOT = 1, CHK_STAGE = 2, CHK_SLOTS = 3, CHK_RECORD = 4, CHK_SITE = 5, CHK_COEF = 6,
  CHK_CASEB = 7, CHK_RERUN = 8, CHK_LIST = 9, CHK_PHASE = 10, CHK_NNZ = 11
};

// Bytes of a global slab for `blocks` 128-thread blocks of 32-lane groups.
size_t global_slab_bytes(int fp32, uint32_t W, uint32_t cap, uint32_t rw, uint32_t blocks);

// Bytes of shared memory one shot group needs for capacity `cap`.
size_t group_smem_bytes(int fp32, uint32_t W, uint32_t cap, uint32_t rw);

// Launch the persistent kernel. group = 8 or 32 lanes per shot.
cudaError_t launch_shots(const ShotParams &p, int fp32, uint32_t W, uint32_t group, int blocks_per_sm,
                         cudaStream_t stream, int *grid_out);

}  // namespace soft
