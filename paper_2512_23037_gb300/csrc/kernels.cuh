// kernels.cuh -- launch interface of the shot kernel (internal to libsoft).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "program.h"

namespace soft {

constexpr int kMaxCirc = 64;  // circuits per launch (descriptors travel in the kernel parameters)

// One compiled circuit as seen by a launch. Work items [item_begin,
// item_begin + n_shots) of the launch's global item range are this circuit's
// shots first_shot + (item - item_begin).
struct CircDev {
  const void *ev;  // Ev<W>
  const Coef *coef;
  const CaseB *cb;
  const Site *sites;
  const uint64_t *thr;
  uint32_t n_events, n_sites, rw, cap;  // cap: this circuit's coefficient cap
  uint32_t n_coef, n_cb;
  uint32_t bucket0;    // lane-per-shot scheduling: the circuit's first bucket (one per event, plus one)
  uint32_t lanes_off;  // 1: its maps outgrow a lane; its shots go straight to the warp pass (no buckets)
  uint64_t item_begin, n_shots, first_shot;
  unsigned long long *tally;  // [5]: shots, discarded, overflow, kept, logical
  double *fsum;               // fidelity mode: sum of F over kept shots (may be null)
  uint8_t *status;            // per shot offset < out_limit
  uint64_t *records;          // rw words per shot offset < out_limit
  uint64_t out_limit;
  // the noiseless run's state at the top of events [0, traj_stop] (null: none);
  // a shot starts at the event that applies its first error, or at traj_stop
  const unsigned char *traj;
  uint32_t traj_stop, traj_stride;
  uint32_t traj_fid_stop, pad_traj;  // first fidelity measurement's event (fidelity mode stops there)
  const uint32_t *site_ev;  // per site: the event that applies its error
  const uint32_t *thr_tab;  // the gap search's index, 2^kThrTabBits + 1 entries (null: plain search)
};

struct ShotParams {
  uint32_t n_circ;
  uint32_t cap;     // capacity of the on-chip map of this launch (first pass: small)
  uint32_t rw_max;  // record words reserved per group
  uint32_t hs_max;  // hash slots per group: power of two >= 4 * cap
  double tau;
  uint64_t seed;
  // work: global items item_base + [0, n_items) or item_base + list[0 .. n_items)
  uint64_t item_base, n_items;
  const unsigned long long *item_base_dev;  // optional: read on the device (graph replay)
  const unsigned long long *n_items_dev;    // optional: item count read on the device
  const uint32_t *list;
  unsigned long long *next_item;  // work counter (zeroed before launch)
  int small_pass;                 // 1: a shot whose |v| exceeds cap but not its circuit's cap is rerun
  uint32_t rerun_cap;
  uint32_t *rerun;                // rerun list of local items (capacity rerun_cap)
  unsigned long long *n_rerun;
  unsigned long long *n_rerun_total;  // reruns over all chunks of a run (may be null)
  // final GS state of circuit 0's first st_limit shots
  uint64_t *st_signs;  // 4 words per shot
  uint64_t *st_keys;   // st_stride entries x 2 words
  double *st_vals;     // st_stride entries x (re, im)
  uint32_t *st_nnz;
  uint64_t st_limit;
  uint32_t st_stride;
  // global-memory mode (caps whose state does not fit in shared memory):
  // group g of block b uses gslab + (b * groups_per_block + g) * group_bytes
  unsigned char *gslab;
  uint32_t gslab_blocks;
  uint32_t groups_per_block;  // 0 = 4 (block of 128 threads for 32-lane groups)
  // first failed in-kernel check: [0] count, [1] code << 32 | event, [2] shot, [3] value
  unsigned long long *diag;
  // fidelity mode: measurements flagged F_FIDELITY project onto +1 and each
  // kept shot adds the product of their conditional probabilities to fsum
  int fid_mode;
  // lane-per-shot scheduling of circuit 0 (lane_kernel): per item its start event;
  // bucket e = al_order[al_start[e] .. al_start[e + 1]); claims per bucket
  uint32_t *al_ev;  // per item (start event, rank in its bucket), 8-byte aligned
  uint32_t *al_order, *al_start;
  unsigned int *al_count, *al_next;
  uint32_t *al_cursor;  // per item the noise cursor after its first draw (nxt, cur, kblk, w2), 16-byte aligned
  uint32_t *al_base;    // per pre-pass block: the block's first rank in each bucket, then its first
                        // slot in the warp pass's list (al_nb + 1 words per block)
  uint32_t al_grid;     // pre-pass blocks (each bins a contiguous range of items)
  uint32_t al_nb;       // buckets over all circuits of the run
  uint32_t al_lo, al_hi;  // a lane launch's buckets [al_lo, al_hi) (circuits of one lane map size)
  // lane-per-shot rounds: a warp left with few active lanes evicts their shots to the spill
  // pool; the next round buckets them by the event they resume at and packs them into warps
  uint32_t lane_round;        // 0: shots from their start buckets; r >= 1: shots evicted before round r
  uint32_t lane_evict;        // 1: this round may evict
  uint32_t lane_hand;         // 1: a lane whose map would outgrow it hands the shot over (a spill record)
  uint32_t lane_wide;         // 1: a wide round takes the handed-over shots (records stay off the rerun list)
  uint32_t lane_wide_round;   // 1: this is the wide round (its records: the handed-over ones)
  unsigned char *sp;          // spill pool, sp_cap records (layout: lane_spill_bytes): evictions in
  uint32_t sp_cap;            // [0, sp_evict_cap), shots handed from a lane to a warp after that
  uint32_t sp_evict_cap;
  unsigned long long *lr;     // [0] eviction records taken, [1] handover records taken;
                              // round r >= 1: [2 + 2r] its first record, [3 + 2r] its count
  CircDev circ[kMaxCirc];
};

// In-kernel check codes (a failed check ends the shot with SOFT_SHOT_ERROR
// and skips the access).
enum : uint32_t {
  CHK_HASH_SLOT = 1, CHK_STAGE = 2, CHK_SLOTS = 3, CHK_RECORD = 4, CHK_SITE = 5, CHK_COEF = 6,
  CHK_CASEB = 7, CHK_RERUN = 8, CHK_LIST = 9, CHK_PHASE = 10, CHK_NNZ = 11
};

// Bytes per event of a noiseless-run snapshot table (see CircDev::traj).
size_t prefix_stride(int fp32, uint32_t W, uint32_t rw);
// Record circuit p.circ[0]'s noiseless run into `out` ((n_events + 1) snapshots);
// stop[0] receives the last valid event, stop[1] the first fidelity measurement's
// event (or n_events), stop[2] the largest map of the recorded snapshots. One
// warp; p.cap is the map capacity used.
cudaError_t launch_prefix(const ShotParams &p, int fp32, uint32_t W, unsigned char *out, uint32_t *stop,
                          cudaStream_t st);

// Bytes of shared memory one shot group needs for capacity `cap`.
size_t group_smem_bytes(int fp32, uint32_t W, uint32_t cap, uint32_t rw);

// Bytes of a global slab for `blocks` blocks of 4 32-lane groups.
size_t global_slab_bytes(int fp32, uint32_t W, uint32_t cap, uint32_t rw, uint32_t blocks);

// A resolved launch of the shot kernel (kernel, grid, block, dynamic smem).
struct LaunchCfg {
  const void *kern;
  unsigned grid, block;
  size_t smem;
};

// Lane-per-shot kernel (lanes.cu): the bucketing pre-pass (start events, bucket
// starts, order), its launch shape, and its map capacity per shot.
cudaError_t launch_lane_prepass(const ShotParams &p, cudaStream_t st);
// round r >= 1: the range of records evicted before it, then their buckets
cudaError_t launch_lane_resume_prepass(const ShotParams &p, int fp32, uint32_t W, cudaStream_t st);
size_t lane_spill_bytes(int fp32, uint32_t W, uint32_t rw, uint32_t cap);
uint32_t lane_rounds();
uint32_t lane_max_buckets();  // lane-per-shot runs hold at most this many buckets (events + 1 per circuit)
uint32_t lane_prepass_grid();  // blocks of the bucketing pre-pass (al_base holds this many rows)
// cap: the lane map's entries: lane_map_cap() for the first rounds, twice that for the wide
// round, or lane_first_cap()'s answer for circuits of larger maps
cudaError_t prepare_lanes(const ShotParams &p, int fp32, uint32_t W, int blocks_per_sm, LaunchCfg *cfg,
                          uint32_t cap);
uint32_t lane_map_cap();
// The smallest lane map (16, 32 or, with FP32 coefficients, 64 entries) that holds a circuit
// whose noiseless run's maps reach max_n entries in max_d directions; 0 if none does.
uint32_t lane_first_cap(uint32_t max_n, uint32_t max_d, int fp32);
uint32_t lane_map_dim();  // directions of a first-round lane's affine map (lane_map_cap = 2^lane_map_dim)
// After launch_prefix: the affine form of each snapshot of the run (events [0, stop[0]]),
// on the same stream; stop[3] (zeroed before) receives the largest dimension.
cudaError_t launch_snap_affine(unsigned char *traj, uint32_t n_snap, uint32_t rw, int fp32, uint32_t W,
                               uint32_t *stop, cudaStream_t st);

// Resolve the launch (sets the kernel's shared-memory attribute, queries
// occupancy). `p.hs_max` must already be hash_slots_for(p.cap). Not a stream
// operation, so it may run before a stream capture.
cudaError_t prepare_shots(const ShotParams &p, int fp32, uint32_t W, uint32_t group, int blocks_per_sm,
                          LaunchCfg *cfg);
// Launch a prepared configuration on `stream` (capturable).
cudaError_t launch_prepared(const LaunchCfg &cfg, const ShotParams &p, cudaStream_t stream);
uint32_t hash_slots_for(uint32_t cap);

// Launch the persistent kernel. group = 8 or 32 lanes per shot.
cudaError_t launch_shots(const ShotParams &p, int fp32, uint32_t W, uint32_t group, int blocks_per_sm,
                         cudaStream_t stream, int *grid_out);

// Device-side item_base += step (advances graph-replayed chunks).
cudaError_t launch_advance(unsigned long long *item_base, unsigned long long step, cudaStream_t stream);

}  // namespace soft
