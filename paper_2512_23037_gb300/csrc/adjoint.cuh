// adjoint.cuh -- launch interface of the fidelity-gradient kernel (internal).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "program.h"

namespace soft {

struct GradParams {
  const void *ev;  // Ev<W>
  const Coef *coef;  // coefficients for the current parameter vector
  const CaseB *cb;
  const Site *sites;
  const uint64_t *thr;
  const uint32_t *thr_tab;  // the gap search's index (program.h; null: plain search)
  uint32_t n_events, n_sites, rw, n_rot, n_params, blocks;
  double tau_rel;  // prune |v|^2 below tau_rel times the squared norm
  uint64_t seed, first_pattern, n_patterns;
  unsigned long long *next;  // work counter (zeroed before launch)
  double *fid, *pacc, *grad;  // per pattern: F, N_acc, dF/dtheta (n_params)
  uint8_t *status;            // per pattern: 0 ok, 1 zero acceptance, 2 unsupported, 3 error
  double *sums;               // optional: sum of N_acc, sum of N_fid, count over ok patterns
  unsigned char *tape;        // one slot of tape_stride bytes per resident warp
  size_t tape_stride;
  // shared noiseless prefix (null psnap: patterns start at event 0)
  const unsigned char *ptape;  // the tracing warp's tape (same layout as a warp's)
  const unsigned char *psnap;  // state at the top of each event, psnap_stride bytes each
  size_t psnap_stride;
  const uint32_t *pstop;       // last event a pattern may start at (device)
  const uint32_t *site_ev;     // per site: the event that applies its error
  // patterns whose maps outgrow 32 entries: listed by the register pass, rerun
  // with shared-memory maps (null wide_list: none)
  uint32_t *wide_list;
  unsigned long long *wide_n, *wide_next;
  uint32_t wide_cap, wide_blocks;
  unsigned char *wide_tape;  // one slot of wide_tape_stride bytes per wide block
  size_t wide_tape_stride;
};

size_t grad_smem_per_warp(int fp32, uint32_t W, uint32_t rw);
size_t grad_tape_bytes(int fp32, uint32_t W, uint32_t n_rot, uint32_t n_events);
uint32_t grad_warps_per_block();
uint32_t grad_blocks_per_sm();  // resident blocks per SM the register budget allows
size_t grad_wide_tape_bytes(int fp32, uint32_t W, uint32_t n_rot, uint32_t n_events);
cudaError_t launch_grad(const GradParams &p, int fp32, uint32_t W, cudaStream_t st);
// Per-event snapshot bytes of the noiseless prefix, and its tracing launch (one
// warp): tape -> p.ptape (writable here), snapshots -> p.psnap, last event -> *stop.
size_t grad_prefix_stride(int fp32, uint32_t W, uint32_t rw);
cudaError_t launch_grad_prefix(const GradParams &p, int fp32, uint32_t W, unsigned char *tape, unsigned char *snaps,
                               uint32_t *stop, cudaStream_t st);

}  // namespace soft
