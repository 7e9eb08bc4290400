// handles.h -- library-internal definition of the circuit handle and the
// numeric constants every run entry point shares.
#pragma once
#include <cstdint>

#include "../../include/soft.h"
#include "compile.h"
#include "program.h"

namespace soft {
constexpr double kTauFp64 = 1e-20;  // prune |v|^2 below this (FP64 coefficients)
constexpr double kTauFp32 = 1e-10;  // FP32 coefficients: well above FP32 cancellation residue
constexpr uint32_t kDefaultFirstCap = 64;
// Records `msg` for soft_last_error() on this thread and returns `code`.
int set_error(int code, const char *msg);
}  // namespace soft

struct soft_circuit {
  soft::HostProgram hp;
  int device = 0;
  void *d_ev = nullptr;  // Ev<W> array, W = hp.W
  soft::Coef *d_coef = nullptr;
  soft::CaseB *d_cb = nullptr;
  soft::Site *d_sites = nullptr;
  uint64_t *d_thr = nullptr;
  uint64_t bytes = 0;
  // the noiseless run's snapshot table per precision (index 0 FP64, 1 FP32),
  // built at compile time; traj_stop = last valid event
  unsigned char *d_traj[2] = {nullptr, nullptr};
  uint32_t *d_stop = nullptr;  // where the noiseless runs report their stop events (6 words)
  uint32_t traj_stop[2] = {0, 0};
  uint32_t traj_fid_stop[2] = {0, 0};
  uint32_t traj_max_n[2] = {0, 0};  // largest map of the recorded noiseless run
  uint32_t traj_max_d[2] = {0, 0};  // largest affine dimension of its maps (0xFF: above 5)
  uint32_t traj_stride[2] = {0, 0};
  // fidelity-gradient workspace, kept between calls (they are synchronous):
  // per-parameter coefficient table, work counter, per-warp tapes
  soft::Coef *d_gcoef = nullptr;
  unsigned long long *d_gnext = nullptr;
  unsigned char *d_gtape = nullptr;
  size_t gtape_bytes = 0;
  unsigned char *d_gprefix = nullptr;  // shared noiseless prefix: tape, snapshots, stop index
  size_t gprefix_bytes = 0;
  unsigned char *d_gwide = nullptr;    // wide rerun: list, counters, tapes
  size_t gwide_bytes = 0;
};

namespace soft {
struct CircDev;
// A launch's descriptor of compiled circuit c: its program, noise tables and
// the gap-search index; with `prefix`, also its noiseless run's snapshots
// for precision fp32 (shots start at their first error).
CircDev circ_desc(const soft_circuit *c, int fp32, bool prefix);
}  // namespace soft
