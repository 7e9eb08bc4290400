// compile.h -- host-side circuit compiler (internal to libsoft).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/soft.h"
#include "program.h"

namespace soft {

struct HostProgram {
  uint32_t n = 0, W = 1;
  uint32_t n_records = 0, rw = 1, n_sites = 0, cap = 0;
  double pmax = 0.0;
  std::vector<Ev<2>> ev;          // events in the two-word layout (narrowed at upload when W = 1)
  std::vector<Coef> coefs;
  std::vector<int32_t> coef_param;  // per coefficient: parameter << 1 | negated, or -1 (fixed angle)
  uint32_t n_params = 0;            // 1 + largest parameter index of a parameterised RZ
  uint32_t n_rot = 0;               // ROT + ROT_DIAG events
  std::vector<CaseB> cb;
  std::vector<Site> sites;
  std::vector<uint64_t> thr;     // gap thresholds, one per site
  std::vector<uint32_t> site_ev; // per site: the first event whose site_begin exceeds it (applies its error)
  std::vector<uint32_t> thr_tab; // 2^kThrTabBits + 1 entries: the gap search's index (program.h)
  std::vector<uint64_t> fin_x;   // final X words, 2n rows x 2 words
  std::vector<uint64_t> fin_z;
  bool fid_ok = true;  // no DETECTOR at or after the first measurement an OBSERVABLE reads
};

// Returns SOFT_OK or a SOFT_E_* code with a message in `err`.
int compile_program(const soft_op *ops, size_t n_ops, uint32_t n_qubits, const soft_noise *noise, uint32_t cap,
                    HostProgram &out, std::string &err);

}  // namespace soft
