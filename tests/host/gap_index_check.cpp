// Host check of the compiled program's gap-search index: for every U the search
// bounded by U's bucket gives the plain binary search's answer (the first gap g
// with U < thr[g], capped at the remaining sites), and thr is non-decreasing.
// Usage: gap_index_check <ops file> <n_qubits> <p> ; prints "ok <checks>" or the
// first failure.
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <iterator>
#include <random>
#include <string>
#include <vector>

#include "../../paper_2512_23037_gb300/csrc/compile.h"

static uint32_t plain(const soft::HostProgram &hp, uint64_t U, uint32_t rem) {
  uint32_t lo = 0, hi = rem;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (U < hp.thr[mid]) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

static uint32_t bounded(const soft::HostProgram &hp, uint64_t U, uint32_t rem) {
  const uint32_t b = (uint32_t)(U >> (64 - soft::kThrTabBits));
  const uint32_t t0 = hp.thr_tab[b], t1 = hp.thr_tab[b + 1];
  uint32_t lo = t0 < rem ? t0 : rem, hi = t1 < rem ? t1 : rem;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (U < hp.thr[mid]) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

int main(int argc, char **argv) {
  if (argc < 4) return 2;
  std::ifstream f(argv[1], std::ios::binary);
  std::vector<char> buf((std::istreambuf_iterator<char>(f)), std::istreambuf_iterator<char>());
  const double p = std::atof(argv[3]);
  const soft_noise nz{p, p, p, p, 0.0};
  soft::HostProgram hp;
  std::string err;
  const int rc = soft::compile_program(reinterpret_cast<const soft_op *>(buf.data()), buf.size() / sizeof(soft_op),
                                       (uint32_t)std::atoi(argv[2]), &nz, 256, hp, err);
  if (rc != 0) {
    std::printf("compile failed: %d %s\n", rc, err.c_str());
    return 1;
  }
  if (hp.thr_tab.size() != (1u << soft::kThrTabBits) + 1u) {
    std::printf("index size %zu\n", hp.thr_tab.size());
    return 1;
  }
  for (uint32_t g = 1; g < hp.n_sites; ++g)
    if (hp.thr[g] < hp.thr[g - 1]) {
      std::printf("thr decreases at %u\n", g);
      return 1;
    }
  std::mt19937_64 gen(12345);
  long checks = 0;
  auto check = [&](uint64_t U, uint32_t rem) -> bool {
    ++checks;
    if (plain(hp, U, rem) == bounded(hp, U, rem)) return true;
    std::printf("mismatch U=%llu rem=%u: %u vs %u\n", (unsigned long long)U, rem, plain(hp, U, rem),
                bounded(hp, U, rem));
    return false;
  };
  for (uint32_t rem : {hp.n_sites, hp.n_sites / 2, hp.n_sites / 7, 1u, 0u}) {
    for (int i = 0; i < 200000; ++i)
      if (!check(gen(), rem)) return 1;
    for (uint64_t b = 0; b <= (1u << soft::kThrTabBits); ++b)
      for (int d = -1; d <= 1; ++d)
        if (!check((b << (64 - soft::kThrTabBits)) + (uint64_t)(int64_t)d, rem)) return 1;
    for (uint32_t k = 0; k < hp.n_sites; ++k)
      for (int d = -1; d <= 1; ++d)
        if (!check(hp.thr[k] + (uint64_t)(int64_t)d, rem)) return 1;
  }
  std::printf("ok %ld\n", checks);
  return 0;
}
