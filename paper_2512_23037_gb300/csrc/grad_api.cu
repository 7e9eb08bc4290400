// grad_api.cu -- soft_fidelity_grad: post-selected fidelity and its gradient
// for fixed error patterns (C ABI, see include/soft.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/soft.h"
#include "adjoint.cuh"
#include "handles.h"

extern "C" int soft_fidelity_grad(soft_circuit *c, const double *theta, uint32_t n_params, uint64_t n_patterns,
                                  uint64_t first_pattern, uint64_t seed, int32_t precision, void *stream,
                                  double *d_fid, double *d_pacc, double *d_grad, uint8_t *d_status,
                                  double *d_sums) {
  if (!c || !d_fid || !d_pacc || !d_status || (n_params && (!theta || !d_grad)))
    return soft::set_error(SOFT_E_ARG, "null argument");
  if (precision != SOFT_FP64 && precision != SOFT_FP32) return soft::set_error(SOFT_E_ARG, "bad precision");
  const auto &hp = c->hp;
  if (n_params < hp.n_params) return soft::set_error(SOFT_E_ARG, "theta shorter than the circuit's parameter count");
  if (n_patterns == 0) return SOFT_OK;
  const int fp32 = precision == SOFT_FP32;
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return soft::set_error(SOFT_E_CUDA, "cudaSetDevice failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // coefficients a I + b Z for this parameter vector: Rz(s theta_k) = cos(s theta_k/2) I - i sin(s theta_k/2) Z
  std::vector<soft::Coef> coefs(hp.coefs);
  for (size_t k = 0; k < coefs.size(); ++k) {
    const int32_t cp = hp.coef_param[k];
    if (cp < 0) continue;
    const double ang = ((cp & 1) ? -1.0 : 1.0) * theta[cp >> 1];
    const double cr = std::cos(0.5 * ang), si = -std::sin(0.5 * ang);
    coefs[k] = soft::Coef{cr, 0.0, 0.0, si, (float)cr, 0.0f, 0.0f, (float)si};
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  const uint32_t wpb = soft::grad_warps_per_block();
  uint64_t blocks = (uint64_t)(sms > 0 ? sms : 1) * soft::grad_blocks_per_sm();
  blocks = std::min<uint64_t>(blocks, (n_patterns + wpb - 1) / wpb);
  const size_t stride = soft::grad_tape_bytes(fp32, hp.W, hp.n_rot, (uint32_t)hp.ev.size());
  // workspace kept in the handle between calls; the tape grows to the largest launch seen
  const size_t tape_need = stride * blocks * wpb;
  if (!c->d_gcoef && (e = cudaMalloc(&c->d_gcoef, std::max<size_t>(1, coefs.size()) * sizeof(soft::Coef))) != cudaSuccess)
    return soft::set_error(e == cudaErrorMemoryAllocation ? SOFT_E_OOM : SOFT_E_CUDA, "device allocation failed");
  if (!c->d_gnext && (e = cudaMalloc(&c->d_gnext, sizeof(unsigned long long))) != cudaSuccess)
    return soft::set_error(e == cudaErrorMemoryAllocation ? SOFT_E_OOM : SOFT_E_CUDA, "device allocation failed");
  if (c->gtape_bytes < tape_need) {
    cudaFree(c->d_gtape);
    c->d_gtape = nullptr;
    c->gtape_bytes = 0;
    if ((e = cudaMalloc(&c->d_gtape, tape_need)) != cudaSuccess)
      return soft::set_error(e == cudaErrorMemoryAllocation ? SOFT_E_OOM : SOFT_E_CUDA, "device allocation failed");
    c->gtape_bytes = tape_need;
  }
  // shared noiseless prefix: one tape slot, (events + 1) snapshots, the stop index
  const size_t snap_stride = soft::grad_prefix_stride(fp32, hp.W, hp.rw);
  const size_t snap_off = (stride + 255) & ~(size_t)255;
  const size_t stop_off = (snap_off + (hp.ev.size() + 1) * snap_stride + 255) & ~(size_t)255;
  const size_t prefix_need = stop_off + 256;
  if (c->gprefix_bytes < prefix_need) {
    cudaFree(c->d_gprefix);
    c->d_gprefix = nullptr;
    c->gprefix_bytes = 0;
    if ((e = cudaMalloc(&c->d_gprefix, prefix_need)) != cudaSuccess)
      return soft::set_error(e == cudaErrorMemoryAllocation ? SOFT_E_OOM : SOFT_E_CUDA, "device allocation failed");
    c->gprefix_bytes = prefix_need;
  }
  // wide rerun (maps above 32 entries): list of up to n_patterns offsets, two counters, and
  // one shared-memory-map tape per block (SMs x 2 blocks of one warp)
  const uint32_t wide_blocks = (uint32_t)(sms > 0 ? sms : 1) * 2;
  const size_t wstride = soft::grad_wide_tape_bytes(fp32, hp.W, hp.n_rot, (uint32_t)hp.ev.size());
  const size_t list_bytes = ((size_t)std::min<uint64_t>(n_patterns, 0xFFFFFFFFull) * 4 + 255) & ~(size_t)255;
  const size_t wide_need = 256 + list_bytes + (size_t)wide_blocks * wstride;
  if (c->gwide_bytes < wide_need) {
    cudaFree(c->d_gwide);
    c->d_gwide = nullptr;
    c->gwide_bytes = 0;
    if ((e = cudaMalloc(&c->d_gwide, wide_need)) != cudaSuccess)
      return soft::set_error(e == cudaErrorMemoryAllocation ? SOFT_E_OOM : SOFT_E_CUDA, "device allocation failed");
    c->gwide_bytes = wide_need;
  }
  if ((e = cudaMemsetAsync(c->d_gwide, 0, 256, st)) != cudaSuccess)
    return soft::set_error(SOFT_E_CUDA, "memset failed");
  soft::Coef *d_coef = c->d_gcoef;
  unsigned long long *d_next = c->d_gnext;
  unsigned char *d_tape = c->d_gtape;
  if ((!coefs.empty() && (e = cudaMemcpyAsync(d_coef, coefs.data(), coefs.size() * sizeof(soft::Coef),
                                              cudaMemcpyHostToDevice, st)) != cudaSuccess) ||
      (e = cudaMemsetAsync(d_next, 0, sizeof(unsigned long long), st)) != cudaSuccess ||
      (d_sums && (e = cudaMemsetAsync(d_sums, 0, 3 * sizeof(double), st)) != cudaSuccess)) {
    return soft::set_error(SOFT_E_CUDA, "upload failed");
  }
  soft::GradParams p{};
  p.ev = c->d_ev;
  p.coef = d_coef;
  p.cb = c->d_cb;
  p.sites = c->d_sites;
  p.thr = c->d_thr;
  p.n_events = (uint32_t)hp.ev.size();
  p.n_sites = hp.n_sites;
  p.rw = hp.rw;
  p.n_rot = hp.n_rot;
  p.n_params = n_params;
  p.blocks = (uint32_t)blocks;
  p.tau_rel = fp32 ? 1e-10 : 1e-20;
  p.seed = seed;
  p.first_pattern = first_pattern;
  p.n_patterns = n_patterns;
  p.next = d_next;
  p.fid = d_fid;
  p.pacc = d_pacc;
  p.grad = d_grad;
  p.status = d_status;
  p.sums = d_sums;
  p.tape = d_tape;
  p.tape_stride = stride;
  unsigned char *ptape = c->d_gprefix, *psnap = c->d_gprefix + snap_off;
  uint32_t *pstop = reinterpret_cast<uint32_t *>(c->d_gprefix + stop_off);
  p.site_ev = reinterpret_cast<const uint32_t *>(c->d_thr + hp.thr.size());
  p.thr_tab = p.site_ev + hp.site_ev.size();
  if ((e = soft::launch_grad_prefix(p, fp32, hp.W, ptape, psnap, pstop, st)) != cudaSuccess)
    return soft::set_error(SOFT_E_CUDA, "prefix kernel launch failed");
  p.wide_n = reinterpret_cast<unsigned long long *>(c->d_gwide);
  p.wide_next = p.wide_n + 1;
  p.wide_list = reinterpret_cast<uint32_t *>(c->d_gwide + 256);
  p.wide_cap = (uint32_t)std::min<uint64_t>(n_patterns, 0xFFFFFFFFull);
  p.wide_blocks = wide_blocks;
  p.wide_tape = c->d_gwide + 256 + list_bytes;
  p.wide_tape_stride = wstride;
  p.ptape = ptape;
  p.psnap = psnap;
  p.psnap_stride = snap_stride;
  p.pstop = pstop;
  if ((e = soft::launch_grad(p, fp32, hp.W, st)) != cudaSuccess)
    return soft::set_error(SOFT_E_CUDA, "gradient kernel launch failed");
  // synchronous: the host coefficient table and the handle's workspace are reused by the next call
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return soft::set_error(SOFT_E_CUDA, "gradient kernel failed");
  return SOFT_OK;
}
