// device_common.cuh -- device helpers shared by the shot kernel and the
// adjoint kernel (complex arithmetic, packed keys, Philox4x32-10).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace soft {
namespace dev {

template <typename R>
struct Cx {
  R x, y;
};
// Real arithmetic with fixed rounding: explicit round-to-nearest intrinsics, so that no
// product is contracted into a fused multiply-add differently in different kernels (the
// noiseless-run snapshots come from one kernel and must equal, bit for bit, what the shot
// kernels compute on the same events). A negated operand of a product or a fused
// multiply-add is an instruction modifier, not an operation.
__device__ __forceinline__ double fmar(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fmar(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double mulr(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mulr(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double addr(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float addr(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double subr(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float subr(float a, float b) { return __fsub_rn(a, b); }
// a b: each component one product and one fused multiply-add
template <typename R>
__device__ __forceinline__ Cx<R> cmul(Cx<R> a, Cx<R> b) {
  return {fmar(a.x, b.x, mulr(-a.y, b.y)), fmar(a.x, b.y, mulr(a.y, b.x))};
}
template <typename R>
__device__ __forceinline__ Cx<R> cadd(Cx<R> a, Cx<R> b) {
  return {addr(a.x, b.x), addr(a.y, b.y)};
}
template <typename R>
__device__ __forceinline__ Cx<R> csub(Cx<R> a, Cx<R> b) {
  return {subr(a.x, b.x), subr(a.y, b.y)};
}
template <typename R>
__device__ __forceinline__ Cx<R> cscale(Cx<R> a, R s) {
  return {mulr(a.x, s), mulr(a.y, s)};
}
// a v + b w as one chain of fused multiply-adds per component
template <typename R>
__device__ __forceinline__ Cx<R> cmad2(Cx<R> a, Cx<R> v, Cx<R> b, Cx<R> w) {
  return {fmar(a.x, v.x, fmar(-a.y, v.y, fmar(b.x, w.x, mulr(-b.y, w.y)))),
          fmar(a.x, v.y, fmar(a.y, v.x, fmar(b.x, w.y, mulr(b.y, w.x))))};
}
// -x by flipping the sign bit, for a negated value that is stored or selected rather than
// fed to an arithmetic instruction. For FP64 the flip is an explicit 32-bit xor of the
// high word in inline PTX: written as a plain negation (or a bit flip the compiler
// recognizes as one) it becomes a DADD on GB300's narrow FP64 pipe, which measured
// 0.91 G DADDs per 2^22 shots of the FP64 lane kernel, 22 % of its time.
__device__ __forceinline__ double negr(double x) {
  int hi = __double2hiint(x);
  const int lo = __double2loint(x);
  asm("xor.b32 %0, %0, 0x80000000;" : "+r"(hi));
  return __hiloint2double(hi, lo);
}
__device__ __forceinline__ float negr(float x) { return -x; }
// v * i^e
template <typename R>
__device__ __forceinline__ Cx<R> ipow(Cx<R> v, uint32_t e) {
  Cx<R> r = (e & 1u) ? Cx<R>{negr(v.y), v.x} : v;
  if (e & 2u) r = {negr(r.x), negr(r.y)};
  return r;
}
template <typename R>
__device__ __forceinline__ R norm2(Cx<R> v) {
  return fmar(v.x, v.x, mulr(v.y, v.y));
}

// The pruning test |v|^2 < tau, decided exactly as the norm computed in R decides it.
// FP64: when both |re| and |im| lie below sqrt(tau/2) (1 - 2^-18), or either lies above
// sqrt(tau) (1 + 2^-18), integer compares of their high words settle it (the computed
// norm's rounding cannot cross tau there); only values in that narrow band compute the
// norm on the FP64 pipe, GB300's narrowest.
template <typename R>
struct PruneTest {
  R tau;
  uint32_t lo = 0, hi = 0;  // high words of the two bounds above (FP64)
  __device__ explicit PruneTest(double t) : tau((R)t) {
    if (sizeof(R) == 8) {
      lo = (uint32_t)((unsigned long long)__double_as_longlong(sqrt(0.5 * t) * (1.0 - 0x1p-18)) >> 32);
      hi = (uint32_t)((unsigned long long)__double_as_longlong(sqrt(t) * (1.0 + 0x1p-18)) >> 32);
    }
  }
  __device__ __forceinline__ bool small(Cx<R> v) const {
    if (sizeof(R) == 4) return norm2(v) < tau;
    const uint32_t hx = (uint32_t)((unsigned long long)__double_as_longlong((double)v.x) >> 32) & 0x7FFFFFFFu;
    const uint32_t hy = (uint32_t)((unsigned long long)__double_as_longlong((double)v.y) >> 32) & 0x7FFFFFFFu;
    if (hx > hi || hy > hi) return false;
    if (hx < lo && hy < lo) return true;
    return norm2(v) < tau;
  }
};
template <typename R>
__device__ __forceinline__ double norm2d(Cx<R> v) {
  const double a = (double)v.x, b = (double)v.y;
  return __fma_rn(a, a, __dmul_rn(b, b));
}
// |v|^2 as it enters the FP64 probability sums of a measurement: computed in FP64 for FP64
// maps; for FP32 maps computed in FP32 (its rounding, 2^-24 relative, is that of the
// coefficients themselves) and widened, which keeps two conversions and two FP64 products
// per entry off GB300's narrow FP64 pipe (w42 FP32: 622 -> 660 M shots/s). The sums stay FP64.
template <typename R>
__device__ __forceinline__ double pnorm(Cx<R> v) {
  if (sizeof(R) == 4) return (double)norm2(v);
  return norm2d(v);
}

template <int W>
struct Key {
  uint64_t w[W];
};
template <int W>
__device__ __forceinline__ Key<W> kxor(const Key<W> &a, const uint64_t *b) {
  Key<W> r;
#pragma unroll
  for (int i = 0; i < W; ++i) r.w[i] = a.w[i] ^ b[i];
  return r;
}
template <int W>
__device__ __forceinline__ uint32_t kpar(const Key<W> &a, const uint64_t *b) {
  uint32_t t = 0;
#pragma unroll
  for (int i = 0; i < W; ++i) t += __popcll(a.w[i] & b[i]);
  return t & 1u;
}
template <int W>
__device__ __forceinline__ bool keq(const Key<W> &a, const Key<W> &b) {
  bool e = true;
#pragma unroll
  for (int i = 0; i < W; ++i) e = e && (a.w[i] == b.w[i]);
  return e;
}
// word (i >> 6) of a W-word vector without dynamic register indexing
template <int W>
__device__ __forceinline__ uint64_t word_of(const uint64_t *a, uint32_t i) {
  return (W == 1 || (i >> 6) == 0u) ? a[0] : a[W - 1];
}
template <int W>
__device__ __forceinline__ uint32_t kbit(const Key<W> &a, uint32_t i) {
  return (uint32_t)((word_of<W>(a.w, i) >> (i & 63)) & 1ull);
}
template <int W>
__device__ __forceinline__ uint32_t khash(const Key<W> &a) {
  uint64_t h = a.w[0];
  if (W == 2) h ^= a.w[W - 1] * 0xC2B2AE3D27D4EB4Full;
  h *= 0x9E3779B97F4A7C15ull;
  return (uint32_t)(h >> 32);
}
template <int W>
__device__ __forceinline__ uint32_t wpar(const uint64_t *a, const uint64_t *b) {
  uint32_t t = 0;
#pragma unroll
  for (int i = 0; i < W; ++i) t += __popcll(a[i] & b[i]);
  return t & 1u;
}
template <int W>
__device__ __forceinline__ uint32_t wbit(const uint64_t *a, uint32_t i) {
  return (uint32_t)((word_of<W>(a, i) >> (i & 63)) & 1ull);
}
template <int W>
__device__ __forceinline__ void wflip(uint64_t *a, uint32_t i) {
#pragma unroll
  for (int w = 0; w < W; ++w)
    if ((int)(i >> 6) == w) a[w] ^= 1ull << (i & 63);
}

// Philox4x32-10, counter (shot_lo, shot_hi, stream, index), key = seed. Rolled: the
// round loop is not unrolled, for kernels whose instruction fetch limits them (the lane
// kernel: 3.6 % faster on w42 FP32); same values.
template <bool Rolled = false>
__device__ __forceinline__ uint4 philox(uint64_t seed, uint64_t shot, uint32_t stream, uint32_t idx) {
  uint32_t c0 = (uint32_t)shot, c1 = (uint32_t)(shot >> 32), c2 = stream, c3 = idx;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll (Rolled ? 1 : 10)
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return make_uint4(c0, c1, c2, c3);
}



}  // namespace dev
}  // namespace soft
