// pf_device.cuh -- small device helpers shared by the kernel translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "pf_internal.h"
#include "pf_model.cuh"

namespace pf {

// Storage codecs.  FP64 / FP32 store populations as they are.  The 16-bit
// forms store each population as its offset from w_i M_o, with M_o the lagged
// moment of the site that holds it (phi for h, psi for g, C for s; kept in
// FP32), so that only the small non-rest part is rounded to 16 bits; the NS
// populations, which are small already, are stored scaled by 2^12.  FP16
// also scales the offsets by 2^14 (exact): its narrow exponent range would
// otherwise put the tiny offsets of a quiet bulk among the subnormals, where
// every site rounds them the same way and the conserved totals drift.
template <typename S>
struct Codec {
  static constexpr bool kOffset = false;
  static constexpr float kOffScale = 1.0f;
  template <typename R>
  __device__ __forceinline__ static R dec(S v) { return static_cast<R>(v); }
  template <typename R>
  __device__ __forceinline__ static S enc(R v) { return static_cast<S>(v); }
};
template <>
struct Codec<__half> {
  static constexpr bool kOffset = true;
  static constexpr float kOffScale = 16384.0f;
  template <typename R>
  __device__ __forceinline__ static R dec(__half v) { return __half2float(v); }
  template <typename R>
  __device__ __forceinline__ static __half enc(R v) { return __float2half_rn(v); }
};
template <>
struct Codec<__nv_bfloat16> {
  static constexpr bool kOffset = true;
  static constexpr float kOffScale = 1.0f;
  template <typename R>
  __device__ __forceinline__ static R dec(__nv_bfloat16 v) { return __bfloat162float(v); }
  template <typename R>
  __device__ __forceinline__ static __nv_bfloat16 enc(R v) { return __float2bfloat16_rn(v); }
};
constexpr float kNSScale = 4096.0f;      // NS populations x 2^12 in the 16-bit forms
constexpr float kNSInvScale = 1.0f / 4096.0f;


template <typename R, typename S, typename I>
__device__ __forceinline__ R ld(const S* __restrict__ p, I i) {
  return Codec<S>::template dec<R>(__ldg(p + i));
}

template <typename S, typename R, typename I>
__device__ __forceinline__ void st(S* __restrict__ p, I i, R v) {
  p[i] = Codec<S>::template enc<R>(v);
}

// Reciprocal and reciprocal square root: IEEE in FP64; in FP32 the hardware
// approximations (relative error a few 1e-7), far inside the FP32 tolerance.
__device__ __forceinline__ double frcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float frcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double frsqrt(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float frsqrt(float x) { return rsqrtf(x); }

// Plane k of a plane-major buffer: a warp-uniform base pointer, so that one
// per-thread element offset serves every plane of a site.
template <typename T>
__device__ __forceinline__ const T* plane(const T* p, int k, unsigned ps) {
  return p + (size_t)k * ps;
}
template <typename T>
__device__ __forceinline__ T* plane(T* p, int k, unsigned ps) {
  return p + (size_t)k * ps;
}

// Weights of the D2Q9 / D2Q5 lattices in the compute type.
template <typename R>
__device__ __forceinline__ R w9(int i) {
  return i == 0 ? R(4.0 / 9.0) : (i < 5 ? R(1.0 / 9.0) : R(1.0 / 36.0));
}
template <typename R>
__device__ __forceinline__ R w5(int i) {
  return i == 0 ? R(1.0 / 3.0) : R(1.0 / 6.0);
}

// Physical value <-> stored value of one population.  kind: 0 NS (scaled in
// the 16-bit forms), 1 offset from w M_o (the caller passes w M_o).
template <typename S, typename R, typename I>
__device__ __forceinline__ R pop_ns(const S* __restrict__ p, I i) {
  if constexpr (Codec<S>::kOffset) return ld<R>(p, i) * R(kNSInvScale);
  else return ld<R>(p, i);
}
template <typename S, typename R, typename I>
__device__ __forceinline__ void st_ns(S* __restrict__ p, I i, R v) {
  if constexpr (Codec<S>::kOffset) st(p, i, v * R(kNSScale));
  else st(p, i, v);
}
// Offset-stored value <-> population (wm = w_i M_o; unused by FP64/FP32).
template <typename S, typename R>
__device__ __forceinline__ R dec_off(S v, R wm) {
  const R raw = Codec<S>::template dec<R>(v);
  if constexpr (!Codec<S>::kOffset) return raw;
  else if constexpr (Codec<S>::kOffScale == 1.0f) return wm + raw;
  else return raw * R(1.0f / Codec<S>::kOffScale) + wm;
}
template <typename S, typename R>
__device__ __forceinline__ S enc_off(R v, R wm) {
  if constexpr (!Codec<S>::kOffset) return Codec<S>::template enc<R>(v);
  else if constexpr (Codec<S>::kOffScale == 1.0f) return Codec<S>::template enc<R>(v - wm);
  else return Codec<S>::template enc<R>((v - wm) * R(Codec<S>::kOffScale));
}
template <typename S, typename R, typename I>
__device__ __forceinline__ R pop_off(const S* __restrict__ p, I i, R wm) {
  return dec_off<S, R>(__ldg(p + i), wm);
}
template <typename S, typename R, typename I>
__device__ __forceinline__ void st_off(S* __restrict__ p, I i, R v, R wm) {
  p[i] = enc_off<S, R>(v, wm);
}
// Same value as st_off(p, i, v, w * M), with the weight w a compile-time
// lattice weight: in FP16 the scale folds into one FMA per population,
// v * 2^14 - (w * 2^14) * M, and (w * 2^14) * M is shared by every population
// of the same weight class.  Scaling by a power of two commutes with rounding,
// so the stored bits equal those of (v - w M) * 2^14.
template <typename S, typename R, typename I>
__device__ __forceinline__ void st_off_w(S* __restrict__ p, I i, R v, R w, R M) {
  if constexpr (Codec<S>::kOffset && Codec<S>::kOffScale != 1.0f) {
    constexpr R sc = R(Codec<S>::kOffScale);
    p[i] = Codec<S>::template enc<R>(fma(v, sc, -((w * sc) * M)));
  } else {
    p[i] = enc_off<S, R>(v, w * M);
  }
}

// Compensated (Neumaier) accumulation: the zeroth moments phi, psi, C are sums
// of 5 or 9 populations of similar size; in FP32 plain summation loses up to
// ~8 ulp(phi), which the W_phi^2-weighted Laplacian in mu_phi then amplifies.
template <typename R>
struct CSum {
  R s = R(0), c = R(0);
  // Fast2Sum: the first term added (the rest population, weight 1/3 or 4/9)
  // is the largest, so |s| >= |v| holds for the later terms.
  __device__ __forceinline__ void add(R v) {
    const R t = s + v;
    c += (s - t) + v;
    s = t;
  }
  __device__ __forceinline__ R value() const { return s + c; }
};

__device__ __forceinline__ int wrapi(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}

}  // namespace pf
