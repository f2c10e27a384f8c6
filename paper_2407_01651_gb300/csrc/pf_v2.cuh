// pf_v2.cuh -- two-lane arithmetic for the per-site math of the step kernels.
//
// Much of one LB site update comes in pairs: x and y components of gradients,
// forces and fluxes, and the populations of the opposite-direction pairs of the
// D2Q9 and D2Q5 lattices.  V2<float> maps each pair operation onto one paired
// FP32 instruction of sm_100+ (__fadd2_rn, __fmul2_rn, __ffma2_rn), which
// halves the issue slots of that arithmetic; V2<double> is two scalar
// operations.  Every lane is an IEEE round-to-nearest operation; fma() is a
// fused multiply-add in both.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

namespace pf {

template <typename R>
struct V2 {
  R x, y;
};

// Scalar fused multiply-add under the name the pair code uses (the lane types
// add their own overloads).
__device__ __forceinline__ float fma(float a, float b, float c) { return ::fmaf(a, b, c); }
__device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }

template <typename R>
__device__ __forceinline__ V2<R> vec2(R x, R y) {
  return {x, y};
}
template <typename R>
__device__ __forceinline__ V2<R> splat(R a) {
  return {a, a};
}

template <typename R>
__device__ __forceinline__ V2<R> operator+(V2<R> a, V2<R> b) {
  return {a.x + b.x, a.y + b.y};
}
template <typename R>
__device__ __forceinline__ V2<R> operator-(V2<R> a, V2<R> b) {
  return {a.x - b.x, a.y - b.y};
}
template <typename R>
__device__ __forceinline__ V2<R> operator*(V2<R> a, V2<R> b) {
  return {a.x * b.x, a.y * b.y};
}
// a * b + c, fused
template <typename R>
__device__ __forceinline__ V2<R> fma(V2<R> a, V2<R> b, V2<R> c) {
  return {fma(a.x, b.x, c.x), fma(a.y, b.y, c.y)};
}

#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
__device__ __forceinline__ float2 f2(V2<float> a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ V2<float> v2f(float2 a) { return {a.x, a.y}; }
template <>
__device__ __forceinline__ V2<float> operator+(V2<float> a, V2<float> b) {
  return v2f(__fadd2_rn(f2(a), f2(b)));
}
// a - b as b * (-1) + a: the product is exact, so this is the rounded difference
template <>
__device__ __forceinline__ V2<float> operator-(V2<float> a, V2<float> b) {
  return v2f(__ffma2_rn(f2(b), make_float2(-1.0f, -1.0f), f2(a)));
}
template <>
__device__ __forceinline__ V2<float> operator*(V2<float> a, V2<float> b) {
  return v2f(__fmul2_rn(f2(a), f2(b)));
}
template <>
__device__ __forceinline__ V2<float> fma(V2<float> a, V2<float> b, V2<float> c) {
  return v2f(__ffma2_rn(f2(a), f2(b), f2(c)));
}
#endif

template <typename U>
struct is_v2 : std::false_type {};
template <typename T>
struct is_v2<V2<T>> : std::true_type {};

// scalar-times-pair helpers (the scalar is converted to the lane type)
template <typename T, typename U, typename = std::enable_if_t<!is_v2<U>::value>>
__device__ __forceinline__ V2<T> operator*(U s, V2<T> a) {
  return splat(T(s)) * a;
}
template <typename T, typename U, typename = std::enable_if_t<!is_v2<U>::value>>
__device__ __forceinline__ V2<T> fma(U s, V2<T> b, V2<T> c) {
  return fma(splat(T(s)), b, c);
}

}  // namespace pf
