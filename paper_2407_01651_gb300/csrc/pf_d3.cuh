// pf_d3.cuh -- pieces shared by the 3-D z-march kernels (pf_step3d.cu,
// pf_step3f.cu): the 32 x 8 column tile with its halo ring, the D3Q7 velocity
// set, plane addressing, periodic wrapping and the isotropic D3Q19-weighted
// gradient and Laplacian over a 4-slot shared-memory ring of planes.
#pragma once
#include <cmath>

#include "pf_device.cuh"

namespace pf {
namespace d3 {

constexpr int TX = 32, TY = 8;                    // interior tile
constexpr int HX = TX + 2, HY = TY + 2;           // tile with its halo ring
constexpr int NIN = TX * TY;                      // 256 interior threads
constexpr int NHALO = HX * HY - NIN;              // 84 halo threads
constexpr int THREADS = 352;                      // 11 warps (340 used)

__device__ __forceinline__ constexpr int cx7(int i) { return i == 1 ? 1 : (i == 2 ? -1 : 0); }
__device__ __forceinline__ constexpr int cy7(int i) { return i == 3 ? 1 : (i == 4 ? -1 : 0); }
__device__ __forceinline__ constexpr int cz7(int i) { return i == 5 ? 1 : (i == 6 ? -1 : 0); }
template <typename R>
__device__ __forceinline__ R w7(int i) { return i == 0 ? R(0.25) : R(0.125); }

template <typename T>
__device__ __forceinline__ const T* pl(const T* p, int k, unsigned long long ps) { return p + (size_t)k * ps; }
template <typename T>
__device__ __forceinline__ T* pl(T* p, int k, unsigned long long ps) { return p + (size_t)k * ps; }
// 32-bit plane stride: the caller guarantees planes x sites < 2^32
template <typename T>
__device__ __forceinline__ const T* pl(const T* p, int k, unsigned ps) { return p + (unsigned)k * ps; }
template <typename T>
__device__ __forceinline__ T* pl(T* p, int k, unsigned ps) { return p + (unsigned)k * ps; }

// Index offset from coordinate v (in [0, n)) to v - c, c in {-1, 0, 1}, with one
// periodic wrap, times the axis stride. Added to a site index in the unsigned
// type I, a negative offset wraps modulo 2^bits and the sum is the exact
// neighbour index.
template <typename I>
__device__ __forceinline__ I step_off(int c, int v, int n, I stride) {
  if (c == 0) return I(0);
  const int d = c > 0 ? (v == 0 ? n - 1 : -1) : (v == n - 1 ? 1 - n : 1);
  return (I)d * stride;
}

// Hint: bring the line that holds p into L2 ahead of its use (no register is
// written, so a z-march can look two planes ahead for free).
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(__cvta_generic_to_global(p)));
}

// one step across a periodic boundary (z), and a full modulo (tile columns,
// which may lie up to a tile beyond a small domain)
__device__ __forceinline__ int wrap1(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }
__device__ __forceinline__ int wrapm(int a, int n) { a %= n; return a < 0 ? a + n : a; }

// 3 sum_q w_q c_q (X(x + c_q) - X(x)) over the 6 face (w = 1/18) and 12 edge
// (w = 1/36) neighbours of the ring column (hy, hx): the isotropic gradient.
template <typename R>
__device__ __forceinline__ void grad18(const R (*Pm)[HX], const R (*P0)[HX], const R (*Pp)[HX],
                                       int hy, int hx, R& gx, R& gy, R& gz) {
  const R X0 = P0[hy][hx];
  auto d = [&](const R (*Pl)[HX], int dx, int dy) { return Pl[hy + dy][hx + dx] - X0; };
  const R w1 = R(1.0 / 18.0), w2 = R(1.0 / 36.0);
  gx = w1 * (d(P0, 1, 0) - d(P0, -1, 0)) +
       w2 * ((d(P0, 1, 1) - d(P0, -1, 1)) + (d(P0, 1, -1) - d(P0, -1, -1)) +
             (d(Pp, 1, 0) - d(Pp, -1, 0)) + (d(Pm, 1, 0) - d(Pm, -1, 0)));
  gy = w1 * (d(P0, 0, 1) - d(P0, 0, -1)) +
       w2 * ((d(P0, 1, 1) - d(P0, 1, -1)) + (d(P0, -1, 1) - d(P0, -1, -1)) +
             (d(Pp, 0, 1) - d(Pp, 0, -1)) + (d(Pm, 0, 1) - d(Pm, 0, -1)));
  gz = w1 * (d(Pp, 0, 0) - d(Pm, 0, 0)) +
       w2 * ((d(Pp, 1, 0) - d(Pm, 1, 0)) + (d(Pp, -1, 0) - d(Pm, -1, 0)) +
             (d(Pp, 0, 1) - d(Pm, 0, 1)) + (d(Pp, 0, -1) - d(Pm, 0, -1)));
  gx *= R(3); gy *= R(3); gz *= R(3);
}

// 6 sum_q w_q (X(x + c_q) - X(x)) over the same 18 neighbours: the isotropic
// Laplacian (2 / c_s^2) sum w (X_q - X_0) with c_s^2 = 1/3.
template <typename R>
__device__ __forceinline__ R lap18(const R (*Pm)[HX], const R (*P0)[HX], const R (*Pp)[HX],
                                   int hy, int hx) {
  const R X0 = P0[hy][hx];
  auto d = [&](const R (*Pl)[HX], int dx, int dy) { return Pl[hy + dy][hx + dx] - X0; };
  const R faces = (d(P0, 1, 0) + d(P0, -1, 0)) + (d(P0, 0, 1) + d(P0, 0, -1)) +
                  (d(Pp, 0, 0) + d(Pm, 0, 0));
  const R edges = ((d(P0, 1, 1) + d(P0, -1, -1)) + (d(P0, 1, -1) + d(P0, -1, 1))) +
                  ((d(Pp, 1, 0) + d(Pm, -1, 0)) + (d(Pp, -1, 0) + d(Pm, 1, 0))) +
                  ((d(Pp, 0, 1) + d(Pm, 0, -1)) + (d(Pp, 0, -1) + d(Pm, 0, 1)));
  return R(1.0 / 3.0) * faces + R(1.0 / 6.0) * edges;
}

// Signed minimum-image offset on a periodic axis of length L.
__device__ __forceinline__ double min_image1(double d, double L) {
  if (d <= -L || d >= L) d = fmod(d, L);
  if (d < -0.5 * L) d += L;
  if (d >= 0.5 * L) d -= L;
  return d;
}

// Grain index of every site: the nearest seed (minimum image, the first seed
// on an exact tie).  seeds: n x 7 (x, y, z, quaternion); a template so that
// both 3-D translation units may instantiate it.
template <int STRIDE>
__global__ void k_grain_nearest(int nx, int ny, int nz, const double* seeds, int n_seeds,
                                int* grain) {
  const unsigned long long n = (unsigned long long)nx * ny * nz;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const double X[3] = {(double)(i % nx), (double)((i / nx) % ny),
                         (double)(i / ((unsigned long long)nx * ny))};
    const double L[3] = {(double)nx, (double)ny, (double)nz};
    int best = 0;
    double bd = 0.0;
    for (int s = 0; s < n_seeds; ++s) {
      double r2 = 0.0;
      for (int q = 0; q < 3; ++q) {
        const double d = min_image1(X[q] - seeds[STRIDE * s + q], L[q]);
        r2 += d * d;
      }
      if (s == 0 || r2 < bd) { bd = r2; best = s; }
    }
    grain[i] = best;
  }
}

// Rotation matrix (row-major) of the quaternion (w, x, y, z) after
// normalisation; false for a zero or non-finite quaternion.
inline bool quat_rows(const double* q, double R[9]) {
  for (int k = 0; k < 4; ++k)
    if (!std::isfinite(q[k])) return false;
  const double nq = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  if (!(nq > 0)) return false;
  const double w = q[0] / nq, x = q[1] / nq, y = q[2] / nq, z = q[3] / nq;
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - z * w);     R[2] = 2 * (x * z + y * w);
  R[3] = 2 * (x * y + z * w);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - x * w);
  R[6] = 2 * (x * z - y * w);     R[7] = 2 * (y * z + x * w);     R[8] = 1 - 2 * (x * x + y * y);
  return true;
}

// Sets *flag when any of the n host-supplied values staged at p is not
// finite (NaN or infinite): the field setters check their input on the
// device before it reaches the state.
static __global__ void k_flag_nonfinite(const double* __restrict__ p, long long n,
                                        unsigned int* flag) {
  bool bad = false;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    bad |= !isfinite(p[i]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1u);
}

}  // namespace d3
}  // namespace pf
