// pf_kernels.cu -- sm_103a support kernels of the coupled lattice Boltzmann step
// of the gas-liquid-dendrite phase-field model (arXiv 2407.01651); the step
// itself is in pf_step.cu:
//   k_init_spec initial fields from seeds and bubbles, equilibrium populations
//   k_set_fields equilibrium populations from given macroscopic fields
//   k_reduce*   FP64 diagnostics (conservation, centroid, Laplace probe)
//   k_*_state   raw state to / from FP64
//
// Layout: structure of arrays, one plane per population / scalar, x fastest,
// periodic domains concatenated in every plane.
#include "pf_internal.h"
#include "pf_device.cuh"

#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include <algorithm>

namespace pf {

// ---------------------------------------------------------------------------
// Initialisation
// ---------------------------------------------------------------------------
// Minimum-image offset; fmod(d, L) == d whenever |d| < L, so it is only taken
// for offsets of a whole period or more.
__device__ __forceinline__ double min_image(double d, double L) {
  if (d <= -L || d >= L) d = fmod(d, L);
  if (d < -0.5 * L) d += L;
  if (d >= 0.5 * L) d -= L;
  return d;
}

// Temperature lattice of one site at equilibrium (thermal mode): H =
// c_p [theta - (c_p^s/c_p) h(psi)], e = g^eq(rho H, theta, rho H v) of
// Appendix B (with the axis base rounded as in collide_th), lagged H = H and
// the lagged dendrite source at its pointwise part Q_psi(theta) / F(U).
template <typename S, typename R>
__device__ void write_thermal(S* out, R* aout, R* fields, long long ps, long long site, R phi,
                              R psi, R U, R vx, R vy, R theta, const KParams<R>& kp) {
  const R rho = kp.rho_g + phi * kp.drho;
  const R H = kp.th_cp * (theta - kp.th_lh * (R(1) + psi));
  const R m0 = rho * H;
  const R b = round_to_multiple(theta * R(1.0 / 6.0), quantum_quarter_ulp(m0));
  const R jx = m0 * vx, jy = m0 * vy;
  const R e[5] = {m0 - R(4) * b, b + R(0.5) * jx, b + R(0.5) * jy, b - R(0.5) * jx,
                  b - R(0.5) * jy};
  for (int i = 0; i < 5; ++i) st<S, R>(out + (P_E + i) * ps, site, e[i]);
  aout[A_HO * ps + site] = H;
  const R omp2 = R(1) - psi * psi, ophi = R(1) - phi;
  const R Q = kp.four_bpsi * psi * omp2 - kp.two_bint * ophi * ophi * (R(1) + psi) -
              kp.lam * omp2 * omp2 * (theta + kp.Mcinf * U);
  const R F = kp.th_iLe + kp.Mcinf * (R(1) + (R(1) - kp.k) * U);
  aout[A_QO * ps + site] = Q / F;
  if (fields) fields[FLD_THETA * ps + site] = theta;
}

// Offset along an axis: minimum image on a periodic axis, plain otherwise.
__device__ __forceinline__ double axis_offset(double d, double L, bool periodic) {
  return periodic ? min_image(d, L) : d;
}

// Write the equilibrium state and the fields of one site.
template <typename S, typename R>
__device__ void write_equilibrium(S* out, R* aout, R* fields, long long ps, long long site,
                                  double phi_d, double psi_d, double C_d, double vx_d,
                                  double vy_d, double p_d, const KParams<R>& kp, int thermal,
                                  double theta_d) {
  const R phi = static_cast<R>(phi_d), psi = static_cast<R>(psi_d), C = static_cast<R>(C_d);
  const R vx = static_cast<R>(vx_d), vy = static_cast<R>(vy_d), p = static_cast<R>(p_d);
  const R rho = kp.rho_g + phi * kp.drho;
  R f[9];
  feq_ns(p, rho, vx, vy, f);
  // CAC h_eq = w_i phi (1 + 3 c.v); dendrite w_i psi; solute w_i C (1 + 3 c.v)
  const R cu[9] = {R(0), vx, vy, -vx, -vy, vx + vy, -vx + vy, -vx - vy, vx - vy};
  for (int i = 0; i < 9; ++i) {
    st_ns<S, R>(out + (P_F + i) * ps, site, f[i]);
    st_off<S, R>(out + (P_H + i) * ps, site, w9<R>(i) * phi * (R(1) + R(3) * cu[i]),
                 w9<R>(i) * phi);
  }
  for (int i = 0; i < 5; ++i) {
    st_off<S, R>(out + (P_GPRE + i) * ps, site, w5<R>(i) * psi, w5<R>(i) * psi);
    st_off<S, R>(out + (P_GPOST + i) * ps, site, w5<R>(i) * psi, w5<R>(i) * psi);
    st_off<S, R>(out + (P_S + i) * ps, site, w5<R>(i) * C * (R(1) + R(3) * cu[i]),
                 w5<R>(i) * C);
  }
  const R omk = R(1) - kp.k;
  const R U = (R(2) * C / (R(1) + kp.k - omk * psi) - R(1)) / omk;
  const R omp2 = R(1) - psi * psi;
  const R ophi = R(1) - phi;
  const R Q = kp.four_bpsi * psi * omp2 - kp.two_bint * ophi * ophi * (R(1) + psi) -
              kp.lam * omp2 * omp2 * (kp.theta + kp.Mcinf * U);
  aout[A_RR * ps + site] = R(1);
  aout[A_PHIO * ps + site] = phi;
  aout[A_CO * ps + site] = C;
  aout[A_VXO * ps + site] = vx;
  aout[A_VYO * ps + site] = vy;
  aout[A_QO * ps + site] = Q;
  aout[A_PSIO * ps + site] = psi;
  if (fields) {
    fields[FLD_PHI * ps + site] = phi;
    fields[FLD_PSI * ps + site] = psi;
    fields[FLD_C * ps + site] = C;
    fields[FLD_U * ps + site] = U;
    fields[FLD_P * ps + site] = p;
    fields[FLD_VX * ps + site] = vx;
    fields[FLD_VY * ps + site] = vy;
    fields[FLD_MU * ps + site] = R(0);
    fields[FLD_THETA * ps + site] = kp.theta;
  }
  if (thermal) write_thermal<S, R>(out, aout, fields, ps, site, phi, psi, U, vx, vy,
                                   static_cast<R>(theta_d), kp);
}

template <typename S, typename R>
__global__ void k_init_spec(InitArgs<S, R> a) {
  const DomDesc d = a.dom;
  const long long n = (long long)d.nx * d.ny;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % d.nx), y = (int)(i / d.nx);
    // tanh of an argument beyond +-30 is exactly +-1 in FP64, so objects that
    // far away are not evaluated (identical result, ~100x fewer tanh).
    const double seed_far = a.R_s + 30.0 * a.W0 / a.sq2bpsi;
    double psi = -1.0, best = 0.0;
    int gid = 0;
    for (int s = 0; s < a.n_seeds; ++s) {
      const double dx = axis_offset((double)x - a.seeds[3 * s], (double)d.nx, d.bc[0] == 0);
      const double dy = axis_offset((double)y - a.seeds[3 * s + 1], (double)d.ny, d.bc[2] == 0);
      const double r2 = dx * dx + dy * dy;
      const double v = r2 > seed_far * seed_far
                           ? -1.0
                           : tanh(a.sq2bpsi * (a.R_s - sqrt(r2)) / a.W0);
      if (s == 0 || v > psi) psi = v;
      if (s == 0 || r2 < best) {
        best = r2;
        gid = s;
      }
    }
    double phi = 1.0;
    for (int b = 0; b < a.n_bub; ++b) {
      const double dx = axis_offset((double)x - a.bubbles[3 * b], (double)d.nx, d.bc[0] == 0);
      const double dy = axis_offset((double)y - a.bubbles[3 * b + 1], (double)d.ny, d.bc[2] == 0);
      const double r2 = dx * dx + dy * dy;
      const double far = a.bubbles[3 * b + 2] + 60.0 * a.Wphi / a.sq2bphi;
      const double v =
          r2 > far * far ? 1.0
                         : 0.5 + 0.5 * tanh(a.sq2bphi * (sqrt(r2) - a.bubbles[3 * b + 2]) /
                                            (2.0 * a.Wphi));
      if (b == 0 || v < phi) phi = v;
    }
    const double C = phi * (1.0 - (1.0 - a.k) * 0.5 * (1.0 + psi));
    const long long site = d.off + i;
    a.grain[site] = (uint8_t)gid;
    write_equilibrium<S, R>(a.out, a.aout, a.fields, a.plane_stride, site, phi, psi, C, 0.0,
                            0.0, 0.0, a.kp, a.thermal, a.theta0);
  }
}

template <typename S, typename R>
__global__ void k_set_fields(SetFieldsArgs<S, R> a) {
  const DomDesc d = a.dom;
  const long long n = (long long)d.nx * d.ny;
  const long long hi = a.i1 > 0 ? a.i1 : n;
  for (long long i = a.i0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < hi;
       i += (long long)gridDim.x * blockDim.x) {
    const long long site = d.off + i;
    const double* F = a.f6;
    const double v0 = F[i], v1 = F[n + i], v2 = F[2 * n + i], v3 = F[3 * n + i],
                 v4 = F[4 * n + i], v5 = F[5 * n + i];
    // the host reads this bit after the launch and rejects the fields
    if (!isfinite(v0) || !isfinite(v1) || !isfinite(v2) || !isfinite(v3) || !isfinite(v4) ||
        !isfinite(v5))
      atomicOr(a.err, ERR_NONFINITE_INPUT);
    write_equilibrium<S, R>(a.out, a.aout, a.fields, a.plane_stride, site, v0, v1, v2, v3, v4,
                            v5, a.kp, a.thermal, a.theta0);
    a.grain[site] = a.grain_ids ? a.grain_ids[i] : (uint8_t)0;
  }
}

// Thermal mode: the temperature lattice of a domain at equilibrium for a given
// theta field, with phi, psi, U and v taken from the field planes (the state
// written by the last initialisation).
template <typename S, typename R>
__global__ void k_set_temperature(S* out, R* aout, R* fields, long long ps, DomDesc d,
                                  const double* __restrict__ theta, KParams<R> kp) {
  const long long n = (long long)d.nx * d.ny;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long site = d.off + i;
    write_thermal<S, R>(out, aout, fields, ps, site, fields[FLD_PHI * ps + site],
                        fields[FLD_PSI * ps + site], fields[FLD_U * ps + site],
                        fields[FLD_VX * ps + site], fields[FLD_VY * ps + site],
                        static_cast<R>(theta[i]), kp);
  }
}

// ---------------------------------------------------------------------------
// Raw state / fields conversion to and from FP64.
// ---------------------------------------------------------------------------
// Raw state of one site <-> the 39 physical planes (f, h, g_pre, g_post, r,
// s, phi, C, vx, vy, Q_psi), decoding / encoding the storage form.  In the
// offset forms a population stored at site x is relative to the lagged
// moment of x itself.
// Thermal mode adds planes 39..43 (e_0..e_4) and 44 (H of the last step).
template <typename S, typename R>
__global__ void k_state_to_f64(const S* __restrict__ pin, const R* __restrict__ ain, long long ps,
                               long long off, long long n, double* __restrict__ out,
                               int thermal) {
  constexpr bool offs = Codec<S>::kOffset;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x) {
    const long long s = off + j;
    const R phio = ain[A_PHIO * ps + s], Co = ain[A_CO * ps + s];
    const R psio = offs ? ain[A_PSIO * ps + s] : R(0);
    for (int i = 0; i < 9; ++i) {
      out[(0 + i) * n + j] = (double)pop_ns<S, R>(pin + (P_F + i) * ps, s);
      out[(9 + i) * n + j] = (double)pop_off<S, R>(pin + (P_H + i) * ps, s, w9<R>(i) * phio);
    }
    for (int i = 0; i < 5; ++i) {
      out[(18 + i) * n + j] = (double)pop_off<S, R>(pin + (P_GPRE + i) * ps, s, w5<R>(i) * psio);
      out[(23 + i) * n + j] = (double)pop_off<S, R>(pin + (P_GPOST + i) * ps, s, w5<R>(i) * psio);
      out[(29 + i) * n + j] = (double)pop_off<S, R>(pin + (P_S + i) * ps, s, w5<R>(i) * Co);
    }
    out[28 * n + j] = (double)ain[A_RR * ps + s];
    out[34 * n + j] = (double)phio;
    out[35 * n + j] = (double)Co;
    out[36 * n + j] = (double)ain[A_VXO * ps + s];
    out[37 * n + j] = (double)ain[A_VYO * ps + s];
    out[38 * n + j] = (double)ain[A_QO * ps + s];
    if (thermal) {
      for (int i = 0; i < 5; ++i) out[(39 + i) * n + j] = (double)ld<R>(pin + (P_E + i) * ps, s);
      out[44 * n + j] = (double)ain[A_HO * ps + s];
    }
  }
}

template <typename S, typename R>
__global__ void k_state_from_f64(S* __restrict__ pout, R* __restrict__ aout, long long ps,
                                 long long off, long long n, const double* __restrict__ in,
                                 int thermal) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x) {
    const long long s = off + j;
    const R phio = (R)in[34 * n + j], Co = (R)in[35 * n + j];
    R psio = R(0);  // psi of the last step = sum of g_pre
    for (int i = 0; i < 5; ++i) psio += (R)in[(18 + i) * n + j];
    for (int i = 0; i < 9; ++i) {
      st_ns<S, R>(pout + (P_F + i) * ps, s, (R)in[(0 + i) * n + j]);
      st_off<S, R>(pout + (P_H + i) * ps, s, (R)in[(9 + i) * n + j], w9<R>(i) * phio);
    }
    for (int i = 0; i < 5; ++i) {
      st_off<S, R>(pout + (P_GPRE + i) * ps, s, (R)in[(18 + i) * n + j], w5<R>(i) * psio);
      st_off<S, R>(pout + (P_GPOST + i) * ps, s, (R)in[(23 + i) * n + j], w5<R>(i) * psio);
      st_off<S, R>(pout + (P_S + i) * ps, s, (R)in[(29 + i) * n + j], w5<R>(i) * Co);
    }
    aout[A_RR * ps + s] = (R)in[28 * n + j];
    aout[A_PHIO * ps + s] = phio;
    aout[A_CO * ps + s] = Co;
    aout[A_VXO * ps + s] = (R)in[36 * n + j];
    aout[A_VYO * ps + s] = (R)in[37 * n + j];
    aout[A_QO * ps + s] = (R)in[38 * n + j];
    aout[A_PSIO * ps + s] = psio;
    if (thermal) {
      for (int i = 0; i < 5; ++i) st<S, R>(pout + (P_E + i) * ps, s, (R)in[(39 + i) * n + j]);
      aout[A_HO * ps + s] = (R)in[44 * n + j];
    }
  }
}

template <typename R>
__global__ void k_fields_to_f64(const R* __restrict__ fields, long long ps, long long off,
                                long long n, uint32_t mask, double* __restrict__ out) {
  int sel[N_FIELDS];
  int ns = 0;
  for (int f = 0; f < N_FIELDS; ++f)
    if (mask & (1u << f)) sel[ns++] = f;
  const long long tot = n * ns;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    const long long q = i / n, j = i % n;
    out[i] = static_cast<double>(fields[sel[q] * ps + off + j]);
  }
}

// ---------------------------------------------------------------------------
// FP64 reductions: each block writes NDIAG partials, one block sums them in a
// fixed order (deterministic).
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_reduce_partial(ReduceArgs<R> a, double* __restrict__ partial) {
  double acc[NDIAG];
  for (int q = 0; q < NDIAG; ++q) acc[q] = 0.0;
  const DomDesc d = a.dom;
  const long long n = (long long)d.nx * d.ny;
  const long long ps = a.plane_stride;
  const double Rin = a.Rp - 2.0 * a.W, Rout = a.Rp + 4.0 * a.W;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long site = d.off + i;
    const double phi = (double)a.fields[FLD_PHI * ps + site];
    const double psi = (double)a.fields[FLD_PSI * ps + site];
    const double C = (double)a.fields[FLD_C * ps + site];
    const double p = (double)a.fields[FLD_P * ps + site];
    const double vx = (double)a.fields[FLD_VX * ps + site];
    const double vy = (double)a.fields[FLD_VY * ps + site];
    const double x = (double)(i % d.nx), y = (double)(i / d.nx);
    acc[0] += phi;
    acc[1] += C;
    acc[2] += 0.5 * (1.0 + psi);
    acc[3] += 1.0 - phi;
    acc[4] += x * (1.0 - phi);
    acc[5] += y * (1.0 - phi);
    if (a.probe) {
      const double dx = min_image(x - a.xc, (double)d.nx), dy = min_image(y - a.yc, (double)d.ny);
      const double r = sqrt(dx * dx + dy * dy);
      if (r < Rin) { acc[6] += p; acc[7] += 1.0; }
      if (r > Rout) { acc[8] += p; acc[9] += 1.0; }
    }
    const double vm = sqrt(vx * vx + vy * vy);
    if (vm > acc[10]) acc[10] = vm;
    if (!isfinite(phi) || !isfinite(psi) || !isfinite(C) || !isfinite(p) || !isfinite(vx) ||
        !isfinite(vy))
      acc[11] += 1.0;
  }
  __shared__ double sh[NDIAG][256];
  for (int q = 0; q < NDIAG; ++q) sh[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int stride = blockDim.x / 2; stride > 0; stride >>= 1) {
    if ((int)threadIdx.x < stride)
      for (int q = 0; q < NDIAG; ++q) {
        if (q == 10)
          sh[q][threadIdx.x] = fmax(sh[q][threadIdx.x], sh[q][threadIdx.x + stride]);
        else
          sh[q][threadIdx.x] += sh[q][threadIdx.x + stride];
      }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < NDIAG; ++q) partial[blockIdx.x * NDIAG + q] = sh[q][0];
}

// Thermal totals (FP64): sum over sites of the five temperature populations
// (the total of rho H), sum theta, sum psi; fixed-order partials as above.
template <typename S, typename R>
__global__ void k_reduce_thermal_partial(const S* __restrict__ pop, const R* __restrict__ fields,
                                         long long ps, DomDesc d, double* __restrict__ partial) {
  double acc[3] = {0.0, 0.0, 0.0};
  const long long n = (long long)d.nx * d.ny;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long site = d.off + i;
    double se = 0.0;
    for (int q = 0; q < 5; ++q) se += (double)ld<R>(pop + (P_E + q) * ps, site);
    acc[0] += se;
    acc[1] += (double)fields[FLD_THETA * ps + site];
    acc[2] += (double)fields[FLD_PSI * ps + site];
  }
  __shared__ double sh[3][256];
  for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int stride = blockDim.x / 2; stride > 0; stride >>= 1) {
    if ((int)threadIdx.x < stride)
      for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + stride];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) partial[blockIdx.x * 3 + q] = sh[q][0];
}

__global__ void k_reduce_thermal_final(const double* __restrict__ partial, int nblocks,
                                       double* __restrict__ out) {
  const int q = threadIdx.x;
  if (q >= 3) return;
  double acc = 0.0;
  for (int b = 0; b < nblocks; ++b) acc += partial[b * 3 + q];
  out[q] = acc;
}

__global__ void k_reduce_final(const double* __restrict__ partial, int nblocks,
                               double* __restrict__ out) {
  const int q = threadIdx.x;
  if (q >= NDIAG) return;
  double acc = 0.0;
  for (int b = 0; b < nblocks; ++b) {
    const double v = partial[b * NDIAG + q];
    acc = (q == 10) ? fmax(acc, v) : acc + v;
  }
  out[q] = acc;
}

// Fields [j0, j1) of a domain to FP64 (the band form of k_fields_to_f64).
template <typename R>
__global__ void k_fields_to_f64_range(const R* __restrict__ fields, long long ps, long long off,
                                      long long n, long long j0, long long j1, uint32_t mask,
                                      double* __restrict__ out) {
  int sel[N_FIELDS];
  int ns = 0;
  for (int f = 0; f < N_FIELDS; ++f)
    if (mask & (1u << f)) sel[ns++] = f;
  const long long m = j1 - j0, tot = m * ns;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    const long long q = i / m, j = j0 + i % m;
    out[q * n + j] = static_cast<double>(fields[sel[q] * ps + off + j]);
  }
}

// FP64 sum of n values rounded to R, with the thread order and block tree of
// the phi sum in k_reduce_partial / k_reduce_final (REDUCE_BLOCKS x 256).
template <typename R>
__global__ void k_sum_as_partial(const double* __restrict__ v, long long n,
                                 double* __restrict__ partial) {
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    acc += (double)static_cast<R>(v[i]);
  __shared__ double sh[256];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int stride = blockDim.x / 2; stride > 0; stride >>= 1) {
    if ((int)threadIdx.x < stride) sh[threadIdx.x] += sh[threadIdx.x + stride];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void k_sum_final(const double* __restrict__ partial, int nblocks,
                            double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double acc = 0.0;
  for (int b = 0; b < nblocks; ++b) acc = acc + partial[b];
  *out = acc;
}

__global__ void k_set_rho_bar(DomDesc* doms, int dom, const double* __restrict__ sum, double n,
                              double rho_g, double drho) {
  if (blockIdx.x == 0 && threadIdx.x == 0) doms[dom].rho_bar = fma(*sum / n, drho, rho_g);
}

// ---------------------------------------------------------------------------
// Host-side launchers (explicit instantiations for FP64 and FP32).
// ---------------------------------------------------------------------------
template <typename S, typename R>
cudaError_t launch_init_spec(const InitArgs<S, R>& a, cudaStream_t st) {
  const long long n = (long long)a.dom.nx * a.dom.ny;
  const int grid = (int)((n + 255) / 256 < 65535 ? (n + 255) / 256 : 65535);
  k_init_spec<S, R><<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

// Sets *flag when any of n staged host values is not finite; run before the
// values reach the state.
__global__ void k_flag_nonfinite(const double* __restrict__ p, long long n,
                                 unsigned int* flag) {
  bool bad = false;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    bad |= !isfinite(p[i]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1u);
}

cudaError_t launch_flag_nonfinite(const double* p, long long n, unsigned int* flag,
                                  cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  const int grid = (int)std::min<long long>((n + 255) / 256, 1024);
  k_flag_nonfinite<<<std::max(grid, 1), 256, 0, st>>>(p, n, flag);
  return cudaGetLastError();
}

template <typename S, typename R>
cudaError_t launch_set_fields(const SetFieldsArgs<S, R>& a, cudaStream_t st) {
  const long long n = (a.i1 > 0 ? a.i1 : (long long)a.dom.nx * a.dom.ny) - a.i0;
  if (n <= 0) return cudaSuccess;
  const int grid = (int)((n + 255) / 256 < 65535 ? (n + 255) / 256 : 65535);
  k_set_fields<S, R><<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

template <typename S, typename R>
cudaError_t launch_state_to_f64(const S* pin, const R* ain, long long ps, long long off,
                                long long n, double* out, int thermal, cudaStream_t st) {
  k_state_to_f64<S, R><<<1024, 256, 0, st>>>(pin, ain, ps, off, n, out, thermal);
  return cudaGetLastError();
}

template <typename S, typename R>
cudaError_t launch_state_from_f64(S* pout, R* aout, long long ps, long long off, long long n,
                                  const double* in, int thermal, cudaStream_t st) {
  k_state_from_f64<S, R><<<1024, 256, 0, st>>>(pout, aout, ps, off, n, in, thermal);
  return cudaGetLastError();
}

template <typename S, typename R>
cudaError_t launch_set_temperature(S* out, R* aout, R* fields, long long ps, const DomDesc& d,
                                   const double* theta, const KParams<R>& kp, cudaStream_t st) {
  const long long n = (long long)d.nx * d.ny;
  const int grid = (int)((n + 255) / 256 < 65535 ? (n + 255) / 256 : 65535);
  k_set_temperature<S, R><<<grid, 256, 0, st>>>(out, aout, fields, ps, d, theta, kp);
  return cudaGetLastError();
}

template <typename S, typename R>
cudaError_t launch_reduce_thermal(const S* pop, const R* fields, long long ps, const DomDesc& d,
                                  double* partial, double* out, cudaStream_t st) {
  k_reduce_thermal_partial<S, R><<<REDUCE_BLOCKS, 256, 0, st>>>(pop, fields, ps, d, partial);
  k_reduce_thermal_final<<<1, 32, 0, st>>>(partial, REDUCE_BLOCKS, out);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_fields_to_f64(const R* fields, long long ps, long long off, long long n,
                                 uint32_t mask, double* out, cudaStream_t st) {
  k_fields_to_f64<R><<<1024, 256, 0, st>>>(fields, ps, off, n, mask, out);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_fields_to_f64_range(const R* fields, long long ps, long long off, long long n,
                                       long long j0, long long j1, uint32_t mask, double* out,
                                       cudaStream_t st) {
  if (j1 <= j0) return cudaSuccess;
  k_fields_to_f64_range<R><<<1024, 256, 0, st>>>(fields, ps, off, n, j0, j1, mask, out);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_sum_as(const double* phi, long long n, double* partial, double* out,
                          cudaStream_t st) {
  k_sum_as_partial<R><<<REDUCE_BLOCKS, 256, 0, st>>>(phi, n, partial);
  k_sum_final<<<1, 32, 0, st>>>(partial, REDUCE_BLOCKS, out);
  return cudaGetLastError();
}

cudaError_t launch_set_rho_bar(DomDesc* doms, int dom, const double* sum, double n, double rho_g,
                               double drho, cudaStream_t st) {
  k_set_rho_bar<<<1, 32, 0, st>>>(doms, dom, sum, n, rho_g, drho);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_reduce(const ReduceArgs<R>& a, double* partial, double* out,
                          cudaStream_t st) {
  k_reduce_partial<R><<<REDUCE_BLOCKS, 256, 0, st>>>(a, partial);
  k_reduce_final<<<1, 32, 0, st>>>(partial, REDUCE_BLOCKS, out);
  return cudaGetLastError();
}

#define PF_INST(S, R)                                                                      \
  template cudaError_t launch_init_spec<S, R>(const InitArgs<S, R>&, cudaStream_t);          \
  template cudaError_t launch_set_fields<S, R>(const SetFieldsArgs<S, R>&, cudaStream_t);    \
  template cudaError_t launch_state_to_f64<S, R>(const S*, const R*, long long, long long,   \
                                                 long long, double*, int, cudaStream_t);     \
  template cudaError_t launch_state_from_f64<S, R>(S*, R*, long long, long long, long long,  \
                                                   const double*, int, cudaStream_t);        \
  template cudaError_t launch_set_temperature<S, R>(S*, R*, R*, long long, const DomDesc&,   \
                                                    const double*, const KParams<R>&,        \
                                                    cudaStream_t);                           \
  template cudaError_t launch_reduce_thermal<S, R>(const S*, const R*, long long,            \
                                                   const DomDesc&, double*, double*,         \
                                                   cudaStream_t);

PF_INST(double, double)
PF_INST(float, float)
PF_INST(__half, float)
PF_INST(__nv_bfloat16, float)

template cudaError_t launch_fields_to_f64<double>(const double*, long long, long long,
                                                  long long, uint32_t, double*, cudaStream_t);
template cudaError_t launch_fields_to_f64<float>(const float*, long long, long long, long long,
                                                 uint32_t, double*, cudaStream_t);
template cudaError_t launch_fields_to_f64_range<double>(const double*, long long, long long,
                                                        long long, long long, long long, uint32_t,
                                                        double*, cudaStream_t);
template cudaError_t launch_fields_to_f64_range<float>(const float*, long long, long long,
                                                       long long, long long, long long, uint32_t,
                                                       double*, cudaStream_t);
template cudaError_t launch_sum_as<double>(const double*, long long, double*, double*,
                                           cudaStream_t);
template cudaError_t launch_sum_as<float>(const double*, long long, double*, double*,
                                          cudaStream_t);
template cudaError_t launch_reduce<double>(const ReduceArgs<double>&, double*, double*,
                                           cudaStream_t);
template cudaError_t launch_reduce<float>(const ReduceArgs<float>&, double*, double*,
                                          cudaStream_t);

}  // namespace pf
