// pf_kernels.cu -- sm_103a kernels of one coupled lattice Boltzmann step of the
// gas-liquid-dendrite phase-field model (arXiv 2407.01651):
//   k_step      fused stream + moments + stencils + sources + four collisions
//   k_init_spec initial fields from seeds and bubbles, equilibrium populations
//   k_set_fields equilibrium populations from given macroscopic fields
//   k_reduce*   FP64 diagnostics (conservation, centroid, Laplace probe)
//   k_*_state   raw state to / from FP64
//
// Layout: structure of arrays, one plane per population / scalar, x fastest,
// periodic domains concatenated in every plane.  The step is a pull scheme with
// two state copies (ping-pong).  One CTA owns a TX x TY tile; it first builds
// phi, psi and the lagged velocity on the tile plus a one-site halo in shared
// memory (the stencils of step 3 need them at the 8 neighbours), then each
// thread streams, collides and stores its own site.
#include "pf_internal.h"
#include "pf_model.cuh"

#include <cuda_fp16.h>
#include <cuda_bf16.h>

namespace pf {

template <typename R, typename S>
__device__ __forceinline__ R ld(const S* __restrict__ p, long long i) {
  return static_cast<R>(__ldg(p + i));
}

template <typename S, typename R>
__device__ __forceinline__ void st(S* __restrict__ p, long long i, R v) {
  p[i] = static_cast<S>(v);
}

// Compensated (Neumaier) accumulation: the zeroth moments phi, psi, C are sums
// of 5 or 9 populations of similar size; in FP32 plain summation loses up to
// ~8 ulp(phi), which the W_phi^2-weighted Laplacian in mu_phi then amplifies.
template <typename R>
struct CSum {
  R s = R(0), c = R(0);
  __device__ __forceinline__ void add(R v) {
    const R t = s + v;
    c += (fabs(s) >= fabs(v)) ? ((s - t) + v) : ((v - t) + s);
    s = t;
  }
  __device__ __forceinline__ R value() const { return s + c; }
};

__device__ __forceinline__ int wrapi(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}

// Zeroth moments phi (CAC) and psi (dendrite, with the a_s^2 time stretch)
// at site (x, y) after streaming.
template <typename S, typename R>
__device__ __forceinline__ void pulled_phi_psi(const StepArgs<S, R>& a, const DomDesc& d,
                                               int x, int y, R& phi, R& psi) {
  const int nx = d.nx, ny = d.ny;
  const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
  const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
  const long long r0 = d.off + (long long)y * nx, rm = d.off + (long long)ym * nx,
                  rp = d.off + (long long)yp * nx;
  const long long src[9] = {r0 + x, r0 + xm, rm + x, r0 + xp, rp + x,
                            rm + xm, rm + xp, rp + xp, rp + xm};
  const long long ps = a.plane_stride;
  CSum<R> s;
#pragma unroll
  for (int i = 0; i < 9; ++i) s.add(ld<R>(a.in + (P_H + i) * ps, src[i]));
  phi = s.value();
  CSum<R> t;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const R gold = ld<R>(a.in + (P_GPRE + i) * ps, src[0]);
    const R gpo = ld<R>(a.in + (P_GPOST + i) * ps, src[i]);
    const R rr = ld<R>(a.in + P_RR * ps, src[i]);
    t.add(gold + (gpo - gold) * rr);
  }
  psi = t.value();
}

template <typename S, typename R>
__global__ void __launch_bounds__(256) k_step(StepArgs<S, R> a) {
  extern __shared__ unsigned char smem_raw[];
  const int TX = blockDim.x, TY = blockDim.y;
  const int SW = TX + 2, SH = TY + 2;
  R* sphi = reinterpret_cast<R*>(smem_raw);
  R* spsi = sphi + SW * SH;
  R* svx = spsi + SW * SH;
  R* svy = svx + SW * SH;
  const int tid = threadIdx.y * TX + threadIdx.x;
  const int nthr = TX * TY;
  const long long ps = a.plane_stride;
  const KParams<R>& kp = a.kp;

  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const DomDesc d = a.doms[a.tile_dom[tile]];
    const int lt = tile - d.tile0;
    const int x0 = (lt % d.tiles_x) * TX, y0 = (lt / d.tiles_x) * TY;
    const int nx = d.nx, ny = d.ny;

    // ---- phase 1: phi, psi, v_o on the tile + halo ----
    for (int i = tid; i < SW * SH; i += nthr) {
      const int gx = wrapi(x0 + (i % SW) - 1, nx), gy = wrapi(y0 + (i / SW) - 1, ny);
      R phi, psi;
      pulled_phi_psi(a, d, gx, gy, phi, psi);
      sphi[i] = phi;
      spsi[i] = psi;
      const long long site = d.off + (long long)gy * nx + gx;
      svx[i] = ld<R>(a.in + P_VXO * ps, site);
      svy[i] = ld<R>(a.in + P_VYO * ps, site);
    }
    __syncthreads();

    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x < nx && y < ny) {
      const int c = (threadIdx.y + 1) * SW + threadIdx.x + 1;
      const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
      const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
      const long long r0 = d.off + (long long)y * nx, rm = d.off + (long long)ym * nx,
                      rp = d.off + (long long)yp * nx;
      const long long src[9] = {r0 + x, r0 + xm, rm + x, r0 + xp, rp + x,
                                rm + xm, rm + xp, rp + xp, rp + xm};
      const long long site = src[0];

      // ---- stream ----
      R f[9], h[9], g[5], s[5];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        f[i] = ld<R>(a.in + (P_F + i) * ps, src[i]);
        h[i] = ld<R>(a.in + (P_H + i) * ps, src[i]);
      }
      R psio = R(0);
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        const R gold = ld<R>(a.in + (P_GPRE + i) * ps, site);
        psio += gold;
        g[i] = gold + (ld<R>(a.in + (P_GPOST + i) * ps, src[i]) - gold) *
                          ld<R>(a.in + P_RR * ps, src[i]);
        s[i] = ld<R>(a.in + (P_S + i) * ps, src[i]);
      }
      const R phi = sphi[c], psi = spsi[c];
      R C;
      {
        CSum<R> cs;
#pragma unroll
        for (int i = 0; i < 5; ++i) cs.add(s[i]);
        C = cs.value();
      }
      const R phio = ld<R>(a.in + P_PHIO * ps, site);
      const R Co = ld<R>(a.in + P_CO * ps, site);
      const R vxo = svx[c], vyo = svy[c];
      const R Qo = ld<R>(a.in + P_QO * ps, site);

      // ---- isotropic stencils, on differences from the centre value so that
      // FP32 keeps the bits of the (small) neighbour differences ----
      const R w1 = R(1.0 / 9.0), w2 = R(1.0 / 36.0);
      auto grad = [&](const R* X, R& gx, R& gy) {
        const R X0 = X[c];
        const R e = X[c + 1] - X0, w = X[c - 1] - X0, n = X[c + SW] - X0, so = X[c - SW] - X0;
        const R ne = X[c + SW + 1] - X0, nw = X[c + SW - 1] - X0;
        const R sw = X[c - SW - 1] - X0, se = X[c - SW + 1] - X0;
        gx = R(3) * (w1 * (e - w) + w2 * ((ne - sw) + (se - nw)));
        gy = R(3) * (w1 * (n - so) + w2 * ((ne - sw) + (nw - se)));
      };
      R gpx, gpy, gsx, gsy, dvxx, dvxy, dvyx, dvyy;
      grad(sphi, gpx, gpy);
      grad(spsi, gsx, gsy);
      grad(svx, dvxx, dvxy);
      grad(svy, dvyx, dvyy);
      R lphi;
      {
        const R X0 = sphi[c];
        const R ax = ((sphi[c + 1] - X0) + (sphi[c - 1] - X0)) +
                     ((sphi[c + SW] - X0) + (sphi[c - SW] - X0));
        const R dg = ((sphi[c + SW + 1] - X0) + (sphi[c - SW - 1] - X0)) +
                     ((sphi[c + SW - 1] - X0) + (sphi[c - SW + 1] - X0));
        lphi = R(6) * (w1 * ax + w2 * dg);
      }

      // ---- gas-liquid interface, forces ----
      const R rho = kp.rho_g + phi * kp.drho;
      const R grx = kp.drho * gpx, gry = kp.drho * gpy;
      const R igm = R(1) / sqrt(gpx * gpx + gpy * gpy + kp.ge2);
      const R nfx = gpx * igm, nfy = gpy * igm;
      const R opsi = R(1) + psi, ophi = R(1) - phi;
      const R mu = kp.two_bphi * phi * ophi * (R(1) - R(2) * phi) -
                   kp.two_bint * ophi * opsi * opsi - kp.Wphi2 * lphi;
      const R Fsx = kp.fs_coef * mu * gpx, Fsy = kp.fs_coef * mu * gpy;
      const R Fby = -(rho - static_cast<R>(d.rho_bar)) * kp.g;
      const R aphi = kp.kappa * phi * ophi;
      const R Dx = kp.M_phi * (gpx - aphi * nfx), Dy = kp.M_phi * (gpy - aphi * nfy);
      const R divD = (phi - phio) + vxo * gpx + vyo * gpy;
      const R Fmx = kp.drho * (divD * vxo + Dx * dvxx + Dy * dvxy);
      const R Fmy = kp.drho * (divD * vyo + Dx * dvyx + Dy * dvyy);

      // ---- NS moments, drag, pressure ----
      const R jx = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
      const R jy = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
      const R sum_nz = f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8];
      const R Fpx = Fsx + Fmx, Fpy = Fsy + Fby + Fmy;
      const R irho = R(1) / rho;
      const R vsx = (jx + R(0.5) * Fpx) * irho, vsy = (jy + R(0.5) * Fpy) * irho;
      const R chi = R(0.5) * opsi;
      const R vx = (R(1) - chi) * vsx, vy = (R(1) - chi) * vsy;
      const R Fx = Fpx - R(2) * chi * rho * vsx, Fy = Fpy - R(2) * chi * rho * vsy;
      const R v2 = vx * vx + vy * vy;
      const R p = R(0.6) * (sum_nz + R(0.5) * (vx * grx + vy * gry) - R(2.0 / 3.0) * rho * v2);
      // c_s^2/(1-w0) = 3/5; w0/(2 c_s^2) = 2/3

      // ---- dendrite geometry in the grain frame ----
      const uint8_t gid = a.grain[site];
      const double2 cs = a.grain_cs[d.grain_off + gid];
      const R ct = static_cast<R>(cs.x), sn = static_cast<R>(cs.y);
      const R eps = static_cast<R>(d.eps_s);
      const R gxr = ct * gsx + sn * gsy, gyr = -sn * gsx + ct * gsy;
      const R gm2 = gsx * gsx + gsy * gsy;
      const R smag = sqrt(gm2 + kp.ge2);
      const R ism = R(1) / smag;
      const R nxr = -gxr * ism, nyr = -gyr * ism;
      const R nx2 = nxr * nxr, ny2 = nyr * nyr;
      const R n2 = nx2 + ny2;
      const R s4 = nx2 * nx2 + ny2 * ny2;
      const R as = R(1) + eps * (R(4) * s4 - R(3) * n2 * n2);
      const R iso = s4 + R(0.75) * n2 * (R(1) - n2);
      const R pre = R(-16) * eps * as * smag;
      const R Nxr = pre * nxr * (nx2 - iso), Nyr = pre * nyr * (ny2 - iso);
      const R Nx = ct * Nxr - sn * Nyr, Ny = sn * Nxr + ct * Nyr;
      const R as2 = as * as;
      const R ias2 = R(1) / as2;

      // ---- solute and dendrite sources ----
      const R omk = R(1) - kp.k;
      const R A = R(1) + kp.k - omk * psi;
      const R iA = R(1) / A;
      const R U = (R(2) * C * iA - R(1)) / omk;
      const R omp2 = R(1) - psi * psi;
      const R Q = kp.four_bpsi * psi * omp2 - kp.two_bint * ophi * ophi * opsi -
                  kp.lam * omp2 * omp2 * (kp.theta + kp.Mcinf * U);
      const R dpsi = psi - psio;
      const R at = -kp.a_at * kp.W0 * as * (R(1) + omk * U) * dpsi / sqrt(gm2 + kp.gat2);
      const R qf = R(0.5) * (R(1) - psi);
      const R jv = kp.D * qf * C * kp.kappa * ophi;

      // ---- collisions ----
      collide_ns(f, p, rho, vx, vy, Fx, Fy, grx, gry, kp);
      {
        const R G1x = (phi * vx - phio * vxo) + R(1.0 / 3.0) * aphi * nfx;
        const R G1y = (phi * vy - phio * vyo) + R(1.0 / 3.0) * aphi * nfy;
        collide_cac(h, phi, vx, vy, G1x, G1y, kp);
      }
      R gpost[5];
      {
        const R Fs = (Q + R(0.5) * (Q - Qo)) * kp.inv_tau0;
        const R s1 = R(1) / (kp.c_s1 * as2 + R(0.5));
#pragma unroll
        for (int i = 0; i < 5; ++i) gpost[i] = g[i];
        collide_q5(gpost, psi + Fs, s1, R(0), R(0), R(-1.0 / 3.0) * Nx * ias2,
                   R(-1.0 / 3.0) * Ny * ias2);
      }
      {
        const R E = R(2) * omk * kp.D * qf * C * iA * iA;
        const R jex = C * vx - E * gsx + omk * (at * gsx + jv * nfx);
        const R jey = C * vy - E * gsy + omk * (at * gsy + jv * nfy);
        const R DC = R(2) * kp.D * qf * iA;
        const R sc = R(1) / (R(3) * DC + R(0.5));
        collide_q5(s, C, sc, jex, jey, C * vx - Co * vxo, C * vy - Co * vyo);
      }

      // ---- store ----
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        st(a.out + (P_F + i) * ps, site, f[i]);
        st(a.out + (P_H + i) * ps, site, h[i]);
      }
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        st(a.out + (P_GPRE + i) * ps, site, g[i]);
        st(a.out + (P_GPOST + i) * ps, site, gpost[i]);
        st(a.out + (P_S + i) * ps, site, s[i]);
      }
      st(a.out + P_RR * ps, site, ias2);
      st(a.out + P_PHIO * ps, site, phi);
      st(a.out + P_CO * ps, site, C);
      st(a.out + P_VXO * ps, site, vx);
      st(a.out + P_VYO * ps, site, vy);
      st(a.out + P_QO * ps, site, Q);
      if (a.fields) {
        R* fl = a.fields;
        fl[FLD_PHI * ps + site] = phi;
        fl[FLD_PSI * ps + site] = psi;
        fl[FLD_C * ps + site] = C;
        fl[FLD_U * ps + site] = U;
        fl[FLD_P * ps + site] = p;
        fl[FLD_VX * ps + site] = vx;
        fl[FLD_VY * ps + site] = vy;
        fl[FLD_MU * ps + site] = mu;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Initialisation
// ---------------------------------------------------------------------------
__device__ __forceinline__ double min_image(double d, double L) {
  d = fmod(d, L);
  if (d < -0.5 * L) d += L;
  if (d >= 0.5 * L) d -= L;
  return d;
}

// Write the equilibrium state and the fields of one site.
template <typename S, typename R>
__device__ void write_equilibrium(S* out, R* fields, long long ps, long long site, double phi_d,
                                  double psi_d, double C_d, double vx_d, double vy_d,
                                  double p_d, const KParams<R>& kp) {
  const R phi = static_cast<R>(phi_d), psi = static_cast<R>(psi_d), C = static_cast<R>(C_d);
  const R vx = static_cast<R>(vx_d), vy = static_cast<R>(vy_d), p = static_cast<R>(p_d);
  const R rho = kp.rho_g + phi * kp.drho;
  R f[9];
  feq_ns(p, rho, vx, vy, f);
  for (int i = 0; i < 9; ++i) st(out + (P_F + i) * ps, site, f[i]);
  // CAC h_eq = w_i phi (1 + 3 c.v)
  const R w[9] = {R(4.0 / 9.0), R(1.0 / 9.0), R(1.0 / 9.0), R(1.0 / 9.0), R(1.0 / 9.0),
                  R(1.0 / 36.0), R(1.0 / 36.0), R(1.0 / 36.0), R(1.0 / 36.0)};
  const R cu[9] = {R(0), vx, vy, -vx, -vy, vx + vy, -vx + vy, -vx - vy, vx - vy};
  for (int i = 0; i < 9; ++i) st(out + (P_H + i) * ps, site, w[i] * phi * (R(1) + R(3) * cu[i]));
  const R w5[5] = {R(1.0 / 3.0), R(1.0 / 6.0), R(1.0 / 6.0), R(1.0 / 6.0), R(1.0 / 6.0)};
  for (int i = 0; i < 5; ++i) {
    st(out + (P_GPRE + i) * ps, site, w5[i] * psi);
    st(out + (P_GPOST + i) * ps, site, w5[i] * psi);
    st(out + (P_S + i) * ps, site, w5[i] * C + w5[i] * R(3) * C * cu[i]);
  }
  st(out + P_RR * ps, site, R(1));
  const R omk = R(1) - kp.k;
  const R U = (R(2) * C / (R(1) + kp.k - omk * psi) - R(1)) / omk;
  const R omp2 = R(1) - psi * psi;
  const R ophi = R(1) - phi;
  const R Q = kp.four_bpsi * psi * omp2 - kp.two_bint * ophi * ophi * (R(1) + psi) -
              kp.lam * omp2 * omp2 * (kp.theta + kp.Mcinf * U);
  st(out + P_PHIO * ps, site, phi);
  st(out + P_CO * ps, site, C);
  st(out + P_VXO * ps, site, vx);
  st(out + P_VYO * ps, site, vy);
  st(out + P_QO * ps, site, Q);
  if (fields) {
    fields[FLD_PHI * ps + site] = phi;
    fields[FLD_PSI * ps + site] = psi;
    fields[FLD_C * ps + site] = C;
    fields[FLD_U * ps + site] = U;
    fields[FLD_P * ps + site] = p;
    fields[FLD_VX * ps + site] = vx;
    fields[FLD_VY * ps + site] = vy;
    fields[FLD_MU * ps + site] = R(0);
  }
}

template <typename S, typename R>
__global__ void k_init_spec(InitArgs<S, R> a) {
  const DomDesc d = a.dom;
  const long long n = (long long)d.nx * d.ny;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % d.nx), y = (int)(i / d.nx);
    double psi = -1.0, best = 0.0;
    int gid = 0;
    for (int s = 0; s < a.n_seeds; ++s) {
      const double dx = min_image((double)x - a.seeds[3 * s], (double)d.nx);
      const double dy = min_image((double)y - a.seeds[3 * s + 1], (double)d.ny);
      const double r2 = dx * dx + dy * dy;
      const double v = tanh(a.sq2bpsi * (a.R_s - sqrt(r2)) / a.W0);
      if (s == 0 || v > psi) psi = v;
      if (s == 0 || r2 < best) {
        best = r2;
        gid = s;
      }
    }
    double phi = 1.0;
    for (int b = 0; b < a.n_bub; ++b) {
      const double dx = min_image((double)x - a.bubbles[3 * b], (double)d.nx);
      const double dy = min_image((double)y - a.bubbles[3 * b + 1], (double)d.ny);
      const double v =
          0.5 + 0.5 * tanh(a.sq2bphi * (sqrt(dx * dx + dy * dy) - a.bubbles[3 * b + 2]) /
                           (2.0 * a.Wphi));
      if (b == 0 || v < phi) phi = v;
    }
    const double C = phi * (1.0 - (1.0 - a.k) * 0.5 * (1.0 + psi));
    const long long site = d.off + i;
    a.grain[site] = (uint8_t)gid;
    write_equilibrium<S, R>(a.out, a.fields, a.plane_stride, site, phi, psi, C, 0.0, 0.0, 0.0,
                            a.kp);
  }
}

template <typename S, typename R>
__global__ void k_set_fields(SetFieldsArgs<S, R> a) {
  const DomDesc d = a.dom;
  const long long n = (long long)d.nx * d.ny;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long site = d.off + i;
    const double* F = a.f6;
    write_equilibrium<S, R>(a.out, a.fields, a.plane_stride, site, F[i], F[n + i], F[2 * n + i],
                            F[3 * n + i], F[4 * n + i], F[5 * n + i], a.kp);
    a.grain[site] = a.grain_ids ? a.grain_ids[i] : (uint8_t)0;
  }
}

// ---------------------------------------------------------------------------
// Raw state / fields conversion to and from FP64.
// ---------------------------------------------------------------------------
template <typename S>
__global__ void k_state_to_f64(const S* __restrict__ in, long long ps, long long off,
                               long long n, int nplanes, double* __restrict__ out) {
  const long long tot = n * nplanes;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    const long long p = i / n, j = i % n;
    out[i] = static_cast<double>(in[p * ps + off + j]);
  }
}

template <typename S>
__global__ void k_state_from_f64(S* __restrict__ out, long long ps, long long off, long long n,
                                 int nplanes, const double* __restrict__ in) {
  const long long tot = n * nplanes;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    const long long p = i / n, j = i % n;
    out[p * ps + off + j] = static_cast<S>(in[i]);
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

// ---------------------------------------------------------------------------
// Host-side launchers (explicit instantiations for FP64 and FP32).
// ---------------------------------------------------------------------------
template <typename S, typename R>
cudaError_t launch_step(const StepArgs<S, R>& a, int tx, int ty, int grid, cudaStream_t st) {
  const size_t smem = 4 * (size_t)(tx + 2) * (ty + 2) * sizeof(R);
  k_step<S, R><<<grid, dim3(tx, ty), smem, st>>>(a);
  return cudaGetLastError();
}

template <typename S, typename R>
cudaError_t launch_init_spec(const InitArgs<S, R>& a, cudaStream_t st) {
  const long long n = (long long)a.dom.nx * a.dom.ny;
  const int grid = (int)((n + 255) / 256 < 65535 ? (n + 255) / 256 : 65535);
  k_init_spec<S, R><<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

template <typename S, typename R>
cudaError_t launch_set_fields(const SetFieldsArgs<S, R>& a, cudaStream_t st) {
  const long long n = (long long)a.dom.nx * a.dom.ny;
  const int grid = (int)((n + 255) / 256 < 65535 ? (n + 255) / 256 : 65535);
  k_set_fields<S, R><<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

template <typename S>
cudaError_t launch_state_to_f64(const S* in, long long ps, long long off, long long n,
                                int nplanes, double* out, cudaStream_t st) {
  k_state_to_f64<S><<<1024, 256, 0, st>>>(in, ps, off, n, nplanes, out);
  return cudaGetLastError();
}

template <typename S>
cudaError_t launch_state_from_f64(S* out, long long ps, long long off, long long n, int nplanes,
                                  const double* in, cudaStream_t st) {
  k_state_from_f64<S><<<1024, 256, 0, st>>>(out, ps, off, n, nplanes, in);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_fields_to_f64(const R* fields, long long ps, long long off, long long n,
                                 uint32_t mask, double* out, cudaStream_t st) {
  k_fields_to_f64<R><<<1024, 256, 0, st>>>(fields, ps, off, n, mask, out);
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
  template cudaError_t launch_step<S, R>(const StepArgs<S, R>&, int, int, int, cudaStream_t); \
  template cudaError_t launch_init_spec<S, R>(const InitArgs<S, R>&, cudaStream_t);          \
  template cudaError_t launch_set_fields<S, R>(const SetFieldsArgs<S, R>&, cudaStream_t);

PF_INST(double, double)
PF_INST(float, float)

template cudaError_t launch_state_to_f64<double>(const double*, long long, long long, long long,
                                                 int, double*, cudaStream_t);
template cudaError_t launch_state_to_f64<float>(const float*, long long, long long, long long,
                                                int, double*, cudaStream_t);
template cudaError_t launch_state_from_f64<double>(double*, long long, long long, long long, int,
                                                   const double*, cudaStream_t);
template cudaError_t launch_state_from_f64<float>(float*, long long, long long, long long, int,
                                                  const double*, cudaStream_t);
template cudaError_t launch_fields_to_f64<double>(const double*, long long, long long,
                                                  long long, uint32_t, double*, cudaStream_t);
template cudaError_t launch_fields_to_f64<float>(const float*, long long, long long, long long,
                                                 uint32_t, double*, cudaStream_t);
template cudaError_t launch_reduce<double>(const ReduceArgs<double>&, double*, double*,
                                           cudaStream_t);
template cudaError_t launch_reduce<float>(const ReduceArgs<float>&, double*, double*,
                                          cudaStream_t);

}  // namespace pf
