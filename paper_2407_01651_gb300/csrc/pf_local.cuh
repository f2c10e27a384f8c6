// pf_local.cuh -- the pointwise part of one coupled LB step at one site
// (interface geometry, forces and sources, the four MRT collisions) and its
// hand-written reverse-mode derivative (discrete adjoint), for the
// gas-liquid-dendrite phase-field model of arXiv 2407.01651.
//
// Inputs of the site (LocalIn): the streamed populations, the stencils of phi,
// psi and of the lagged velocity, and the lagged scalars of the site.  Outputs
// (LocalOut): the 39 state values the step stores at the site.  The forward is
// the arithmetic of the step kernel; local_reverse recomputes it and
// back-propagates output adjoints to input adjoints and to the three
// differentiable parameters (eps_s, Omega, sigma).
//
// Host-and-device code: the same header is compiled into the CUDA kernels and
// into a host harness that checks the reverse against central differences.
#pragma once

#include <cmath>

#if defined(__CUDACC__)
#define PF_HD __host__ __device__ __forceinline__
#else
#define PF_HD inline
#endif

namespace pf {
namespace local {

using std::sqrt;

template <typename R>
struct Coef {
  R rho_g, drho, ge2, gat2, kappa, fs_coef, Wphi2, M_phi;
  R two_bphi, two_bint, four_bpsi, lam, theta, Mcinf, inv_tau0, c_s1, W0, a_at, k, D, g;
  R s_e, s_eps, s_q, s_nu, s_phi;
  R eps, ct, sn, rho_bar;  // per site: anisotropy, grain frame, buoyancy reference
};

template <typename R>
struct In {
  R f[9], h[9], g[5], s[5];     // streamed populations
  R psio;                       // psi of the previous step
  R gpx, gpy, lphi;             // grad phi, lap phi
  R gsx, gsy;                   // grad psi
  R dvxx, dvxy, dvyx, dvyy;     // d_x vx_o, d_y vx_o, d_x vy_o, d_y vy_o
  R phio, Co, Qo, vxo, vyo;     // lagged scalars of the site
};

template <typename R>
struct Out {
  R f[9], h[9], gpre[5], gpost[5], rr, s[5], phi, C, vx, vy, Q;
  // diagnostics (not state)
  R U, p, mu;
};

// Parameter adjoints: d/d eps_s, d/d Omega, d/d sigma.
template <typename R>
struct ParGrad {
  R eps, Omega, sigma;
};

// --- D2Q9 moment transforms (Lallemand-Luo) ---------------------------------
template <typename R>
PF_HD void m9(const R f[9], R m[9]) {
  const R a14 = f[1] + f[2] + f[3] + f[4];
  const R a58 = f[5] + f[6] + f[7] + f[8];
  m[0] = f[0] + a14 + a58;
  m[1] = R(-4) * f[0] - a14 + R(2) * a58;
  m[2] = R(4) * f[0] - R(2) * a14 + a58;
  const R dx = f[5] - f[6] - f[7] + f[8];
  const R dy = f[5] + f[6] - f[7] - f[8];
  m[3] = f[1] - f[3] + dx;
  m[4] = R(-2) * (f[1] - f[3]) + dx;
  m[5] = f[2] - f[4] + dy;
  m[6] = R(-2) * (f[2] - f[4]) + dy;
  m[7] = f[1] - f[2] + f[3] - f[4];
  m[8] = f[5] - f[6] + f[7] - f[8];
}

// f = M^T m (no scaling); M^-1 m = M^T diag(1/|row|^2) m.
template <typename R>
PF_HD void mt9(const R m[9], R f[9]) {
  const R a = m[0], b = m[1], c = m[2], d = m[3], e = m[4], fy = m[5], gy = m[6];
  const R h = m[7], k = m[8];
  const R axis = a - b - R(2) * c;
  const R diag = a + R(2) * b + c;
  f[0] = a - R(4) * b + R(4) * c;
  f[1] = axis + d - R(2) * e + h;
  f[2] = axis + fy - R(2) * gy - h;
  f[3] = axis - d + R(2) * e + h;
  f[4] = axis - fy + R(2) * gy - h;
  f[5] = diag + d + e + fy + gy + k;
  f[6] = diag - d - e + fy + gy - k;
  f[7] = diag - d - e - fy - gy + k;
  f[8] = diag + d + e - fy - gy - k;
}

template <typename R>
PF_HD void scale_d9(R m[9]) {
  const R inv[9] = {R(1.0 / 9.0), R(1.0 / 36.0), R(1.0 / 36.0), R(1.0 / 6.0), R(1.0 / 12.0),
                    R(1.0 / 6.0), R(1.0 / 12.0), R(0.25), R(0.25)};
  for (int i = 0; i < 9; ++i) m[i] *= inv[i];
}

// --- forward ------------------------------------------------------------------
template <typename R>
PF_HD void forward(const In<R>& in, const Coef<R>& c, Out<R>& o) {
  R phi = R(0), psi = R(0), C = R(0);
  for (int i = 0; i < 9; ++i) phi += in.h[i];
  for (int i = 0; i < 5; ++i) psi += in.g[i];
  for (int i = 0; i < 5; ++i) C += in.s[i];
  const R gpx = in.gpx, gpy = in.gpy, gsx = in.gsx, gsy = in.gsy;

  const R rho = c.rho_g + phi * c.drho;
  const R grx = c.drho * gpx, gry = c.drho * gpy;
  const R igm = R(1) / sqrt(gpx * gpx + gpy * gpy + c.ge2);
  const R nfx = gpx * igm, nfy = gpy * igm;
  const R opsi = R(1) + psi, ophi = R(1) - phi;
  const R mu = c.two_bphi * phi * ophi * (R(1) - R(2) * phi) - c.two_bint * ophi * opsi * opsi -
               c.Wphi2 * in.lphi;
  const R Fsx = c.fs_coef * mu * gpx, Fsy = c.fs_coef * mu * gpy;
  const R Fby = -(rho - c.rho_bar) * c.g;
  const R aphi = c.kappa * phi * ophi;
  const R Dx = c.M_phi * (gpx - aphi * nfx), Dy = c.M_phi * (gpy - aphi * nfy);
  const R divD = (phi - in.phio) + in.vxo * gpx + in.vyo * gpy;
  const R Fmx = c.drho * (divD * in.vxo + Dx * in.dvxx + Dy * in.dvxy);
  const R Fmy = c.drho * (divD * in.vyo + Dx * in.dvyx + Dy * in.dvyy);
  const R* f = in.f;
  const R jx = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
  const R jy = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
  const R snz = f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8];
  const R Fpx = Fsx + Fmx, Fpy = Fsy + Fby + Fmy;
  const R irho = R(1) / rho;
  const R vsx = (jx + R(0.5) * Fpx) * irho, vsy = (jy + R(0.5) * Fpy) * irho;
  const R chi = R(0.5) * opsi;
  const R vx = (R(1) - chi) * vsx, vy = (R(1) - chi) * vsy;
  const R Fx = Fpx - R(2) * chi * rho * vsx, Fy = Fpy - R(2) * chi * rho * vsy;
  const R v2 = vx * vx + vy * vy;
  const R p = R(0.6) * (snz + R(0.5) * (vx * grx + vy * gry) - R(2.0 / 3.0) * rho * v2);

  const R gxr = c.ct * gsx + c.sn * gsy, gyr = -c.sn * gsx + c.ct * gsy;
  const R gm2 = gsx * gsx + gsy * gsy;
  const R smag = sqrt(gm2 + c.ge2);
  const R ism = R(1) / smag;
  const R nxr = -gxr * ism, nyr = -gyr * ism;
  const R nx2 = nxr * nxr, ny2 = nyr * nyr;
  const R n2 = nx2 + ny2;
  const R s4 = nx2 * nx2 + ny2 * ny2;
  const R as = R(1) + c.eps * (R(4) * s4 - R(3) * n2 * n2);
  const R iso = s4 + R(0.75) * n2 * (R(1) - n2);
  const R pre = R(-16) * c.eps * as * smag;
  const R Nxr = pre * nxr * (nx2 - iso), Nyr = pre * nyr * (ny2 - iso);
  const R Nx = c.ct * Nxr - c.sn * Nyr, Ny = c.sn * Nxr + c.ct * Nyr;
  const R as2 = as * as;
  const R ias2 = R(1) / as2;

  const R omk = R(1) - c.k;
  const R A = R(1) + c.k - omk * psi;
  const R iA = R(1) / A;
  const R U = (R(2) * C * iA - R(1)) / omk;
  const R omp2 = R(1) - psi * psi;
  const R drive = c.theta + c.Mcinf * U;
  const R Q = c.four_bpsi * psi * omp2 - c.two_bint * ophi * ophi * opsi -
              c.lam * omp2 * omp2 * drive;
  const R dpsi = psi - in.psio;
  const R sat = sqrt(gm2 + c.gat2);
  const R at = -c.a_at * c.W0 * as * (R(1) + omk * U) * dpsi / sat;
  const R qf = R(0.5) * (R(1) - psi);
  const R jv = c.D * qf * C * c.kappa * ophi;

  // NS collision
  {
    R m[9], ms[9];
    m9(f, m);
    const R vg = vx * grx + vy * gry;
    const R rv2 = rho * v2;
    const R hn = R(1) - R(0.5) * c.s_nu;
    ms[0] = R(0.5) * vg;
    ms[1] = m[1] - c.s_e * (m[1] - (R(6) * p + R(3) * rv2));
    ms[2] = m[2] - c.s_eps * (m[2] - (R(-9) * p - R(3) * rv2)) - (R(1) - R(0.5) * c.s_eps) * vg;
    ms[3] = rho * vx + R(0.5) * Fx;
    ms[4] = m[4] - c.s_q * (m[4] + rho * vx) - (R(1) - R(0.5) * c.s_q) * Fx;
    ms[5] = rho * vy + R(0.5) * Fy;
    ms[6] = m[6] - c.s_q * (m[6] + rho * vy) - (R(1) - R(0.5) * c.s_q) * Fy;
    ms[7] = m[7] - c.s_nu * (m[7] - rho * (vx * vx - vy * vy)) +
            hn * R(2.0 / 3.0) * (vx * grx - vy * gry);
    ms[8] = m[8] - c.s_nu * (m[8] - rho * vx * vy) + hn * R(1.0 / 3.0) * (vx * gry + vy * grx);
    scale_d9(ms);
    mt9(ms, o.f);
  }
  // CAC collision
  {
    const R* h = in.h;
    const R hjx = h[1] - h[3] + h[5] - h[6] - h[7] + h[8];
    const R hjy = h[2] - h[4] + h[5] + h[6] - h[7] - h[8];
    const R G1x = (phi * vx - in.phio * in.vxo) + R(1.0 / 3.0) * aphi * nfx;
    const R G1y = (phi * vy - in.phio * in.vyo) + R(1.0 / 3.0) * aphi * nfy;
    const R hs = R(1) - R(0.5) * c.s_phi;
    R ms[9];
    ms[0] = phi;
    ms[1] = R(-2) * phi;
    ms[2] = phi;
    ms[3] = hjx - c.s_phi * (hjx - phi * vx) + hs * G1x;
    ms[4] = -phi * vx - R(0.5) * G1x;
    ms[5] = hjy - c.s_phi * (hjy - phi * vy) + hs * G1y;
    ms[6] = -phi * vy - R(0.5) * G1y;
    ms[7] = R(0);
    ms[8] = R(0);
    scale_d9(ms);
    mt9(ms, o.h);
  }
  // dendrite collision (D2Q5)
  {
    const R Fs = (R(1.5) * Q - R(0.5) * in.Qo) * c.inv_tau0;
    const R s1 = R(1) / (c.c_s1 * as2 + R(0.5));
    const R m0 = psi + Fs;
    const R* g = in.g;
    const R gjx = g[1] - g[3], gjy = g[2] - g[4];
    const R hs = R(1) - R(0.5) * s1;
    const R Gx = R(-1.0 / 3.0) * Nx * ias2, Gy = R(-1.0 / 3.0) * Ny * ias2;
    const R jsx = gjx - s1 * gjx + hs * Gx, jsy = gjy - s1 * gjy + hs * Gy;
    const R a = m0 * R(1.0 / 6.0);
    o.gpost[0] = m0 * R(1.0 / 3.0);
    o.gpost[1] = a + R(0.5) * jsx;
    o.gpost[3] = a - R(0.5) * jsx;
    o.gpost[2] = a + R(0.5) * jsy;
    o.gpost[4] = a - R(0.5) * jsy;
  }
  // solute collision (D2Q5)
  {
    const R E = R(2) * omk * c.D * qf * C * iA * iA;
    const R jex = C * vx - E * gsx + omk * (at * gsx + jv * nfx);
    const R jey = C * vy - E * gsy + omk * (at * gsy + jv * nfy);
    const R DC = R(2) * c.D * qf * iA;
    const R sc = R(1) / (R(3) * DC + R(0.5));
    const R* s = in.s;
    const R sjx = s[1] - s[3], sjy = s[2] - s[4];
    const R hs = R(1) - R(0.5) * sc;
    const R Gx = C * vx - in.Co * in.vxo, Gy = C * vy - in.Co * in.vyo;
    const R jsx = sjx - sc * (sjx - jex) + hs * Gx, jsy = sjy - sc * (sjy - jey) + hs * Gy;
    const R a = C * R(1.0 / 6.0);
    o.s[0] = C * R(1.0 / 3.0);
    o.s[1] = a + R(0.5) * jsx;
    o.s[3] = a - R(0.5) * jsx;
    o.s[2] = a + R(0.5) * jsy;
    o.s[4] = a - R(0.5) * jsy;
  }
  for (int i = 0; i < 5; ++i) o.gpre[i] = in.g[i];
  o.rr = ias2;
  o.phi = phi;
  o.C = C;
  o.vx = vx;
  o.vy = vy;
  o.Q = Q;
  o.U = U;
  o.p = p;
  o.mu = mu;
}

// --- reverse ------------------------------------------------------------------
// Given the adjoints of the stored outputs (ao: f, h, gpre, gpost, rr, s, phi,
// C, vx, vy, Q; the diagnostics U, p, mu are ignored), accumulate into ai the
// adjoints of every input and into pg the parameter adjoints.  ai and pg are
// overwritten (ai) / accumulated (pg).  dfs_dsigma = d fs_coef / d sigma.
template <typename R>
PF_HD void reverse(const In<R>& in, const Coef<R>& c, R dfs_dsigma, const Out<R>& ao, In<R>& ai,
                   ParGrad<R>& pg) {
  // ---- recompute the forward intermediates ----
  R phi = R(0), psi = R(0), C = R(0);
  for (int i = 0; i < 9; ++i) phi += in.h[i];
  for (int i = 0; i < 5; ++i) psi += in.g[i];
  for (int i = 0; i < 5; ++i) C += in.s[i];
  const R gpx = in.gpx, gpy = in.gpy, gsx = in.gsx, gsy = in.gsy;
  const R rho = c.rho_g + phi * c.drho;
  const R grx = c.drho * gpx, gry = c.drho * gpy;
  const R gmp = sqrt(gpx * gpx + gpy * gpy + c.ge2);
  const R igm = R(1) / gmp;
  const R nfx = gpx * igm, nfy = gpy * igm;
  const R opsi = R(1) + psi, ophi = R(1) - phi;
  const R mu = c.two_bphi * phi * ophi * (R(1) - R(2) * phi) - c.two_bint * ophi * opsi * opsi -
               c.Wphi2 * in.lphi;
  const R aphi = c.kappa * phi * ophi;
  const R Dx = c.M_phi * (gpx - aphi * nfx), Dy = c.M_phi * (gpy - aphi * nfy);
  const R divD = (phi - in.phio) + in.vxo * gpx + in.vyo * gpy;
  const R Fsx = c.fs_coef * mu * gpx, Fsy = c.fs_coef * mu * gpy;
  const R Fby = -(rho - c.rho_bar) * c.g;
  const R Fmx = c.drho * (divD * in.vxo + Dx * in.dvxx + Dy * in.dvxy);
  const R Fmy = c.drho * (divD * in.vyo + Dx * in.dvyx + Dy * in.dvyy);
  const R* f = in.f;
  const R jx = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
  const R jy = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
  const R Fpx = Fsx + Fmx, Fpy = Fsy + Fby + Fmy;
  const R irho = R(1) / rho;
  const R vsx = (jx + R(0.5) * Fpx) * irho, vsy = (jy + R(0.5) * Fpy) * irho;
  const R chi = R(0.5) * opsi;
  const R vx = (R(1) - chi) * vsx, vy = (R(1) - chi) * vsy;
  const R Fx = Fpx - R(2) * chi * rho * vsx, Fy = Fpy - R(2) * chi * rho * vsy;
  const R v2 = vx * vx + vy * vy;
  const R snz = f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8];
  const R p = R(0.6) * (snz + R(0.5) * (vx * grx + vy * gry) - R(2.0 / 3.0) * rho * v2);

  const R gxr = c.ct * gsx + c.sn * gsy, gyr = -c.sn * gsx + c.ct * gsy;
  const R gm2 = gsx * gsx + gsy * gsy;
  const R smag = sqrt(gm2 + c.ge2);
  const R ism = R(1) / smag;
  const R nxr = -gxr * ism, nyr = -gyr * ism;
  const R nx2 = nxr * nxr, ny2 = nyr * nyr;
  const R n2 = nx2 + ny2;
  const R s4 = nx2 * nx2 + ny2 * ny2;
  const R as = R(1) + c.eps * (R(4) * s4 - R(3) * n2 * n2);
  const R iso = s4 + R(0.75) * n2 * (R(1) - n2);
  const R pre = R(-16) * c.eps * as * smag;
  const R Nxr = pre * nxr * (nx2 - iso), Nyr = pre * nyr * (ny2 - iso);
  const R Nx = c.ct * Nxr - c.sn * Nyr, Ny = c.sn * Nxr + c.ct * Nyr;
  const R as2 = as * as;
  const R ias2 = R(1) / as2;
  const R omk = R(1) - c.k;
  const R A = R(1) + c.k - omk * psi;
  const R iA = R(1) / A;
  const R U = (R(2) * C * iA - R(1)) / omk;
  const R omp2 = R(1) - psi * psi;
  const R drive = c.theta + c.Mcinf * U;
  const R Q = c.four_bpsi * psi * omp2 - c.two_bint * ophi * ophi * opsi -
              c.lam * omp2 * omp2 * drive;
  const R dpsi = psi - in.psio;
  const R sat = sqrt(gm2 + c.gat2);
  const R tat = -c.a_at * c.W0 * as * (R(1) + omk * U);  // at = tat * dpsi / sat
  const R at = tat * dpsi / sat;
  const R qf = R(0.5) * (R(1) - psi);
  const R jv = c.D * qf * C * c.kappa * ophi;

  // ---- adjoint accumulators of the intermediates ----
  R a_phi = ao.phi, a_psi = R(0), a_C = ao.C, a_vx = ao.vx, a_vy = ao.vy, a_Q = ao.Q;
  R a_ias2 = ao.rr, a_rho = R(0), a_p = R(0), a_Fx = R(0), a_Fy = R(0), a_grx = R(0),
    a_gry = R(0);
  R a_f[9], a_h[9], a_g[5], a_s[5];
  for (int i = 0; i < 9; ++i) { a_f[i] = R(0); a_h[i] = R(0); }
  for (int i = 0; i < 5; ++i) { a_g[i] = ao.gpre[i]; a_s[i] = R(0); }
  R a_nfx = R(0), a_nfy = R(0), a_aphi = R(0), a_Nx = R(0), a_Ny = R(0), a_at = R(0),
    a_jv = R(0), a_U = R(0), a_gsx = R(0), a_gsy = R(0), a_as = R(0);
  R a_phio = R(0), a_vxo = R(0), a_vyo = R(0), a_Co = R(0), a_Qo = R(0), a_qf = R(0);
  R a_eps = R(0), a_dpsi = R(0);

  // ---- solute collision ----
  {
    const R E = R(2) * omk * c.D * qf * C * iA * iA;
    const R jex = C * vx - E * gsx + omk * (at * gsx + jv * nfx);
    const R jey = C * vy - E * gsy + omk * (at * gsy + jv * nfy);
    const R DC = R(2) * c.D * qf * iA;
    const R den = R(3) * DC + R(0.5);
    const R sc = R(1) / den;
    const R* s = in.s;
    const R sjx = s[1] - s[3], sjy = s[2] - s[4];
    const R Gx = C * vx - in.Co * in.vxo, Gy = C * vy - in.Co * in.vyo;
    // q5 from m: o.s[0] = C/3, o.s[1,3] = C/6 +- jsx/2, o.s[2,4] = C/6 +- jsy/2
    const R* as_ = ao.s;
    a_C += as_[0] * R(1.0 / 3.0) + (as_[1] + as_[2] + as_[3] + as_[4]) * R(1.0 / 6.0);
    const R a_jsx = R(0.5) * (as_[1] - as_[3]), a_jsy = R(0.5) * (as_[2] - as_[4]);
    // jsx = (1 - sc) sjx + sc jex + (1 - sc/2) Gx
    const R a_sjx = (R(1) - sc) * a_jsx, a_sjy = (R(1) - sc) * a_jsy;
    const R a_jex = sc * a_jsx, a_jey = sc * a_jsy;
    const R a_Gx = (R(1) - R(0.5) * sc) * a_jsx, a_Gy = (R(1) - R(0.5) * sc) * a_jsy;
    const R a_sc = (jex - sjx - R(0.5) * Gx) * a_jsx + (jey - sjy - R(0.5) * Gy) * a_jsy;
    a_s[1] += a_sjx; a_s[3] -= a_sjx; a_s[2] += a_sjy; a_s[4] -= a_sjy;
    // sc = 1 / (3 DC + 1/2)
    const R a_DC = -R(3) * sc * sc * a_sc;
    // DC = 2 D qf iA
    a_qf += R(2) * c.D * iA * a_DC;
    R a_iA = R(2) * c.D * qf * a_DC;
    // Gx = C vx - Co vxo
    a_C += vx * a_Gx + vy * a_Gy;
    a_vx += C * a_Gx;
    a_vy += C * a_Gy;
    a_Co += -in.vxo * a_Gx - in.vyo * a_Gy;
    a_vxo += -in.Co * a_Gx;
    a_vyo += -in.Co * a_Gy;
    // jex = C vx - E gsx + omk (at gsx + jv nfx)
    a_C += vx * a_jex + vy * a_jey;
    a_vx += C * a_jex;
    a_vy += C * a_jey;
    const R a_E = -gsx * a_jex - gsy * a_jey;
    a_gsx += (-E + omk * at) * a_jex;
    a_gsy += (-E + omk * at) * a_jey;
    a_at += omk * (gsx * a_jex + gsy * a_jey);
    a_jv += omk * (nfx * a_jex + nfy * a_jey);
    a_nfx += omk * jv * a_jex;
    a_nfy += omk * jv * a_jey;
    // E = 2 omk D qf C iA^2
    a_qf += R(2) * omk * c.D * C * iA * iA * a_E;
    a_C += R(2) * omk * c.D * qf * iA * iA * a_E;
    a_iA += R(4) * omk * c.D * qf * C * iA * a_E;
    // iA = 1 / A, A = 1 + k - omk psi
    const R a_A = -iA * iA * a_iA;
    a_psi += -omk * a_A;
  }
  // ---- dendrite collision ----
  {
    const R den = c.c_s1 * as2 + R(0.5);
    const R s1 = R(1) / den;
    const R* g = in.g;
    const R gjx = g[1] - g[3], gjy = g[2] - g[4];
    const R Gx = R(-1.0 / 3.0) * Nx * ias2, Gy = R(-1.0 / 3.0) * Ny * ias2;
    const R* ag = ao.gpost;
    const R a_m0 = ag[0] * R(1.0 / 3.0) + (ag[1] + ag[2] + ag[3] + ag[4]) * R(1.0 / 6.0);
    const R a_jsx = R(0.5) * (ag[1] - ag[3]), a_jsy = R(0.5) * (ag[2] - ag[4]);
    // jsx = (1 - s1) gjx + (1 - s1/2) Gx
    const R a_gjx = (R(1) - s1) * a_jsx, a_gjy = (R(1) - s1) * a_jsy;
    const R a_Gx = (R(1) - R(0.5) * s1) * a_jsx, a_Gy = (R(1) - R(0.5) * s1) * a_jsy;
    const R a_s1 = (-gjx - R(0.5) * Gx) * a_jsx + (-gjy - R(0.5) * Gy) * a_jsy;
    a_g[1] += a_gjx; a_g[3] -= a_gjx; a_g[2] += a_gjy; a_g[4] -= a_gjy;
    // Gx = -Nx ias2 / 3
    a_Nx += R(-1.0 / 3.0) * ias2 * a_Gx;
    a_Ny += R(-1.0 / 3.0) * ias2 * a_Gy;
    a_ias2 += R(-1.0 / 3.0) * (Nx * a_Gx + Ny * a_Gy);
    // s1 = 1 / (c_s1 as2 + 1/2)  ->  d s1 / d as2 = -c_s1 s1^2
    const R a_as2_s = -c.c_s1 * s1 * s1 * a_s1;
    // m0 = psi + Fs, Fs = (1.5 Q - 0.5 Qo) / tau0
    a_psi += a_m0;
    a_Q += R(1.5) * c.inv_tau0 * a_m0;
    a_Qo += R(-0.5) * c.inv_tau0 * a_m0;
    // ias2 = 1/as2
    const R a_as2 = a_as2_s - ias2 * ias2 * a_ias2;
    a_as += R(2) * as * a_as2;
  }
  // ---- CAC collision ----
  R a_G1x, a_G1y;
  {
    R am[9];
    for (int i = 0; i < 9; ++i) am[i] = ao.h[i];
    R ams[9];
    m9(am, ams);
    scale_d9(ams);  // adjoint of ms = D^-1 M a_h*
    const R hs = R(1) - R(0.5) * c.s_phi;
    a_phi += ams[0] - R(2) * ams[1] + ams[2] + c.s_phi * (vx * ams[3] + vy * ams[5]) -
             vx * ams[4] - vy * ams[6];
    const R a_hjx = (R(1) - c.s_phi) * ams[3], a_hjy = (R(1) - c.s_phi) * ams[5];
    a_vx += c.s_phi * phi * ams[3] - phi * ams[4];
    a_vy += c.s_phi * phi * ams[5] - phi * ams[6];
    a_G1x = hs * ams[3] - R(0.5) * ams[4];
    a_G1y = hs * ams[5] - R(0.5) * ams[6];
    const int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    for (int i = 0; i < 9; ++i) a_h[i] += R(cx[i]) * a_hjx + R(cy[i]) * a_hjy;
    // G1x = phi vx - phio vxo + aphi nfx / 3
    a_phi += vx * a_G1x + vy * a_G1y;
    a_vx += phi * a_G1x;
    a_vy += phi * a_G1y;
    a_phio += -in.vxo * a_G1x - in.vyo * a_G1y;
    a_vxo += -in.phio * a_G1x;
    a_vyo += -in.phio * a_G1y;
    a_aphi += R(1.0 / 3.0) * (nfx * a_G1x + nfy * a_G1y);
    a_nfx += R(1.0 / 3.0) * aphi * a_G1x;
    a_nfy += R(1.0 / 3.0) * aphi * a_G1y;
  }
  // ---- NS collision ----
  {
    R am[9];
    for (int i = 0; i < 9; ++i) am[i] = ao.f[i];
    R ams[9];
    m9(am, ams);
    scale_d9(ams);
    const R hn = R(1) - R(0.5) * c.s_nu;
    R a_m[9];
    for (int i = 0; i < 9; ++i) a_m[i] = R(0);
    R a_vg = R(0.5) * ams[0], a_rv2 = R(0);
    a_m[1] += (R(1) - c.s_e) * ams[1];
    a_p += R(6) * c.s_e * ams[1];
    a_rv2 += R(3) * c.s_e * ams[1];
    a_m[2] += (R(1) - c.s_eps) * ams[2];
    a_p += R(-9) * c.s_eps * ams[2];
    a_rv2 += R(-3) * c.s_eps * ams[2];
    a_vg += -(R(1) - R(0.5) * c.s_eps) * ams[2];
    a_rho += vx * ams[3] + vy * ams[5];
    a_vx += rho * ams[3];
    a_vy += rho * ams[5];
    a_Fx += R(0.5) * ams[3];
    a_Fy += R(0.5) * ams[5];
    a_m[4] += (R(1) - c.s_q) * ams[4];
    a_rho += -c.s_q * (vx * ams[4] + vy * ams[6]);
    a_vx += -c.s_q * rho * ams[4];
    a_vy += -c.s_q * rho * ams[6];
    a_Fx += -(R(1) - R(0.5) * c.s_q) * ams[4];
    a_Fy += -(R(1) - R(0.5) * c.s_q) * ams[6];
    a_m[6] += (R(1) - c.s_q) * ams[6];
    // ms7 = (1 - s_nu) m7 + s_nu rho (vx^2 - vy^2) + hn 2/3 (vx grx - vy gry)
    a_m[7] += (R(1) - c.s_nu) * ams[7];
    a_rho += c.s_nu * (vx * vx - vy * vy) * ams[7];
    a_vx += (R(2) * c.s_nu * rho * vx + hn * R(2.0 / 3.0) * grx) * ams[7];
    a_vy += (R(-2) * c.s_nu * rho * vy - hn * R(2.0 / 3.0) * gry) * ams[7];
    a_grx += hn * R(2.0 / 3.0) * vx * ams[7];
    a_gry += -hn * R(2.0 / 3.0) * vy * ams[7];
    // ms8 = (1 - s_nu) m8 + s_nu rho vx vy + hn/3 (vx gry + vy grx)
    a_m[8] += (R(1) - c.s_nu) * ams[8];
    a_rho += c.s_nu * vx * vy * ams[8];
    a_vx += (c.s_nu * rho * vy + hn * R(1.0 / 3.0) * gry) * ams[8];
    a_vy += (c.s_nu * rho * vx + hn * R(1.0 / 3.0) * grx) * ams[8];
    a_grx += hn * R(1.0 / 3.0) * vy * ams[8];
    a_gry += hn * R(1.0 / 3.0) * vx * ams[8];
    // vg = vx grx + vy gry; rv2 = rho (vx^2 + vy^2)
    a_vx += grx * a_vg + R(2) * rho * vx * a_rv2;
    a_vy += gry * a_vg + R(2) * rho * vy * a_rv2;
    a_grx += vx * a_vg;
    a_gry += vy * a_vg;
    a_rho += v2 * a_rv2;
    // m = M f
    R af[9];
    mt9(a_m, af);
    for (int i = 0; i < 9; ++i) a_f[i] += af[i];
  }
  // ---- pressure: p = 0.6 (snz + 0.5 (vx grx + vy gry) - 2/3 rho v2) ----
  for (int i = 1; i < 9; ++i) a_f[i] += R(0.6) * a_p;
  a_vx += R(0.6) * (R(0.5) * grx - R(4.0 / 3.0) * rho * vx) * a_p;
  a_vy += R(0.6) * (R(0.5) * gry - R(4.0 / 3.0) * rho * vy) * a_p;
  a_grx += R(0.3) * vx * a_p;
  a_gry += R(0.3) * vy * a_p;
  a_rho += R(-0.4) * v2 * a_p;
  // ---- drag: vx = (1 - chi) vsx, Fx = Fpx - 2 chi rho vsx ----
  R a_vsx = (R(1) - chi) * a_vx - R(2) * chi * rho * a_Fx;
  R a_vsy = (R(1) - chi) * a_vy - R(2) * chi * rho * a_Fy;
  R a_chi = -vsx * a_vx - vsy * a_vy - R(2) * rho * (vsx * a_Fx + vsy * a_Fy);
  a_rho += R(-2) * chi * (vsx * a_Fx + vsy * a_Fy);
  R a_Fpx = a_Fx, a_Fpy = a_Fy;
  a_psi += R(0.5) * a_chi;
  // vsx = (jx + 0.5 Fpx) irho
  const R a_jx = irho * a_vsx, a_jy = irho * a_vsy;
  a_Fpx += R(0.5) * irho * a_vsx;
  a_Fpy += R(0.5) * irho * a_vsy;
  const R a_irho = (jx + R(0.5) * Fpx) * a_vsx + (jy + R(0.5) * Fpy) * a_vsy;
  a_rho += -irho * irho * a_irho;
  {
    const int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    for (int i = 0; i < 9; ++i) a_f[i] += R(cx[i]) * a_jx + R(cy[i]) * a_jy;
  }
  // ---- forces: Fpx = Fsx + Fmx, Fpy = Fsy + Fby + Fmy ----
  const R a_Fsx = a_Fpx, a_Fsy = a_Fpy, a_Fmx = a_Fpx, a_Fmy = a_Fpy, a_Fby = a_Fpy;
  // Fmx = drho (divD vxo + Dx dvxx + Dy dvxy)
  const R a_divD = c.drho * (in.vxo * a_Fmx + in.vyo * a_Fmy);
  a_vxo += c.drho * divD * a_Fmx;
  a_vyo += c.drho * divD * a_Fmy;
  const R a_Dx = c.drho * (in.dvxx * a_Fmx + in.dvyx * a_Fmy);
  const R a_Dy = c.drho * (in.dvxy * a_Fmx + in.dvyy * a_Fmy);
  ai.dvxx = c.drho * Dx * a_Fmx;
  ai.dvxy = c.drho * Dy * a_Fmx;
  ai.dvyx = c.drho * Dx * a_Fmy;
  ai.dvyy = c.drho * Dy * a_Fmy;
  // divD = phi - phio + vxo gpx + vyo gpy
  a_phi += a_divD;
  a_phio += -a_divD;
  a_vxo += gpx * a_divD;
  a_vyo += gpy * a_divD;
  R a_gpx = in.vxo * a_divD, a_gpy = in.vyo * a_divD;
  // Dx = M (gpx - aphi nfx)
  a_gpx += c.M_phi * a_Dx;
  a_gpy += c.M_phi * a_Dy;
  a_aphi += -c.M_phi * (nfx * a_Dx + nfy * a_Dy);
  a_nfx += -c.M_phi * aphi * a_Dx;
  a_nfy += -c.M_phi * aphi * a_Dy;
  // Fby = -(rho - rho_bar) g
  a_rho += -c.g * a_Fby;
  // Fsx = fs mu gpx
  const R a_mu = c.fs_coef * (gpx * a_Fsx + gpy * a_Fsy);
  a_gpx += c.fs_coef * mu * a_Fsx;
  a_gpy += c.fs_coef * mu * a_Fsy;
  pg.sigma += dfs_dsigma * mu * (gpx * a_Fsx + gpy * a_Fsy);
  // mu = 2bphi phi (1-phi)(1-2phi) - 2bint (1-phi)(1+psi)^2 - Wphi^2 lphi
  a_phi += (c.two_bphi * (R(1) - R(6) * phi + R(6) * phi * phi) + c.two_bint * opsi * opsi) * a_mu;
  a_psi += R(-2) * c.two_bint * ophi * opsi * a_mu;
  ai.lphi = -c.Wphi2 * a_mu;
  // ---- solute sources: jv = D qf C kappa (1-phi) ----
  a_qf += c.D * C * c.kappa * ophi * a_jv;
  a_C += c.D * qf * c.kappa * ophi * a_jv;
  a_phi += -c.D * qf * C * c.kappa * a_jv;
  a_psi += R(-0.5) * a_qf;
  // at = tat dpsi / sat, tat = -a_at W0 as (1 + omk U), sat = sqrt(gm2 + gat2)
  {
    const R a_tat = dpsi / sat * a_at;
    a_dpsi += tat / sat * a_at;
    const R a_sat = -tat * dpsi / (sat * sat) * a_at;
    a_as += -c.a_at * c.W0 * (R(1) + omk * U) * a_tat;
    a_U += -c.a_at * c.W0 * as * omk * a_tat;
    // sat^2 = gsx^2 + gsy^2 + gat2
    a_gsx += gsx / sat * a_sat;
    a_gsy += gsy / sat * a_sat;
  }
  a_psi += a_dpsi;
  const R a_psio = -a_dpsi;
  // Q = 4bpsi psi omp2 - 2bint (1-phi)^2 (1+psi) - lam omp2^2 drive
  {
    const R a_omp2 = (c.four_bpsi * psi - R(2) * c.lam * omp2 * drive) * a_Q;
    const R a_drive = -c.lam * omp2 * omp2 * a_Q;
    a_psi += (c.four_bpsi * omp2 - c.two_bint * ophi * ophi) * a_Q - R(2) * psi * a_omp2;
    a_phi += R(2) * c.two_bint * ophi * opsi * a_Q;
    // drive = theta + Mcinf U; d theta / d Omega = -Mcinf/(1-(1-k)Omega)
    // - Omega (1-k) ... = -1 for the isothermal closure, d Mcinf / d Omega = -(1-k)
    a_U += c.Mcinf * a_drive;
    pg.Omega += (R(-1) - omk * U) * a_drive;
  }
  // U = (2 C iA - 1) / omk
  a_C += R(2) * iA / omk * a_U;
  {
    const R a_iA = R(2) * C / omk * a_U;
    a_psi += -omk * (-iA * iA * a_iA);
  }
  // ---- anisotropy: as, N from (gsx, gsy) and eps ----
  {
    // Nx = ct Nxr - sn Nyr, Ny = sn Nxr + ct Nyr
    const R a_Nxr = c.ct * a_Nx + c.sn * a_Ny;
    const R a_Nyr = -c.sn * a_Nx + c.ct * a_Ny;
    // Nxr = pre nxr (nx2 - iso)
    const R a_pre = nxr * (nx2 - iso) * a_Nxr + nyr * (ny2 - iso) * a_Nyr;
    R a_nxr = pre * (nx2 - iso) * a_Nxr;
    R a_nyr = pre * (ny2 - iso) * a_Nyr;
    R a_nx2 = pre * nxr * a_Nxr;
    R a_ny2 = pre * nyr * a_Nyr;
    const R a_iso = -pre * (nxr * a_Nxr + nyr * a_Nyr);
    // pre = -16 eps as smag
    a_eps += R(-16) * as * smag * a_pre;
    a_as += R(-16) * c.eps * smag * a_pre;
    R a_smag = R(-16) * c.eps * as * a_pre;
    // iso = s4 + 0.75 n2 (1 - n2)
    R a_s4 = a_iso;
    R a_n2 = R(0.75) * (R(1) - R(2) * n2) * a_iso;
    // as = 1 + eps (4 s4 - 3 n2^2)
    a_eps += (R(4) * s4 - R(3) * n2 * n2) * a_as;
    a_s4 += R(4) * c.eps * a_as;
    a_n2 += R(-6) * c.eps * n2 * a_as;
    // s4 = nx2^2 + ny2^2, n2 = nx2 + ny2
    a_nx2 += R(2) * nx2 * a_s4 + a_n2;
    a_ny2 += R(2) * ny2 * a_s4 + a_n2;
    a_nxr += R(2) * nxr * a_nx2;
    a_nyr += R(2) * nyr * a_ny2;
    // nxr = -gxr ism, nyr = -gyr ism
    const R a_gxr = -ism * a_nxr, a_gyr = -ism * a_nyr;
    const R a_ism = -gxr * a_nxr - gyr * a_nyr;
    a_smag += -ism * ism * a_ism;
    // smag = sqrt(gm2 + ge2)
    a_gsx += gsx / smag * a_smag;
    a_gsy += gsy / smag * a_smag;
    // gxr = ct gsx + sn gsy, gyr = -sn gsx + ct gsy
    a_gsx += c.ct * a_gxr - c.sn * a_gyr;
    a_gsy += c.sn * a_gxr + c.ct * a_gyr;
  }
  pg.eps += a_eps;
  // ---- gas-liquid interface ----
  // aphi = kappa phi (1-phi)
  a_phi += c.kappa * (R(1) - R(2) * phi) * a_aphi;
  // nfx = gpx igm, igm = 1/sqrt(gpx^2 + gpy^2 + ge2)
  {
    const R a_igm = gpx * a_nfx + gpy * a_nfy;
    a_gpx += igm * a_nfx;
    a_gpy += igm * a_nfy;
    const R a_gmp = -igm * igm * a_igm;
    a_gpx += gpx / gmp * a_gmp;
    a_gpy += gpy / gmp * a_gmp;
  }
  // grx = drho gpx; rho = rho_g + phi drho
  a_gpx += c.drho * a_grx;
  a_gpy += c.drho * a_gry;
  a_phi += c.drho * a_rho;
  // ---- moments: phi = sum h, psi = sum g, C = sum s ----
  for (int i = 0; i < 9; ++i) ai.h[i] = a_h[i] + a_phi;
  for (int i = 0; i < 5; ++i) ai.g[i] = a_g[i] + a_psi;
  for (int i = 0; i < 5; ++i) ai.s[i] = a_s[i] + a_C;
  for (int i = 0; i < 9; ++i) ai.f[i] = a_f[i];
  ai.psio = a_psio;
  ai.gpx = a_gpx;
  ai.gpy = a_gpy;
  ai.gsx = a_gsx;
  ai.gsy = a_gsy;
  ai.phio = a_phio;
  ai.Co = a_Co;
  ai.Qo = a_Qo;
  ai.vxo = a_vxo;
  ai.vyo = a_vyo;
}

}  // namespace local
}  // namespace pf
