// pf_model.cuh -- device-side pieces of one coupled LB step of the
// gas-liquid-dendrite phase-field model (arXiv 2407.01651): parameters, state
// layout, equilibria and the closed-form MRT collisions.
//
// The collisions below are Lambda = M^-1 S M (Appendix B) written out in
// moment space: the moments of the equilibria and of the forcing terms are
// evaluated analytically and the back-transform uses M^-1 = M^T diag(1/|row|^2)
// of the orthogonal Lallemand-Luo (D2Q9) and (1, cx, cy, 5|c|^2-4, cx^2-cy^2)
// (D2Q5) bases.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pf {

// ---------------------------------------------------------------------------
// State planes.  Each plane holds one value per site of every domain (plane
// stride = total padded sites); domain d starts at DomDesc::off.  Populations
// live in one buffer of the storage type, the lagged scalars in another of
// the compute type.
// ---------------------------------------------------------------------------
enum PopPlane : int {
  P_F = 0,        // NS populations f_0..f_8 (post-collision)
  P_H = 9,        // CAC populations h_0..h_8 (post-collision)
  P_GPRE = 18,    // dendrite populations before collision g_0..g_4
  P_GPOST = 23,   // dendrite populations after collision
  P_S = 28,       // solute populations s_0..s_4 (post-collision)
  N_POP = 33
};

enum AuxPlane : int {
  A_RR = 0,       // 1 / a_s^2 of the last collision
  A_PHIO = 1,     // phi of the last step
  A_CO = 2,       // C of the last step
  A_VXO = 3,      // vx of the last step
  A_VYO = 4,      // vy of the last step
  A_QO = 5,       // Q_psi of the last step
  A_PSIO = 6,     // psi of the last step (offset storage forms only)
  N_AUX = 7
};

// Raw state exchanged with the host (pf_get_state / pf_set_state): 39 planes
// f[9], h[9], g_pre[5], g_post[5], r, s[5], phi, C, vx, vy, Q_psi.
constexpr int N_PHYS = 39;

enum Field : int { FLD_PHI, FLD_PSI, FLD_C, FLD_U, FLD_P, FLD_VX, FLD_VY, FLD_MU, N_FIELDS };

struct DomDesc {
  long long off;      // first site of the domain in every plane
  int nx, ny;
  int tiles_x, tile0; // tiling of the step kernel
  int grain_off;      // first entry of the domain in the grain table
  int pad;
  double eps_s;       // anisotropy strength of this domain
  double rho_bar;     // domain-mean density (buoyancy reference)
};

// Coefficients of one step, precomputed on the host in FP64.
template <typename R>
struct KParams {
  R rho_g, drho;            // rho_g, rho_l - rho_g
  R ge2, gat2;              // grad_eps^2, grad_eps_at^2
  R kappa;                  // sqrt(2 beta_phi) / W_phi
  R fs_coef;                // 6 sigma / (W_phi sqrt(2 beta_phi))
  R Wphi2, M_phi;
  R two_bphi, two_bint, four_bpsi;
  R lam, theta, Mcinf;      // lambda', theta_sys, M c_inf
  R inv_tau0, c_s1;         // 1/tau0, 3 W0^2 / tau0
  R W0, a_at;               // W0, a(psi) = 1/(2 sqrt2)
  R k, D, g;
  R inv_omk;                // 1 / (1 - k)
  R s_e, s_eps, s_q, s_nu, s_phi;
};

// ---------------------------------------------------------------------------
// Equilibria (also used to initialise the populations).
// ---------------------------------------------------------------------------
// NS: f_i^eq = w_i p/cs2 - delta_i0 p/cs2 + rho w_i [3 c.v + 4.5 (c.v)^2 - 1.5 v^2]
template <typename R>
__device__ __forceinline__ void feq_ns(R p, R rho, R vx, R vy, R f[9]) {
  const R w0 = R(4.0 / 9.0), w1 = R(1.0 / 9.0), w5 = R(1.0 / 36.0);
  const R v2 = R(1.5) * (vx * vx + vy * vy);
  const R p3 = R(3) * p;
  f[0] = w0 * p3 - p3 + rho * w0 * (-v2);
  const R ax[4] = {vx, vy, -vx, -vy};
  for (int i = 0; i < 4; ++i) {
    const R cu = ax[i];
    f[1 + i] = w1 * p3 + rho * w1 * (R(3) * cu + R(4.5) * cu * cu - v2);
  }
  const R dg[4] = {vx + vy, -vx + vy, -vx - vy, vx - vy};
  for (int i = 0; i < 4; ++i) {
    const R cu = dg[i];
    f[5 + i] = w5 * p3 + rho * w5 * (R(3) * cu + R(4.5) * cu * cu - v2);
  }
}

// ---------------------------------------------------------------------------
// D2Q9 moment transforms (Lallemand-Luo order rho, e, eps, jx, qx, jy, qy,
// pxx, pxy) and the inverse via M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12,
// 1/6, 1/12, 1/4, 1/4).
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void m9_from_f(const R f[9], R m[9]) {
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

template <typename R>
__device__ __forceinline__ void f_from_m9(const R m[9], R f[9]) {
  const R a = m[0] * R(1.0 / 9.0), b = m[1] * R(1.0 / 36.0), c = m[2] * R(1.0 / 36.0);
  const R d = m[3] * R(1.0 / 6.0), e = m[4] * R(1.0 / 12.0);
  const R fy = m[5] * R(1.0 / 6.0), gy = m[6] * R(1.0 / 12.0);
  const R h = m[7] * R(0.25), k = m[8] * R(0.25);
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

// D2Q5 post-collision populations from (m0, jx, jy) with the energy moment at
// -(2/3) m0 and the anisotropic moment at 0 (their equilibria, rate 1):
// s_0 = m0/3, s_{1,3} = m0/6 +- jx/2, s_{2,4} = m0/6 +- jy/2.
template <typename R>
__device__ __forceinline__ void q5_from_m(R m0, R jx, R jy, R s[5]) {
  const R a = m0 * R(1.0 / 6.0);
  s[0] = m0 * R(1.0 / 3.0);
  s[1] = a + R(0.5) * jx;
  s[3] = a - R(0.5) * jx;
  s[2] = a + R(0.5) * jy;
  s[4] = a - R(0.5) * jy;
}

// NS collision, D2Q9 MRT with forcing through (I - S/2):
//   m* = m - S (m - m_eq) + (I - S/2) M G,
// m_eq = (0, 6p + 3 rho v^2, -9p - 3 rho v^2, rho vx, -rho vx, rho vy, -rho vy,
//         rho (vx^2 - vy^2), rho vx vy),
// M G  = (v.g, 0, -v.g, Fx, -Fx, Fy, -Fy, 2/3 (vx gx - vy gy), 1/3 (vx gy + vy gx))
// with G_i = w_i [c_i.F/cs2 + (c_i.v)(c_i.g)/cs2], g = grad rho.
template <typename R>
__device__ __forceinline__ void collide_ns(R f[9], R p, R rho, R vx, R vy, R Fx, R Fy,
                                           R gx, R gy, const KParams<R>& kp) {
  R m[9];
  m9_from_f(f, m);
  const R v2 = vx * vx + vy * vy;
  const R vg = vx * gx + vy * gy;
  const R rv2 = rho * v2;
  R ms[9];
  ms[0] = R(0.5) * vg;
  ms[1] = m[1] - kp.s_e * (m[1] - (R(6) * p + R(3) * rv2));
  ms[2] = m[2] - kp.s_eps * (m[2] - (R(-9) * p - R(3) * rv2)) - (R(1) - R(0.5) * kp.s_eps) * vg;
  ms[3] = rho * vx + R(0.5) * Fx;
  ms[4] = m[4] - kp.s_q * (m[4] + rho * vx) - (R(1) - R(0.5) * kp.s_q) * Fx;
  ms[5] = rho * vy + R(0.5) * Fy;
  ms[6] = m[6] - kp.s_q * (m[6] + rho * vy) - (R(1) - R(0.5) * kp.s_q) * Fy;
  const R hn = R(1) - R(0.5) * kp.s_nu;
  ms[7] = m[7] - kp.s_nu * (m[7] - rho * (vx * vx - vy * vy)) +
          hn * R(2.0 / 3.0) * (vx * gx - vy * gy);
  ms[8] = m[8] - kp.s_nu * (m[8] - rho * vx * vy) + hn * R(1.0 / 3.0) * (vx * gy + vy * gx);
  f_from_m9(ms, f);
}

// CAC collision, D2Q9: h_eq = w_i phi (1 + 3 c.v), G_i = 3 w_i c.G1.  Flux
// moments relax with s_phi, all others with 1:
// m* = (phi, -2 phi, phi, j*x, -phi vx - G1x/2, j*y, -phi vy - G1y/2, 0, 0).
template <typename R>
__device__ __forceinline__ void collide_cac(R h[9], R phi, R vx, R vy, R G1x, R G1y,
                                            const KParams<R>& kp) {
  const R jx = h[1] - h[3] + h[5] - h[6] - h[7] + h[8];
  const R jy = h[2] - h[4] + h[5] + h[6] - h[7] - h[8];
  const R hs = R(1) - R(0.5) * kp.s_phi;
  R ms[9];
  ms[0] = phi;
  ms[1] = R(-2) * phi;
  ms[2] = phi;
  ms[3] = jx - kp.s_phi * (jx - phi * vx) + hs * G1x;
  ms[4] = -phi * vx - R(0.5) * G1x;
  ms[5] = jy - kp.s_phi * (jy - phi * vy) + hs * G1y;
  ms[6] = -phi * vy - R(0.5) * G1y;
  ms[7] = R(0);
  ms[8] = R(0);
  f_from_m9(ms, h);
}

// D2Q5 collision with conserved zeroth moment m0 (after the direct source),
// flux moments j relaxing with rate s towards jeq plus (1 - s/2) Gj, and the
// other moments at their equilibria.
template <typename R>
__device__ __forceinline__ void collide_q5(R q[5], R m0, R s, R jeqx, R jeqy, R Gx, R Gy) {
  const R jx = q[1] - q[3];
  const R jy = q[2] - q[4];
  const R hs = R(1) - R(0.5) * s;
  const R jsx = jx - s * (jx - jeqx) + hs * Gx;
  const R jsy = jy - s * (jy - jeqy) + hs * Gy;
  q5_from_m(m0, jsx, jsy, q);
}

}  // namespace pf
