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

#include "pf_v2.cuh"

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
  N_POP = 33,
  P_E = 33,       // temperature populations e_0..e_4 (post-collision; thermal mode)
  N_POP_TH = 38
};

enum AuxPlane : int {
  A_RR = 0,       // 1 / a_s^2 of the last collision
  A_PHIO = 1,     // phi of the last step
  A_CO = 2,       // C of the last step
  A_VXO = 3,      // vx of the last step
  A_VYO = 4,      // vy of the last step
  A_QO = 5,       // Q_psi of the last step
  A_PSIO = 6,     // psi of the last step (offset storage forms only)
  N_AUX = 7,
  A_HO = 7,       // H = c_p theta - c_p^s h(psi) of the last step (thermal mode)
  N_AUX_TH = 8
};

// Raw state exchanged with the host (pf_get_state / pf_set_state): 39 planes
// f[9], h[9], g_pre[5], g_post[5], r, s[5], phi, C, vx, vy, Q_psi.
constexpr int N_PHYS = 39;
// Thermal mode: + e[5], H_o.
constexpr int N_PHYS_TH = 45;

enum Field : int { FLD_PHI, FLD_PSI, FLD_C, FLD_U, FLD_P, FLD_VX, FLD_VY, FLD_MU, FLD_THETA, N_FIELDS };

// Boundary type of a domain side, placed half-way between the last site and
// its ghost: periodic; symmetric plane (populations and the normal velocity
// mirrored); wall (half-way bounce-back: no slip, no flux); far field (wall
// for the flow and phi, Dirichlet psi = -1, C = 1, theta = theta0 by
// anti-bounce-back).
// Inlet: velocity u_in by moving-wall bounce-back, liquid phi = 1 and the far
// field for psi, C, theta; outlet: pressure p = 0 for the flow, zero gradient
// for the rest; extrapolation inlet: velocity u_in at the ghost node by
// non-equilibrium extrapolation for the flow, the rest as the inlet.
enum BoundaryType : int { BC_PERIODIC = 0, BC_SYMMETRIC = 1, BC_WALL = 2, BC_FARFIELD = 3,
                          BC_INLET = 4, BC_OUTLET = 5, BC_INLET_NEE = 6 };

struct DomDesc {
  long long off;      // first site of the domain in every plane
  int nx, ny;
  int tiles_x, tile0; // tiling of the step kernel
  int grain_off;      // first entry of the domain in the grain table
  unsigned char bc[4];  // side types x-, x+, y-, y+ (BoundaryType; 0 = periodic)
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
  // temperature coupling (thermal mode)
  R th_cp, th_icp;          // c_p, 1 / c_p
  R th_lh;                  // (c_p^s / c_p) / 2: theta = H / c_p + th_lh (1 + psi)
  R th_s;                   // flux rate of the temperature lattice, k_T = (1/s - 1/2) c_s^2
  R th_iLe;                 // 1 / Le
  R th_dF;                  // M c_inf (1 - k): grad F = th_dF grad U
  R W0sq;                   // W0^2
  R th_far;                 // theta at a far-field side (theta0)
  R vin_x, vin_y;           // velocity at an inlet side
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
// Collisions.  Moments follow the Lallemand-Luo order (rho, e, eps, jx, qx,
// jy, qy, pxx, pxy); the back-transform is M^-1 = M^T diag(1/9, 1/36, 1/36,
// 1/6, 1/12, 1/6, 1/12, 1/4, 1/4).  Both transforms are written on the
// opposite-direction pairs (f1, f2) / (f3, f4) and (f5, f6) / (f7, f8) and on
// (x, y) pairs of moments, so that the FP32 build issues paired instructions.
// ---------------------------------------------------------------------------

// Populations f1..f8 from the moments, given as the scalars of the rest/energy
// group (m0/9, m1/36, m2/36 folded into axis, diag, f0), the flux pairs
// DF = (m3, m5)/6 and EG = (m4, m6)/12, and h = m7/4, k = m8/4.
template <typename T>
__device__ __forceinline__ void f_from_moments(T axis, T diag, V2<T> DF, V2<T> EG, T h, T k,
                                               T f[9]) {
  const V2<T> Q = fma(T(-2), EG, DF);            // (d - 2e, fy - 2gy)
  const V2<T> A = vec2(axis + h, axis - h);
  const V2<T> f12 = A + Q, f34 = A - Q;
  const V2<T> S = DF + EG;                       // (d + e, fy + gy)
  const T P = S.x + k, N = S.x - k;
  const V2<T> f56 = splat(diag + S.y) + vec2(P, -P);
  const V2<T> f78 = splat(diag - S.y) + vec2(-N, N);
  f[1] = f12.x; f[2] = f12.y; f[3] = f34.x; f[4] = f34.y;
  f[5] = f56.x; f[6] = f56.y; f[7] = f78.x; f[8] = f78.y;
}

// D2Q5 post-collision populations from (m0, jx, jy) with the energy moment at
// -(2/3) m0 and the anisotropic moment at 0 (their equilibria, rate 1):
// s_0 = m0/3, s_{1,3} = m0/6 +- jx/2, s_{2,4} = m0/6 +- jy/2.
// s_0 is formed as m0 - 4 (m0/6): by Sterbenz's lemma that difference is
// exact, so sum_i s_i = m0 up to the unbiased rounding of the +-j/2 terms.
// (Rounding m0 * fl(1/3) and m0 * fl(1/6) separately would bias every site's
// sum the same way, a drift of ~0.5 ulp per step in a conserved total.)
template <typename T>
__device__ __forceinline__ void q5_from_m(T m0, V2<T> J, T s[5]) {
  const T a0 = m0 * T(1.0 / 6.0);
  const V2<T> a = splat(a0);
  const V2<T> s12 = fma(T(0.5), J, a), s34 = fma(T(-0.5), J, a);
  s[0] = m0 - T(4) * a0;
  s[1] = s12.x; s[2] = s12.y; s[3] = s34.x; s[4] = s34.y;
}

// NS collision, D2Q9 MRT with forcing through (I - S/2):
//   m* = m - S (m - m_eq) + (I - S/2) M G,
// m_eq = (0, 6p + 3 rho v^2, -9p - 3 rho v^2, rho vx, -rho vx, rho vy, -rho vy,
//         rho (vx^2 - vy^2), rho vx vy),
// M G  = (v.g, 0, -v.g, Fx, -Fx, Fy, -Fy, 2/3 (vx gx - vy gy), 1/3 (vx gy + vy gx))
// with G_i = w_i [c_i.F/cs2 + (c_i.v)(c_i.g)/cs2], g = grad rho.  The
// conserved moments come out as m*_0 = v.g/2 and m*_{3,5} = rho v + F/2.
template <typename T, typename R>
__device__ __forceinline__ void collide_ns(T f[9], T p, T rho, V2<T> v, V2<T> F, V2<T> g,
                                           const KParams<R>& kp) {
  const V2<T> A = vec2(f[1], f[2]), B = vec2(f[3], f[4]), C = vec2(f[5], f[6]),
              D = vec2(f[7], f[8]);
  const V2<T> S = A + B, Dl = A - B, Tt = C + D, U = C - D;
  const T a14 = S.x + S.y, a58 = Tt.x + Tt.y;
  const T m1 = T(-4) * f[0] - a14 + T(2) * a58;
  const T m2 = T(4) * f[0] - T(2) * a14 + a58;
  const V2<T> dxy = vec2(U.x - U.y, U.x + U.y);
  const V2<T> m46 = fma(T(-2), Dl, dxy);
  const V2<T> m78 = vec2(S.x - S.y, Tt.x - Tt.y);

  const V2<T> vv = v * v;
  const T v2s = vv.x + vv.y;
  const V2<T> vgp = v * g;
  const T vg = vgp.x + vgp.y;
  const T rv2 = rho * v2s;
  const T ms0 = T(0.5) * vg;
  const T ms1 = m1 - T(kp.s_e) * (m1 - (T(6) * p + T(3) * rv2));
  const T ms2 = m2 - T(kp.s_eps) * (m2 - (T(-9) * p - T(3) * rv2)) -
                T(R(1) - R(0.5) * kp.s_eps) * vg;
  const V2<T> rv = rho * v;
  const V2<T> ms35 = fma(T(0.5), F, rv);
  const V2<T> ms46 = fma(splat(T(-kp.s_q)), m46 + rv, m46) - (R(1) - R(0.5) * kp.s_q) * F;
  const R hn = R(1) - R(0.5) * kp.s_nu;
  const V2<T> eq78 = vec2(rho * (vv.x - vv.y), rho * v.x * v.y);
  const V2<T> fr78 = vec2(T(2.0 / 3.0) * (vgp.x - vgp.y), T(1.0 / 3.0) * (v.x * g.y + v.y * g.x));
  const V2<T> ms78 = fma(splat(T(hn)), fr78, fma(splat(T(-kp.s_nu)), m78 - eq78, m78));

  const T a = ms0 * T(1.0 / 9.0), b = ms1 * T(1.0 / 36.0), c = ms2 * T(1.0 / 36.0);
  f[0] = a - T(4) * b + T(4) * c;
  f_from_moments(a - b - T(2) * c, a + T(2) * b + c, T(1.0 / 6.0) * ms35,
                 T(1.0 / 12.0) * ms46, T(0.25) * ms78.x, T(0.25) * ms78.y, f);
}

// CAC collision, D2Q9: h_eq = w_i phi (1 + 3 c.v), G_i = 3 w_i c.G1.  Flux
// moments relax with s_phi, all others with 1:
// m* = (phi, -2 phi, phi, j*x, -phi vx - G1x/2, j*y, -phi vy - G1y/2, 0, 0),
// whose back-transform has axis = phi/9, diag = phi/36, h_0 = 4 phi/9.  The
// rest population is formed as h_0 = phi - 4 t with t = fl(axis + diag), an
// exact difference (Sterbenz), and the diagonal base is shifted by the exact
// rounding error of t (Fast2Sum), so that h_0 + 4 axis + 4 diag = phi holds
// exactly.  Otherwise a uniform bulk, where every site rounds the same value
// the same way, would lose a fixed fraction of phi at every step.
template <typename T, typename R>
__device__ __forceinline__ void collide_cac(T h[9], T phi, V2<T> v, V2<T> G1,
                                            const KParams<R>& kp) {
  const V2<T> Dl = vec2(h[1], h[2]) - vec2(h[3], h[4]);
  const V2<T> U = vec2(h[5], h[6]) - vec2(h[7], h[8]);
  const V2<T> J = Dl + vec2(U.x - U.y, U.x + U.y);
  const R hs = R(1) - R(0.5) * kp.s_phi;
  const V2<T> pv = phi * v;
  const V2<T> JS = fma(splat(T(hs)), G1, fma(splat(T(-kp.s_phi)), J - pv, J));
  const V2<T> q46 = fma(T(-0.5), G1, splat(T(0)) - pv);   // (-phi vx - G1x/2, ...)
  const T axis = phi * T(1.0 / 9.0), diag = phi * T(1.0 / 36.0);
  const T t = axis + diag;
  const T e = diag - (t - axis);   // axis + diag - t, exact (|axis| >= |diag|)
  h[0] = phi - T(4) * t;
  f_from_moments(axis, diag - e, T(1.0 / 6.0) * JS, T(1.0 / 12.0) * q46, T(0), T(0), h);
}

// D2Q5 collision with conserved zeroth moment m0 (after the direct source),
// flux moments j relaxing with rate s towards jeq plus (1 - s/2) Gj, and the
// other moments at their equilibria.
template <typename T>
__device__ __forceinline__ void collide_q5(T q[5], T m0, T s, V2<T> Jeq, V2<T> G) {
  const V2<T> J = vec2(q[1], q[2]) - vec2(q[3], q[4]);
  const T hs = T(1) - T(0.5) * s;
  const V2<T> JS = fma(splat(hs), G, fma(splat(-s), J - Jeq, J));
  q5_from_m(m0, JS, q);
}

// Temperature collision, D2Q5 (Appendix B): g_0^eq = rho H + (w_0 - 1) theta,
// g_i^eq = w_i theta + w_i c_i.(rho H v)/c_s^2, G_i = w_i c_i.dJ/c_s^2 with
// dJ = d_t(rho H v); flux moments relax with s, the others with 1.  In moment
// space the energy moment is at -4 m0 + (10/3) theta and the anisotropic one
// at 0, whose back-transform is e_0 = m0 - (2/3) theta, e_{1,3} = theta/6 +- j*x/2,
// e_{2,4} = theta/6 +- j*y/2.  m0 = rho H is conserved as it came in.  The
// base theta/6 of the axis populations is rounded to a multiple of ulp(m0)/4,
// which makes m0 - 4 (theta/6) exact in the common case: a uniform region
// would otherwise round every site's e_0 the same way and drift the conserved
// total of rho H by a fixed fraction per step.
template <typename T>
__device__ __forceinline__ T quantum_quarter_ulp(T m) {
  if constexpr (sizeof(T) == 4) {
    const unsigned e = __float_as_uint(m) & 0x7f800000u;   // 2^E of m, E >= -126
    // 2^(E - 25) = ulp(m) / 4 for a normal m; a tiny m gets the smallest normal
    return e > (25u << 23) ? __uint_as_float(e - (25u << 23)) : __uint_as_float(1u << 23);
  } else {
    const unsigned long long e =
        (unsigned long long)__double_as_longlong(m) & 0x7ff0000000000000ull;
    return e > (54ull << 52) ? __longlong_as_double((long long)(e - (54ull << 52)))
                             : __longlong_as_double(1ll << 52);
  }
}
template <typename T>
__device__ __forceinline__ T round_to_multiple(T v, T q) {
  // q is a power of two, so 1/q and both products are exact
  if constexpr (sizeof(T) == 4) return rintf(v * __frcp_rn(q)) * q;
  else return rint(v * __drcp_rn(q)) * q;
}
template <typename T>
__device__ __forceinline__ void collide_th(T e[5], T m0, T theta, T s, V2<T> Jeq, V2<T> G) {
  const V2<T> J = vec2(e[1], e[2]) - vec2(e[3], e[4]);
  const T hs = T(1) - T(0.5) * s;
  const V2<T> JS = fma(splat(hs), G, fma(splat(-s), J - Jeq, J));
  const T b = round_to_multiple(theta * T(1.0 / 6.0), quantum_quarter_ulp(m0));
  const V2<T> a = splat(b);
  const V2<T> e12 = fma(T(0.5), JS, a), e34 = fma(T(-0.5), JS, a);
  e[0] = m0 - T(4) * b;
  e[1] = e12.x; e[2] = e12.y; e[3] = e34.x; e[4] = e34.y;
}

}  // namespace pf
