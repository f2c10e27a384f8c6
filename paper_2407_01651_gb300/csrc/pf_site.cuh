// pf_site.cuh -- the per-site part of one coupled LB step of the
// gas-liquid-dendrite phase-field model (arXiv 2407.01651), shared by every
// traversal of the step kernel: isotropic stencils, interface geometry,
// forces and sources (Sections 2.1-2.2), the four MRT collisions
// (Appendix B) and the stores of the new state.
//
// site_math takes its inputs as values (the streamed populations, the lagged
// scalars and the 3 x 3 stencil neighbourhoods) and returns the new state as
// values; each traversal gathers the inputs from its own memory layout and
// stores the outputs.  It is templated on the lane type T and the parameter
// type R (T = R for every traversal here).
#pragma once

#include "pf_pull.cuh"

namespace pf {

// Values of a field on the 3 x 3 neighbourhood of a site: v[row][dx + 1],
// rows 0 = y-1, 1 = y, 2 = y+1.
template <typename T>
struct Nb9 {
  T v[3][3];
};

// New state and diagnostic fields of a site.
template <typename T>
struct SiteOut {
  T f[9], h[9], s[5], gpost[5];
  T ias2, phi, psi, C, U, p, vx, vy, Q, mu;
};

// Temperature coupling (thermal mode): inputs and outputs of a site.
template <typename T>
struct ThermIn {
  T e[5];     // streamed temperature populations
  T Ho;       // H of the previous step
  Nb9<T> U;   // supersaturation on the 3 x 3 neighbourhood (for grad F)
};
template <typename T>
struct ThermOut {
  T e[5];     // post-collision temperature populations
  T H, theta;
};

// Everything after streaming at one site:
//   f, h, g, s   streamed populations (g after the a_s^2 time stretch)
//   psio         psi of the previous step
//   phio, Co, Qo lagged phi, C, Q_psi of the site
//   P, S, VX, VY phi, psi and the lagged velocity on the 3 x 3 neighbourhood
//   ct, sn       grain rotation; eps anisotropy strength; rho_bar mean density
// g is stored unchanged as the next g_pre; everything else goes to `o`.
// TH (thermal mode, Section 2.1 and Appendix B): theta comes from the
// temperature lattice (ti, to) instead of theta_sys, and the dendrite lattice
// takes F(U) = 1/Le + M c_inf [1 + (1-k) U] in its rate and the source
//   Q_eff = Q / F + W0^2 / F^2 grad F . (a_s^2 grad psi + N),
// stored as the lagged source (o.Q) in place of Q.
template <typename T, typename R, bool TH = false>
__device__ __forceinline__ void site_math(const KParams<R>& kp, T rho_bar, T eps, T ct, T sn,
                                          const T (&f_in)[9], const T (&h_in)[9],
                                          const T (&g)[5], const T (&s_in)[5], T psio, T phio,
                                          T Co, T Qo, const Nb9<T>& P, const Nb9<T>& S,
                                          const Nb9<T>& VX, const Nb9<T>& VY, SiteOut<T>& o,
                                          const ThermIn<T>* ti = nullptr,
                                          ThermOut<T>* to = nullptr) {
  T* f = o.f;
  T* h = o.h;
  T* s = o.s;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    f[i] = f_in[i];
    h[i] = h_in[i];
  }
#pragma unroll
  for (int i = 0; i < 5; ++i) s[i] = s_in[i];

  const T phi = P.v[1][1], psi = S.v[1][1];
  const V2<T> vo = vec2(VX.v[1][1], VY.v[1][1]);
  T C;
  {
    CSum<T> cs;
#pragma unroll
    for (int i = 0; i < 5; ++i) cs.add(s[i]);
    C = cs.value();
  }

  // ---- isotropic stencils (9-point D2Q9 weights), on differences from the
  // centre value so that FP32 keeps the bits of the small neighbour
  // differences.  e/w = x+-1, n/s = y+-1.
  const T w1 = T(1.0 / 9.0), w2 = T(1.0 / 36.0);
  // gradient (d/dx, d/dy) of one scalar field
  auto grad = [&](const Nb9<T>& X) {
    const V2<T> X0 = splat(X.v[1][1]);
    const V2<T> en = vec2(X.v[1][2], X.v[2][1]) - X0;   // (e, n)
    const V2<T> ws = vec2(X.v[1][0], X.v[0][1]) - X0;   // (w, s)
    const V2<T> nen = vec2(X.v[2][2], X.v[2][0]) - X0;  // (ne, nw)
    const V2<T> sws = vec2(X.v[0][0], X.v[0][2]) - X0;  // (sw, se)
    const V2<T> dd = nen - sws;                         // (ne - sw, nw - se)
    const V2<T> cr = vec2(dd.x - dd.y, dd.x + dd.y);    // ((ne-sw)+(se-nw), (ne-sw)+(nw-se))
    return T(3) * fma(splat(w1), en - ws, w2 * cr);
  };
  // gradients of a pair of fields (U, V): (dU/dx, dV/dx) and (dU/dy, dV/dy)
  auto grad_pair = [&](const Nb9<T>& U, const Nb9<T>& V, V2<T>& gx, V2<T>& gy) {
    auto at = [&](int r, int k) { return vec2(U.v[r][k], V.v[r][k]); };
    const V2<T> X0 = at(1, 1);
    const V2<T> e = at(1, 2) - X0, w = at(1, 0) - X0, n = at(2, 1) - X0, so = at(0, 1) - X0;
    const V2<T> ne = at(2, 2) - X0, nw = at(2, 0) - X0, sw = at(0, 0) - X0, se = at(0, 2) - X0;
    const V2<T> a = ne - sw, b = se - nw;
    gx = T(3) * fma(splat(w1), e - w, w2 * (a + b));
    gy = T(3) * fma(splat(w1), n - so, w2 * (a - b));
  };
  const V2<T> gp = grad(P);   // grad phi
  const V2<T> gs = grad(S);   // grad psi
  V2<T> dvx, dvy;             // (d vx_o/dx, d vy_o/dx), (d vx_o/dy, d vy_o/dy)
  grad_pair(VX, VY, dvx, dvy);
  T lphi;
  {
    const V2<T> X0 = splat(P.v[1][1]);
    const V2<T> ax = (vec2(P.v[1][2], P.v[2][1]) - X0) + (vec2(P.v[1][0], P.v[0][1]) - X0);
    const V2<T> dg = (vec2(P.v[2][2], P.v[2][0]) - X0) + (vec2(P.v[0][0], P.v[0][2]) - X0);
    lphi = T(6) * (w1 * (ax.x + ax.y) + w2 * (dg.x + dg.y));
  }

  // ---- gas-liquid interface, forces ----
  const T rho = T(kp.rho_g) + phi * T(kp.drho);
  const V2<T> gr = kp.drho * gp;                       // grad rho
  const V2<T> gp2 = gp * gp;
  const T igm = frsqrt(gp2.x + gp2.y + T(kp.ge2));
  const V2<T> nf = igm * gp;                           // n_phi
  const T opsi = T(1) + psi, ophi = T(1) - phi;
  const T mu = T(kp.two_bphi) * phi * ophi * (T(1) - T(2) * phi) -
               T(kp.two_bint) * ophi * opsi * opsi - T(kp.Wphi2) * lphi;
  const V2<T> Fsb = fma(T(kp.fs_coef) * mu, gp, vec2(T(0), -(rho - rho_bar) * T(kp.g)));
  const T aphi = T(kp.kappa) * phi * ophi;
  const V2<T> D = kp.M_phi * fma(-aphi, nf, gp);
  const V2<T> vg = vo * gp;
  const T divD = (phi - phio) + (vg.x + vg.y);
  const V2<T> Fm = kp.drho * fma(D.x, dvx, fma(D.y, dvy, divD * vo));

  // ---- NS moments, drag, pressure ----
  const V2<T> fA = vec2(f[1], f[2]) - vec2(f[3], f[4]), fU = vec2(f[5], f[6]) - vec2(f[7], f[8]);
  const V2<T> j = fA + vec2(fU.x - fU.y, fU.x + fU.y);
  const V2<T> fS = vec2(f[1], f[2]) + vec2(f[3], f[4]), fT = vec2(f[5], f[6]) + vec2(f[7], f[8]);
  const T sum_nz = (fS.x + fS.y) + (fT.x + fT.y);
  const V2<T> Fp = Fsb + Fm;
  const T irho = frcp(rho);
  const V2<T> vs = irho * fma(T(0.5), Fp, j);
  const T chi = T(0.5) * opsi;
  const V2<T> v = (T(1) - chi) * vs;
  const V2<T> F = fma(T(-2) * chi * rho, vs, Fp);
  const V2<T> vv = v * v, vgr = v * gr;
  const T v2 = vv.x + vv.y;
  // c_s^2/(1-w0) = 3/5; w0/(2 c_s^2) = 2/3
  const T p = T(0.6) * (sum_nz + T(0.5) * (vgr.x + vgr.y) - T(2.0 / 3.0) * rho * v2);

  // ---- dendrite geometry in the grain frame ----
  const T gxr = ct * gs.x + sn * gs.y, gyr = -sn * gs.x + ct * gs.y;
  const V2<T> gs2 = gs * gs;
  const T gm2 = gs2.x + gs2.y;
  const T ism = frsqrt(gm2 + T(kp.ge2));
  const T smag = (gm2 + T(kp.ge2)) * ism;
  const V2<T> nr = (-ism) * vec2(gxr, gyr);            // n' = -grad psi / |grad psi|, grain frame
  const V2<T> n2v = nr * nr;
  const T n2 = n2v.x + n2v.y;
  const V2<T> n4v = n2v * n2v;
  const T s4 = n4v.x + n4v.y;
  const T as = T(1) + eps * (T(4) * s4 - T(3) * n2 * n2);
  const T iso = s4 + T(0.75) * n2 * (T(1) - n2);
  const T pre = T(-16) * eps * as * smag;
  const V2<T> Nr = pre * (nr * (n2v - splat(iso)));
  const T Nx = ct * Nr.x - sn * Nr.y, Ny = sn * Nr.x + ct * Nr.y;
  const T as2 = as * as;
  const T ias2 = frcp(as2);

  // ---- solute and dendrite sources ----
  const T omk = T(R(1) - kp.k);
  const T A = T(R(1) + kp.k) - omk * psi;
  const T iA = frcp(A);
  const T U = (T(2) * C * iA - T(1)) * T(kp.inv_omk);
  const T omp2 = T(1) - psi * psi;
  // temperature: rho H = sum of the streamed e (rest population first, the
  // largest), theta = H / c_p + (c_p^s / c_p) h(psi)
  T rhoH = T(0), theta = T(kp.theta);
  if constexpr (TH) {
    CSum<T> es;
#pragma unroll
    for (int i = 0; i < 5; ++i) es.add(ti->e[i]);
    rhoH = es.value();
    theta = fma(rhoH * irho, T(kp.th_icp), T(kp.th_lh) * opsi);
  }
  const T Q = T(kp.four_bpsi) * psi * omp2 - T(kp.two_bint) * ophi * ophi * opsi -
              T(kp.lam) * omp2 * omp2 * (theta + T(kp.Mcinf) * U);
  const T dpsi = psi - psio;
  const T at = T(-kp.a_at * kp.W0) * as * (T(1) + omk * U) * dpsi * frsqrt(gm2 + T(kp.gat2));
  const T qf = T(0.5) * (T(1) - psi);
  const T jv = T(kp.D) * qf * C * T(kp.kappa) * ophi;

  // ---- collisions ----
  collide_ns(f, p, rho, v, F, gr, kp);
  collide_cac(h, phi, v, fma(T(1.0 / 3.0) * aphi, nf, fma(phi, v, (-phio) * vo)), kp);
  T Qs = Q;        // source stored as the lagged value
  {
    T s1;
    if constexpr (TH) {
      const T iF = frcp(T(kp.th_iLe) + T(kp.Mcinf) * (T(1) + omk * U));
      V2<T> gu;
      {
        const Nb9<T>& X = ti->U;
        const V2<T> X0 = splat(X.v[1][1]);
        const V2<T> en = vec2(X.v[1][2], X.v[2][1]) - X0;
        const V2<T> ws = vec2(X.v[1][0], X.v[0][1]) - X0;
        const V2<T> nen = vec2(X.v[2][2], X.v[2][0]) - X0;
        const V2<T> sws = vec2(X.v[0][0], X.v[0][2]) - X0;
        const V2<T> dd = nen - sws;
        const V2<T> cr = vec2(dd.x - dd.y, dd.x + dd.y);
        gu = T(3) * fma(splat(w1), en - ws, w2 * cr);   // grad U
      }
      const V2<T> Xv = fma(splat(as2), gs, vec2(Nx, Ny));   // a_s^2 grad psi + N
      const V2<T> gX = gu * Xv;
      Qs = fma(T(kp.W0sq) * T(kp.th_dF) * iF * iF, gX.x + gX.y, Q * iF);
      s1 = frcp(T(kp.c_s1) * as2 * iF + T(0.5));
    } else {
      s1 = frcp(T(kp.c_s1) * as2 + T(0.5));
    }
    const T Fs = (Qs + T(0.5) * (Qs - Qo)) * T(kp.inv_tau0);
#pragma unroll
    for (int i = 0; i < 5; ++i) o.gpost[i] = g[i];
    collide_q5(o.gpost, psi + Fs, s1, vec2(T(0), T(0)), (T(-1.0 / 3.0) * ias2) * vec2(Nx, Ny));
  }
  {
    const T E = T(2) * omk * T(kp.D) * qf * C * iA * iA;
    const V2<T> jeq = fma(C, v, fma(-E, gs, omk * fma(at, gs, jv * nf)));
    const T DC = T(2 * kp.D) * qf * iA;
    const T sc = frcp(T(3) * DC + T(0.5));
    collide_q5(s, C, sc, jeq, fma(C, v, (-Co) * vo));
  }
  if constexpr (TH) {
    // d_t(rho H v) with rho_o H_o v_o of the previous step (backward difference)
    const T rho_o = T(kp.rho_g) + phio * T(kp.drho);
    const V2<T> jH = rhoH * v;
    const V2<T> dJ = fma(-(rho_o * ti->Ho), vo, jH);
#pragma unroll
    for (int i = 0; i < 5; ++i) to->e[i] = ti->e[i];
    collide_th(to->e, rhoH, theta, T(kp.th_s), jH, dJ);
    to->H = rhoH * irho;
    to->theta = theta;
  }
  o.ias2 = ias2;
  o.phi = phi;
  o.psi = psi;
  o.C = C;
  o.U = U;
  o.p = p;
  o.vx = v.x;
  o.vy = v.y;
  o.Q = Qs;
  o.mu = mu;
}

// One site: gather the stencil values from the traversal's shared-memory rows,
// run site_math and store the new state and (if requested) the fields.
// TH: thermal mode, with SU the supersaturation rows and in.e / in.Ho loaded.
template <typename S, typename R, bool TH = false>
__device__ __forceinline__ void site_update(const StepArgs<S, R>& a, const DomDesc& d,
                                            const Src9& src, const SiteIn<R>& in,
                                            const R (&h_in)[9], const R (&g_in)[5], R psio,
                                            Rows3<R> SP, Rows3<R> SS, Rows3<R> SVX,
                                            Rows3<R> SVY, int c, Rows3<R> SU = Rows3<R>{}) {
  const unsigned ps = (unsigned)a.plane_stride;
  const unsigned site = src.s[0];
  auto nb = [&](const Rows3<R>& X) {
    Nb9<R> n;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      n.v[0][k] = X.m[c - 1 + k];
      n.v[1][k] = X.c[c - 1 + k];
      n.v[2][k] = X.p[c - 1 + k];
    }
    return n;
  };
  const double2 cs = a.grain_cs[d.grain_off + in.gid];
  SiteOut<R> o;
  ThermIn<R> ti;
  ThermOut<R> to;
  if constexpr (TH) {
#pragma unroll
    for (int i = 0; i < 5; ++i) ti.e[i] = in.e[i];
    ti.Ho = in.Ho;
    ti.U = nb(SU);
  }
  site_math<R, R, TH>(a.kp, static_cast<R>(d.rho_bar), static_cast<R>(d.eps_s),
                      static_cast<R>(cs.x), static_cast<R>(cs.y), in.f, h_in, g_in, in.s, psio,
                      in.phio, in.Co, in.Qo, nb(SP), nb(SS), nb(SVX), nb(SVY), o, &ti, &to);

  // ---- store ----
  const R phi = o.phi, psi = o.psi, C = o.C;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    st_ns<S, R>(plane(a.out, P_F + i, ps), site, o.f[i]);
    st_off_w<S, R>(plane(a.out, P_H + i, ps), site, o.h[i], w9<R>(i), phi);
  }
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    st_off_w<S, R>(plane(a.out, P_GPRE + i, ps), site, g_in[i], w5<R>(i), psi);
    st_off_w<S, R>(plane(a.out, P_GPOST + i, ps), site, o.gpost[i], w5<R>(i), psi);
    st_off_w<S, R>(plane(a.out, P_S + i, ps), site, o.s[i], w5<R>(i), C);
  }
  plane(a.aout, A_RR, ps)[site] = o.ias2;
  plane(a.aout, A_PHIO, ps)[site] = phi;
  plane(a.aout, A_CO, ps)[site] = C;
  plane(a.aout, A_VXO, ps)[site] = o.vx;
  plane(a.aout, A_VYO, ps)[site] = o.vy;
  plane(a.aout, A_QO, ps)[site] = o.Q;
  if constexpr (Codec<S>::kOffset) plane(a.aout, A_PSIO, ps)[site] = psi;
  if constexpr (TH) {
#pragma unroll
    for (int i = 0; i < 5; ++i) st<S, R>(plane(a.out, P_E + i, ps), site, to.e[i]);
    plane(a.aout, A_HO, ps)[site] = to.H;
  }
  if (a.fields) {
    R* fl = a.fields;
    plane(fl, FLD_PHI, ps)[site] = phi;
    plane(fl, FLD_PSI, ps)[site] = psi;
    plane(fl, FLD_C, ps)[site] = C;
    plane(fl, FLD_U, ps)[site] = o.U;
    plane(fl, FLD_P, ps)[site] = o.p;
    plane(fl, FLD_VX, ps)[site] = o.vx;
    plane(fl, FLD_VY, ps)[site] = o.vy;
    plane(fl, FLD_MU, ps)[site] = o.mu;
    if constexpr (TH) plane(fl, FLD_THETA, ps)[site] = to.theta;
  }
}

}  // namespace pf
