// pf_site.cuh -- the per-site part of one coupled LB step of the
// gas-liquid-dendrite phase-field model (arXiv 2407.01651), shared by every
// traversal of the step kernel: isotropic stencils, interface geometry,
// forces and sources (Sections 2.1-2.2), the four MRT collisions
// (Appendix B) and the stores of the new state.
#pragma once

#include "pf_pull.cuh"

namespace pf {

// Everything after streaming at one site: stencils, interface geometry,
// forces, sources, the four collisions and the stores.  h, g: streamed
// populations of the site; `in` holds the rest of its inputs.
template <typename S, typename R>
__device__ __forceinline__ void site_update(const StepArgs<S, R>& a, const DomDesc& d,
                                            const Src9& src, const SiteIn<R>& in,
                                            const R (&h_in)[9], const R (&g_in)[5], R psio,
                                            Rows3<R> SP, Rows3<R> SS, Rows3<R> SVX,
                                            Rows3<R> SVY, int c) {
  const unsigned ps = (unsigned)a.plane_stride;
  const KParams<R>& kp = a.kp;
  const unsigned site = src.s[0];
  R f[9], h[9], g[5], s[5];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    f[i] = in.f[i];
    h[i] = h_in[i];
  }
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    s[i] = in.s[i];
    g[i] = g_in[i];
  }
  const R phio = in.phio, Co = in.Co, Qo = in.Qo;
  const uint8_t gid = in.gid;

  const R phi = SP.c[c], psi = SS.c[c];
  const R vxo = SVX.c[c], vyo = SVY.c[c];
  R C;
  {
    CSum<R> cs;
#pragma unroll
    for (int i = 0; i < 5; ++i) cs.add(s[i]);
    C = cs.value();
  }

  // ---- isotropic stencils, on differences from the centre value so that
  // FP32 keeps the bits of the (small) neighbour differences ----
  const R w1 = R(1.0 / 9.0), w2 = R(1.0 / 36.0);
  auto grad = [&](const Rows3<R>& X, R& gx, R& gy) {
    const R X0 = X.c[c];
    const R e = X.c[c + 1] - X0, w = X.c[c - 1] - X0, n = X.p[c] - X0, so = X.m[c] - X0;
    const R ne = X.p[c + 1] - X0, nw = X.p[c - 1] - X0;
    const R sw = X.m[c - 1] - X0, se = X.m[c + 1] - X0;
    gx = R(3) * (w1 * (e - w) + w2 * ((ne - sw) + (se - nw)));
    gy = R(3) * (w1 * (n - so) + w2 * ((ne - sw) + (nw - se)));
  };
  R gpx, gpy, gsx, gsy, dvxx, dvxy, dvyx, dvyy;
  grad(SP, gpx, gpy);
  grad(SS, gsx, gsy);
  grad(SVX, dvxx, dvxy);
  grad(SVY, dvyx, dvyy);
  R lphi;
  {
    const R X0 = SP.c[c];
    const R ax = ((SP.c[c + 1] - X0) + (SP.c[c - 1] - X0)) + ((SP.p[c] - X0) + (SP.m[c] - X0));
    const R dg = ((SP.p[c + 1] - X0) + (SP.m[c - 1] - X0)) +
                 ((SP.p[c - 1] - X0) + (SP.m[c + 1] - X0));
    lphi = R(6) * (w1 * ax + w2 * dg);
  }

  // ---- gas-liquid interface, forces ----
  const R rho = kp.rho_g + phi * kp.drho;
  const R grx = kp.drho * gpx, gry = kp.drho * gpy;
  const R igm = frsqrt(gpx * gpx + gpy * gpy + kp.ge2);
  const R nfx = gpx * igm, nfy = gpy * igm;
  const R opsi = R(1) + psi, ophi = R(1) - phi;
  const R mu = kp.two_bphi * phi * ophi * (R(1) - R(2) * phi) - kp.two_bint * ophi * opsi * opsi -
               kp.Wphi2 * lphi;
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
  const R irho = frcp(rho);
  const R vsx = (jx + R(0.5) * Fpx) * irho, vsy = (jy + R(0.5) * Fpy) * irho;
  const R chi = R(0.5) * opsi;
  const R vx = (R(1) - chi) * vsx, vy = (R(1) - chi) * vsy;
  const R Fx = Fpx - R(2) * chi * rho * vsx, Fy = Fpy - R(2) * chi * rho * vsy;
  const R v2 = vx * vx + vy * vy;
  // c_s^2/(1-w0) = 3/5; w0/(2 c_s^2) = 2/3
  const R p = R(0.6) * (sum_nz + R(0.5) * (vx * grx + vy * gry) - R(2.0 / 3.0) * rho * v2);

  // ---- dendrite geometry in the grain frame ----
  const double2 cs = a.grain_cs[d.grain_off + gid];
  const R ct = static_cast<R>(cs.x), sn = static_cast<R>(cs.y);
  const R eps = static_cast<R>(d.eps_s);
  const R gxr = ct * gsx + sn * gsy, gyr = -sn * gsx + ct * gsy;
  const R gm2 = gsx * gsx + gsy * gsy;
  const R ism = frsqrt(gm2 + kp.ge2);
  const R smag = (gm2 + kp.ge2) * ism;
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
  const R ias2 = frcp(as2);

  // ---- solute and dendrite sources ----
  const R omk = R(1) - kp.k;
  const R A = R(1) + kp.k - omk * psi;
  const R iA = frcp(A);
  const R U = (R(2) * C * iA - R(1)) * kp.inv_omk;
  const R omp2 = R(1) - psi * psi;
  const R Q = kp.four_bpsi * psi * omp2 - kp.two_bint * ophi * ophi * opsi -
              kp.lam * omp2 * omp2 * (kp.theta + kp.Mcinf * U);
  const R dpsi = psi - psio;
  const R at = -kp.a_at * kp.W0 * as * (R(1) + omk * U) * dpsi * frsqrt(gm2 + kp.gat2);
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
    const R s1 = frcp(kp.c_s1 * as2 + R(0.5));
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
    const R sc = frcp(R(3) * DC + R(0.5));
    collide_q5(s, C, sc, jex, jey, C * vx - Co * vxo, C * vy - Co * vyo);
  }

  // ---- store ----
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    st_ns<S, R>(a.out, (P_F + i) * ps + site, f[i]);
    st_off<S, R>(a.out, (P_H + i) * ps + site, h[i], w9<R>(i) * phi);
  }
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    st_off<S, R>(a.out, (P_GPRE + i) * ps + site, g[i], w5<R>(i) * psi);
    st_off<S, R>(a.out, (P_GPOST + i) * ps + site, gpost[i], w5<R>(i) * psi);
    st_off<S, R>(a.out, (P_S + i) * ps + site, s[i], w5<R>(i) * C);
  }
  a.aout[A_RR * ps + site] = ias2;
  a.aout[A_PHIO * ps + site] = phi;
  a.aout[A_CO * ps + site] = C;
  a.aout[A_VXO * ps + site] = vx;
  a.aout[A_VYO * ps + site] = vy;
  a.aout[A_QO * ps + site] = Q;
  if constexpr (Codec<S>::kOffset) a.aout[A_PSIO * ps + site] = psi;
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

}  // namespace pf
