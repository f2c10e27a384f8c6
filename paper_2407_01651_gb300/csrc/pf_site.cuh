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
  const V2<R> vo = vec2(SVX.c[c], SVY.c[c]);
  R C;
  {
    CSum<R> cs;
#pragma unroll
    for (int i = 0; i < 5; ++i) cs.add(s[i]);
    C = cs.value();
  }

  // ---- isotropic stencils (9-point D2Q9 weights), on differences from the
  // centre value so that FP32 keeps the bits of the small neighbour
  // differences.  Neighbours: e/w = x+-1, n/s = y+-1 (rows p/m).
  const R w1 = R(1.0 / 9.0), w2 = R(1.0 / 36.0);
  // gradient (d/dx, d/dy) of one scalar field
  auto grad = [&](const Rows3<R>& X) {
    const V2<R> X0 = splat(X.c[c]);
    const V2<R> en = vec2(X.c[c + 1], X.p[c]) - X0;        // (e, n)
    const V2<R> ws = vec2(X.c[c - 1], X.m[c]) - X0;        // (w, s)
    const V2<R> nen = vec2(X.p[c + 1], X.p[c - 1]) - X0;   // (ne, nw)
    const V2<R> sws = vec2(X.m[c - 1], X.m[c + 1]) - X0;   // (sw, se)
    const V2<R> dd = nen - sws;                            // (ne - sw, nw - se)
    const V2<R> cr = vec2(dd.x - dd.y, dd.x + dd.y);       // ((ne-sw)+(se-nw), (ne-sw)+(nw-se))
    return R(3) * fma(splat(w1), en - ws, w2 * cr);
  };
  // gradients of a pair of fields (U, V): returns (dU/dx, dV/dx) and (dU/dy, dV/dy)
  auto grad_pair = [&](const Rows3<R>& U, const Rows3<R>& V, V2<R>& gx, V2<R>& gy) {
    const V2<R> X0 = vec2(U.c[c], V.c[c]);
    const V2<R> e = vec2(U.c[c + 1], V.c[c + 1]) - X0, w = vec2(U.c[c - 1], V.c[c - 1]) - X0;
    const V2<R> n = vec2(U.p[c], V.p[c]) - X0, so = vec2(U.m[c], V.m[c]) - X0;
    const V2<R> ne = vec2(U.p[c + 1], V.p[c + 1]) - X0, nw = vec2(U.p[c - 1], V.p[c - 1]) - X0;
    const V2<R> sw = vec2(U.m[c - 1], V.m[c - 1]) - X0, se = vec2(U.m[c + 1], V.m[c + 1]) - X0;
    const V2<R> a = ne - sw, b = se - nw;
    gx = R(3) * fma(splat(w1), e - w, w2 * (a + b));
    gy = R(3) * fma(splat(w1), n - so, w2 * (a - b));
  };
  const V2<R> gp = grad(SP);   // grad phi
  const V2<R> gs = grad(SS);   // grad psi
  V2<R> dvx, dvy;              // (d vx_o/dx, d vy_o/dx), (d vx_o/dy, d vy_o/dy)
  grad_pair(SVX, SVY, dvx, dvy);
  R lphi;
  {
    const V2<R> X0 = splat(SP.c[c]);
    const V2<R> ax = (vec2(SP.c[c + 1], SP.p[c]) - X0) + (vec2(SP.c[c - 1], SP.m[c]) - X0);
    const V2<R> dg = (vec2(SP.p[c + 1], SP.p[c - 1]) - X0) + (vec2(SP.m[c - 1], SP.m[c + 1]) - X0);
    lphi = R(6) * (w1 * (ax.x + ax.y) + w2 * (dg.x + dg.y));
  }

  // ---- gas-liquid interface, forces ----
  const R rho = kp.rho_g + phi * kp.drho;
  const V2<R> gr = kp.drho * gp;                       // grad rho
  const V2<R> gp2 = gp * gp;
  const R igm = frsqrt(gp2.x + gp2.y + kp.ge2);
  const V2<R> nf = igm * gp;                           // n_phi
  const R opsi = R(1) + psi, ophi = R(1) - phi;
  const R mu = kp.two_bphi * phi * ophi * (R(1) - R(2) * phi) - kp.two_bint * ophi * opsi * opsi -
               kp.Wphi2 * lphi;
  const V2<R> Fsb = fma(kp.fs_coef * mu, gp, vec2(R(0), -(rho - static_cast<R>(d.rho_bar)) * kp.g));
  const R aphi = kp.kappa * phi * ophi;
  const V2<R> D = kp.M_phi * fma(-aphi, nf, gp);
  const V2<R> vg = vo * gp;
  const R divD = (phi - phio) + (vg.x + vg.y);
  const V2<R> Fm = kp.drho * fma(D.x, dvx, fma(D.y, dvy, divD * vo));

  // ---- NS moments, drag, pressure ----
  const V2<R> fA = vec2(f[1], f[2]) - vec2(f[3], f[4]), fU = vec2(f[5], f[6]) - vec2(f[7], f[8]);
  const V2<R> j = fA + vec2(fU.x - fU.y, fU.x + fU.y);
  const V2<R> fS = vec2(f[1], f[2]) + vec2(f[3], f[4]), fT = vec2(f[5], f[6]) + vec2(f[7], f[8]);
  const R sum_nz = (fS.x + fS.y) + (fT.x + fT.y);
  const V2<R> Fp = Fsb + Fm;
  const R irho = frcp(rho);
  const V2<R> vs = irho * fma(R(0.5), Fp, j);
  const R chi = R(0.5) * opsi;
  const V2<R> v = (R(1) - chi) * vs;
  const V2<R> F = fma(R(-2) * chi * rho, vs, Fp);
  const V2<R> vv = v * v, vgr = v * gr;
  const R v2 = vv.x + vv.y;
  // c_s^2/(1-w0) = 3/5; w0/(2 c_s^2) = 2/3
  const R p = R(0.6) * (sum_nz + R(0.5) * (vgr.x + vgr.y) - R(2.0 / 3.0) * rho * v2);
  const R vx = v.x, vy = v.y;

  // ---- dendrite geometry in the grain frame ----
  const double2 cs = a.grain_cs[d.grain_off + gid];
  const R ct = static_cast<R>(cs.x), sn = static_cast<R>(cs.y);
  const R eps = static_cast<R>(d.eps_s);
  const R gxr = ct * gs.x + sn * gs.y, gyr = -sn * gs.x + ct * gs.y;
  const V2<R> gs2 = gs * gs;
  const R gm2 = gs2.x + gs2.y;
  const R ism = frsqrt(gm2 + kp.ge2);
  const R smag = (gm2 + kp.ge2) * ism;
  const V2<R> nr = (-ism) * vec2(gxr, gyr);            // n' = -grad psi / |grad psi|, grain frame
  const V2<R> n2v = nr * nr;
  const R n2 = n2v.x + n2v.y;
  const V2<R> n4v = n2v * n2v;
  const R s4 = n4v.x + n4v.y;
  const R as = R(1) + eps * (R(4) * s4 - R(3) * n2 * n2);
  const R iso = s4 + R(0.75) * n2 * (R(1) - n2);
  const R pre = R(-16) * eps * as * smag;
  const V2<R> Nr = pre * (nr * (n2v - splat(iso)));
  const R Nx = ct * Nr.x - sn * Nr.y, Ny = sn * Nr.x + ct * Nr.y;
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
  collide_ns(f, p, rho, v, F, gr, kp);
  collide_cac(h, phi, v, fma(R(1.0 / 3.0) * aphi, nf, fma(phi, v, (-phio) * vo)), kp);
  R gpost[5];
  {
    const R Fs = (Q + R(0.5) * (Q - Qo)) * kp.inv_tau0;
    const R s1 = frcp(kp.c_s1 * as2 + R(0.5));
#pragma unroll
    for (int i = 0; i < 5; ++i) gpost[i] = g[i];
    collide_q5(gpost, psi + Fs, s1, vec2(R(0), R(0)),
               (R(-1.0 / 3.0) * ias2) * vec2(Nx, Ny));
  }
  {
    const R E = R(2) * omk * kp.D * qf * C * iA * iA;
    const V2<R> jeq = fma(C, v, fma(-E, gs, omk * fma(at, gs, jv * nf)));
    const R DC = R(2) * kp.D * qf * iA;
    const R sc = frcp(R(3) * DC + R(0.5));
    collide_q5(s, C, sc, jeq, fma(C, v, (-Co) * vo));
  }

  // ---- store ----
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    st_ns<S, R>(plane(a.out, P_F + i, ps), site, f[i]);
    st_off<S, R>(plane(a.out, P_H + i, ps), site, h[i], w9<R>(i) * phi);
  }
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    st_off<S, R>(plane(a.out, P_GPRE + i, ps), site, g[i], w5<R>(i) * psi);
    st_off<S, R>(plane(a.out, P_GPOST + i, ps), site, gpost[i], w5<R>(i) * psi);
    st_off<S, R>(plane(a.out, P_S + i, ps), site, s[i], w5<R>(i) * C);
  }
  plane(a.aout, A_RR, ps)[site] = ias2;
  plane(a.aout, A_PHIO, ps)[site] = phi;
  plane(a.aout, A_CO, ps)[site] = C;
  plane(a.aout, A_VXO, ps)[site] = vx;
  plane(a.aout, A_VYO, ps)[site] = vy;
  plane(a.aout, A_QO, ps)[site] = Q;
  if constexpr (Codec<S>::kOffset) plane(a.aout, A_PSIO, ps)[site] = psi;
  if (a.fields) {
    R* fl = a.fields;
    plane(fl, FLD_PHI, ps)[site] = phi;
    plane(fl, FLD_PSI, ps)[site] = psi;
    plane(fl, FLD_C, ps)[site] = C;
    plane(fl, FLD_U, ps)[site] = U;
    plane(fl, FLD_P, ps)[site] = p;
    plane(fl, FLD_VX, ps)[site] = vx;
    plane(fl, FLD_VY, ps)[site] = vy;
    plane(fl, FLD_MU, ps)[site] = mu;
  }
}

}  // namespace pf
