// pf_pull.cuh -- streaming (pull) helpers shared by the step kernel and the
// adjoint kernels: source sites of the D2Q9 / D2Q5 pull, the streamed CAC and
// dendrite populations with the a_s^2 time stretch, and the per-site inputs
// that no neighbour needs.
#pragma once

#include "pf_device.cuh"

namespace pf {

// Source sites of the pull for the 9 D2Q9 directions at (x, y):
// src[i] = (x - cx_i, y - cy_i), periodic.
struct Src9 {
  unsigned s[9];   // element offsets (a handle holds < 2^32 elements per buffer)
};

__device__ __forceinline__ Src9 sources(const DomDesc& d, int x, int y) {
  const int nx = d.nx, ny = d.ny;
  const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
  const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
  const unsigned off = (unsigned)d.off;
  const unsigned unx = (unsigned)nx;
  const unsigned r0 = off + (unsigned)y * unx, rm = off + (unsigned)ym * unx,
                 rp = off + (unsigned)yp * unx;
  Src9 o;
  o.s[0] = r0 + x; o.s[1] = r0 + xm; o.s[2] = rm + x; o.s[3] = r0 + xp; o.s[4] = rp + x;
  o.s[5] = rm + xm; o.s[6] = rm + xp; o.s[7] = rp + xp; o.s[8] = rp + xm;
  return o;
}

// Element offsets of plane k at site index s.  A handle whose buffers hold
// fewer than 2^32 elements addresses them with one 32-bit offset k*ps + s from
// the buffer base (the fast form); a larger one (BIG) takes a 64-bit base per
// plane and the 32-bit site index (a handle holds fewer than 2^32 sites).
template <bool BIG, typename T>
__device__ __forceinline__ const T* pbase(const T* p, int k, unsigned ps) {
  if constexpr (BIG) return plane(p, k, ps);
  else return p;
}
template <bool BIG>
__device__ __forceinline__ unsigned pidx(int k, unsigned ps, unsigned s) {
  if constexpr (BIG) return s;
  else return (unsigned)k * ps + s;
}

// Streamed CAC populations h and dendrite populations g (with the a_s^2 time
// stretch g = g_pre + r_src (g_post,src - g_pre)) at (x, y); returns phi, psi
// (compensated sums) and psi_o, the psi of the previous step (sum of g_pre, or
// the stored lagged psi in the offset forms).  In the offset forms a
// population held by site s decodes as w_i M_o(s) + stored value.
template <typename S, typename R, bool BIG = false>
__device__ __forceinline__ void pull_hg(const StepArgs<S, R>& a, const Src9& src, R h[9],
                                        R g[5], R& phi, R& psi, R& psio) {
  const unsigned ps = (unsigned)a.plane_stride;
  constexpr bool off = Codec<S>::kOffset;
  CSum<R> sh;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const R wm = off ? w9<R>(i) * ld<R>(pbase<BIG>(a.ain, A_PHIO, ps), pidx<BIG>(A_PHIO, ps, src.s[i])) : R(0);
    h[i] = pop_off<S, R>(pbase<BIG>(a.in, P_H + i, ps), pidx<BIG>(P_H + i, ps, src.s[i]), wm);
    sh.add(h[i]);
  }
  phi = sh.value();
  CSum<R> sg;
  R po = R(0);
  const R psio_own = off ? ld<R>(pbase<BIG>(a.ain, A_PSIO, ps), pidx<BIG>(A_PSIO, ps, src.s[0])) : R(0);
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const R gold = pop_off<S, R>(pbase<BIG>(a.in, P_GPRE + i, ps), pidx<BIG>(P_GPRE + i, ps, src.s[0]), w5<R>(i) * psio_own);
    const R wm = off ? w5<R>(i) * ld<R>(pbase<BIG>(a.ain, A_PSIO, ps), pidx<BIG>(A_PSIO, ps, src.s[i])) : R(0);
    const R gpo = pop_off<S, R>(pbase<BIG>(a.in, P_GPOST + i, ps), pidx<BIG>(P_GPOST + i, ps, src.s[i]), wm);
    const R rr = ld<R>(pbase<BIG>(a.ain, A_RR, ps), pidx<BIG>(A_RR, ps, src.s[i]));
    g[i] = gold + (gpo - gold) * rr;
    sg.add(g[i]);
    po += gold;
  }
  psi = sg.value();
  psio = off ? psio_own : po;
}

// Three rows of a shared-memory field around a site: row y-1, y, y+1.
template <typename R>
struct Rows3 {
  const R* m;
  const R* c;
  const R* p;
};

// Per-site inputs that do not feed the neighbours' stencils: streamed NS and
// solute populations and the lagged scalars of the site.
template <typename R>
struct SiteIn {
  R f[9], s[5];
  R phio, Co, Qo;
  uint8_t gid;
  R e[5], Ho;     // thermal mode: streamed temperature populations, lagged H
};

template <typename S, typename R, bool BIG = false, bool TH = false>
__device__ __forceinline__ void load_site(const StepArgs<S, R>& a, const Src9& src,
                                          SiteIn<R>& in) {
  const unsigned ps = (unsigned)a.plane_stride;
  constexpr bool off = Codec<S>::kOffset;
#pragma unroll
  for (int i = 0; i < 9; ++i) in.f[i] = pop_ns<S, R>(pbase<BIG>(a.in, P_F + i, ps), pidx<BIG>(P_F + i, ps, src.s[i]));
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const R wm = off ? w5<R>(i) * ld<R>(pbase<BIG>(a.ain, A_CO, ps), pidx<BIG>(A_CO, ps, src.s[i])) : R(0);
    in.s[i] = pop_off<S, R>(pbase<BIG>(a.in, P_S + i, ps), pidx<BIG>(P_S + i, ps, src.s[i]), wm);
  }
  in.phio = ld<R>(pbase<BIG>(a.ain, A_PHIO, ps), pidx<BIG>(A_PHIO, ps, src.s[0]));
  in.Co = ld<R>(pbase<BIG>(a.ain, A_CO, ps), pidx<BIG>(A_CO, ps, src.s[0]));
  in.Qo = ld<R>(pbase<BIG>(a.ain, A_QO, ps), pidx<BIG>(A_QO, ps, src.s[0]));
  in.gid = a.grain[src.s[0]];
  if constexpr (TH) {
#pragma unroll
    for (int i = 0; i < 5; ++i)
      in.e[i] = ld<R>(pbase<BIG>(a.in, P_E + i, ps), pidx<BIG>(P_E + i, ps, src.s[i]));
    in.Ho = ld<R>(pbase<BIG>(a.ain, A_HO, ps), pidx<BIG>(A_HO, ps, src.s[0]));
  }
}

// Supersaturation U of a site from its streamed solute populations (thermal
// mode: U on the stencil neighbourhood feeds grad F), with the arithmetic of
// the site update's own C and U.
template <typename S, typename R, bool BIG = false>
__device__ __forceinline__ R pull_U(const StepArgs<S, R>& a, const Src9& src, R psi) {
  const unsigned ps = (unsigned)a.plane_stride;
  CSum<R> cs;
#pragma unroll
  for (int i = 0; i < 5; ++i)
    cs.add(ld<R>(pbase<BIG>(a.in, P_S + i, ps), pidx<BIG>(P_S + i, ps, src.s[i])));
  const R C = cs.value();
  const R omk = R(1) - a.kp.k;
  const R A = (R(1) + a.kp.k) - omk * psi;
  return (R(2) * C * frcp(A) - R(1)) * a.kp.inv_omk;
}

}  // namespace pf
