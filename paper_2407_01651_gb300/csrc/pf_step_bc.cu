// pf_step_bc.cu -- the y-march step kernel for domains with non-periodic
// sides (arXiv 2407.01651, Section 3: half-way bounce-back for no-slip walls
// and no-flux scalars, the symmetric scheme for symmetry planes; Section 4:
// far-field Dirichlet values psi = psi_l, C = 1, theta = -Omega).
//
// Same traversal and per-site arithmetic as k_step_ymarch (pf_step.cu); what
// differs is where values come from at a non-periodic side:
//   - pull streaming: a symmetric side reflects the source site and the
//     direction; a wall returns the site's own post-collision population of
//     the opposite direction; a far-field side does the same for NS and CAC
//     and an anti-bounce-back -f*_opp + 2 w_i X_far for psi, C and theta; an
//     inlet adds the moving-wall term 2 rho_l w_i c_i.u_in / c_s^2 for NS and
//     anti-bounces CAC to phi = 1; an outlet anti-bounces NS to p = 0 and
//     clamps the other lattices' source to the last site; an extrapolation
//     inlet gives NS the ghost node's populations f*(x_f) + rho_l s(u_in) -
//     rho_f s(v_f) from the fluid site x_f next to it and treats the other
//     lattices as an inlet; a bounce wins where two sides are crossed, then
//     the extrapolation, then the clamp, then the reflection;
//   - stencils: ghost rows and columns of the shared-memory ring hold the
//     mirror site's values mapped per side (phi, psi, U unchanged, or
//     2 X_far - X for psi and U at a far-field side or inlet, 2 - phi at an
//     inlet; the velocity's normal component flipped at a symmetric side, both
//     components at a wall or far field, 2 u_in - v at an inlet, u_in at an
//     extrapolation inlet; everything
//     copied at an outlet; corners: the y side's map, then the x side's).
// Sites away from a non-periodic side take the periodic pulls of pf_pull.cuh.
// FP32 and FP64 storage only.
#include <type_traits>

#include "pf_site.cuh"

namespace pf {

namespace {

__device__ __forceinline__ constexpr int cx9(int i) {
  return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__device__ __forceinline__ constexpr int cy9(int i) {
  return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__device__ __forceinline__ constexpr int opp9(int i) {
  return i == 0 ? 0 : (i <= 4 ? (i + 1) % 4 + 1 : (i + 1) % 4 + 5);
}
// reflections that flip c_x / c_y
__device__ __forceinline__ int mirx9(int i) {
  switch (i) {
    case 1: return 3; case 3: return 1; case 5: return 6; case 6: return 5;
    case 7: return 8; case 8: return 7; default: return i;
  }
}
__device__ __forceinline__ int miry9(int i) {
  switch (i) {
    case 2: return 4; case 4: return 2; case 5: return 8; case 8: return 5;
    case 6: return 7; case 7: return 6; default: return i;
  }
}

__device__ __forceinline__ unsigned site_at(const DomDesc& d, int x, int y) {
  return (unsigned)d.off + (unsigned)y * (unsigned)d.nx + (unsigned)x;
}

// Source of the population of direction i pulled by (x, y): site, direction
// to read and mode (0 plain or reflected, 1 wall bounce, 2 far-field bounce,
// 3 inlet bounce, 4 outlet: source clamped to the last site, 5 extrapolation
// inlet: the source is the ghost node beyond the side, whose NS population is
// built from the fluid site next to it, the one returned).
struct PullSrc {
  unsigned site;
  int q, mode;
};
// IO: some side of the launch is an inlet or an outlet; without them the
// compiler drops those branches from the boundary pulls
template <bool IO>
__device__ __forceinline__ int bounce_rank(int t) {
  return t == BC_WALL ? 1 : (t == BC_FARFIELD ? 2 : (IO && t == BC_INLET ? 3 : 0));
}
template <bool IO>
__device__ __forceinline__ PullSrc pull_src(const DomDesc& d, int x, int y, int i) {
  const int nx = d.nx, ny = d.ny;
  int sx = x - cx9(i), sy = y - cy9(i), q = i, bounce = 0, outlet = 0, nee = 0;
  if (sx < 0 || sx >= nx) {
    const int t = d.bc[sx < 0 ? 0 : 1];
    if (t == BC_PERIODIC) sx += sx < 0 ? nx : -nx;
    else if (t == BC_SYMMETRIC) { sx = sx < 0 ? -1 - sx : 2 * nx - 1 - sx; q = mirx9(q); }
    else if (IO && t == BC_OUTLET) { sx = sx < 0 ? 0 : nx - 1; outlet = 1; }
    else if (IO && t == BC_INLET_NEE) { sx = sx < 0 ? 0 : nx - 1; nee = 1; }
    else bounce = bounce_rank<IO>(t);
  }
  if (sy < 0 || sy >= ny) {
    const int t = d.bc[sy < 0 ? 2 : 3];
    if (t == BC_PERIODIC) sy += sy < 0 ? ny : -ny;
    else if (t == BC_SYMMETRIC) { sy = sy < 0 ? -1 - sy : 2 * ny - 1 - sy; q = miry9(q); }
    else if (IO && t == BC_OUTLET) { sy = sy < 0 ? 0 : ny - 1; outlet = 1; }
    else if (IO && t == BC_INLET_NEE) { sy = sy < 0 ? 0 : ny - 1; nee = 1; }
    else bounce = max(bounce, bounce_rank<IO>(t));
  }
  if (bounce) return {site_at(d, x, y), opp9(i), bounce};
  return {site_at(d, sx, sy), q, nee ? 5 : (outlet ? 4 : 0)};
}

// The lattices other than NS see an extrapolation inlet as an inlet:
// anti-bounce-back at the site itself.
template <bool IO>
__device__ __forceinline__ PullSrc scalar_src(const DomDesc& d, int x, int y, int i) {
  PullSrc p = pull_src<IO>(d, x, y, i);
  if (IO && p.mode == 5) p = {site_at(d, x, y), opp9(i), 3};
  return p;
}

// A pull source of (x, y) lies beyond a non-periodic side.
__device__ __forceinline__ bool near_side(const DomDesc& d, int x, int y) {
  return (x == 0 && d.bc[0]) || (x == d.nx - 1 && d.bc[1]) || (y == 0 && d.bc[2]) ||
         (y == d.ny - 1 && d.bc[3]);
}

// Ring fields: 0 phi, 1 psi, 2 vx_o, 3 vy_o, 4 U.  Ghost value across one side
// of type t on axis (0: x, 1: y) from the mirror site's value v.
template <typename R, bool IO>
__device__ __forceinline__ R ghost_map(const KParams<R>& kp, int t, int axis, int field, R v) {
  if (IO && t == BC_OUTLET) return v;
  if (field == 2 || field == 3) {
    const bool normal = (field == 2) == (axis == 0);
    if (t == BC_SYMMETRIC) return normal ? -v : v;
    if (IO && t == BC_INLET) return R(2) * (field == 2 ? kp.vin_x : kp.vin_y) - v;
    if (IO && t == BC_INLET_NEE) return field == 2 ? kp.vin_x : kp.vin_y;   // the ghost is the node
    return -v;
  }
  if (t == BC_FARFIELD || (IO && (t == BC_INLET || t == BC_INLET_NEE))) {
    if (field == 1) return R(-2) - v;   // 2 psi_far - psi, psi_far = -1
    if (field == 4) return -v;          // 2 U_far - U, U_far = 0
    if (IO && field == 0 && t != BC_FARFIELD) return R(2) - v;   // liquid inflow, phi = 1
  }
  return v;
}

template <typename S, typename R, bool BIG, bool IO>
__device__ __forceinline__ void pull_hg_b(const StepArgs<S, R>& a, const DomDesc& d, int x,
                                          int y, R h[9], R g[5], R& phi, R& psi, R& psio) {
  const unsigned ps = (unsigned)a.plane_stride;
  const unsigned own = site_at(d, x, y);
  CSum<R> sh;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const PullSrc p = scalar_src<IO>(d, x, y, i);
    R v = ld<R>(pbase<BIG>(a.in, P_H + p.q, ps), pidx<BIG>(P_H + p.q, ps, p.site));
    if (IO && p.mode == 3) v = -v + R(2) * w9<R>(i) * R(1);   // inlet: phi = 1
    h[i] = v;
    sh.add(h[i]);
  }
  phi = sh.value();
  CSum<R> sg;
  R po = R(0);
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const PullSrc p = scalar_src<IO>(d, x, y, i);
    const R gold = ld<R>(pbase<BIG>(a.in, P_GPRE + i, ps), pidx<BIG>(P_GPRE + i, ps, own));
    R gpo = ld<R>(pbase<BIG>(a.in, P_GPOST + p.q, ps), pidx<BIG>(P_GPOST + p.q, ps, p.site));
    if (p.mode == 2 || p.mode == 3) gpo = -gpo + R(2) * w5<R>(i) * R(-1);
    const R rr = ld<R>(pbase<BIG>(a.ain, A_RR, ps), pidx<BIG>(A_RR, ps, p.site));
    g[i] = gold + (gpo - gold) * rr;
    sg.add(g[i]);
    po += gold;
  }
  psi = sg.value();
  psio = po;
}

template <typename S, typename R, bool BIG, bool TH, bool IO>
__device__ __forceinline__ void load_site_b(const StepArgs<S, R>& a, const DomDesc& d, int x,
                                            int y, SiteIn<R>& in) {
  const unsigned ps = (unsigned)a.plane_stride;
  const unsigned own = site_at(d, x, y);
  in.phio = ld<R>(pbase<BIG>(a.ain, A_PHIO, ps), pidx<BIG>(A_PHIO, ps, own));
  R vxo = R(0), vyo = R(0);
  if constexpr (IO) {
    vxo = ld<R>(pbase<BIG>(a.ain, A_VXO, ps), pidx<BIG>(A_VXO, ps, own));
    vyo = ld<R>(pbase<BIG>(a.ain, A_VYO, ps), pidx<BIG>(A_VYO, ps, own));
  }
  const R rho_o = a.kp.rho_g + in.phio * a.kp.drho;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const PullSrc p = pull_src<IO>(d, x, y, i);
    if (IO && p.mode == 4) {
      // pressure outlet p = 0: -f*_opp(own) + 2 rho_o w_i [(c.v_o)^2 / (2 cs^4) - v_o^2 / (2 cs^2)]
      const R fo = ld<R>(pbase<BIG>(a.in, P_F + opp9(i), ps), pidx<BIG>(P_F + opp9(i), ps, own));
      const R cu = R(cx9(i)) * vxo + R(cy9(i)) * vyo;
      in.f[i] = -fo + R(2) * rho_o * w9<R>(i) * (R(4.5) * cu * cu - R(1.5) * (vxo * vxo + vyo * vyo));
    } else {
      R v = ld<R>(pbase<BIG>(a.in, P_F + p.q, ps), pidx<BIG>(P_F + p.q, ps, p.site));
      if (IO && p.mode == 3)   // inlet: moving-wall bounce-back
        v += R(2) * (a.kp.rho_g + a.kp.drho) * w9<R>(i) * R(3) *
             (R(cx9(i)) * a.kp.vin_x + R(cy9(i)) * a.kp.vin_y);
      if (IO && p.mode == 5) {
        // extrapolation inlet: the ghost node's post-collision population is
        // f_q^eq(p_b, rho_l, u_in) + f*_q(x_f) - f_q^eq(p_f, rho_f, v_f) with
        // p_b = p_f, i.e. f*_q(x_f) + rho_l s_q(u_in) - rho_f s_q(v_f), with
        // s_q(v) = w_q [3 c.v + 4.5 (c.v)^2 - 1.5 v^2] and the fluid site's
        // last-step rho and v
        const R fx = ld<R>(pbase<BIG>(a.ain, A_VXO, ps), pidx<BIG>(A_VXO, ps, p.site));
        const R fy = ld<R>(pbase<BIG>(a.ain, A_VYO, ps), pidx<BIG>(A_VYO, ps, p.site));
        const R fphi = ld<R>(pbase<BIG>(a.ain, A_PHIO, ps), pidx<BIG>(A_PHIO, ps, p.site));
        const R cb = R(cx9(p.q)) * a.kp.vin_x + R(cy9(p.q)) * a.kp.vin_y;
        const R cf = R(cx9(p.q)) * fx + R(cy9(p.q)) * fy;
        const R sb = R(3) * cb + R(4.5) * cb * cb -
                     R(1.5) * (a.kp.vin_x * a.kp.vin_x + a.kp.vin_y * a.kp.vin_y);
        const R sf = R(3) * cf + R(4.5) * cf * cf - R(1.5) * (fx * fx + fy * fy);
        v += w9<R>(p.q) * ((a.kp.rho_g + a.kp.drho) * sb - (a.kp.rho_g + fphi * a.kp.drho) * sf);
      }
      in.f[i] = v;
    }
  }
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const PullSrc p = scalar_src<IO>(d, x, y, i);
    R v = ld<R>(pbase<BIG>(a.in, P_S + p.q, ps), pidx<BIG>(P_S + p.q, ps, p.site));
    if (p.mode == 2 || p.mode == 3) v = -v + R(2) * w5<R>(i) * R(1);   // C_far = 1
    in.s[i] = v;
    if constexpr (TH) {
      R e = ld<R>(pbase<BIG>(a.in, P_E + p.q, ps), pidx<BIG>(P_E + p.q, ps, p.site));
      if (p.mode == 2 || p.mode == 3) e = -e + R(2) * w5<R>(i) * a.kp.th_far;
      in.e[i] = e;
    }
  }
  in.Co = ld<R>(pbase<BIG>(a.ain, A_CO, ps), pidx<BIG>(A_CO, ps, own));
  in.Qo = ld<R>(pbase<BIG>(a.ain, A_QO, ps), pidx<BIG>(A_QO, ps, own));
  in.gid = a.grain[own];
  if constexpr (TH) in.Ho = ld<R>(pbase<BIG>(a.ain, A_HO, ps), pidx<BIG>(A_HO, ps, own));
}

template <typename S, typename R, bool BIG, bool IO>
__device__ __forceinline__ R pull_U_b(const StepArgs<S, R>& a, const DomDesc& d, int x, int y,
                                      R psi) {
  const unsigned ps = (unsigned)a.plane_stride;
  CSum<R> cs;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const PullSrc p = scalar_src<IO>(d, x, y, i);
    R v = ld<R>(pbase<BIG>(a.in, P_S + p.q, ps), pidx<BIG>(P_S + p.q, ps, p.site));
    if (p.mode == 2 || p.mode == 3) v = -v + R(2) * w5<R>(i) * R(1);
    cs.add(v);
  }
  const R C = cs.value();
  const R omk = R(1) - a.kp.k;
  const R A = (R(1) + a.kp.k) - omk * psi;
  return (R(2) * C * frcp(A) - R(1)) * a.kp.inv_omk;
}

}  // namespace

template <typename S, typename R, bool BIG, bool TH, bool IO>
__global__ void __launch_bounds__(YM_THREADS, sizeof(R) == 4 ? 3 : 2)
    k_step_ymarch_bc(StepArgs<S, R> a) {
  constexpr int RW = YM_W + 2;
  constexpr int NF = TH ? 5 : 4;
  __shared__ R ring[NF][4][RW];
  const int t = threadIdx.x;
  const unsigned ps = (unsigned)a.plane_stride;

  for (int tile = a.tile_base + blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const DomDesc d = a.doms[a.tile_dom[tile]];
    const int lt = tile - d.tile0;
    const int nx = d.nx, ny = d.ny;
    const int x0 = (lt % d.tiles_x) * YM_W;
    const int ya = (lt / d.tiles_x) * a.chunk;
    const int yb = min(ya + a.chunk, ny);
    const int w = min(YM_W, nx - x0);
    bool interior = false, active = false;
    int col = 0, sc = 0, tx = -1;   // column of the values, ring column, x ghost side type
    if (t < YM_W) {
      interior = active = t < w;
      col = x0 + t;
      sc = t + 1;
    } else if (t == YM_W) {
      active = true;
      sc = 0;
      if (x0 == 0 && d.bc[0]) { col = 0; tx = d.bc[0]; }
      else col = x0 == 0 ? nx - 1 : x0 - 1;
    } else if (t == YM_W + 1) {
      active = true;
      sc = w + 1;
      if (x0 + w >= nx && d.bc[1]) { col = nx - 1; tx = d.bc[1]; }
      else col = x0 + w >= nx ? x0 + w - nx : x0 + w;
    }

    // ring values of row yr (ya-1 .. yb, possibly a ghost row) and the
    // streamed h, g of the site (col, row) they were computed at
    auto fill = [&](int yr, R (&h)[9], R (&g)[5], R& po) {
      int ey = yr, ty = -1;
      if (yr < 0) {
        if (d.bc[2]) { ey = 0; ty = d.bc[2]; } else ey = yr + ny;
      } else if (yr >= ny) {
        if (d.bc[3]) { ey = ny - 1; ty = d.bc[3]; } else ey = yr - ny;
      }
      R v[NF];
      const bool near = near_side(d, col, ey);
      if (near) pull_hg_b<S, R, BIG, IO>(a, d, col, ey, h, g, v[0], v[1], po);
      else pull_hg<S, R, BIG>(a, sources(d, col, ey), h, g, v[0], v[1], po);
      const unsigned s0 = site_at(d, col, ey);
      v[2] = ld<R>(pbase<BIG>(a.ain, A_VXO, ps), pidx<BIG>(A_VXO, ps, s0));
      v[3] = ld<R>(pbase<BIG>(a.ain, A_VYO, ps), pidx<BIG>(A_VYO, ps, s0));
      if constexpr (TH)
        v[4] = near ? pull_U_b<S, R, BIG, IO>(a, d, col, ey, v[1])
                    : pull_U<S, R, BIG>(a, sources(d, col, ey), v[1]);
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        R u = v[f];
        if (ty >= 0) u = ghost_map<R, IO>(a.kp, ty, 1, f, u);
        if (tx >= 0) u = ghost_map<R, IO>(a.kp, tx, 0, f, u);
        ring[f][yr & 3][sc] = u;
      }
    };

    R hC[9], gC[5], poC = R(0);
    for (int k = 0; k < 2; ++k) {
      if (active) {
        R h[9], g[5], po;
        fill(ya - 1 + k, h, g, po);
        if (k == 1) {
#pragma unroll
          for (int i = 0; i < 9; ++i) hC[i] = h[i];
#pragma unroll
          for (int i = 0; i < 5; ++i) gC[i] = g[i];
          poC = po;
        }
      }
    }

    for (int j = ya; j < yb; ++j) {
      SiteIn<R> in;
      Src9 srcj;
      if (interior) {
        if (near_side(d, col, j)) {
          load_site_b<S, R, BIG, TH, IO>(a, d, col, j, in);
          srcj.s[0] = site_at(d, col, j);
        } else {
          srcj = sources(d, col, j);
          load_site<S, R, BIG, TH>(a, srcj, in);
        }
      }
      R hL[9], gL[5], poL = R(0);
      if (active) fill(j + 1, hL, gL, poL);
      __syncthreads();
      if (interior) {
        const int m = (j - 1) & 3, c0 = j & 3, pp = (j + 1) & 3;
        auto rows = [&](int f) { return Rows3<R>{ring[f][m], ring[f][c0], ring[f][pp]}; };
        site_update<S, R, TH>(a, d, srcj, in, hC, gC, poC, rows(0), rows(1), rows(2), rows(3),
                              sc, rows(NF - 1));
      }
#pragma unroll
      for (int i = 0; i < 9; ++i) hC[i] = hL[i];
#pragma unroll
      for (int i = 0; i < 5; ++i) gC[i] = gL[i];
      poC = poL;
    }
    __syncthreads();
  }
}

template <typename S, typename R>
cudaError_t launch_ymarch_bc(const StepArgs<S, R>& a, bool big, int grid, cudaStream_t st) {
  if constexpr (sizeof(S) == sizeof(R)) {
    // a.bc: 1 boundary sides, 2 among them an inlet or an outlet
    auto go = [&](auto io) {
      constexpr bool IO = decltype(io)::value;
      if (big) {
        if (a.thermal) k_step_ymarch_bc<S, R, true, true, IO><<<grid, YM_THREADS, 0, st>>>(a);
        else k_step_ymarch_bc<S, R, true, false, IO><<<grid, YM_THREADS, 0, st>>>(a);
      } else {
        if (a.thermal) k_step_ymarch_bc<S, R, false, true, IO><<<grid, YM_THREADS, 0, st>>>(a);
        else k_step_ymarch_bc<S, R, false, false, IO><<<grid, YM_THREADS, 0, st>>>(a);
      }
    };
    if (a.bc == 2) go(std::true_type{});
    else go(std::false_type{});
    return cudaGetLastError();
  } else {
    return cudaErrorInvalidValue;   // boundaries need FP32 or FP64 storage (checked on the host)
  }
}

template <typename S, typename R>
int ymarch_bc_blocks_per_sm(bool big, bool thermal) {
  int n = 0;
  if constexpr (sizeof(S) == sizeof(R)) {
    if (big) {
      if (thermal)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_ymarch_bc<S, R, true, true, true>, YM_THREADS, 0);
      else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_ymarch_bc<S, R, true, false, true>, YM_THREADS, 0);
    } else {
      if (thermal)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_ymarch_bc<S, R, false, true, true>, YM_THREADS, 0);
      else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_ymarch_bc<S, R, false, false, true>, YM_THREADS, 0);
    }
  }
  return n > 0 ? n : 1;
}

#define PF_BC_INST(S, R)                                                                  \
  template cudaError_t launch_ymarch_bc<S, R>(const StepArgs<S, R>&, bool, int, cudaStream_t); \
  template int ymarch_bc_blocks_per_sm<S, R>(bool, bool);
PF_BC_INST(double, double)
PF_BC_INST(float, float)
PF_BC_INST(__half, float)
PF_BC_INST(__nv_bfloat16, float)

}  // namespace pf
