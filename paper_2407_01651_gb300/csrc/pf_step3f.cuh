// pf_step3f.cuh -- the 3-D two-phase step kernel k_step3f and its device
// helpers (see pf_step3f.cu for the model, the traversal and the C ABI); shared
// by the translation units that instantiate its variants.
#pragma once
#include <cmath>
#include <cstdint>

#include "../../include/pf.h"
#include "pf_d3.cuh"

namespace pf {
namespace d3f {

// column tile of the z-march: TX x TY interior columns and their halo ring
// (the stencil helpers of pf_d3.cuh take rows of HX = TX + 2)
constexpr int TX = d3::TX, TY = 8;
constexpr int HX = TX + 2, HY = TY + 2;
constexpr int NIN = TX * TY;
constexpr int NHALO = HX * HY - NIN;
constexpr int THREADS = (NIN + NHALO + 31) / 32 * 32;
constexpr int MIN_CTAS = 1;
#ifndef PF3F_PREFETCH
#define PF3F_PREFETCH 0   // planes ahead of the z-march warmed in L2 (0: none)
#endif
static_assert(HX == d3::HX, "the stencil helpers assume rows of d3::HX");
using d3::cx7;
using d3::cy7;
using d3::cz7;
using d3::pl;
using d3::w7;
using d3::wrap1;
using d3::wrapm;

// populations (storage type): f 0..18, h 19..37, g_pre 38..44, g_post 45..51,
// s 52..58; auxiliaries (compute type): r, Q_o, phi_o, C_o, v_o (3)
constexpr int F_POP = 0, H_POP = 19, G_PRE = 38, G_POST = 45, S_POP = 52, NPOPF = 59;
constexpr int AX_RR = 0, AX_QO = 1, AX_PHIO = 2, AX_CO = 3, AX_VO = 4, NAUXF = 7;
constexpr int NSTATEF = 66, NFIELDSF = 9;
// thermal mode: temperature populations e after s, the lagged H after v_o, theta
// as a tenth field
constexpr int E_POP = 59, NPOPF_TH = 66, AX_HO = 7, NAUXF_TH = 8, NSTATEF_TH = 74,
              NFIELDSF_TH = 10;
// shared memory of k_step3f: 5 rings (phi, psi, v_o) of 4 planes of the halo tile
// (a sixth ring, of U, in thermal mode), then, for two planes, the 9 pair
// differences h_{2j-1} - h_{2j} of each interior site's streamed CAC populations
template <typename R>
__host__ __device__ constexpr size_t rings_only_bytes(bool th) { return (th ? 6 : 5) * 4 * HY * HX * sizeof(R); }
template <typename R>
__host__ __device__ constexpr size_t ring_bytes(bool th) { return rings_only_bytes<R>(th) + 2 * 9 * NIN * sizeof(R); }

// D3Q19: rest, faces, edges; opposite directions in pairs (2j-1, 2j)
__host__ __device__ constexpr int c19(int i, int a) {
  constexpr int C[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},  {0, -1, 0},
                            {0, 0, 1},  {0, 0, -1},  {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},
                            {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                            {0, 1, 1},  {0, -1, -1}, {0, 1, -1},  {0, -1, 1}};
  return C[i][a];
}
__host__ __device__ constexpr int c2_19(int i) {
  return c19(i, 0) * c19(i, 0) + c19(i, 1) * c19(i, 1) + c19(i, 2) * c19(i, 2);
}
template <typename R>
__device__ __forceinline__ constexpr R w19(int i) {
  return c2_19(i) == 0 ? R(1.0 / 3.0) : (c2_19(i) == 1 ? R(1.0 / 18.0) : R(1.0 / 36.0));
}
// the moments of the NS collision whose rate may differ from 1 (d'Humieres
// rows e, eps, q_x, q_y, q_z, 3p_xx, p_ww, p_xy, p_yz, p_xz, m_x, m_y, m_z)
constexpr int NMOM = 13;
__host__ __device__ constexpr int mrow(int k, int i) {
  const int x = c19(i, 0), y = c19(i, 1), z = c19(i, 2), c2 = c2_19(i);
  switch (k) {
    case 0: return 19 * c2 - 30;
    case 1: return (21 * c2 * c2 - 53 * c2 + 24) / 2;
    case 2: return (5 * c2 - 9) * x;
    case 3: return (5 * c2 - 9) * y;
    case 4: return (5 * c2 - 9) * z;
    case 5: return 3 * x * x - c2;
    case 6: return y * y - z * z;
    case 7: return x * y;
    case 8: return y * z;
    case 9: return x * z;
    case 10: return (y * y - z * z) * x;
    case 11: return (z * z - x * x) * y;
    default: return (x * x - y * y) * z;
  }
}
__host__ __device__ constexpr int mnorm(int k) {
  int s = 0;
  for (int i = 0; i < 19; ++i) s += mrow(k, i) * mrow(k, i);
  return s;
}

template <typename R>
struct CoefF {
  R rl, rg, drho, rho_bar, g, kappa, fs_coef, bphi2, binter2, Wphi2, Mphi;
  R eps, ge2, gat2, four_bpsi, lam, theta, Mcinf, inv_tau0, c4W0sq_tau0, k, inv_omk, D, aW0;
  R s_phi;
  R cm[NMOM];          // (1 - s_k) / |M_k|^2 of the NS moments above
  // thermal mode: c_p, latent / 2, 1/Le, W0^2, s_T and 1 - s_T/2 (k_T = Le D rho_l c_p)
  R cp, halfL, iLe, W0sq, sth, hsth;
  R th0;               // theta at a far-field side
};

// I: the type of site indices and plane offsets (32-bit when planes x sites
// fits, which saves address arithmetic in the pulls; 64-bit otherwise)
template <typename S, typename R, typename I = unsigned long long>
struct ArgsF {
  const S* in;
  S* out;
  const R* ain;
  R* aout;
  R* fields;            // phi, psi, C, U, p, vx, vy, vz, mu planes, or nullptr
  const int* grain;     // ROT: grain index per site
  const R* rot;         // ROT: 9 entries (row-major R) per grain
  int bc[6];            // BC: side types x-, x+, y-, y+, z-, z+ (0 periodic, 1 symmetric,
                        // 2 wall, 3 far field)
  I ps;
  int nx, ny, nz, chunk;
  int tiles_x, tiles_y, tiles_z;
  CoefF<R> c;
};

template <typename S, typename R, typename I>
__device__ __forceinline__ unsigned long long site_of(const ArgsF<S, R, I>& a, int x, int y, int z) {
  return ((I)z * (I)a.ny + (I)y) * (I)a.nx + (I)x;
}
// pull source of D3Q19 direction i (x, y, z in range; one step wraps)
// (the site's own index plus one offset per axis: the own index and the
// offsets are shared by all directions)
template <typename S, typename R, typename I>
__device__ __forceinline__ unsigned long long src19(const ArgsF<S, R, I>& a, int x, int y, int z, int i) {
  const I own = (I)site_of(a, x, y, z);
  return own + d3::step_off<I>(c19(i, 0), x, a.nx, I(1)) + d3::step_off<I>(c19(i, 1), y, a.ny, (I)a.nx) +
         d3::step_off<I>(c19(i, 2), z, a.nz, (I)a.nx * (I)a.ny);
}
template <typename S, typename R, typename I>
__device__ __forceinline__ unsigned long long src7(const ArgsF<S, R, I>& a, int x, int y, int z, int i) {
  const I own = (I)site_of(a, x, y, z);
  return own + d3::step_off<I>(cx7(i), x, a.nx, I(1)) + d3::step_off<I>(cy7(i), y, a.ny, (I)a.nx) +
         d3::step_off<I>(cz7(i), z, a.nz, (I)a.nx * (I)a.ny);
}

// D3Q19 index of the velocity (cx, cy, cz)
__host__ __device__ constexpr int idx19(int x, int y, int z) {
  for (int j = 0; j < 19; ++j)
    if (c19(j, 0) == x && c19(j, 1) == y && c19(j, 2) == z) return j;
  return 0;
}
__host__ __device__ constexpr int opp19(int i) { return i == 0 ? 0 : (i % 2 ? i + 1 : i - 1); }

// BC: pull source of D3Q19 direction i at (x, y, z): periodic sides wrap, a
// symmetric side reflects the source site and the direction's normal
// component, a wall or far-field side returns the site's own opposite
// population (a bounce wins over a reflection).
template <typename S, typename R, bool BC, typename I>
__device__ __forceinline__ unsigned long long pull19(const ArgsF<S, R, I>& a, int x, int y, int z, int i,
                                                     int& q) {
  if constexpr (BC) {
    int X[3] = {x - c19(i, 0), y - c19(i, 1), z - c19(i, 2)};
    int c[3] = {c19(i, 0), c19(i, 1), c19(i, 2)};
    const int L[3] = {a.nx, a.ny, a.nz};
    bool bounce = false;
#pragma unroll
    for (int d = 0; d < 3; ++d)
      if (X[d] < 0 || X[d] >= L[d]) {
        const int t = a.bc[2 * d + (X[d] < 0 ? 0 : 1)];
        if (t == 0) X[d] = X[d] < 0 ? X[d] + L[d] : X[d] - L[d];
        else if (t == 1) { X[d] = X[d] < 0 ? -1 - X[d] : 2 * L[d] - 1 - X[d]; c[d] = -c[d]; }
        else bounce = true;
      }
    if (bounce) {
      q = opp19(i);
      return site_of(a, x, y, z);
    }
    q = idx19(c[0], c[1], c[2]);
    return site_of(a, X[0], X[1], X[2]);
  } else {
    q = i;
    return src19(a, x, y, z, i);
  }
}

// BC: D3Q7 pull (axis directions): a symmetric side and a wall both give the
// site's own opposite population (mode 1), a far-field side its anti-bounce-back
// (mode 2).
__device__ __forceinline__ constexpr int opp7f(int i) { return i == 0 ? 0 : (i % 2 ? i + 1 : i - 1); }
template <typename S, typename R, bool BC, typename I>
__device__ __forceinline__ int pull7(const ArgsF<S, R, I>& a, int x, int y, int z, int i,
                                     unsigned long long& src, int& q) {
  if constexpr (BC) {
    const int X = x - cx7(i), Y = y - cy7(i), Z = z - cz7(i);
    int t = 0;
    if (X < 0) t = a.bc[0]; else if (X >= a.nx) t = a.bc[1];
    else if (Y < 0) t = a.bc[2]; else if (Y >= a.ny) t = a.bc[3];
    else if (Z < 0) t = a.bc[4]; else if (Z >= a.nz) t = a.bc[5];
    if (t) {
      src = site_of(a, x, y, z);
      q = opp7f(i);
      return t == 3 ? 2 : 1;
    }
  }
  src = src7(a, x, y, z, i);
  q = i;
  return 0;
}

// Streamed D3Q7 populations (plane base P) at (x, y, z); far: the far-field value
template <typename S, typename R, bool BC, typename I>
__device__ __forceinline__ void stream7f(const ArgsF<S, R, I>& a, int P, int x, int y, int z, R f[7],
                                         R far) {
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    unsigned long long src;
    int q;
    const int mode = pull7<S, R, BC>(a, x, y, z, i, src, q);
    f[i] = ld<R>(pl(a.in, P + q, a.ps), src);
    if (BC && mode == 2) f[i] = -f[i] + R(2) * w7<R>(i) * far;
  }
}

// BC: coordinate of a ring column or plane c on an axis of n sites with sides
// t0 / t1: in range as is, wrapped at periodic sides, else the mirror site
// (clamped: columns further out are never read); t returns the side crossed.
__device__ __forceinline__ int side_coord(int c, int n, int t0, int t1, int& t) {
  t = 0;
  if (c >= 0 && c < n) return c;
  const int tt = c < 0 ? t0 : t1;
  if (tt == 0) return wrapm(c, n);
  if (c == -1 || c == n) t = tt;
  const int m = c < 0 ? -1 - c : 2 * n - 1 - c;
  return m < 0 ? 0 : (m >= n ? n - 1 : m);
}

// phi = sum of the streamed h at (x, y, z); with pd (stride ps), also the 9
// pair differences h_{2j-1} - h_{2j} that the CAC collision takes
template <typename S, typename R, bool BC, typename I>
__device__ __forceinline__ R stream_phi(const ArgsF<S, R, I>& a, int x, int y, int z,
                                        R* pd = nullptr, int pstride = 0) {
  CSum<R> s;
  R hodd = R(0);
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    int q;
    const unsigned long long src = pull19<S, R, BC>(a, x, y, z, i, q);
    const R hv = ld<R>(pl(a.in, H_POP + q, a.ps), src);
    s.add(hv);
    if (i & 1) hodd = hv;
    else if (i > 0 && pd) pd[(i / 2 - 1) * pstride] = hodd - hv;
  }
  return s.value();
}

// streamed g with the time stretch, psi and psi_o (as in the melt-only step)
template <typename S, typename R, bool BC, typename I>
__device__ __forceinline__ void stream_g(const ArgsF<S, R, I>& a, int x, int y, int z, R g[7],
                                         R& psi, R& psio) {
  const unsigned long long own = site_of(a, x, y, z);
  CSum<R> sg;
  R po = R(0);
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    unsigned long long src;
    int q;
    const int mode = pull7<S, R, BC>(a, x, y, z, i, src, q);
    const R gold = ld<R>(pl(a.in, G_PRE + i, a.ps), own);
    R gpo = ld<R>(pl(a.in, G_POST + q, a.ps), src);
    if (BC && mode == 2) gpo = -gpo + R(2) * w7<R>(i) * R(-1);     // psi_far = -1
    const R rr = pl(a.ain, AX_RR, a.ps)[src];
    g[i] = gold + (gpo - gold) * rr;
    sg.add(g[i]);
    po += gold;
  }
  psi = sg.value();
  psio = po;
}

// U = (2C/A - 1)/(1-k) of the streamed solute at (x, y, z), for the U ring
template <typename S, typename R, bool BC, typename I>
__device__ __forceinline__ R stream_U(const ArgsF<S, R, I>& a, int x, int y, int z, R psi) {
  CSum<R> cs;
  R sv[7];
  stream7f<S, R, BC>(a, S_POP, x, y, z, sv, R(1));
#pragma unroll
  for (int i = 0; i < 7; ++i) cs.add(sv[i]);
  const R A = (R(1) + a.c.k) - (R(1) - a.c.k) * psi;
  return (R(2) * cs.value() * frcp(A) - R(1)) * a.c.inv_omk;
}

// BC: non-periodic sides (pull19, pull7, side_coord): ghost ring columns and
// planes take the mirror site's values, mapped per side (psi and U across a far
// side, the velocity's normal component at a symmetric side and all of it at a
// wall or far side).
template <typename S, typename R, bool ROT, bool TH, bool BC, typename I = unsigned long long>
__global__ void __launch_bounds__(THREADS, MIN_CTAS) k_step3f(ArgsF<S, R, I> a) {
  // rings of phi, psi, v_o (and U) (dynamic: 54 KB in FP64)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R (*rphi)[HY][HX] = reinterpret_cast<R (*)[HY][HX]>(smem_raw);
  R (*rpsi)[HY][HX] = rphi + 4;
  R (*rv0)[HY][HX] = rphi + 8;
  R (*rv[3])[HY][HX] = {rv0, rv0 + 4, rv0 + 8};
  R (*rU)[HY][HX] = rphi + 20;         // TH only
  // pair differences of the streamed h of interior site t, plane z in [z & 1]
  R (*hd)[9][NIN] = reinterpret_cast<R (*)[9][NIN]>(smem_raw + rings_only_bytes<R>(TH));
  const int t = threadIdx.x;
  int hx = 0, hy = 0;
  const bool interior = t < NIN;
  if (interior) {
    hx = 1 + t % TX;
    hy = 1 + t / TX;
  } else if (t < NIN + NHALO) {
    const int h = t - NIN;            // halo ring: bottom row, top row, left, right
    if (h < HX) { hx = h; hy = 0; }
    else if (h < 2 * HX) { hx = h - HX; hy = HY - 1; }
    else if (h < 2 * HX + TY) { hx = 0; hy = 1 + h - 2 * HX; }
    else { hx = HX - 1; hy = 1 + h - 2 * HX - TY; }
  }
  const bool active = t < NIN + NHALO;
  const int ntiles = a.tiles_x * a.tiles_y * a.tiles_z;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int tx = tile % a.tiles_x, ty = (tile / a.tiles_x) % a.tiles_y;
    const int tz = tile / (a.tiles_x * a.tiles_y);
    const int za = tz * a.chunk, zb = min(za + a.chunk, a.nz);
    int x, y, sx = 0, sy = 0;      // column, and the side a ghost column lies beyond
    if constexpr (BC) {
      x = side_coord(tx * TX + hx - 1, a.nx, a.bc[0], a.bc[1], sx);
      y = side_coord(ty * TY + hy - 1, a.ny, a.bc[2], a.bc[3], sy);
    } else {
      x = wrapm(tx * TX + hx - 1, a.nx);
      y = wrapm(ty * TY + hy - 1, a.ny);
    }
    const bool mine = interior && tx * TX + hx - 1 < a.nx && ty * TY + hy - 1 < a.ny;
    // ghost maps of a ring value: kind 1 psi, 2 U, 3..5 velocity component
    auto gmap = [&](R v, int kind, int sz) {
      if constexpr (BC) {
        const int ts[3] = {sx, sy, sz};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const int t = ts[d];
          if (!t) continue;
          if (kind == 1 && t == 3) v = R(-2) - v;
          else if (kind == 2 && t == 3) v = -v;
          else if (kind >= 3 && (t != 1 || kind - 3 == d)) v = -v;
        }
      }
      return v;
    };
    R gC[7], gL[7], poC = R(0), poL = R(0);
    // ring planes za-1 and za
    for (int k = 0; k < 2; ++k) {
      if (active) {
        int sz = 0;
        const int z = BC ? side_coord(za - 1 + k, a.nz, a.bc[4], a.bc[5], sz) : wrap1(za - 1 + k, a.nz);
        const int slot = (za - 1 + k) & 3;
        R g[7], psi, po;
        stream_g<S, R, BC>(a, x, y, z, g, psi, po);
        rpsi[slot][hy][hx] = gmap(psi, 1, sz);
        rphi[slot][hy][hx] = stream_phi<S, R, BC>(a, x, y, z, mine ? &hd[(za - 1 + k) & 1][0][t] : nullptr, NIN);
        const unsigned long long s0 = site_of(a, x, y, z);
#pragma unroll
        for (int c = 0; c < 3; ++c) rv[c][slot][hy][hx] = gmap(pl(a.ain, AX_VO + c, a.ps)[s0], 3 + c, sz);
        if constexpr (TH) rU[slot][hy][hx] = gmap(stream_U<S, R, BC>(a, x, y, z, psi), 2, sz);
        if (k == 1) {
#pragma unroll
          for (int i = 0; i < 7; ++i) gC[i] = g[i];
          poC = po;
        }
      }
    }
    for (int z = za; z < zb; ++z) {
      const unsigned long long site = site_of(a, x, y, z);
      R sv[7], Qo = R(0), phio = R(0), Co = R(0), vo[3] = {R(0), R(0), R(0)};
      if (active) {
        int sz = 0;
        const int zn = BC ? side_coord(z + 1, a.nz, a.bc[4], a.bc[5], sz) : wrap1(z + 1, a.nz);
        const int slot = (z + 1) & 3;
        R psi;
        stream_g<S, R, BC>(a, x, y, zn, gL, psi, poL);
        rpsi[slot][hy][hx] = gmap(psi, 1, sz);
        rphi[slot][hy][hx] = stream_phi<S, R, BC>(a, x, y, zn, mine ? &hd[(z + 1) & 1][0][t] : nullptr, NIN);
        const unsigned long long sn = site_of(a, x, y, zn);
#pragma unroll
        for (int c = 0; c < 3; ++c) rv[c][slot][hy][hx] = gmap(pl(a.ain, AX_VO + c, a.ps)[sn], 3 + c, sz);
        if constexpr (TH) rU[slot][hy][hx] = gmap(stream_U<S, R, BC>(a, x, y, zn, psi), 2, sz);
      }
      // the site's own streamed s and lagged scalars: needed after the barrier
      // only, so issued after the fill whose loads the barrier waits on
      if (mine) {
        stream7f<S, R, BC>(a, S_POP, x, y, z, sv, R(1));
        Qo = pl(a.ain, AX_QO, a.ps)[site];
        phio = pl(a.ain, AX_PHIO, a.ps)[site];
        Co = pl(a.ain, AX_CO, a.ps)[site];
        if constexpr (PF3F_PREFETCH > 0) {
          // warm L2 with this column's planes PF3F_PREFETCH planes ahead (one
          // instruction per plane and warp; no register holds the data)
          const int z2 = z + PF3F_PREFETCH < a.nz ? z + PF3F_PREFETCH : z + PF3F_PREFETCH - a.nz;
          const unsigned long long pf2 = site_of(a, x, y, z2);
          constexpr int NP = TH ? NPOPF_TH : NPOPF, NA = TH ? NAUXF_TH : NAUXF;
#pragma unroll
          for (int q = 0; q < NP; ++q) d3::prefetch_l2(pl(a.in, q, a.ps) + pf2);
#pragma unroll
          for (int q = 0; q < NA; ++q) d3::prefetch_l2(pl(a.ain, q, a.ps) + pf2);
        }
      }
      // the streamed f of this plane, issued before the barrier so that their
      // latency overlaps the wait and the stencils (FP32 periodic kernels; in
      // the boundary and FP64 variants the registers they hold there cost spills)
      R fv[19];
      auto pull_f = [&]() {
#pragma unroll
        for (int i = 0; i < 19; ++i) {
          int qf;
          const unsigned long long sf = pull19<S, R, BC>(a, x, y, z, i, qf);
          fv[i] = ld<R>(pl(a.in, F_POP + qf, a.ps), sf);
        }
      };
      constexpr bool EARLY_F = !BC && sizeof(R) == 4;
      R ev[7], Ho = R(0);   // TH: streamed temperature populations, lagged H
      if constexpr (EARLY_F) {
        if (mine) {
          pull_f();
          if constexpr (TH) {
            stream7f<S, R, BC>(a, E_POP, x, y, z, ev, a.c.th0);
            Ho = pl(a.ain, AX_HO, a.ps)[site];
          }
        }
      }
      __syncthreads();
      if (mine) {
        const CoefF<R>& c = a.c;
        const int sm = (z - 1) & 3, s0 = z & 3, sp = (z + 1) & 3;
        const R phi = rphi[s0][hy][hx], psi = rpsi[s0][hy][hx];
#pragma unroll
        for (int q = 0; q < 3; ++q) vo[q] = rv[q][s0][hy][hx];
        // stencils
        R gp[3], gs[3], dv[3][3];
        d3::grad18<R>(rphi[sm], rphi[s0], rphi[sp], hy, hx, gp[0], gp[1], gp[2]);
        const R lphi = d3::lap18<R>(rphi[sm], rphi[s0], rphi[sp], hy, hx);
        d3::grad18<R>(rpsi[sm], rpsi[s0], rpsi[sp], hy, hx, gs[0], gs[1], gs[2]);
#pragma unroll
        for (int q = 0; q < 3; ++q)
          d3::grad18<R>(rv[q][sm], rv[q][s0], rv[q][sp], hy, hx, dv[q][0], dv[q][1], dv[q][2]);
        // gas-liquid interface
        const R rho = c.rg + phi * c.drho;
        const R gr[3] = {c.drho * gp[0], c.drho * gp[1], c.drho * gp[2]};
        const R igm = frsqrt(gp[0] * gp[0] + gp[1] * gp[1] + gp[2] * gp[2] + c.ge2);
        const R nf[3] = {gp[0] * igm, gp[1] * igm, gp[2] * igm};
        const R opsi = R(1) + psi;
        const R mu = c.bphi2 * phi * (R(1) - phi) * (R(1) - R(2) * phi) -
                     c.binter2 * (R(1) - phi) * opsi * opsi - c.Wphi2 * lphi;
        const R aphi = c.kappa * phi * (R(1) - phi);
        R Dm[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) Dm[q] = c.Mphi * (gp[q] - aphi * nf[q]);
        const R divD = (phi - phio) + (vo[0] * gp[0] + vo[1] * gp[1] + vo[2] * gp[2]);
        R Fp[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const R Fm = c.drho * (divD * vo[q] + (Dm[0] * dv[q][0] + Dm[1] * dv[q][1] + Dm[2] * dv[q][2]));
          Fp[q] = c.fs_coef * mu * gp[q] + Fm;
        }
        Fp[1] -= (rho - c.rho_bar) * c.g;
        // NS moments of the pulled f, drag, pressure
        if constexpr (!EARLY_F) pull_f();
        R j[3] = {R(0), R(0), R(0)};
        CSum<R> snz;
#pragma unroll
        for (int i = 0; i < 19; ++i) {
          if (i) snz.add(fv[i]);
          if (c19(i, 0)) j[0] += R(c19(i, 0)) * fv[i];
          if (c19(i, 1)) j[1] += R(c19(i, 1)) * fv[i];
          if (c19(i, 2)) j[2] += R(c19(i, 2)) * fv[i];
        }
        const R chi = R(0.5) * opsi;
        const R irho = frcp(rho);
        R v[3], F[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const R vs = (j[q] + R(0.5) * Fp[q]) * irho;
          v[q] = (R(1) - chi) * vs;
          F[q] = Fp[q] - R(2) * chi * rho * vs;
        }
        const R v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        // p = c_s^2 / (1 - w0) [sum_{i != 0} f_i + v.grad(rho)/2 - w0 rho v^2 / (2 c_s^2)]
        const R pr = R(0.5) * (snz.value() + R(0.5) * (v[0] * gr[0] + v[1] * gr[1] + v[2] * gr[2]) -
                               R(0.5) * rho * v2);
        // NS collision on opposite pairs (2j-1, 2j), c = +-c_j.  With G_i = 3 w_i
        // [c.F + (c.v)(c.grad rho)], f_eq + G/2 = E_j +- O_j where
        //   E_j = w (3p + rho (4.5 cu^2 - 1.5 v^2) + 1.5 cu cg),  O_j = w (3 rho cu + 1.5 cF),
        // and d = f - f_eq + G/2 has the pair sum De_j and difference Do_j.  The
        // even moment rows (e, eps, p's) see only De, the odd ones (q, m) only Do.
        {
          const R w0 = R(1.0 / 3.0);
          R n[NMOM];
#pragma unroll
          for (int k = 0; k < NMOM; ++k) n[k] = R(0);
          const R e0 = w0 * (R(3) * pr - R(1.5) * rho * v2) - R(3) * pr;   // f_eq_0, G_0 = 0
          {
            const R d0 = fv[0] - e0;
#pragma unroll
            for (int k = 0; k < NMOM; ++k)
              if (mrow(k, 0) != 0) n[k] += R(mrow(k, 0)) * d0;
          }
          auto pair_eo = [&](int jp, R& E, R& O) {
            const int i = 2 * jp - 1;
            const R cu = R(c19(i, 0)) * v[0] + R(c19(i, 1)) * v[1] + R(c19(i, 2)) * v[2];
            const R cF = R(c19(i, 0)) * F[0] + R(c19(i, 1)) * F[1] + R(c19(i, 2)) * F[2];
            const R cg = R(c19(i, 0)) * gr[0] + R(c19(i, 1)) * gr[1] + R(c19(i, 2)) * gr[2];
            const R wi = w19<R>(i);
            E = wi * (R(3) * pr + rho * (R(4.5) * cu * cu - R(1.5) * v2) + R(1.5) * cu * cg);
            O = wi * (R(3) * rho * cu + R(1.5) * cF);
            return wi * R(3) * cu * cg;          // G_e: the even part of G (2 x its half)
          };
#pragma unroll
          for (int jp = 1; jp <= 9; ++jp) {
            const int i = 2 * jp - 1;
            R E, O;
            const R Ge = pair_eo(jp, E, O);
            // f_eq = (E - Ge/2) +- (O - Go/2), G/2 = Ge/2 +- Go/2, Go = 3 w cF
            const R Go = w19<R>(i) * R(3) * (R(c19(i, 0)) * F[0] + R(c19(i, 1)) * F[1] +
                                             R(c19(i, 2)) * F[2]);
            const R De = (fv[i] + fv[i + 1]) - R(2) * E + R(2) * Ge;
            const R Do = (fv[i] - fv[i + 1]) - R(2) * O + R(2) * Go;
#pragma unroll
            for (int k = 0; k < NMOM; ++k)
              if (mrow(k, i) != 0) n[k] += R(mrow(k, i)) * (mrow(k, i) == mrow(k, i + 1) ? De : Do);
          }
#pragma unroll
          for (int k = 0; k < NMOM; ++k) n[k] *= c.cm[k];
          {
            R o = e0;
#pragma unroll
            for (int k = 0; k < NMOM; ++k)
              if (mrow(k, 0) != 0) o += R(mrow(k, 0)) * n[k];
            st<S, R>(pl(a.out, F_POP, a.ps), site, o);
          }
#pragma unroll
          for (int jp = 1; jp <= 9; ++jp) {
            const int i = 2 * jp - 1;
            R E, O;
            pair_eo(jp, E, O);
#pragma unroll
            for (int k = 0; k < NMOM; ++k) {
              if (mrow(k, i) == 0) continue;
              if (mrow(k, i) == mrow(k, i + 1)) E += R(mrow(k, i)) * n[k];
              else O += R(mrow(k, i)) * n[k];
            }
            st<S, R>(pl(a.out, F_POP + i, a.ps), site, E + O);
            st<S, R>(pl(a.out, F_POP + i + 1, a.ps), site, E - O);
          }
        }
        // CAC collision: h_eq = w phi (1 + 3 c.v), G_i = 3 w c.G1 with G1 =
        // d_t(phi v) + c_s^2 kappa phi (1-phi) n; fluxes at s_phi, the rest at 1.
        // On pairs: h_eq + G/2 = w phi +- O_j, O_j = w (3 phi cu + 1.5 cG); the
        // flux of d = h - h_eq + G/2 is sum_j c_j [(h+ - h-) - 2 w (3 phi cu - 1.5 cG)].
        {
          R G1[3];
#pragma unroll
          for (int q = 0; q < 3; ++q) G1[q] = (phi * v[q] - phio * vo[q]) + R(1.0 / 3.0) * aphi * nf[q];
          R nj[3] = {R(0), R(0), R(0)};
#pragma unroll
          for (int jp = 1; jp <= 9; ++jp) {
            const int i = 2 * jp - 1;
            // h_i - h_{i+1} of this site, kept by the ring fill of plane z
            const R dh = hd[z & 1][jp - 1][t];
            const R cu = R(c19(i, 0)) * v[0] + R(c19(i, 1)) * v[1] + R(c19(i, 2)) * v[2];
            const R cG = R(c19(i, 0)) * G1[0] + R(c19(i, 1)) * G1[1] + R(c19(i, 2)) * G1[2];
            const R Do = dh - R(2) * w19<R>(i) * (R(3) * phi * cu - R(1.5) * cG);
            if (c19(i, 0)) nj[0] += R(c19(i, 0)) * Do;
            if (c19(i, 1)) nj[1] += R(c19(i, 1)) * Do;
            if (c19(i, 2)) nj[2] += R(c19(i, 2)) * Do;
          }
          const R cj = (R(1) - c.s_phi) * R(0.1);           // |row j|^2 = 10
#pragma unroll
          for (int q = 0; q < 3; ++q) nj[q] *= cj;
          // h*_i = w_i phi + (odd part).  The even bases are b = phi/36 (edges)
          // and 2b (faces), b rounded to a multiple of ulp(phi)/8, so that the
          // rest population phi - 24 b is exact (one FMA) and h* sums to phi
          // exactly: otherwise a uniform bulk, where every site rounds w_i phi
          // the same way, would change sum phi by a fixed fraction per step.
          const R b = round_to_multiple(phi * R(1.0 / 36.0), R(0.5) * quantum_quarter_ulp(phi));
          st<S, R>(pl(a.out, H_POP, a.ps), site, fma(R(-24), b, phi));
#pragma unroll
          for (int jp = 1; jp <= 9; ++jp) {
            const int i = 2 * jp - 1;
            const R cu = R(c19(i, 0)) * v[0] + R(c19(i, 1)) * v[1] + R(c19(i, 2)) * v[2];
            const R cG = R(c19(i, 0)) * G1[0] + R(c19(i, 1)) * G1[1] + R(c19(i, 2)) * G1[2];
            R odd = w19<R>(i) * (R(3) * phi * cu + R(1.5) * cG);
            if (c19(i, 0)) odd += R(c19(i, 0)) * nj[0];
            if (c19(i, 1)) odd += R(c19(i, 1)) * nj[1];
            if (c19(i, 2)) odd += R(c19(i, 2)) * nj[2];
            const R base = c2_19(i) == 1 ? R(2) * b : b;
            st<S, R>(pl(a.out, H_POP + i, a.ps), site, base + odd);
            st<S, R>(pl(a.out, H_POP + i + 1, a.ps), site, base - odd);
          }
        }
        // dendrite geometry, sources (anisotropy summed over three axes)
        const R gm2 = gs[0] * gs[0] + gs[1] * gs[1] + gs[2] * gs[2];
        const R im = frsqrt(gm2 + c.ge2);
        const R m = (gm2 + c.ge2) * im;
        R gc0 = gs[0], gc1 = gs[1], gc2 = gs[2];
        const R* Rm = nullptr;
        if constexpr (ROT) {
          Rm = a.rot + 9 * a.grain[site];
          gc0 = Rm[0] * gs[0] + Rm[3] * gs[1] + Rm[6] * gs[2];
          gc1 = Rm[1] * gs[0] + Rm[4] * gs[1] + Rm[7] * gs[2];
          gc2 = Rm[2] * gs[0] + Rm[5] * gs[1] + Rm[8] * gs[2];
        }
        const R n0 = -gc0 * im, n1 = -gc1 * im, n2v = -gc2 * im;
        const R q0 = n0 * n0, q1 = n1 * n1, q2 = n2v * n2v;
        const R n2 = q0 + q1 + q2, s4 = q0 * q0 + q1 * q1 + q2 * q2;
        const R as = R(1) + c.eps * (R(4) * s4 - R(3) * n2 * n2);
        const R iso = s4 + R(0.75) * n2 * (R(1) - n2);
        const R pre = R(-16) * c.eps * as * m;
        R Nx = pre * n0 * (q0 - iso), Ny = pre * n1 * (q1 - iso), Nz = pre * n2v * (q2 - iso);
        if constexpr (ROT) {
          const R Ncx = Nx, Ncy = Ny, Ncz = Nz;
          Nx = Rm[0] * Ncx + Rm[1] * Ncy + Rm[2] * Ncz;
          Ny = Rm[3] * Ncx + Rm[4] * Ncy + Rm[5] * Ncz;
          Nz = Rm[6] * Ncx + Rm[7] * Ncy + Rm[8] * Ncz;
        }
        const R as2 = as * as, ias2 = frcp(as2);
        CSum<R> cs;
#pragma unroll
        for (int i = 0; i < 7; ++i) cs.add(sv[i]);
        const R C = cs.value();
        const R omk = R(1) - c.k;
        const R A = (R(1) + c.k) - omk * psi;
        const R iA = frcp(A);
        const R U = (R(2) * C * iA - R(1)) * c.inv_omk;
        const R omp2 = R(1) - psi * psi;
        // TH: rho H = sum e, theta from the local density
        R rhoH = R(0), theta = c.theta, iF = R(1);
        if constexpr (TH) {
          if constexpr (!EARLY_F) stream7f<S, R, BC>(a, E_POP, x, y, z, ev, c.th0);
          CSum<R> ce;
#pragma unroll
          for (int i = 0; i < 7; ++i) ce.add(ev[i]);
          rhoH = ce.value();
          theta = rhoH * frcp(rho * c.cp) + c.halfL * opsi;
        }
        R Q = c.four_bpsi * psi * omp2 - c.binter2 * (R(1) - phi) * (R(1) - phi) * opsi -
              c.lam * omp2 * omp2 * (theta + c.Mcinf * U);
        if constexpr (TH) {
          R ux, uy, uz;
          d3::grad18<R>(rU[sm], rU[s0], rU[sp], hy, hx, ux, uy, uz);
          iF = frcp(c.iLe + c.Mcinf * (R(1) + omk * U));
          const R dot = c.Mcinf * omk *
                        (ux * (as2 * gs[0] + Nx) + uy * (as2 * gs[1] + Ny) + uz * (as2 * gs[2] + Nz));
          Q = Q * iF + c.W0sq * iF * iF * dot;
        }
        const R at = -c.aW0 * as * (R(1) + omk * U) * (psi - poC) * frsqrt(gm2 + c.gat2);
        // psi: D3Q7 as in the melt-only step
        {
          const R m0 = psi + (Q + R(0.5) * (Q - Qo)) * c.inv_tau0;
          const R s1 = frcp(c.c4W0sq_tau0 * as2 * iF + R(0.5));
          const R hs = R(1) - R(0.5) * s1;
          const R Jx = gC[1] - gC[2], Jy = gC[3] - gC[4], Jz = gC[5] - gC[6];
          const R gq = R(-0.25) * ias2;
          const R Sx = fma(hs, gq * Nx, Jx - s1 * Jx), Sy = fma(hs, gq * Ny, Jy - s1 * Jy),
                  Sz = fma(hs, gq * Nz, Jz - s1 * Jz);
          const R b = m0 * R(0.125);
          R go[7];
          go[0] = fma(R(-6), b, m0);           // m0 - 6 m0/8 = m0/4, exact
          go[1] = fma(R(0.5), Sx, b); go[2] = fma(R(-0.5), Sx, b);
          go[3] = fma(R(0.5), Sy, b); go[4] = fma(R(-0.5), Sy, b);
          go[5] = fma(R(0.5), Sz, b); go[6] = fma(R(-0.5), Sz, b);
#pragma unroll
          for (int i = 0; i < 7; ++i) {
            st<S, R>(pl(a.out, G_PRE + i, a.ps), site, gC[i]);
            st<S, R>(pl(a.out, G_POST + i, a.ps), site, go[i]);
          }
          pl(a.aout, AX_RR, a.ps)[site] = ias2;
          pl(a.aout, AX_QO, a.ps)[site] = Q;
        }
        // solute: D3Q7; equilibrium flux C v - E grad psi + (1-k)(J_at + J),
        // J = D q C kappa (1-phi) n_phi; G = w c . d_t(C v) / c_s^2 through
        // (I - S/2); rate from D_C = 2 D q / A = (1/s - 1/2) c_s^2
        {
          const R qf = R(0.5) * (R(1) - psi);
          const R E = R(2) * omk * c.D * qf * C * iA * iA;
          const R DC = R(2) * c.D * qf * iA;
          const R sc = frcp(R(4) * DC + R(0.5));
          const R jv = c.D * qf * C * c.kappa * (R(1) - phi);
          const R hsc = R(1) - R(0.5) * sc;
          R Sf[3];
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            const R Jeq = C * v[q] - E * gs[q] + omk * (at * gs[q] + jv * nf[q]);
            const R Jq = sv[2 * q + 1] - sv[2 * q + 2];
            Sf[q] = Jq - sc * (Jq - Jeq) + hsc * (C * v[q] - Co * vo[q]);
          }
          const R b = C * R(0.125);
          R so[7];
          so[0] = fma(R(-6), b, C);            // C - 6 C/8 = C/4, exact
          so[1] = fma(R(0.5), Sf[0], b); so[2] = fma(R(-0.5), Sf[0], b);
          so[3] = fma(R(0.5), Sf[1], b); so[4] = fma(R(-0.5), Sf[1], b);
          so[5] = fma(R(0.5), Sf[2], b); so[6] = fma(R(-0.5), Sf[2], b);
#pragma unroll
          for (int i = 0; i < 7; ++i) st<S, R>(pl(a.out, S_POP + i, a.ps), site, so[i]);
        }
        // TH: temperature collision, D3Q7: equilibrium flux j = rho H v, G = w c .
        // d_t(rho H v) / c_s^2 (backward difference) through (I - S/2), flux rate
        // s_T, the rest at 1; base theta/8 rounded to a multiple of ulp(rho H)/2 so
        // that the rest population rho H - 6 theta/8 is exact in the common case
        if constexpr (TH) {
          const R rho_o = c.rg + phio * c.drho;
          if constexpr (!EARLY_F) Ho = pl(a.ain, AX_HO, a.ps)[site];
          R Sf[3];
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            const R jq = rhoH * v[q];
            const R Jq = ev[2 * q + 1] - ev[2 * q + 2];
            Sf[q] = Jq - c.sth * (Jq - jq) + c.hsth * (jq - rho_o * Ho * vo[q]);
          }
          const R b = round_to_multiple(theta * R(0.125), R(2) * quantum_quarter_ulp(rhoH));
          R eo[7];
          eo[0] = fma(R(-6), b, rhoH);
          eo[1] = fma(R(0.5), Sf[0], b); eo[2] = fma(R(-0.5), Sf[0], b);
          eo[3] = fma(R(0.5), Sf[1], b); eo[4] = fma(R(-0.5), Sf[1], b);
          eo[5] = fma(R(0.5), Sf[2], b); eo[6] = fma(R(-0.5), Sf[2], b);
#pragma unroll
          for (int i = 0; i < 7; ++i) st<S, R>(pl(a.out, E_POP + i, a.ps), site, eo[i]);
          pl(a.aout, AX_HO, a.ps)[site] = rhoH * irho;
        }
        pl(a.aout, AX_PHIO, a.ps)[site] = phi;
        pl(a.aout, AX_CO, a.ps)[site] = C;
#pragma unroll
        for (int q = 0; q < 3; ++q) pl(a.aout, AX_VO + q, a.ps)[site] = v[q];
        if (a.fields) {
          const R vals[NFIELDSF] = {phi, psi, C, U, pr, v[0], v[1], v[2], mu};
#pragma unroll
          for (int f = 0; f < NFIELDSF; ++f) pl(a.fields, f, a.ps)[site] = vals[f];
          if constexpr (TH) pl(a.fields, NFIELDSF, a.ps)[site] = theta;
        }
      }
#pragma unroll
      for (int i = 0; i < 7; ++i) gC[i] = gL[i];
      poC = poL;
    }
    __syncthreads();
  }
}

// One step launch over all tiles (dynamic shared memory smem): the variant for
// the thermal and rotated modes, with sides (BC) or periodic, in index type I.
// Each set of (BC, I) is instantiated in one translation unit.
template <typename S, typename R, bool BC, typename I>
cudaError_t launch3f(const ArgsF<S, R, I>& a, bool rotated, bool thermal, int tiles, size_t smem,
                     cudaStream_t st) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaSuccess;
    auto big = [&](auto kern) {
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    };
    big(k_step3f<S, R, false, false, BC, I>);
    big(k_step3f<S, R, true, false, BC, I>);
    big(k_step3f<S, R, false, true, BC, I>);
    big(k_step3f<S, R, true, true, BC, I>);
    if (e != cudaSuccess) return e;
  }
  if (thermal) {
    if (rotated) k_step3f<S, R, true, true, BC, I><<<tiles, THREADS, smem, st>>>(a);
    else k_step3f<S, R, false, true, BC, I><<<tiles, THREADS, smem, st>>>(a);
  } else {
    if (rotated) k_step3f<S, R, true, false, BC, I><<<tiles, THREADS, smem, st>>>(a);
    else k_step3f<S, R, false, false, BC, I><<<tiles, THREADS, smem, st>>>(a);
  }
  return cudaGetLastError();
}

// instantiated in pf_step3f_bc.cu (sides, 64-bit) and pf_step3f_wide.cu
// (periodic, 64-bit: grids whose plane offsets exceed 32 bits)
#define PF3F_LAUNCH_SET(EXT, BC, I)                                                              \
  EXT template cudaError_t launch3f<float, float, BC, I>(const ArgsF<float, float, I>&, bool,    \
                                                         bool, int, size_t, cudaStream_t);      \
  EXT template cudaError_t launch3f<double, double, BC, I>(const ArgsF<double, double, I>&, bool, \
                                                           bool, int, size_t, cudaStream_t);
PF3F_LAUNCH_SET(extern, true, unsigned long long)
PF3F_LAUNCH_SET(extern, false, unsigned long long)

}  // namespace d3f
}  // namespace pf
