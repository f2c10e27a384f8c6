// pf_step3d.cu -- the three-dimensional dendrite step of arXiv 2407.01651
// (Section 2.1 with the anisotropy summed over three axes; the anisotropic
// Allen-Cahn equation with the a_s^2 time stretch of Appendix B and the
// solute equation with antitrapping) on D3Q7 lattices, in a melt without gas
// or flow, and the C ABI of its handle (pf3_* in include/pf.h).
//
// Kernel: k_step3d, a z-march.  A CTA owns a 32 x 8 column tile and walks
// `chunk` planes along z; 256 threads own the interior columns and 84 more
// the halo ring of the tile.  At plane k every thread pulls g of plane k+1 at
// its column (the a_s^2-stretched streaming) and writes psi into a 4-slot
// shared-memory ring; after one barrier the interior threads update plane k
// with the 18-neighbour gradient read from slots k-1, k, k+1.  D3Q7 weights
// w0 = 1/4, wi = 1/8, c_s^2 = 1/4; gradient with D3Q19 weights (1/18 faces,
// 1/36 edges).  Layout: one plane per population, [z][y][x], x fastest.
#include <cmath>
#include <cstdint>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/pf.h"
#include "pf_d3.cuh"

namespace pf {
namespace d3 {

// planes: g_pre 0..6, g_post 7..13, s 14..20, thermal e 21..27 (storage
// type); r, Q_o (compute type)
constexpr int G_PRE = 0, G_POST = 7, S_POP = 14, E_POP = 21, NPOP3 = 21, NPOP3_TH = 28;
constexpr int A3_RR = 0, A3_QO = 1, NAUX3 = 2;
constexpr int NSTATE3 = 23, NSTATE3_TH = 30;      // raw FP64 state planes

template <typename R>
struct Coef3 {
  R eps, ge2, gat2, four_bpsi, lam, theta, Mcinf, inv_tau0, c4W0sq_tau0, k, inv_omk, D, aW0;
  R th0;                // theta at a far-field side
  // thermal mode: rho_l c_p and its inverse, latent / 2, 1/Le, W0^2, 1 - s_T
  R rcp, irc, halfL, iLe, W0sq, omsth;
};

// I: the type of site indices and plane offsets (32-bit when planes x sites
// fits, which saves address arithmetic in the pulls; 64-bit otherwise)
template <typename S, typename R, typename I = unsigned long long>
struct Args3 {
  const S* in;
  S* out;
  const R* ain;
  R* aout;
  R* fields;            // psi, C, U (and theta) planes, or nullptr
  const int* grain;     // ROT: grain index per site
  const R* rot;         // ROT: 9 entries (row-major R) per grain
  int bc[6];            // BC: side types x-, x+, y-, y+, z-, z+ (0 periodic, 1 symmetric,
                        // 2 wall, 3 far field)
  I ps;
  int nx, ny, nz, chunk;
  int tiles_x, tiles_y, tiles_z;
  Coef3<R> c;
};

template <typename S, typename R, typename I>
__device__ __forceinline__ unsigned long long site3(const Args3<S, R, I>& a, int x, int y, int z) {
  return ((I)z * (I)a.ny + (I)y) * (I)a.nx + (I)x;
}
template <typename S, typename R, typename I>
__device__ __forceinline__ unsigned long long src7(const Args3<S, R, I>& a, int x, int y, int z, int i) {
  // x, y, z in range: the own index plus one offset per axis (one step wraps)
  const I own = (I)site3(a, x, y, z);
  return own + d3::step_off<I>(cx7(i), x, a.nx, I(1)) + d3::step_off<I>(cy7(i), y, a.ny, (I)a.nx) +
         d3::step_off<I>(cz7(i), z, a.nz, (I)a.nx * (I)a.ny);
}

// BC: pull source of direction i at (x, y, z): a source beyond a non-periodic
// side is the site's own opposite population, bounced (symmetric side or wall:
// mode 1) or anti-bounced to the far-field value (mode 2); D3Q7 crosses at most
// one side.
__device__ __forceinline__ constexpr int opp7(int i) { return i == 0 ? 0 : (i % 2 ? i + 1 : i - 1); }
template <typename S, typename R, bool BC, typename I>
__device__ __forceinline__ int pull7(const Args3<S, R, I>& a, int x, int y, int z, int i,
                                     unsigned long long& src, int& q) {
  if constexpr (BC) {
    const int X = x - cx7(i), Y = y - cy7(i), Z = z - cz7(i);
    int t = 0;
    if (X < 0) t = a.bc[0]; else if (X >= a.nx) t = a.bc[1];
    else if (Y < 0) t = a.bc[2]; else if (Y >= a.ny) t = a.bc[3];
    else if (Z < 0) t = a.bc[4]; else if (Z >= a.nz) t = a.bc[5];
    if (t) {
      src = site3(a, x, y, z);
      q = opp7(i);
      return t == 3 ? 2 : 1;
    }
  }
  src = src7(a, x, y, z, i);
  q = i;
  return 0;
}

// Streamed g at (x, y, z) (time stretch g = g_pre + r_src (g_post,src - g_pre))
// and psi, psi_o (compensated sums).
template <typename S, typename R, bool BC, typename I>
__device__ __forceinline__ void stream_g(const Args3<S, R, I>& a, int x, int y, int z, R g[7],
                                         R& psi, R& psio) {
  const unsigned long long own = site3(a, x, y, z);
  CSum<R> sg;
  R po = R(0);
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    unsigned long long src;
    int q;
    const int mode = pull7<S, R, BC>(a, x, y, z, i, src, q);
    const R gold = ld<R>(pl(a.in, G_PRE + i, a.ps), own);
    R gpo = ld<R>(pl(a.in, G_POST + q, a.ps), src);
    if (BC && mode == 2) gpo = -gpo + R(2) * w7<R>(i) * R(-1);    // psi_far = -1
    const R rr = ld<R>(pl(a.ain, A3_RR, a.ps), src);
    g[i] = gold + (gpo - gold) * rr;
    sg.add(g[i]);
    po += gold;
  }
  psi = sg.value();
  psio = po;
}

// Streamed populations of one D3Q7 lattice (plane base P) at (x, y, z); far:
// the lattice's far-field value (BC).
template <typename S, typename R, bool BC, typename I>
__device__ __forceinline__ void stream7(const Args3<S, R, I>& a, int P, int x, int y, int z, R f[7],
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

// BC: lattice coordinate of a ring column or plane c of an axis of n sites with
// sides t0 (below) and t1 (above): in range as is, periodic sides wrap, across
// a non-periodic side the mirror site (clamped: columns further out are never
// read); far marks a far-field ghost, whose value is 2 X_far - X.
__device__ __forceinline__ int ghost_coord(int c, int n, int t0, int t1, bool& far) {
  far = false;
  if (c >= 0 && c < n) return c;
  const int t = c < 0 ? t0 : t1;
  if (t == 0) return wrapm(c, n);
  far = t == 3 && (c == -1 || c == n);
  const int m = c < 0 ? -1 - c : 2 * n - 1 - c;
  return m < 0 ? 0 : (m >= n ? n - 1 : m);
}

template <typename R>
__device__ __forceinline__ R sum7(const R f[7]) {
  CSum<R> cs;
#pragma unroll
  for (int i = 0; i < 7; ++i) cs.add(f[i]);
  return cs.value();
}

// U = (2C/A - 1)/(1-k), A = 1+k - (1-k) psi (Eq. eq-u with phi = 1)
template <typename R>
__device__ __forceinline__ R supersat3(const Coef3<R>& c, R C, R psi) {
  const R A = (R(1) + c.k) - (R(1) - c.k) * psi;
  return (R(2) * C * frcp(A) - R(1)) * c.inv_omk;
}

// Resident CTAs per SM of k_step3d: three for the FP32 isothermal aligned-grain
// form with 32-bit indices (56 registers, no spills), else two (80 registers).
template <typename R, bool TH, bool ROT, typename I>
constexpr int ctas3d() { return (!TH && !ROT && sizeof(R) == 4 && sizeof(I) == 4) ? 3 : 2; }

// TH: the temperature lattice of Appendix B on D3Q7 (rho H conserved, theta =
// H / c_p + (c_p^s/c_p) h(psi)), F(U) = 1/Le + M c_inf [1 + (1-k) U] in the
// relaxation of psi, and the source Q / F + W0^2 / F^2 grad F . (a_s^2 grad psi
// + N) with grad F = M c_inf (1-k) grad U; U is kept in a second ring.
// ROT: grain orientations (the site's grain rotation R; the anisotropy is
// evaluated on g' = R^T grad psi and N = R N'(g')).
// BC: non-periodic sides (pull7, ghost_coord): ghost ring columns and planes
// take the mirror site's psi (and U), mapped to 2 X_far - X across a far side.
template <typename S, typename R, bool TH, bool ROT, bool BC, typename I = unsigned long long>
__global__ void __launch_bounds__(THREADS, (ctas3d<R, TH, ROT, I>())) k_step3d(Args3<S, R, I> a) {
  __shared__ R ring[4][HY][HX];
  __shared__ R uring[TH ? 4 : 1][HY][HX];
  const int t = threadIdx.x;
  // column of this thread within the halo tile
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
    bool fx = false, fy = false;
    int x, y;
    if constexpr (BC) {
      x = ghost_coord(tx * TX + hx - 1, a.nx, a.bc[0], a.bc[1], fx);
      y = ghost_coord(ty * TY + hy - 1, a.ny, a.bc[2], a.bc[3], fy);
    } else {
      x = wrapm(tx * TX + hx - 1, a.nx);
      y = wrapm(ty * TY + hy - 1, a.ny);
    }
    const bool mine = interior && tx * TX + hx - 1 < a.nx && ty * TY + hy - 1 < a.ny;
    // ghost maps of the ring values: 2 X_far - X per far-field side crossed
    // (psi_far = -1, U_far = 0)
    auto gpsi = [&](R v, bool fz) {
      if constexpr (BC) {
        if (fx) v = R(-2) - v;
        if (fy) v = R(-2) - v;
        if (fz) v = R(-2) - v;
      }
      return v;
    };
    auto gU = [&](R v, bool fz) {
      if constexpr (BC) {
        if (fx) v = -v;
        if (fy) v = -v;
        if (fz) v = -v;
      }
      return v;
    };
    R gC[7], gL[7], poC = R(0), poL = R(0);
    R sC[7], sL[7], CC = R(0), CL = R(0);   // TH: streamed s and C carried a plane ahead
    // ring planes za-1 and za
    for (int k = 0; k < 2; ++k) {
      if (active) {
        bool fz = false;
        const int z = BC ? ghost_coord(za - 1 + k, a.nz, a.bc[4], a.bc[5], fz) : wrap1(za - 1 + k, a.nz);
        R g[7], psi, po;
        stream_g<S, R, BC>(a, x, y, z, g, psi, po);
        ring[(za - 1 + k) & 3][hy][hx] = gpsi(psi, fz);
        if constexpr (TH) {
          R sv[7];
          stream7<S, R, BC>(a, S_POP, x, y, z, sv, R(1));
          const R C = sum7(sv);
          uring[(za - 1 + k) & 3][hy][hx] = gU(supersat3(a.c, C, psi), fz);
          if (k == 1) {
#pragma unroll
            for (int i = 0; i < 7; ++i) sC[i] = sv[i];
            CC = C;
          }
        }
        if (k == 1) {
#pragma unroll
          for (int i = 0; i < 7; ++i) gC[i] = g[i];
          poC = po;
        }
      }
    }
    for (int z = za; z < zb; ++z) {
      // own inputs of plane z: streamed solute (and temperature) populations
      // and the lagged source
      R sv[7], ev[7], Qo = R(0);
      const unsigned long long site = site3(a, x, y, z);
      if (mine) {
        if constexpr (TH) {
#pragma unroll
          for (int i = 0; i < 7; ++i) sv[i] = sC[i];
          stream7<S, R, BC>(a, E_POP, x, y, z, ev, a.c.th0);
        } else {
          stream7<S, R, BC>(a, S_POP, x, y, z, sv, R(1));
        }
        Qo = ld<R>(pl(a.ain, A3_QO, a.ps), site);
        // warm L2 with this column's populations two planes ahead
        const int z2 = z + 2 >= a.nz ? z + 2 - a.nz : z + 2;
        const unsigned long long pf2 = site3(a, x, y, z2);
        constexpr int NPF = TH ? NPOP3_TH : NPOP3;
#pragma unroll
        for (int q = 0; q < NPF; ++q) prefetch_l2(pl(a.in, q, a.ps) + pf2);
        prefetch_l2(pl(a.ain, A3_RR, a.ps) + pf2);
        prefetch_l2(pl(a.ain, A3_QO, a.ps) + pf2);
      }
      if (active) {
        R psi;
        bool fz = false;
        const int zn = BC ? ghost_coord(z + 1, a.nz, a.bc[4], a.bc[5], fz) : wrap1(z + 1, a.nz);
        stream_g<S, R, BC>(a, x, y, zn, gL, psi, poL);
        ring[(z + 1) & 3][hy][hx] = gpsi(psi, fz);
        if constexpr (TH) {
          stream7<S, R, BC>(a, S_POP, x, y, zn, sL, R(1));
          CL = sum7(sL);
          uring[(z + 1) & 3][hy][hx] = gU(supersat3(a.c, CL, psi), fz);
        }
      }
      __syncthreads();
      if (mine) {
        const Coef3<R>& c = a.c;
        const R psi = ring[z & 3][hy][hx];
        R gx, gy, gz;
        grad18<R>(ring[(z - 1) & 3], ring[z & 3], ring[(z + 1) & 3], hy, hx, gx, gy, gz);
        // anisotropy (three axes), regularised normal, in the crystal frame
        const R gm2 = gx * gx + gy * gy + gz * gz;
        const R im = frsqrt(gm2 + c.ge2);
        const R m = (gm2 + c.ge2) * im;
        R gxc = gx, gyc = gy, gzc = gz;
        const R* Rm = nullptr;
        if constexpr (ROT) {
          Rm = a.rot + 9 * a.grain[site];
          gxc = Rm[0] * gx + Rm[3] * gy + Rm[6] * gz;
          gyc = Rm[1] * gx + Rm[4] * gy + Rm[7] * gz;
          gzc = Rm[2] * gx + Rm[5] * gy + Rm[8] * gz;
        }
        const R n0 = -gxc * im, n1 = -gyc * im, n2v = -gzc * im;
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
        // moments, sources
        const R C = TH ? CC : sum7(sv);
        const R omk = R(1) - c.k;
        const R A = (R(1) + c.k) - omk * psi;
        const R iA = frcp(A);
        const R U = (R(2) * C * iA - R(1)) * c.inv_omk;
        const R omp2 = R(1) - psi * psi;
        R theta = c.theta, m0e = R(0), iF = R(1);
        if constexpr (TH) {
          m0e = sum7(ev);
          theta = m0e * c.irc + c.halfL * (R(1) + psi);
        }
        const R Q = c.four_bpsi * psi * omp2 - c.lam * omp2 * omp2 * (theta + c.Mcinf * U);
        R Qeff = Q;
        if constexpr (TH) {
          R ux, uy, uz;
          grad18<R>(uring[(z - 1) & 3], uring[z & 3], uring[(z + 1) & 3], hy, hx, ux, uy, uz);
          iF = frcp(c.iLe + c.Mcinf * (R(1) + omk * U));
          const R dot = c.Mcinf * omk *
                        (ux * (as2 * gx + Nx) + uy * (as2 * gy + Ny) + uz * (as2 * gz + Nz));
          Qeff = Q * iF + c.W0sq * iF * iF * dot;
        }
        const R at = -c.aW0 * as * (R(1) + omk * U) * (psi - poC) * frsqrt(gm2 + c.gat2);
        // psi: D3Q7, m0 = psi + (Q + (Q - Q_o)/2) / tau0, flux rate s1 from
        // W0^2 a_s^2 / (tau0 F) = (1/s1 - 1/2) c_s^2, forcing flux -c_s^2 N / a_s^2
        {
          const R m0 = psi + (Qeff + R(0.5) * (Qeff - Qo)) * c.inv_tau0;
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
          pl(a.aout, A3_RR, a.ps)[site] = ias2;
          pl(a.aout, A3_QO, a.ps)[site] = Qeff;
        }
        // solute: D3Q7, Jeq = -E grad psi + (1-k) J_at, rate from
        // D_C = 2 D q / A = (1/s - 1/2) c_s^2
        {
          const R qf = R(0.5) * (R(1) - psi);
          const R E = R(2) * omk * c.D * qf * C * iA * iA;
          const R DC = R(2) * c.D * qf * iA;
          const R sc = frcp(R(4) * DC + R(0.5));
          const R coef = omk * at - E;
          const R Ex = coef * gx, Ey = coef * gy, Ez = coef * gz;
          const R Jx = sv[1] - sv[2], Jy = sv[3] - sv[4], Jz = sv[5] - sv[6];
          const R Sx = Jx - sc * (Jx - Ex), Sy = Jy - sc * (Jy - Ey), Sz = Jz - sc * (Jz - Ez);
          const R b = C * R(0.125);
          R so[7];
          so[0] = fma(R(-6), b, C);            // C - 6 C/8 = C/4, exact
          so[1] = fma(R(0.5), Sx, b); so[2] = fma(R(-0.5), Sx, b);
          so[3] = fma(R(0.5), Sy, b); so[4] = fma(R(-0.5), Sy, b);
          so[5] = fma(R(0.5), Sz, b); so[6] = fma(R(-0.5), Sz, b);
#pragma unroll
          for (int i = 0; i < 7; ++i) st<S, R>(pl(a.out, S_POP + i, a.ps), site, so[i]);
        }
        // temperature (TH): at rest the equilibrium is e_0 = rho H - (3/4) theta,
        // e_i = theta / 8; the flux relaxes to 0 at s_T from k_T = (1/s_T - 1/2)
        // c_s^2, every other moment to its equilibrium.  theta/8 is rounded to
        // a multiple of ulp(rho H)/2 so that rho H - 6 (theta/8) is exact in the
        // common case and a uniform region keeps sum rho H to the last bit.
        if constexpr (TH) {
          const R b = round_to_multiple(theta * R(0.125), R(2) * quantum_quarter_ulp(m0e));
          const R Sx = c.omsth * (ev[1] - ev[2]), Sy = c.omsth * (ev[3] - ev[4]),
                  Sz = c.omsth * (ev[5] - ev[6]);
          R eo[7];
          eo[0] = fma(R(-6), b, m0e);
          eo[1] = fma(R(0.5), Sx, b); eo[2] = fma(R(-0.5), Sx, b);
          eo[3] = fma(R(0.5), Sy, b); eo[4] = fma(R(-0.5), Sy, b);
          eo[5] = fma(R(0.5), Sz, b); eo[6] = fma(R(-0.5), Sz, b);
#pragma unroll
          for (int i = 0; i < 7; ++i) st<S, R>(pl(a.out, E_POP + i, a.ps), site, eo[i]);
        }
        if (a.fields) {
          pl(a.fields, 0, a.ps)[site] = psi;
          pl(a.fields, 1, a.ps)[site] = C;
          pl(a.fields, 2, a.ps)[site] = U;
          if constexpr (TH) pl(a.fields, 3, a.ps)[site] = theta;
        }
      }
#pragma unroll
      for (int i = 0; i < 7; ++i) gC[i] = gL[i];
      poC = poL;
      if constexpr (TH) {
#pragma unroll
        for (int i = 0; i < 7; ++i) sC[i] = sL[i];
        CC = CL;
      }
    }
    __syncthreads();
  }
}

// Temperature populations at rest (Appendix B) for theta: rho H = rho_l c_p
// (theta - (c_p^s/c_p) h(psi)), e_0 = rho H - (3/4) theta, e_i = theta / 8;
// the lagged source becomes Q_psi(theta) / F(U); theta is written to the fields.
template <typename S, typename R>
__device__ void write_th3(const Args3<S, R>& a, unsigned long long site, R psi, R C, R theta) {
  const Coef3<R>& c = a.c;
  const R m0 = c.rcp * (theta - c.halfL * (R(1) + psi));
#pragma unroll
  for (int i = 1; i < 7; ++i) st<S, R>(pl(a.out, E_POP + i, a.ps), site, R(0.125) * theta);
  st<S, R>(pl(a.out, E_POP, a.ps), site, m0 - R(0.75) * theta);
  const R U = supersat3(c, C, psi);
  const R omp2 = R(1) - psi * psi;
  const R Q = c.four_bpsi * psi * omp2 - c.lam * omp2 * omp2 * (theta + c.Mcinf * U);
  pl(a.aout, A3_QO, a.ps)[site] = Q / (c.iLe + c.Mcinf * (R(1) + (R(1) - c.k) * U));
  pl(a.fields, 3, a.ps)[site] = theta;
}

// Equilibrium state of a site from psi and C (populations w psi / w C, r = 1,
// lagged source Q_psi), fields written; TH: temperature populations at theta.
template <typename S, typename R, bool TH>
__device__ void write_eq3(const Args3<S, R>& a, unsigned long long site, R psi, R C, R theta) {
  const Coef3<R>& c = a.c;
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    st<S, R>(pl(a.out, G_PRE + i, a.ps), site, w7<R>(i) * psi);
    st<S, R>(pl(a.out, G_POST + i, a.ps), site, w7<R>(i) * psi);
    st<S, R>(pl(a.out, S_POP + i, a.ps), site, w7<R>(i) * C);
  }
  const R omk = R(1) - c.k;
  const R U = (R(2) * C / ((R(1) + c.k) - omk * psi) - R(1)) * c.inv_omk;
  const R omp2 = R(1) - psi * psi;
  pl(a.aout, A3_RR, a.ps)[site] = R(1);
  pl(a.aout, A3_QO, a.ps)[site] = c.four_bpsi * psi * omp2 - c.lam * omp2 * omp2 * (c.theta + c.Mcinf * U);
  pl(a.fields, 0, a.ps)[site] = psi;
  pl(a.fields, 1, a.ps)[site] = C;
  pl(a.fields, 2, a.ps)[site] = U;
  if constexpr (TH) write_th3(a, site, psi, C, theta);
}


template <typename S, typename R, bool TH>
__global__ void k_init3(Args3<S, R> a, const double* seeds, int n_seeds, double R_s, double sq2b,
                        double W0, double k, double theta0) {
  // minimum image along periodic axes, plain distance along bounded ones
  auto off = [&](double d, double L, int t) { return t == 0 ? min_image1(d, L) : d; };
  const unsigned long long n = (unsigned long long)a.nx * a.ny * a.nz;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % a.nx), y = (int)((i / a.nx) % a.ny), z = (int)(i / ((unsigned long long)a.nx * a.ny));
    double psi = -1.0;
    const double far = R_s + 30.0 * W0 / sq2b;
    for (int s = 0; s < n_seeds; ++s) {
      const double dx = off(x - seeds[3 * s], a.nx, a.bc[0]), dy = off(y - seeds[3 * s + 1], a.ny, a.bc[2]);
      const double dz = off(z - seeds[3 * s + 2], a.nz, a.bc[4]);
      const double r2 = dx * dx + dy * dy + dz * dz;
      const double v = r2 > far * far ? -1.0 : tanh(sq2b * (R_s - sqrt(r2)) / W0);
      if (s == 0 || v > psi) psi = v;
    }
    const double C = 1.0 - (1.0 - k) * 0.5 * (1.0 + psi);
    write_eq3<S, R, TH>(a, i, (R)psi, (R)C, (R)theta0);
  }
}

template <typename S, typename R, bool TH>
__global__ void k_set3(Args3<S, R> a, const double* psi, const double* C, double theta0) {
  const unsigned long long n = (unsigned long long)a.nx * a.ny * a.nz;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x)
    write_eq3<S, R, TH>(a, i, (R)psi[i], (R)C[i], (R)theta0);
}

// Temperature field of the initial state (psi and C from the field planes).
template <typename S, typename R>
__global__ void k_settemp3(Args3<S, R> a, const double* theta) {
  const unsigned long long n = (unsigned long long)a.nx * a.ny * a.nz;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x)
    write_th3(a, i, pl(a.fields, 0, a.ps)[i], pl(a.fields, 1, a.ps)[i], (R)theta[i]);
}

template <typename S, typename R>
__global__ void k_state3(const S* pin, const R* ain, unsigned long long ps, unsigned long long n,
                         int thermal, double* out) {
  for (unsigned long long j = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j < n;
       j += (unsigned long long)gridDim.x * blockDim.x) {
    for (int i = 0; i < 7; ++i) {
      out[(0 + i) * n + j] = (double)ld<R>(pl(pin, G_PRE + i, ps), j);
      out[(7 + i) * n + j] = (double)ld<R>(pl(pin, G_POST + i, ps), j);
      out[(15 + i) * n + j] = (double)ld<R>(pl(pin, S_POP + i, ps), j);
    }
    out[14 * n + j] = (double)ain[A3_RR * ps + j];
    out[22 * n + j] = (double)ain[A3_QO * ps + j];
    if (thermal)
      for (int i = 0; i < 7; ++i) out[(23 + i) * n + j] = (double)ld<R>(pl(pin, E_POP + i, ps), j);
  }
}

template <typename R>
__global__ void k_fields3(const R* f, unsigned long long ps, unsigned long long n, int planes,
                          double* out) {
  for (unsigned long long j = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j < planes * n;
       j += (unsigned long long)gridDim.x * blockDim.x)
    out[j] = (double)f[(j / n) * ps + j % n];
}

// FP64 totals: sum C, sum h(psi) = sum (1 + psi) / 2; fixed-order partials.
template <typename R>
__global__ void k_reduce3(const R* f, unsigned long long ps, unsigned long long n, double* part) {
  double a0 = 0.0, a1 = 0.0;
  for (unsigned long long j = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j < n;
       j += (unsigned long long)gridDim.x * blockDim.x) {
    a1 += 0.5 * (1.0 + (double)f[j]);
    a0 += (double)f[ps + j];
  }
  __shared__ double sh[2][256];
  sh[0][threadIdx.x] = a0;
  sh[1][threadIdx.x] = a1;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) { part[2 * blockIdx.x] = sh[0][0]; part[2 * blockIdx.x + 1] = sh[1][0]; }
}
__global__ void k_reduce3_final(const double* part, int nb, int k, double* out) {
  if ((int)threadIdx.x >= k) return;
  double acc = 0.0;
  for (int b = 0; b < nb; ++b) acc += part[k * b + threadIdx.x];
  out[threadIdx.x] = acc;
}

// Thermal totals: sum of the seven temperature populations (rho H), sum theta,
// sum psi; fixed-order partials.
template <typename S, typename R>
__global__ void k_reduce3_th(const S* pin, const R* f, unsigned long long ps, unsigned long long n,
                             double* part) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (unsigned long long j = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j < n;
       j += (unsigned long long)gridDim.x * blockDim.x) {
    for (int i = 0; i < 7; ++i) a0 += (double)ld<R>(pl(pin, E_POP + i, ps), j);
    a1 += (double)f[3 * ps + j];
    a2 += (double)f[j];
  }
  __shared__ double sh[3][256];
  sh[0][threadIdx.x] = a0;
  sh[1][threadIdx.x] = a1;
  sh[2][threadIdx.x] = a2;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) part[3 * blockIdx.x + q] = sh[q][0];
}

}  // namespace d3
}  // namespace pf

using namespace pf;
using namespace pf::d3;

struct pf3_handle {
  pf_params p{};
  pf_precision prec = PF_FP32;
  cudaStream_t stream = nullptr;
  int nx = 0, ny = 0, nz = 0, chunk = 16;
  int index64 = 0;  // periodic step in 64-bit indices at any size
  int thermal = 0, npop = NPOP3, nfields = 3, nstate = NSTATE3;
  int rotated = 0;                // grain orientations set
  int bc[6] = {0, 0, 0, 0, 0, 0}; // side types x-, x+, y-, y+, z-, z+
  int any_bc = 0;
  int* grain = nullptr;           // grain index per site
  void* rot = nullptr;            // 9 x n_grains rotation entries (compute type)
  unsigned long long n = 0;
  size_t elem = 4, celem = 4;
  void* pop[2] = {nullptr, nullptr};
  void* aux[2] = {nullptr, nullptr};
  void* fields = nullptr;
  double* scratch = nullptr;      // FP64 staging and reduction partials
  size_t scratch_elems = 0;
  int cur = 0, inited = 0;
  long long steps = 0, launches = 0;
  std::string err;
};

static std::string g3_err;

static pf_status fail3(pf3_handle* h, pf_status code, const std::string& m) {
  if (h) h->err = m; else g3_err = m;
  return code;
}
#define PF3_CUDA(h, ...)                                                                \
  do {                                                                                  \
    cudaError_t e_ = (__VA_ARGS__);                                                     \
    if (e_ != cudaSuccess) return fail3((h), PF_ERR_CUDA, std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename R>
static Coef3<R> coef3(const pf_params& p) {
  Coef3<R> c{};
  double der[3];
  pf_params_derived(&p, der);
  c.eps = (R)p.eps_s;
  c.ge2 = (R)(p.grad_eps * p.grad_eps);
  c.gat2 = (R)(p.grad_eps_at * p.grad_eps_at);
  c.four_bpsi = (R)(4.0 * p.beta_psi);
  c.lam = (R)der[0];
  c.Mcinf = (R)der[1];
  c.theta = (R)der[2];
  c.inv_tau0 = (R)(1.0 / p.tau0);
  c.c4W0sq_tau0 = (R)(4.0 * p.W0 * p.W0 / p.tau0);   // W0^2 / (tau0 c_s^2), c_s^2 = 1/4
  c.k = (R)p.k;
  c.inv_omk = (R)(1.0 / (1.0 - p.k));
  c.D = (R)p.D;
  c.aW0 = (R)(p.W0 / (2.0 * std::sqrt(2.0)));
  c.th0 = (R)p.theta0;
  if (p.thermal) {
    const double rcp = p.rho_l * p.cp;
    const double kT = p.Le * p.D * rcp;                 // k_T = alpha rho_l c_p, alpha = Le D
    c.rcp = (R)rcp;
    c.irc = (R)(1.0 / rcp);
    c.halfL = (R)(0.5 * p.latent);
    c.iLe = (R)(1.0 / p.Le);
    c.W0sq = (R)(p.W0 * p.W0);
    c.omsth = (R)(1.0 - 1.0 / (4.0 * kT + 0.5));       // 1 - s_T, c_s^2 = 1/4
  }
  return c;
}

template <typename S, typename R, typename I = unsigned long long>
static Args3<S, R, I> args3(const pf3_handle* h, bool fields) {
  Args3<S, R, I> a{};
  a.in = (const S*)h->pop[h->cur];
  a.out = (S*)h->pop[h->cur ^ 1];
  a.ain = (const R*)h->aux[h->cur];
  a.aout = (R*)h->aux[h->cur ^ 1];
  a.fields = fields ? (R*)h->fields : nullptr;
  a.grain = h->grain;
  a.rot = (const R*)h->rot;
  for (int k = 0; k < 6; ++k) a.bc[k] = h->bc[k];
  a.ps = (I)h->n;
  a.nx = h->nx; a.ny = h->ny; a.nz = h->nz; a.chunk = h->chunk;
  a.tiles_x = (h->nx + TX - 1) / TX;
  a.tiles_y = (h->ny + TY - 1) / TY;
  a.tiles_z = (h->nz + h->chunk - 1) / h->chunk;
  a.c = coef3<R>(h->p);
  return a;
}

static pf_status ensure_scratch3(pf3_handle* h, size_t elems) {
  if (elems <= h->scratch_elems) return PF_OK;
  cudaStreamSynchronize(h->stream);
  cudaFree(h->scratch);
  h->scratch = nullptr;
  h->scratch_elems = 0;
  if (cudaMalloc(&h->scratch, elems * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail3(h, PF_ERR_OOM, "staging allocation failed");
  }
  h->scratch_elems = elems;
  return PF_OK;
}

template <typename F>
static pf_status dispatch3(const pf3_handle* h, F&& f) {
  if (h->prec == PF_FP64) return f(double{}, double{});
  return f(float{}, float{});
}

extern "C" pf_status pf3_create(const pf_params* p, int nx, int ny, int nz, pf_precision prec,
                                void* cuda_stream, pf3_handle** out) {
  if (!out || !p) return fail3(nullptr, PF_ERR_BAD_ARG, "NULL argument");
  *out = nullptr;
  if (prec != PF_FP32 && prec != PF_FP64)
    return fail3(nullptr, PF_ERR_BAD_ARG, "the 3-D step takes FP32 or FP64 storage");
  if (nx < 4 || ny < 4 || nz < 4 || nx > 4096 || ny > 4096 || nz > 4096)
    return fail3(nullptr, PF_ERR_BAD_ARG, "sizes must be in [4, 4096]");
  if (!(p->W0 > 0) || !(p->tau0 > 0) || !(p->D > 0) || !(p->k > 0 && p->k < 1) ||
      !(p->eps_s >= 0 && p->eps_s < 0.25) || !(p->grad_eps > 0) || !(p->grad_eps_at > 0) ||
      1.0 - (1.0 - p->k) * p->Omega == 0.0)
    return fail3(nullptr, PF_ERR_BAD_ARG, "a parameter is out of range");
  if (p->thermal != 0 && p->thermal != 1) return fail3(nullptr, PF_ERR_BAD_ARG, "thermal must be 0 or 1");
  if (p->thermal) {
    auto pos = [](double v) { return std::isfinite(v) && v > 0; };
    if (!pos(p->Le) || !pos(p->cp) || !pos(p->rho_l) || !std::isfinite(p->latent) ||
        !std::isfinite(p->theta0))
      return fail3(nullptr, PF_ERR_BAD_ARG, "thermal mode needs Le, cp, rho_l > 0, finite latent, theta0");
    if (p->rho_l * p->cp < 0.75)
      return fail3(nullptr, PF_ERR_BAD_ARG, "thermal mode needs rho_l * cp >= 3/4 (stability)");
  }
  const unsigned long long n = (unsigned long long)nx * ny * nz;
  pf3_handle* h = new (std::nothrow) pf3_handle();
  if (!h) return fail3(nullptr, PF_ERR_OOM, "host allocation failed");
  h->p = *p; h->prec = prec; h->stream = (cudaStream_t)cuda_stream;
  h->nx = nx; h->ny = ny; h->nz = nz; h->n = n;
  h->thermal = p->thermal;
  h->npop = p->thermal ? NPOP3_TH : NPOP3;
  h->nfields = p->thermal ? 4 : 3;
  h->nstate = p->thermal ? NSTATE3_TH : NSTATE3;
  h->elem = h->celem = prec == PF_FP64 ? 8 : 4;
  bool ok = true;
  for (int c = 0; c < 2; ++c) {
    ok = ok && cudaMalloc(&h->pop[c], n * h->npop * h->elem) == cudaSuccess;
    ok = ok && cudaMalloc(&h->aux[c], n * NAUX3 * h->celem) == cudaSuccess;
  }
  ok = ok && cudaMalloc(&h->fields, n * h->nfields * h->celem) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    pf3_destroy(h);
    return fail3(nullptr, PF_ERR_OOM, "device allocation failed");
  }
  *out = h;
  return PF_OK;
}

extern "C" pf_status pf3_destroy(pf3_handle* h) {
  if (!h) return PF_OK;
  cudaStreamSynchronize(h->stream);
  for (int c = 0; c < 2; ++c) { cudaFree(h->pop[c]); cudaFree(h->aux[c]); }
  cudaFree(h->fields);
  cudaFree(h->scratch);
  cudaFree(h->grain);
  cudaFree(h->rot);
  const cudaError_t e = cudaGetLastError();
  delete h;
  return e == cudaSuccess ? PF_OK : PF_ERR_CUDA;
}

extern "C" const char* pf3_last_error(const pf3_handle* h) { return h ? h->err.c_str() : g3_err.c_str(); }
extern "C" long long pf3_launch_count(const pf3_handle* h) { return h ? h->launches : -1; }
extern "C" int pf3_state_planes(const pf3_handle* h) { return h ? h->nstate : -1; }
extern "C" int pf3_field_planes(const pf3_handle* h) { return h ? h->nfields : -1; }

extern "C" pf_status pf3_init_seeds(pf3_handle* h, const double* seeds, int n_seeds, double R_s) {
  if (!h) return PF_ERR_BAD_ARG;
  if (n_seeds < 0 || (n_seeds > 0 && !seeds) || !std::isfinite(R_s))
    return fail3(h, PF_ERR_BAD_ARG, "bad seeds");
  pf_status st = ensure_scratch3(h, 3 * (size_t)n_seeds + 1);
  if (st != PF_OK) return st;
  if (n_seeds)
    PF3_CUDA(h, cudaMemcpyAsync(h->scratch, seeds, 3 * (size_t)n_seeds * sizeof(double),
                                cudaMemcpyHostToDevice, h->stream));
  h->cur = 0;
  st = dispatch3(h, [&](auto s_t, auto r_t) {
    using S = decltype(s_t);
    using R = decltype(r_t);
    Args3<S, R> a = args3<S, R>(h, true);
    a.out = (S*)h->pop[0];
    a.aout = (R*)h->aux[0];
    const double sq2b = std::sqrt(2.0 * h->p.beta_psi);
    if (h->thermal)
      k_init3<S, R, true><<<1024, 256, 0, h->stream>>>(a, h->scratch, n_seeds, R_s, sq2b, h->p.W0,
                                                       h->p.k, h->p.theta0);
    else
      k_init3<S, R, false><<<1024, 256, 0, h->stream>>>(a, h->scratch, n_seeds, R_s, sq2b, h->p.W0,
                                                        h->p.k, 0.0);
    PF3_CUDA(h, cudaGetLastError());
    return PF_OK;
  });
  if (st != PF_OK) return st;
  h->launches++;
  PF3_CUDA(h, cudaStreamSynchronize(h->stream));
  h->inited = 1;
  h->steps = 0;
  return PF_OK;
}

extern "C" pf_status pf3_set_fields(pf3_handle* h, const double* psi, const double* C, size_t n) {
  if (!h) return PF_ERR_BAD_ARG;
  if (!psi || !C || n != h->n) return fail3(h, PF_ERR_BAD_ARG, "need psi and C of nx*ny*nz");
  pf_status st = ensure_scratch3(h, 2 * n + 1);
  if (st != PF_OK) return st;
  PF3_CUDA(h, cudaMemcpyAsync(h->scratch, psi, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  PF3_CUDA(h, cudaMemcpyAsync(h->scratch + n, C, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  {
    // non-finite values are found on the device, before the state is touched
    unsigned int* flag = reinterpret_cast<unsigned int*>(h->scratch + 2 * n);
    unsigned int bits = 0;
    PF3_CUDA(h, cudaMemsetAsync(flag, 0, sizeof(unsigned int), h->stream));
    k_flag_nonfinite<<<1024, 256, 0, h->stream>>>(h->scratch, (long long)(2 * n), flag);
    PF3_CUDA(h, cudaGetLastError());
    h->launches++;
    PF3_CUDA(h, cudaMemcpyAsync(&bits, flag, sizeof(bits), cudaMemcpyDeviceToHost, h->stream));
    PF3_CUDA(h, cudaStreamSynchronize(h->stream));
    if (bits) return fail3(h, PF_ERR_BAD_ARG, "non-finite field");
  }
  h->cur = 0;
  st = dispatch3(h, [&](auto s_t, auto r_t) {
    using S = decltype(s_t);
    using R = decltype(r_t);
    Args3<S, R> a = args3<S, R>(h, true);
    a.out = (S*)h->pop[0];
    a.aout = (R*)h->aux[0];
    if (h->thermal)
      k_set3<S, R, true><<<1024, 256, 0, h->stream>>>(a, h->scratch, h->scratch + n, h->p.theta0);
    else
      k_set3<S, R, false><<<1024, 256, 0, h->stream>>>(a, h->scratch, h->scratch + n, 0.0);
    PF3_CUDA(h, cudaGetLastError());
    return PF_OK;
  });
  if (st != PF_OK) return st;
  h->launches++;
  PF3_CUDA(h, cudaStreamSynchronize(h->stream));
  h->inited = 1;
  h->steps = 0;
  return PF_OK;
}

extern "C" pf_status pf3_set_temperature(pf3_handle* h, const double* theta, size_t n) {
  if (!h) return PF_ERR_BAD_ARG;
  if (!h->thermal) return fail3(h, PF_ERR_BAD_ARG, "the handle is not in thermal mode");
  if (!theta || n != h->n) return fail3(h, PF_ERR_BAD_ARG, "need theta of nx*ny*nz");
  if (!h->inited || h->steps != 0)
    return fail3(h, PF_ERR_STATE, "set the temperature after initialisation, before stepping");
  pf_status st = ensure_scratch3(h, n + 1);
  if (st != PF_OK) return st;
  PF3_CUDA(h, cudaMemcpyAsync(h->scratch, theta, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  {
    // non-finite values are found on the device, before the state is touched
    unsigned int* flag = reinterpret_cast<unsigned int*>(h->scratch + n);
    unsigned int bits = 0;
    PF3_CUDA(h, cudaMemsetAsync(flag, 0, sizeof(unsigned int), h->stream));
    k_flag_nonfinite<<<1024, 256, 0, h->stream>>>(h->scratch, (long long)n, flag);
    PF3_CUDA(h, cudaGetLastError());
    h->launches++;
    PF3_CUDA(h, cudaMemcpyAsync(&bits, flag, sizeof(bits), cudaMemcpyDeviceToHost, h->stream));
    PF3_CUDA(h, cudaStreamSynchronize(h->stream));
    if (bits) return fail3(h, PF_ERR_BAD_ARG, "non-finite theta");
  }
  st = dispatch3(h, [&](auto s_t, auto r_t) {
    using S = decltype(s_t);
    using R = decltype(r_t);
    Args3<S, R> a = args3<S, R>(h, true);
    a.out = (S*)h->pop[0];
    a.aout = (R*)h->aux[0];
    k_settemp3<S, R><<<1024, 256, 0, h->stream>>>(a, h->scratch);
    PF3_CUDA(h, cudaGetLastError());
    return PF_OK;
  });
  if (st != PF_OK) return st;
  h->launches++;
  PF3_CUDA(h, cudaStreamSynchronize(h->stream));
  return PF_OK;
}

extern "C" pf_status pf3_set_orientation(pf3_handle* h, const double* seeds7, int n_seeds) {
  if (!h) return PF_ERR_BAD_ARG;
  if (n_seeds < 0 || (n_seeds > 0 && !seeds7)) return fail3(h, PF_ERR_BAD_ARG, "bad seeds");
  if (n_seeds == 0) {                      // back to the lattice-aligned grain
    h->rotated = 0;
    return PF_OK;
  }
  std::vector<double> rot(9 * (size_t)n_seeds);
  for (int s = 0; s < n_seeds; ++s) {
    const double* q = seeds7 + 7 * s;
    if (!std::isfinite(q[0]) || !std::isfinite(q[1]) || !std::isfinite(q[2]) ||
        !quat_rows(q + 3, rot.data() + 9 * s))
      return fail3(h, PF_ERR_BAD_ARG, "non-finite seed or zero quaternion");
  }
  PF3_CUDA(h, cudaStreamSynchronize(h->stream));
  if (!h->grain && cudaMalloc(&h->grain, h->n * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    h->grain = nullptr;
    return fail3(h, PF_ERR_OOM, "device allocation failed");
  }
  cudaFree(h->rot);
  h->rot = nullptr;
  if (cudaMalloc(&h->rot, 9 * (size_t)n_seeds * h->celem) != cudaSuccess) {
    cudaGetLastError();
    h->rot = nullptr;
    return fail3(h, PF_ERR_OOM, "device allocation failed");
  }
  pf_status st = ensure_scratch3(h, 7 * (size_t)n_seeds);
  if (st != PF_OK) return st;
  PF3_CUDA(h, cudaMemcpyAsync(h->scratch, seeds7, 7 * (size_t)n_seeds * sizeof(double),
                              cudaMemcpyHostToDevice, h->stream));
  k_grain_nearest<7><<<1024, 256, 0, h->stream>>>(h->nx, h->ny, h->nz, h->scratch, n_seeds, h->grain);
  PF3_CUDA(h, cudaGetLastError());
  h->launches++;
  if (h->prec == PF_FP64) {
    PF3_CUDA(h, cudaMemcpyAsync(h->rot, rot.data(), rot.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  } else {
    std::vector<float> rf(rot.begin(), rot.end());
    PF3_CUDA(h, cudaMemcpyAsync(h->rot, rf.data(), rf.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream));
  }
  PF3_CUDA(h, cudaStreamSynchronize(h->stream));
  h->rotated = 1;
  return PF_OK;
}

extern "C" pf_status pf3_set_boundaries(pf3_handle* h, const int bc[6]) {
  if (!h) return PF_ERR_BAD_ARG;
  if (!bc) return fail3(h, PF_ERR_BAD_ARG, "NULL bc");
  for (int k = 0; k < 6; ++k)
    if (bc[k] < 0 || bc[k] > 3)
      return fail3(h, PF_ERR_BAD_ARG, "side types are 0 (periodic) .. 3 (far field)");
  for (int a = 0; a < 3; ++a)
    if ((bc[2 * a] == 0) != (bc[2 * a + 1] == 0))
      return fail3(h, PF_ERR_BAD_ARG, "a periodic side needs a periodic opposite side");
  if (h->inited) return fail3(h, PF_ERR_STATE, "set the sides before initialising");
  h->any_bc = 0;
  for (int k = 0; k < 6; ++k) {
    h->bc[k] = bc[k];
    if (bc[k]) h->any_bc = 1;
  }
  return PF_OK;
}

extern "C" pf_status pf3_set_chunk(pf3_handle* h, int chunk) {
  if (!h) return PF_ERR_BAD_ARG;
  if (chunk < 1 || chunk > 4096) return fail3(h, PF_ERR_BAD_ARG, "chunk must be in [1, 4096]");
  h->chunk = chunk;
  return PF_OK;
}

extern "C" pf_status pf3_set_index64(pf3_handle* h, int on) {
  if (!h) return PF_ERR_BAD_ARG;
  h->index64 = on != 0;
  return PF_OK;
}

extern "C" pf_status pf3_step(pf3_handle* h, int n_steps) {
  if (!h) return PF_ERR_BAD_ARG;
  if (n_steps < 0) return fail3(h, PF_ERR_BAD_ARG, "n_steps must be >= 0");
  if (!h->inited) return fail3(h, PF_ERR_STATE, "initialise before stepping");
  return dispatch3(h, [&](auto s_t, auto r_t) {
    using S = decltype(s_t);
    using R = decltype(r_t);
    // periodic launches index sites and planes in 32 bits while every plane
    // offset (below NSTATE3_TH x sites) fits
    const bool a32 = !h->any_bc && !h->index64 && (unsigned long long)NSTATE3_TH * h->n <= 0xFFFFFFFFull;
    for (int t = 0; t < n_steps; ++t) {
      const bool last = t == n_steps - 1;
      const int tiles = (int)((long long)((h->nx + TX - 1) / TX) * ((h->ny + TY - 1) / TY) *
                              ((h->nz + h->chunk - 1) / h->chunk));
      auto go = [&](auto bcv, const auto& a) {
        constexpr bool BC = decltype(bcv)::value;
        using I = decltype(a.ps);
        if (h->rotated) {
          if (h->thermal) k_step3d<S, R, true, true, BC, I><<<tiles, THREADS, 0, h->stream>>>(a);
          else k_step3d<S, R, false, true, BC, I><<<tiles, THREADS, 0, h->stream>>>(a);
        } else {
          if (h->thermal) k_step3d<S, R, true, false, BC, I><<<tiles, THREADS, 0, h->stream>>>(a);
          else k_step3d<S, R, false, false, BC, I><<<tiles, THREADS, 0, h->stream>>>(a);
        }
      };
      if (h->any_bc) go(std::true_type{}, args3<S, R>(h, last));
      else if (a32) go(std::false_type{}, args3<S, R, unsigned>(h, last));
      else go(std::false_type{}, args3<S, R>(h, last));
      PF3_CUDA(h, cudaGetLastError());
      h->cur ^= 1;
      h->steps++;
      h->launches++;
    }
    return PF_OK;
  });
}

extern "C" pf_status pf3_get_fields(pf3_handle* h, double* out, size_t n) {
  if (!h) return PF_ERR_BAD_ARG;
  const size_t need = (size_t)h->nfields * h->n;
  if (!out || n < need) return fail3(h, PF_ERR_BAD_ARG, "output must hold pf3_field_planes planes");
  pf_status st = ensure_scratch3(h, need);
  if (st != PF_OK) return st;
  if (h->prec == PF_FP64)
    k_fields3<double><<<1024, 256, 0, h->stream>>>((const double*)h->fields, h->n, h->n, h->nfields, h->scratch);
  else
    k_fields3<float><<<1024, 256, 0, h->stream>>>((const float*)h->fields, h->n, h->n, h->nfields, h->scratch);
  PF3_CUDA(h, cudaGetLastError());
  h->launches++;
  PF3_CUDA(h, cudaMemcpyAsync(out, h->scratch, need * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  PF3_CUDA(h, cudaStreamSynchronize(h->stream));
  return PF_OK;
}

extern "C" pf_status pf3_get_state(pf3_handle* h, double* out, size_t n) {
  if (!h) return PF_ERR_BAD_ARG;
  const size_t need = (size_t)h->nstate * h->n;
  if (!out || n < need) return fail3(h, PF_ERR_BAD_ARG, "output must hold pf3_state_planes planes");
  pf_status st = ensure_scratch3(h, need);
  if (st != PF_OK) return st;
  st = dispatch3(h, [&](auto s_t, auto r_t) {
    using S = decltype(s_t);
    using R = decltype(r_t);
    k_state3<S, R><<<1024, 256, 0, h->stream>>>((const S*)h->pop[h->cur], (const R*)h->aux[h->cur],
                                                 h->n, h->n, h->thermal, h->scratch);
    PF3_CUDA(h, cudaGetLastError());
    return PF_OK;
  });
  if (st != PF_OK) return st;
  h->launches++;
  PF3_CUDA(h, cudaMemcpyAsync(out, h->scratch, need * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  PF3_CUDA(h, cudaStreamSynchronize(h->stream));
  return PF_OK;
}

extern "C" pf_status pf3_reduce(pf3_handle* h, double out[2]) {
  if (!h) return PF_ERR_BAD_ARG;
  if (!out) return fail3(h, PF_ERR_BAD_ARG, "NULL output");
  const int nb = 1024;
  pf_status st = ensure_scratch3(h, 2 * nb + 2);
  if (st != PF_OK) return st;
  if (h->prec == PF_FP64) k_reduce3<double><<<nb, 256, 0, h->stream>>>((const double*)h->fields, h->n, h->n, h->scratch);
  else k_reduce3<float><<<nb, 256, 0, h->stream>>>((const float*)h->fields, h->n, h->n, h->scratch);
  k_reduce3_final<<<1, 32, 0, h->stream>>>(h->scratch, nb, 2, h->scratch + 2 * nb);
  PF3_CUDA(h, cudaGetLastError());
  h->launches += 2;
  PF3_CUDA(h, cudaMemcpyAsync(out, h->scratch + 2 * nb, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  PF3_CUDA(h, cudaStreamSynchronize(h->stream));
  return PF_OK;
}

extern "C" pf_status pf3_reduce_thermal(pf3_handle* h, double out[3]) {
  if (!h) return PF_ERR_BAD_ARG;
  if (!out) return fail3(h, PF_ERR_BAD_ARG, "NULL output");
  if (!h->thermal) return fail3(h, PF_ERR_BAD_ARG, "the handle is not in thermal mode");
  const int nb = 1024;
  pf_status st = ensure_scratch3(h, 3 * nb + 3);
  if (st != PF_OK) return st;
  st = dispatch3(h, [&](auto s_t, auto r_t) {
    using S = decltype(s_t);
    using R = decltype(r_t);
    k_reduce3_th<S, R><<<nb, 256, 0, h->stream>>>((const S*)h->pop[h->cur], (const R*)h->fields,
                                                   h->n, h->n, h->scratch);
    k_reduce3_final<<<1, 32, 0, h->stream>>>(h->scratch, nb, 3, h->scratch + 3 * nb);
    PF3_CUDA(h, cudaGetLastError());
    return PF_OK;
  });
  if (st != PF_OK) return st;
  h->launches += 2;
  PF3_CUDA(h, cudaMemcpyAsync(out, h->scratch + 3 * nb, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  PF3_CUDA(h, cudaStreamSynchronize(h->stream));
  return PF_OK;
}
