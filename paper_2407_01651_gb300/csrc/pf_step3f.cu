// pf_step3f.cu -- the three-dimensional two-phase coupled step of arXiv
// 2407.01651: incompressible Navier-Stokes and the conservative Allen-Cahn
// equation on D3Q19 lattices (MRT with the d'Humieres basis), the anisotropic
// dendrite equation (a_s^2 time stretch of Appendix B) and the solute equation
// with antitrapping and the gas-vacuum flux on D3Q7 lattices, coupled through
// surface tension, buoyancy, the mass-flux correction and the diffuse drag of
// the solid exactly as in the 2-D step; and the C ABI of its handle (pf3f_* in
// include/pf.h).
//
// Kernel: k_step3f, a z-march over 32 x 8 column tiles (the geometry of
// pf_d3.cuh).  At plane k every ring column (256 interior + 84 halo threads)
// pulls h and g of plane k+1, and reads the lagged velocity there, and writes
// phi, psi and v_o into 4-slot shared-memory rings; after one barrier the
// interior threads update plane k: D3Q19-weighted gradients and Laplacian
// from the rings, the forces, the NS collision (f pulled here), the CAC
// collision (h pulled again, an L1/L2 hit), the dendrite collision with the
// carried g and the solute collision.  Collisions are the MRT operator of
// Appendix B in closed form: f* = f_eq + G/2 + sum over the moments k with a
// rate s_k != 1 of (1 - s_k) [M (f - f_eq + G/2)]_k M_k / |M_k|^2.
// Layout: one plane per population, [z][y][x], x fastest.
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

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
// (a sixth ring, of U, in thermal mode)
template <typename R>
constexpr size_t ring_bytes(bool th) { return (th ? 6 : 5) * 4 * HY * HX * sizeof(R); }

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
};

template <typename S, typename R>
struct ArgsF {
  const S* in;
  S* out;
  const R* ain;
  R* aout;
  R* fields;            // phi, psi, C, U, p, vx, vy, vz, mu planes, or nullptr
  const int* grain;     // ROT: grain index per site
  const R* rot;         // ROT: 9 entries (row-major R) per grain
  unsigned long long ps;
  int nx, ny, nz, chunk;
  int tiles_x, tiles_y, tiles_z;
  CoefF<R> c;
};

template <typename S, typename R>
__device__ __forceinline__ unsigned long long site_of(const ArgsF<S, R>& a, int x, int y, int z) {
  return ((unsigned long long)z * a.ny + y) * a.nx + x;
}
// pull source of D3Q19 direction i (x, y in range; one step wraps)
template <typename S, typename R>
__device__ __forceinline__ unsigned long long src19(const ArgsF<S, R>& a, int x, int y, int z, int i) {
  return site_of(a, wrap1(x - c19(i, 0), a.nx), wrap1(y - c19(i, 1), a.ny), wrap1(z - c19(i, 2), a.nz));
}
template <typename S, typename R>
__device__ __forceinline__ unsigned long long src7(const ArgsF<S, R>& a, int x, int y, int z, int i) {
  return site_of(a, wrap1(x - cx7(i), a.nx), wrap1(y - cy7(i), a.ny), wrap1(z - cz7(i), a.nz));
}

// phi = sum of the streamed h at (x, y, z)
template <typename S, typename R>
__device__ __forceinline__ R stream_phi(const ArgsF<S, R>& a, int x, int y, int z) {
  CSum<R> s;
#pragma unroll
  for (int i = 0; i < 19; ++i) s.add(ld<R>(pl(a.in, H_POP + i, a.ps), src19(a, x, y, z, i)));
  return s.value();
}

// streamed g with the time stretch, psi and psi_o (as in the melt-only step)
template <typename S, typename R>
__device__ __forceinline__ void stream_g(const ArgsF<S, R>& a, int x, int y, int z, R g[7],
                                         R& psi, R& psio) {
  const unsigned long long own = site_of(a, x, y, z);
  CSum<R> sg;
  R po = R(0);
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    const unsigned long long src = src7(a, x, y, z, i);
    const R gold = ld<R>(pl(a.in, G_PRE + i, a.ps), own);
    const R gpo = ld<R>(pl(a.in, G_POST + i, a.ps), src);
    const R rr = pl(a.ain, AX_RR, a.ps)[src];
    g[i] = gold + (gpo - gold) * rr;
    sg.add(g[i]);
    po += gold;
  }
  psi = sg.value();
  psio = po;
}

// ROT: grain orientations (anisotropy on g' = R^T grad psi, N = R N'(g')).
// TH: the temperature lattice of Appendix B on D3Q7 with the flux rho H v and
// d_t(rho H v) through (I - S/2); theta = H / c_p + (c_p^s/c_p) h(psi) from the
// local density; F(U) in the psi relaxation and the source Q / F + W0^2 / F^2
// grad F . (a_s^2 grad psi + N), grad F = M c_inf (1-k) grad U from a U ring.
// U = (2C/A - 1)/(1-k) of the streamed solute at (x, y, z), for the U ring
template <typename S, typename R>
__device__ __forceinline__ R stream_U(const ArgsF<S, R>& a, int x, int y, int z, R psi) {
  CSum<R> cs;
#pragma unroll
  for (int i = 0; i < 7; ++i) cs.add(ld<R>(pl(a.in, S_POP + i, a.ps), src7(a, x, y, z, i)));
  const R A = (R(1) + a.c.k) - (R(1) - a.c.k) * psi;
  return (R(2) * cs.value() * frcp(A) - R(1)) * a.c.inv_omk;
}

template <typename S, typename R, bool ROT, bool TH>
__global__ void __launch_bounds__(THREADS, MIN_CTAS) k_step3f(ArgsF<S, R> a) {
  // rings of phi, psi, v_o (and U) (dynamic: 54 KB in FP64)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R (*rphi)[HY][HX] = reinterpret_cast<R (*)[HY][HX]>(smem_raw);
  R (*rpsi)[HY][HX] = rphi + 4;
  R (*rv0)[HY][HX] = rphi + 8;
  R (*rv[3])[HY][HX] = {rv0, rv0 + 4, rv0 + 8};
  R (*rU)[HY][HX] = rphi + 20;         // TH only
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
    const int x = wrapm(tx * TX + hx - 1, a.nx), y = wrapm(ty * TY + hy - 1, a.ny);
    const bool mine = interior && tx * TX + hx - 1 < a.nx && ty * TY + hy - 1 < a.ny;
    R gC[7], gL[7], poC = R(0), poL = R(0);
    // ring planes za-1 and za
    for (int k = 0; k < 2; ++k) {
      if (active) {
        const int z = wrap1(za - 1 + k, a.nz);
        const int slot = (za - 1 + k) & 3;
        R g[7], psi, po;
        stream_g(a, x, y, z, g, psi, po);
        rpsi[slot][hy][hx] = psi;
        rphi[slot][hy][hx] = stream_phi(a, x, y, z);
        const unsigned long long s0 = site_of(a, x, y, z);
#pragma unroll
        for (int c = 0; c < 3; ++c) rv[c][slot][hy][hx] = pl(a.ain, AX_VO + c, a.ps)[s0];
        if constexpr (TH) rU[slot][hy][hx] = stream_U(a, x, y, z, psi);
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
      if (mine) {
#pragma unroll
        for (int i = 0; i < 7; ++i) sv[i] = ld<R>(pl(a.in, S_POP + i, a.ps), src7(a, x, y, z, i));
        Qo = pl(a.ain, AX_QO, a.ps)[site];
        phio = pl(a.ain, AX_PHIO, a.ps)[site];
        Co = pl(a.ain, AX_CO, a.ps)[site];
      }
      if (active) {
        const int zn = wrap1(z + 1, a.nz);
        const int slot = (z + 1) & 3;
        R psi;
        stream_g(a, x, y, zn, gL, psi, poL);
        rpsi[slot][hy][hx] = psi;
        rphi[slot][hy][hx] = stream_phi(a, x, y, zn);
        const unsigned long long sn = site_of(a, x, y, zn);
#pragma unroll
        for (int c = 0; c < 3; ++c) rv[c][slot][hy][hx] = pl(a.ain, AX_VO + c, a.ps)[sn];
        if constexpr (TH) rU[slot][hy][hx] = stream_U(a, x, y, zn, psi);
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
        R fv[19], j[3] = {R(0), R(0), R(0)};
        CSum<R> snz;
#pragma unroll
        for (int i = 0; i < 19; ++i) {
          fv[i] = ld<R>(pl(a.in, F_POP + i, a.ps), src19(a, x, y, z, i));
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
            const R hp = ld<R>(pl(a.in, H_POP + i, a.ps), src19(a, x, y, z, i));
            const R hm = ld<R>(pl(a.in, H_POP + i + 1, a.ps), src19(a, x, y, z, i + 1));
            const R cu = R(c19(i, 0)) * v[0] + R(c19(i, 1)) * v[1] + R(c19(i, 2)) * v[2];
            const R cG = R(c19(i, 0)) * G1[0] + R(c19(i, 1)) * G1[1] + R(c19(i, 2)) * G1[2];
            const R Do = (hp - hm) - R(2) * w19<R>(i) * (R(3) * phi * cu - R(1.5) * cG);
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
        R ev[7];
        if constexpr (TH) {
#pragma unroll
          for (int i = 0; i < 7; ++i) ev[i] = ld<R>(pl(a.in, E_POP + i, a.ps), src7(a, x, y, z, i));
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
          const R Ho = pl(a.ain, AX_HO, a.ps)[site];
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

// Equilibrium state of a site (Appendix B at the given phi, psi, C, v, p):
// f = f_eq(p, rho, v), h = w phi (1 + 3 c.v), g = w psi, s = w C (1 + 4 c.v),
// r = 1, lagged values equal to the current ones; fields written.
template <typename S, typename R>
__device__ void write_eqf(const ArgsF<S, R>& a, unsigned long long site, R phi, R psi, R C,
                          const R v[3], R p) {
  const CoefF<R>& c = a.c;
  const R rho = c.rg + phi * c.drho;
  const R v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  // h bases as in the collision: the even parts sum to phi exactly
  const R b = round_to_multiple(phi * R(1.0 / 36.0), R(0.5) * quantum_quarter_ulp(phi));
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    const R cu = R(c19(i, 0)) * v[0] + R(c19(i, 1)) * v[1] + R(c19(i, 2)) * v[2];
    R feq = w19<R>(i) * (R(3) * p + rho * (R(3) * cu + R(4.5) * cu * cu - R(1.5) * v2));
    if (i == 0) feq -= R(3) * p;
    st<S, R>(pl(a.out, F_POP + i, a.ps), site, feq);
    const R base = i == 0 ? fma(R(-24), b, phi) : (c2_19(i) == 1 ? R(2) * b : b);
    st<S, R>(pl(a.out, H_POP + i, a.ps), site, base + w19<R>(i) * R(3) * phi * cu);
  }
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    const R cu = R(cx7(i)) * v[0] + R(cy7(i)) * v[1] + R(cz7(i)) * v[2];
    st<S, R>(pl(a.out, G_PRE + i, a.ps), site, w7<R>(i) * psi);
    st<S, R>(pl(a.out, G_POST + i, a.ps), site, w7<R>(i) * psi);
    st<S, R>(pl(a.out, S_POP + i, a.ps), site, w7<R>(i) * C + w7<R>(i) * C * cu * R(4));
  }
  const R omk = R(1) - c.k;
  const R U = (R(2) * C / ((R(1) + c.k) - omk * psi) - R(1)) * c.inv_omk;
  const R omp2 = R(1) - psi * psi;
  const R Q = c.four_bpsi * psi * omp2 - c.binter2 * (R(1) - phi) * (R(1) - phi) * (R(1) + psi) -
              c.lam * omp2 * omp2 * (c.theta + c.Mcinf * U);
  pl(a.aout, AX_RR, a.ps)[site] = R(1);
  pl(a.aout, AX_QO, a.ps)[site] = Q;
  pl(a.aout, AX_PHIO, a.ps)[site] = phi;
  pl(a.aout, AX_CO, a.ps)[site] = C;
#pragma unroll
  for (int q = 0; q < 3; ++q) pl(a.aout, AX_VO + q, a.ps)[site] = v[q];
  const R vals[NFIELDSF] = {phi, psi, C, U, p, v[0], v[1], v[2], R(0)};
#pragma unroll
  for (int f = 0; f < NFIELDSF; ++f) pl(a.fields, f, a.ps)[site] = vals[f];
}

// Thermal mode: temperature populations at equilibrium for theta (rho H = rho c_p
// (theta - latent h(psi)), flux rho H v), lagged H, the lagged source Q_psi(theta)
// / F(U) and the theta field; phi, psi, C, v as initialised.
template <typename S, typename R>
__device__ void write_thf(const ArgsF<S, R>& a, unsigned long long site, R phi, R psi, R C,
                          const R v[3], R theta) {
  const CoefF<R>& c = a.c;
  const R rho = c.rg + phi * c.drho;
  const R H = c.cp * (theta - c.halfL * (R(1) + psi));
  const R rhoH = rho * H;
  st<S, R>(pl(a.out, E_POP, a.ps), site, rhoH - R(0.75) * theta);
#pragma unroll
  for (int i = 1; i < 7; ++i) {
    const R cj = rhoH * (R(cx7(i)) * v[0] + R(cy7(i)) * v[1] + R(cz7(i)) * v[2]);
    st<S, R>(pl(a.out, E_POP + i, a.ps), site, R(0.125) * theta + R(0.5) * cj);
  }
  pl(a.aout, AX_HO, a.ps)[site] = H;
  const R omk = R(1) - c.k;
  const R U = (R(2) * C / ((R(1) + c.k) - omk * psi) - R(1)) * c.inv_omk;
  const R omp2 = R(1) - psi * psi;
  const R Q = c.four_bpsi * psi * omp2 - c.binter2 * (R(1) - phi) * (R(1) - phi) * (R(1) + psi) -
              c.lam * omp2 * omp2 * (theta + c.Mcinf * U);
  pl(a.aout, AX_QO, a.ps)[site] = Q / (c.iLe + c.Mcinf * (R(1) + omk * U));
  pl(a.fields, NFIELDSF, a.ps)[site] = theta;
}

// Temperature field of the initial state (phi, psi, C, v from the field planes).
template <typename S, typename R>
__global__ void k_settempf(ArgsF<S, R> a, const double* theta, int uniform, double theta0) {
  const unsigned long long n = (unsigned long long)a.nx * a.ny * a.nz;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const R v[3] = {pl(a.fields, 5, a.ps)[i], pl(a.fields, 6, a.ps)[i], pl(a.fields, 7, a.ps)[i]};
    write_thf<S, R>(a, i, pl(a.fields, 0, a.ps)[i], pl(a.fields, 1, a.ps)[i],
                    pl(a.fields, 2, a.ps)[i], v, uniform ? (R)theta0 : (R)theta[i]);
  }
}

__device__ __forceinline__ double min_image(double d, double L) {
  d = fmod(d, L);
  if (d < -0.5 * L) d += L;
  if (d >= 0.5 * L) d -= L;
  return d;
}

// Fields from seeds (x, y, z) and bubbles (x, y, z, R): psi = max tanh(sqrt(2
// beta_psi) (R_s - r)/W0), phi = min [1/2 + 1/2 tanh(sqrt(2 beta_phi) (r -
// R_b)/(2 W_phi))], C = phi (1 - (1-k) h(psi)); at rest, p = 0.
template <typename S, typename R>
__global__ void k_initf(ArgsF<S, R> a, const double* seeds, int n_seeds, double R_s,
                        const double* bub, int n_bub, double sb, double W0, double sp, double Wphi,
                        double k) {
  const unsigned long long n = (unsigned long long)a.nx * a.ny * a.nz;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const double X[3] = {(double)(i % a.nx), (double)((i / a.nx) % a.ny),
                         (double)(i / ((unsigned long long)a.nx * a.ny))};
    const double L[3] = {(double)a.nx, (double)a.ny, (double)a.nz};
    double psi = -1.0, phi = 1.0;
    for (int s = 0; s < n_seeds; ++s) {
      double r2 = 0;
      for (int q = 0; q < 3; ++q) {
        const double d = min_image(X[q] - seeds[3 * s + q], L[q]);
        r2 += d * d;
      }
      const double v = tanh(sb * (R_s - sqrt(r2)) / W0);
      if (s == 0 || v > psi) psi = v;
    }
    for (int b = 0; b < n_bub; ++b) {
      double r2 = 0;
      for (int q = 0; q < 3; ++q) {
        const double d = min_image(X[q] - bub[4 * b + q], L[q]);
        r2 += d * d;
      }
      const double v = 0.5 + 0.5 * tanh(sp * (sqrt(r2) - bub[4 * b + 3]) / (2.0 * Wphi));
      if (b == 0 || v < phi) phi = v;
    }
    const double C = phi * (1.0 - (1.0 - k) * 0.5 * (1.0 + psi));
    const R v0[3] = {R(0), R(0), R(0)};
    write_eqf<S, R>(a, i, (R)phi, (R)psi, (R)C, v0, R(0));
  }
}

// Fields from host arrays: phi, psi, C, vx, vy, vz, p planes of n (FP64).
template <typename S, typename R>
__global__ void k_setf(ArgsF<S, R> a, const double* in) {
  const unsigned long long n = (unsigned long long)a.nx * a.ny * a.nz;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const R v[3] = {(R)in[3 * n + i], (R)in[4 * n + i], (R)in[5 * n + i]};
    write_eqf<S, R>(a, i, (R)in[i], (R)in[n + i], (R)in[2 * n + i], v, (R)in[6 * n + i]);
  }
}

template <typename S, typename R>
__global__ void k_statef(const S* pin, const R* ain, unsigned long long ps, unsigned long long n,
                         int thermal, double* out) {
  for (unsigned long long j = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j < n;
       j += (unsigned long long)gridDim.x * blockDim.x) {
    int q = 0;
    for (int i = 0; i < 19; ++i) out[(q++) * n + j] = (double)ld<R>(pl(pin, F_POP + i, ps), j);
    for (int i = 0; i < 19; ++i) out[(q++) * n + j] = (double)ld<R>(pl(pin, H_POP + i, ps), j);
    for (int i = 0; i < 7; ++i) out[(q++) * n + j] = (double)ld<R>(pl(pin, G_PRE + i, ps), j);
    for (int i = 0; i < 7; ++i) out[(q++) * n + j] = (double)ld<R>(pl(pin, G_POST + i, ps), j);
    out[(q++) * n + j] = (double)ain[AX_RR * ps + j];
    for (int i = 0; i < 7; ++i) out[(q++) * n + j] = (double)ld<R>(pl(pin, S_POP + i, ps), j);
    out[(q++) * n + j] = (double)ain[AX_QO * ps + j];
    out[(q++) * n + j] = (double)ain[AX_PHIO * ps + j];
    out[(q++) * n + j] = (double)ain[AX_CO * ps + j];
    for (int c = 0; c < 3; ++c) out[(q++) * n + j] = (double)ain[(AX_VO + c) * ps + j];
    if (thermal) {
      for (int i = 0; i < 7; ++i) out[(q++) * n + j] = (double)ld<R>(pl(pin, E_POP + i, ps), j);
      out[(q++) * n + j] = (double)ain[AX_HO * ps + j];
    }
  }
}

template <typename R>
__global__ void k_fieldsf(const R* f, unsigned long long ps, unsigned long long n, int planes,
                          double* out) {
  for (unsigned long long j = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
       j < planes * n; j += (unsigned long long)gridDim.x * blockDim.x)
    out[j] = (double)f[(j / n) * ps + j % n];
}

// FP64 totals: sum phi, sum C, sum h(psi); fixed-order partials.
template <typename R>
__global__ void k_reducef(const R* f, unsigned long long ps, unsigned long long n, double* part) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (unsigned long long j = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j < n;
       j += (unsigned long long)gridDim.x * blockDim.x) {
    a0 += (double)f[j];
    a2 += 0.5 * (1.0 + (double)f[ps + j]);
    a1 += (double)f[2 * ps + j];
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
__global__ void k_reducef_final(const double* part, int nb, double* out) {
  if (threadIdx.x >= 3) return;
  double acc = 0.0;
  for (int b = 0; b < nb; ++b) acc += part[3 * b + threadIdx.x];
  out[threadIdx.x] = acc;
}

}  // namespace d3f
}  // namespace pf

using namespace pf;
using namespace pf::d3f;

struct pf3f_handle {
  pf_params p{};
  pf_precision prec = PF_FP32;
  cudaStream_t stream = nullptr;
  int nx = 0, ny = 0, nz = 0, chunk = 16;
  unsigned long long n = 0;
  size_t elem = 4;
  double rho_bar = 0.0;
  void* pop[2] = {nullptr, nullptr};
  void* aux[2] = {nullptr, nullptr};
  void* fields = nullptr;
  double* scratch = nullptr;
  size_t scratch_elems = 0;
  int rotated = 0;                // grain orientations set
  int* grain = nullptr;           // grain index per site
  void* rot = nullptr;            // 9 x n_grains rotation entries (storage precision)
  int thermal = 0, npop = NPOPF, naux = NAUXF, nfields = NFIELDSF, nstate = NSTATEF;
  int cur = 0, inited = 0;
  long long steps = 0, launches = 0;
  std::string err;
};

static std::string g3f_err;

static pf_status failf(pf3f_handle* h, pf_status code, const std::string& m) {
  if (h) h->err = m; else g3f_err = m;
  return code;
}
#define PF3F_CUDA(h, ...)                                                               \
  do {                                                                                  \
    cudaError_t e_ = (__VA_ARGS__);                                                     \
    if (e_ != cudaSuccess) return failf((h), PF_ERR_CUDA, std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename R>
static CoefF<R> coeff(const pf3f_handle* h) {
  const pf_params& p = h->p;
  CoefF<R> c{};
  double der[3];
  pf_params_derived(&p, der);
  c.rl = (R)p.rho_l;
  c.rg = (R)p.rho_g;
  c.drho = (R)(p.rho_l - p.rho_g);
  c.rho_bar = (R)h->rho_bar;
  c.g = (R)p.g;
  c.kappa = (R)(std::sqrt(2.0 * p.beta_phi) / p.W_phi);
  c.fs_coef = (R)(6.0 * p.sigma / (p.W_phi * std::sqrt(2.0 * p.beta_phi)));
  c.bphi2 = (R)(2.0 * p.beta_phi);
  c.binter2 = (R)(2.0 * p.beta_inter);
  c.Wphi2 = (R)(p.W_phi * p.W_phi);
  c.Mphi = (R)p.M_phi;
  c.eps = (R)p.eps_s;
  c.ge2 = (R)(p.grad_eps * p.grad_eps);
  c.gat2 = (R)(p.grad_eps_at * p.grad_eps_at);
  c.four_bpsi = (R)(4.0 * p.beta_psi);
  c.lam = (R)der[0];
  c.Mcinf = (R)der[1];
  c.theta = (R)der[2];
  c.inv_tau0 = (R)(1.0 / p.tau0);
  c.c4W0sq_tau0 = (R)(4.0 * p.W0 * p.W0 / p.tau0);
  c.k = (R)p.k;
  c.inv_omk = (R)(1.0 / (1.0 - p.k));
  c.D = (R)p.D;
  c.aW0 = (R)(p.W0 / (2.0 * std::sqrt(2.0)));
  c.s_phi = (R)(1.0 / (3.0 * p.M_phi + 0.5));          // M_phi = (1/s - 1/2) c_s^2
  const double s_nu = 1.0 / (3.0 * p.nu + 0.5);
  const double s_q = 8.0 * (2.0 - s_nu) / (8.0 - s_nu);
  const double rate[NMOM] = {p.s_e, p.s_eps, s_q, s_q, s_q, s_nu, s_nu, s_nu, s_nu, s_nu,
                             s_q, s_q, s_q};
  for (int k = 0; k < NMOM; ++k) c.cm[k] = (R)((1.0 - rate[k]) / mnorm(k));
  if (p.thermal) {
    const double kT = p.Le * p.D * p.rho_l * p.cp;      // k_T = alpha rho_l c_p, alpha = Le D
    const double sth = 1.0 / (4.0 * kT + 0.5);          // c_s^2 = 1/4
    c.cp = (R)p.cp;
    c.halfL = (R)(0.5 * p.latent);
    c.iLe = (R)(1.0 / p.Le);
    c.W0sq = (R)(p.W0 * p.W0);
    c.sth = (R)sth;
    c.hsth = (R)(1.0 - 0.5 * sth);
  }
  return c;
}

template <typename S, typename R>
static ArgsF<S, R> argsf(const pf3f_handle* h, bool fields) {
  ArgsF<S, R> a{};
  a.in = (const S*)h->pop[h->cur];
  a.out = (S*)h->pop[h->cur ^ 1];
  a.ain = (const R*)h->aux[h->cur];
  a.aout = (R*)h->aux[h->cur ^ 1];
  a.fields = fields ? (R*)h->fields : nullptr;
  a.grain = h->grain;
  a.rot = (const R*)h->rot;
  a.ps = h->n;
  a.nx = h->nx; a.ny = h->ny; a.nz = h->nz; a.chunk = h->chunk;
  a.tiles_x = (h->nx + TX - 1) / TX;
  a.tiles_y = (h->ny + TY - 1) / TY;
  a.tiles_z = (h->nz + h->chunk - 1) / h->chunk;
  a.c = coeff<R>(h);
  return a;
}

static pf_status ensure_scratchf(pf3f_handle* h, size_t elems) {
  if (elems <= h->scratch_elems) return PF_OK;
  cudaStreamSynchronize(h->stream);
  cudaFree(h->scratch);
  h->scratch = nullptr;
  h->scratch_elems = 0;
  if (cudaMalloc(&h->scratch, elems * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return failf(h, PF_ERR_OOM, "staging allocation failed");
  }
  h->scratch_elems = elems;
  return PF_OK;
}

template <typename F>
static pf_status dispatchf(const pf3f_handle* h, F&& f) {
  if (h->prec == PF_FP64) return f(double{}, double{});
  return f(float{}, float{});
}

// sums of the field planes into out[3] (sum phi, sum C, sum h(psi))
static pf_status reduce_fields(pf3f_handle* h, double out[3]) {
  const int nb = 1024;
  pf_status st = ensure_scratchf(h, 3 * nb + 3);
  if (st != PF_OK) return st;
  if (h->prec == PF_FP64) k_reducef<double><<<nb, 256, 0, h->stream>>>((const double*)h->fields, h->n, h->n, h->scratch);
  else k_reducef<float><<<nb, 256, 0, h->stream>>>((const float*)h->fields, h->n, h->n, h->scratch);
  k_reducef_final<<<1, 32, 0, h->stream>>>(h->scratch, nb, h->scratch + 3 * nb);
  PF3F_CUDA(h, cudaGetLastError());
  h->launches += 2;
  PF3F_CUDA(h, cudaMemcpyAsync(out, h->scratch + 3 * nb, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  PF3F_CUDA(h, cudaStreamSynchronize(h->stream));
  return PF_OK;
}

// after an initialisation: rho_bar = rho_g + mean(phi) (rho_l - rho_g) (reading R13)
static pf_status finish_init(pf3f_handle* h) {
  double t[3];
  pf_status st = reduce_fields(h, t);
  if (st != PF_OK) return st;
  h->rho_bar = h->p.rho_g + (t[0] / (double)h->n) * (h->p.rho_l - h->p.rho_g);
  h->inited = 1;
  h->steps = 0;
  return PF_OK;
}

extern "C" pf_status pf3f_create(const pf_params* p, int nx, int ny, int nz, pf_precision prec,
                                 void* cuda_stream, pf3f_handle** out) {
  if (!out || !p) return failf(nullptr, PF_ERR_BAD_ARG, "NULL argument");
  *out = nullptr;
  if (prec != PF_FP32 && prec != PF_FP64)
    return failf(nullptr, PF_ERR_BAD_ARG, "the 3-D two-phase step takes FP32 or FP64 storage");
  if (nx < 4 || ny < 4 || nz < 4 || nx > 2048 || ny > 2048 || nz > 2048)
    return failf(nullptr, PF_ERR_BAD_ARG, "sizes must be in [4, 2048]");
  auto pos = [](double v) { return std::isfinite(v) && v > 0; };
  if (!pos(p->rho_l) || !pos(p->rho_g) || !pos(p->nu) || !pos(p->W_phi) || !pos(p->M_phi) ||
      !pos(p->beta_phi) || !std::isfinite(p->sigma) || !std::isfinite(p->g) ||
      !(p->s_e > 0 && p->s_e < 2) || !(p->s_eps > 0 && p->s_eps < 2) || !std::isfinite(p->beta_inter))
    return failf(nullptr, PF_ERR_BAD_ARG, "a flow parameter is out of range");
  if (!(p->W0 > 0) || !(p->tau0 > 0) || !(p->D > 0) || !(p->k > 0 && p->k < 1) ||
      !(p->eps_s >= 0 && p->eps_s < 0.25) || !(p->grad_eps > 0) || !(p->grad_eps_at > 0) ||
      1.0 - (1.0 - p->k) * p->Omega == 0.0)
    return failf(nullptr, PF_ERR_BAD_ARG, "a dendrite parameter is out of range");
  if (p->thermal != 0 && p->thermal != 1) return failf(nullptr, PF_ERR_BAD_ARG, "thermal must be 0 or 1");
  if (p->thermal) {
    if (!pos(p->Le) || !pos(p->cp) || !std::isfinite(p->latent) || !std::isfinite(p->theta0))
      return failf(nullptr, PF_ERR_BAD_ARG, "thermal mode needs Le, cp > 0, finite latent, theta0");
    if (p->rho_g * p->cp < 0.75)
      return failf(nullptr, PF_ERR_BAD_ARG, "thermal mode needs rho_g * cp >= 3/4 (stability)");
  }
  const unsigned long long n = (unsigned long long)nx * ny * nz;
  pf3f_handle* h = new (std::nothrow) pf3f_handle();
  if (!h) return failf(nullptr, PF_ERR_OOM, "host allocation failed");
  h->p = *p; h->prec = prec; h->stream = (cudaStream_t)cuda_stream;
  h->nx = nx; h->ny = ny; h->nz = nz; h->n = n;
  h->elem = prec == PF_FP64 ? 8 : 4;
  h->thermal = p->thermal;
  h->npop = p->thermal ? NPOPF_TH : NPOPF;
  h->naux = p->thermal ? NAUXF_TH : NAUXF;
  h->nfields = p->thermal ? NFIELDSF_TH : NFIELDSF;
  h->nstate = p->thermal ? NSTATEF_TH : NSTATEF;
  bool ok = true;
  for (int c = 0; c < 2; ++c) {
    ok = ok && cudaMalloc(&h->pop[c], n * h->npop * h->elem) == cudaSuccess;
    ok = ok && cudaMalloc(&h->aux[c], n * h->naux * h->elem) == cudaSuccess;
  }
  ok = ok && cudaMalloc(&h->fields, n * h->nfields * h->elem) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    pf3f_destroy(h);
    return failf(nullptr, PF_ERR_OOM, "device allocation failed");
  }
  *out = h;
  return PF_OK;
}

extern "C" pf_status pf3f_destroy(pf3f_handle* h) {
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

extern "C" const char* pf3f_last_error(const pf3f_handle* h) { return h ? h->err.c_str() : g3f_err.c_str(); }
extern "C" long long pf3f_launch_count(const pf3f_handle* h) { return h ? h->launches : -1; }

extern "C" pf_status pf3f_init_spec(pf3f_handle* h, const double* seeds, int n_seeds, double R_s,
                                    const double* bubbles, int n_bub) {
  if (!h) return PF_ERR_BAD_ARG;
  if (n_seeds < 0 || n_bub < 0 || (n_seeds > 0 && !seeds) || (n_bub > 0 && !bubbles) ||
      !std::isfinite(R_s))
    return failf(h, PF_ERR_BAD_ARG, "bad seeds or bubbles");
  pf_status st = ensure_scratchf(h, 3 * (size_t)n_seeds + 4 * (size_t)n_bub + 1);
  if (st != PF_OK) return st;
  if (n_seeds)
    PF3F_CUDA(h, cudaMemcpyAsync(h->scratch, seeds, 3 * (size_t)n_seeds * sizeof(double),
                                 cudaMemcpyHostToDevice, h->stream));
  if (n_bub)
    PF3F_CUDA(h, cudaMemcpyAsync(h->scratch + 3 * n_seeds, bubbles, 4 * (size_t)n_bub * sizeof(double),
                                 cudaMemcpyHostToDevice, h->stream));
  h->cur = 0;
  st = dispatchf(h, [&](auto s_t, auto r_t) {
    using S = decltype(s_t);
    using R = decltype(r_t);
    ArgsF<S, R> a = argsf<S, R>(h, true);
    a.out = (S*)h->pop[0];
    a.aout = (R*)h->aux[0];
    k_initf<S, R><<<1024, 256, 0, h->stream>>>(a, h->scratch, n_seeds, R_s, h->scratch + 3 * n_seeds,
                                                n_bub, std::sqrt(2.0 * h->p.beta_psi), h->p.W0,
                                                std::sqrt(2.0 * h->p.beta_phi), h->p.W_phi, h->p.k);
    PF3F_CUDA(h, cudaGetLastError());
    if (h->thermal) {
      k_settempf<S, R><<<1024, 256, 0, h->stream>>>(a, nullptr, 1, h->p.theta0);
      PF3F_CUDA(h, cudaGetLastError());
      h->launches++;
    }
    return PF_OK;
  });
  if (st != PF_OK) return st;
  h->launches++;
  return finish_init(h);
}

extern "C" pf_status pf3f_set_fields(pf3f_handle* h, const double* fields7, size_t n) {
  if (!h) return PF_ERR_BAD_ARG;
  if (!fields7 || n != 7 * h->n) return failf(h, PF_ERR_BAD_ARG, "need 7 planes of nx*ny*nz");
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(fields7[i])) return failf(h, PF_ERR_BAD_ARG, "non-finite field");
  pf_status st = ensure_scratchf(h, n);
  if (st != PF_OK) return st;
  PF3F_CUDA(h, cudaMemcpyAsync(h->scratch, fields7, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  h->cur = 0;
  st = dispatchf(h, [&](auto s_t, auto r_t) {
    using S = decltype(s_t);
    using R = decltype(r_t);
    ArgsF<S, R> a = argsf<S, R>(h, true);
    a.out = (S*)h->pop[0];
    a.aout = (R*)h->aux[0];
    k_setf<S, R><<<1024, 256, 0, h->stream>>>(a, h->scratch);
    PF3F_CUDA(h, cudaGetLastError());
    if (h->thermal) {
      k_settempf<S, R><<<1024, 256, 0, h->stream>>>(a, nullptr, 1, h->p.theta0);
      PF3F_CUDA(h, cudaGetLastError());
      h->launches++;
    }
    return PF_OK;
  });
  if (st != PF_OK) return st;
  h->launches++;
  return finish_init(h);
}

extern "C" pf_status pf3f_set_rho_bar(pf3f_handle* h, double rho_bar) {
  if (!h) return PF_ERR_BAD_ARG;
  if (!std::isfinite(rho_bar)) return failf(h, PF_ERR_BAD_ARG, "non-finite rho_bar");
  h->rho_bar = rho_bar;
  return PF_OK;
}
extern "C" double pf3f_get_rho_bar(const pf3f_handle* h) { return h ? h->rho_bar : 0.0; }

extern "C" pf_status pf3f_set_orientation(pf3f_handle* h, const double* seeds7, int n_seeds) {
  if (!h) return PF_ERR_BAD_ARG;
  if (n_seeds < 0 || (n_seeds > 0 && !seeds7)) return failf(h, PF_ERR_BAD_ARG, "bad seeds");
  if (n_seeds == 0) {
    h->rotated = 0;
    return PF_OK;
  }
  std::vector<double> rot(9 * (size_t)n_seeds);
  for (int s = 0; s < n_seeds; ++s) {
    const double* q = seeds7 + 7 * s;
    if (!std::isfinite(q[0]) || !std::isfinite(q[1]) || !std::isfinite(q[2]) ||
        !d3::quat_rows(q + 3, rot.data() + 9 * s))
      return failf(h, PF_ERR_BAD_ARG, "non-finite seed or zero quaternion");
  }
  PF3F_CUDA(h, cudaStreamSynchronize(h->stream));
  if (!h->grain && cudaMalloc(&h->grain, h->n * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    h->grain = nullptr;
    return failf(h, PF_ERR_OOM, "device allocation failed");
  }
  cudaFree(h->rot);
  h->rot = nullptr;
  if (cudaMalloc(&h->rot, 9 * (size_t)n_seeds * h->elem) != cudaSuccess) {
    cudaGetLastError();
    h->rot = nullptr;
    return failf(h, PF_ERR_OOM, "device allocation failed");
  }
  pf_status st = ensure_scratchf(h, 7 * (size_t)n_seeds);
  if (st != PF_OK) return st;
  PF3F_CUDA(h, cudaMemcpyAsync(h->scratch, seeds7, 7 * (size_t)n_seeds * sizeof(double),
                               cudaMemcpyHostToDevice, h->stream));
  d3::k_grain_nearest<7><<<1024, 256, 0, h->stream>>>(h->nx, h->ny, h->nz, h->scratch, n_seeds, h->grain);
  PF3F_CUDA(h, cudaGetLastError());
  h->launches++;
  if (h->prec == PF_FP64) {
    PF3F_CUDA(h, cudaMemcpyAsync(h->rot, rot.data(), rot.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  } else {
    std::vector<float> rf(rot.begin(), rot.end());
    PF3F_CUDA(h, cudaMemcpyAsync(h->rot, rf.data(), rf.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream));
  }
  PF3F_CUDA(h, cudaStreamSynchronize(h->stream));
  h->rotated = 1;
  return PF_OK;
}

extern "C" pf_status pf3f_set_chunk(pf3f_handle* h, int chunk) {
  if (!h) return PF_ERR_BAD_ARG;
  if (chunk < 1 || chunk > 2048) return failf(h, PF_ERR_BAD_ARG, "chunk must be in [1, 2048]");
  h->chunk = chunk;
  return PF_OK;
}

extern "C" pf_status pf3f_step(pf3f_handle* h, int n_steps) {
  if (!h) return PF_ERR_BAD_ARG;
  if (n_steps < 0) return failf(h, PF_ERR_BAD_ARG, "n_steps must be >= 0");
  if (!h->inited) return failf(h, PF_ERR_STATE, "initialise before stepping");
  return dispatchf(h, [&](auto s_t, auto r_t) {
    using S = decltype(s_t);
    using R = decltype(r_t);
    const size_t smem = ring_bytes<R>(h->thermal != 0);
    if (smem > 48 * 1024) {
      auto big = [&](auto kern) {
        return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      };
      PF3F_CUDA(h, big(k_step3f<S, R, false, false>));
      PF3F_CUDA(h, big(k_step3f<S, R, true, false>));
      PF3F_CUDA(h, big(k_step3f<S, R, false, true>));
      PF3F_CUDA(h, big(k_step3f<S, R, true, true>));
    }
    for (int t = 0; t < n_steps; ++t) {
      const ArgsF<S, R> a = argsf<S, R>(h, t == n_steps - 1);
      const int tiles = a.tiles_x * a.tiles_y * a.tiles_z;
      if (h->thermal) {
        if (h->rotated) k_step3f<S, R, true, true><<<tiles, THREADS, smem, h->stream>>>(a);
        else k_step3f<S, R, false, true><<<tiles, THREADS, smem, h->stream>>>(a);
      } else {
        if (h->rotated) k_step3f<S, R, true, false><<<tiles, THREADS, smem, h->stream>>>(a);
        else k_step3f<S, R, false, false><<<tiles, THREADS, smem, h->stream>>>(a);
      }
      PF3F_CUDA(h, cudaGetLastError());
      h->cur ^= 1;
      h->steps++;
      h->launches++;
    }
    return PF_OK;
  });
}

extern "C" pf_status pf3f_get_fields(pf3f_handle* h, double* out, size_t n) {
  if (!h) return PF_ERR_BAD_ARG;
  const size_t need = (size_t)h->nfields * h->n;
  if (!out || n < need) return failf(h, PF_ERR_BAD_ARG, "output must hold pf3f_field_planes planes");
  pf_status st = ensure_scratchf(h, need);
  if (st != PF_OK) return st;
  if (h->prec == PF_FP64)
    k_fieldsf<double><<<1024, 256, 0, h->stream>>>((const double*)h->fields, h->n, h->n, h->nfields, h->scratch);
  else
    k_fieldsf<float><<<1024, 256, 0, h->stream>>>((const float*)h->fields, h->n, h->n, h->nfields, h->scratch);
  PF3F_CUDA(h, cudaGetLastError());
  h->launches++;
  PF3F_CUDA(h, cudaMemcpyAsync(out, h->scratch, need * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  PF3F_CUDA(h, cudaStreamSynchronize(h->stream));
  return PF_OK;
}

extern "C" pf_status pf3f_get_state(pf3f_handle* h, double* out, size_t n) {
  if (!h) return PF_ERR_BAD_ARG;
  const size_t need = (size_t)h->nstate * h->n;
  if (!out || n < need) return failf(h, PF_ERR_BAD_ARG, "output must hold pf3f_state_planes planes");
  pf_status st = ensure_scratchf(h, need);
  if (st != PF_OK) return st;
  st = dispatchf(h, [&](auto s_t, auto r_t) {
    using S = decltype(s_t);
    using R = decltype(r_t);
    k_statef<S, R><<<1024, 256, 0, h->stream>>>((const S*)h->pop[h->cur], (const R*)h->aux[h->cur],
                                                 h->n, h->n, h->thermal, h->scratch);
    PF3F_CUDA(h, cudaGetLastError());
    return PF_OK;
  });
  if (st != PF_OK) return st;
  h->launches++;
  PF3F_CUDA(h, cudaMemcpyAsync(out, h->scratch, need * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  PF3F_CUDA(h, cudaStreamSynchronize(h->stream));
  return PF_OK;
}

extern "C" pf_status pf3f_reduce(pf3f_handle* h, double out[3]) {
  if (!h) return PF_ERR_BAD_ARG;
  if (!out) return failf(h, PF_ERR_BAD_ARG, "NULL output");
  return reduce_fields(h, out);
}

extern "C" int pf3f_field_planes(const pf3f_handle* h) { return h ? h->nfields : -1; }
extern "C" int pf3f_state_planes(const pf3f_handle* h) { return h ? h->nstate : -1; }

extern "C" pf_status pf3f_set_temperature(pf3f_handle* h, const double* theta, size_t n) {
  if (!h) return PF_ERR_BAD_ARG;
  if (!h->thermal) return failf(h, PF_ERR_BAD_ARG, "the handle is not in thermal mode");
  if (!theta || n != h->n) return failf(h, PF_ERR_BAD_ARG, "need theta of nx*ny*nz");
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(theta[i])) return failf(h, PF_ERR_BAD_ARG, "non-finite theta");
  if (!h->inited || h->steps != 0)
    return failf(h, PF_ERR_STATE, "set the temperature after initialisation, before stepping");
  pf_status st = ensure_scratchf(h, n);
  if (st != PF_OK) return st;
  PF3F_CUDA(h, cudaMemcpyAsync(h->scratch, theta, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  st = dispatchf(h, [&](auto s_t, auto r_t) {
    using S = decltype(s_t);
    using R = decltype(r_t);
    ArgsF<S, R> a = argsf<S, R>(h, true);
    a.out = (S*)h->pop[0];
    a.aout = (R*)h->aux[0];
    k_settempf<S, R><<<1024, 256, 0, h->stream>>>(a, h->scratch, 0, 0.0);
    PF3F_CUDA(h, cudaGetLastError());
    return PF_OK;
  });
  if (st != PF_OK) return st;
  h->launches++;
  PF3F_CUDA(h, cudaStreamSynchronize(h->stream));
  return PF_OK;
}

// Thermal totals: sum of the seven temperature populations (rho H), sum theta,
// sum psi; fixed-order partials.
template <typename S, typename R>
__global__ void k_reducef_th(const S* pin, const R* f, unsigned long long ps, unsigned long long n,
                             double* part) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (unsigned long long j = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j < n;
       j += (unsigned long long)gridDim.x * blockDim.x) {
    for (int i = 0; i < 7; ++i) a0 += (double)ld<R>(pl(pin, E_POP + i, ps), j);
    a1 += (double)f[NFIELDSF * ps + j];
    a2 += (double)f[ps + j];
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

extern "C" pf_status pf3f_reduce_thermal(pf3f_handle* h, double out[3]) {
  if (!h) return PF_ERR_BAD_ARG;
  if (!out) return failf(h, PF_ERR_BAD_ARG, "NULL output");
  if (!h->thermal) return failf(h, PF_ERR_BAD_ARG, "the handle is not in thermal mode");
  const int nb = 1024;
  pf_status st = ensure_scratchf(h, 3 * nb + 3);
  if (st != PF_OK) return st;
  st = dispatchf(h, [&](auto s_t, auto r_t) {
    using S = decltype(s_t);
    using R = decltype(r_t);
    k_reducef_th<S, R><<<nb, 256, 0, h->stream>>>((const S*)h->pop[h->cur], (const R*)h->fields,
                                                   h->n, h->n, h->scratch);
    k_reducef_final<<<1, 32, 0, h->stream>>>(h->scratch, nb, h->scratch + 3 * nb);
    PF3F_CUDA(h, cudaGetLastError());
    return PF_OK;
  });
  if (st != PF_OK) return st;
  h->launches += 2;
  PF3F_CUDA(h, cudaMemcpyAsync(out, h->scratch + 3 * nb, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  PF3F_CUDA(h, cudaStreamSynchronize(h->stream));
  return PF_OK;
}
