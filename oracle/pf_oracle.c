/*
 * pf_oracle.c -- plain FP64 CPU oracle for one coupled lattice Boltzmann (LB)
 * time step of the gas-liquid-dendrite phase-field model of Zhan, Chai, Sun,
 * Shi, Geng and Jiang, "Phase-field modeling of dendritic growth with gas
 * bubbles in the solidification of binary alloys" (arXiv 2407.01651).
 *
 * TEST INFRASTRUCTURE.  This file is the checker, not the product.  Only the
 * test-suite, __graft_entry__.smoke() and the CPU-baseline leg of bench.py may
 * build, load or call it; the library path never does.  It shares no code,
 * header, table or helper with the CUDA path.
 *
 * It is written to be read against the paper: one lattice site at a time, one
 * field at a time, dense moment matrices M and M^-1, and two plain passes per
 * step (1: streaming + zeroth moments, 2: gradients + sources + collisions).
 * There is no blocking, no fusion and no reordering of the arithmetic beyond
 * what the formulas state.  Where the paper leaves a choice open (the CAC,
 * Navier-Stokes and solute LB models are only cited, the drag force and the
 * time-stretch realisation are not spelled out), this file takes one reading
 * per open point, numbered R1..R32; each is stated where it is used.
 *
 * Compiled twice from this one source:
 *   real_t = double                          -> liboracle_d.so
 *   real_t = double complex (-DPF_ORACLE_Z)  -> liboracle_z.so
 * and, for the flop count per lattice update only, a third time as C++ with
 * an instrumented scalar (-DPF_ORACLE_COUNT, counting.h) -> liboracle_count.so.
 * The complex build is the complex-step derivative (Squire & Trapp, SIAM Rev.
 * 1998; Martins, Sturdza & Alonso, ACM TOMS 2003): a parameter is perturbed by
 * i*h and Im(J)/h is dJ/dparameter to rounding error, with no subtractive
 * cancellation.  Every operation on the step path is analytic (no abs, min,
 * max or comparison of a perturbed value), so the derivative is the exact
 * derivative of the discrete map.
 *
 * Parity status: every function here is pinned by the not-gpu tests (closed
 * forms, invariants, special cases) except the long-time morphology and the
 * Gibbs-Thomson trend, which are "parity unpinned" (the paper shows figures
 * only).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

#ifdef PF_ORACLE_Z
#include <complex.h>
typedef double complex real_t;
#define RSQRT_(x) csqrt(x)
#define RE_(x) creal(x)
#define IM_(x) cimag(x)
#elif defined(PF_ORACLE_COUNT)
/* the flop-counting build: this file compiled as C++ (counting.h) */
#include "counting.h"
typedef pf_count::Counting real_t;
#define RSQRT_(x) pf_count::sqrt(x)
#define RE_(x) ((x).v)
#define IM_(x) (0.0)
pf_count::Tally pf_count::g_tally = {0, 0, 0, 0};
extern "C" {
#else
typedef double real_t;
#define RSQRT_(x) sqrt(x)
#define RE_(x) (x)
#define IM_(x) (0.0)
#endif

/* ------------------------------------------------------------------------ */
/* Lattices (Appendix B: D2Q9 for Navier-Stokes and the conservative        */
/* Allen-Cahn equation, D2Q5 for the dendrite, solute and temperature).     */
/* ------------------------------------------------------------------------ */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double W9[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                             1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
/* D2Q5 weights: the paper gives none; reading R12: w0 = 1/3, wi = 1/6. */
static const double W5[5] = {1.0 / 3, 1.0 / 6, 1.0 / 6, 1.0 / 6, 1.0 / 6};
static const double CS2 = 1.0 / 3.0;

/* Moment matrices M0 (Appendix B, Lambda = M^-1 S M with lattice speed 1 so
 * C_d = I).  D2Q9: Lallemand-Luo order (rho, e, eps, jx, qx, jy, qy, pxx, pxy).
 * D2Q5: (zeroth, jx, jy, energy, pxx-pyy).  Rows are mutually orthogonal, so
 * M^-1 = M^T diag(1/|row_k|^2); built in build_inverse(). */
static const double M9[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},
    {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},
    {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},
    {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},
    {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1}};
static const double M5[5][5] = {
    {1, 1, 1, 1, 1},
    {0, 1, 0, -1, 0},
    {0, 0, 1, 0, -1},
    {-4, 1, 1, 1, 1},
    {0, 1, -1, 1, -1}};
static double M9I[9][9], M5I[5][5];
static int inverse_built = 0;

static void build_inverse(void) {
  if (inverse_built) return;
  for (int k = 0; k < 9; ++k) {
    double n2 = 0;
    for (int j = 0; j < 9; ++j) n2 += M9[k][j] * M9[k][j];
    for (int j = 0; j < 9; ++j) M9I[j][k] = M9[k][j] / n2;
  }
  for (int k = 0; k < 5; ++k) {
    double n2 = 0;
    for (int j = 0; j < 5; ++j) n2 += M5[k][j] * M5[k][j];
    for (int j = 0; j < 5; ++j) M5I[j][k] = M5[k][j] / n2;
  }
  inverse_built = 1;
}

/* ------------------------------------------------------------------------ */
/* Parameters, in the paper's symbols (lattice units, dx = dt = 1).         */
/* ------------------------------------------------------------------------ */
enum {
  P_RHO_L, P_RHO_G, P_NU, P_SIGMA, P_W_PHI, P_M_PHI, P_BETA_PHI, P_BETA_PSI,
  P_BETA_INTER, P_W0, P_TAU0, P_EPS_S, P_K, P_D, P_OMEGA, P_G, P_GRAD_EPS,
  P_S_E, P_S_EPS, P_GRAD_EPS_AT,
  /* temperature coupling (Section 2.1 and Appendix B): P_THERMAL = 0 keeps the
   * isothermal closure theta = theta_sys, F(U) = 1 (Eq. eq-Tsys); 1 solves the
   * temperature equation with Lewis number Le = alpha / D, latent-heat factor
   * c_p^s / c_p, uniform initial temperature theta0 and lattice heat capacity
   * c_p (reading R28). */
  P_THERMAL, P_LE, P_LATENT, P_THETA0, P_CP,
  /* velocity at an inlet side (reading R32) */
  P_VIN_X, P_VIN_Y, NPAR
};

/* Boundary type of each side (reading R31): x- (left), x+ (right), y- (bottom),
 * y+ (top), all at the half-way position between the last site and its ghost. */
enum { BC_PERIODIC = 0, BC_SYMMETRIC = 1, BC_WALL = 2, BC_FARFIELD = 3, BC_INLET = 4,
       BC_OUTLET = 5, BC_INLET_NEE = 6 };

typedef struct {
  int nx, ny, n;
  int NX, NY, x0, y0;       /* placement of this lattice in a periodic NX x NY one */
  int bc[4];                /* boundary types: x-, x+, y-, y+ */
  real_t par[NPAR];
  real_t rho_bar;           /* domain-mean density (reading R13) */
  int rho_bar_fixed;
  long steps;
  /* state after the last step: post-collision populations + lagged values */
  real_t *f[9], *h[9], *gpre[5], *gpost[5], *rr, *s[5];
  real_t *phi_o, *C_o, *vx_o, *vy_o, *Q_o;
  real_t *e[5], *H_o;       /* temperature populations and lagged H (thermal mode) */
  double *cth, *sth;        /* grain orientation per site (reading R10) */
  /* macroscopic fields of the last step: phi, psi, C, U, p, vx, vy, mu_phi, theta */
  real_t *fld[9];
  /* scratch for the streaming pass */
  real_t *fS[9], *hS[9], *gS[5], *sS[5], *phiS, *psiS, *CS, *psiOld;
  real_t *eS[5], *US;
  /* next-state buffers */
  real_t *nf[9], *nh[9], *ngpre[5], *ngpost[5], *nrr, *ns[5];
  real_t *nphi_o, *nC_o, *nvx_o, *nvy_o, *nQ_o;
  real_t *ne[5], *nH_o;
  real_t *block;
} ostate;

enum { F_PHI, F_PSI, F_C, F_U, F_P, F_VX, F_VY, F_MU, F_THETA, NFLD };

/* Derived coefficients of the isothermal closure and the thin-interface map. */
typedef struct {
  real_t lam;      /* lambda' = 15 lambda / 16 = D tau0 / (a2' W0^2), a2' = 47/75 */
  real_t Mcinf;    /* M c_inf = 1 - (1-k) Omega                                  */
  real_t theta;    /* theta_sys = -M c_inf Omega / (1 - (1-k) Omega)             */
  real_t kappa;    /* sqrt(2 beta_phi) / W_phi                                   */
  real_t fs_coef;  /* 6 sigma / ((phi_l-phi_g)^3 W_phi sqrt(2 beta_phi))          */
  real_t s_nu, s_q, s_phi;
  real_t kT;       /* thermal conductivity k_T = Le D rho_l c_p                   */
  real_t s_th;     /* k_T = (1/s_th - 1/2) c_s^2 (Appendix B, temperature)       */
} derived_t;

static derived_t derive(const ostate *st) {
  derived_t d;
  const real_t *p = st->par;
  /* Appendix A (end): tau0 D / W^2 = a2' lambda' with a2' = 47/75. */
  d.lam = p[P_D] * p[P_TAU0] / ((47.0 / 75.0) * p[P_W0] * p[P_W0]);
  /* Eq. (eq-Tsys): theta_sys and M c_inf for the solutal case (B). */
  d.Mcinf = 1.0 - (1.0 - p[P_K]) * p[P_OMEGA];
  d.theta = -d.Mcinf * p[P_OMEGA] / (1.0 - (1.0 - p[P_K]) * p[P_OMEGA]);
  d.kappa = RSQRT_(2.0 * p[P_BETA_PHI]) / p[P_W_PHI];
  /* Surface tension force, Section 2.2, with phi_l - phi_g = 1. */
  d.fs_coef = 6.0 * p[P_SIGMA] / (p[P_W_PHI] * RSQRT_(2.0 * p[P_BETA_PHI]));
  /* mu = rho nu (reading R23): nu = (1/s_nu - 1/2) c_s^2. */
  d.s_nu = 1.0 / (p[P_NU] / CS2 + 0.5);
  d.s_q = 8.0 * (2.0 - d.s_nu) / (8.0 - d.s_nu);   /* reading R7 */
  /* CAC mobility M_phi = (1/s - 1/2) c_s^2. */
  d.s_phi = 1.0 / (p[P_M_PHI] / CS2 + 0.5);
  /* Temperature (reading R28): Le = alpha / D (Section 2.1) with alpha =
   * k_T / (rho_l c_p) the liquid's diffusivity and k_T uniform. */
  d.kT = p[P_LE] * p[P_D] * p[P_RHO_L] * p[P_CP];
  d.s_th = 1.0 / (d.kT / CS2 + 0.5);
  return d;
}

/* ------------------------------------------------------------------------ */
/* Allocation                                                               */
/* ------------------------------------------------------------------------ */
#define NPLANES (9 + 9 + 5 + 5 + 1 + 5 + 5)  /* one state copy */

ostate *or_new(int nx, int ny) {
  build_inverse();
  if (nx < 1 || ny < 1) return NULL;
  ostate *st = (ostate *)calloc(1, sizeof(ostate));
  if (!st) return NULL;
  st->nx = nx; st->ny = ny; st->n = nx * ny;
  st->NX = nx; st->NY = ny; st->x0 = 0; st->y0 = 0;
  size_t n = (size_t)st->n;
  /* 2 state copies (+ 6 temperature planes each) + 9 fields + streaming
   * scratch (28 pops + 4 moments, + 5 temperature pops + U) */
  size_t nplanes = 2 * (NPLANES + 6) + 9 + 28 + 4 + 6;
  st->block = (real_t *)calloc(nplanes * n, sizeof(real_t));
  st->cth = (double *)calloc(n, sizeof(double));
  st->sth = (double *)calloc(n, sizeof(double));
  if (!st->block || !st->cth || !st->sth) {
    free(st->block); free(st->cth); free(st->sth); free(st);
    return NULL;
  }
  real_t *q = st->block;
#define TAKE(ptr) do { (ptr) = q; q += n; } while (0)
  for (int i = 0; i < 9; ++i) TAKE(st->f[i]);
  for (int i = 0; i < 9; ++i) TAKE(st->h[i]);
  for (int i = 0; i < 5; ++i) TAKE(st->gpre[i]);
  for (int i = 0; i < 5; ++i) TAKE(st->gpost[i]);
  TAKE(st->rr);
  for (int i = 0; i < 5; ++i) TAKE(st->s[i]);
  TAKE(st->phi_o); TAKE(st->C_o); TAKE(st->vx_o); TAKE(st->vy_o); TAKE(st->Q_o);
  for (int i = 0; i < 5; ++i) TAKE(st->e[i]);
  TAKE(st->H_o);
  for (int i = 0; i < 9; ++i) TAKE(st->nf[i]);
  for (int i = 0; i < 9; ++i) TAKE(st->nh[i]);
  for (int i = 0; i < 5; ++i) TAKE(st->ngpre[i]);
  for (int i = 0; i < 5; ++i) TAKE(st->ngpost[i]);
  TAKE(st->nrr);
  for (int i = 0; i < 5; ++i) TAKE(st->ns[i]);
  TAKE(st->nphi_o); TAKE(st->nC_o); TAKE(st->nvx_o); TAKE(st->nvy_o); TAKE(st->nQ_o);
  for (int i = 0; i < 5; ++i) TAKE(st->ne[i]);
  TAKE(st->nH_o);
  for (int i = 0; i < NFLD; ++i) TAKE(st->fld[i]);
  for (int i = 0; i < 9; ++i) TAKE(st->fS[i]);
  for (int i = 0; i < 9; ++i) TAKE(st->hS[i]);
  for (int i = 0; i < 5; ++i) TAKE(st->gS[i]);
  for (int i = 0; i < 5; ++i) TAKE(st->sS[i]);
  TAKE(st->phiS); TAKE(st->psiS); TAKE(st->CS); TAKE(st->psiOld);
  for (int i = 0; i < 5; ++i) TAKE(st->eS[i]);
  TAKE(st->US);
#undef TAKE
  for (size_t i = 0; i < n; ++i) st->cth[i] = 1.0;
  return st;
}

void or_free(ostate *st) {
  if (!st) return;
  free(st->block); free(st->cth); free(st->sth); free(st);
}

int or_npar(void) { return NPAR; }

void or_set_params(ostate *st, const double *pv) {
  for (int i = 0; i < NPAR; ++i) st->par[i] = pv[i];
}

/* Complex build only: add i*h to parameter idx (complex-step direction). */
void or_perturb_param(ostate *st, int idx, double h) {
#ifdef PF_ORACLE_Z
  if (idx >= 0 && idx < NPAR) st->par[idx] += I * h;
#else
  (void)st; (void)idx; (void)h;
#endif
}

void or_set_window(ostate *st, int NX, int NY, int x0, int y0) {
  st->NX = NX; st->NY = NY; st->x0 = x0; st->y0 = y0;
}

void or_set_rho_bar(ostate *st, double rho_bar) {
  st->rho_bar = rho_bar; st->rho_bar_fixed = 1;
}

double or_get_rho_bar(const ostate *st) { return RE_(st->rho_bar); }
long or_get_steps(const ostate *st) { return st->steps; }

/* ------------------------------------------------------------------------ */
/* Pointwise model functions (Section 2.1, Appendix B).                     */
/* ------------------------------------------------------------------------ */

/* Supersaturation from the dimensionless concentration, Eq. for u with
 * beta_psi = 1/4, psi_s = 1, psi_l = -1 and U = (e^u - 1)/(1 - k). */
static real_t supersat(const ostate *st, real_t C, real_t psi) {
  real_t k = st->par[P_K];
  return (2.0 * C / (1.0 + k - (1.0 - k) * psi) - 1.0) / (1.0 - k);
}

/* Q_psi = -[f2' + d_psi f3 + lambda p'(psi) (theta + M c_inf U)], Appendix B,
 * with f2 = beta_psi (1-psi^2)^2, f3 = beta_inter (1-phi)^2 (1+psi)^2
 * (Eq. eq-douWell, eq-f3Inter) and lambda p' = lambda' (1-psi^2)^2. */
static real_t q_psi_at(const ostate *st, const derived_t *d, real_t phi, real_t psi,
                       real_t U, real_t theta) {
  const real_t *p = st->par;
  real_t one_m = 1.0 - psi * psi;
  real_t f2p = -4.0 * p[P_BETA_PSI] * psi * one_m;
  real_t f3p = 2.0 * p[P_BETA_INTER] * (1.0 - phi) * (1.0 - phi) * (1.0 + psi);
  real_t drive = d->lam * one_m * one_m * (theta + d->Mcinf * U);
  return -(f2p + f3p + drive);
}

/* Isothermal form: theta = theta_sys everywhere (Eq. eq-Tsys). */
static real_t q_psi(const ostate *st, const derived_t *d, real_t phi, real_t psi,
                    real_t U) {
  return q_psi_at(st, d, phi, psi, U, d->theta);
}

/* F(U) = 1/Le + M c_inf [1 + (1-k) U] (Section 2.1, thin-interface limit). */
static real_t f_of_u(const ostate *st, const derived_t *d, real_t U) {
  return 1.0 / st->par[P_LE] + d->Mcinf * (1.0 + (1.0 - st->par[P_K]) * U);
}

static int thermal_on(const ostate *st) { return RE_(st->par[P_THERMAL]) != 0.0; }

/* Anisotropy of the solid-liquid interface for a grain rotated by theta
 * (reading R10).  g = grad psi, n_psi = -g/|g|_reg (Section 2.1, regularised
 * norm of reading R6), expressed in the crystal frame n' = R(-theta) n.
 * The anisotropy function of Section 3.3,
 *   a_s = (1 - 3 eps) [1 + 4 eps/(1 - 3 eps) sum n'_a^4],
 * is written as a_s = 1 + eps (4 sum n'^4 - 3 |n'|^4), equal to it for a unit
 * normal and tending to 1 where the normal is undefined (reading R6).  The
 * anisotropy vector N_a = |g|^2 a_s d a_s / d(d_a psi) (Section 2.1) of this
 * function of g is, with |g| -> |g|_reg,
 *   N'_a = -16 eps a_s |g|_reg n'_a [n'_a^2 - sum n'^4 - 3/4 |n'|^2 (1 - |n'|^2)],
 * and N = R(theta) N'.  Returns a_s, N and |g|_reg. */
static void aniso(real_t gx, real_t gy, double ct, double sn, real_t eps, real_t geps,
                  real_t *as_out, real_t *Nx, real_t *Ny, real_t *gmag) {
  const real_t gx_r = ct * gx + sn * gy;
  const real_t gy_r = -sn * gx + ct * gy;
  const real_t smag = RSQRT_(gx * gx + gy * gy + geps * geps);
  const real_t nx_r = -gx_r / smag, ny_r = -gy_r / smag;
  const real_t n2 = nx_r * nx_r + ny_r * ny_r;
  const real_t s4 = nx_r * nx_r * nx_r * nx_r + ny_r * ny_r * ny_r * ny_r;
  const real_t as = 1.0 + eps * (4.0 * s4 - 3.0 * n2 * n2);
  const real_t iso = s4 + 0.75 * n2 * (1.0 - n2);
  const real_t Nx_r = -16.0 * eps * as * smag * nx_r * (nx_r * nx_r - iso);
  const real_t Ny_r = -16.0 * eps * as * smag * ny_r * (ny_r * ny_r - iso);
  *Nx = ct * Nx_r - sn * Ny_r;
  *Ny = sn * Nx_r + ct * Ny_r;
  *as_out = as;
  *gmag = smag;
}

/* ------------------------------------------------------------------------ */
/* Equilibria (readings R1 for the cited CAC / NS / solute models).          */
/* ------------------------------------------------------------------------ */

/* Pressure-based incompressible NS equilibrium:
 * f_i^eq = w_i p/cs2 - delta_i0 p/cs2 + rho w_i [c.v/cs2 + (c.v)^2/(2cs4) - v^2/(2cs2)]. */
static void feq_ns(real_t p, real_t rho, real_t vx, real_t vy, real_t out[9]) {
  real_t v2 = vx * vx + vy * vy;
  for (int i = 0; i < 9; ++i) {
    real_t cu = CX[i] * vx + CY[i] * vy;
    real_t s_i = W9[i] * (cu / CS2 + cu * cu / (2 * CS2 * CS2) - v2 / (2 * CS2));
    out[i] = W9[i] * p / CS2 + rho * s_i;
    if (i == 0) out[i] -= p / CS2;
  }
}

/* CAC equilibrium h_i^eq = w_i phi (1 + c.v/cs2). */
static void heq_cac(real_t phi, real_t vx, real_t vy, real_t out[9]) {
  for (int i = 0; i < 9; ++i)
    out[i] = W9[i] * phi * (1.0 + (CX[i] * vx + CY[i] * vy) / CS2);
}

/* Solute equilibrium (reading R1): C is the conserved and diffused variable,
 * s_i^eq = w_i C + w_i c_i.Jeq / cs2, with the remaining fluxes in Jeq. */
static void seq_sol(real_t C, real_t jx, real_t jy, real_t out[5]) {
  for (int i = 0; i < 5; ++i)
    out[i] = W5[i] * C + W5[i] * (CX[i] * jx + CY[i] * jy) / CS2;
}

/* Temperature equilibrium (Appendix B) for the variable H = c_p theta -
 * c_p^s h(psi):  g_0^eq = rho H + (w_0 - 1) theta,
 *                g_i^eq = w_i theta + w_i c_i . (rho H v) / c_s^2  (i != 0),
 * so that sum g^eq = rho H, sum c g^eq = rho H v, sum c c g^eq = c_s^2 theta I. */
static void teq_th(real_t rhoH, real_t theta, real_t jx, real_t jy, real_t out[5]) {
  for (int i = 0; i < 5; ++i)
    out[i] = W5[i] * theta + W5[i] * (CX[i] * jx + CY[i] * jy) / CS2;
  out[0] = rhoH + (W5[0] - 1.0) * theta;
}

/* ------------------------------------------------------------------------ */
/* MRT collision in moment space (Appendix B, Lambda = M^-1 S M):           */
/*   m* = m - S (m - m_eq) + (I - S/2) M G + M Fd,    f* = M^-1 m*          */
/* G: terms that enter through (delta_ij - Lambda_ij/2); Fd: terms that     */
/* enter directly (the dendrite source F + dt/2 dF/dt).                     */
/* ------------------------------------------------------------------------ */
static void collide9(const real_t f[9], const real_t feq[9], const real_t S[9],
                     const real_t G[9], real_t out[9]) {
  real_t m[9], meq[9], mg[9], ms[9];
  for (int k = 0; k < 9; ++k) {
    m[k] = meq[k] = mg[k] = 0;
    for (int j = 0; j < 9; ++j) {
      m[k] += M9[k][j] * f[j];
      meq[k] += M9[k][j] * feq[j];
      mg[k] += M9[k][j] * G[j];
    }
    ms[k] = m[k] - S[k] * (m[k] - meq[k]) + (1.0 - 0.5 * S[k]) * mg[k];
  }
  for (int j = 0; j < 9; ++j) {
    out[j] = 0;
    for (int k = 0; k < 9; ++k) out[j] += M9I[j][k] * ms[k];
  }
}

static void collide5(const real_t f[5], const real_t feq[5], const real_t S[5],
                     const real_t G[5], const real_t Fd[5], real_t out[5]) {
  real_t m[5], meq[5], mg[5], mf[5], ms[5];
  for (int k = 0; k < 5; ++k) {
    m[k] = meq[k] = mg[k] = mf[k] = 0;
    for (int j = 0; j < 5; ++j) {
      m[k] += M5[k][j] * f[j];
      meq[k] += M5[k][j] * feq[j];
      mg[k] += M5[k][j] * G[j];
      mf[k] += M5[k][j] * Fd[j];
    }
    ms[k] = m[k] - S[k] * (m[k] - meq[k]) + (1.0 - 0.5 * S[k]) * mg[k] + mf[k];
  }
  for (int j = 0; j < 5; ++j) {
    out[j] = 0;
    for (int k = 0; k < 5; ++k) out[j] += M5I[j][k] * ms[k];
  }
}

/* ------------------------------------------------------------------------ */
/* Initial state                                                             */
/* ------------------------------------------------------------------------ */

/* Minimum-image signed offset of a periodic coordinate. */
static double min_image(double d, double L) {
  d = fmod(d, L);
  if (d < -0.5 * L) d += L;
  if (d >= 0.5 * L) d -= L;
  return d;
}

/* Signed offset along an axis: the minimum image on a periodic axis, the
 * plain difference otherwise. */
static double axis_offset(double d, double L, int periodic) {
  return periodic ? min_image(d, L) : d;
}

void or_set_bc(ostate *st, int xm, int xp, int ym, int yp) {
  st->bc[0] = xm; st->bc[1] = xp; st->bc[2] = ym; st->bc[3] = yp;
}

/* Set every population to its equilibrium for given macroscopic fields, the
 * lagged values equal to the current ones (first-step time derivatives are
 * zero) and the dendrite time-stretch factor 1/a_s^2 = 1.  Reading R20 of the
 * initial state.  Arrays: phi, psi, C, vx, vy, p, theta (host, n each; vx, vy,
 * p and theta may be NULL: zero velocity and pressure, theta0).  In thermal
 * mode the lagged dendrite source starts at its pointwise part Q_psi / F(U)
 * (reading R29). */
void or_init_from_fields(ostate *st, const double *phi, const double *psi,
                         const double *C, const double *vx, const double *vy,
                         const double *p, const double *theta) {
  derived_t d = derive(st);
  const real_t *par = st->par;
  double sphi = 0;
  for (int idx = 0; idx < st->n; ++idx) {
    real_t ph = phi[idx], ps = psi[idx], c = C[idx];
    real_t ux = vx ? vx[idx] : 0.0, uy = vy ? vy[idx] : 0.0;
    real_t pp = p ? p[idx] : 0.0;
    real_t rho = par[P_RHO_G] + ph * (par[P_RHO_L] - par[P_RHO_G]);
    real_t tmp[9];
    feq_ns(pp, rho, ux, uy, tmp);
    for (int i = 0; i < 9; ++i) st->f[i][idx] = tmp[i];
    heq_cac(ph, ux, uy, tmp);
    for (int i = 0; i < 9; ++i) st->h[i][idx] = tmp[i];
    for (int i = 0; i < 5; ++i) st->gpre[i][idx] = st->gpost[i][idx] = W5[i] * ps;
    st->rr[idx] = 1.0;
    real_t U = supersat(st, c, ps);
    real_t t5[5];
    seq_sol(c, c * ux, c * uy, t5);
    for (int i = 0; i < 5; ++i) st->s[i][idx] = t5[i];
    st->phi_o[idx] = ph; st->C_o[idx] = c;
    st->vx_o[idx] = ux; st->vy_o[idx] = uy;
    if (thermal_on(st)) {
      /* H = c_p theta - c_p^s h(psi) = c_p [theta - (c_p^s/c_p) h(psi)],
       * h = (1+psi)/2 (Appendix B) */
      real_t th = theta ? theta[idx] : par[P_THETA0];
      real_t H = par[P_CP] * (th - par[P_LATENT] * 0.5 * (1.0 + ps));
      teq_th(rho * H, th, rho * H * ux, rho * H * uy, t5);
      for (int i = 0; i < 5; ++i) st->e[i][idx] = t5[i];
      st->H_o[idx] = H;
      st->Q_o[idx] = q_psi_at(st, &d, ph, ps, U, th) / f_of_u(st, &d, U);
      st->fld[F_THETA][idx] = th;
    } else {
      for (int i = 0; i < 5; ++i) st->e[i][idx] = 0.0;
      st->H_o[idx] = 0.0;
      st->Q_o[idx] = q_psi(st, &d, ph, ps, U);
      st->fld[F_THETA][idx] = d.theta;
    }
    st->fld[F_PHI][idx] = ph; st->fld[F_PSI][idx] = ps; st->fld[F_C][idx] = c;
    st->fld[F_U][idx] = U; st->fld[F_P][idx] = pp;
    st->fld[F_VX][idx] = ux; st->fld[F_VY][idx] = uy; st->fld[F_MU][idx] = 0.0;
    sphi += phi[idx];
  }
  if (!st->rho_bar_fixed)
    st->rho_bar = par[P_RHO_G] + (sphi / st->n) * (par[P_RHO_L] - par[P_RHO_G]);
  st->steps = 0;
}

/* Grain orientation per site: the angle of the nearest seed (minimum image,
 * first seed on an exact tie), reading R10.  seeds: n x (x, y, theta). */
void or_set_orientation(ostate *st, const double *seeds, int n_seeds) {
  for (int y = 0; y < st->ny; ++y)
    for (int x = 0; x < st->nx; ++x) {
      int idx = y * st->nx + x;
      double th = 0.0, best = 0.0;
      for (int s = 0; s < n_seeds; ++s) {
        double dx = axis_offset((st->x0 + x) - seeds[3 * s], st->NX, st->bc[0] == BC_PERIODIC);
        double dy = axis_offset((st->y0 + y) - seeds[3 * s + 1], st->NY, st->bc[2] == BC_PERIODIC);
        double r2 = dx * dx + dy * dy;
        if (s == 0 || r2 < best) { best = r2; th = seeds[3 * s + 2]; }
      }
      st->cth[idx] = cos(th);
      st->sth[idx] = sin(th);
    }
}

/* Macroscopic initial fields from seeds and bubbles (readings R9, R21):
 *   psi = max_s tanh( sqrt(2 beta_psi) (R_s - r_s) / W0 )      (Eq. eq-psiEq)
 *   phi = min_b [1/2 + 1/2 tanh( sqrt(2 beta_phi) (r_b - R_b) / (2 W_phi) )]
 *                                                               (Eq. eq-phiEq)
 *   C   = phi [1 - (1-k) h(psi)],  h = (1+psi)/2   (U = 0 in melt and solid,
 *                                                   solute vacuum in the gas)
 * Outputs phi, psi, C (n each). */
void or_fields_from_spec(const ostate *st, const double *seeds, int n_seeds,
                         double R_s, const double *bubbles, int n_bub,
                         double *phi, double *psi, double *C) {
  double bpsi = RE_(st->par[P_BETA_PSI]), bphi = RE_(st->par[P_BETA_PHI]);
  double W0 = RE_(st->par[P_W0]), Wphi = RE_(st->par[P_W_PHI]);
  double k = RE_(st->par[P_K]);
  for (int y = 0; y < st->ny; ++y)
    for (int x = 0; x < st->nx; ++x) {
      int idx = y * st->nx + x;
      double ps = -1.0;
      for (int s = 0; s < n_seeds; ++s) {
        double dx = axis_offset((st->x0 + x) - seeds[3 * s], st->NX, st->bc[0] == BC_PERIODIC);
        double dy = axis_offset((st->y0 + y) - seeds[3 * s + 1], st->NY, st->bc[2] == BC_PERIODIC);
        double v = tanh(sqrt(2.0 * bpsi) * (R_s - sqrt(dx * dx + dy * dy)) / W0);
        if (s == 0 || v > ps) ps = v;
      }
      double ph = 1.0;
      for (int b = 0; b < n_bub; ++b) {
        double dx = axis_offset((st->x0 + x) - bubbles[3 * b], st->NX, st->bc[0] == BC_PERIODIC);
        double dy = axis_offset((st->y0 + y) - bubbles[3 * b + 1], st->NY, st->bc[2] == BC_PERIODIC);
        double v = 0.5 + 0.5 * tanh(sqrt(2.0 * bphi) *
                                    (sqrt(dx * dx + dy * dy) - bubbles[3 * b + 2]) /
                                    (2.0 * Wphi));
        if (b == 0 || v < ph) ph = v;
      }
      phi[idx] = ph;
      psi[idx] = ps;
      C[idx] = ph * (1.0 - (1.0 - k) * 0.5 * (1.0 + ps));
    }
}

/* Mean of the initial phi over the whole periodic NX x NY lattice (the
 * buoyancy reference rho_bar of reading R13 for a windowed oracle). */
double or_mean_phi_global(const ostate *st, const double *bubbles, int n_bub) {
  double bphi = RE_(st->par[P_BETA_PHI]), Wphi = RE_(st->par[P_W_PHI]);
  double total = 0.0;
#pragma omp parallel for reduction(+ : total) schedule(static)
  for (int y = 0; y < st->NY; ++y) {
    double row = 0.0;
    for (int x = 0; x < st->NX; ++x) {
      double ph = 1.0;
      for (int b = 0; b < n_bub; ++b) {
        double dx = axis_offset(x - bubbles[3 * b], st->NX, st->bc[0] == BC_PERIODIC);
        double dy = axis_offset(y - bubbles[3 * b + 1], st->NY, st->bc[2] == BC_PERIODIC);
        double v = 0.5 + 0.5 * tanh(sqrt(2.0 * bphi) *
                                    (sqrt(dx * dx + dy * dy) - bubbles[3 * b + 2]) /
                                    (2.0 * Wphi));
        if (b == 0 || v < ph) ph = v;
      }
      row += ph;
    }
    total += row;
  }
  return total / ((double)st->NX * st->NY);
}

/* Convenience: orientation + fields + equilibrium populations. */
int or_init_spec(ostate *st, const double *seeds, int n_seeds, double R_s,
                 const double *bubbles, int n_bub) {
  size_t n = (size_t)st->n;
  double *buf = (double *)malloc(3 * n * sizeof(double));
  if (!buf) return -1;
  or_set_orientation(st, seeds, n_seeds);
  or_fields_from_spec(st, seeds, n_seeds, R_s, bubbles, n_bub, buf, buf + n,
                      buf + 2 * n);
  or_init_from_fields(st, buf, buf + n, buf + 2 * n, NULL, NULL, NULL, NULL);
  free(buf);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* One coupled step                                                          */
/* ------------------------------------------------------------------------ */
static inline int wrap(int a, int n) { a %= n; return a < 0 ? a + n : a; }

/* Direction maps of D2Q9 (and of its D2Q5 subset 0..4): opposite, and the
 * reflections that flip c_x or c_y. */
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const int MIRX[9] = {0, 3, 2, 1, 4, 6, 5, 8, 7};
static const int MIRY[9] = {0, 1, 4, 3, 2, 8, 7, 6, 5};

/* Far-field values of the Dirichlet sides (Section 4: psi = psi_l, C = 1,
 * theta = -Omega, here theta0), and U of that state (0). */
static const double PSI_FAR = -1.0, C_FAR = 1.0;

/* Source of the population of direction i pulled by site (x, y) (readings
 * R31, R32).  Periodic sides wrap; a symmetric side reflects the source site
 * about the half-way plane and the direction with it; an outlet clamps the
 * source to the last site (zero gradient; the NS lattice instead takes a
 * pressure anti-bounce-back, applied by the caller); a wall, far-field or
 * inlet side returns the site's own post-collision population of the opposite
 * direction (half-way bounce-back), which the far-field side turns into an
 * anti-bounce-back on the lattices with a Dirichlet value and the inlet into a
 * moving-wall bounce-back for the flow and anti-bounce-backs for the scalars.
 * Returns 0 (plain or reflected source), 1 (wall), 2 (far field), 3 (inlet),
 * 4 (outlet, clamped source) or 5 (non-equilibrium extrapolation inlet: the
 * source is the boundary node, a ghost one site beyond the side, whose
 * populations the caller builds from the fluid site next to it, returned in
 * *src), a bounce winning over the rest where two sides are crossed, then
 * the extrapolation, then the clamp; *src and *q give the site and the
 * direction to read. */
static int bounce_rank(int t) {
  return t == BC_WALL ? 1 : (t == BC_FARFIELD ? 2 : (t == BC_INLET ? 3 : 0));
}

static int pull_src(const ostate *st, int x, int y, int i, int *src, int *q) {
  const int nx = st->nx, ny = st->ny;
  int sx = x - CX[i], sy = y - CY[i], qi = i, bounce = 0, outlet = 0, nee = 0;
  if (sx < 0 || sx >= nx) {
    const int t = st->bc[sx < 0 ? 0 : 1];
    if (t == BC_PERIODIC) sx = wrap(sx, nx);
    else if (t == BC_SYMMETRIC) { sx = sx < 0 ? -1 - sx : 2 * nx - 1 - sx; qi = MIRX[qi]; }
    else if (t == BC_OUTLET) { sx = sx < 0 ? 0 : nx - 1; outlet = 1; }
    else if (t == BC_INLET_NEE) { sx = sx < 0 ? 0 : nx - 1; nee = 1; }
    else if (bounce_rank(t) > bounce) bounce = bounce_rank(t);
  }
  if (sy < 0 || sy >= ny) {
    const int t = st->bc[sy < 0 ? 2 : 3];
    if (t == BC_PERIODIC) sy = wrap(sy, ny);
    else if (t == BC_SYMMETRIC) { sy = sy < 0 ? -1 - sy : 2 * ny - 1 - sy; qi = MIRY[qi]; }
    else if (t == BC_OUTLET) { sy = sy < 0 ? 0 : ny - 1; outlet = 1; }
    else if (t == BC_INLET_NEE) { sy = sy < 0 ? 0 : ny - 1; nee = 1; }
    else if (bounce_rank(t) > bounce) bounce = bounce_rank(t);
  }
  if (bounce) { *src = y * nx + x; *q = OPP[i]; return bounce; }
  *src = sy * nx + sx;
  *q = qi;
  return nee ? 5 : (outlet ? 4 : 0);
}

/* The lattices other than NS see a non-equilibrium-extrapolation inlet as an
 * inlet (reading R37): anti-bounce-back at the site itself. */
static int scalar_src(const ostate *st, int x, int y, int i, int *src, int *q) {
  const int mode = pull_src(st, x, y, i, src, q);
  if (mode != 5) return mode;
  *src = y * st->nx + x;
  *q = OPP[i];
  return 3;
}

/* Kinds of field read on the stencil neighbourhood, for the ghost values. */
enum { GK_NOFLUX, GK_PSI, GK_U, GK_VX, GK_VY };

/* Ghost value across one non-periodic side of type t on axis a (0: x, 1: y)
 * from the value v at the mirror site (readings R31, R32): zero normal
 * gradient for phi, and for psi and U except at a far-field side or an inlet,
 * where the ghost is the linear extrapolation 2 X_far - v through the boundary
 * value (phi_far = 1 at an inlet); the velocity flips its normal component at
 * a symmetric side and both components at a wall or far-field side (no slip),
 * and is extrapolated through the inlet velocity; an outlet copies every
 * value (zero gradient). */
static real_t ghost_map(const ostate *st, int t, int axis, int kind, real_t v) {
  if (t == BC_OUTLET) return v;
  if (kind == GK_VX || kind == GK_VY) {
    const int normal = (kind == GK_VX) == (axis == 0);
    if (t == BC_SYMMETRIC) return normal ? -v : v;
    if (t == BC_INLET) return 2.0 * st->par[kind == GK_VX ? P_VIN_X : P_VIN_Y] - v;
    /* the extrapolation inlet's boundary node is the ghost itself */
    if (t == BC_INLET_NEE) return st->par[kind == GK_VX ? P_VIN_X : P_VIN_Y];
    return -v;
  }
  if (t == BC_FARFIELD || t == BC_INLET || t == BC_INLET_NEE) {
    if (kind == GK_PSI) return 2.0 * PSI_FAR - v;
    if (kind == GK_U) return -v;                 /* U = 0 at psi = -1, C = 1 */
    if (kind == GK_NOFLUX && t != BC_FARFIELD) return 2.0 * 1.0 - v;   /* liquid inflow */
  }
  return v;
}

/* X at (x, y), one site beyond the lattice at most: periodic sides wrap, the
 * others read the mirror site and map the value (y side first, then x). */
static real_t field_at(const ostate *st, const real_t *X, int x, int y, int kind) {
  const int nx = st->nx, ny = st->ny;
  int tx = -1, ty = -1;
  if (x < 0 || x >= nx) {
    const int t = st->bc[x < 0 ? 0 : 1];
    if (t == BC_PERIODIC) x = wrap(x, nx);
    else { tx = t; x = x < 0 ? -1 - x : 2 * nx - 1 - x; }
  }
  if (y < 0 || y >= ny) {
    const int t = st->bc[y < 0 ? 2 : 3];
    if (t == BC_PERIODIC) y = wrap(y, ny);
    else { ty = t; y = y < 0 ? -1 - y : 2 * ny - 1 - y; }
  }
  real_t v = X[y * nx + x];
  if (ty >= 0) v = ghost_map(st, ty, 1, kind, v);
  if (tx >= 0) v = ghost_map(st, tx, 0, kind, v);
  return v;
}

/* Pass 1: streaming (Eq. of the unified LBE, pull form) and zeroth moments.
 * NS, CAC and solute: f_i(x, t+1) = f*_i(x - c_i, t).
 * Dendrite, with the time stretch a_n = a_s^2 of Appendix B realised as
 * linear interpolation in time (reading R3):
 *   g_i(x, t+1) = g_i(x, t) + [g*_i(x - c_i, t) - g_i(x, t)] / a_s^2(x - c_i, t). */
static void pass_stream(ostate *st) {
  const int nx = st->nx, ny = st->ny;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      int idx = y * nx + x;
      real_t phi = 0, psi = 0, C = 0, psio = 0;
      int src, q;
      for (int i = 0; i < 9; ++i) {
        int mode = pull_src(st, x, y, i, &src, &q);
        /* NS and CAC: bounce-back at walls and far-field sides; at an inlet the
         * moving-wall bounce-back f*_opp + 2 rho_l w_i c_i.u_in / cs2 and the
         * anti-bounce-back to phi = 1 (reading R32) */
        if (mode == 5) {
          /* non-equilibrium extrapolation (Section 3, reading R37): the ghost
           * node's post-collision population is the equilibrium at u_in and
           * the liquid density plus the fluid neighbour's non-equilibrium
           * part, f_q^eq(p_b, rho_l, u_in) + f*_q(x_f) - f_q^eq(p_f, rho_f, v_f),
           * with the pressure extrapolated (p_b = p_f), so that only the
           * momentum parts of the equilibria remain (last step's rho and v
           * of the fluid site) */
          const real_t vbx = st->par[P_VIN_X], vby = st->par[P_VIN_Y];
          const real_t ux = st->vx_o[src], uy = st->vy_o[src];
          const real_t rho_f = st->par[P_RHO_G] + st->phi_o[src] * (st->par[P_RHO_L] - st->par[P_RHO_G]);
          const real_t cb = CX[q] * vbx + CY[q] * vby, cf = CX[q] * ux + CY[q] * uy;
          const real_t sb = W9[q] * (cb / CS2 + cb * cb / (2.0 * CS2 * CS2) - (vbx * vbx + vby * vby) / (2.0 * CS2));
          const real_t sf = W9[q] * (cf / CS2 + cf * cf / (2.0 * CS2 * CS2) - (ux * ux + uy * uy) / (2.0 * CS2));
          st->fS[i][idx] = st->f[q][src] + st->par[P_RHO_L] * sb - rho_f * sf;
          mode = scalar_src(st, x, y, i, &src, &q);
          st->hS[i][idx] = -st->h[q][src] + 2.0 * W9[i] * 1.0;
        } else if (mode == 3) {
          const real_t cu = CX[i] * st->par[P_VIN_X] + CY[i] * st->par[P_VIN_Y];
          st->fS[i][idx] = st->f[q][src] + 2.0 * st->par[P_RHO_L] * W9[i] * cu / CS2;
          st->hS[i][idx] = -st->h[q][src] + 2.0 * W9[i] * 1.0;
        } else if (mode == 4) {
          /* pressure outlet p = 0: anti-bounce-back of the site's own opposite
           * population plus twice the even part of the equilibrium at p = 0,
           * with the site's velocity and density of the last step */
          const real_t ux = st->vx_o[idx], uy = st->vy_o[idx];
          const real_t rho_o = st->par[P_RHO_G] + st->phi_o[idx] * (st->par[P_RHO_L] - st->par[P_RHO_G]);
          const real_t cu = CX[i] * ux + CY[i] * uy;
          st->fS[i][idx] = -st->f[OPP[i]][idx] +
                           2.0 * rho_o * W9[i] * (cu * cu / (2.0 * CS2 * CS2) - (ux * ux + uy * uy) / (2.0 * CS2));
          st->hS[i][idx] = st->h[q][src];
        } else {
          st->fS[i][idx] = st->f[q][src];
          st->hS[i][idx] = st->h[q][src];
        }
        phi += st->hS[i][idx];
      }
      for (int i = 0; i < 5; ++i) {
        const int mode = scalar_src(st, x, y, i, &src, &q);
        /* anti-bounce-back to the far-field values: -f*_opp + 2 w_i X_far */
        st->sS[i][idx] = (mode == 2 || mode == 3) ? -st->s[q][src] + 2.0 * W5[i] * C_FAR : st->s[q][src];
        C += st->sS[i][idx];
        real_t gold = st->gpre[i][idx];
        const real_t gsrc = (mode == 2 || mode == 3) ? -st->gpost[q][src] + 2.0 * W5[i] * PSI_FAR
                                      : st->gpost[q][src];
        st->gS[i][idx] = gold + (gsrc - gold) * st->rr[src];
        psi += st->gS[i][idx];
        psio += gold;
      }
      st->phiS[idx] = phi;
      st->psiS[idx] = psi;
      st->CS[idx] = C;
      st->psiOld[idx] = psio;
      /* temperature populations (thermal mode): plain pull, and the
       * supersaturation field whose gradient enters grad F(U) */
      for (int i = 0; i < 5; ++i) {
        const int mode = scalar_src(st, x, y, i, &src, &q);
        st->eS[i][idx] = (mode == 2 || mode == 3) ? -st->e[q][src] + 2.0 * W5[i] * st->par[P_THETA0]
                                   : st->e[q][src];
      }
      st->US[idx] = supersat(st, C, psi);
    }
}

/* Isotropic 9-point gradient and Laplacian (reading R5):
 *   grad X = (1/cs2) sum_i w_i c_i X(x + c_i)
 *   lap  X = (2/cs2) sum_i w_i [X(x + c_i) - X(x)]                       */
static void grad9(const ostate *st, const real_t *X, int kind, int x, int y, real_t *gx,
                  real_t *gy) {
  real_t ax = 0, ay = 0;
  for (int i = 1; i < 9; ++i) {
    real_t v = field_at(st, X, x + CX[i], y + CY[i], kind);
    ax += W9[i] * CX[i] * v;
    ay += W9[i] * CY[i] * v;
  }
  *gx = ax / CS2;
  *gy = ay / CS2;
}

static real_t lap9(const ostate *st, const real_t *X, int kind, int x, int y) {
  real_t c = X[y * st->nx + x], a = 0;
  for (int i = 1; i < 9; ++i)
    a += W9[i] * (field_at(st, X, x + CX[i], y + CY[i], kind) - c);
  return 2.0 * a / CS2;
}

/* Pass 2: gradients, interface geometry, forces and sources, collisions. */
static void pass_collide(ostate *st) {
  const int nx = st->nx, ny = st->ny;
  const real_t *par = st->par;
  const derived_t d = derive(st);
  const real_t rl = par[P_RHO_L], rg = par[P_RHO_G];
  const real_t eps = par[P_EPS_S], k = par[P_K];
  const real_t ge2 = par[P_GRAD_EPS] * par[P_GRAD_EPS];
  const int thermal = thermal_on(st);
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const int idx = y * nx + x;
      const real_t phi = st->phiS[idx], psi = st->psiS[idx], C = st->CS[idx];
      const real_t psio = st->psiOld[idx];
      const real_t phio = st->phi_o[idx], Co = st->C_o[idx];
      const real_t vxo = st->vx_o[idx], vyo = st->vy_o[idx], Qo = st->Q_o[idx];

      /* --- stencils --- */
      real_t gpx, gpy, gsx, gsy, dvxx, dvxy, dvyx, dvyy;
      grad9(st, st->phiS, GK_NOFLUX, x, y, &gpx, &gpy);
      real_t lphi = lap9(st, st->phiS, GK_NOFLUX, x, y);
      grad9(st, st->psiS, GK_PSI, x, y, &gsx, &gsy);
      grad9(st, st->vx_o, GK_VX, x, y, &dvxx, &dvxy);  /* d_x vx, d_y vx */
      grad9(st, st->vy_o, GK_VY, x, y, &dvyx, &dvyy);  /* d_x vy, d_y vy */

      /* --- gas-liquid interface --- */
      const real_t rho = rg + phi * (rl - rg);
      const real_t grx = (rl - rg) * gpx, gry = (rl - rg) * gpy;
      const real_t gmag = RSQRT_(gpx * gpx + gpy * gpy + ge2);  /* reading R6 */
      const real_t nfx = gpx / gmag, nfy = gpy / gmag;
      /* chemical potential incl. d_phi f3 (reading R15) */
      const real_t mu = 2.0 * par[P_BETA_PHI] * phi * (1.0 - phi) * (1.0 - 2.0 * phi)
                      - 2.0 * par[P_BETA_INTER] * (1.0 - phi) * (1.0 + psi) * (1.0 + psi)
                      - par[P_W_PHI] * par[P_W_PHI] * lphi;
      const real_t Fsx = d.fs_coef * mu * gpx, Fsy = d.fs_coef * mu * gpy;
      /* body force, periodic reading R13 */
      const real_t Fbx = 0.0, Fby = -(rho - st->rho_bar) * par[P_G];
      /* CAC diffusive flux D(phi) (Section 2.2) */
      const real_t aphi = d.kappa * phi * (1.0 - phi);
      const real_t Dx = par[P_M_PHI] * (gpx - aphi * nfx);
      const real_t Dy = par[P_M_PHI] * (gpy - aphi * nfy);
      /* mass-flux correction (rho_l - rho_g) div(D v), reading R14 */
      const real_t divD = (phi - phio) + vxo * gpx + vyo * gpy;
      const real_t Fmx = (rl - rg) * (divD * vxo + Dx * dvxx + Dy * dvxy);
      const real_t Fmy = (rl - rg) * (divD * vyo + Dx * dvyx + Dy * dvyy);

      /* --- Navier-Stokes moments, drag (reading R2), pressure --- */
      real_t f[9], jx = 0, jy = 0, sum_nz = 0;
      for (int i = 0; i < 9; ++i) {
        f[i] = st->fS[i][idx];
        jx += CX[i] * f[i];
        jy += CY[i] * f[i];
        if (i) sum_nz += f[i];
      }
      const real_t Fpx = Fsx + Fbx + Fmx, Fpy = Fsy + Fby + Fmy;
      const real_t vsx = (jx + 0.5 * Fpx) / rho, vsy = (jy + 0.5 * Fpy) / rho;
      const real_t chi = 0.5 * (1.0 + psi);
      const real_t vx = (1.0 - chi) * vsx, vy = (1.0 - chi) * vsy;
      const real_t Fx = Fpx - 2.0 * chi * rho * vsx, Fy = Fpy - 2.0 * chi * rho * vsy;
      const real_t v2 = vx * vx + vy * vy;
      const real_t p = CS2 / (1.0 - W9[0]) *
                       (sum_nz + 0.5 * (vx * grx + vy * gry) - W9[0] * rho * v2 / (2.0 * CS2));

      /* --- dendrite geometry: rotated normal, a_s, N (Sections 2.1, 3.3) --- */
      real_t as, Nx, Ny, smag;
      aniso(gsx, gsy, st->cth[idx], st->sth[idx], eps, par[P_GRAD_EPS], &as, &Nx, &Ny,
            &smag);
      const real_t as2 = as * as;

      /* --- solute --- */
      const real_t U = supersat(st, C, psi);
      /* --- temperature (thermal mode, Appendix B): rho H = sum_i g_i and
       * theta = H / c_p + (c_p^s / c_p) h(psi), h = (1+psi)/2 --- */
      real_t rhoH = 0.0, theta = d.theta;
      if (thermal) {
        for (int i = 0; i < 5; ++i) rhoH += st->eS[i][idx];
        theta = rhoH / (rho * par[P_CP]) + par[P_LATENT] * 0.5 * (1.0 + psi);
      }
      const real_t Q = thermal ? q_psi_at(st, &d, phi, psi, U, theta) : q_psi(st, &d, phi, psi, U);
      const real_t Wpsi = par[P_W0] * as;                /* reading R11 */
      const real_t dpsi = psi - psio;                    /* reading R4 */
      /* antitrapping direction grad psi / |grad psi| with its own, larger
       * regularisation scale (reading R6b): at the centre of a seed smaller than
       * the interface d_t psi is finite while the normal is 0/0 */
      const real_t at = -(1.0 / (2.0 * RSQRT_(2.0))) * Wpsi * (1.0 + (1.0 - k) * U) * dpsi / RSQRT_(gsx * gsx + gsy * gsy + par[P_GRAD_EPS_AT] * par[P_GRAD_EPS_AT]);
      const real_t Jatx = at * gsx, Jaty = at * gsy;
      const real_t qf = 0.5 * (1.0 - psi);
      const real_t jv = par[P_D] * qf * C * d.kappa * (1.0 - phi);
      const real_t Jx = jv * nfx, Jy = jv * nfy;

      /* --- NS collision: D2Q9 MRT with forcing (reading R1, R7) --- */
      {
        real_t feq[9], G[9], out[9];
        feq_ns(p, rho, vx, vy, feq);
        for (int i = 0; i < 9; ++i) {
          real_t cF = CX[i] * Fx + CY[i] * Fy;
          real_t cv = CX[i] * vx + CY[i] * vy;
          real_t cg = CX[i] * grx + CY[i] * gry;
          G[i] = W9[i] * (cF / CS2 + cv * cg / CS2);
        }
        const real_t S[9] = {1.0, par[P_S_E], par[P_S_EPS], 1.0, d.s_q, 1.0, d.s_q,
                             d.s_nu, d.s_nu};
        collide9(f, feq, S, G, out);
        for (int i = 0; i < 9; ++i) st->nf[i][idx] = out[i];
      }
      /* --- CAC collision: D2Q9 MRT, Eq. (eq-ACE) --- */
      {
        real_t hh[9], heq[9], G[9], out[9];
        for (int i = 0; i < 9; ++i) hh[i] = st->hS[i][idx];
        heq_cac(phi, vx, vy, heq);
        const real_t G1x = (phi * vx - phio * vxo) + CS2 * aphi * nfx;
        const real_t G1y = (phi * vy - phio * vyo) + CS2 * aphi * nfy;
        for (int i = 0; i < 9; ++i) G[i] = W9[i] * (CX[i] * G1x + CY[i] * G1y) / CS2;
        const real_t S[9] = {1, 1, 1, d.s_phi, 1, d.s_phi, 1, 1, 1};
        collide9(hh, heq, S, G, out);
        for (int i = 0; i < 9; ++i) st->nh[i][idx] = out[i];
      }
      /* --- dendrite collision: D2Q5 MRT of Appendix B.  Isothermal: F == 1
       * (reading R8).  Thermal: the source of the rewritten equation,
       *   tau0 F_psi = Q_psi / F + W0^2 / F^2 grad F . (a_s^2 grad psi + N),
       * with grad F = M c_inf (1-k) grad U, and the rate from
       *   W0^2 a_s^2 / (tau0 F) = (1/s1 - 1/2) cs2. --- */
      real_t Qeff = Q;
      {
        real_t gg[5], geq[5], G[5], Fd[5], out[5];
        real_t Fu = 1.0;
        if (thermal) {
          Fu = f_of_u(st, &d, U);
          real_t gux, guy;
          grad9(st, st->US, GK_U, x, y, &gux, &guy);
          const real_t Xx = as2 * gsx + Nx, Xy = as2 * gsy + Ny;
          const real_t dFx = d.Mcinf * (1.0 - k) * gux, dFy = d.Mcinf * (1.0 - k) * guy;
          Qeff = Q / Fu + par[P_W0] * par[P_W0] / (Fu * Fu) * (dFx * Xx + dFy * Xy);
        }
        for (int i = 0; i < 5; ++i) {
          gg[i] = st->gS[i][idx];
          geq[i] = W5[i] * psi;
          G[i] = -W5[i] * (CX[i] * Nx + CY[i] * Ny) / as2;
          /* dt F + dt^2/2 dF/dt with a backward difference (reading R4) */
          Fd[i] = W5[i] * Qeff / par[P_TAU0] + 0.5 * W5[i] * (Qeff - Qo) / par[P_TAU0];
        }
        /* W0^2 a_s^2 / (tau0 F) = (1/s1 - 1/2) cs2 */
        const real_t s1 = thermal
            ? 1.0 / (par[P_W0] * par[P_W0] * as2 / (par[P_TAU0] * Fu * CS2) + 0.5)
            : 1.0 / (par[P_W0] * par[P_W0] * as2 / (par[P_TAU0] * CS2) + 0.5);
        const real_t S[5] = {1, s1, s1, 1, 1};
        collide5(gg, geq, S, G, Fd, out);
        for (int i = 0; i < 5; ++i) {
          st->ngpost[i][idx] = out[i];
          st->ngpre[i][idx] = gg[i];
        }
        st->nrr[idx] = 1.0 / as2;
      }
      /* --- solute collision: D2Q5 MRT (reading R1) ---
       * (1-k) D q grad U = D_C grad C + E grad psi with
       * A = 1 + k - (1-k) psi, D_C = 2 D q / A, E = 2 (1-k) D q C / A^2;
       * D_C sets the local rate, E grad psi joins the fluxes in Jeq. */
      {
        real_t ss[5], seq[5], G[5], Fd[5] = {0, 0, 0, 0, 0}, out[5];
        const real_t A = 1.0 + k - (1.0 - k) * psi;
        const real_t DC = 2.0 * par[P_D] * qf / A;
        const real_t E = 2.0 * (1.0 - k) * par[P_D] * qf * C / (A * A);
        const real_t jex = C * vx - E * gsx + (1.0 - k) * (Jatx + Jx);
        const real_t jey = C * vy - E * gsy + (1.0 - k) * (Jaty + Jy);
        seq_sol(C, jex, jey, seq);
        const real_t Gx = C * vx - Co * vxo, Gy = C * vy - Co * vyo;
        for (int i = 0; i < 5; ++i) {
          ss[i] = st->sS[i][idx];
          G[i] = W5[i] * (CX[i] * Gx + CY[i] * Gy) / CS2;
        }
        /* D_C = (1/s - 1/2) cs2 */
        const real_t sc = 1.0 / (DC / CS2 + 0.5);
        const real_t S[5] = {1, sc, sc, 1, 1};
        collide5(ss, seq, S, G, Fd, out);
        for (int i = 0; i < 5; ++i) st->ns[i][idx] = out[i];
      }
      /* --- temperature collision (thermal mode): D2Q5 MRT of Appendix B,
       * equilibrium teq_th with rho H v, G_i = w_i c_i . d_t(rho H v) / cs2 with
       * a backward difference (reading R4), k_T = (1/s - 1/2) cs2 --- */
      if (thermal) {
        real_t ee[5], teq[5], G[5], Fd[5] = {0, 0, 0, 0, 0}, out[5];
        const real_t rho_o = rg + phio * (rl - rg);
        const real_t jx = rhoH * vx, jy = rhoH * vy;
        teq_th(rhoH, theta, jx, jy, teq);
        const real_t Gx = jx - rho_o * st->H_o[idx] * vxo;
        const real_t Gy = jy - rho_o * st->H_o[idx] * vyo;
        for (int i = 0; i < 5; ++i) {
          ee[i] = st->eS[i][idx];
          G[i] = W5[i] * (CX[i] * Gx + CY[i] * Gy) / CS2;
        }
        const real_t S[5] = {1, d.s_th, d.s_th, 1, 1};
        collide5(ee, teq, S, G, Fd, out);
        for (int i = 0; i < 5; ++i) st->ne[i][idx] = out[i];
        st->nH_o[idx] = rhoH / rho;
      }
      st->fld[F_THETA][idx] = theta;
      st->nphi_o[idx] = phi;
      st->nC_o[idx] = C;
      st->nvx_o[idx] = vx;
      st->nvy_o[idx] = vy;
      st->nQ_o[idx] = Qeff;
      st->fld[F_PHI][idx] = phi; st->fld[F_PSI][idx] = psi; st->fld[F_C][idx] = C;
      st->fld[F_U][idx] = U; st->fld[F_P][idx] = p;
      st->fld[F_VX][idx] = vx; st->fld[F_VY][idx] = vy; st->fld[F_MU][idx] = mu;
    }
}

static void swap_state(ostate *st) {
  real_t *t;
#define SW(a, b) do { t = (a); (a) = (b); (b) = t; } while (0)
  for (int i = 0; i < 9; ++i) { SW(st->f[i], st->nf[i]); SW(st->h[i], st->nh[i]); }
  for (int i = 0; i < 5; ++i) {
    SW(st->gpre[i], st->ngpre[i]); SW(st->gpost[i], st->ngpost[i]); SW(st->s[i], st->ns[i]);
  }
  SW(st->rr, st->nrr);
  SW(st->phi_o, st->nphi_o); SW(st->C_o, st->nC_o);
  SW(st->vx_o, st->nvx_o); SW(st->vy_o, st->nvy_o); SW(st->Q_o, st->nQ_o);
  if (thermal_on(st)) {
    for (int i = 0; i < 5; ++i) SW(st->e[i], st->ne[i]);
    SW(st->H_o, st->nH_o);
  }
#undef SW
}

void or_step(ostate *st, int n_steps) {
  for (int t = 0; t < n_steps; ++t) {
    pass_stream(st);
    pass_collide(st);
    swap_state(st);
    st->steps++;
  }
}

/* ------------------------------------------------------------------------ */
/* Outputs                                                                   */
/* ------------------------------------------------------------------------ */

/* Fields of the last step (real part), field-major: out[f * n + idx] for the
 * fields selected by mask bits (phi, psi, C, U, p, vx, vy, mu_phi, theta). */
void or_get_fields(const ostate *st, unsigned mask, double *out) {
  int o = 0;
  for (int fi = 0; fi < NFLD; ++fi)
    if (mask & (1u << fi)) {
      for (int idx = 0; idx < st->n; ++idx) out[(size_t)o * st->n + idx] = RE_(st->fld[fi][idx]);
      ++o;
    }
}

/* Imaginary parts (complex build; zeros otherwise). */
void or_get_fields_im(const ostate *st, unsigned mask, double *out) {
  int o = 0;
  for (int fi = 0; fi < NFLD; ++fi)
    if (mask & (1u << fi)) {
      for (int idx = 0; idx < st->n; ++idx) out[(size_t)o * st->n + idx] = IM_(st->fld[fi][idx]);
      ++o;
    }
}

/* Raw state, 39 planes in the documented order:
 * f[9], h[9], gpre[5], gpost[5], rr, s[5], phi_o, C_o, vx_o, vy_o, Q_o,
 * then in thermal mode 6 more: e[5] (temperature populations), H_o. */
int or_state_planes(const ostate *st) { return thermal_on(st) ? 45 : 39; }

void or_get_state(const ostate *st, double *out) {
  const real_t *planes[45];
  int q = 0;
  for (int i = 0; i < 9; ++i) planes[q++] = st->f[i];
  for (int i = 0; i < 9; ++i) planes[q++] = st->h[i];
  for (int i = 0; i < 5; ++i) planes[q++] = st->gpre[i];
  for (int i = 0; i < 5; ++i) planes[q++] = st->gpost[i];
  planes[q++] = st->rr;
  for (int i = 0; i < 5; ++i) planes[q++] = st->s[i];
  planes[q++] = st->phi_o; planes[q++] = st->C_o;
  planes[q++] = st->vx_o; planes[q++] = st->vy_o; planes[q++] = st->Q_o;
  if (thermal_on(st)) {
    for (int i = 0; i < 5; ++i) planes[q++] = st->e[i];
    planes[q++] = st->H_o;
  }
  for (int p = 0; p < q; ++p)
    for (int idx = 0; idx < st->n; ++idx) out[(size_t)p * st->n + idx] = RE_(planes[p][idx]);
}

/* FP64 diagnostics of the last step's fields (readings R16-R18):
 * out[0]  sum phi            out[1]  sum C          out[2]  sum h(psi)
 * out[3]  sum (1-phi)        out[4]  sum x (1-phi)  out[5]  sum y (1-phi)
 * out[6]  sum p, r < R-2W    out[7]  count          out[8]  sum p, r > R+4W
 * out[9]  count              out[10] max |v|        out[11] non-finite count
 * Coordinates are global site indices.  (xc, yc, R, W) is the Laplace probe. */
void or_diag(const ostate *st, double xc, double yc, double R, double W, double *out) {
  for (int i = 0; i < 12; ++i) out[i] = 0;
  for (int y = 0; y < st->ny; ++y)
    for (int x = 0; x < st->nx; ++x) {
      int idx = y * st->nx + x;
      double phi = RE_(st->fld[F_PHI][idx]), psi = RE_(st->fld[F_PSI][idx]);
      double C = RE_(st->fld[F_C][idx]), p = RE_(st->fld[F_P][idx]);
      double vx = RE_(st->fld[F_VX][idx]), vy = RE_(st->fld[F_VY][idx]);
      double gx = st->x0 + x, gy = st->y0 + y;
      out[0] += phi; out[1] += C; out[2] += 0.5 * (1.0 + psi);
      out[3] += 1.0 - phi; out[4] += gx * (1.0 - phi); out[5] += gy * (1.0 - phi);
      double dx = min_image(gx - xc, st->NX), dy = min_image(gy - yc, st->NY);
      double r = sqrt(dx * dx + dy * dy);
      if (r < R - 2.0 * W) { out[6] += p; out[7] += 1; }
      if (r > R + 4.0 * W) { out[8] += p; out[9] += 1; }
      double vm = sqrt(vx * vx + vy * vy);
      if (vm > out[10]) out[10] = vm;
      if (!isfinite(phi) || !isfinite(psi) || !isfinite(C) || !isfinite(p) ||
          !isfinite(vx) || !isfinite(vy))
        out[11] += 1;
    }
}

/* Final-state objective J = mean h(psi) + y_c / L_y with
 * y_c = sum y (1-phi) / sum (1-phi) (readings R16, R17).  Returns Re and Im. */
void or_objective(const ostate *st, double *re, double *im) {
  real_t sh = 0, gas = 0, gy = 0;
  for (int y = 0; y < st->ny; ++y)
    for (int x = 0; x < st->nx; ++x) {
      int idx = y * st->nx + x;
      sh += 0.5 * (1.0 + st->fld[F_PSI][idx]);
      gas += 1.0 - st->fld[F_PHI][idx];
      gy += (double)(st->y0 + y) * (1.0 - st->fld[F_PHI][idx]);
    }
  real_t J = sh / (double)st->n + (gy / gas) / (double)st->NY;
  *re = RE_(J);
  *im = IM_(J);
}

/* ------------------------------------------------------------------------ */
/* Pointwise pieces exported for the pin tests (double build).               */
/* ------------------------------------------------------------------------ */
void or_aniso(double gx, double gy, double theta, double eps, double geps, double *out) {
  real_t as, Nx, Ny, gm;
  aniso(gx, gy, cos(theta), sin(theta), eps, geps, &as, &Nx, &Ny, &gm);
  out[0] = RE_(as); out[1] = RE_(Nx); out[2] = RE_(Ny); out[3] = RE_(gm);
}

void or_feq_ns(double p, double rho, double vx, double vy, double *out) {
  real_t o[9];
  feq_ns(p, rho, vx, vy, o);
  for (int i = 0; i < 9; ++i) out[i] = RE_(o[i]);
}

void or_heq_cac(double phi, double vx, double vy, double *out) {
  real_t o[9];
  heq_cac(phi, vx, vy, o);
  for (int i = 0; i < 9; ++i) out[i] = RE_(o[i]);
}

void or_seq_sol(double C, double jx, double jy, double *out) {
  real_t o[5];
  seq_sol(C, jx, jy, o);
  for (int i = 0; i < 5; ++i) out[i] = RE_(o[i]);
}

void or_collide9(const double *f, const double *feq, const double *S, const double *G,
                 double *out) {
  real_t a[9], b[9], c[9], d[9], o[9];
  build_inverse();
  for (int i = 0; i < 9; ++i) { a[i] = f[i]; b[i] = feq[i]; c[i] = S[i]; d[i] = G[i]; }
  collide9(a, b, c, d, o);
  for (int i = 0; i < 9; ++i) out[i] = RE_(o[i]);
}

void or_collide5(const double *f, const double *feq, const double *S, const double *G,
                 const double *Fd, double *out) {
  real_t a[5], b[5], c[5], d[5], e[5], o[5];
  build_inverse();
  for (int i = 0; i < 5; ++i) { a[i] = f[i]; b[i] = feq[i]; c[i] = S[i]; d[i] = G[i]; e[i] = Fd[i]; }
  collide5(a, b, c, d, e, o);
  for (int i = 0; i < 5; ++i) out[i] = RE_(o[i]);
}

/* Gradient and Laplacian of a periodic nx x ny array at (x, y). */
void or_stencil(const double *X, int nx, int ny, int x, int y, double *out) {
  real_t *tmp = (real_t *)malloc((size_t)nx * ny * sizeof(real_t));
  if (!tmp) return;
  for (int i = 0; i < nx * ny; ++i) tmp[i] = X[i];
  ostate per;                       /* a periodic lattice of the array's size */
  memset(&per, 0, sizeof(per));
  per.nx = nx; per.ny = ny; per.n = nx * ny;
  real_t gx, gy;
  grad9(&per, tmp, GK_NOFLUX, x, y, &gx, &gy);
  out[0] = RE_(gx); out[1] = RE_(gy); out[2] = RE_(lap9(&per, tmp, GK_NOFLUX, x, y));
  free(tmp);
}

/* lambda', M c_inf, theta_sys, kappa, surface-tension coefficient, s_nu, s_q, s_phi. */
void or_derived(const ostate *st, double *out) {
  derived_t d = derive(st);
  out[0] = RE_(d.lam); out[1] = RE_(d.Mcinf); out[2] = RE_(d.theta);
  out[3] = RE_(d.kappa); out[4] = RE_(d.fs_coef); out[5] = RE_(d.s_nu);
  out[6] = RE_(d.s_q); out[7] = RE_(d.s_phi);
}

/* Supersaturation U(C, psi) and the dendrite source Q_psi(phi, psi, U). */
void or_pointwise(const ostate *st, double phi, double psi, double C, double *out) {
  derived_t d = derive(st);
  real_t U = supersat(st, C, psi);
  out[0] = RE_(U);
  out[1] = RE_(q_psi(st, &d, phi, psi, U));
}

/* Temperature equilibrium of Appendix B (for the pin tests). */
void or_teq_th(double rhoH, double theta, double jx, double jy, double *out) {
  real_t o[5];
  teq_th(rhoH, theta, jx, jy, o);
  for (int i = 0; i < 5; ++i) out[i] = RE_(o[i]);
}

/* F(U) of Section 2.1 and the thermal rate s_th (for the pin tests). */
void or_thermal_coefs(const ostate *st, double U, double *out) {
  derived_t d = derive(st);
  out[0] = RE_(f_of_u(st, &d, U));
  out[1] = RE_(d.kT);
  out[2] = RE_(d.s_th);
}

/* Totals of the thermal state: out[0] = sum over sites and directions of the
 * temperature populations (the total of rho H, conserved by the collision and
 * the streaming), out[1] = sum theta, out[2] = sum psi. */
static void neumaier_add(double *s, double *c, double v) {
  double t = *s + v;
  if (fabs(*s) >= fabs(v)) *c += (*s - t) + v;
  else *c += (v - t) + *s;
  *s = t;
}

void or_thermal_totals(const ostate *st, double *out) {
  /* compensated (Neumaier) sums, so that the totals carry no summation-order
   * error at the 1e-12 level of the conservation checks */
  double s[3] = {0, 0, 0}, c[3] = {0, 0, 0};
  for (int idx = 0; idx < st->n; ++idx) {
    for (int i = 0; i < 5; ++i) neumaier_add(&s[0], &c[0], RE_(st->e[i][idx]));
    neumaier_add(&s[1], &c[1], RE_(st->fld[F_THETA][idx]));
    neumaier_add(&s[2], &c[2], RE_(st->fld[F_PSI][idx]));
  }
  for (int k = 0; k < 3; ++k) out[k] = s[k] + c[k];
}

#ifdef PF_ORACLE_COUNT
/* Operation counts since the last reset: additions and subtractions,
 * multiplications, divisions, square roots. */
void or_count_get(unsigned long long out[4]) {
  out[0] = pf_count::g_tally.add; out[1] = pf_count::g_tally.mul;
  out[2] = pf_count::g_tally.div; out[3] = pf_count::g_tally.sqrt;
}
void or_count_reset(void) { pf_count::g_tally = pf_count::Tally{0, 0, 0, 0}; }
}  /* extern "C" */
#endif
