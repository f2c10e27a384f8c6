/*
 * pf_oracle3d.c -- plain FP64 CPU oracle of the three-dimensional dendrite
 * step of the phase-field model of arXiv 2407.01651: the anisotropic
 * Allen-Cahn equation for psi (Eq. eq-AnACE with the a_s^2 time stretch of
 * Appendix B) and the solute equation with antitrapping (Section 2.1), on
 * D3Q7 lattices, in a melt without gas or flow (phi = 1, v = 0).  The
 * anisotropy sums over the three axes (Section 2.1: alpha = 1, ..., d).
 *
 * TEST INFRASTRUCTURE, like pf_oracle.c: only the tests, the smoke check and
 * the CPU baseline of the benchmark may build, load or call it; it shares no
 * code with the CUDA path.  Reading R33: D3Q7 weights w0 = 1/4, wi = 1/8,
 * c_s^2 = 1/4; the isotropic gradient with D3Q19 weights; one grain
 * orientation, aligned with the lattice axes.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double real;

/* D3Q7: rest, +x, -x, +y, -y, +z, -z */
static const int C7[7][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0},
                             {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
static const double W7[7] = {0.25, 0.125, 0.125, 0.125, 0.125, 0.125, 0.125};
static const double CS2_7 = 0.25;
/* D3Q7 moments: zeroth, three fluxes, energy and two anisotropic second
 * moments (3 cx^2 - |c|^2, cy^2 - cz^2); the rows are orthogonal. */
static double M7[7][7], M7I[7][7];
static int m7_built = 0;

static void build_m7(void) {
  if (m7_built) return;
  for (int j = 0; j < 7; ++j) {
    const double cx = C7[j][0], cy = C7[j][1], cz = C7[j][2];
    const double c2 = cx * cx + cy * cy + cz * cz;
    M7[0][j] = 1;
    M7[1][j] = cx;
    M7[2][j] = cy;
    M7[3][j] = cz;
    M7[4][j] = 7 * c2 - 6;
    M7[5][j] = 3 * cx * cx - c2;
    M7[6][j] = cy * cy - cz * cz;
  }
  for (int k = 0; k < 7; ++k) {
    double n2 = 0;
    for (int j = 0; j < 7; ++j) n2 += M7[k][j] * M7[k][j];
    for (int j = 0; j < 7; ++j) M7I[j][k] = M7[k][j] / n2;
  }
  m7_built = 1;
}

/* the 18 neighbours of the D3Q19 stencil with their weights (1/18 faces,
 * 1/36 edges), for the isotropic gradient (reading R33) */
static int N18[18][3];
static double WN18[18];
static int n18_built = 0;
static void build_n18(void) {
  if (n18_built) return;
  int k = 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int a = abs(dx) + abs(dy) + abs(dz);
        if (a == 0 || a == 3) continue;
        N18[k][0] = dx; N18[k][1] = dy; N18[k][2] = dz;
        WN18[k] = a == 1 ? 1.0 / 18.0 : 1.0 / 36.0;
        ++k;
      }
  n18_built = 1;
}

/* Parameters (same symbols as the 2-D oracle). */
enum { Q_BETA_PSI, Q_W0, Q_TAU0, Q_EPS_S, Q_K, Q_D, Q_OMEGA, Q_GRAD_EPS, Q_GRAD_EPS_AT,
       /* temperature coupling (as in 2-D, readings R28-R30): thermal 0/1, Le,
        * latent = c_p^s/c_p, theta0, c_p; rho = rho_l (no gas) */
       Q_THERMAL, Q_LE, Q_LATENT, Q_THETA0, Q_CP, Q_RHO_L, NPAR3 };

typedef struct {
  int nx, ny, nz, n;
  int NX, NY, NZ, x0, y0, z0;  /* placement of this lattice in a periodic NX x NY x NZ one */
  double par[NPAR3];
  long steps;
  real *gpre[7], *gpost[7], *rr, *s[7], *Q_o;      /* state */
  real *ngpre[7], *ngpost[7], *nrr, *ns[7], *nQ_o; /* next state */
  real *psiS, *CS, *psiOld, *gS[7], *sS[7];        /* streaming scratch */
  real *e[7], *ne[7], *eS[7], *US;                  /* temperature populations (thermal) */
  real *fld[4];                                     /* psi, C, U, theta of the last step */
  real *block;
} o3state;

static inline int wrap3(int a, int n) { a %= n; return a < 0 ? a + n : a; }
static inline int idx3(const o3state *st, int x, int y, int z) {
  return (wrap3(z, st->nz) * st->ny + wrap3(y, st->ny)) * st->nx + wrap3(x, st->nx);
}

o3state *or3_new(int nx, int ny, int nz) {
  build_m7();
  build_n18();
  if (nx < 1 || ny < 1 || nz < 1) return NULL;
  o3state *st = (o3state *)calloc(1, sizeof(o3state));
  if (!st) return NULL;
  st->nx = nx; st->ny = ny; st->nz = nz; st->n = nx * ny * nz;
  st->NX = nx; st->NY = ny; st->NZ = nz;
  const size_t n = (size_t)st->n, planes = 2 * (7 + 7 + 1 + 7 + 1) + 3 + 14 + 4 + 22;
  st->block = (real *)calloc(planes * n, sizeof(real));
  if (!st->block) { free(st); return NULL; }
  real *q = st->block;
#define TAKE(p) do { (p) = q; q += n; } while (0)
  for (int i = 0; i < 7; ++i) { TAKE(st->gpre[i]); TAKE(st->gpost[i]); TAKE(st->s[i]); }
  TAKE(st->rr); TAKE(st->Q_o);
  for (int i = 0; i < 7; ++i) { TAKE(st->ngpre[i]); TAKE(st->ngpost[i]); TAKE(st->ns[i]); }
  TAKE(st->nrr); TAKE(st->nQ_o);
  TAKE(st->psiS); TAKE(st->CS); TAKE(st->psiOld);
  for (int i = 0; i < 7; ++i) { TAKE(st->gS[i]); TAKE(st->sS[i]); }
  for (int i = 0; i < 7; ++i) { TAKE(st->e[i]); TAKE(st->ne[i]); TAKE(st->eS[i]); }
  TAKE(st->US);
  for (int f = 0; f < 4; ++f) TAKE(st->fld[f]);
#undef TAKE
  return st;
}

void or3_free(o3state *st) {
  if (!st) return;
  free(st->block);
  free(st);
}

/* A window of a larger periodic lattice: the initial seeds are placed with
 * global coordinates and minimum images in NX x NY x NZ; the window itself
 * stays periodic, so only sites far enough from its faces follow the large
 * lattice (two sites per step). */
void or3_set_window(o3state *st, int NX, int NY, int NZ, int x0, int y0, int z0) {
  st->NX = NX; st->NY = NY; st->NZ = NZ; st->x0 = x0; st->y0 = y0; st->z0 = z0;
}

void or3_set_params(o3state *st, const double *p) {
  for (int i = 0; i < NPAR3; ++i) st->par[i] = p[i];
}

/* lambda' (Appendix A), M c_inf and theta_sys (Eq. eq-Tsys), as in 2-D */
static void derived3(const o3state *st, double *lam, double *Mc, double *th) {
  const double *p = st->par;
  *lam = p[Q_D] * p[Q_TAU0] / ((47.0 / 75.0) * p[Q_W0] * p[Q_W0]);
  *Mc = 1.0 - (1.0 - p[Q_K]) * p[Q_OMEGA];
  *th = -*Mc * p[Q_OMEGA] / (1.0 - (1.0 - p[Q_K]) * p[Q_OMEGA]);
}

static double supersat3(const o3state *st, double C, double psi) {
  const double k = st->par[Q_K];
  return (2.0 * C / (1.0 + k - (1.0 - k) * psi) - 1.0) / (1.0 - k);
}

/* Q_psi with phi = 1 (no interaction with gas), at temperature theta */
static double qpsi3_at(const o3state *st, double psi, double U, double theta) {
  double lam, Mc, th;
  derived3(st, &lam, &Mc, &th);
  const double om = 1.0 - psi * psi;
  return 4.0 * st->par[Q_BETA_PSI] * psi * om - lam * om * om * (theta + Mc * U);
}

/* isothermal: theta = theta_sys (Eq. eq-Tsys) */
static double qpsi3(const o3state *st, double psi, double U) {
  double lam, Mc, th;
  derived3(st, &lam, &Mc, &th);
  return qpsi3_at(st, psi, U, th);
}

static int thermal3(const o3state *st) { return st->par[Q_THERMAL] != 0.0; }

/* F(U) = 1/Le + M c_inf [1 + (1-k) U] (Section 2.1) */
static double f_of_u3(const o3state *st, double U) {
  double lam, Mc, th;
  derived3(st, &lam, &Mc, &th);
  return 1.0 / st->par[Q_LE] + Mc * (1.0 + (1.0 - st->par[Q_K]) * U);
}

/* Temperature equilibrium on D3Q7 at rest (no flow): e_0 = rho H + (w_0 - 1)
 * theta, e_i = w_i theta (Appendix B). */
static void teq3(double rhoH, double theta, real out[7]) {
  for (int i = 0; i < 7; ++i) out[i] = W7[i] * theta;
  out[0] = rhoH + (W7[0] - 1.0) * theta;
}

/* thermal initial populations and lagged source at theta */
static void init_thermal_site(o3state *st, int id, double psi, double C, double theta) {
  const double *p = st->par;
  const double H = p[Q_CP] * (theta - p[Q_LATENT] * 0.5 * (1.0 + psi));
  real t[7];
  teq3(p[Q_RHO_L] * H, theta, t);
  for (int i = 0; i < 7; ++i) st->e[i][id] = t[i];
  const double U = supersat3(st, C, psi);
  st->Q_o[id] = qpsi3_at(st, psi, U, theta) / f_of_u3(st, U);
  st->fld[3][id] = theta;
}

/* Anisotropy in 3-D (Section 2.1, sum over alpha = 1..3), the same regularised
 * form as in 2-D: n = -g/|g|_r, a_s = 1 + eps (4 sum n^4 - 3 |n|^4),
 * N_a = |g|_r^2 a_s da_s/dg_a = -16 eps a_s |g|_r n_a [n_a^2 - sum n^4 -
 * 3/4 |n|^2 (1 - |n|^2)]. */
static void aniso3(const double g[3], double eps, double geps, double *as, double N[3],
                   double *gmag) {
  const double m = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2] + geps * geps);
  double n[3], n2 = 0, s4 = 0;
  for (int a = 0; a < 3; ++a) {
    n[a] = -g[a] / m;
    n2 += n[a] * n[a];
    s4 += n[a] * n[a] * n[a] * n[a];
  }
  *as = 1.0 + eps * (4.0 * s4 - 3.0 * n2 * n2);
  const double iso = s4 + 0.75 * n2 * (1.0 - n2);
  for (int a = 0; a < 3; ++a) N[a] = -16.0 * eps * (*as) * m * n[a] * (n[a] * n[a] - iso);
  *gmag = m;
}

/* MRT collision on D3Q7: m* = m - S (m - m_eq) + (I - S/2) M G + M Fd */
static void collide7(const real f[7], const real feq[7], const real S[7], const real G[7],
                     const real Fd[7], real out[7]) {
  real m[7], ms[7];
  for (int k = 0; k < 7; ++k) {
    real a = 0, b = 0, c = 0, d = 0;
    for (int j = 0; j < 7; ++j) {
      a += M7[k][j] * f[j];
      b += M7[k][j] * feq[j];
      c += M7[k][j] * G[j];
      d += M7[k][j] * Fd[j];
    }
    m[k] = a;
    ms[k] = a - S[k] * (a - b) + (1.0 - 0.5 * S[k]) * c + d;
  }
  (void)m;
  for (int j = 0; j < 7; ++j) {
    real o = 0;
    for (int k = 0; k < 7; ++k) o += M7I[j][k] * ms[k];
    out[j] = o;
  }
}

/* Initial state: psi = max over seeds of tanh(sqrt(2 beta) (R_s - r) / W0)
 * (spheres, minimum image), C = 1 - (1-k) h(psi) (U = 0), populations at
 * equilibrium, r = 1, lagged Q_psi = its current value. */
void or3_init(o3state *st, const double *seeds, int n_seeds, double R_s) {
  const double *p = st->par;
  const double k = p[Q_K];
  for (int z = 0; z < st->nz; ++z)
    for (int y = 0; y < st->ny; ++y)
      for (int x = 0; x < st->nx; ++x) {
        const int id = (z * st->ny + y) * st->nx + x;
        double psi = -1.0;
        for (int s = 0; s < n_seeds; ++s) {
          double d[3] = {st->x0 + x - seeds[3 * s], st->y0 + y - seeds[3 * s + 1],
                         st->z0 + z - seeds[3 * s + 2]};
          const double L[3] = {st->NX, st->NY, st->NZ};
          double r2 = 0;
          for (int a = 0; a < 3; ++a) {
            d[a] = fmod(d[a], L[a]);
            if (d[a] < -0.5 * L[a]) d[a] += L[a];
            if (d[a] >= 0.5 * L[a]) d[a] -= L[a];
            r2 += d[a] * d[a];
          }
          const double v = tanh(sqrt(2.0 * p[Q_BETA_PSI]) * (R_s - sqrt(r2)) / p[Q_W0]);
          if (s == 0 || v > psi) psi = v;
        }
        const double C = 1.0 - (1.0 - k) * 0.5 * (1.0 + psi);
        for (int i = 0; i < 7; ++i) {
          st->gpre[i][id] = st->gpost[i][id] = W7[i] * psi;
          st->s[i][id] = W7[i] * C;
        }
        st->rr[id] = 1.0;
        const double U = supersat3(st, C, psi);
        st->Q_o[id] = qpsi3(st, psi, U);
        st->fld[0][id] = psi; st->fld[1][id] = C; st->fld[2][id] = U;
        double lam, Mc, th;
        derived3(st, &lam, &Mc, &th);
        st->fld[3][id] = th;
        if (thermal3(st)) init_thermal_site(st, id, psi, C, p[Q_THETA0]);
      }
  st->steps = 0;
}

/* Initial state from given psi and C fields (n each) and, in thermal mode,
 * theta (NULL: theta0). */
void or3_init_fields(o3state *st, const double *psi, const double *C, const double *theta) {
  for (int id = 0; id < st->n; ++id) {
    for (int i = 0; i < 7; ++i) {
      st->gpre[i][id] = st->gpost[i][id] = W7[i] * psi[id];
      st->s[i][id] = W7[i] * C[id];
    }
    st->rr[id] = 1.0;
    const double U = supersat3(st, C[id], psi[id]);
    st->Q_o[id] = qpsi3(st, psi[id], U);
    st->fld[0][id] = psi[id]; st->fld[1][id] = C[id]; st->fld[2][id] = U;
    double lam, Mc, th;
    derived3(st, &lam, &Mc, &th);
    st->fld[3][id] = th;
    if (thermal3(st))
      init_thermal_site(st, id, psi[id], C[id], theta ? theta[id] : st->par[Q_THETA0]);
  }
  st->steps = 0;
}

static void step3(o3state *st) {
  const int nx = st->nx, ny = st->ny, nz = st->nz;
  const double *p = st->par;
  const double k = p[Q_K], eps = p[Q_EPS_S], W0 = p[Q_W0], tau0 = p[Q_TAU0];
  /* pass 1: streaming with the time stretch of psi (reading R3), moments */
#pragma omp parallel for schedule(static)
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const int id = (z * ny + y) * nx + x;
        real psi = 0, psio = 0, C = 0;
        for (int i = 0; i < 7; ++i) {
          const int src = idx3(st, x - C7[i][0], y - C7[i][1], z - C7[i][2]);
          const real gold = st->gpre[i][id];
          st->gS[i][id] = gold + (st->gpost[i][src] - gold) * st->rr[src];
          st->sS[i][id] = st->s[i][src];
          psi += st->gS[i][id];
          psio += gold;
          C += st->sS[i][id];
        }
        st->psiS[id] = psi; st->psiOld[id] = psio; st->CS[id] = C;
        st->US[id] = supersat3(st, C, psi);
        if (thermal3(st))
          for (int i = 0; i < 7; ++i)
            st->eS[i][id] = st->e[i][idx3(st, x - C7[i][0], y - C7[i][1], z - C7[i][2])];
      }
  /* pass 2: gradient, anisotropy, sources, collisions */
#pragma omp parallel for schedule(static)
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const int id = (z * ny + y) * nx + x;
        const real psi = st->psiS[id], psio = st->psiOld[id], C = st->CS[id];
        double g[3] = {0, 0, 0};
        for (int q = 0; q < 18; ++q) {
          const real v = st->psiS[idx3(st, x + N18[q][0], y + N18[q][1], z + N18[q][2])];
          for (int a = 0; a < 3; ++a) g[a] += WN18[q] * N18[q][a] * v;
        }
        for (int a = 0; a < 3; ++a) g[a] /= (1.0 / 3.0);   /* D3Q19 c_s^2 = 1/3 */
        double as, N[3], gm;
        aniso3(g, eps, p[Q_GRAD_EPS], &as, N, &gm);
        const double as2 = as * as;
        const double U = supersat3(st, C, psi);
        /* temperature (thermal mode): rho H = sum e, theta = H / c_p + L h(psi) */
        const int th_on = thermal3(st);
        double rhoH = 0.0, theta = 0.0, Fu = 1.0, Qeff;
        if (th_on) {
          for (int i = 0; i < 7; ++i) rhoH += st->eS[i][id];
          theta = rhoH / (p[Q_RHO_L] * p[Q_CP]) + p[Q_LATENT] * 0.5 * (1.0 + psi);
        }
        const double Q = th_on ? qpsi3_at(st, psi, U, theta) : qpsi3(st, psi, U);
        Qeff = Q;
        if (th_on) {
          /* rewritten dendrite equation of Appendix B: source Q/F + W0^2/F^2
           * grad F . (a_s^2 grad psi + N), grad F = M c_inf (1-k) grad U */
          double lam, Mc, thsys;
          derived3(st, &lam, &Mc, &thsys);
          double gu[3] = {0, 0, 0};
          for (int q = 0; q < 18; ++q) {
            const real v = st->US[idx3(st, x + N18[q][0], y + N18[q][1], z + N18[q][2])];
            for (int a2 = 0; a2 < 3; ++a2) gu[a2] += WN18[q] * N18[q][a2] * v;
          }
          double dot = 0;
          for (int a2 = 0; a2 < 3; ++a2) {
            gu[a2] /= (1.0 / 3.0);
            dot += Mc * (1.0 - k) * gu[a2] * (as2 * g[a2] + N[a2]);
          }
          Fu = f_of_u3(st, U);
          Qeff = Q / Fu + W0 * W0 / (Fu * Fu) * dot;
        }
        /* antitrapping with the direction's own regularisation (reading R6b) */
        const double at = -(1.0 / (2.0 * sqrt(2.0))) * W0 * as * (1.0 + (1.0 - k) * U) *
                          (psi - psio) /
                          sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2] +
                               p[Q_GRAD_EPS_AT] * p[Q_GRAD_EPS_AT]);
        /* psi: D3Q7 MRT, f_eq = w psi, G = -w c.N / a_s^2, Fd = w (Q + dQ/2) / tau0 */
        {
          real gg[7], geq[7], G[7], Fd[7], out[7];
          for (int i = 0; i < 7; ++i) {
            gg[i] = st->gS[i][id];
            geq[i] = W7[i] * psi;
            G[i] = -W7[i] * (C7[i][0] * N[0] + C7[i][1] * N[1] + C7[i][2] * N[2]) / as2;
            Fd[i] = W7[i] * Qeff / tau0 + 0.5 * W7[i] * (Qeff - st->Q_o[id]) / tau0;
          }
          const double s1 = th_on ? 1.0 / (W0 * W0 * as2 / (tau0 * Fu * CS2_7) + 0.5)
                                  : 1.0 / (W0 * W0 * as2 / (tau0 * CS2_7) + 0.5);
          const real S[7] = {1, s1, s1, s1, 1, 1, 1};
          collide7(gg, geq, S, G, Fd, out);
          for (int i = 0; i < 7; ++i) { st->ngpost[i][id] = out[i]; st->ngpre[i][id] = gg[i]; }
          st->nrr[id] = 1.0 / as2;
        }
        /* solute: (1-k) D q grad U = D_C grad C + E grad psi (reading R1) with
         * no flow and no gas: Jeq = -E grad psi + (1-k) J_at */
        {
          real ss[7], seq[7], G[7] = {0, 0, 0, 0, 0, 0, 0}, Fd[7] = {0, 0, 0, 0, 0, 0, 0};
          real out[7];
          const double qf = 0.5 * (1.0 - psi);
          const double A = 1.0 + k - (1.0 - k) * psi;
          const double DC = 2.0 * p[Q_D] * qf / A;
          const double E = 2.0 * (1.0 - k) * p[Q_D] * qf * C / (A * A);
          double J[3];
          for (int a = 0; a < 3; ++a) J[a] = -E * g[a] + (1.0 - k) * at * g[a];
          for (int i = 0; i < 7; ++i) {
            ss[i] = st->sS[i][id];
            seq[i] = W7[i] * C + W7[i] * (C7[i][0] * J[0] + C7[i][1] * J[1] + C7[i][2] * J[2]) / CS2_7;
          }
          const double sc = 1.0 / (DC / CS2_7 + 0.5);
          const real S[7] = {1, sc, sc, sc, 1, 1, 1};
          collide7(ss, seq, S, G, Fd, out);
          for (int i = 0; i < 7; ++i) st->ns[i][id] = out[i];
        }
        /* temperature collision (D3Q7, no flow): flux rate from
         * k_T = Le D rho_l c_p = (1/s - 1/2) c_s^2, other moments at 1 */
        if (th_on) {
          real ee[7], teq[7], G0[7] = {0, 0, 0, 0, 0, 0, 0}, out[7];
          teq3(rhoH, theta, teq);
          for (int i = 0; i < 7; ++i) ee[i] = st->eS[i][id];
          const double kT = p[Q_LE] * p[Q_D] * p[Q_RHO_L] * p[Q_CP];
          const double sth = 1.0 / (kT / CS2_7 + 0.5);
          const real S[7] = {1, sth, sth, sth, 1, 1, 1};
          collide7(ee, teq, S, G0, G0, out);
          for (int i = 0; i < 7; ++i) st->ne[i][id] = out[i];
          st->fld[3][id] = theta;
        }
        st->nQ_o[id] = Qeff;
        st->fld[0][id] = psi; st->fld[1][id] = C; st->fld[2][id] = U;
      }
  real *t;
#define SW(a, b) do { t = (a); (a) = (b); (b) = t; } while (0)
  for (int i = 0; i < 7; ++i) { SW(st->gpre[i], st->ngpre[i]); SW(st->gpost[i], st->ngpost[i]); SW(st->s[i], st->ns[i]); }
  SW(st->rr, st->nrr); SW(st->Q_o, st->nQ_o);
  if (thermal3(st))
    for (int i = 0; i < 7; ++i) SW(st->e[i], st->ne[i]);
#undef SW
  st->steps++;
}

void or3_step(o3state *st, int n) {
  for (int t = 0; t < n; ++t) step3(st);
}

/* Fields psi, C, U, theta of the last step, field-major (4 x n). */
void or3_fields(const o3state *st, double *out) {
  for (int f = 0; f < 4; ++f) memcpy(out + (size_t)f * st->n, st->fld[f], st->n * sizeof(double));
}

/* Sum over sites of the temperature populations (total rho H) and of theta,
 * compensated (Neumaier). */
void or3_thermal_totals(const o3state *st, double *out) {
  double s[2] = {0, 0}, c[2] = {0, 0};
  for (int id = 0; id < st->n; ++id)
    for (int k2 = 0; k2 < 8; ++k2) {
      const double v = k2 < 7 ? st->e[k2][id] : st->fld[3][id];
      const int j = k2 < 7 ? 0 : 1;
      const double t = s[j] + v;
      c[j] += fabs(s[j]) >= fabs(v) ? (s[j] - t) + v : (v - t) + s[j];
      s[j] = t;
    }
  out[0] = s[0] + c[0];
  out[1] = s[1] + c[1];
}

/* Raw state: g_pre[7], g_post[7], r, s[7], Q_o (23 planes), then in thermal
 * mode e[7] (30 planes). */
int or3_state_planes(const o3state *st) { return thermal3(st) ? 30 : 23; }

void or3_state(const o3state *st, double *out) {
  const real *pl[30];
  int q = 0;
  for (int i = 0; i < 7; ++i) pl[q++] = st->gpre[i];
  for (int i = 0; i < 7; ++i) pl[q++] = st->gpost[i];
  pl[q++] = st->rr;
  for (int i = 0; i < 7; ++i) pl[q++] = st->s[i];
  pl[q++] = st->Q_o;
  if (thermal3(st))
    for (int i = 0; i < 7; ++i) pl[q++] = st->e[i];
  for (int p = 0; p < q; ++p) memcpy(out + (size_t)p * st->n, pl[p], st->n * sizeof(double));
}

/* Pointwise pieces for the pin tests. */
void or3_aniso(const double *g, double eps, double geps, double *out) {
  double as, N[3], gm;
  aniso3(g, eps, geps, &as, N, &gm);
  out[0] = as; out[1] = N[0]; out[2] = N[1]; out[3] = N[2]; out[4] = gm;
}

void or3_collide7(const double *f, const double *feq, const double *S, const double *G,
                  const double *Fd, double *out) {
  build_m7();
  collide7(f, feq, S, G, Fd, out);
}

/* gradient of a periodic field at (x, y, z) with the D3Q19-weighted stencil */
void or3_grad(const double *X, int nx, int ny, int nz, int x, int y, int z, double *out) {
  build_n18();
  o3state tmp;
  memset(&tmp, 0, sizeof(tmp));
  tmp.nx = nx; tmp.ny = ny; tmp.nz = nz;
  double g[3] = {0, 0, 0};
  for (int q = 0; q < 18; ++q) {
    const double v = X[idx3(&tmp, x + N18[q][0], y + N18[q][1], z + N18[q][2])];
    for (int a = 0; a < 3; ++a) g[a] += WN18[q] * N18[q][a] * v;
  }
  for (int a = 0; a < 3; ++a) out[a] = 3.0 * g[a];
}
