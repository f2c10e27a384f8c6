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
  int bc[6];                    /* side types x-, x+, y-, y+, z-, z+ (B3_*) */
  double par[NPAR3];
  long steps;
  real *gpre[7], *gpost[7], *rr, *s[7], *Q_o;      /* state */
  real *ngpre[7], *ngpost[7], *nrr, *ns[7], *nQ_o; /* next state */
  real *psiS, *CS, *psiOld, *gS[7], *sS[7];        /* streaming scratch */
  real *e[7], *ne[7], *eS[7], *US;                  /* temperature populations (thermal) */
  real *fld[4];                                     /* psi, C, U, theta of the last step */
  real *block;
  double *rot;     /* grain orientation per site (9 per site, row-major R), or NULL */
} o3state;

static inline int wrap3(int a, int n) { a %= n; return a < 0 ? a + n : a; }
/* Side types of the melt step (reading R35; the 2-D types of reading R31 that
 * act on D3Q7 lattices): periodic, symmetric, wall, far field. */
enum { B3_PERIODIC = 0, B3_SYMMETRIC = 1, B3_WALL = 2, B3_FARFIELD = 3 };

static inline int idx3(const o3state *st, int x, int y, int z) {
  return (wrap3(z, st->nz) * st->ny + wrap3(y, st->ny)) * st->nx + wrap3(x, st->nx);
}

void or3_set_bc(o3state *st, const int *bc) {
  for (int k = 0; k < 6; ++k) st->bc[k] = bc[k];
}

/* Pull source of D3Q7 direction i at (x, y, z): the site and direction read,
 * and the mode: 0 plain (periodic wrap), 1 bounce-back (symmetric or wall: on
 * D3Q7 the mirror of an axis population is its opposite at the site itself),
 * 2 anti-bounce-back to the far-field value (reading R35). */
static int pull7(const o3state *st, int x, int y, int z, int i, int *src, int *q) {
  const int X[3] = {x - C7[i][0], y - C7[i][1], z - C7[i][2]};
  const int L[3] = {st->nx, st->ny, st->nz};
  int mode = 0;
  for (int a = 0; a < 3; ++a)
    if (X[a] < 0 || X[a] >= L[a]) {
      const int t = st->bc[2 * a + (X[a] < 0 ? 0 : 1)];
      if (t == B3_FARFIELD) mode = 2;
      else if (t != B3_PERIODIC) mode = 1;
    }
  if (mode) {
    *src = idx3(st, x, y, z);
    *q = i == 0 ? 0 : (i % 2 ? i + 1 : i - 1);     /* opposite of an axis direction */
  } else {
    *src = idx3(st, X[0], X[1], X[2]);
    *q = i;
  }
  return mode;
}

/* Value of a field at (x, y, z), one site beyond the lattice at most: periodic
 * sides wrap; across a non-periodic side the mirror site's value, unchanged at
 * a symmetric side or wall (zero normal gradient) and 2 X_far - X at a far-field
 * side (far = -1 for psi, 0 for U); the axes are mapped in the order x, y, z. */
static real field3(const o3state *st, const real *X, int x, int y, int z, double far) {
  int c[3] = {x, y, z};
  const int L[3] = {st->nx, st->ny, st->nz};
  int ff[3] = {0, 0, 0};
  for (int a = 0; a < 3; ++a)
    if (c[a] < 0 || c[a] >= L[a]) {
      const int t = st->bc[2 * a + (c[a] < 0 ? 0 : 1)];
      if (t == B3_PERIODIC) continue;
      c[a] = c[a] < 0 ? -1 - c[a] : 2 * L[a] - 1 - c[a];
      ff[a] = t == B3_FARFIELD;
    }
  real v = X[idx3(st, c[0], c[1], c[2])];
  for (int a = 0; a < 3; ++a)
    if (ff[a]) v = 2.0 * far - v;
  return v;
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
  free(st->rot);
  free(st->block);
  free(st);
}

/* Rotation matrix (row-major) of the unit quaternion q = (w, x, y, z) after
 * normalisation: the crystal axes are the columns of R. */
static void quat_rot(const double *q, double R[9]) {
  const double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  const double w = q[0] / n, x = q[1] / n, y = q[2] / n, z = q[3] / n;
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - z * w);     R[2] = 2 * (x * z + y * w);
  R[3] = 2 * (x * y + z * w);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - x * w);
  R[6] = 2 * (x * z - y * w);     R[7] = 2 * (y * z + x * w);     R[8] = 1 - 2 * (x * x + y * y);
}

/* Grain orientations (the 3-D form of reading R10): each site takes the
 * orientation of the nearest seed (minimum image in the NX x NY x NZ lattice,
 * the first seed on an exact tie).  seeds: n x (x, y, z, qw, qx, qy, qz). */
/* Rotation of the nearest seed for every site of an nx x ny x nz lattice
 * placed at (x0, y0, z0) in a periodic NX x NY x NZ one; NULL on failure. */
static double *nearest_rotations(int nx, int ny, int nz, int NX, int NY, int NZ, int x0, int y0,
                                 int z0, const double *seeds, int n_seeds) {
  double *rot = (double *)malloc((size_t)nx * ny * nz * 9 * sizeof(double));
  if (!rot) return NULL;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const int id = (z * ny + y) * nx + x;
        const double X[3] = {x0 + x, y0 + y, z0 + z}, L[3] = {NX, NY, NZ};
        int best = 0;
        double bd = 0;
        for (int s2 = 0; s2 < n_seeds; ++s2) {
          double r2 = 0;
          for (int a = 0; a < 3; ++a) {
            double d = fmod(X[a] - seeds[7 * s2 + a], L[a]);
            if (d < -0.5 * L[a]) d += L[a];
            if (d >= 0.5 * L[a]) d -= L[a];
            r2 += d * d;
          }
          if (s2 == 0 || r2 < bd) { bd = r2; best = s2; }
        }
        quat_rot(seeds + 7 * best + 3, rot + 9 * (size_t)id);
      }
  return rot;
}

int or3_set_orientation(o3state *st, const double *seeds, int n_seeds) {
  free(st->rot);
  st->rot = NULL;
  if (n_seeds <= 0) return 0;
  st->rot = nearest_rotations(st->nx, st->ny, st->nz, st->NX, st->NY, st->NZ, st->x0, st->y0,
                              st->z0, seeds, n_seeds);
  return st->rot ? 0 : -1;
}

/* Orientation of a site (9 values of R; the identity without orientations). */
void or3_orientation(const o3state *st, int id, double *out) {
  for (int k = 0; k < 9; ++k) out[k] = st->rot ? st->rot[9 * (size_t)id + k] : (k % 4 == 0);
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
            if (st->bc[2 * a] == B3_PERIODIC) {    /* minimum image; plain distance otherwise */
              d[a] = fmod(d[a], L[a]);
              if (d[a] < -0.5 * L[a]) d[a] += L[a];
              if (d[a] >= 0.5 * L[a]) d[a] -= L[a];
            }
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
          int src, q;
          const int mode = pull7(st, x, y, z, i, &src, &q);
          const real gold = st->gpre[i][id];
          /* far field: anti-bounce-back -f*_opp + 2 w_i X_far (psi -1, C 1) */
          const real gsrc = mode == 2 ? -st->gpost[q][src] + 2.0 * W7[i] * (-1.0) : st->gpost[q][src];
          st->gS[i][id] = gold + (gsrc - gold) * st->rr[src];
          st->sS[i][id] = mode == 2 ? -st->s[q][src] + 2.0 * W7[i] * 1.0 : st->s[q][src];
          psi += st->gS[i][id];
          psio += gold;
          C += st->sS[i][id];
        }
        st->psiS[id] = psi; st->psiOld[id] = psio; st->CS[id] = C;
        st->US[id] = supersat3(st, C, psi);
        if (thermal3(st))
          for (int i = 0; i < 7; ++i) {
            int src, q;
            const int mode = pull7(st, x, y, z, i, &src, &q);
            st->eS[i][id] = mode == 2 ? -st->e[q][src] + 2.0 * W7[i] * p[Q_THETA0] : st->e[q][src];
          }
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
          const real v = field3(st, st->psiS, x + N18[q][0], y + N18[q][1], z + N18[q][2], -1.0);
          for (int a = 0; a < 3; ++a) g[a] += WN18[q] * N18[q][a] * v;
        }
        for (int a = 0; a < 3; ++a) g[a] /= (1.0 / 3.0);   /* D3Q19 c_s^2 = 1/3 */
        double as, N[3], gm;
        if (st->rot) {
          /* crystal frame g' = R^T g, N = R N'(g') (R10 in 3-D) */
          const double *R = st->rot + 9 * (size_t)id;
          double gr[3], Nr[3];
          for (int a = 0; a < 3; ++a) gr[a] = R[a] * g[0] + R[3 + a] * g[1] + R[6 + a] * g[2];
          aniso3(gr, eps, p[Q_GRAD_EPS], &as, Nr, &gm);
          for (int a = 0; a < 3; ++a) N[a] = R[3 * a] * Nr[0] + R[3 * a + 1] * Nr[1] + R[3 * a + 2] * Nr[2];
        } else {
          aniso3(g, eps, p[Q_GRAD_EPS], &as, N, &gm);
        }
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
            const real v = field3(st, st->US, x + N18[q][0], y + N18[q][1], z + N18[q][2], 0.0);
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

/* ======================================================================== */
/* Three-dimensional two-phase step (reading R34): the coupled step of the   */
/* 2-D oracle written for d = 3.  Incompressible Navier-Stokes and the       */
/* conservative Allen-Cahn equation on D3Q19 lattices (w0 = 1/3, faces 1/18, */
/* edges 1/36, c_s^2 = 1/3) with the MRT of d'Humieres et al. (2002) in the  */
/* role of the paper's M0 (the paper gives the D2Q9 one only); psi and C on  */
/* the D3Q7 lattices above, coupled to the flow and the gas as in 2-D.       */
/* Periodic cube, one grain orientation aligned with the lattice.            */
/* ======================================================================== */

/* D3Q19: rest, six faces, twelve edges; opposite directions in pairs
 * (2j-1, 2j). */
static const int C19[19][3] = {
    {0, 0, 0},   {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},  {0, -1, 0},  {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},  {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1},
    {1, 0, -1},  {-1, 0, 1},  {0, 1, 1},   {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static double W19[19];
static const double CS2_19 = 1.0 / 3.0;
/* Moment basis: rho, e, eps, jx, qx, jy, qy, jz, qz, 3pxx, 3pixx, pww, piww,
 * pxy, pyz, pxz, mx, my, mz, as polynomials of c; mutually orthogonal rows,
 * so M^-1 = M^T diag(1 / |row|^2). */
static double M19[19][19], M19I[19][19];
static int m19_built = 0;

static void build_m19(void) {
  if (m19_built) return;
  for (int j = 0; j < 19; ++j) {
    const double x = C19[j][0], y = C19[j][1], z = C19[j][2];
    const double c2 = x * x + y * y + z * z;
    W19[j] = c2 == 0 ? 1.0 / 3.0 : (c2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
    const double r[19] = {1.0,
                          19 * c2 - 30,
                          (21 * c2 * c2 - 53 * c2 + 24) / 2,
                          x, (5 * c2 - 9) * x,
                          y, (5 * c2 - 9) * y,
                          z, (5 * c2 - 9) * z,
                          3 * x * x - c2, (3 * c2 - 5) * (3 * x * x - c2),
                          y * y - z * z, (3 * c2 - 5) * (y * y - z * z),
                          x * y, y * z, x * z,
                          (y * y - z * z) * x, (z * z - x * x) * y, (x * x - y * y) * z};
    for (int k = 0; k < 19; ++k) M19[k][j] = r[k];
  }
  for (int k = 0; k < 19; ++k) {
    double n2 = 0;
    for (int j = 0; j < 19; ++j) n2 += M19[k][j] * M19[k][j];
    for (int j = 0; j < 19; ++j) M19I[j][k] = M19[k][j] / n2;
  }
  m19_built = 1;
}

/* m* = m - S (m - m_eq) + (I - S/2) M G, f* = M^-1 m* (Appendix B's operator). */
static void collide19(const real f[19], const real feq[19], const real S[19], const real G[19],
                      real out[19]) {
  real ms[19];
  for (int k = 0; k < 19; ++k) {
    real a = 0, b = 0, c = 0;
    for (int j = 0; j < 19; ++j) {
      a += M19[k][j] * f[j];
      b += M19[k][j] * feq[j];
      c += M19[k][j] * G[j];
    }
    ms[k] = a - S[k] * (a - b) + (1.0 - 0.5 * S[k]) * c;
  }
  for (int j = 0; j < 19; ++j) {
    real o = 0;
    for (int k = 0; k < 19; ++k) o += M19I[j][k] * ms[k];
    out[j] = o;
  }
}

/* Parameters of the two-phase step (the 2-D symbols). */
enum { F3_RHO_L, F3_RHO_G, F3_NU, F3_SIGMA, F3_W_PHI, F3_M_PHI, F3_BETA_PHI, F3_BETA_PSI,
       F3_BETA_INTER, F3_W0, F3_TAU0, F3_EPS_S, F3_K, F3_D, F3_OMEGA, F3_G, F3_GRAD_EPS,
       F3_GRAD_EPS_AT, F3_S_E, F3_S_EPS,
       /* temperature coupling (thermal mode, as in 2-D: readings R28-R30) */
       F3_THERMAL, F3_LE, F3_LATENT, F3_THETA0, F3_CP, NPAR3F };

enum { G3_PHI, G3_PSI, G3_C, G3_U, G3_P, G3_VX, G3_VY, G3_VZ, G3_MU, G3_THETA, NFLD3F };

typedef struct {
  int nx, ny, nz, n;
  int NX, NY, NZ, x0, y0, z0;
  double par[NPAR3F];
  double rho_bar;
  int rho_bar_fixed;
  long steps;
  /* state */
  real *f[19], *h[19], *gpre[7], *gpost[7], *rr, *s[7], *Q_o, *phi_o, *C_o, *v_o[3];
  /* next state */
  real *nf[19], *nh[19], *ngpre[7], *ngpost[7], *nrr, *ns[7], *nQ_o, *nphi_o, *nC_o, *nv_o[3];
  /* streaming scratch */
  real *fS[19], *hS[19], *gS[7], *sS[7], *phiS, *psiS, *CS, *psiOld;
  /* thermal mode: temperature populations, lagged H, streamed e and U */
  real *e[7], *ne[7], *eS[7], *H_o, *nH_o, *US;
  real *fld[NFLD3F];
  real *block;
  double *rot;     /* grain orientation per site (9 per site), or NULL */
  int bc[6];       /* side types x-, x+, y-, y+, z-, z+ (B3_*) */
} o3fstate;

static int thermalf(const o3fstate *st) { return st->par[F3_THERMAL] != 0.0; }

static double derivedf(const o3fstate *st, double *lam, double *Mc, double *th) {
  const double *p = st->par;
  *lam = p[F3_D] * p[F3_TAU0] / ((47.0 / 75.0) * p[F3_W0] * p[F3_W0]);
  *Mc = 1.0 - (1.0 - p[F3_K]) * p[F3_OMEGA];
  *th = -*Mc * p[F3_OMEGA] / (1.0 - (1.0 - p[F3_K]) * p[F3_OMEGA]);
  return *lam;
}

o3fstate *or3f_new(int nx, int ny, int nz) {
  build_m7();
  build_n18();
  build_m19();
  if (nx < 1 || ny < 1 || nz < 1) return NULL;
  o3fstate *st = (o3fstate *)calloc(1, sizeof(o3fstate));
  if (!st) return NULL;
  st->nx = nx; st->ny = ny; st->nz = nz; st->n = nx * ny * nz;
  st->NX = nx; st->NY = ny; st->NZ = nz;
  const size_t n = (size_t)st->n;
  const size_t planes = 2 * (19 + 19 + 7 + 7 + 1 + 7 + 1 + 1 + 1 + 3) + (19 + 19 + 7 + 7 + 4) + NFLD3F +
                        3 * 7 + 3;
  st->block = (real *)calloc(planes * n, sizeof(real));
  if (!st->block) { free(st); return NULL; }
  real *q = st->block;
#define TAKE(p) do { (p) = q; q += n; } while (0)
  for (int i = 0; i < 19; ++i) { TAKE(st->f[i]); TAKE(st->h[i]); TAKE(st->nf[i]); TAKE(st->nh[i]); }
  for (int i = 0; i < 7; ++i) {
    TAKE(st->gpre[i]); TAKE(st->gpost[i]); TAKE(st->s[i]);
    TAKE(st->ngpre[i]); TAKE(st->ngpost[i]); TAKE(st->ns[i]);
  }
  TAKE(st->rr); TAKE(st->Q_o); TAKE(st->phi_o); TAKE(st->C_o);
  TAKE(st->nrr); TAKE(st->nQ_o); TAKE(st->nphi_o); TAKE(st->nC_o);
  for (int a = 0; a < 3; ++a) { TAKE(st->v_o[a]); TAKE(st->nv_o[a]); }
  for (int i = 0; i < 19; ++i) { TAKE(st->fS[i]); TAKE(st->hS[i]); }
  for (int i = 0; i < 7; ++i) { TAKE(st->gS[i]); TAKE(st->sS[i]); }
  TAKE(st->phiS); TAKE(st->psiS); TAKE(st->CS); TAKE(st->psiOld);
  for (int i = 0; i < 7; ++i) { TAKE(st->e[i]); TAKE(st->ne[i]); TAKE(st->eS[i]); }
  TAKE(st->H_o); TAKE(st->nH_o); TAKE(st->US);
  for (int f = 0; f < NFLD3F; ++f) TAKE(st->fld[f]);
#undef TAKE
  return st;
}

void or3f_free(o3fstate *st) {
  if (!st) return;
  free(st->rot);
  free(st->block);
  free(st);
}

/* Grain orientations as for the melt step: seeds n x (x, y, z, qw, qx, qy, qz). */
int or3f_set_orientation(o3fstate *st, const double *seeds, int n_seeds) {
  free(st->rot);
  st->rot = NULL;
  if (n_seeds <= 0) return 0;
  st->rot = nearest_rotations(st->nx, st->ny, st->nz, st->NX, st->NY, st->NZ, st->x0, st->y0,
                              st->z0, seeds, n_seeds);
  return st->rot ? 0 : -1;
}

void or3f_set_params(o3fstate *st, const double *p) {
  for (int i = 0; i < NPAR3F; ++i) st->par[i] = p[i];
}

void or3f_set_window(o3fstate *st, int NX, int NY, int NZ, int x0, int y0, int z0) {
  st->NX = NX; st->NY = NY; st->NZ = NZ; st->x0 = x0; st->y0 = y0; st->z0 = z0;
}

/* Fix the buoyancy reference density (reading R13) instead of taking it from
 * the initial phi of this lattice (a window of a larger one). */
void or3f_set_rho_bar(o3fstate *st, double rho_bar) { st->rho_bar = rho_bar; st->rho_bar_fixed = 1; }
double or3f_get_rho_bar(const o3fstate *st) { return st->rho_bar; }

static inline int idx3f(const o3fstate *st, int x, int y, int z) {
  return (wrap3(z, st->nz) * st->ny + wrap3(y, st->ny)) * st->nx + wrap3(x, st->nx);
}

void or3f_set_bc(o3fstate *st, const int *bc) {
  for (int k = 0; k < 6; ++k) st->bc[k] = bc[k];
}

/* D3Q19 direction with the component along axis a reversed, and the opposite */
static int mirror19(int i, int a) {
  int c[3] = {C19[i][0], C19[i][1], C19[i][2]};
  c[a] = -c[a];
  for (int j = 0; j < 19; ++j)
    if (C19[j][0] == c[0] && C19[j][1] == c[1] && C19[j][2] == c[2]) return j;
  return i;
}
static int opp19(int i) { return i == 0 ? 0 : (i % 2 ? i + 1 : i - 1); }

/* Pull source of a population of direction c = (cx, cy, cz) at (x, y, z) with
 * the sides of the 2-D reading R31 in 3-D (R36): periodic wrap; a symmetric
 * side reflects the source site and the direction (mirror(a)); a wall or a
 * far-field side returns the site's own opposite population (mode 1 wall, 2 far
 * field); a bounce wins over a reflection where both are crossed.  Returns the
 * mode; *q is the direction read (in the lattice's own numbering via map). */
static int pull_side(const o3fstate *st, int x, int y, int z, const int c[3], int *src, int *refl) {
  int X[3] = {x - c[0], y - c[1], z - c[2]};
  const int L[3] = {st->nx, st->ny, st->nz};
  int mode = 0;
  *refl = 0;
  for (int a = 0; a < 3; ++a)
    if (X[a] < 0 || X[a] >= L[a]) {
      const int t = st->bc[2 * a + (X[a] < 0 ? 0 : 1)];
      if (t == B3_PERIODIC) continue;
      if (t == B3_SYMMETRIC) {
        X[a] = X[a] < 0 ? -1 - X[a] : 2 * L[a] - 1 - X[a];
        *refl |= 1 << a;
      } else {
        const int m = t == B3_FARFIELD ? 2 : 1;
        if (m > mode) mode = m;
      }
    }
  *src = mode ? idx3f(st, x, y, z) : idx3f(st, X[0], X[1], X[2]);
  return mode;
}

/* Field value one site beyond the lattice at most: the mirror site's value
 * across a non-periodic side, mapped per side (kind 0 phi: unchanged; 1 psi:
 * 2 psi_far - psi at a far side; 2 U: -U at a far side; 3..5 the velocity
 * component a = kind - 3: its sign flipped at a symmetric side if normal to it,
 * flipped at a wall or far-field side always); axes mapped in the order x, y, z. */
static real field3f(const o3fstate *st, const real *X, int x, int y, int z, int kind) {
  int c[3] = {x, y, z};
  const int L[3] = {st->nx, st->ny, st->nz};
  int t3[3] = {0, 0, 0};
  for (int a = 0; a < 3; ++a)
    if (c[a] < 0 || c[a] >= L[a]) {
      const int t = st->bc[2 * a + (c[a] < 0 ? 0 : 1)];
      if (t == B3_PERIODIC) continue;
      c[a] = c[a] < 0 ? -1 - c[a] : 2 * L[a] - 1 - c[a];
      t3[a] = t;
    }
  real v = X[idx3f(st, c[0], c[1], c[2])];
  for (int a = 0; a < 3; ++a) {
    const int t = t3[a];
    if (!t) continue;
    if (kind == 1 && t == B3_FARFIELD) v = -2.0 - v;
    else if (kind == 2 && t == B3_FARFIELD) v = -v;
    else if (kind >= 3) {
      if (t == B3_SYMMETRIC) { if (kind - 3 == a) v = -v; }
      else v = -v;
    }
  }
  return v;
}

static double supersatf(const o3fstate *st, double C, double psi) {
  const double k = st->par[F3_K];
  return (2.0 * C / (1.0 + k - (1.0 - k) * psi) - 1.0) / (1.0 - k);
}

/* Q_psi = -[f2' + d_psi f3 + lambda' (1-psi^2)^2 (theta_sys + M c_inf U)] with
 * f3 = beta_inter (1-phi)^2 (1+psi)^2 (Appendix B, Eq. eq-f3Inter) */
static double qpsif(const o3fstate *st, double phi, double psi, double U) {
  const double *p = st->par;
  double lam, Mc, th;
  derivedf(st, &lam, &Mc, &th);
  const double om = 1.0 - psi * psi;
  return 4.0 * p[F3_BETA_PSI] * psi * om - 2.0 * p[F3_BETA_INTER] * (1.0 - phi) * (1.0 - phi) * (1.0 + psi) -
         lam * om * om * (th + Mc * U);
}

/* Q_psi at temperature theta (thermal mode) */
static double qpsif_at(const o3fstate *st, double phi, double psi, double U, double theta) {
  const double *p = st->par;
  double lam, Mc, th;
  derivedf(st, &lam, &Mc, &th);
  const double om = 1.0 - psi * psi;
  return 4.0 * p[F3_BETA_PSI] * psi * om - 2.0 * p[F3_BETA_INTER] * (1.0 - phi) * (1.0 - phi) * (1.0 + psi) -
         lam * om * om * (theta + Mc * U);
}

/* F(U) = 1/Le + M c_inf [1 + (1-k) U] */
static double f_of_uf(const o3fstate *st, double U) {
  double lam, Mc, th;
  derivedf(st, &lam, &Mc, &th);
  return 1.0 / st->par[F3_LE] + Mc * (1.0 + (1.0 - st->par[F3_K]) * U);
}

/* Temperature equilibrium on D3Q7 with the flux rho H v (Appendix B):
 * e_0 = rho H + (w0 - 1) theta, e_i = w_i theta + w_i c_i . j / c_s^2 */
static void teqf(double rhoH, double theta, const double j[3], real out[7]) {
  for (int i = 0; i < 7; ++i)
    out[i] = W7[i] * theta + W7[i] * (C7[i][0] * j[0] + C7[i][1] * j[1] + C7[i][2] * j[2]) / CS2_7;
  out[0] = rhoH + (W7[0] - 1.0) * theta;
}

/* Pressure-based incompressible equilibrium on D3Q19: w p / c_s^2 off the
 * rest direction, -(1 - w0) p / c_s^2 on it, plus rho w [c.v/c_s^2 +
 * (c.v)^2/(2 c_s^4) - v^2/(2 c_s^2)] (reading R1 in 3-D). */
static void feq19(double p, double rho, const double v[3], real out[19]) {
  const double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  for (int i = 0; i < 19; ++i) {
    const double cu = C19[i][0] * v[0] + C19[i][1] * v[1] + C19[i][2] * v[2];
    out[i] = W19[i] * p / CS2_19 +
             rho * W19[i] * (cu / CS2_19 + cu * cu / (2 * CS2_19 * CS2_19) - v2 / (2 * CS2_19));
    if (i == 0) out[i] -= p / CS2_19;
  }
}

/* CAC equilibrium w phi (1 + c.v / c_s^2) */
static void heq19(double phi, const double v[3], real out[19]) {
  for (int i = 0; i < 19; ++i)
    out[i] = W19[i] * phi * (1.0 + (C19[i][0] * v[0] + C19[i][1] * v[1] + C19[i][2] * v[2]) / CS2_19);
}

/* Initial state from fields (n each; v and p may be NULL: rest, p = 0):
 * populations at equilibrium, lagged values equal to the current ones,
 * r = 1 (reading R20 in 3-D). */
void or3f_init_fields(o3fstate *st, const double *phi, const double *psi, const double *C,
                      const double *vx, const double *vy, const double *vz, const double *p) {
  const double *par = st->par;
  double sphi = 0.0;
  for (int id = 0; id < st->n; ++id) {
    const double ph = phi[id], ps = psi[id], c = C[id];
    const double v[3] = {vx ? vx[id] : 0.0, vy ? vy[id] : 0.0, vz ? vz[id] : 0.0};
    const double pp = p ? p[id] : 0.0;
    const double rho = par[F3_RHO_G] + ph * (par[F3_RHO_L] - par[F3_RHO_G]);
    real t[19];
    feq19(pp, rho, v, t);
    for (int i = 0; i < 19; ++i) st->f[i][id] = t[i];
    heq19(ph, v, t);
    for (int i = 0; i < 19; ++i) st->h[i][id] = t[i];
    for (int i = 0; i < 7; ++i) {
      st->gpre[i][id] = st->gpost[i][id] = W7[i] * ps;
      st->s[i][id] = W7[i] * c + W7[i] * c * (C7[i][0] * v[0] + C7[i][1] * v[1] + C7[i][2] * v[2]) / CS2_7;
    }
    st->rr[id] = 1.0;
    const double U = supersatf(st, c, ps);
    st->Q_o[id] = qpsif(st, ph, ps, U);
    st->phi_o[id] = ph; st->C_o[id] = c;
    for (int a = 0; a < 3; ++a) st->v_o[a][id] = v[a];
    st->fld[G3_PHI][id] = ph; st->fld[G3_PSI][id] = ps; st->fld[G3_C][id] = c;
    st->fld[G3_U][id] = U; st->fld[G3_P][id] = pp;
    st->fld[G3_VX][id] = v[0]; st->fld[G3_VY][id] = v[1]; st->fld[G3_VZ][id] = v[2];
    st->fld[G3_MU][id] = 0.0;
    {
      double lam, Mc, th;
      derivedf(st, &lam, &Mc, &th);
      st->fld[G3_THETA][id] = th;
    }
    if (thermalf(st)) {
      /* H = c_p [theta0 - (c_p^s/c_p) h(psi)], e at equilibrium with rho H v,
       * lagged source Q_psi(theta0) / F(U) (readings R28, R29) */
      const double th0 = par[F3_THETA0];
      const double H = par[F3_CP] * (th0 - par[F3_LATENT] * 0.5 * (1.0 + ps));
      const double j[3] = {rho * H * v[0], rho * H * v[1], rho * H * v[2]};
      real t7[7];
      teqf(rho * H, th0, j, t7);
      for (int i = 0; i < 7; ++i) st->e[i][id] = t7[i];
      st->H_o[id] = H;
      st->Q_o[id] = qpsif_at(st, ph, ps, U, th0) / f_of_uf(st, U);
      st->fld[G3_THETA][id] = th0;
    }
    sphi += ph;
  }
  if (!st->rho_bar_fixed)
    st->rho_bar = par[F3_RHO_G] + (sphi / st->n) * (par[F3_RHO_L] - par[F3_RHO_G]);
  st->steps = 0;
}

/* Thermal mode: set the initial temperature field theta (n) after
 * or3f_init_fields / or3f_init_spec (the lagged values follow). */
void or3f_set_temperature(o3fstate *st, const double *theta) {
  const double *par = st->par;
  for (int id = 0; id < st->n; ++id) {
    const double ph = st->fld[G3_PHI][id], ps = st->fld[G3_PSI][id], c = st->fld[G3_C][id];
    const double v[3] = {st->fld[G3_VX][id], st->fld[G3_VY][id], st->fld[G3_VZ][id]};
    const double rho = par[F3_RHO_G] + ph * (par[F3_RHO_L] - par[F3_RHO_G]);
    const double H = par[F3_CP] * (theta[id] - par[F3_LATENT] * 0.5 * (1.0 + ps));
    const double j[3] = {rho * H * v[0], rho * H * v[1], rho * H * v[2]};
    real t7[7];
    teqf(rho * H, theta[id], j, t7);
    for (int i = 0; i < 7; ++i) st->e[i][id] = t7[i];
    st->H_o[id] = H;
    const double U = supersatf(st, c, ps);
    st->Q_o[id] = qpsif_at(st, ph, ps, U, theta[id]) / f_of_uf(st, U);
    st->fld[G3_THETA][id] = theta[id];
  }
}

/* Signed minimum-image offset on a periodic axis of length L */
static double min_image3(double d, double L) {
  d = fmod(d, L);
  if (d < -0.5 * L) d += L;
  if (d >= 0.5 * L) d -= L;
  return d;
}

/* Initial fields from spherical seeds (x, y, z) of radius R_s and bubbles
 * (x, y, z, R_b) (readings R9, R21 in 3-D): psi = max tanh(sqrt(2 beta_psi)
 * (R_s - r)/W0), phi = min [1/2 + 1/2 tanh(sqrt(2 beta_phi) (r - R_b)/(2 W_phi))],
 * C = phi [1 - (1-k) h(psi)]. */
void or3f_fields_from_spec(const o3fstate *st, const double *seeds, int n_seeds, double R_s,
                           const double *bubbles, int n_bub, double *phi, double *psi, double *C) {
  const double *p = st->par;
  const double sb = sqrt(2.0 * p[F3_BETA_PSI]), sp = sqrt(2.0 * p[F3_BETA_PHI]);
  for (int z = 0; z < st->nz; ++z)
    for (int y = 0; y < st->ny; ++y)
      for (int x = 0; x < st->nx; ++x) {
        const int id = (z * st->ny + y) * st->nx + x;
        const double X[3] = {st->x0 + x, st->y0 + y, st->z0 + z}, L[3] = {st->NX, st->NY, st->NZ};
        double ps = -1.0, ph = 1.0;
        for (int s = 0; s < n_seeds; ++s) {
          double r2 = 0;
          for (int a = 0; a < 3; ++a) {
            const double d = st->bc[2 * a] == B3_PERIODIC ? min_image3(X[a] - seeds[3 * s + a], L[a])
                                                          : X[a] - seeds[3 * s + a];
            r2 += d * d;
          }
          const double v = tanh(sb * (R_s - sqrt(r2)) / p[F3_W0]);
          if (s == 0 || v > ps) ps = v;
        }
        for (int b = 0; b < n_bub; ++b) {
          double r2 = 0;
          for (int a = 0; a < 3; ++a) {
            const double d = st->bc[2 * a] == B3_PERIODIC ? min_image3(X[a] - bubbles[4 * b + a], L[a])
                                                          : X[a] - bubbles[4 * b + a];
            r2 += d * d;
          }
          const double v = 0.5 + 0.5 * tanh(sp * (sqrt(r2) - bubbles[4 * b + 3]) / (2.0 * p[F3_W_PHI]));
          if (b == 0 || v < ph) ph = v;
        }
        phi[id] = ph;
        psi[id] = ps;
        C[id] = ph * (1.0 - (1.0 - p[F3_K]) * 0.5 * (1.0 + ps));
      }
}

/* mean phi of the spec over the whole NX x NY x NZ lattice */
double or3f_mean_phi_global(const o3fstate *st, const double *bubbles, int n_bub) {
  const double sp = sqrt(2.0 * st->par[F3_BETA_PHI]);
  double total = 0.0;
#pragma omp parallel for reduction(+ : total) schedule(static)
  for (int z = 0; z < st->NZ; ++z)
    for (int y = 0; y < st->NY; ++y)
      for (int x = 0; x < st->NX; ++x) {
        const double X[3] = {x, y, z}, L[3] = {st->NX, st->NY, st->NZ};
        double ph = 1.0;
        for (int b = 0; b < n_bub; ++b) {
          double r2 = 0;
          for (int a = 0; a < 3; ++a) {
            const double d = min_image3(X[a] - bubbles[4 * b + a], L[a]);
            r2 += d * d;
          }
          const double v = 0.5 + 0.5 * tanh(sp * (sqrt(r2) - bubbles[4 * b + 3]) / (2.0 * st->par[F3_W_PHI]));
          if (b == 0 || v < ph) ph = v;
        }
        total += ph;
      }
  return total / ((double)st->NX * st->NY * st->NZ);
}

int or3f_init_spec(o3fstate *st, const double *seeds, int n_seeds, double R_s,
                   const double *bubbles, int n_bub) {
  const size_t n = (size_t)st->n;
  double *buf = (double *)malloc(3 * n * sizeof(double));
  if (!buf) return -1;
  or3f_fields_from_spec(st, seeds, n_seeds, R_s, bubbles, n_bub, buf, buf + n, buf + 2 * n);
  or3f_init_fields(st, buf, buf + n, buf + 2 * n, NULL, NULL, NULL, NULL);
  free(buf);
  return 0;
}

/* isotropic gradient and Laplacian with the D3Q19 weights (reading R5 in 3-D):
 * grad X = (1/c_s^2) sum w c X(x+c), lap X = (2/c_s^2) sum w [X(x+c) - X(x)] */
static void grad19(const o3fstate *st, const real *X, int kind, int x, int y, int z, double g[3]) {
  g[0] = g[1] = g[2] = 0.0;
  for (int i = 1; i < 19; ++i) {
    const double v = field3f(st, X, x + C19[i][0], y + C19[i][1], z + C19[i][2], kind);
    for (int a = 0; a < 3; ++a) g[a] += W19[i] * C19[i][a] * v;
  }
  for (int a = 0; a < 3; ++a) g[a] /= CS2_19;
}
static double lap19(const o3fstate *st, const real *X, int kind, int x, int y, int z) {
  const double c = X[idx3f(st, x, y, z)];
  double a = 0.0;
  for (int i = 1; i < 19; ++i)
    a += W19[i] * (field3f(st, X, x + C19[i][0], y + C19[i][1], z + C19[i][2], kind) - c);
  return 2.0 * a / CS2_19;
}

static void step3f(o3fstate *st) {
  const int nx = st->nx, ny = st->ny, nz = st->nz;
  const double *p = st->par;
  /* pass 1: pull streaming of f, h, s and of g with the time stretch (R3) */
#pragma omp parallel for schedule(static)
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const int id = (z * ny + y) * nx + x;
        real phi = 0, psi = 0, psio = 0, C = 0;
        for (int i = 0; i < 19; ++i) {
          /* NS and CAC: reflection at a symmetric side, the own opposite
           * population (no slip, no flux) at a wall or far-field side */
          int src, refl;
          const int mode = pull_side(st, x, y, z, C19[i], &src, &refl);
          int q = i;
          if (mode) q = opp19(i);
          else
            for (int a2 = 0; a2 < 3; ++a2)
              if (refl & (1 << a2)) q = mirror19(q, a2);
          st->fS[i][id] = st->f[q][src];
          st->hS[i][id] = st->h[q][src];
          phi += st->hS[i][id];
        }
        for (int i = 0; i < 7; ++i) {
          /* D3Q7: reflection and bounce coincide (the own opposite population);
           * a far-field side anti-bounces to psi = -1, C = 1 */
          int src, refl;
          const int mode = pull_side(st, x, y, z, C7[i], &src, &refl);
          const int q = (mode || refl) ? (i == 0 ? 0 : (i % 2 ? i + 1 : i - 1)) : i;
          if (refl) src = idx3f(st, x, y, z);
          const real gold = st->gpre[i][id];
          const real gsrc = mode == 2 ? -st->gpost[q][src] + 2.0 * W7[i] * (-1.0) : st->gpost[q][src];
          st->gS[i][id] = gold + (gsrc - gold) * st->rr[src];
          st->sS[i][id] = mode == 2 ? -st->s[q][src] + 2.0 * W7[i] * 1.0 : st->s[q][src];
          psi += st->gS[i][id];
          psio += gold;
          C += st->sS[i][id];
        }
        st->phiS[id] = phi; st->psiS[id] = psi; st->psiOld[id] = psio; st->CS[id] = C;
        if (thermalf(st)) {
          /* temperature populations (plain pull) and U, whose gradient gives grad F */
          for (int i = 0; i < 7; ++i) {
            int src, refl;
            const int mode = pull_side(st, x, y, z, C7[i], &src, &refl);
            const int q = (mode || refl) ? (i == 0 ? 0 : (i % 2 ? i + 1 : i - 1)) : i;
            if (refl) src = idx3f(st, x, y, z);
            st->eS[i][id] = mode == 2 ? -st->e[q][src] + 2.0 * W7[i] * p[F3_THETA0] : st->e[q][src];
          }
          st->US[id] = supersatf(st, C, psi);
        }
      }
  double lam, Mc, thsys;
  derivedf(st, &lam, &Mc, &thsys);
  const double rl = p[F3_RHO_L], rg = p[F3_RHO_G], k = p[F3_K], W0 = p[F3_W0], tau0 = p[F3_TAU0];
  const double kappa = sqrt(2.0 * p[F3_BETA_PHI]) / p[F3_W_PHI];
  /* F_s = 6 sigma / (W_phi sqrt(2 beta_phi)) mu grad phi (Section 2.2, phi_l - phi_g = 1) */
  const double fs_coef = 6.0 * p[F3_SIGMA] / (p[F3_W_PHI] * sqrt(2.0 * p[F3_BETA_PHI]));
  const double s_nu = 1.0 / (p[F3_NU] / CS2_19 + 0.5);
  const double s_q = 8.0 * (2.0 - s_nu) / (8.0 - s_nu);          /* reading R7 */
  const double s_phi = 1.0 / (p[F3_M_PHI] / CS2_19 + 0.5);
  /* pass 2 */
#pragma omp parallel for schedule(static)
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const int id = (z * ny + y) * nx + x;
        const double phi = st->phiS[id], psi = st->psiS[id], C = st->CS[id], psio = st->psiOld[id];
        const double phio = st->phi_o[id], Co = st->C_o[id], Qo = st->Q_o[id];
        const double vo[3] = {st->v_o[0][id], st->v_o[1][id], st->v_o[2][id]};
        /* stencils */
        double gp[3], gs[3], dv[3][3];   /* dv[a][b] = d_b v_o,a */
        grad19(st, st->phiS, 0, x, y, z, gp);
        const double lphi = lap19(st, st->phiS, 0, x, y, z);
        grad19(st, st->psiS, 1, x, y, z, gs);
        for (int a = 0; a < 3; ++a) grad19(st, st->v_o[a], 3 + a, x, y, z, dv[a]);
        /* gas-liquid interface */
        const double rho = rg + phi * (rl - rg);
        double gr[3], nf[3];
        const double gm = sqrt(gp[0] * gp[0] + gp[1] * gp[1] + gp[2] * gp[2] + p[F3_GRAD_EPS] * p[F3_GRAD_EPS]);
        for (int a = 0; a < 3; ++a) { gr[a] = (rl - rg) * gp[a]; nf[a] = gp[a] / gm; }
        const double mu = 2.0 * p[F3_BETA_PHI] * phi * (1.0 - phi) * (1.0 - 2.0 * phi) -
                          2.0 * p[F3_BETA_INTER] * (1.0 - phi) * (1.0 + psi) * (1.0 + psi) -
                          p[F3_W_PHI] * p[F3_W_PHI] * lphi;
        const double aphi = kappa * phi * (1.0 - phi);
        double Dm[3];
        for (int a = 0; a < 3; ++a) Dm[a] = p[F3_M_PHI] * (gp[a] - aphi * nf[a]);
        const double divD = (phi - phio) + vo[0] * gp[0] + vo[1] * gp[1] + vo[2] * gp[2];
        double Fp[3];
        for (int a = 0; a < 3; ++a) {
          const double Fs = fs_coef * mu * gp[a];
          const double Fb = a == 1 ? -(rho - st->rho_bar) * p[F3_G] : 0.0;   /* reading R13 */
          const double Fm = (rl - rg) * (divD * vo[a] + Dm[0] * dv[a][0] + Dm[1] * dv[a][1] + Dm[2] * dv[a][2]);
          Fp[a] = Fs + Fb + Fm;
        }
        /* NS moments, drag (reading R2), pressure */
        real f[19];
        double j[3] = {0, 0, 0}, sum_nz = 0;
        for (int i = 0; i < 19; ++i) {
          f[i] = st->fS[i][id];
          for (int a = 0; a < 3; ++a) j[a] += C19[i][a] * f[i];
          if (i) sum_nz += f[i];
        }
        const double chi = 0.5 * (1.0 + psi);
        double vs[3], v[3], F[3];
        for (int a = 0; a < 3; ++a) {
          vs[a] = (j[a] + 0.5 * Fp[a]) / rho;
          v[a] = (1.0 - chi) * vs[a];
          F[a] = Fp[a] - 2.0 * chi * rho * vs[a];
        }
        const double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        const double pr = CS2_19 / (1.0 - W19[0]) *
                          (sum_nz + 0.5 * (v[0] * gr[0] + v[1] * gr[1] + v[2] * gr[2]) -
                           W19[0] * rho * v2 / (2.0 * CS2_19));
        /* dendrite geometry and sources */
        double as, N[3], gmag;
        if (st->rot) {
          /* crystal frame g' = R^T grad psi, N = R N'(g') */
          const double *R = st->rot + 9 * (size_t)id;
          double gr2[3], Nr[3];
          for (int a = 0; a < 3; ++a) gr2[a] = R[a] * gs[0] + R[3 + a] * gs[1] + R[6 + a] * gs[2];
          aniso3(gr2, p[F3_EPS_S], p[F3_GRAD_EPS], &as, Nr, &gmag);
          for (int a = 0; a < 3; ++a) N[a] = R[3 * a] * Nr[0] + R[3 * a + 1] * Nr[1] + R[3 * a + 2] * Nr[2];
        } else {
          aniso3(gs, p[F3_EPS_S], p[F3_GRAD_EPS], &as, N, &gmag);
        }
        const double as2 = as * as;
        const double U = supersatf(st, C, psi);
        /* thermal mode: rho H = sum e, theta = H / c_p + (c_p^s/c_p) h(psi) with the
         * local rho; the source of the rewritten equation (Appendix B)
         *   Q / F + W0^2 / F^2 grad F . (a_s^2 grad psi + N), grad F = M c_inf (1-k) grad U */
        const int th_on = thermalf(st);
        double rhoH = 0.0, theta = 0.0, Fu = 1.0, Q;
        if (th_on) {
          for (int i = 0; i < 7; ++i) rhoH += st->eS[i][id];
          theta = rhoH / (rho * p[F3_CP]) + p[F3_LATENT] * 0.5 * (1.0 + psi);
          const double Q0 = qpsif_at(st, phi, psi, U, theta);
          double lam, Mc, thsys, gu[3];
          derivedf(st, &lam, &Mc, &thsys);
          grad19(st, st->US, 2, x, y, z, gu);
          double dot = 0;
          for (int a = 0; a < 3; ++a) dot += Mc * (1.0 - k) * gu[a] * (as2 * gs[a] + N[a]);
          Fu = f_of_uf(st, U);
          Q = Q0 / Fu + W0 * W0 / (Fu * Fu) * dot;
        } else {
          Q = qpsif(st, phi, psi, U);
        }
        const double at = -(1.0 / (2.0 * sqrt(2.0))) * W0 * as * (1.0 + (1.0 - k) * U) * (psi - psio) /
                          sqrt(gs[0] * gs[0] + gs[1] * gs[1] + gs[2] * gs[2] +
                               p[F3_GRAD_EPS_AT] * p[F3_GRAD_EPS_AT]);
        const double qf = 0.5 * (1.0 - psi);
        const double jv = p[F3_D] * qf * C * kappa * (1.0 - phi);     /* gas-vacuum flux J */
        /* NS collision: D3Q19 MRT with forcing */
        {
          real feq[19], G[19], out[19];
          feq19(pr, rho, v, feq);
          for (int i = 0; i < 19; ++i) {
            const double cF = C19[i][0] * F[0] + C19[i][1] * F[1] + C19[i][2] * F[2];
            const double cv = C19[i][0] * v[0] + C19[i][1] * v[1] + C19[i][2] * v[2];
            const double cg = C19[i][0] * gr[0] + C19[i][1] * gr[1] + C19[i][2] * gr[2];
            G[i] = W19[i] * (cF / CS2_19 + cv * cg / CS2_19);
          }
          const real S[19] = {1, p[F3_S_E], p[F3_S_EPS], 1, s_q, 1, s_q, 1, s_q,
                              s_nu, 1, s_nu, 1, s_nu, s_nu, s_nu, s_q, s_q, s_q};
          collide19(f, feq, S, G, out);
          for (int i = 0; i < 19; ++i) st->nf[i][id] = out[i];
        }
        /* CAC collision: D3Q19 MRT, fluxes at s_phi from M_phi = (1/s - 1/2) c_s^2 */
        {
          real hh[19], heq[19], G[19], out[19];
          for (int i = 0; i < 19; ++i) hh[i] = st->hS[i][id];
          heq19(phi, v, heq);
          double G1[3];
          for (int a = 0; a < 3; ++a) G1[a] = (phi * v[a] - phio * vo[a]) + CS2_19 * aphi * nf[a];
          for (int i = 0; i < 19; ++i)
            G[i] = W19[i] * (C19[i][0] * G1[0] + C19[i][1] * G1[1] + C19[i][2] * G1[2]) / CS2_19;
          real S[19];
          for (int kk = 0; kk < 19; ++kk) S[kk] = 1.0;
          S[3] = S[5] = S[7] = s_phi;
          collide19(hh, heq, S, G, out);
          for (int i = 0; i < 19; ++i) st->nh[i][id] = out[i];
        }
        /* psi: D3Q7 MRT as in the melt-only step */
        {
          real gg[7], geq[7], G[7], Fd[7], out[7];
          for (int i = 0; i < 7; ++i) {
            gg[i] = st->gS[i][id];
            geq[i] = W7[i] * psi;
            G[i] = -W7[i] * (C7[i][0] * N[0] + C7[i][1] * N[1] + C7[i][2] * N[2]) / as2;
            Fd[i] = W7[i] * Q / tau0 + 0.5 * W7[i] * (Q - Qo) / tau0;
          }
          const double s1 = 1.0 / (W0 * W0 * as2 / (tau0 * Fu * CS2_7) + 0.5);
          const real S[7] = {1, s1, s1, s1, 1, 1, 1};
          collide7(gg, geq, S, G, Fd, out);
          for (int i = 0; i < 7; ++i) { st->ngpost[i][id] = out[i]; st->ngpre[i][id] = gg[i]; }
          st->nrr[id] = 1.0 / as2;
        }
        /* solute: D3Q7, C v - E grad psi + (1-k)(J_at + J) in the equilibrium
         * flux, G = w c . d_t(C v) / c_s^2 (backward difference) */
        {
          real ss[7], seq[7], G[7], Fd[7] = {0, 0, 0, 0, 0, 0, 0}, out[7];
          const double A = 1.0 + k - (1.0 - k) * psi;
          const double DC = 2.0 * p[F3_D] * qf / A;
          const double E = 2.0 * (1.0 - k) * p[F3_D] * qf * C / (A * A);
          double Jq[3], Gq[3];
          for (int a = 0; a < 3; ++a) {
            Jq[a] = C * v[a] - E * gs[a] + (1.0 - k) * (at * gs[a] + jv * nf[a]);
            Gq[a] = C * v[a] - Co * vo[a];
          }
          for (int i = 0; i < 7; ++i) {
            ss[i] = st->sS[i][id];
            seq[i] = W7[i] * C + W7[i] * (C7[i][0] * Jq[0] + C7[i][1] * Jq[1] + C7[i][2] * Jq[2]) / CS2_7;
            G[i] = W7[i] * (C7[i][0] * Gq[0] + C7[i][1] * Gq[1] + C7[i][2] * Gq[2]) / CS2_7;
          }
          const double sc = 1.0 / (DC / CS2_7 + 0.5);
          const real S[7] = {1, sc, sc, sc, 1, 1, 1};
          collide7(ss, seq, S, G, Fd, out);
          for (int i = 0; i < 7; ++i) st->ns[i][id] = out[i];
        }
        /* temperature collision (thermal mode): D3Q7 MRT with the equilibrium
         * flux rho H v and G = w c . d_t(rho H v) / c_s^2 (backward difference),
         * flux rate from k_T = Le D rho_l c_p = (1/s - 1/2) c_s^2 */
        if (th_on) {
          real ee[7], teq[7], G[7], Fd[7] = {0, 0, 0, 0, 0, 0, 0}, out[7];
          const double rho_o = rg + phio * (rl - rg);
          double j[3], Gq[3];
          for (int a = 0; a < 3; ++a) {
            j[a] = rhoH * v[a];
            Gq[a] = j[a] - rho_o * st->H_o[id] * vo[a];
          }
          teqf(rhoH, theta, j, teq);
          for (int i = 0; i < 7; ++i) {
            ee[i] = st->eS[i][id];
            G[i] = W7[i] * (C7[i][0] * Gq[0] + C7[i][1] * Gq[1] + C7[i][2] * Gq[2]) / CS2_7;
          }
          const double kT = p[F3_LE] * p[F3_D] * rl * p[F3_CP];
          const double sth = 1.0 / (kT / CS2_7 + 0.5);
          const real S[7] = {1, sth, sth, sth, 1, 1, 1};
          collide7(ee, teq, S, G, Fd, out);
          for (int i = 0; i < 7; ++i) st->ne[i][id] = out[i];
          st->nH_o[id] = rhoH / rho;
          st->fld[G3_THETA][id] = theta;
        } else {
          double lam, Mc, thsys;
          derivedf(st, &lam, &Mc, &thsys);
          st->fld[G3_THETA][id] = thsys;
        }
        st->nQ_o[id] = Q;
        st->nphi_o[id] = phi;
        st->nC_o[id] = C;
        for (int a = 0; a < 3; ++a) st->nv_o[a][id] = v[a];
        st->fld[G3_PHI][id] = phi; st->fld[G3_PSI][id] = psi; st->fld[G3_C][id] = C;
        st->fld[G3_U][id] = U; st->fld[G3_P][id] = pr;
        st->fld[G3_VX][id] = v[0]; st->fld[G3_VY][id] = v[1]; st->fld[G3_VZ][id] = v[2];
        st->fld[G3_MU][id] = mu;
      }
  real *t;
#define SW(a, b) do { t = (a); (a) = (b); (b) = t; } while (0)
  for (int i = 0; i < 19; ++i) { SW(st->f[i], st->nf[i]); SW(st->h[i], st->nh[i]); }
  for (int i = 0; i < 7; ++i) { SW(st->gpre[i], st->ngpre[i]); SW(st->gpost[i], st->ngpost[i]); SW(st->s[i], st->ns[i]); }
  SW(st->rr, st->nrr); SW(st->Q_o, st->nQ_o); SW(st->phi_o, st->nphi_o); SW(st->C_o, st->nC_o);
  for (int a = 0; a < 3; ++a) SW(st->v_o[a], st->nv_o[a]);
  if (thermalf(st)) {
    for (int i = 0; i < 7; ++i) SW(st->e[i], st->ne[i]);
    SW(st->H_o, st->nH_o);
  }
#undef SW
  st->steps++;
}

void or3f_step(o3fstate *st, int n) {
  for (int t = 0; t < n; ++t) step3f(st);
}

int or3f_nfields(void) { return NFLD3F; }
int or3f_npar(void) { return NPAR3F; }

/* Fields phi, psi, C, U, p, vx, vy, vz, mu_phi, theta of the last step (10 x n). */
void or3f_fields(const o3fstate *st, double *out) {
  for (int f = 0; f < NFLD3F; ++f) memcpy(out + (size_t)f * st->n, st->fld[f], st->n * sizeof(double));
}

/* Raw state, 66 planes: f[19], h[19], g_pre[7], g_post[7], r, s[7], Q_o,
 * phi_o, C_o, vx_o, vy_o, vz_o; in thermal mode 74 (e[7] and H_o follow). */
int or3f_state_planes(const o3fstate *st) { return thermalf(st) ? 74 : 66; }
void or3f_state(const o3fstate *st, double *out) {
  const real *pl[74];
  int q = 0;
  for (int i = 0; i < 19; ++i) pl[q++] = st->f[i];
  for (int i = 0; i < 19; ++i) pl[q++] = st->h[i];
  for (int i = 0; i < 7; ++i) pl[q++] = st->gpre[i];
  for (int i = 0; i < 7; ++i) pl[q++] = st->gpost[i];
  pl[q++] = st->rr;
  for (int i = 0; i < 7; ++i) pl[q++] = st->s[i];
  pl[q++] = st->Q_o; pl[q++] = st->phi_o; pl[q++] = st->C_o;
  for (int a = 0; a < 3; ++a) pl[q++] = st->v_o[a];
  if (thermalf(st)) {             /* then e[7] and the lagged H */
    for (int i = 0; i < 7; ++i) pl[q++] = st->e[i];
    pl[q++] = st->H_o;
  }
  for (int p = 0; p < q; ++p) memcpy(out + (size_t)p * st->n, pl[p], st->n * sizeof(double));
}

/* Thermal mode: compensated sums of the temperature populations (rho H) and
 * of theta. */
void or3f_thermal_totals(const o3fstate *st, double *out) {
  double s2[2] = {0, 0}, c2[2] = {0, 0};
  for (int id = 0; id < st->n; ++id)
    for (int k2 = 0; k2 < 8; ++k2) {
      const double v = k2 < 7 ? st->e[k2][id] : st->fld[G3_THETA][id];
      const int j = k2 < 7 ? 0 : 1;
      const double t = s2[j] + v;
      c2[j] += fabs(s2[j]) >= fabs(v) ? (s2[j] - t) + v : (v - t) + s2[j];
      s2[j] = t;
    }
  out[0] = s2[0] + c2[0];
  out[1] = s2[1] + c2[1];
}

/* Totals (compensated): sum phi, sum C, sum of the NS momentum j = sum c f
 * (three components) of the current populations. */
void or3f_totals(const o3fstate *st, double *out) {
  double s[5] = {0, 0, 0, 0, 0}, c[5] = {0, 0, 0, 0, 0};
  for (int id = 0; id < st->n; ++id) {
    double v[5] = {st->fld[G3_PHI][id], st->fld[G3_C][id], 0, 0, 0};
    for (int i = 0; i < 19; ++i)
      for (int a = 0; a < 3; ++a) v[2 + a] += C19[i][a] * st->f[i][id];
    for (int q = 0; q < 5; ++q) {
      const double t = s[q] + v[q];
      c[q] += fabs(s[q]) >= fabs(v[q]) ? (s[q] - t) + v[q] : (v[q] - t) + s[q];
      s[q] = t;
    }
  }
  for (int q = 0; q < 5; ++q) out[q] = s[q] + c[q];
}

/* Pointwise pieces for the pin tests: the D3Q19 basis and weights, the MRT
 * collision, the equilibria. */
void or3f_basis(double *M, double *W, int *C) {
  build_m19();
  for (int k = 0; k < 19; ++k)
    for (int j = 0; j < 19; ++j) M[k * 19 + j] = M19[k][j];
  for (int j = 0; j < 19; ++j) {
    W[j] = W19[j];
    for (int a = 0; a < 3; ++a) C[3 * j + a] = C19[j][a];
  }
}
void or3f_collide19(const double *f, const double *feq, const double *S, const double *G, double *out) {
  build_m19();
  collide19(f, feq, S, G, out);
}
void or3f_feq(double p, double rho, const double *v, double *out) {
  build_m19();
  feq19(p, rho, v, out);
}
