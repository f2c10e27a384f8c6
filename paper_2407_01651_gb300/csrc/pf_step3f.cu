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
#include <type_traits>
#include <vector>

#include "pf_step3f.cuh"

namespace pf {
namespace d3f {

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
      for (int q = 0; q < 3; ++q) {     // minimum image along periodic axes only
        const double d = a.bc[2 * q] == 0 ? min_image(X[q] - seeds[3 * s + q], L[q]) : X[q] - seeds[3 * s + q];
        r2 += d * d;
      }
      const double v = tanh(sb * (R_s - sqrt(r2)) / W0);
      if (s == 0 || v > psi) psi = v;
    }
    for (int b = 0; b < n_bub; ++b) {
      double r2 = 0;
      for (int q = 0; q < 3; ++q) {
        const double d = a.bc[2 * q] == 0 ? min_image(X[q] - bub[4 * b + q], L[q]) : X[q] - bub[4 * b + q];
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
  int nx = 0, ny = 0, nz = 0, chunk = 36;  // z-march tile (tuned at 256^3 on 152 SMs)
  int index64 = 0;  // periodic step in 64-bit indices at any size
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
  int bc[6] = {0, 0, 0, 0, 0, 0}; // side types x-, x+, y-, y+, z-, z+
  int any_bc = 0;
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
  c.th0 = (R)p.theta0;
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

template <typename S, typename R, typename I = unsigned long long>
static ArgsF<S, R, I> argsf(const pf3f_handle* h, bool fields) {
  ArgsF<S, R, I> a{};
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
  pf_status st = ensure_scratchf(h, n + 1);
  if (st != PF_OK) return st;
  PF3F_CUDA(h, cudaMemcpyAsync(h->scratch, fields7, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  {
    // non-finite values are found on the device, before the state is touched
    unsigned int* flag = reinterpret_cast<unsigned int*>(h->scratch + n);
    unsigned int bits = 0;
    PF3F_CUDA(h, cudaMemsetAsync(flag, 0, sizeof(unsigned int), h->stream));
    pf::d3::k_flag_nonfinite<<<1024, 256, 0, h->stream>>>(h->scratch, (long long)n, flag);
    PF3F_CUDA(h, cudaGetLastError());
    h->launches++;
    PF3F_CUDA(h, cudaMemcpyAsync(&bits, flag, sizeof(bits), cudaMemcpyDeviceToHost, h->stream));
    PF3F_CUDA(h, cudaStreamSynchronize(h->stream));
    if (bits) return failf(h, PF_ERR_BAD_ARG, "non-finite field");
  }
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

extern "C" pf_status pf3f_set_boundaries(pf3f_handle* h, const int bc[6]) {
  if (!h) return PF_ERR_BAD_ARG;
  if (!bc) return failf(h, PF_ERR_BAD_ARG, "NULL bc");
  for (int k = 0; k < 6; ++k)
    if (bc[k] < 0 || bc[k] > 3)
      return failf(h, PF_ERR_BAD_ARG, "side types are 0 (periodic) .. 3 (far field)");
  for (int d = 0; d < 3; ++d)
    if ((bc[2 * d] == 0) != (bc[2 * d + 1] == 0))
      return failf(h, PF_ERR_BAD_ARG, "a periodic side needs a periodic opposite side");
  if (h->inited) return failf(h, PF_ERR_STATE, "set the sides before initialising");
  h->any_bc = 0;
  for (int k = 0; k < 6; ++k) {
    h->bc[k] = bc[k];
    if (bc[k]) h->any_bc = 1;
  }
  return PF_OK;
}

extern "C" pf_status pf3f_set_chunk(pf3f_handle* h, int chunk) {
  if (!h) return PF_ERR_BAD_ARG;
  if (chunk < 1 || chunk > 2048) return failf(h, PF_ERR_BAD_ARG, "chunk must be in [1, 2048]");
  h->chunk = chunk;
  return PF_OK;
}

extern "C" pf_status pf3f_set_index64(pf3f_handle* h, int on) {
  if (!h) return PF_ERR_BAD_ARG;
  h->index64 = on != 0;
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
    // periodic launches index sites and planes in 32 bits while every plane
    // offset (below NSTATEF_TH x sites) fits
    const bool a32 = !h->any_bc && !h->index64 && (unsigned long long)NSTATEF_TH * h->n <= 0xFFFFFFFFull;
    const bool rot = h->rotated != 0, th = h->thermal != 0;
    for (int t = 0; t < n_steps; ++t) {
      const bool last = t == n_steps - 1;
      const ArgsF<S, R> a = argsf<S, R>(h, last);
      const int tiles = a.tiles_x * a.tiles_y * a.tiles_z;
      if (a32)
        PF3F_CUDA(h, (launch3f<S, R, false, unsigned>(argsf<S, R, unsigned>(h, last), rot, th, tiles,
                                                      smem, h->stream)));
      else if (h->any_bc)
        PF3F_CUDA(h, (launch3f<S, R, true>(a, rot, th, tiles, smem, h->stream)));
      else
        PF3F_CUDA(h, (launch3f<S, R, false>(a, rot, th, tiles, smem, h->stream)));
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
  if (!h->inited || h->steps != 0)
    return failf(h, PF_ERR_STATE, "set the temperature after initialisation, before stepping");
  pf_status st = ensure_scratchf(h, n + 1);
  if (st != PF_OK) return st;
  PF3F_CUDA(h, cudaMemcpyAsync(h->scratch, theta, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  {
    // non-finite values are found on the device, before the state is touched
    unsigned int* flag = reinterpret_cast<unsigned int*>(h->scratch + n);
    unsigned int bits = 0;
    PF3F_CUDA(h, cudaMemsetAsync(flag, 0, sizeof(unsigned int), h->stream));
    pf::d3::k_flag_nonfinite<<<1024, 256, 0, h->stream>>>(h->scratch, (long long)n, flag);
    PF3F_CUDA(h, cudaGetLastError());
    h->launches++;
    PF3F_CUDA(h, cudaMemcpyAsync(&bits, flag, sizeof(bits), cudaMemcpyDeviceToHost, h->stream));
    PF3F_CUDA(h, cudaStreamSynchronize(h->stream));
    if (bits) return failf(h, PF_ERR_BAD_ARG, "non-finite theta");
  }
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
