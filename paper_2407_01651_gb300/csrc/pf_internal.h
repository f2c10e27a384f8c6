// pf_internal.h -- kernel argument blocks and launchers shared by the kernel
// translation unit and the C-ABI implementation.
#pragma once

#include <cstdint>
#include <string>
#include <cuda_runtime.h>

#include "pf_model.cuh"

namespace pf {

constexpr int NDIAG = 12;            // entries of pf_diag
constexpr int REDUCE_BLOCKS = 1024;  // blocks of the first reduction pass
constexpr int MAX_GRAINS = 256;      // grain ids are uint8
#define PF_RUN_BANDS 32              // row bands of pf_run (at most)

// Step kernel variants (same arithmetic, different traversal).
enum StepVariant : int { STEP_TILE = 0, STEP_YMARCH = 1, STEP_STAGED = 2 };
constexpr int YM_W = 128;            // interior columns of a y-march strip
constexpr int YM_THREADS = YM_W + 32;  // + one warp whose lanes 0, 1 own the halo columns

template <typename S, typename R>
struct StepArgs {
  const S* __restrict__ in;     // population planes read this step
  S* __restrict__ out;          // population planes written this step
  const R* __restrict__ ain;    // lagged-scalar planes read this step
  R* __restrict__ aout;         // lagged-scalar planes written this step
  long long plane_stride;       // sites per plane (all domains, padded)
  const uint8_t* __restrict__ grain;    // grain id per site
  const double2* __restrict__ grain_cs; // (cos, sin) of each grain angle
  const DomDesc* __restrict__ doms;
  const int* __restrict__ tile_dom;     // domain of each tile
  int tile_base;                // first tile of this launch
  int ntiles;                   // one past the last tile of this launch
  int chunk;                    // rows per y-march tile
  R* fields;                    // 8 field planes, or nullptr
  unsigned int* err;            // device error bits (1: a staged copy timed out), or nullptr
  int drop_copies;              // testing only: the staged kernel skips its bulk copies
  int thermal;                  // 1: temperature lattice and finite-Le F(U) (FP32 / FP64)
  int bc;                       // 1: some domain has a non-periodic side (y-march only)
  KParams<R> kp;
};

template <typename S, typename R>
struct InitArgs {
  S* out;
  R* aout;
  R* fields;
  uint8_t* grain;
  long long plane_stride;
  DomDesc dom;
  const double* seeds;    // device, n_seeds x 3
  const double* bubbles;  // device, n_bub x 3
  int n_seeds, n_bub;
  double R_s, W0, Wphi, sq2bpsi, sq2bphi, k;
  KParams<R> kp;
  int thermal;           // also initialise the temperature lattice at theta0
  double theta0;
};

template <typename S, typename R>
struct SetFieldsArgs {
  S* out;
  R* aout;
  R* fields;
  uint8_t* grain;
  long long plane_stride;
  DomDesc dom;
  const double* f6;          // device, 6 x n
  const uint8_t* grain_ids;  // device, n, or nullptr
  KParams<R> kp;
  int thermal;               // also initialise the temperature lattice at theta0
  double theta0;
  unsigned int* err;         // device error bits: ERR_NONFINITE_INPUT set on a non-finite value
  long long i0, i1;          // sites [i0, i1) of the domain (i1 <= 0: the whole domain)
};

// Device error bits (pf_handle::d_err).
constexpr unsigned int ERR_STAGED_TIMEOUT = 1u;   // a staged bulk copy did not complete
constexpr unsigned int ERR_NONFINITE_INPUT = 2u;  // pf_set_fields met a non-finite value

template <typename R>
struct ReduceArgs {
  const R* fields;
  long long plane_stride;
  DomDesc dom;
  int probe;
  double xc, yc, Rp, W;
};

template <typename S, typename R>
cudaError_t launch_step(const StepArgs<S, R>& a, int variant, int tx, int ty, int grid,
                        cudaStream_t st);
// Staged variant (bulk copies of the input rows into shared memory): launch,
// dynamic shared memory, the x granularity it needs (nx a multiple of it), and
// resident CTAs per SM.
template <typename S, typename R>
cudaError_t launch_step_staged(const StepArgs<S, R>& a, int grid, cudaStream_t st);
// y-march for handles with non-periodic domain sides (FP32 / FP64 storage).
template <typename S, typename R>
cudaError_t launch_ymarch_bc(const StepArgs<S, R>& a, bool big, int grid, cudaStream_t st);
template <typename S, typename R>
int ymarch_bc_blocks_per_sm(bool big, bool thermal);
template <typename S, typename R>
int staged_smem_bytes();
template <typename S, typename R>
int staged_halo_columns();
template <typename S, typename R>
int staged_blocks_per_sm();
// Every step of a call in one cooperative launch (y-march, periodic domains),
// and the resident CTAs per SM of that kernel.
// ctr: two device ints (tile counters), owned by the caller.
template <typename S, typename R>
cudaError_t launch_ymarch_steps(const StepArgs<S, R>& a, int nsteps, int* ctr, int grid,
                                cudaStream_t st);
template <typename S, typename R>
int ymarch_steps_blocks_per_sm(long long plane_stride, bool thermal);
// Resident CTAs per SM of the step kernel (for persistent grids).
template <typename S, typename R>
int step_blocks_per_sm(int variant, int tx, int ty, long long plane_stride, bool thermal,
                       bool bc);
template <typename S, typename R>
cudaError_t launch_init_spec(const InitArgs<S, R>& a, cudaStream_t st);
template <typename S, typename R>
cudaError_t launch_set_fields(const SetFieldsArgs<S, R>& a, cudaStream_t st);
// *flag = 1 if any of the n device values at p is NaN or infinite, else 0.
cudaError_t launch_flag_nonfinite(const double* p, long long n, unsigned int* flag,
                                  cudaStream_t st);
template <typename S, typename R>
cudaError_t launch_state_to_f64(const S* pin, const R* ain, long long ps, long long off,
                                long long n, double* out, int thermal, cudaStream_t st);
template <typename S, typename R>
cudaError_t launch_state_from_f64(S* pout, R* aout, long long ps, long long off, long long n,
                                  const double* in, int thermal, cudaStream_t st);
// Thermal mode: temperature lattice at equilibrium for a theta field (device,
// n of the domain), and the FP64 totals (sum e, sum theta, sum psi).
template <typename S, typename R>
cudaError_t launch_set_temperature(S* out, R* aout, R* fields, long long ps, const DomDesc& d,
                                   const double* theta, const KParams<R>& kp, cudaStream_t st);
template <typename S, typename R>
cudaError_t launch_reduce_thermal(const S* pop, const R* fields, long long ps, const DomDesc& d,
                                  double* partial, double* out, cudaStream_t st);
template <typename R>
cudaError_t launch_fields_to_f64(const R* fields, long long ps, long long off, long long n,
                                 uint32_t mask, double* out, cudaStream_t st);
// The same for sites [j0, j1) of the domain only (out keeps the stride n per field).
template <typename R>
cudaError_t launch_fields_to_f64_range(const R* fields, long long ps, long long off, long long n,
                                       long long j0, long long j1, uint32_t mask, double* out,
                                       cudaStream_t st);
// *out = the FP64 sum over the n values phi[i] rounded to R, in the order of
// the diagnostics reduction (launch_reduce): equal to its sum of phi over the
// fields that pf_set_fields writes from the same values.  partial: REDUCE_BLOCKS doubles.
template <typename R>
cudaError_t launch_sum_as(const double* phi, long long n, double* partial, double* out,
                          cudaStream_t st);
// doms[dom].rho_bar = fma(*sum / n, drho, rho_g), on the device.
cudaError_t launch_set_rho_bar(DomDesc* doms, int dom, const double* sum, double n, double rho_g,
                               double drho, cudaStream_t st);
template <typename R>
cudaError_t launch_reduce(const ReduceArgs<R>& a, double* partial, double* out,
                          cudaStream_t st);

// ---------------------------------------------------------------------------
// Discrete adjoint
// ---------------------------------------------------------------------------
constexpr int ADJ_TX = 32, ADJ_TY = 8;  // tile of the local reverse kernel
constexpr int ADJ_LAUNCHES_PER_STEP = 2;  // kernels of one reverse step
// Planes of the per-site input adjoints (layout of local::In).
enum AiPlane : int {
  AI_F = 0, AI_H = 9, AI_G = 18, AI_S = 23, AI_PSIO = 28, AI_GPX = 29, AI_GPY = 30,
  AI_LPHI = 31, AI_GSX = 32, AI_GSY = 33, AI_DVXX = 34, AI_DVXY = 35, AI_DVYX = 36,
  AI_DVYY = 37, AI_PHIO = 38, AI_CO = 39, AI_QO = 40, AI_VXO = 41, AI_VYO = 42, N_AI = 43
};

template <typename S, typename R>
struct AdjArgs {
  StepArgs<S, R> step;     // the state x_t (in / ain) and the coefficients
  DomDesc dom;
  const R* lam_in;         // lambda_{t+1}, 39 planes
  R* lam_out;              // lambda_t, 39 planes
  R* ai;                   // input adjoints, N_AI planes
  double* partial;         // per-block parameter adjoints (eps, Omega, sigma), accumulated
  double dfs_dsigma;       // d(surface-tension coefficient)/d sigma
};

template <typename S, typename R>
cudaError_t launch_adjoint_step(const AdjArgs<S, R>& a, int grid, cudaStream_t st);
template <typename R>
cudaError_t launch_adj_objective(R* lam, DomDesc d, long long ps, double w_s, double w_c,
                                 double yc, double gas, cudaStream_t st);
template <typename S, typename R>
cudaError_t launch_adj_omega_init(const R* lam, const S* pop, const R* aux, DomDesc d,
                                  long long ps, double lam_p, double k, double* partial,
                                  int blocks, cudaStream_t st);

// Message returned by pf_last_error(NULL) (entry points without a handle).
void set_global_error(const std::string& msg);

}  // namespace pf
