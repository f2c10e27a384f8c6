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

// Step kernel variants (same arithmetic, different traversal).
enum StepVariant : int { STEP_TILE = 0, STEP_YMARCH = 1 };
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
  int ntiles;
  int chunk;                    // rows per y-march tile
  R* fields;                    // 8 field planes, or nullptr
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
};

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
template <typename S, typename R>
cudaError_t launch_init_spec(const InitArgs<S, R>& a, cudaStream_t st);
template <typename S, typename R>
cudaError_t launch_set_fields(const SetFieldsArgs<S, R>& a, cudaStream_t st);
template <typename S, typename R>
cudaError_t launch_state_to_f64(const S* pin, const R* ain, long long ps, long long off,
                                long long n, double* out, cudaStream_t st);
template <typename S, typename R>
cudaError_t launch_state_from_f64(S* pout, R* aout, long long ps, long long off, long long n,
                                  const double* in, cudaStream_t st);
template <typename R>
cudaError_t launch_fields_to_f64(const R* fields, long long ps, long long off, long long n,
                                 uint32_t mask, double* out, cudaStream_t st);
template <typename R>
cudaError_t launch_reduce(const ReduceArgs<R>& a, double* partial, double* out,
                          cudaStream_t st);

// Message returned by pf_last_error(NULL) (entry points without a handle).
void set_global_error(const std::string& msg);

}  // namespace pf
