// pf_step3f_bc.cu -- the boundary-aware variants of the 3-D two-phase step
// kernel (k_step3f with BC = true: non-periodic sides), compiled apart from
// the periodic ones so that the two sets build in parallel.
#include "pf_step3f.cuh"

namespace pf {
namespace d3f {

template <typename S, typename R>
cudaError_t launch3f_bc(const ArgsF<S, R>& a, bool rotated, bool thermal, int tiles, size_t smem,
                        cudaStream_t st) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaSuccess;
    auto big = [&](auto kern) {
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    };
    big(k_step3f<S, R, false, false, true>);
    big(k_step3f<S, R, true, false, true>);
    big(k_step3f<S, R, false, true, true>);
    big(k_step3f<S, R, true, true, true>);
    if (e != cudaSuccess) return e;
  }
  if (thermal) {
    if (rotated) k_step3f<S, R, true, true, true><<<tiles, THREADS, smem, st>>>(a);
    else k_step3f<S, R, false, true, true><<<tiles, THREADS, smem, st>>>(a);
  } else {
    if (rotated) k_step3f<S, R, true, false, true><<<tiles, THREADS, smem, st>>>(a);
    else k_step3f<S, R, false, false, true><<<tiles, THREADS, smem, st>>>(a);
  }
  return cudaGetLastError();
}

template cudaError_t launch3f_bc<float, float>(const ArgsF<float, float>&, bool, bool, int, size_t,
                                               cudaStream_t);
template cudaError_t launch3f_bc<double, double>(const ArgsF<double, double>&, bool, bool, int,
                                                 size_t, cudaStream_t);

}  // namespace d3f
}  // namespace pf
