// pf_noalloc.cu -- FP64 diagnostics of a field stack without any device
// memory allocation.
//
// Some callers cannot allocate device memory, neither themselves nor through
// this library: a plugin living inside a host framework that owns the whole
// device-memory budget and hands out only pre-allocated buffers, or a loop
// that must never hit cudaMalloc / cudaFree (they may synchronise the device
// and stall every other stream).  pf_reduce_noalloc serves them.  The caller
// passes the field planes (device memory it already owns) and a host pf_diag;
// the per-block partial sums live in the file-scope device array below, whose
// size is fixed: every GPU that loads this library holds it until the process
// exits.
//
// Capacity: one block of 256 threads reduces 4096 consecutive sites into one
// partial record of 12 doubles; at most 16384 blocks, i.e. 67,108,864 sites
// per call (an 8192 x 8192 lattice), 1.5 MiB of device memory.
#include <cstring>

#include "../../include/pf.h"
#include "pf_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kSitesPerThread = 16;
constexpr int kSitesPerBlock = kThreads * kSitesPerThread;
constexpr int kMaxBlocks = 16384;
constexpr long long kMaxSites = (long long)kMaxBlocks * kSitesPerBlock;

// partial records of every block, then the final record
static __device__ __align__(256) double g_noalloc_scratch[(kMaxBlocks + 1) * pf::NDIAG];

__device__ __forceinline__ double wrap_offset(double d, double L) {
  d = fmod(d, L);
  if (d < -0.5 * L) d += L;
  if (d >= 0.5 * L) d -= L;
  return d;
}

// Block b reduces sites [b * kSitesPerBlock, (b + 1) * kSitesPerBlock) into
// record b: the same 12 quantities as pf_reduce (sums, gas moments, Laplace
// probe, max |v|, non-finite count).
template <typename R>
__global__ void __launch_bounds__(kThreads) k_noalloc_partial(
    const R* __restrict__ fields, long long ps, long long off, int nx, int ny, int probe,
    double xc, double yc, double Rp, double W, double* __restrict__ scratch) {
  double acc[pf::NDIAG];
#pragma unroll
  for (int q = 0; q < pf::NDIAG; ++q) acc[q] = 0.0;
  const long long n = (long long)nx * ny;
  const long long first = (long long)blockIdx.x * kSitesPerBlock;
  const double r_in = Rp - 2.0 * W, r_out = Rp + 4.0 * W;
  for (int k = 0; k < kSitesPerThread; ++k) {
    const long long i = first + (long long)k * kThreads + threadIdx.x;
    if (i >= n) break;
    const long long s = off + i;
    const double phi = (double)fields[pf::FLD_PHI * ps + s];
    const double psi = (double)fields[pf::FLD_PSI * ps + s];
    const double C = (double)fields[pf::FLD_C * ps + s];
    const double p = (double)fields[pf::FLD_P * ps + s];
    const double vx = (double)fields[pf::FLD_VX * ps + s];
    const double vy = (double)fields[pf::FLD_VY * ps + s];
    const double x = (double)(i % nx), y = (double)(i / nx);
    acc[0] += phi;
    acc[1] += C;
    acc[2] += 0.5 * (1.0 + psi);
    acc[3] += 1.0 - phi;
    acc[4] += x * (1.0 - phi);
    acc[5] += y * (1.0 - phi);
    if (probe) {
      const double dx = wrap_offset(x - xc, (double)nx), dy = wrap_offset(y - yc, (double)ny);
      const double r = sqrt(dx * dx + dy * dy);
      if (r < r_in) { acc[6] += p; acc[7] += 1.0; }
      if (r > r_out) { acc[8] += p; acc[9] += 1.0; }
    }
    acc[10] = fmax(acc[10], sqrt(vx * vx + vy * vy));
    if (!isfinite(phi) || !isfinite(psi) || !isfinite(C) || !isfinite(p) || !isfinite(vx) ||
        !isfinite(vy))
      acc[11] += 1.0;
  }
  __shared__ double red[pf::NDIAG][kThreads];
#pragma unroll
  for (int q = 0; q < pf::NDIAG; ++q) red[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int half = kThreads / 2; half > 0; half >>= 1) {
    if ((int)threadIdx.x < half) {
#pragma unroll
      for (int q = 0; q < pf::NDIAG; ++q) {
        const double o = red[q][threadIdx.x + half];
        red[q][threadIdx.x] = q == 10 ? fmax(red[q][threadIdx.x], o) : red[q][threadIdx.x] + o;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x < pf::NDIAG) scratch[blockIdx.x * pf::NDIAG + threadIdx.x] = red[threadIdx.x][0];
}

// One warp: record q of the final result sums (or maxes) the block records
// in block order, so the result does not depend on scheduling.
__global__ void k_noalloc_final(double* __restrict__ scratch, int nblocks) {
  const int q = threadIdx.x;
  if (q >= pf::NDIAG) return;
  double acc = 0.0;
  for (int b = 0; b < nblocks; ++b) {
    const double v = scratch[b * pf::NDIAG + q];
    acc = q == 10 ? fmax(acc, v) : acc + v;
  }
  scratch[kMaxBlocks * pf::NDIAG + q] = acc;
}

// Device address of the scratch array in the current context.  The host-side
// name of a __device__ array is not its address, and the address belongs to
// the module loaded into the current context: a context that was reset and
// re-created may place it elsewhere.  So it is looked up on every call (a host
// lookup; it allocates nothing) instead of being cached per device.
pf_status scratch_for_current_context(double** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    pf::set_global_error(std::string("pf_reduce_noalloc: cudaGetSymbolAddress: ") +
                         cudaGetErrorString(e));
    return PF_ERR_CUDA;
  }
  *out = static_cast<double*>(p);
  return PF_OK;
}

}  // namespace

extern "C" pf_status pf_reduce_noalloc(const void* fields, int fields_fp64, long long plane_stride,
                                       long long offset, int nx, int ny, const pf_probe* probe,
                                       pf_diag* out, void* cuda_stream) {
  if (!fields || !out) {
    pf::set_global_error("pf_reduce_noalloc: fields and out must be non-NULL");
    return PF_ERR_BAD_ARG;
  }
  if (nx < 1 || ny < 1 || offset < 0) {
    pf::set_global_error("pf_reduce_noalloc: nx, ny must be >= 1 and offset >= 0");
    return PF_ERR_BAD_ARG;
  }
  const long long n = (long long)nx * ny;
  if (n > kMaxSites) {
    pf::set_global_error("pf_reduce_noalloc: lattice exceeds the 67,108,864-site capacity of "
                         "its fixed scratch");
    return PF_ERR_BAD_ARG;
  }
  if (plane_stride < offset + n) {
    pf::set_global_error("pf_reduce_noalloc: plane_stride must cover offset + nx*ny");
    return PF_ERR_BAD_ARG;
  }
  double* scratch = nullptr;
  pf_status st = scratch_for_current_context(&scratch);
  if (st != PF_OK) return st;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  const int nblocks = (int)((n + kSitesPerBlock - 1) / kSitesPerBlock);
  const int pr = probe != nullptr;
  const double xc = pr ? probe->xc : 0.0, yc = pr ? probe->yc : 0.0;
  const double R = pr ? probe->R : 0.0, W = pr ? probe->W : 0.0;
  if (fields_fp64)
    k_noalloc_partial<double><<<nblocks, kThreads, 0, stream>>>(
        static_cast<const double*>(fields), plane_stride, offset, nx, ny, pr, xc, yc, R, W, scratch);
  else
    k_noalloc_partial<float><<<nblocks, kThreads, 0, stream>>>(
        static_cast<const float*>(fields), plane_stride, offset, nx, ny, pr, xc, yc, R, W, scratch);
  k_noalloc_final<<<1, 32, 0, stream>>>(scratch, nblocks);
  double res[pf::NDIAG];
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(res, scratch + (size_t)kMaxBlocks * pf::NDIAG, sizeof(res),
                        cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) {
    pf::set_global_error(std::string("pf_reduce_noalloc: ") + cudaGetErrorString(e));
    return PF_ERR_CUDA;
  }
  static_assert(sizeof(pf_diag) == sizeof(res), "pf_diag layout");
  std::memcpy(out, res, sizeof(res));
  return PF_OK;
}
