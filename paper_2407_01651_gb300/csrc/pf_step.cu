// pf_step.cu -- the fused sm_103a kernel of one coupled lattice Boltzmann step
// of the gas-liquid-dendrite phase-field model (arXiv 2407.01651): streaming
// (with the a_s^2 time stretch of the dendrite lattice), zeroth moments,
// isotropic stencils, interface geometry, forces and sources, and the four
// MRT collisions (NS and CAC on D2Q9, dendrite and solute on D2Q5), fused in
// one pull-scheme launch per step over a tile list that spans any number of
// periodic domains.  Two traversals with the same arithmetic:
//   k_step_tile    2-D tiles with a shared-memory halo of phi, psi, v
//   k_step_ymarch  column strips marched along y
// (and k_step_staged, pf_step_staged.cu: the y-march with its input rows
// staged in shared memory by bulk copies)
#include <cooperative_groups.h>

#include "pf_site.cuh"

namespace pf {

namespace cg = cooperative_groups;

// Variant A: 2-D tiles.  The CTA builds phi, psi and the lagged velocity on
// its TX x TY tile plus a one-site halo in shared memory, then each thread
// streams, collides and stores its own site.
template <typename S, typename R, bool BIG>
__global__ void __launch_bounds__(256) k_step_tile(StepArgs<S, R> a) {
  extern __shared__ unsigned char smem_raw[];
  const int TX = blockDim.x, TY = blockDim.y;
  const int SW = TX + 2, SH = TY + 2;
  R* sphi = reinterpret_cast<R*>(smem_raw);
  R* spsi = sphi + SW * SH;
  R* svx = spsi + SW * SH;
  R* svy = svx + SW * SH;
  const int tid = threadIdx.y * TX + threadIdx.x;
  const int nthr = TX * TY;
  const unsigned ps = (unsigned)a.plane_stride;

  for (int tile = a.tile_base + blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const DomDesc d = a.doms[a.tile_dom[tile]];
    const int lt = tile - d.tile0;
    const int x0 = (lt % d.tiles_x) * TX, y0 = (lt / d.tiles_x) * TY;
    const int nx = d.nx, ny = d.ny;

    for (int i = tid; i < SW * SH; i += nthr) {
      const int gx = wrapi(x0 + (i % SW) - 1, nx), gy = wrapi(y0 + (i / SW) - 1, ny);
      R h[9], g[5], phi, psi, po;
      pull_hg<S, R, BIG>(a, sources(d, gx, gy), h, g, phi, psi, po);
      sphi[i] = phi;
      spsi[i] = psi;
      const unsigned site = (unsigned)d.off + (unsigned)gy * (unsigned)nx + (unsigned)gx;
      svx[i] = ld<R>(pbase<BIG>(a.ain, A_VXO, ps), pidx<BIG>(A_VXO, ps, site));
      svy[i] = ld<R>(pbase<BIG>(a.ain, A_VYO, ps), pidx<BIG>(A_VYO, ps, site));
    }
    __syncthreads();

    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x < nx && y < ny) {
      const Src9 src = sources(d, x, y);
      R h[9], g[5], phi, psi, po;
      pull_hg<S, R, BIG>(a, src, h, g, phi, psi, po);
      const int r = threadIdx.y + 1;
      auto rows = [&](const R* X) { return Rows3<R>{X + (r - 1) * SW, X + r * SW, X + (r + 1) * SW}; };
      SiteIn<R> in;
      load_site<S, R, BIG>(a, src, in);
      site_update(a, d, src, in, h, g, po, rows(sphi), rows(spsi), rows(svx), rows(svy),
                  threadIdx.x + 1);
    }
    __syncthreads();
  }
}

// Variant B: column strips marched along y.  Each of the YM_W interior
// threads owns one column and walks down the rows of its tile (YM_W columns x
// `chunk` rows); lanes 0 and 1 of one extra warp own the two halo columns.  At
// row j every thread streams h and g of row j+1 (one-row lookahead kept in
// registers) and puts phi, psi and the lagged velocity of row j+1 into a
// 4-slot shared-memory ring; after one barrier the interior threads update row
// j with the stencils read from slots j-1, j, j+1.  Every population is loaded
// from memory once (plus 2 halo columns per YM_W).  TH (thermal mode) adds the
// supersaturation U of row j+1 to the ring (for grad F) and the temperature
// lattice to the site update; it runs 3 CTAs per SM.
// The tile loop of the y-march.  Tiles are taken by CTA index and stride
// (DYN = false), or claimed one at a time from the counter *ctr (DYN = true),
// which balances the CTAs of a persistent grid over tiles of uneven cost.
template <typename S, typename R, bool BIG, bool TH, bool DYN = false>
__device__ __forceinline__ void ymarch_tiles(const StepArgs<S, R>& a,
                                             R (&ring)[TH ? 5 : 4][4][YM_W + 2],
                                             int* ctr = nullptr) {
  constexpr int NF = TH ? 5 : 4;
  const int t = threadIdx.x;
  const unsigned ps = (unsigned)a.plane_stride;
  __shared__ int s_tile;
  auto next_tile = [&](int cur) {
    if constexpr (DYN) {
      if (t == 0) s_tile = a.tile_base + atomicAdd(ctr, 1);
      __syncthreads();
      return s_tile;
    } else {
      return cur < 0 ? a.tile_base + (int)blockIdx.x : cur + (int)gridDim.x;
    }
  };

  for (int tile = next_tile(-1); tile < a.ntiles; tile = next_tile(tile)) {
    const DomDesc d = a.doms[a.tile_dom[tile]];
    const int lt = tile - d.tile0;
    const int nx = d.nx, ny = d.ny;
    const int x0 = (lt % d.tiles_x) * YM_W;
    const int ya = (lt / d.tiles_x) * a.chunk;
    const int yb = min(ya + a.chunk, ny);
    const int w = min(YM_W, nx - x0);
    bool interior = false, active = false;
    int col = 0, sc = 0;
    if (t < YM_W) {
      interior = active = t < w;
      col = x0 + t;
      sc = t + 1;
    } else if (t == YM_W) {
      active = true;
      col = x0 == 0 ? nx - 1 : x0 - 1;
      sc = 0;
    } else if (t == YM_W + 1) {
      active = true;
      col = x0 + w >= nx ? x0 + w - nx : x0 + w;
      sc = w + 1;
    }

    R hC[9], gC[5], poC = R(0);
    // rows ya-1 and ya into the ring (warm-up)
    for (int k = 0; k < 2; ++k) {
      const int yy = wrapi(ya - 1 + k, ny);
      const int slot = (ya - 1 + k) & 3;
      if (active) {
        const Src9 src = sources(d, col, yy);
        R h[9], g[5], phi, psi, po;
        pull_hg<S, R, BIG>(a, src, h, g, phi, psi, po);
        ring[0][slot][sc] = phi;
        ring[1][slot][sc] = psi;
        ring[2][slot][sc] = ld<R>(pbase<BIG>(a.ain, A_VXO, ps), pidx<BIG>(A_VXO, ps, src.s[0]));
        ring[3][slot][sc] = ld<R>(pbase<BIG>(a.ain, A_VYO, ps), pidx<BIG>(A_VYO, ps, src.s[0]));
        if constexpr (TH) ring[NF - 1][slot][sc] = pull_U<S, R, BIG>(a, src, psi);
        if (k == 1) {
#pragma unroll
          for (int i = 0; i < 9; ++i) hC[i] = h[i];
#pragma unroll
          for (int i = 0; i < 5; ++i) gC[i] = g[i];
          poC = po;
        }
      }
    }

    for (int j = ya; j < yb; ++j) {
      // inputs of row j that no neighbour needs: issued before the barrier so
      // their latency overlaps the lookahead of row j+1
      SiteIn<R> in;
      const Src9 srcj = sources(d, col, j);
      if (interior) load_site<S, R, BIG, TH>(a, srcj, in);
      R hL[9], gL[5], poL = R(0);
      if (active) {
        const int yn = j + 1 >= ny ? j + 1 - ny : j + 1;
        const Src9 src = sources(d, col, yn);
        R phi, psi;
        pull_hg<S, R, BIG>(a, src, hL, gL, phi, psi, poL);
        const int slot = (j + 1) & 3;
        ring[0][slot][sc] = phi;
        ring[1][slot][sc] = psi;
        ring[2][slot][sc] = ld<R>(pbase<BIG>(a.ain, A_VXO, ps), pidx<BIG>(A_VXO, ps, src.s[0]));
        ring[3][slot][sc] = ld<R>(pbase<BIG>(a.ain, A_VYO, ps), pidx<BIG>(A_VYO, ps, src.s[0]));
        if constexpr (TH) ring[NF - 1][slot][sc] = pull_U<S, R, BIG>(a, src, psi);
      }
      __syncthreads();
      if (interior) {
        const int m = (j - 1) & 3, c0 = j & 3, pp = (j + 1) & 3;
        auto rows = [&](int f) { return Rows3<R>{ring[f][m], ring[f][c0], ring[f][pp]}; };
        site_update<S, R, TH>(a, d, srcj, in, hC, gC, poC, rows(0), rows(1), rows(2), rows(3),
                              sc, rows(NF - 1));
      }
#pragma unroll
      for (int i = 0; i < 9; ++i) hC[i] = hL[i];
#pragma unroll
      for (int i = 0; i < 5; ++i) gC[i] = gL[i];
      poC = poL;
    }
    __syncthreads();
  }
}

template <typename S, typename R, bool BIG, bool TH = false>
__global__ void __launch_bounds__(YM_THREADS, sizeof(R) == 4 ? (TH ? 3 : 4) : 2)
    k_step_ymarch(StepArgs<S, R> a) {
  __shared__ R ring[TH ? 5 : 4][4][YM_W + 2];  // [phi, psi, vx_o, vy_o (, U)][slot][column]
  ymarch_tiles<S, R, BIG, TH>(a, ring);
}

// All steps of a call in one launch: the device's resident CTAs march the
// tiles of every domain, meet at a grid-wide barrier, swap the two state
// buffers and go on with the next step.  Launched cooperatively (every CTA
// resident), so the barrier always completes; the fields are written on the
// last step only.
template <typename S, typename R, bool BIG, bool TH = false>
__global__ void __launch_bounds__(YM_THREADS, sizeof(R) == 4 ? (TH ? 3 : 4) : 2)
    k_step_ymarch_steps(StepArgs<S, R> a, int nsteps, int* ctr) {
  __shared__ R ring[TH ? 5 : 4][4][YM_W + 2];
  cg::grid_group grid = cg::this_grid();
  R* fields = a.fields;
  for (int step = 0; step < nsteps; ++step) {
    // tile counters: ctr[step & 1] counts this step's tiles (zeroed by the
    // host for step 0, by this CTA one step ahead otherwise); no CTA touches
    // ctr[(step + 1) & 1] until every CTA has passed the barrier below
    if (blockIdx.x == 0 && threadIdx.x == 0) ctr[(step + 1) & 1] = 0;
    StepArgs<S, R> b = a;
    if (step & 1) {
      b.in = a.out;
      b.ain = a.aout;
      b.out = const_cast<S*>(a.in);
      b.aout = const_cast<R*>(a.ain);
    }
    b.fields = step + 1 == nsteps ? fields : nullptr;
    ymarch_tiles<S, R, BIG, TH, true>(b, ring, ctr + (step & 1));
    if (step + 1 < nsteps) grid.sync();
  }
}

// Buffers of more than 2^32 elements (plane stride x 33 population planes)
// take the 64-bit plane-base addressing of the pull helpers.
inline bool big_handle(long long plane_stride, bool thermal) {
  return (unsigned long long)plane_stride * (thermal ? N_POP_TH : N_POP) >= (1ull << 32);
}

template <typename S, typename R, bool BIG>
static void launch_traversal(const StepArgs<S, R>& a, int variant, int tx, int ty, int grid,
                             cudaStream_t st) {
  if (variant == STEP_YMARCH) {
    if constexpr (sizeof(S) == sizeof(R)) {
      if (a.thermal) {
        k_step_ymarch<S, R, BIG, true><<<grid, YM_THREADS, 0, st>>>(a);
        return;
      }
    }
    k_step_ymarch<S, R, BIG><<<grid, YM_THREADS, 0, st>>>(a);
  } else {
    const size_t smem = 4 * (size_t)(tx + 2) * (ty + 2) * sizeof(R);
    k_step_tile<S, R, BIG><<<grid, dim3(tx, ty), smem, st>>>(a);
  }
}

template <typename S, typename R>
cudaError_t launch_step(const StepArgs<S, R>& a, int variant, int tx, int ty, int grid,
                        cudaStream_t st) {
  if (variant == STEP_STAGED) return launch_step_staged<S, R>(a, grid, st);
  if (variant == STEP_YMARCH && a.bc)
    return launch_ymarch_bc<S, R>(a, big_handle(a.plane_stride, a.thermal != 0), grid, st);
  if (big_handle(a.plane_stride, a.thermal != 0))
    launch_traversal<S, R, true>(a, variant, tx, ty, grid, st);
  else launch_traversal<S, R, false>(a, variant, tx, ty, grid, st);
  return cudaGetLastError();
}

// All n steps in one cooperative launch of the resident grid (y-march,
// periodic domains).  grid <= SMs x ymarch_steps_blocks_per_sm.
template <typename S, typename R, bool BIG>
static cudaError_t launch_steps_t(const StepArgs<S, R>& a, int nsteps, int* ctr, int grid,
                                  cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(ctr, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<StepArgs<S, R>*>(&a), &nsteps, &ctr};
  if constexpr (sizeof(S) == sizeof(R)) {
    if (a.thermal)
      return cudaLaunchCooperativeKernel((const void*)k_step_ymarch_steps<S, R, BIG, true>,
                                         grid, YM_THREADS, args, 0, st);
  }
  return cudaLaunchCooperativeKernel((const void*)k_step_ymarch_steps<S, R, BIG, false>, grid,
                                     YM_THREADS, args, 0, st);
}

template <typename S, typename R>
cudaError_t launch_ymarch_steps(const StepArgs<S, R>& a, int nsteps, int* ctr, int grid,
                                cudaStream_t st) {
  if (a.bc) return cudaErrorInvalidValue;
  return big_handle(a.plane_stride, a.thermal != 0)
             ? launch_steps_t<S, R, true>(a, nsteps, ctr, grid, st)
             : launch_steps_t<S, R, false>(a, nsteps, ctr, grid, st);
}

template <typename S, typename R, bool BIG>
static int steps_blocks_t(bool thermal) {
  int n = 0;
  if constexpr (sizeof(S) == sizeof(R)) {
    if (thermal) {
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_ymarch_steps<S, R, BIG, true>,
                                                    YM_THREADS, 0);
      return n > 0 ? n : 1;
    }
  }
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_ymarch_steps<S, R, BIG, false>,
                                                YM_THREADS, 0);
  return n > 0 ? n : 1;
}

template <typename S, typename R>
int ymarch_steps_blocks_per_sm(long long plane_stride, bool thermal) {
  return big_handle(plane_stride, thermal) ? steps_blocks_t<S, R, true>(thermal)
                                           : steps_blocks_t<S, R, false>(thermal);
}

template <typename S, typename R, bool BIG>
static int traversal_blocks_per_sm(int variant, int tx, int ty, bool thermal) {
  int n = 0;
  if (variant == STEP_YMARCH && thermal) {
    if constexpr (sizeof(S) == sizeof(R))
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_ymarch<S, R, BIG, true>,
                                                    YM_THREADS, 0);
  } else if (variant == STEP_YMARCH)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_ymarch<S, R, BIG>, YM_THREADS, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_tile<S, R, BIG>, tx * ty,
                                                  4 * (size_t)(tx + 2) * (ty + 2) * sizeof(R));
  return n > 0 ? n : 1;
}

template <typename S, typename R>
int step_blocks_per_sm(int variant, int tx, int ty, long long plane_stride, bool thermal,
                       bool bc) {
  if (variant == STEP_STAGED) return staged_blocks_per_sm<S, R>();
  if (variant == STEP_YMARCH && bc)
    return ymarch_bc_blocks_per_sm<S, R>(big_handle(plane_stride, thermal), thermal);
  return big_handle(plane_stride, thermal)
             ? traversal_blocks_per_sm<S, R, true>(variant, tx, ty, thermal)
             : traversal_blocks_per_sm<S, R, false>(variant, tx, ty, thermal);
}

#define PF_STEPS_INST(S, R)                                                                   \
  template cudaError_t launch_ymarch_steps<S, R>(const StepArgs<S, R>&, int, int*, int,       \
                                                 cudaStream_t);                                \
  template int ymarch_steps_blocks_per_sm<S, R>(long long, bool);
PF_STEPS_INST(double, double)
PF_STEPS_INST(float, float)
PF_STEPS_INST(__half, float)
PF_STEPS_INST(__nv_bfloat16, float)

template int step_blocks_per_sm<double, double>(int, int, int, long long, bool, bool);
template int step_blocks_per_sm<float, float>(int, int, int, long long, bool, bool);
template int step_blocks_per_sm<__half, float>(int, int, int, long long, bool, bool);
template int step_blocks_per_sm<__nv_bfloat16, float>(int, int, int, long long, bool, bool);

template cudaError_t launch_step<double, double>(const StepArgs<double, double>&, int, int, int,
                                                int, cudaStream_t);
template cudaError_t launch_step<float, float>(const StepArgs<float, float>&, int, int, int, int,
                                              cudaStream_t);
template cudaError_t launch_step<__half, float>(const StepArgs<__half, float>&, int, int, int,
                                               int, cudaStream_t);
template cudaError_t launch_step<__nv_bfloat16, float>(const StepArgs<__nv_bfloat16, float>&,
                                                      int, int, int, int, cudaStream_t);

}  // namespace pf
