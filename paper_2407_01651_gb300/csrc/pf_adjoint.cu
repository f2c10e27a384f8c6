// pf_adjoint.cu -- discrete adjoint of one coupled LB step (reverse mode), for
// gradients of a final-state objective with respect to the anisotropy
// strength eps_s, the undercooling Omega and the surface tension sigma.
//
// One reverse step maps lambda_{t+1} (the adjoint of the stored state after
// step t+1) to lambda_t, given the state x_t:
//   k_adj_local    per site: rebuild the step's inputs at the site from x_t
//                  (pull, stencils from a shared-memory halo), run the
//                  hand-written reverse of the site update (pf_local.cuh) and
//                  store the adjoints of its inputs (43 planes); accumulate
//                  the parameter adjoints per block.
//   k_adj_transpose transpose the isotropic stencils (adjoints of the phi,
//                  psi and lagged-velocity fields, phi and psi on a tile with
//                  a one-site ring in shared memory), the streaming (a gather
//                  from x + c_i) and the a_s^2 time stretch of the dendrite
//                  lattice: lambda_t.
// Adjoint planes are in the compute precision.  The FP32 and FP64 storage
// forms are supported.
#include "pf_local.cuh"
#include "pf_pull.cuh"

namespace pf {

namespace {

__device__ constexpr int CX9[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__device__ constexpr int CY9[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

template <typename R>
__device__ __forceinline__ local::Coef<R> make_coef(const KParams<R>& kp, const DomDesc& d,
                                                    double2 cs) {
  local::Coef<R> c;
  c.rho_g = kp.rho_g; c.drho = kp.drho; c.ge2 = kp.ge2; c.gat2 = kp.gat2; c.kappa = kp.kappa;
  c.fs_coef = kp.fs_coef; c.Wphi2 = kp.Wphi2; c.M_phi = kp.M_phi; c.two_bphi = kp.two_bphi;
  c.two_bint = kp.two_bint; c.four_bpsi = kp.four_bpsi; c.lam = kp.lam; c.theta = kp.theta;
  c.Mcinf = kp.Mcinf; c.inv_tau0 = kp.inv_tau0; c.c_s1 = kp.c_s1; c.W0 = kp.W0; c.a_at = kp.a_at;
  c.k = kp.k; c.D = kp.D; c.g = kp.g; c.s_e = kp.s_e; c.s_eps = kp.s_eps; c.s_q = kp.s_q;
  c.s_nu = kp.s_nu; c.s_phi = kp.s_phi;
  c.eps = static_cast<R>(d.eps_s);
  c.ct = static_cast<R>(cs.x);
  c.sn = static_cast<R>(cs.y);
  c.rho_bar = static_cast<R>(d.rho_bar);
  return c;
}

}  // namespace

// ---------------------------------------------------------------------------
template <typename S, typename R, bool BIG>
__global__ void __launch_bounds__(256, 2) k_adj_local(AdjArgs<S, R> a) {
  __shared__ R sphi[ADJ_TY + 2][ADJ_TX + 2], spsi[ADJ_TY + 2][ADJ_TX + 2];
  __shared__ R svx[ADJ_TY + 2][ADJ_TX + 2], svy[ADJ_TY + 2][ADJ_TX + 2];
  __shared__ R red[3][256];
  const StepArgs<S, R>& st = a.step;
  const DomDesc d = a.dom;
  const long long ps = st.plane_stride;
  const int tid = threadIdx.y * ADJ_TX + threadIdx.x;
  const int tiles_x = (d.nx + ADJ_TX - 1) / ADJ_TX;
  const int ntiles = tiles_x * ((d.ny + ADJ_TY - 1) / ADJ_TY);
  R pe = R(0), po = R(0), psg = R(0);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int x0 = (tile % tiles_x) * ADJ_TX, y0 = (tile / tiles_x) * ADJ_TY;
    // Each thread pulls its own site once (kept in registers for the
    // reverse) and stores phi, psi and the lagged velocity in the tile; 84
    // threads then pull the one-site ring around it.  Positions beyond a
    // ragged edge hold the periodic images their neighbours read.
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const bool inside = x < d.nx && y < d.ny;
    local::In<R> in;
    Src9 src;
    {
      R phi, psi;
      src = sources(d, x % d.nx, y % d.ny);
      pull_hg<S, R, BIG>(st, src, in.h, in.g, phi, psi, in.psio);
      sphi[threadIdx.y + 1][threadIdx.x + 1] = phi;
      spsi[threadIdx.y + 1][threadIdx.x + 1] = psi;
      svx[threadIdx.y + 1][threadIdx.x + 1] = ld<R>(st.ain + A_VXO * ps, src.s[0]);
      svy[threadIdx.y + 1][threadIdx.x + 1] = ld<R>(st.ain + A_VYO * ps, src.s[0]);
    }
    if (tid < 2 * (ADJ_TX + 2) + 2 * ADJ_TY) {
      int lx, ly;
      if (tid < ADJ_TX + 2) { lx = tid; ly = 0; }
      else if (tid < 2 * (ADJ_TX + 2)) { lx = tid - (ADJ_TX + 2); ly = ADJ_TY + 1; }
      else if (tid < 2 * (ADJ_TX + 2) + ADJ_TY) { lx = 0; ly = tid - 2 * (ADJ_TX + 2) + 1; }
      else { lx = ADJ_TX + 1; ly = tid - 2 * (ADJ_TX + 2) - ADJ_TY + 1; }
      int gx = x0 + lx - 1, gy = y0 + ly - 1;
      gx = ((gx % d.nx) + d.nx) % d.nx;
      gy = ((gy % d.ny) + d.ny) % d.ny;
      R h[9], g[5], phi, psi, pso;
      const Src9 hs = sources(d, gx, gy);
      pull_hg<S, R, BIG>(st, hs, h, g, phi, psi, pso);
      sphi[ly][lx] = phi;
      spsi[ly][lx] = psi;
      svx[ly][lx] = ld<R>(st.ain + A_VXO * ps, hs.s[0]);
      svy[ly][lx] = ld<R>(st.ain + A_VYO * ps, hs.s[0]);
    }
    __syncthreads();
    if (inside) {
      SiteIn<R> si;
      load_site<S, R, BIG>(st, src, si);
      for (int i = 0; i < 9; ++i) in.f[i] = si.f[i];
      for (int i = 0; i < 5; ++i) in.s[i] = si.s[i];
      in.phio = si.phio;
      in.Co = si.Co;
      in.Qo = si.Qo;
      const int cx = threadIdx.x + 1, cy = threadIdx.y + 1;
      in.vxo = svx[cy][cx];
      in.vyo = svy[cy][cx];
      const R w1 = R(1.0 / 9.0), w2 = R(1.0 / 36.0);
      auto grad = [&](R (*X)[ADJ_TX + 2], R& gx, R& gy) {
        const R X0 = X[cy][cx];
        const R e = X[cy][cx + 1] - X0, w = X[cy][cx - 1] - X0;
        const R n = X[cy + 1][cx] - X0, so = X[cy - 1][cx] - X0;
        const R ne = X[cy + 1][cx + 1] - X0, nw = X[cy + 1][cx - 1] - X0;
        const R sw = X[cy - 1][cx - 1] - X0, se = X[cy - 1][cx + 1] - X0;
        gx = R(3) * (w1 * (e - w) + w2 * ((ne - sw) + (se - nw)));
        gy = R(3) * (w1 * (n - so) + w2 * ((ne - sw) + (nw - se)));
      };
      grad(sphi, in.gpx, in.gpy);
      grad(spsi, in.gsx, in.gsy);
      grad(svx, in.dvxx, in.dvxy);
      grad(svy, in.dvyx, in.dvyy);
      {
        const R X0 = sphi[cy][cx];
        const R ax = ((sphi[cy][cx + 1] - X0) + (sphi[cy][cx - 1] - X0)) +
                     ((sphi[cy + 1][cx] - X0) + (sphi[cy - 1][cx] - X0));
        const R dg = ((sphi[cy + 1][cx + 1] - X0) + (sphi[cy - 1][cx - 1] - X0)) +
                     ((sphi[cy + 1][cx - 1] - X0) + (sphi[cy - 1][cx + 1] - X0));
        in.lphi = R(6) * (w1 * ax + w2 * dg);
      }
      const local::Coef<R> c = make_coef(st.kp, d, st.grain_cs[d.grain_off + si.gid]);
      // output adjoints of the site (39 physical planes)
      const long long site = src.s[0];
      const R* L = a.lam_in;
      local::Out<R> ao;
      for (int i = 0; i < 9; ++i) {
        ao.f[i] = L[(0 + i) * ps + site];
        ao.h[i] = L[(9 + i) * ps + site];
      }
      for (int i = 0; i < 5; ++i) {
        ao.gpre[i] = L[(18 + i) * ps + site];
        ao.gpost[i] = L[(23 + i) * ps + site];
        ao.s[i] = L[(29 + i) * ps + site];
      }
      ao.rr = L[28 * ps + site];
      ao.phi = L[34 * ps + site];
      ao.C = L[35 * ps + site];
      ao.vx = L[36 * ps + site];
      ao.vy = L[37 * ps + site];
      ao.Q = L[38 * ps + site];
      ao.U = ao.p = ao.mu = R(0);
      local::In<R> ai;
      local::ParGrad<R> pg{R(0), R(0), R(0)};
      local::reverse(in, c, static_cast<R>(a.dfs_dsigma), ao, ai, pg);
      pe += pg.eps;
      po += pg.Omega;
      psg += pg.sigma;
      R* A = a.ai;
      for (int i = 0; i < 9; ++i) {
        A[(AI_F + i) * ps + site] = ai.f[i];
        A[(AI_H + i) * ps + site] = ai.h[i];
      }
      for (int i = 0; i < 5; ++i) {
        A[(AI_G + i) * ps + site] = ai.g[i];
        A[(AI_S + i) * ps + site] = ai.s[i];
      }
      A[AI_PSIO * ps + site] = ai.psio;
      A[AI_GPX * ps + site] = ai.gpx;
      A[AI_GPY * ps + site] = ai.gpy;
      A[AI_LPHI * ps + site] = ai.lphi;
      A[AI_GSX * ps + site] = ai.gsx;
      A[AI_GSY * ps + site] = ai.gsy;
      A[AI_DVXX * ps + site] = ai.dvxx;
      A[AI_DVXY * ps + site] = ai.dvxy;
      A[AI_DVYX * ps + site] = ai.dvyx;
      A[AI_DVYY * ps + site] = ai.dvyy;
      A[AI_PHIO * ps + site] = ai.phio;
      A[AI_CO * ps + site] = ai.Co;
      A[AI_QO * ps + site] = ai.Qo;
      A[AI_VXO * ps + site] = ai.vxo;
      A[AI_VYO * ps + site] = ai.vyo;
    }
    __syncthreads();
  }
  // block sum of the parameter adjoints, accumulated into this block's record
  red[0][tid] = pe;
  red[1][tid] = po;
  red[2][tid] = psg;
  __syncthreads();
  for (int half = 128; half > 0; half >>= 1) {
    if (tid < half)
      for (int q = 0; q < 3; ++q) red[q][tid] += red[q][tid + half];
    __syncthreads();
  }
  if (tid < 3) a.partial[blockIdx.x * 3 + tid] += static_cast<double>(red[tid][0]);
}

// Transposes of the stencils, the streaming and the a_s^2 time stretch:
// lambda_t from the per-site input adjoints (ai).  One CTA per tile of
// ADJ_TX x ADJ_TY sites.
//
// Stencils: grad X(z) = 3 sum_j w_j c_j X(z + c_j) and
// lap X(z) = 6 sum_{j>0} w_j (X(z + c_j) - X(z)) give
//   adj X(x) = sum_j 3 w_j c_j . adj grad(x - c_j)
//            + sum_{j>0} 6 w_j adj lap(x - c_j) - 6 (1 - w_0) adj lap(x).
// The gather below needs adj phi and adj psi at the site and at its eight
// neighbours, so they are formed for the tile and a one-site ring in shared
// memory first; adj vx_o and adj vy_o are needed at the site only.
//
// Streaming and stretch: g_i(x) = g_pre,i(x) + r(x - c_i) [g_post,i(x - c_i)
// - g_pre,i(x)] and psi_o(x) = sum_i g_pre,i(x).  The population of direction
// q leaving x lands on x + c_q, the source x - c_{opp(q)} of the pull with the
// opposite direction.
template <typename S, typename R>
__global__ void __launch_bounds__(ADJ_TX * ADJ_TY) k_adj_transpose(AdjArgs<S, R> a) {
  constexpr int SX = ADJ_TX + 2, SY = ADJ_TY + 2;
  __shared__ R s_aphi[SY][SX], s_apsi[SY][SX];
  const DomDesc d = a.dom;
  const unsigned ps = (unsigned)a.step.plane_stride;
  const R* __restrict__ A = a.ai;
  const S* __restrict__ P = a.step.in;
  const R* __restrict__ X = a.step.ain;
  R* __restrict__ L = a.lam_out;
  constexpr int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
  const R w[9] = {R(4.0 / 9.0), R(1.0 / 9.0), R(1.0 / 9.0), R(1.0 / 9.0), R(1.0 / 9.0),
                  R(1.0 / 36.0), R(1.0 / 36.0), R(1.0 / 36.0), R(1.0 / 36.0)};
  const int tiles_x = (d.nx + ADJ_TX - 1) / ADJ_TX;
  const int x0 = (blockIdx.x % tiles_x) * ADJ_TX, y0 = (blockIdx.x / tiles_x) * ADJ_TY;
  const int tid = threadIdx.y * ADJ_TX + threadIdx.x;
  // adj phi and adj psi on the tile and its ring (periodic images beyond the
  // domain's edges)
  for (int i = tid; i < SX * SY; i += ADJ_TX * ADJ_TY) {
    const int lx = i % SX, ly = i / SX;
    int gx = x0 + lx - 1, gy = y0 + ly - 1;
    gx = ((gx % d.nx) + d.nx) % d.nx;
    gy = ((gy % d.ny) + d.ny) % d.ny;
    const Src9 src = sources(d, gx, gy);   // src.s[j] = z - c_j
    R aphi = R(-6) * (R(1) - w[0]) * __ldg(plane(A, AI_LPHI, ps) + src.s[0]);
    R apsi = R(0);
#pragma unroll
    for (int j = 1; j < 9; ++j) {
      const unsigned z = src.s[j];
      const R wx = R(3) * w[j] * R(CX9[j]), wy = R(3) * w[j] * R(CY9[j]);
      aphi += wx * __ldg(plane(A, AI_GPX, ps) + z) + wy * __ldg(plane(A, AI_GPY, ps) + z) +
              R(6) * w[j] * __ldg(plane(A, AI_LPHI, ps) + z);
      apsi += wx * __ldg(plane(A, AI_GSX, ps) + z) + wy * __ldg(plane(A, AI_GSY, ps) + z);
    }
    s_aphi[ly][lx] = aphi;
    s_apsi[ly][lx] = apsi;
  }
  // the site's gathers that need no shared value are issued (and the planes
  // they complete stored) before the barrier, so that their latency overlaps
  // the wait for the ring
  const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
  const bool valid = x < d.nx && y < d.ny;
  const int cx = threadIdx.x + 1, cy = threadIdx.y + 1;
  const Src9 src = sources(d, valid ? x : 0, valid ? y : 0);
  const unsigned site = src.s[0];
  R hraw[9], gown[5], gdst[5], rsrc[5], gdiff[5], rr_own = R(0), apsio = R(0);
  if (valid) {
    R avx = __ldg(plane(A, AI_VXO, ps) + site), avy = __ldg(plane(A, AI_VYO, ps) + site);
#pragma unroll
    for (int j = 1; j < 9; ++j) {
      const unsigned z = src.s[j];
      const R wx = R(3) * w[j] * R(CX9[j]), wy = R(3) * w[j] * R(CY9[j]);
      avx += wx * __ldg(plane(A, AI_DVXX, ps) + z) + wy * __ldg(plane(A, AI_DVXY, ps) + z);
      avy += wx * __ldg(plane(A, AI_DVYX, ps) + z) + wy * __ldg(plane(A, AI_DVYY, ps) + z);
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      const unsigned t = src.s[OPP[q]];   // x + c_q
      plane(L, 0 + q, ps)[site] = __ldg(plane(A, AI_F + q, ps) + t);
      hraw[q] = __ldg(plane(A, AI_H + q, ps) + t);
    }
    rr_own = __ldg(plane(X, A_RR, ps) + site);
    apsio = __ldg(plane(A, AI_PSIO, ps) + site);
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const unsigned t = src.s[OPP[q]];   // destination of q
      const unsigned sq = src.s[q];       // source of q
      plane(L, 29 + q, ps)[site] = __ldg(plane(A, AI_S + q, ps) + t);
      gown[q] = __ldg(plane(A, AI_G + q, ps) + site);
      gdst[q] = __ldg(plane(A, AI_G + q, ps) + t);
      rsrc[q] = __ldg(plane(X, A_RR, ps) + sq);
      gdiff[q] = ld<R>(plane(P, P_GPOST + q, ps), site) - ld<R>(plane(P, P_GPRE + q, ps), t);
    }
    plane(L, 34, ps)[site] = __ldg(plane(A, AI_PHIO, ps) + site);
    plane(L, 35, ps)[site] = __ldg(plane(A, AI_CO, ps) + site);
    plane(L, 36, ps)[site] = avx;
    plane(L, 37, ps)[site] = avy;
    plane(L, 38, ps)[site] = __ldg(plane(A, AI_QO, ps) + site);
  }
  __syncthreads();
  if (!valid) return;
#pragma unroll
  for (int q = 0; q < 9; ++q)
    plane(L, 9 + q, ps)[site] = hraw[q] + s_aphi[cy + CY9[q]][cx + CX9[q]];
  const R as1 = s_apsi[cy][cx];
  R lrr = R(0);
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const R ag_own = gown[q] + as1;
    const R ag_dst = gdst[q] + s_apsi[cy + CY9[q]][cx + CX9[q]];
    plane(L, 18 + q, ps)[site] = ag_own * (R(1) - rsrc[q]) + apsio;
    plane(L, 23 + q, ps)[site] = ag_dst * rr_own;
    lrr += ag_dst * gdiff[q];
  }
  plane(L, 28, ps)[site] = lrr;
}

// Adjoint of the final-state objective
//   J = w_s mean h(psi_T) + w_c y_c(T) / L_y,  y_c = sum y (1 - phi) / sum (1 - phi),
// with psi_T = sum g_pre and phi_T the stored lagged phi of x_T.
template <typename R>
__global__ void k_adj_objective(R* __restrict__ L, DomDesc d, long long ps, double w_s,
                                double w_c, double yc, double gas) {
  const long long n = (long long)d.nx * d.ny;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long site = d.off + i;
    const double y = (double)(i / d.nx);
    for (int q = 0; q < N_PHYS; ++q) L[q * ps + site] = R(0);
    for (int q = 0; q < 5; ++q) L[(18 + q) * ps + site] = static_cast<R>(0.5 * w_s / (double)n);
    L[34 * ps + site] = static_cast<R>(w_c * (yc - y) / (gas * (double)d.ny));
  }
}

// Initial-condition term of d J / d Omega: the initial lagged Q_psi is
// Q(phi0, psi0, U0), whose Omega-derivative is lambda' (1-psi0^2)^2 (1 + (1-k) U0)
// (d theta_sys / d Omega = -1, d M c_inf / d Omega = -(1-k)).
template <typename S, typename R>
__global__ void k_adj_omega_init(const R* __restrict__ L, const S* __restrict__ P,
                                 const R* __restrict__ X, DomDesc d, long long ps, double lam,
                                 double k, double* __restrict__ partial) {
  __shared__ double red[256];
  const long long n = (long long)d.nx * d.ny;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long site = d.off + i;
    double psi = 0.0;
    for (int q = 0; q < 5; ++q) psi += (double)ld<R>(P + (P_GPRE + q) * ps, site);
    const double C = (double)X[A_CO * ps + site];
    const double U = (2.0 * C / (1.0 + k - (1.0 - k) * psi) - 1.0) / (1.0 - k);
    const double om = 1.0 - psi * psi;
    acc += (double)L[38 * ps + site] * lam * om * om * (1.0 + (1.0 - k) * U);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int half = blockDim.x / 2; half > 0; half >>= 1) {
    if ((int)threadIdx.x < half) red[threadIdx.x] += red[threadIdx.x + half];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// ---------------------------------------------------------------------------
template <typename S, typename R>
cudaError_t launch_adjoint_step(const AdjArgs<S, R>& a, int grid, cudaStream_t st) {
  if ((unsigned long long)a.step.plane_stride * N_POP >= (1ull << 32))
    k_adj_local<S, R, true><<<grid, dim3(ADJ_TX, ADJ_TY), 0, st>>>(a);
  else
    k_adj_local<S, R, false><<<grid, dim3(ADJ_TX, ADJ_TY), 0, st>>>(a);
  const int tiles = ((a.dom.nx + ADJ_TX - 1) / ADJ_TX) * ((a.dom.ny + ADJ_TY - 1) / ADJ_TY);
  k_adj_transpose<S, R><<<tiles, dim3(ADJ_TX, ADJ_TY), 0, st>>>(a);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_adj_objective(R* lam, DomDesc d, long long ps, double w_s, double w_c,
                                 double yc, double gas, cudaStream_t st) {
  const long long n = (long long)d.nx * d.ny;
  const int g = (int)std::min<long long>((n + 255) / 256, 4096);
  k_adj_objective<R><<<g, 256, 0, st>>>(lam, d, ps, w_s, w_c, yc, gas);
  return cudaGetLastError();
}

template <typename S, typename R>
cudaError_t launch_adj_omega_init(const R* lam, const S* pop, const R* aux, DomDesc d,
                                  long long ps, double lam_p, double k, double* partial,
                                  int blocks, cudaStream_t st) {
  k_adj_omega_init<S, R><<<blocks, 256, 0, st>>>(lam, pop, aux, d, ps, lam_p, k, partial);
  return cudaGetLastError();
}

template cudaError_t launch_adjoint_step<double, double>(const AdjArgs<double, double>&, int,
                                                        cudaStream_t);
template cudaError_t launch_adjoint_step<float, float>(const AdjArgs<float, float>&, int,
                                                      cudaStream_t);
template cudaError_t launch_adj_objective<double>(double*, DomDesc, long long, double, double,
                                                  double, double, cudaStream_t);
template cudaError_t launch_adj_objective<float>(float*, DomDesc, long long, double, double,
                                                 double, double, cudaStream_t);
template cudaError_t launch_adj_omega_init<double, double>(const double*, const double*,
                                                          const double*, DomDesc, long long,
                                                          double, double, double*, int,
                                                          cudaStream_t);
template cudaError_t launch_adj_omega_init<float, float>(const float*, const float*,
                                                        const float*, DomDesc, long long,
                                                        double, double, double*, int,
                                                        cudaStream_t);

}  // namespace pf
