// pf_step_staged.cu -- k_step_staged: the coupled LB step (arXiv 2407.01651)
// as a y-marched column strip whose input rows are staged in shared memory by
// the bulk-copy (TMA) engine a few rows ahead of the arithmetic.
//
// The arithmetic per site is the one of every other traversal (pf_site.cuh);
// what differs is how the inputs reach it.  Every plane that a site reads at
// its neighbours (f, h, g_post, s and r = 1/a_s^2; in the 16-bit forms also
// the lagged phi, C, psi that decode the neighbours' offsets) is copied row by
// row with cp.async.bulk into a ring of NSLOT row slots, each completing on
// its own mbarrier.  Planes that only the site itself reads (g_pre, the lagged
// velocity, Q_psi, the grain id; phi_o and C_o in FP32/FP64) are loaded into
// registers one row ahead of their use.  So no warp waits on HBM inside the
// arithmetic of a row: the copies of row j+4 are in flight while row j is
// computed.
//
// Row slots: with NSLOT = 6, iteration j (the update of row j and the
// streaming of row j+1) reads rows j-1 .. j+2; row j+3 and j+4 are in flight.
// Each slot row holds, per staged plane, the strip's interior columns plus
// 16 bytes of halo on each side (the two copies of the halo wrap around the
// periodic x boundary on their own).  Requirements (checked on the host):
// nx a multiple of 16 / sizeof(storage) and of 16 / sizeof(compute), and
// 16-byte aligned plane bases.
#include "pf_site.cuh"

namespace pf {

namespace {

template <typename S, typename R>
struct Stage {
  static constexpr int HS = 16 / (int)sizeof(S);   // halo columns of a storage plane
  static constexpr int HR = 16 / (int)sizeof(R);   // halo columns of a compute plane
  static constexpr int PWS = YM_W + 2 * HS;        // staged width, storage planes
  static constexpr int PWR = YM_W + 2 * HR;        // staged width, compute planes
  static constexpr int NPS = 28;                   // f[9], h[9], g_post[5], s[5]
  static constexpr bool OFF = Codec<S>::kOffset;
  static constexpr int NAS = OFF ? 4 : 1;          // r (+ phi_o, C_o, psi_o)
  static constexpr int POP_BYTES = NPS * PWS * (int)sizeof(S);
  static constexpr int SLOT_BYTES = POP_BYTES + NAS * PWR * (int)sizeof(R);
  static constexpr int NSLOT = 6;
  static constexpr int RW = YM_W + 2;
  static constexpr int RING_BYTES = 4 * 4 * RW * (int)sizeof(R);
  static constexpr int SMEM = NSLOT * SLOT_BYTES + RING_BYTES + NSLOT * 8;
  static constexpr int MIN_BLOCKS = sizeof(S) == 8 ? 1 : (sizeof(S) == 4 ? 2 : 3);
  static_assert(POP_BYTES % 16 == 0 && SLOT_BYTES % 16 == 0, "16-byte staged planes");
  static_assert(HS >= 2 && HR >= 2, "the halo streaming reaches two columns out");
};

// staged aux planes
constexpr int U_RR = 0, U_PHIO = 1, U_CO = 2, U_PSIO = 3;
__device__ __forceinline__ int aux_plane(int u) {
  return u == U_RR ? A_RR : (u == U_PHIO ? A_PHIO : (u == U_CO ? A_CO : A_PSIO));
}
// staged storage plane q -> population plane (f, h, then g_post, s)
__device__ __forceinline__ int pop_plane(int q) { return q < 18 ? q : q + 5; }

// ---- mbarrier and bulk copy (PTX) ----
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void bar_init(unsigned bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void bar_expect(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool bar_try(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for the phase of `bar` with parity `parity`; gives up after about one
// second (or 2^24 polls) and returns false.
__device__ __forceinline__ bool bar_wait(unsigned bar, unsigned parity) {
  if (bar_try(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  for (unsigned it = 0; it < (1u << 24); ++it) {
    if (bar_try(bar, parity)) return true;
    if ((it & 255u) == 255u && globaltimer() - t0 > 1000000000ull) break;
  }
  return false;
}
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes,
                                         unsigned bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// Copy one staged plane row: columns [x0 - H, x0 + w + H) of the strip, the
// halos wrapping around the periodic x boundary.  A strip away from both x
// boundaries is one contiguous piece.
template <typename E>
__device__ __forceinline__ void copy_plane_row(unsigned dst, const E* src, int x0, int w, int nx,
                                               int H, unsigned bar) {
  const bool wl = x0 == 0, wr = x0 + w == nx;
  const unsigned hb = (unsigned)(H * sizeof(E)), wb = (unsigned)(w * sizeof(E));
  if (!wl && !wr) {
    bulk_g2s(dst, src + x0 - H, wb + 2 * hb, bar);
  } else if (!wr) {
    bulk_g2s(dst, src + nx - H, hb, bar);
    bulk_g2s(dst + hb, src + x0, wb + hb, bar);
  } else if (!wl) {
    bulk_g2s(dst, src + x0 - H, hb + wb, bar);
    bulk_g2s(dst + hb + wb, src, hb, bar);
  } else {
    bulk_g2s(dst, src + nx - H, hb, bar);
    bulk_g2s(dst + hb, src + x0, wb, bar);
    bulk_g2s(dst + hb + wb, src, hb, bar);
  }
}

// Issue the copies of one strip row (global row gy) into a slot; called by
// every thread of the CTA.  Thread 0 announces the byte count on the slot's
// mbarrier; staged plane q is copied by lane q / 5 of warp q % 5, so that the
// issue of the bulk copies is spread over the warps.
template <typename S, typename R>
__device__ __forceinline__ void issue_row(const StepArgs<S, R>& a, const DomDesc& d, int gy,
                                          int x0, int w, unsigned char* slot, unsigned bar,
                                          int t) {
  using G = Stage<S, R>;
  constexpr int NW = YM_THREADS / 32;
  if (a.drop_copies) return;   // testing only: the waits on this row time out
  if (t == 0) {
    const unsigned bytes =
        G::NPS * (w + 2 * G::HS) * sizeof(S) + G::NAS * (w + 2 * G::HR) * sizeof(R);
    bar_expect(bar, bytes);
  }
  const int q = (t & 31) * NW + (t >> 5);
  if (q >= G::NPS + G::NAS) return;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  const unsigned ps = (unsigned)a.plane_stride;
  const unsigned row = (unsigned)d.off + (unsigned)gy * (unsigned)d.nx;
  if (q < G::NPS) {
    copy_plane_row<S>(smem_u32(slot + q * G::PWS * sizeof(S)),
                      plane(a.in, pop_plane(q), ps) + row, x0, w, d.nx, G::HS, bar);
  } else {
    const int u = q - G::NPS;
    copy_plane_row<R>(smem_u32(slot + G::POP_BYTES + u * G::PWR * sizeof(R)),
                      plane(a.ain, aux_plane(u), ps) + row, x0, w, d.nx, G::HR, bar);
  }
}

// One staged row slot seen from a thread.
template <typename S, typename R>
struct SlotView {
  const S* pop;
  const R* aux;
  __device__ __forceinline__ S p(int q, int dx) const {
    return pop[q * Stage<S, R>::PWS + dx + Stage<S, R>::HS];
  }
  __device__ __forceinline__ R x(int u, int dx) const {
    return aux[u * Stage<S, R>::PWR + dx + Stage<S, R>::HR];
  }
};

template <typename S, typename R>
__device__ __forceinline__ SlotView<S, R> slot_view(unsigned char* slots, int s) {
  unsigned char* b = slots + s * Stage<S, R>::SLOT_BYTES;
  return {reinterpret_cast<const S*>(b), reinterpret_cast<const R*>(b + Stage<S, R>::POP_BYTES)};
}

template <typename S, typename R>
__device__ __forceinline__ R dec(S v) {
  return Codec<S>::template dec<R>(v);
}
template <typename S, typename R>
__device__ __forceinline__ R dec_ns(S v) {
  if constexpr (Codec<S>::kOffset) return dec<S, R>(v) * R(kNSInvScale);
  else return dec<S, R>(v);
}

// Source row of D2Q9 direction i: row - cy_i, as 0 (row-1), 1 (row), 2 (row+1).
__device__ __forceinline__ constexpr int src_row(int i) {
  return (i == 2 || i == 5 || i == 6) ? 0 : ((i == 4 || i == 7 || i == 8) ? 2 : 1);
}
// Source column offset of direction i: -cx_i.
__device__ __forceinline__ constexpr int src_dx(int i) {
  return (i == 1 || i == 5 || i == 8) ? -1 : ((i == 3 || i == 6 || i == 7) ? 1 : 0);
}

// Own-site inputs of the streaming of one row (loaded a row ahead).
template <typename S, typename R>
struct OwnHG {
  S gpre[5];
  R vxo, vyo;
};
// Own-site inputs of the update of one row (loaded a row ahead).
template <typename S, typename R>
struct OwnSite {
  R phio, Co, Qo;
  uint8_t gid;
};

template <typename S, typename R>
__device__ __forceinline__ void load_own_hg(const StepArgs<S, R>& a, unsigned site, OwnHG<S, R>& o) {
  const unsigned ps = (unsigned)a.plane_stride;
#pragma unroll
  for (int i = 0; i < 5; ++i) o.gpre[i] = __ldg(plane(a.in, P_GPRE + i, ps) + site);
  o.vxo = __ldg(plane(a.ain, A_VXO, ps) + site);
  o.vyo = __ldg(plane(a.ain, A_VYO, ps) + site);
}
template <typename S, typename R>
__device__ __forceinline__ void load_own_site(const StepArgs<S, R>& a, unsigned site,
                                              OwnSite<S, R>& o) {
  const unsigned ps = (unsigned)a.plane_stride;
  if constexpr (!Codec<S>::kOffset) {
    o.phio = __ldg(plane(a.ain, A_PHIO, ps) + site);
    o.Co = __ldg(plane(a.ain, A_CO, ps) + site);
  }
  o.Qo = __ldg(plane(a.ain, A_QO, ps) + site);
  o.gid = __ldg(a.grain + site);
}

// Streamed h and g of the site at column offset dx of the middle row of
// (rm, rc, rp), from the staged rows; same arithmetic as pull_hg.
template <typename S, typename R>
__device__ __forceinline__ void stream_hg(const SlotView<S, R> (&rows)[3], int dx,
                                          const OwnHG<S, R>& own, R h[9], R g[5], R& phi,
                                          R& psi, R& psio) {
  constexpr bool off = Codec<S>::kOffset;
  CSum<R> sh;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const SlotView<S, R>& r = rows[src_row(i)];
    const int sx = dx + src_dx(i);
    h[i] = dec_off<S, R>(r.p(9 + i, sx), off ? w9<R>(i) * r.x(U_PHIO, sx) : R(0));
    sh.add(h[i]);
  }
  phi = sh.value();
  CSum<R> sg;
  R po = R(0);
  const R psio_own = off ? rows[1].x(U_PSIO, dx) : R(0);
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const SlotView<S, R>& r = rows[src_row(i)];
    const int sx = dx + src_dx(i);
    const R gold = dec_off<S, R>(own.gpre[i], w5<R>(i) * psio_own);
    const R gpo = dec_off<S, R>(r.p(18 + i, sx), off ? w5<R>(i) * r.x(U_PSIO, sx) : R(0));
    const R rr = r.x(U_RR, sx);
    g[i] = gold + (gpo - gold) * rr;
    sg.add(g[i]);
    po += gold;
  }
  psi = sg.value();
  psio = off ? psio_own : po;
}

// Streamed f and s and the lagged scalars of the site at column offset dx.
template <typename S, typename R>
__device__ __forceinline__ void site_inputs(const SlotView<S, R> (&rows)[3], int dx,
                                            const OwnSite<S, R>& own, SiteIn<R>& in) {
  constexpr bool off = Codec<S>::kOffset;
#pragma unroll
  for (int i = 0; i < 9; ++i) in.f[i] = dec_ns<S, R>(rows[src_row(i)].p(i, dx + src_dx(i)));
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const SlotView<S, R>& r = rows[src_row(i)];
    const int sx = dx + src_dx(i);
    in.s[i] = dec_off<S, R>(r.p(23 + i, sx), off ? w5<R>(i) * r.x(U_CO, sx) : R(0));
  }
  if constexpr (off) {
    in.phio = rows[1].x(U_PHIO, dx);
    in.Co = rows[1].x(U_CO, dx);
  } else {
    in.phio = own.phio;
    in.Co = own.Co;
  }
  in.Qo = own.Qo;
  in.gid = own.gid;
}

}  // namespace

template <typename S, typename R>
__global__ void __launch_bounds__(YM_THREADS, Stage<S, R>::MIN_BLOCKS)
    k_step_staged(StepArgs<S, R> a) {
  using G = Stage<S, R>;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* slots = smem;
  R(*ring)[4][G::RW] = reinterpret_cast<R(*)[4][G::RW]>(smem + G::NSLOT * G::SLOT_BYTES);
  const unsigned bar0 = smem_u32(smem + G::NSLOT * G::SLOT_BYTES + G::RING_BYTES);
  const int t = threadIdx.x;

  if (t < G::NSLOT) bar_init(bar0 + 8 * t);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();

  unsigned phase = 0;   // bit s: parity of the next completion of slot s
  bool bad = false;     // a copy did not arrive within the time limit

  for (int tile = a.tile_base + blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const DomDesc d = a.doms[a.tile_dom[tile]];
    const int lt = tile - d.tile0;
    const int nx = d.nx, ny = d.ny;
    const int x0 = (lt % d.tiles_x) * YM_W;
    const int ya = (lt / d.tiles_x) * a.chunk;
    const int yb = min(ya + a.chunk, ny);
    const int w = min(YM_W, nx - x0);
    const int k0 = ya - 2;           // first staged row of the tile
    const int klast = yb + 1;        // last staged row of the tile
    bool interior = false, active = false;
    int col = 0, dx = 0;
    if (t < YM_W) {
      interior = active = t < w;
      col = x0 + t;
      dx = t;
    } else if (t == YM_W) {
      active = true;
      col = x0 == 0 ? nx - 1 : x0 - 1;
      dx = -1;
    } else if (t == YM_W + 1) {
      active = true;
      col = x0 + w >= nx ? x0 + w - nx : x0 + w;
      dx = w;
    }
    const int sc = dx + 1;   // ring column
    auto site_of = [&](int row) {
      return (unsigned)d.off + (unsigned)wrapi(row, ny) * (unsigned)nx + (unsigned)col;
    };
    auto slot_of = [&](int row) { return (row - k0) % G::NSLOT; };
    auto wait_row = [&](int row) {
      const int s = slot_of(row);
      if (!bar_wait(bar0 + 8 * s, (phase >> s) & 1u)) bad = true;
      phase ^= 1u << s;
    };

    // the first rows of the tile
    for (int r = k0; r <= min(k0 + G::NSLOT - 1, klast); ++r)
      issue_row(a, d, wrapi(r, ny), x0, w, slots + slot_of(r) * G::SLOT_BYTES,
                bar0 + 8 * slot_of(r), t);
    int issued = min(k0 + G::NSLOT - 1, klast), waited = k0 - 1;

    // ring rows ya-1 and ya (streaming reads staged rows ya-2 .. ya+1)
    OwnHG<S, R> ohg;
    R hC[9], gC[5], poC = R(0);
    for (int r = k0; r <= ya + 1; ++r) wait_row(r);
    waited = ya + 1;
    for (int k = 0; k < 2; ++k) {
      const int y = ya - 1 + k;
      if (active) {
        load_own_hg(a, site_of(y), ohg);
        const SlotView<S, R> rows[3] = {slot_view<S, R>(slots, slot_of(y - 1)),
                                        slot_view<S, R>(slots, slot_of(y)),
                                        slot_view<S, R>(slots, slot_of(y + 1))};
        R h[9], g[5], phi, psi, po;
        stream_hg(rows, dx, ohg, h, g, phi, psi, po);
        ring[0][y & 3][sc] = phi;
        ring[1][y & 3][sc] = psi;
        ring[2][y & 3][sc] = ohg.vxo;
        ring[3][y & 3][sc] = ohg.vyo;
        if (k == 1) {
#pragma unroll
          for (int i = 0; i < 9; ++i) hC[i] = h[i];
#pragma unroll
          for (int i = 0; i < 5; ++i) gC[i] = g[i];
          poC = po;
        }
      }
    }
    // own inputs one row ahead
    OwnSite<S, R> osC{};
    if (active) load_own_hg(a, site_of(ya + 1), ohg);
    if (interior) load_own_site(a, site_of(ya), osC);

    for (int j = ya; j < yb; ++j) {
      wait_row(j + 2);
      waited = j + 2;
      // streaming of row j+1 into the ring
      R hL[9], gL[5], poL = R(0);
      if (active) {
        const int y = j + 1;
        const SlotView<S, R> rows[3] = {slot_view<S, R>(slots, slot_of(y - 1)),
                                        slot_view<S, R>(slots, slot_of(y)),
                                        slot_view<S, R>(slots, slot_of(y + 1))};
        R phi, psi;
        stream_hg(rows, dx, ohg, hL, gL, phi, psi, poL);
        ring[0][y & 3][sc] = phi;
        ring[1][y & 3][sc] = psi;
        ring[2][y & 3][sc] = ohg.vxo;
        ring[3][y & 3][sc] = ohg.vyo;
        if (j + 2 < yb + 1) load_own_hg(a, site_of(j + 2), ohg);
      }
      OwnSite<S, R> osN{};
      if (interior && j + 1 < yb) load_own_site(a, site_of(j + 1), osN);
      if (__syncthreads_or(bad)) {
        // drain the copies still in flight (bounded), report, stop
        for (int r = waited + 1; r <= issued; ++r) {
          const int s = slot_of(r);
          bar_wait(bar0 + 8 * s, (phase >> s) & 1u);
          phase ^= 1u << s;
        }
        if (t == 0 && a.err) atomicOr(a.err, 1u);
        return;
      }
      // refill the slot of row j-2 (free: its last reader was the update of
      // row j-1, before this barrier) with row j-2+NSLOT
      const int rn = j - 2 + G::NSLOT;
      if (rn <= klast)
        issue_row(a, d, wrapi(rn, ny), x0, w, slots + slot_of(rn) * G::SLOT_BYTES,
                  bar0 + 8 * slot_of(rn), t);
      if (rn <= klast) issued = rn;
      if (interior) {
        const SlotView<S, R> rows[3] = {slot_view<S, R>(slots, slot_of(j - 1)),
                                        slot_view<S, R>(slots, slot_of(j)),
                                        slot_view<S, R>(slots, slot_of(j + 1))};
        SiteIn<R> in;
        site_inputs(rows, dx, osC, in);
        Src9 src;
        src.s[0] = site_of(j);
        const int m = (j - 1) & 3, c0 = j & 3, pp = (j + 1) & 3;
        auto rws = [&](int f) { return Rows3<R>{ring[f][m], ring[f][c0], ring[f][pp]}; };
        site_update(a, d, src, in, hC, gC, poC, rws(0), rws(1), rws(2), rws(3), sc);
      }
#pragma unroll
      for (int i = 0; i < 9; ++i) hC[i] = hL[i];
#pragma unroll
      for (int i = 0; i < 5; ++i) gC[i] = gL[i];
      poC = poL;
      osC = osN;
    }
    __syncthreads();
  }
}

template <typename S, typename R>
int staged_smem_bytes() {
  return Stage<S, R>::SMEM;
}

template <typename S, typename R>
int staged_halo_columns() {
  return Stage<S, R>::HS > Stage<S, R>::HR ? Stage<S, R>::HS : Stage<S, R>::HR;
}

template <typename S, typename R>
cudaError_t launch_step_staged(const StepArgs<S, R>& a, int grid, cudaStream_t st) {
  static int configured[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && !configured[dev]) {
    e = cudaFuncSetAttribute(k_step_staged<S, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             Stage<S, R>::SMEM);
    if (e != cudaSuccess) return e;
    configured[dev] = 1;
  }
  k_step_staged<S, R><<<grid, YM_THREADS, Stage<S, R>::SMEM, st>>>(a);
  return cudaGetLastError();
}

template <typename S, typename R>
int staged_blocks_per_sm() {
  int n = 0;
  cudaFuncSetAttribute(k_step_staged<S, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       Stage<S, R>::SMEM);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_staged<S, R>, YM_THREADS,
                                                Stage<S, R>::SMEM);
  return n > 0 ? n : 1;
}

#define PF_STAGED_INST(S, R)                                                          \
  template cudaError_t launch_step_staged<S, R>(const StepArgs<S, R>&, int, cudaStream_t); \
  template int staged_smem_bytes<S, R>();                                             \
  template int staged_halo_columns<S, R>();                                           \
  template int staged_blocks_per_sm<S, R>();
PF_STAGED_INST(double, double)
PF_STAGED_INST(float, float)
PF_STAGED_INST(__half, float)
PF_STAGED_INST(__nv_bfloat16, float)

}  // namespace pf
