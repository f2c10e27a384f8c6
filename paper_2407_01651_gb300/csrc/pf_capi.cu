// pf_capi.cu -- implementation of the C ABI declared in include/pf.h.
//
// A handle owns, for all of its domains together:
//   - two copies of the 39-plane state (45 in thermal mode; ping-pong of the
//     pull scheme),
//   - 9 field planes in compute precision (written by the last step of each
//     pf_step call and by the initialisation),
//   - a uint8 grain id per site and a (cos, sin) table per domain,
//   - the domain and tile tables of the step kernel,
//   - FP64 reduction scratch and a staging buffer for FP64 host transfers.
// Domains are concatenated in every plane; each starts on a 64-site boundary.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "../../include/pf.h"
#include "pf_internal.h"

using namespace pf;

struct pf_handle {
  pf_params p{};
  pf_precision prec = PF_FP32;
  cudaStream_t stream = nullptr;
  pf_allocator alloc{};
  bool has_alloc = false;
  int device = 0;
  std::vector<pf_domain> doms;
  std::vector<DomDesc> ddesc;
  std::vector<int> inited;
  long long plane_stride = 0;
  size_t elem = 4;          // bytes per stored value
  size_t celem = 4;         // bytes per compute value
  int thermal = 0;          // temperature lattice and finite-Le F(U)
  int n_pop = N_POP;        // population planes per state copy
  int n_aux = N_AUX;        // lagged-scalar planes per state copy
  int n_phys = N_PHYS;      // planes of the raw FP64 state
  int any_bc = 0;           // some domain has a non-periodic side
  int any_io = 0;           // ... among them an inlet or an outlet
  // With non-periodic sides (y-march): tiles touching such a side ("edge"
  // tiles) run the boundary-aware kernel, the others the periodic one.  Tiles
  // are ordered [plain tiles of every domain][edge tiles of every domain]; each
  // run of consecutive tiles of one domain has its own descriptor in d_runs,
  // whose tile0 maps the launch index back to the tile of the domain.
  DomDesc* d_runs = nullptr;
  int n_plain = 0;
  std::vector<int> plain0, plain1, edge0, edge1;   // per-domain tile ranges
  // the edge tiles run on a side stream, forked from and joined to the step's
  // stream by events, so that they fill the SMs beside the plain tiles
  cudaStream_t side = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  int variant = STEP_YMARCH;  // step kernel traversal
  int tx = 32, ty = 8;      // tile of the 2-D variant
  int chunk = 32;           // rows per tile of the y-march variants (tuned at 4096^2)
  int ntiles = 0;
  int grid = 0;
  int launch_mode = 0;      // 0: one launch over all domains; 1: one launch per domain
  int persistent = 0;       // 1: grid = resident CTAs, each loops over tiles;
                            // 2: as 1, and every step of a call in one cooperative launch
  int coop_graph_failed = 0;  // capturing the cooperative launch failed: replay without graphs
  int sms = 0;
  // CUDA-graph replay of the stepping: one executable graph per buffer parity
  int graph_steps = 0;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  cudaStream_t cap_stream = nullptr;
  cudaStream_t adj_stream = nullptr;   // recomputation stream of the adjoint
  void* pop[2] = {nullptr, nullptr};   // population planes, storage type
  void* aux[2] = {nullptr, nullptr};   // lagged-scalar planes, compute type
  int cur = 0;
  void* fields = nullptr;
  uint8_t* grain = nullptr;
  double2* grain_cs = nullptr;
  DomDesc* d_doms = nullptr;
  int* d_tile_dom = nullptr;
  double* partial = nullptr;
  double* d_diag = nullptr;
  unsigned int* d_err = nullptr;  // device error bits written by the step kernels
  int* d_tile_ctr = nullptr;      // two tile counters of the one-launch mode
  int drop_copies = 0;            // testing only (pf_test_drop_staged_copies)
  double* staging = nullptr;    // FP64 device staging (largest domain x 39 planes)
  size_t staging_elems = 0;
  long long steps = 0;
  long long launches = 0;
  std::string err;
  // discrete-adjoint workspace (grown on demand, released by pf_destroy)
  void* adj_ws = nullptr;
  size_t adj_ws_bytes = 0;
  // pf_run: one stream per row band, the events that order the bands' steps
  // (two steps alternate) and the event that releases the bands' first step
  cudaStream_t run_st[PF_RUN_BANDS] = {};
  int run_nb = 0;                      // bands the streams' priorities were set for
  cudaEvent_t run_ev[2][PF_RUN_BANDS] = {};
  cudaEvent_t run_phi = nullptr, run_ctl = nullptr;
};

static std::string g_create_err;

void pf::set_global_error(const std::string& msg) { g_create_err = msg; }

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
// Call f(S{}, R{}) with the storage and compute types of the handle.
template <typename F>
static pf_status dispatch(const pf_handle* h, F&& f) {
  switch (h->prec) {
    case PF_FP64: return f(double{}, double{});
    case PF_FP32: return f(float{}, float{});
    case PF_FP16_OFFSET: return f(__half{}, float{});
    case PF_BF16_OFFSET: return f(__nv_bfloat16{}, float{});
  }
  return PF_ERR_BAD_ARG;
}
#define PF_TYPES(s_tag, r_tag)     \
  using S = decltype(s_tag);       \
  using R = decltype(r_tag);
static pf_status fail(pf_handle* h, pf_status code, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_err = msg;
  return code;
}

static bool staged_ok(const pf_handle* h);

static pf_status cuda_fail(pf_handle* h, cudaError_t e, const char* where) {
  return fail(h, PF_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define PF_CUDA(h, ...)                                           \
  do {                                                            \
    cudaError_t e_ = (__VA_ARGS__);                               \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #__VA_ARGS__); \
  } while (0)

// Device address of host memory the GPU can reach directly: page-locked
// (cudaHostAlloc or cudaHostRegister) memory, which the kernels then read or
// write over the CPU-GPU link without a staging copy.  nullptr for ordinary
// pageable memory (the caller stages through device memory).
static const void* host_device_view(const void* host) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, host) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

static void* dev_alloc(pf_handle* h, size_t bytes) {
  if (bytes == 0) bytes = 256;
  void* p = nullptr;
  if (h->has_alloc) {
    p = h->alloc.alloc(h->alloc.ctx, bytes, (void*)h->stream);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  return p;
}

static void dev_free(pf_handle* h, void* p) {
  if (!p) return;
  if (h->has_alloc) h->alloc.free(h->alloc.ctx, p, (void*)h->stream);
  else cudaFree(p);
}

static bool finite_pos(double v) { return std::isfinite(v) && v > 0; }

template <typename R>
static KParams<R> make_kparams(const pf_params& p) {
  KParams<R> k{};
  const double kappa = std::sqrt(2.0 * p.beta_phi) / p.W_phi;
  const double s_nu = 1.0 / (3.0 * p.nu + 0.5);
  k.rho_g = (R)p.rho_g;
  k.drho = (R)(p.rho_l - p.rho_g);
  k.ge2 = (R)(p.grad_eps * p.grad_eps);
  k.gat2 = (R)(p.grad_eps_at * p.grad_eps_at);
  k.kappa = (R)kappa;
  k.fs_coef = (R)(6.0 * p.sigma / (p.W_phi * std::sqrt(2.0 * p.beta_phi)));
  k.Wphi2 = (R)(p.W_phi * p.W_phi);
  k.M_phi = (R)p.M_phi;
  k.two_bphi = (R)(2.0 * p.beta_phi);
  k.two_bint = (R)(2.0 * p.beta_inter);
  k.four_bpsi = (R)(4.0 * p.beta_psi);
  double der[3];
  pf_params_derived(&p, der);
  k.lam = (R)der[0];
  k.Mcinf = (R)der[1];
  k.theta = (R)der[2];
  k.inv_tau0 = (R)(1.0 / p.tau0);
  k.c_s1 = (R)(3.0 * p.W0 * p.W0 / p.tau0);
  k.W0 = (R)p.W0;
  k.a_at = (R)(1.0 / (2.0 * std::sqrt(2.0)));
  k.k = (R)p.k;
  k.D = (R)p.D;
  k.g = (R)p.g;
  k.inv_omk = (R)(1.0 / (1.0 - p.k));
  k.s_e = (R)p.s_e;
  k.s_eps = (R)p.s_eps;
  k.s_q = (R)(8.0 * (2.0 - s_nu) / (8.0 - s_nu));
  k.s_nu = (R)s_nu;
  k.s_phi = (R)(1.0 / (3.0 * p.M_phi + 0.5));
  k.vin_x = (R)p.vin_x;
  k.vin_y = (R)p.vin_y;
  // temperature coupling: alpha = k_T / (rho_l c_p) = Le D, k_T = (1/s - 1/2) / 3
  if (p.thermal) {
    const double kT = p.Le * p.D * p.rho_l * p.cp;
    k.th_cp = (R)p.cp;
    k.th_icp = (R)(1.0 / p.cp);
    k.th_lh = (R)(0.5 * p.latent);
    k.th_s = (R)(1.0 / (3.0 * kT + 0.5));
    k.th_iLe = (R)(1.0 / p.Le);
    k.th_dF = (R)(der[1] * (1.0 - p.k));
    k.W0sq = (R)(p.W0 * p.W0);
    k.th_far = (R)p.theta0;
  }
  return k;
}

static pf_status check_params(const pf_params* p) {
  if (!p) return fail(nullptr, PF_ERR_BAD_ARG, "params is NULL");
  if (!finite_pos(p->rho_l) || !finite_pos(p->rho_g) || !finite_pos(p->nu) ||
      !finite_pos(p->W_phi) || !finite_pos(p->M_phi) || !finite_pos(p->W0) ||
      !finite_pos(p->tau0) || !finite_pos(p->D) || !finite_pos(p->beta_phi) ||
      !finite_pos(p->beta_psi) || !std::isfinite(p->beta_inter) || !std::isfinite(p->sigma) ||
      !std::isfinite(p->g) || !std::isfinite(p->Omega) || !std::isfinite(p->eps_s) ||
      !finite_pos(p->grad_eps) || !finite_pos(p->grad_eps_at) || !finite_pos(p->s_e) ||
      !finite_pos(p->s_eps) || p->s_e >= 2.0 || p->s_eps >= 2.0 || !std::isfinite(p->vin_x) ||
      !std::isfinite(p->vin_y))
    return fail(nullptr, PF_ERR_BAD_ARG, "a parameter is non-finite or out of range");
  if (!(p->k > 0.0 && p->k < 1.0)) return fail(nullptr, PF_ERR_BAD_ARG, "k must be in (0, 1)");
  // a_s >= 1 - eps > 0 needs eps < 1; beyond 1/15 the interface stiffness
  // a_s + a_s'' turns negative along the <11> directions (sharp corners)
  if (!(p->eps_s >= 0.0 && p->eps_s < 0.25))
    return fail(nullptr, PF_ERR_BAD_ARG, "eps_s must be in [0, 0.25)");
  if (1.0 - (1.0 - p->k) * p->Omega == 0.0)
    return fail(nullptr, PF_ERR_BAD_ARG, "1 - (1-k) Omega must be non-zero");
  if (p->thermal != 0 && p->thermal != 1)
    return fail(nullptr, PF_ERR_BAD_ARG, "thermal must be 0 or 1");
  if (p->reserved != 0) return fail(nullptr, PF_ERR_BAD_ARG, "reserved must be 0");
  if (p->thermal) {
    if (!finite_pos(p->Le) || !finite_pos(p->cp) || !std::isfinite(p->latent) ||
        !std::isfinite(p->theta0))
      return fail(nullptr, PF_ERR_BAD_ARG, "thermal mode needs Le > 0, cp > 0, finite latent, theta0");
    // the rest population rho H + (w_0 - 1) theta keeps the update of theta a
    // positive average only for rho c_p >= 1 - w_0 = 2/3 (gas included)
    if (p->rho_g * p->cp < 2.0 / 3.0)
      return fail(nullptr, PF_ERR_BAD_ARG, "thermal mode needs rho_g * cp >= 2/3 (stability)");
  }
  return PF_OK;
}

template <typename R>
static R* fields_ptr(pf_handle* h) { return reinterpret_cast<R*>(h->fields); }

// FP64 device staging for host transfers, grown on demand (never on the
// stepping path).
static pf_status ensure_staging(pf_handle* h, size_t elems) {
  if (elems <= h->staging_elems) return PF_OK;
  cudaStreamSynchronize(h->stream);
  dev_free(h, h->staging);
  h->staging = (double*)dev_alloc(h, elems * sizeof(double));
  h->staging_elems = h->staging ? elems : 0;
  if (!h->staging) return fail(h, PF_ERR_OOM, "staging allocation failed");
  return PF_OK;
}

// ---------------------------------------------------------------------------
// parameters
// ---------------------------------------------------------------------------
extern "C" pf_status pf_params_default(pf_params* out) {
  if (!out) return PF_ERR_BAD_ARG;
  pf_params p{};
  p.rho_l = 1.0; p.rho_g = 0.1; p.nu = 0.1; p.sigma = 1e-3; p.W_phi = 4.0; p.M_phi = 0.1;
  p.beta_phi = 0.25; p.beta_psi = 0.25; p.beta_inter = 0.75;
  p.W0 = 4.0; p.tau0 = 320.0; p.eps_s = 0.05; p.k = 0.15; p.D = 0.1; p.Omega = 0.55;
  p.g = 1e-6; p.grad_eps = 1e-3; p.grad_eps_at = 1e-2; p.s_e = 1.0; p.s_eps = 1.0;
  p.Le = 1.0; p.latent = 1.0; p.theta0 = -0.55; p.cp = 10.0; p.thermal = 0;
  *out = p;
  return PF_OK;
}

extern "C" pf_status pf_params_derived(const pf_params* p, double out[3]) {
  if (!p || !out) return PF_ERR_BAD_ARG;
  // thin-interface limit: tau0 D / W0^2 = a2' lambda', a2' = 47/75
  out[0] = p->D * p->tau0 / ((47.0 / 75.0) * p->W0 * p->W0);
  // isothermal closure of the solutal case (B)
  out[1] = 1.0 - (1.0 - p->k) * p->Omega;
  out[2] = -out[1] * p->Omega / (1.0 - (1.0 - p->k) * p->Omega);
  return PF_OK;
}

// ---------------------------------------------------------------------------
// create / destroy
// ---------------------------------------------------------------------------
static void release(pf_handle* h) {
  if (!h) return;
  for (void*& s : h->pop) { dev_free(h, s); s = nullptr; }
  for (void*& s : h->aux) { dev_free(h, s); s = nullptr; }
  dev_free(h, h->fields);
  dev_free(h, h->grain);
  dev_free(h, h->grain_cs);
  dev_free(h, h->d_doms);
  dev_free(h, h->d_runs);
  h->d_runs = nullptr;
  dev_free(h, h->d_tile_dom);
  dev_free(h, h->partial);
  dev_free(h, h->d_diag);
  dev_free(h, h->d_err);
  h->d_err = nullptr;
  dev_free(h, h->d_tile_ctr);
  h->d_tile_ctr = nullptr;
  dev_free(h, h->staging);
  dev_free(h, h->adj_ws);
  h->adj_ws = nullptr;
  for (auto& g : h->gexec)
    if (g) { cudaGraphExecDestroy(g); g = nullptr; }
  if (h->cap_stream) { cudaStreamDestroy(h->cap_stream); h->cap_stream = nullptr; }
  if (h->adj_stream) { cudaStreamDestroy(h->adj_stream); h->adj_stream = nullptr; }
  if (h->side) { cudaStreamDestroy(h->side); h->side = nullptr; }
  if (h->fork_ev) { cudaEventDestroy(h->fork_ev); h->fork_ev = nullptr; }
  if (h->join_ev) { cudaEventDestroy(h->join_ev); h->join_ev = nullptr; }
  h->run_nb = 0;
  for (int b = 0; b < PF_RUN_BANDS; ++b) {
    if (h->run_st[b]) { cudaStreamDestroy(h->run_st[b]); h->run_st[b] = nullptr; }
    for (int k = 0; k < 2; ++k)
      if (h->run_ev[k][b]) { cudaEventDestroy(h->run_ev[k][b]); h->run_ev[k][b] = nullptr; }
  }
  if (h->run_phi) { cudaEventDestroy(h->run_phi); h->run_phi = nullptr; }
  if (h->run_ctl) { cudaEventDestroy(h->run_ctl); h->run_ctl = nullptr; }
  h->fields = h->grain = nullptr;
}

static pf_status upload_tables(pf_handle* h) {
  // tiles of every domain, in domain order
  std::vector<int> tile_dom;
  std::vector<int> tiles_y(h->ddesc.size());
  for (size_t d = 0; d < h->ddesc.size(); ++d) {
    DomDesc& dd = h->ddesc[d];
    const bool strip = h->variant == STEP_YMARCH || h->variant == STEP_STAGED;
    const int tw = strip ? YM_W : h->tx;
    const int th = strip ? h->chunk : h->ty;
    dd.tiles_x = (dd.nx + tw - 1) / tw;
    tiles_y[d] = (dd.ny + th - 1) / th;
    dd.tile0 = (int)tile_dom.size();
    for (int t = 0; t < dd.tiles_x * tiles_y[d]; ++t) tile_dom.push_back((int)d);
  }
  h->ntiles = (int)tile_dom.size();
  if (h->any_bc) {
    // plain tiles first, then edge tiles, in runs with their own descriptors
    const size_t nd = h->ddesc.size();
    std::vector<DomDesc> runs;
    std::vector<int> order;
    h->plain0.assign(nd, 0); h->plain1.assign(nd, 0);
    h->edge0.assign(nd, 0); h->edge1.assign(nd, 0);
    for (int pass = 0; pass < 2; ++pass) {
      for (size_t d = 0; d < nd; ++d) {
        const DomDesc& dd = h->ddesc[d];
        const int tx = dd.tiles_x, ty = tiles_y[d];
        (pass ? h->edge0 : h->plain0)[d] = (int)order.size();
        int prev = -2;
        for (int lt = 0; lt < tx * ty; ++lt) {
          const int sx = lt % tx, cy = lt / tx;
          const bool edge = (sx == 0 && dd.bc[0]) || (sx == tx - 1 && dd.bc[1]) ||
                            (cy == 0 && dd.bc[2]) || (cy == ty - 1 && dd.bc[3]);
          if (edge != (pass == 1)) continue;
          if (lt != prev + 1) {
            DomDesc r = dd;
            r.tile0 = (int)order.size() - lt;
            runs.push_back(r);
          }
          order.push_back((int)runs.size() - 1);
          prev = lt;
        }
        (pass ? h->edge1 : h->plain1)[d] = (int)order.size();
      }
      if (pass == 0) h->n_plain = (int)order.size();
    }
    tile_dom.swap(order);
    dev_free(h, h->d_runs);
    h->d_runs = (DomDesc*)dev_alloc(h, runs.size() * sizeof(DomDesc));
    if (!h->d_runs) return fail(h, PF_ERR_OOM, "tile table allocation failed");
    PF_CUDA(h, cudaMemcpyAsync(h->d_runs, runs.data(), runs.size() * sizeof(DomDesc),
                               cudaMemcpyHostToDevice, h->stream));
  }
  dev_free(h, h->d_tile_dom);
  h->d_tile_dom = (int*)dev_alloc(h, tile_dom.size() * sizeof(int));
  if (!h->d_tile_dom) return fail(h, PF_ERR_OOM, "tile table allocation failed");
  PF_CUDA(h, cudaMemcpyAsync(h->d_tile_dom, tile_dom.data(), tile_dom.size() * sizeof(int),
                             cudaMemcpyHostToDevice, h->stream));
  PF_CUDA(h, cudaMemcpyAsync(h->d_doms, h->ddesc.data(), h->ddesc.size() * sizeof(DomDesc),
                             cudaMemcpyHostToDevice, h->stream));
  PF_CUDA(h, cudaStreamSynchronize(h->stream));
  for (auto& g : h->gexec)
    if (g) { cudaGraphExecDestroy(g); g = nullptr; }
  cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
  h->grid = h->ntiles;  // one CTA per tile; the kernel also accepts fewer (grid-stride)
  return PF_OK;
}

extern "C" pf_status pf_create(const pf_params* p, const pf_domain* doms, int n_doms,
                               pf_precision prec, void* cuda_stream, const pf_allocator* alloc,
                               pf_handle** out) {
  if (!out) return fail(nullptr, PF_ERR_BAD_ARG, "out is NULL");
  *out = nullptr;
  pf_status st = check_params(p);
  if (st != PF_OK) return st;
  if (!doms || n_doms < 1) return fail(nullptr, PF_ERR_BAD_ARG, "need at least one domain");
  if (prec != PF_FP64 && prec != PF_FP32 && prec != PF_FP16_OFFSET && prec != PF_BF16_OFFSET)
    return fail(nullptr, PF_ERR_BAD_ARG, "unknown precision");
  for (int d = 0; d < n_doms; ++d) {
    if (doms[d].nx < 4 || doms[d].ny < 4 || doms[d].nx > (1 << 16) || doms[d].ny > (1 << 16))
      return fail(nullptr, PF_ERR_BAD_ARG, "domain sizes must be in [4, 65536]");
    if (doms[d].eps_s >= 0.25 || !std::isfinite(doms[d].eps_s))
      return fail(nullptr, PF_ERR_BAD_ARG, "domain eps_s must be < 0.25");
  }
  if (alloc && (!alloc->alloc || !alloc->free))
    return fail(nullptr, PF_ERR_BAD_ARG, "allocator needs alloc and free");
  if (p->thermal && prec != PF_FP32 && prec != PF_FP64)
    return fail(nullptr, PF_ERR_BAD_ARG, "thermal mode needs FP32 or FP64 storage");

  pf_handle* h = new (std::nothrow) pf_handle();
  if (!h) return fail(nullptr, PF_ERR_OOM, "host allocation failed");
  h->p = *p;
  h->prec = prec;
  h->stream = (cudaStream_t)cuda_stream;
  if (alloc) { h->alloc = *alloc; h->has_alloc = true; }
  cudaGetDevice(&h->device);
  h->elem = prec == PF_FP64 ? 8 : (prec == PF_FP32 ? 4 : 2);
  h->celem = prec == PF_FP64 ? 8 : 4;
  h->thermal = p->thermal;
  h->n_pop = p->thermal ? N_POP_TH : N_POP;
  h->n_aux = p->thermal ? N_AUX_TH : N_AUX;
  h->n_phys = p->thermal ? N_PHYS_TH : N_PHYS;
  h->doms.assign(doms, doms + n_doms);
  h->inited.assign(n_doms, 0);
  long long off = 0;
  size_t max_n = 0;
  for (int d = 0; d < n_doms; ++d) {
    DomDesc dd{};
    dd.off = off;
    dd.nx = doms[d].nx;
    dd.ny = doms[d].ny;
    dd.grain_off = d * MAX_GRAINS;
    dd.eps_s = doms[d].eps_s >= 0.0 ? doms[d].eps_s : p->eps_s;
    dd.rho_bar = p->rho_l;
    h->ddesc.push_back(dd);
    const long long n = (long long)dd.nx * dd.ny;
    max_n = std::max(max_n, (size_t)n);
    off += (n + 63) / 64 * 64;
  }
  h->plane_stride = off;
  const size_t ps = (size_t)off;
  // site indices are 32-bit (handles with more than 2^32 buffer elements
  // switch the step kernels to 64-bit plane bases)
  if ((unsigned long long)ps >= (1ull << 32)) {
    g_create_err = "too many sites for one handle (at most 2^32 including padding)";
    delete h;
    return PF_ERR_BAD_ARG;
  }

  auto bail = [&](pf_status code, const char* msg) {
    g_create_err = msg;
    release(h);
    delete h;
    return code;
  };
  for (int c = 0; c < 2; ++c) {
    h->pop[c] = dev_alloc(h, ps * h->n_pop * h->elem);
    h->aux[c] = dev_alloc(h, ps * h->n_aux * h->celem);
    if (!h->pop[c] || !h->aux[c]) return bail(PF_ERR_OOM, "state allocation failed");
  }
  h->fields = dev_alloc(h, ps * N_FIELDS * h->celem);
  h->grain = (uint8_t*)dev_alloc(h, ps);
  h->grain_cs = (double2*)dev_alloc(h, (size_t)n_doms * MAX_GRAINS * sizeof(double2));
  h->d_doms = (DomDesc*)dev_alloc(h, (size_t)n_doms * sizeof(DomDesc));
  h->partial = (double*)dev_alloc(h, (size_t)REDUCE_BLOCKS * NDIAG * sizeof(double));
  h->d_diag = (double*)dev_alloc(h, NDIAG * sizeof(double));
  h->d_err = (unsigned int*)dev_alloc(h, sizeof(unsigned int));
  (void)max_n;
  if (!h->fields || !h->grain || !h->grain_cs || !h->d_doms || !h->partial || !h->d_diag ||
      !h->d_err)
    return bail(PF_ERR_OOM, "device allocation failed");
  if (cudaMemsetAsync(h->fields, 0, ps * N_FIELDS * h->celem, h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->d_err, 0, sizeof(unsigned int), h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->grain, 0, ps, h->stream) != cudaSuccess)
    return bail(PF_ERR_CUDA, "memset failed");
  std::vector<double2> cs((size_t)n_doms * MAX_GRAINS, make_double2(1.0, 0.0));
  if (cudaMemcpyAsync(h->grain_cs, cs.data(), cs.size() * sizeof(double2), cudaMemcpyHostToDevice,
                      h->stream) != cudaSuccess)
    return bail(PF_ERR_CUDA, "grain table upload failed");
  // default traversal: the staged y-march for the 16-bit storage forms
  // (measured faster at 4096^2), the plain y-march otherwise
  if ((prec == PF_FP16_OFFSET || prec == PF_BF16_OFFSET) && staged_ok(h)) {
    h->variant = STEP_STAGED;
    h->chunk = 48;
  }
  if (upload_tables(h) != PF_OK) return bail(PF_ERR_CUDA, h->err.c_str());
  *out = h;
  return PF_OK;
}

extern "C" pf_status pf_destroy(pf_handle* h) {
  if (!h) return PF_OK;
  cudaStreamSynchronize(h->stream);
  cudaError_t e = cudaGetLastError();
  release(h);
  delete h;
  return e == cudaSuccess ? PF_OK : PF_ERR_CUDA;
}

extern "C" const char* pf_last_error(const pf_handle* h) {
  return h ? h->err.c_str() : g_create_err.c_str();
}

extern "C" long long pf_steps_taken(const pf_handle* h) { return h ? h->steps : -1; }
extern "C" long long pf_launch_count(const pf_handle* h) { return h ? h->launches : -1; }

// Device error bits set by the step kernels (read after a synchronisation).
static pf_status check_device_error(pf_handle* h) {
  unsigned int bits = 0;
  PF_CUDA(h, cudaMemcpy(&bits, h->d_err, sizeof(bits), cudaMemcpyDeviceToHost));
  if (bits & ERR_STAGED_TIMEOUT)
    return fail(h, PF_ERR_TIMEOUT,
                "staged step: a bulk copy of an input row did not complete within 1 s; the "
                "state is invalid");
  return PF_OK;
}

// A re-initialised state is valid again: clear the device error bits.
static pf_status clear_device_error(pf_handle* h) {
  PF_CUDA(h, cudaMemsetAsync(h->d_err, 0, sizeof(unsigned int), h->stream));
  return PF_OK;
}

extern "C" pf_status pf_test_drop_staged_copies(pf_handle* h, int on) {
  if (!h) return PF_ERR_BAD_ARG;
  if (on != 0 && on != 1) return fail(h, PF_ERR_BAD_ARG, "on must be 0 or 1");
  PF_CUDA(h, cudaStreamSynchronize(h->stream));
  h->drop_copies = on;
  for (auto& g : h->gexec)
    if (g) { cudaGraphExecDestroy(g); g = nullptr; }
  return PF_OK;
}

extern "C" pf_status pf_sync(pf_handle* h) {
  if (!h) return PF_ERR_BAD_ARG;
  PF_CUDA(h, cudaStreamSynchronize(h->stream));
  PF_CUDA(h, cudaGetLastError());
  return check_device_error(h);
}

// ---------------------------------------------------------------------------
// initialisation
// ---------------------------------------------------------------------------
// rho_bar of a domain from its initial fields (FP64 reduction), then upload.
static pf_status finish_init(pf_handle* h, int dom) {
  pf_diag dg{};
  pf_status st = pf_reduce(h, dom, nullptr, &dg);
  if (st != PF_OK) return st;
  DomDesc& dd = h->ddesc[dom];
  const double n = (double)dd.nx * dd.ny;
  // one rounding of the product-sum (fused), as the device-side form in pf_run
  dd.rho_bar = std::fma(dg.sum_phi / n, h->p.rho_l - h->p.rho_g, h->p.rho_g);
  if (h->any_bc) {
    pf_status st2 = upload_tables(h);   // the run descriptors carry rho_bar too
    if (st2 != PF_OK) return st2;
  }
  PF_CUDA(h, cudaMemcpyAsync(h->d_doms + dom, &dd, sizeof(DomDesc), cudaMemcpyHostToDevice,
                             h->stream));
  PF_CUDA(h, cudaStreamSynchronize(h->stream));
  h->inited[dom] = 1;
  h->steps = 0;
  return PF_OK;
}

template <typename S, typename R>
static pf_status init_spec_t(pf_handle* h, int dom, const pf_init_spec* spec, const double* d_s,
                             const double* d_b) {
  InitArgs<S, R> a{};
  a.out = reinterpret_cast<S*>(h->pop[h->cur]);
  a.aout = reinterpret_cast<R*>(h->aux[h->cur]);
  a.fields = fields_ptr<R>(h);
  a.grain = h->grain;
  a.plane_stride = h->plane_stride;
  a.dom = h->ddesc[dom];
  a.seeds = d_s;
  a.bubbles = d_b;
  a.n_seeds = spec->n_seeds;
  a.n_bub = spec->n_bubbles;
  a.R_s = spec->R_s;
  a.W0 = h->p.W0;
  a.Wphi = h->p.W_phi;
  a.sq2bpsi = std::sqrt(2.0 * h->p.beta_psi);
  a.sq2bphi = std::sqrt(2.0 * h->p.beta_phi);
  a.k = h->p.k;
  a.kp = make_kparams<R>(h->p);
  a.thermal = h->thermal;
  a.theta0 = h->p.theta0;
  PF_CUDA(h, launch_init_spec<S, R>(a, h->stream));
  h->launches++;
  return PF_OK;
}

static pf_status upload_grain_table(pf_handle* h, int dom, const std::vector<double>& angles) {
  std::vector<double2> cs(MAX_GRAINS, make_double2(1.0, 0.0));
  for (size_t i = 0; i < angles.size(); ++i) cs[i] = make_double2(std::cos(angles[i]), std::sin(angles[i]));
  PF_CUDA(h, cudaMemcpyAsync(h->grain_cs + (size_t)dom * MAX_GRAINS, cs.data(),
                             MAX_GRAINS * sizeof(double2), cudaMemcpyHostToDevice, h->stream));
  PF_CUDA(h, cudaStreamSynchronize(h->stream));
  return PF_OK;
}

extern "C" pf_status pf_init_fields(pf_handle* h, int dom, const pf_init_spec* spec) {
  if (!h) return PF_ERR_BAD_ARG;
  if (!spec || dom < 0 || dom >= (int)h->doms.size())
    return fail(h, PF_ERR_BAD_ARG, "bad domain index or NULL spec");
  if (spec->n_seeds < 0 || spec->n_seeds > MAX_GRAINS || spec->n_bubbles < 0 ||
      (spec->n_seeds > 0 && !spec->seeds) || (spec->n_bubbles > 0 && !spec->bubbles) ||
      !std::isfinite(spec->R_s))
    return fail(h, PF_ERR_BAD_ARG, "bad init spec (at most 256 seeds)");
  for (int i = 0; i < 3 * spec->n_seeds; ++i)
    if (!std::isfinite(spec->seeds[i])) return fail(h, PF_ERR_BAD_ARG, "non-finite seed");
  for (int i = 0; i < 3 * spec->n_bubbles; ++i)
    if (!std::isfinite(spec->bubbles[i])) return fail(h, PF_ERR_BAD_ARG, "non-finite bubble");
  std::vector<double> angles;
  for (int s = 0; s < spec->n_seeds; ++s) angles.push_back(spec->seeds[3 * s + 2]);
  pf_status st = clear_device_error(h);
  if (st != PF_OK) return st;
  st = upload_grain_table(h, dom, angles);
  if (st != PF_OK) return st;
  const size_t ns = 3 * (size_t)spec->n_seeds, nb = 3 * (size_t)spec->n_bubbles;
  double* buf = (double*)dev_alloc(h, (ns + nb + 1) * sizeof(double));
  if (!buf) return fail(h, PF_ERR_OOM, "init buffer allocation failed");
  if (ns) PF_CUDA(h, cudaMemcpyAsync(buf, spec->seeds, ns * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  if (nb) PF_CUDA(h, cudaMemcpyAsync(buf + ns, spec->bubbles, nb * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  st = dispatch(h, [&](auto s_t, auto r_t) {
    PF_TYPES(s_t, r_t);
    return init_spec_t<S, R>(h, dom, spec, buf, buf + ns);
  });
  cudaError_t e = cudaStreamSynchronize(h->stream);
  dev_free(h, buf);
  if (st != PF_OK) return st;
  if (e != cudaSuccess) return cuda_fail(h, e, "init");
  return finish_init(h, dom);
}

template <typename S, typename R>
static pf_status set_fields_t(pf_handle* h, int dom, const double* d_f6, const uint8_t* d_ids) {
  SetFieldsArgs<S, R> a{};
  a.out = reinterpret_cast<S*>(h->pop[h->cur]);
  a.aout = reinterpret_cast<R*>(h->aux[h->cur]);
  a.fields = fields_ptr<R>(h);
  a.grain = h->grain;
  a.plane_stride = h->plane_stride;
  a.dom = h->ddesc[dom];
  a.f6 = d_f6;
  a.grain_ids = d_ids;
  a.kp = make_kparams<R>(h->p);
  a.thermal = h->thermal;
  a.theta0 = h->p.theta0;
  a.err = h->d_err;
  PF_CUDA(h, launch_set_fields<S, R>(a, h->stream));
  h->launches++;
  return PF_OK;
}

extern "C" pf_status pf_set_fields(pf_handle* h, int dom, const double* fields6,
                                   const double* theta, size_t n) {
  if (!h) return PF_ERR_BAD_ARG;
  if (dom < 0 || dom >= (int)h->doms.size() || !fields6)
    return fail(h, PF_ERR_BAD_ARG, "bad domain index or NULL fields");
  const size_t nn = (size_t)h->ddesc[dom].nx * h->ddesc[dom].ny;
  if (n != nn) return fail(h, PF_ERR_BAD_ARG, "n must equal nx*ny of the domain");
  // The six planes are checked for non-finite values on the device, by the
  // kernel that writes the equilibria (a host scan of 6 n doubles on one
  // thread cost more than the copy itself).
  // grain angles: distinct values -> ids
  std::vector<uint8_t> ids;
  std::vector<double> angles;
  if (theta) {
    std::map<double, int> idx;
    ids.resize(nn);
    for (size_t i = 0; i < nn; ++i) {
      if (!std::isfinite(theta[i])) return fail(h, PF_ERR_BAD_ARG, "non-finite angle");
      auto it = idx.find(theta[i]);
      if (it == idx.end()) {
        if ((int)angles.size() >= MAX_GRAINS)
          return fail(h, PF_ERR_BAD_ARG, "more than 256 distinct grain angles");
        it = idx.emplace(theta[i], (int)angles.size()).first;
        angles.push_back(theta[i]);
      }
      ids[i] = (uint8_t)it->second;
    }
  }
  pf_status st = clear_device_error(h);
  if (st != PF_OK) return st;
  st = upload_grain_table(h, dom, angles);
  if (st != PF_OK) return st;
  // page-locked fields are read by the kernel in place; others are staged
  const double* direct = static_cast<const double*>(host_device_view(fields6));
  st = ensure_staging(h, (direct ? 0 : 6 * nn) + (theta ? (nn + 7) / 8 : 0));
  if (st != PF_OK) return st;
  const double* buf = direct ? direct : h->staging;
  uint8_t* d_ids = nullptr;
  if (!direct)
    PF_CUDA(h, cudaMemcpyAsync(h->staging, fields6, 6 * nn * sizeof(double),
                               cudaMemcpyHostToDevice, h->stream));
  if (theta) {
    d_ids = reinterpret_cast<uint8_t*>(h->staging + (direct ? 0 : 6 * nn));
    PF_CUDA(h, cudaMemcpyAsync(d_ids, ids.data(), nn, cudaMemcpyHostToDevice, h->stream));
  }
  st = dispatch(h, [&](auto s_t, auto r_t) {
    PF_TYPES(s_t, r_t);
    return set_fields_t<S, R>(h, dom, buf, d_ids);
  });
  if (st != PF_OK) return st;
  unsigned int bits = 0;
  PF_CUDA(h, cudaMemcpyAsync(&bits, h->d_err, sizeof(bits), cudaMemcpyDeviceToHost, h->stream));
  PF_CUDA(h, cudaStreamSynchronize(h->stream));
  if (bits & ERR_NONFINITE_INPUT) {
    // the domain's state now holds the rejected values: it must be set again
    h->inited[dom] = 0;
    pf_status c = clear_device_error(h);
    if (c != PF_OK) return c;
    PF_CUDA(h, cudaStreamSynchronize(h->stream));
    return fail(h, PF_ERR_BAD_ARG, "non-finite field value; the domain must be initialised again");
  }
  return finish_init(h, dom);
}

// ---------------------------------------------------------------------------
// stepping
// ---------------------------------------------------------------------------
template <typename S, typename R>
static StepArgs<S, R> make_step_args(const pf_handle* h, const void* pin, const void* ain,
                                     void* pout, void* aout, bool write_fields) {
  StepArgs<S, R> a{};
  a.in = reinterpret_cast<const S*>(pin);
  a.out = reinterpret_cast<S*>(pout);
  a.ain = reinterpret_cast<const R*>(ain);
  a.aout = reinterpret_cast<R*>(aout);
  a.plane_stride = h->plane_stride;
  a.grain = h->grain;
  a.grain_cs = h->grain_cs;
  a.doms = h->any_bc ? h->d_runs : h->d_doms;
  a.tile_dom = h->d_tile_dom;
  a.ntiles = h->ntiles;
  a.chunk = h->chunk;
  a.fields = write_fields ? reinterpret_cast<R*>(h->fields) : nullptr;
  a.err = h->d_err;
  a.drop_copies = h->drop_copies;
  a.thermal = h->thermal;
  a.bc = h->any_bc ? (h->any_io ? 2 : 1) : 0;
  a.kp = make_kparams<R>(h->p);
  return a;
}

// Launch the step over every domain: one launch over the whole tile list, or
// one launch per domain; the grid is one CTA per tile, or the resident CTAs
// of the device looping over the tiles (persistent).
template <typename S, typename R>
static pf_status launch_all(pf_handle* h, StepArgs<S, R> a, cudaStream_t stream) {
  auto cap_of = [&](bool bc) {
    return h->persistent ? std::max(1, h->sms) *
                               step_blocks_per_sm<S, R>(h->variant, h->tx, h->ty,
                                                        h->plane_stride, h->thermal != 0, bc)
                         : 1 << 30;
  };
  // one launch over tiles [t0, t1) of the periodic (bc = 0) or boundary-aware kernel
  auto go = [&](int t0, int t1, int bc, cudaStream_t sx) -> pf_status {
    if (t1 <= t0) return PF_OK;
    a.tile_base = t0;
    a.ntiles = t1;
    a.bc = bc;
    PF_CUDA(h, launch_step<S, R>(a, h->variant, h->tx, h->ty, std::min(t1 - t0, cap_of(bc != 0)),
                                 sx));
    h->launches++;
    return PF_OK;
  };
  auto go1 = [&](int t0, int t1, int bc) { return go(t0, t1, bc, stream); };
  const int edge_kind = h->any_io ? 2 : 1;   // boundary kernel with or without inlet/outlet code
  pf_status st = PF_OK;
  if (h->any_bc) {
    // plain tiles: the periodic kernel; edge tiles: the boundary-aware one, on
    // the side stream (both read the same state and write disjoint sites)
    if (h->launch_mode == 0) {
      if (h->ntiles > h->n_plain && h->n_plain > 0) {
        if (!h->side) {
          PF_CUDA(h, cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
          PF_CUDA(h, cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming));
          PF_CUDA(h, cudaEventCreateWithFlags(&h->join_ev, cudaEventDisableTiming));
        }
        PF_CUDA(h, cudaEventRecord(h->fork_ev, stream));
        PF_CUDA(h, cudaStreamWaitEvent(h->side, h->fork_ev, 0));
        if ((st = go(h->n_plain, h->ntiles, edge_kind, h->side)) != PF_OK) return st;
        if ((st = go1(0, h->n_plain, 0)) != PF_OK) return st;
        PF_CUDA(h, cudaEventRecord(h->join_ev, h->side));
        PF_CUDA(h, cudaStreamWaitEvent(stream, h->join_ev, 0));
        return PF_OK;
      }
      if ((st = go1(0, h->n_plain, 0)) != PF_OK) return st;
      return go1(h->n_plain, h->ntiles, edge_kind);
    }
    for (size_t d = 0; d < h->ddesc.size(); ++d) {
      if ((st = go1(h->plain0[d], h->plain1[d], 0)) != PF_OK) return st;
      if ((st = go1(h->edge0[d], h->edge1[d], edge_kind)) != PF_OK) return st;
    }
    return PF_OK;
  }
  if (h->launch_mode == 0) return go1(0, h->ntiles, 0);
  for (size_t d = 0; d < h->ddesc.size(); ++d) {
    const int t0 = h->ddesc[d].tile0;
    const int t1 = d + 1 < h->ddesc.size() ? h->ddesc[d + 1].tile0 : h->ntiles;
    if ((st = go1(t0, t1, 0)) != PF_OK) return st;
  }
  return PF_OK;
}

// Kernel launches of one step (the graph replay counts them without launching).
static int launches_per_step(const pf_handle* h) {
  if (!h->any_bc) return h->launch_mode == 0 ? 1 : (int)h->ddesc.size();
  int n = 0;
  if (h->launch_mode == 0) return (h->n_plain > 0) + (h->ntiles > h->n_plain);
  for (size_t d = 0; d < h->ddesc.size(); ++d)
    n += (h->plain1[d] > h->plain0[d]) + (h->edge1[d] > h->edge0[d]);
  return n;
}

// The one-launch mode applies to the y-march over periodic domains with one
// launch over the whole tile list; elsewhere mode 2 runs as mode 1.
static bool steps_in_one_launch(const pf_handle* h) {
  return h->persistent == 2 && h->variant == STEP_YMARCH && !h->any_bc && h->launch_mode == 0;
}

// n steps (n >= 1) in one cooperative launch of the resident grid.
template <typename S, typename R>
static pf_status steps_one_launch(pf_handle* h, int n, bool write_fields, cudaStream_t stream) {
  StepArgs<S, R> a = make_step_args<S, R>(h, h->pop[h->cur], h->aux[h->cur], h->pop[h->cur ^ 1],
                                          h->aux[h->cur ^ 1], write_fields);
  a.tile_base = 0;
  a.ntiles = h->ntiles;
  a.bc = 0;
  const int cap = std::max(1, h->sms) * ymarch_steps_blocks_per_sm<S, R>(h->plane_stride,
                                                                        h->thermal != 0);
  if (!h->d_tile_ctr) return fail(h, PF_ERR_STATE, "tile counters missing (pf_set_launch)");
  PF_CUDA(h, launch_ymarch_steps<S, R>(a, n, h->d_tile_ctr, std::max(1, std::min(cap, h->ntiles)),
                                       stream));
  h->launches++;
  h->cur ^= (n & 1);
  h->steps += n;
  return PF_OK;
}

template <typename S, typename R>
static pf_status step_t(pf_handle* h, bool write_fields, cudaStream_t stream = nullptr) {
  const StepArgs<S, R> a = make_step_args<S, R>(h, h->pop[h->cur], h->aux[h->cur],
                                                h->pop[h->cur ^ 1], h->aux[h->cur ^ 1],
                                                write_fields);
  pf_status st = launch_all<S, R>(h, a, stream ? stream : h->stream);
  if (st != PF_OK) return st;
  h->cur ^= 1;
  h->steps++;
  return PF_OK;
}

// Executable graph of graph_steps steps (no field output) starting from the
// current buffer parity; captured on an internal stream, replayed on the
// handle's stream.  graph_steps is even, so the parity is unchanged.
template <typename S, typename R>
static pf_status ensure_graph(pf_handle* h) {
  const int par = h->cur;
  if (h->gexec[par]) return PF_OK;
  if (!h->cap_stream) PF_CUDA(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  const long long steps0 = h->steps, launches0 = h->launches;
  PF_CUDA(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  pf_status st = PF_OK;
  const bool one = steps_in_one_launch(h);
  if (one) st = steps_one_launch<S, R>(h, h->graph_steps, false, h->cap_stream);
  else
    for (int t = 0; t < h->graph_steps && st == PF_OK; ++t)
      st = step_t<S, R>(h, false, h->cap_stream);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
  h->cur = par;
  h->steps = steps0;
  h->launches = launches0;
  if (one && (st != PF_OK || e != cudaSuccess)) {
    // the cooperative launch could not be captured: replay it directly
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    h->err.clear();
    h->coop_graph_failed = 1;
    return PF_OK;
  }
  if (st != PF_OK) { if (g) cudaGraphDestroy(g); return st; }
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&h->gexec[par], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) { h->gexec[par] = nullptr; return cuda_fail(h, e, "cudaGraphInstantiate"); }
  return PF_OK;
}

template <typename S, typename R>
static pf_status step_n(pf_handle* h, int n_steps) {
  int done = 0;
  if (steps_in_one_launch(h)) {
    // graph_steps > 0: whole graph_steps-step launches replayed from graphs,
    // then the rest (with the field output) in one more launch
    if (h->graph_steps > 0 && !h->coop_graph_failed) {
      while (n_steps - 1 - done >= h->graph_steps) {
        pf_status st = ensure_graph<S, R>(h);
        if (st != PF_OK) return st;
        if (h->coop_graph_failed) break;
        PF_CUDA(h, cudaGraphLaunch(h->gexec[h->cur], h->stream));
        done += h->graph_steps;
        h->steps += h->graph_steps;
        h->launches += 1;
      }
    }
    return n_steps - done > 0 ? steps_one_launch<S, R>(h, n_steps - done, true, h->stream) : PF_OK;
  }
  if (h->graph_steps > 0) {
    const int per_step = launches_per_step(h);
    while (n_steps - 1 - done >= h->graph_steps) {
      pf_status st = ensure_graph<S, R>(h);
      if (st != PF_OK) return st;
      PF_CUDA(h, cudaGraphLaunch(h->gexec[h->cur], h->stream));
      done += h->graph_steps;
      h->steps += h->graph_steps;
      h->launches += (long long)h->graph_steps * per_step;
    }
  }
  for (; done < n_steps; ++done) {
    pf_status st = step_t<S, R>(h, done == n_steps - 1);
    if (st != PF_OK) return st;
  }
  return PF_OK;
}

// The staged variant needs every domain's nx to be a multiple of its copy
// granularity and 16-byte aligned state buffers.
template <typename S, typename R>
static bool staged_ok_t(const pf_handle* h) {
  const int g = staged_halo_columns<S, R>();
  for (const DomDesc& d : h->ddesc)
    if (d.nx % g != 0) return false;
  for (int c = 0; c < 2; ++c)
    if ((reinterpret_cast<uintptr_t>(h->pop[c]) | reinterpret_cast<uintptr_t>(h->aux[c])) & 15u)
      return false;
  return true;
}

static bool staged_ok(const pf_handle* h) {
  return dispatch(h, [&](auto s_t, auto r_t) {
           PF_TYPES(s_t, r_t);
           return staged_ok_t<S, R>(h) ? PF_OK : PF_ERR_BAD_ARG;
         }) == PF_OK;
}

extern "C" pf_status pf_set_step_config(pf_handle* h, int variant, int a, int b) {
  if (!h) return PF_ERR_BAD_ARG;
  if (h->thermal && variant != STEP_YMARCH)
    return fail(h, PF_ERR_BAD_ARG, "thermal mode runs the y-march traversal (variant 1) only");
  if (h->any_bc && variant != STEP_YMARCH)
    return fail(h, PF_ERR_BAD_ARG,
                "domains with non-periodic sides run the y-march traversal (variant 1) only");
  if (variant == STEP_TILE) {
    if (a < 1 || b < 1 || a * b > 256 || a % 32 != 0)
      return fail(h, PF_ERR_BAD_ARG, "tile variant needs tx a multiple of 32 and tx*ty <= 256");
    h->tx = a;
    h->ty = b;
  } else if (variant == STEP_YMARCH || variant == STEP_STAGED) {
    if (a < 1 || a > 65536) return fail(h, PF_ERR_BAD_ARG, "y-march chunk must be in [1, 65536]");
    if (variant == STEP_STAGED && !staged_ok(h))
      return fail(h, PF_ERR_BAD_ARG,
                  "staged variant needs nx a multiple of 16 bytes of storage (4 FP32, 8 FP16/BF16, "
                  "2 FP64 sites) in every domain");
    h->chunk = a;
  } else {
    return fail(h, PF_ERR_BAD_ARG, "unknown step variant");
  }
  PF_CUDA(h, cudaStreamSynchronize(h->stream));
  h->variant = variant;
  // captured graphs hold the old tile table's size and chunk: drop them
  for (auto& g : h->gexec)
    if (g) { cudaGraphExecDestroy(g); g = nullptr; }
  h->coop_graph_failed = 0;
  return upload_tables(h);
}

extern "C" pf_status pf_set_launch(pf_handle* h, int per_domain, int persistent,
                                   int graph_steps) {
  if (!h) return PF_ERR_BAD_ARG;
  if (per_domain < 0 || per_domain > 1 || persistent < 0 || persistent > 2 || graph_steps < 0 ||
      (graph_steps % 2) != 0 || graph_steps > 4096)
    return fail(h, PF_ERR_BAD_ARG,
                "per_domain in {0,1}, persistent in {0,1,2}; graph_steps even in [0, 4096]");
  if (persistent == 2 && per_domain)
    return fail(h, PF_ERR_BAD_ARG, "the one-launch mode takes one launch over every domain");
  if (persistent == 2) {
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device);
    if (!coop) return fail(h, PF_ERR_BAD_ARG, "the device has no cooperative launch");
    // allocated here, never under a graph capture
    if (!h->d_tile_ctr) {
      h->d_tile_ctr = static_cast<int*>(dev_alloc(h, 2 * sizeof(int)));
      if (!h->d_tile_ctr) return fail(h, PF_ERR_OOM, "tile counter allocation failed");
    }
  }
  PF_CUDA(h, cudaStreamSynchronize(h->stream));
  h->launch_mode = per_domain;
  h->persistent = persistent;
  h->graph_steps = graph_steps;
  h->coop_graph_failed = 0;
  for (auto& g : h->gexec)
    if (g) { cudaGraphExecDestroy(g); g = nullptr; }
  return PF_OK;
}

template <typename S, typename R>
static pf_status autotune_t(pf_handle* h, int trial_steps, int out[4]) {
  const size_t ps = (size_t)h->plane_stride;
  const size_t pop_b = ps * h->n_pop * sizeof(S), aux_b = ps * h->n_aux * sizeof(R);
  void* snap_p = dev_alloc(h, pop_b);
  void* snap_a = dev_alloc(h, aux_b);
  if (!snap_p || !snap_a) {
    dev_free(h, snap_p);
    dev_free(h, snap_a);
    return fail(h, PF_ERR_OOM, "autotune snapshot allocation failed");
  }
  const int cur0 = h->cur;
  const long long steps0 = h->steps, launches0 = h->launches;
  PF_CUDA(h, cudaMemcpyAsync(snap_p, h->pop[cur0], pop_b, cudaMemcpyDeviceToDevice, h->stream));
  PF_CUDA(h, cudaMemcpyAsync(snap_a, h->aux[cur0], aux_b, cudaMemcpyDeviceToDevice, h->stream));
  struct Cand { int variant, a, b, persistent; };
  std::vector<Cand> cands;
  for (int ch : {4, 8, 16, 24, 32, 48, 64, 96})
    for (int pers : {0, 1}) cands.push_back({STEP_YMARCH, ch, 0, pers});
  if (!h->thermal && !h->any_bc) {
    if (staged_ok_t<S, R>(h))
      for (int ch : {16, 32, 48, 64, 96, 128})
        for (int pers : {0, 1}) cands.push_back({STEP_STAGED, ch, 0, pers});
    cands.push_back({STEP_TILE, 32, 8, 0});
    cands.push_back({STEP_TILE, 64, 4, 0});
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  Cand bc = cands[0];
  pf_status st = PF_OK;
  for (const Cand& c : cands) {
    h->variant = c.variant;
    if (c.variant != STEP_TILE) h->chunk = c.a; else { h->tx = c.a; h->ty = c.b; }
    h->persistent = c.persistent;
    st = upload_tables(h);
    if (st != PF_OK) break;
    for (int t = 0; t < 2 && st == PF_OK; ++t) st = step_t<S, R>(h, false);
    cudaEventRecord(e0, h->stream);
    for (int t = 0; t < trial_steps && st == PF_OK; ++t) st = step_t<S, R>(h, false);
    cudaEventRecord(e1, h->stream);
    if (st != PF_OK) break;
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) { best = ms; bc = c; }
    // every candidate starts from the same state
    h->cur = cur0;
    cudaMemcpyAsync(h->pop[cur0], snap_p, pop_b, cudaMemcpyDeviceToDevice, h->stream);
    cudaMemcpyAsync(h->aux[cur0], snap_a, aux_b, cudaMemcpyDeviceToDevice, h->stream);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(h->stream);
  dev_free(h, snap_p);
  dev_free(h, snap_a);
  h->cur = cur0;
  h->steps = steps0;
  h->launches = launches0;
  if (st != PF_OK) return st;
  h->variant = bc.variant;
  if (bc.variant != STEP_TILE) h->chunk = bc.a; else { h->tx = bc.a; h->ty = bc.b; }
  h->persistent = bc.persistent;
  for (auto& g : h->gexec)   // graphs captured before hold the old tiles
    if (g) { cudaGraphExecDestroy(g); g = nullptr; }
  h->coop_graph_failed = 0;
  st = upload_tables(h);
  if (st != PF_OK) return st;
  if (out) { out[0] = bc.variant; out[1] = bc.a; out[2] = bc.b; out[3] = bc.persistent; }
  return PF_OK;
}

extern "C" pf_status pf_autotune(pf_handle* h, int trial_steps, int out[4]) {
  if (!h) return PF_ERR_BAD_ARG;
  if (trial_steps < 1 || trial_steps > 10000)
    return fail(h, PF_ERR_BAD_ARG, "trial_steps must be in [1, 10000]");
  for (int d : h->inited)
    if (!d) return fail(h, PF_ERR_STATE, "initialise every domain before autotuning");
  PF_CUDA(h, cudaStreamSynchronize(h->stream));
  return dispatch(h, [&](auto s_t, auto r_t) {
    PF_TYPES(s_t, r_t);
    return autotune_t<S, R>(h, trial_steps, out);
  });
}

extern "C" pf_status pf_get_step_config(const pf_handle* h, int out[3]) {
  if (!h || !out) return PF_ERR_BAD_ARG;
  out[0] = h->variant;
  out[1] = h->variant != STEP_TILE ? h->chunk : h->tx;
  out[2] = h->variant == STEP_TILE ? h->ty : 0;
  return PF_OK;
}

extern "C" pf_status pf_step(pf_handle* h, int n_steps) {
  if (!h) return PF_ERR_BAD_ARG;
  if (n_steps < 0) return fail(h, PF_ERR_BAD_ARG, "n_steps must be >= 0");
  for (int d : h->inited)
    if (!d) return fail(h, PF_ERR_STATE, "every domain must be initialised before stepping");
  return dispatch(h, [&](auto s_t, auto r_t) {
    PF_TYPES(s_t, r_t);
    return step_n<S, R>(h, n_steps);
  });
}

// ---------------------------------------------------------------------------
// outputs
// ---------------------------------------------------------------------------
extern "C" pf_status pf_get_fields(pf_handle* h, int dom, uint32_t mask, double* host_out,
                                   size_t n) {
  if (!h) return PF_ERR_BAD_ARG;
  if (dom < 0 || dom >= (int)h->doms.size() || !host_out || (mask & ~0x1FFu) || !mask)
    return fail(h, PF_ERR_BAD_ARG, "bad domain, mask or output");
  const DomDesc& dd = h->ddesc[dom];
  const size_t nn = (size_t)dd.nx * dd.ny;
  const size_t need = nn * __builtin_popcount(mask);
  if (n < need) return fail(h, PF_ERR_BAD_ARG, "output buffer too small");
  // a page-locked output is written by the kernel in place; others are staged
  double* direct = static_cast<double*>(const_cast<void*>(host_device_view(host_out)));
  pf_status st = ensure_staging(h, direct ? 0 : need);
  if (st != PF_OK) return st;
  double* dst = direct ? direct : h->staging;
  if (h->prec == PF_FP64)
    PF_CUDA(h, launch_fields_to_f64<double>(fields_ptr<double>(h), h->plane_stride, dd.off,
                                            (long long)nn, mask, dst, h->stream));
  else
    PF_CUDA(h, launch_fields_to_f64<float>(fields_ptr<float>(h), h->plane_stride, dd.off,
                                           (long long)nn, mask, dst, h->stream));
  h->launches++;
  if (!direct)
    PF_CUDA(h, cudaMemcpyAsync(host_out, h->staging, need * sizeof(double), cudaMemcpyDeviceToHost,
                               h->stream));
  PF_CUDA(h, cudaStreamSynchronize(h->stream));
  return check_device_error(h);
}

// ---------------------------------------------------------------------------
// fields in, n steps, fields out, with the host copies overlapped
// ---------------------------------------------------------------------------
// The lattice is cut into B row bands of whole tile rows (B <= PF_RUN_BANDS,
// each band at least four tile rows, so that a step of a band reads state
// only from its own band and the two next to it).  Band b lives on its own
// stream: the copy of its rows of psi, C, vx, vy, p, the equilibria of its
// sites, its tiles of every step, its rows of the output fields and their
// copy back.  Its step s waits for step s-1 of bands b-1 and b+1 (periodic),
// which covers both what the step reads and the rows of the buffer it
// overwrites; its first step also waits for the buoyancy reference rho_bar,
// which needs the whole phi plane: that plane is copied first, its FP64 sum
// taken in the order of pf_reduce and rho_bar formed from it on the device
// with the fused product-sum the host uses, so that it is bit for bit the one
// pf_set_fields sets.
template <typename S, typename R>
static pf_status run_banded(pf_handle* h, const double* in6, int n_steps, uint32_t mask,
                            double* out, int B, int th) {
  const DomDesc dd = h->ddesc[0];
  const long long nn = (long long)dd.nx * dd.ny;
  const int ns = __builtin_popcount(mask);
  const int tiles_y = (dd.ny + th - 1) / th;
  std::vector<int> tr(B + 1);
  for (int b = 0; b <= B; ++b) tr[b] = (int)((long long)tiles_y * b / B);
  auto row = [&](int b) { return std::min(tr[b] * th, dd.ny); };
  pf_status st = ensure_staging(h, (size_t)(6 + ns) * nn + REDUCE_BLOCKS + 1);
  if (st != PF_OK) return st;
  double* d_in = h->staging;
  double* d_out = d_in + 6 * nn;
  double* d_part = d_out + (size_t)ns * nn;
  double* d_sum = d_part + REDUCE_BLOCKS;
  // Streams by distance from the periodic seam (between bands B-1 and 0):
  // the bands far from it can run steps ahead of it, so they get the higher
  // priorities, finish first and start their copies back while the bands at
  // the seam still step.
  if (h->run_nb != B) {
    PF_CUDA(h, cudaStreamSynchronize(h->stream));
    int lo = 0, hi = 0;   // least and greatest priority (numerically lo >= hi)
    PF_CUDA(h, cudaDeviceGetStreamPriorityRange(&lo, &hi));
    for (int b = 0; b < B; ++b) {
      if (h->run_st[b]) {
        PF_CUDA(h, cudaStreamSynchronize(h->run_st[b]));
        cudaStreamDestroy(h->run_st[b]);
        h->run_st[b] = nullptr;
      }
      const int dist = std::min(b, B - 1 - b);                 // 0 at the seam
      const int pri = lo - (int)((long long)(lo - hi) * dist / std::max(1, (B - 1) / 2));
      PF_CUDA(h, cudaStreamCreateWithPriority(&h->run_st[b], cudaStreamNonBlocking, pri));
    }
    h->run_nb = B;
  }
  for (int b = 0; b < B; ++b) {
    for (int k = 0; k < 2; ++k)
      if (!h->run_ev[k][b])
        PF_CUDA(h, cudaEventCreateWithFlags(&h->run_ev[k][b], cudaEventDisableTiming));
  }
  if (!h->run_phi) PF_CUDA(h, cudaEventCreateWithFlags(&h->run_phi, cudaEventDisableTiming));
  if (!h->run_ctl) PF_CUDA(h, cudaEventCreateWithFlags(&h->run_ctl, cudaEventDisableTiming));
  cudaStream_t S0 = h->stream;
  st = clear_device_error(h);
  if (st != PF_OK) return st;
  st = upload_grain_table(h, 0, {});
  if (st != PF_OK) return st;
  // phi first; the bands' copies follow it
  PF_CUDA(h, cudaMemcpyAsync(d_in, in6, nn * sizeof(double), cudaMemcpyHostToDevice, S0));
  PF_CUDA(h, cudaEventRecord(h->run_phi, S0));
  PF_CUDA(h, launch_sum_as<R>(d_in, nn, d_part, d_sum, S0));
  // rho_bar written into the device descriptor by a kernel: a copy from the
  // host would queue on the copy engine behind the bands' copies
  PF_CUDA(h, launch_set_rho_bar(h->d_doms, 0, d_sum, (double)nn, h->p.rho_g,
                                h->p.rho_l - h->p.rho_g, S0));
  PF_CUDA(h, cudaEventRecord(h->run_ctl, S0));
  h->launches += 3;
  const int cur = h->cur;
  // the bands' copies one after the other, from the middle band outwards to
  // the seam, so that the middle bands' data arrive (and their steps start)
  // while the rest is still on the way
  std::vector<int> order;
  for (int k = 0; (int)order.size() < B; ++k) {
    const int b = B / 2 + ((k & 1) ? -(k + 1) / 2 : k / 2);
    if (b >= 0 && b < B) order.push_back(b);
  }
  for (int k = 0; k < B; ++k) {
    const int b = order[k];
    cudaStream_t sb = h->run_st[b];
    const long long i0 = (long long)row(b) * dd.nx, i1 = (long long)row(b + 1) * dd.nx;
    PF_CUDA(h, cudaStreamWaitEvent(sb, k == 0 ? h->run_phi : h->run_ev[0][order[k - 1]], 0));
    PF_CUDA(h, cudaMemcpy2DAsync(d_in + nn + i0, nn * sizeof(double), in6 + nn + i0,
                                 nn * sizeof(double), (i1 - i0) * sizeof(double), 5,
                                 cudaMemcpyHostToDevice, sb));
    PF_CUDA(h, cudaEventRecord(h->run_ev[0][b], sb));
    SetFieldsArgs<S, R> a{};
    a.out = reinterpret_cast<S*>(h->pop[cur]);
    a.aout = reinterpret_cast<R*>(h->aux[cur]);
    a.fields = fields_ptr<R>(h);
    a.grain = h->grain;
    a.plane_stride = h->plane_stride;
    a.dom = dd;
    a.f6 = d_in;
    a.grain_ids = nullptr;
    a.kp = make_kparams<R>(h->p);
    a.thermal = 0;
    a.theta0 = h->p.theta0;
    a.err = h->d_err;
    a.i0 = i0;
    a.i1 = i1;
    PF_CUDA(h, launch_set_fields<S, R>(a, sb));
    h->launches++;
    PF_CUDA(h, cudaEventRecord(h->run_ev[1][b], sb));   // "step -1" of band b
  }
  for (int s = 0; s < n_steps; ++s) {
    const int pin = cur ^ (s & 1), pout = pin ^ 1;
    StepArgs<S, R> a = make_step_args<S, R>(h, h->pop[pin], h->aux[pin], h->pop[pout],
                                            h->aux[pout], s + 1 == n_steps);
    for (int b = 0; b < B; ++b) {
      cudaStream_t sb = h->run_st[b];
      if (s == 0) PF_CUDA(h, cudaStreamWaitEvent(sb, h->run_ctl, 0));
      if (B > 1) {
        PF_CUDA(h, cudaStreamWaitEvent(sb, h->run_ev[(s + 1) & 1][(b + B - 1) % B], 0));
        PF_CUDA(h, cudaStreamWaitEvent(sb, h->run_ev[(s + 1) & 1][(b + 1) % B], 0));
      }
      a.tile_base = dd.tile0 + tr[b] * dd.tiles_x;
      a.ntiles = dd.tile0 + tr[b + 1] * dd.tiles_x;
      PF_CUDA(h, launch_step<S, R>(a, h->variant, h->tx, h->ty, a.ntiles - a.tile_base, sb));
      h->launches++;
      PF_CUDA(h, cudaEventRecord(h->run_ev[s & 1][b], sb));
    }
  }
  for (int b = 0; b < B; ++b) {
    cudaStream_t sb = h->run_st[b];
    const long long i0 = (long long)row(b) * dd.nx, i1 = (long long)row(b + 1) * dd.nx;
    PF_CUDA(h, launch_fields_to_f64_range<R>(fields_ptr<R>(h), h->plane_stride, dd.off, nn, i0,
                                             i1, mask, d_out, sb));
    h->launches++;
    PF_CUDA(h, cudaMemcpy2DAsync(out + i0, nn * sizeof(double), d_out + i0, nn * sizeof(double),
                                 (i1 - i0) * sizeof(double), ns, cudaMemcpyDeviceToHost, sb));
    PF_CUDA(h, cudaEventRecord(h->run_ev[0][b], sb));
    PF_CUDA(h, cudaStreamWaitEvent(S0, h->run_ev[0][b], 0));
  }
  PF_CUDA(h, cudaStreamSynchronize(S0));
  PF_CUDA(h, cudaMemcpy(&h->ddesc[0].rho_bar, &h->d_doms[0].rho_bar, sizeof(double),
                        cudaMemcpyDeviceToHost));
  h->cur = cur ^ (n_steps & 1);
  h->steps = n_steps;
  unsigned int bits = 0;
  PF_CUDA(h, cudaMemcpy(&bits, h->d_err, sizeof(bits), cudaMemcpyDeviceToHost));
  if (bits & ERR_NONFINITE_INPUT) {
    h->inited[0] = 0;
    pf_status c = clear_device_error(h);
    if (c != PF_OK) return c;
    PF_CUDA(h, cudaStreamSynchronize(S0));
    return fail(h, PF_ERR_BAD_ARG, "non-finite field value; the domain must be initialised again");
  }
  h->inited[0] = 1;
  return check_device_error(h);
}

extern "C" pf_status pf_run(pf_handle* h, const double* fields6, size_t n, int n_steps,
                            uint32_t mask, double* host_out, size_t n_out) {
  if (!h) return PF_ERR_BAD_ARG;
  if (h->doms.size() != 1) return fail(h, PF_ERR_BAD_ARG, "pf_run takes a single-domain handle");
  if (!fields6 || !host_out || n_steps < 0 || (mask & ~0x1FFu) || !mask)
    return fail(h, PF_ERR_BAD_ARG, "need fields, an output, n_steps >= 0 and a field mask");
  const DomDesc& dd = h->ddesc[0];
  const size_t nn = (size_t)dd.nx * dd.ny;
  if (n != nn) return fail(h, PF_ERR_BAD_ARG, "n must equal nx*ny of the domain");
  if (n_out < nn * __builtin_popcount(mask))
    return fail(h, PF_ERR_BAD_ARG, "output buffer too small");
  const bool strip = h->variant == STEP_YMARCH || h->variant == STEP_STAGED;
  const int th = strip ? h->chunk : h->ty;
  const int B = std::min(PF_RUN_BANDS, ((dd.ny + th - 1) / th) / 4);
  if (n_steps == 0 || h->thermal || h->any_bc || B < 3) {
    // one after the other
    pf_status st = pf_set_fields(h, 0, fields6, nullptr, n);
    if (st != PF_OK) return st;
    st = pf_step(h, n_steps);
    if (st != PF_OK) return st;
    return pf_get_fields(h, 0, mask, host_out, n_out);
  }
  PF_CUDA(h, cudaStreamSynchronize(h->stream));
  return dispatch(h, [&](auto s_t, auto r_t) {
    PF_TYPES(s_t, r_t);
    return run_banded<S, R>(h, fields6, n_steps, mask, host_out, B, th);
  });
}

extern "C" pf_status pf_get_state(pf_handle* h, int dom, double* host_out, size_t n) {
  if (!h) return PF_ERR_BAD_ARG;
  if (dom < 0 || dom >= (int)h->doms.size() || !host_out)
    return fail(h, PF_ERR_BAD_ARG, "bad domain or output");
  const DomDesc& dd = h->ddesc[dom];
  const size_t nn = (size_t)dd.nx * dd.ny;
  const size_t np = (size_t)h->n_phys;
  if (n < nn * np) return fail(h, PF_ERR_BAD_ARG, "output buffer too small");
  pf_status st = ensure_staging(h, nn * np);
  if (st != PF_OK) return st;
  st = dispatch(h, [&](auto s_t, auto r_t) {
    PF_TYPES(s_t, r_t);
    PF_CUDA(h, launch_state_to_f64<S, R>((const S*)h->pop[h->cur], (const R*)h->aux[h->cur],
                                         h->plane_stride, dd.off, (long long)nn, h->staging,
                                         h->thermal, h->stream));
    return PF_OK;
  });
  if (st != PF_OK) return st;
  h->launches++;
  PF_CUDA(h, cudaMemcpyAsync(host_out, h->staging, nn * np * sizeof(double),
                             cudaMemcpyDeviceToHost, h->stream));
  PF_CUDA(h, cudaStreamSynchronize(h->stream));
  return check_device_error(h);
}

extern "C" pf_status pf_set_state(pf_handle* h, int dom, const double* host_in, size_t n) {
  if (!h) return PF_ERR_BAD_ARG;
  if (dom < 0 || dom >= (int)h->doms.size() || !host_in)
    return fail(h, PF_ERR_BAD_ARG, "bad domain or input");
  const DomDesc& dd = h->ddesc[dom];
  const size_t nn = (size_t)dd.nx * dd.ny;
  const size_t np = (size_t)h->n_phys;
  if (n != nn * np)
    return fail(h, PF_ERR_BAD_ARG, "input must hold pf_state_planes(h) planes of nx*ny");
  pf_status st = clear_device_error(h);
  if (st != PF_OK) return st;
  st = ensure_staging(h, nn * np);
  if (st != PF_OK) return st;
  PF_CUDA(h, cudaMemcpyAsync(h->staging, host_in, nn * np * sizeof(double),
                             cudaMemcpyHostToDevice, h->stream));
  st = dispatch(h, [&](auto s_t, auto r_t) {
    PF_TYPES(s_t, r_t);
    PF_CUDA(h, launch_state_from_f64<S, R>((S*)h->pop[h->cur], (R*)h->aux[h->cur],
                                           h->plane_stride, dd.off, (long long)nn, h->staging,
                                           h->thermal, h->stream));
    return PF_OK;
  });
  if (st != PF_OK) return st;
  h->launches++;
  PF_CUDA(h, cudaStreamSynchronize(h->stream));
  h->inited[dom] = 1;
  return PF_OK;
}

template <typename R>
static pf_status reduce_t(pf_handle* h, int dom, const pf_probe* probe) {
  ReduceArgs<R> a{};
  a.fields = fields_ptr<R>(h);
  a.plane_stride = h->plane_stride;
  a.dom = h->ddesc[dom];
  a.probe = probe != nullptr;
  if (probe) { a.xc = probe->xc; a.yc = probe->yc; a.Rp = probe->R; a.W = probe->W; }
  PF_CUDA(h, launch_reduce<R>(a, h->partial, h->d_diag, h->stream));
  h->launches += 2;
  return PF_OK;
}

extern "C" pf_status pf_reduce(pf_handle* h, int dom, const pf_probe* probe, pf_diag* out) {
  if (!h) return PF_ERR_BAD_ARG;
  if (dom < 0 || dom >= (int)h->doms.size() || !out)
    return fail(h, PF_ERR_BAD_ARG, "bad domain or output");
  pf_status st = h->prec == PF_FP64 ? reduce_t<double>(h, dom, probe) : reduce_t<float>(h, dom, probe);
  if (st != PF_OK) return st;
  double buf[NDIAG];
  PF_CUDA(h, cudaMemcpyAsync(buf, h->d_diag, sizeof(buf), cudaMemcpyDeviceToHost, h->stream));
  PF_CUDA(h, cudaStreamSynchronize(h->stream));
  static_assert(sizeof(pf_diag) == NDIAG * sizeof(double), "pf_diag layout");
  std::memcpy(out, buf, sizeof(buf));
  return check_device_error(h);
}

// ---------------------------------------------------------------------------
// boundaries
// ---------------------------------------------------------------------------
extern "C" pf_status pf_set_boundaries(pf_handle* h, int dom, const int bc[4]) {
  if (!h) return PF_ERR_BAD_ARG;
  if (dom < 0 || dom >= (int)h->doms.size() || !bc)
    return fail(h, PF_ERR_BAD_ARG, "bad domain index or NULL bc");
  for (int k = 0; k < 4; ++k)
    if (bc[k] < PF_BC_PERIODIC || bc[k] > PF_BC_INLET_NEE)
      return fail(h, PF_ERR_BAD_ARG, "boundary types are 0 (periodic) .. 6 (extrapolation inlet)");
  if ((bc[0] == PF_BC_PERIODIC) != (bc[1] == PF_BC_PERIODIC) ||
      (bc[2] == PF_BC_PERIODIC) != (bc[3] == PF_BC_PERIODIC))
    return fail(h, PF_ERR_BAD_ARG, "a periodic side needs a periodic opposite side");
  const bool open = bc[0] || bc[1] || bc[2] || bc[3];
  if (open && h->prec != PF_FP32 && h->prec != PF_FP64)
    return fail(h, PF_ERR_BAD_ARG, "non-periodic sides need FP32 or FP64 storage");
  if (h->inited[dom])
    return fail(h, PF_ERR_STATE, "set the boundaries before initialising the domain");
  PF_CUDA(h, cudaStreamSynchronize(h->stream));
  for (int k = 0; k < 4; ++k) h->ddesc[dom].bc[k] = (unsigned char)bc[k];
  h->any_bc = h->any_io = 0;
  for (const DomDesc& d : h->ddesc)
    for (int k = 0; k < 4; ++k) {
      if (d.bc[k]) h->any_bc = 1;
      if (d.bc[k] == PF_BC_INLET || d.bc[k] == PF_BC_OUTLET || d.bc[k] == PF_BC_INLET_NEE)
        h->any_io = 1;
    }
  if (h->any_bc && h->variant != STEP_YMARCH) {
    h->variant = STEP_YMARCH;
    h->chunk = 32;
  }
  for (auto& g : h->gexec)
    if (g) { cudaGraphExecDestroy(g); g = nullptr; }
  return upload_tables(h);
}

// ---------------------------------------------------------------------------
// thermal mode
// ---------------------------------------------------------------------------
extern "C" int pf_state_planes(const pf_handle* h) { return h ? h->n_phys : -1; }

extern "C" pf_status pf_set_temperature(pf_handle* h, int dom, const double* theta, size_t n) {
  if (!h) return PF_ERR_BAD_ARG;
  if (!h->thermal) return fail(h, PF_ERR_BAD_ARG, "the handle is not in thermal mode");
  if (dom < 0 || dom >= (int)h->doms.size() || !theta)
    return fail(h, PF_ERR_BAD_ARG, "bad domain index or NULL theta");
  if (!h->inited[dom]) return fail(h, PF_ERR_STATE, "initialise the domain first");
  if (h->steps != 0) return fail(h, PF_ERR_STATE, "set the temperature before the first step");
  const DomDesc& dd = h->ddesc[dom];
  const size_t nn = (size_t)dd.nx * dd.ny;
  if (n != nn) return fail(h, PF_ERR_BAD_ARG, "n must equal nx*ny of the domain");
  pf_status st = ensure_staging(h, nn + 1);
  if (st != PF_OK) return st;
  PF_CUDA(h, cudaMemcpyAsync(h->staging, theta, nn * sizeof(double), cudaMemcpyHostToDevice,
                             h->stream));
  {
    // non-finite values are found on the device, before the state is touched
    unsigned int* flag = reinterpret_cast<unsigned int*>(h->staging + nn);
    unsigned int bits = 0;
    PF_CUDA(h, launch_flag_nonfinite(h->staging, (long long)nn, flag, h->stream));
    h->launches++;
    PF_CUDA(h, cudaMemcpyAsync(&bits, flag, sizeof(bits), cudaMemcpyDeviceToHost, h->stream));
    PF_CUDA(h, cudaStreamSynchronize(h->stream));
    if (bits) return fail(h, PF_ERR_BAD_ARG, "non-finite temperature");
  }
  st = dispatch(h, [&](auto s_t, auto r_t) {
    PF_TYPES(s_t, r_t);
    PF_CUDA(h, launch_set_temperature<S, R>((S*)h->pop[h->cur], (R*)h->aux[h->cur],
                                            fields_ptr<R>(h), h->plane_stride, dd, h->staging,
                                            make_kparams<R>(h->p), h->stream));
    return PF_OK;
  });
  if (st != PF_OK) return st;
  h->launches++;
  PF_CUDA(h, cudaStreamSynchronize(h->stream));
  return PF_OK;
}

extern "C" pf_status pf_reduce_thermal(pf_handle* h, int dom, double out[3]) {
  if (!h) return PF_ERR_BAD_ARG;
  if (!h->thermal) return fail(h, PF_ERR_BAD_ARG, "the handle is not in thermal mode");
  if (dom < 0 || dom >= (int)h->doms.size() || !out)
    return fail(h, PF_ERR_BAD_ARG, "bad domain or output");
  const DomDesc& dd = h->ddesc[dom];
  pf_status st = dispatch(h, [&](auto s_t, auto r_t) {
    PF_TYPES(s_t, r_t);
    PF_CUDA(h, launch_reduce_thermal<S, R>((const S*)h->pop[h->cur], fields_ptr<R>(h),
                                           h->plane_stride, dd, h->partial, h->d_diag,
                                           h->stream));
    return PF_OK;
  });
  if (st != PF_OK) return st;
  h->launches += 2;
  PF_CUDA(h, cudaMemcpyAsync(out, h->d_diag, 3 * sizeof(double), cudaMemcpyDeviceToHost,
                             h->stream));
  PF_CUDA(h, cudaStreamSynchronize(h->stream));
  return check_device_error(h);
}

// ---------------------------------------------------------------------------
// discrete adjoint
// ---------------------------------------------------------------------------
template <typename S, typename R>
static pf_status adjoint_t(pf_handle* h, int n, const pf_objective* obj, double* J_out,
                           double* grad) {
  const DomDesc dd = h->ddesc[0];
  const size_t ps = (size_t)h->plane_stride;
  const size_t pop_b = ps * N_POP * sizeof(S), aux_b = ps * N_AUX * sizeof(R);
  const size_t state_b = (pop_b + 255) / 256 * 256 + (aux_b + 255) / 256 * 256;
  const int K = obj->checkpoint_every;
  const int nseg = (n + K - 1) / K;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  const int tiles = ((dd.nx + ADJ_TX - 1) / ADJ_TX) * ((dd.ny + ADJ_TY - 1) / ADJ_TY);
  const int grid = std::max(1, std::min(tiles, 4 * std::max(sms, 1)));
  const int oblocks = 256;
  const size_t lam_b = ps * N_PHYS * sizeof(R), ai_b = ps * N_AI * sizeof(R);
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  // Workspace: a checkpoint per segment but the last, whose states the
  // forward sweep keeps in full; two segment buffers, so that the
  // recomputation of segment s-1 (on a second stream) overlaps the reverse
  // sweep of segment s, or one if the device cannot hold two.
  auto need_for = [&](int nbuf) {
    return (size_t)(nseg - 1) * state_b + (size_t)nbuf * K * state_b + 2 * up(lam_b) +
           up(ai_b) + up((size_t)grid * 3 * sizeof(double)) +
           up((size_t)oblocks * sizeof(double));
  };
  int nbuf = nseg > 1 ? 2 : 1;
  if (need_for(nbuf) > h->adj_ws_bytes) {
    PF_CUDA(h, cudaStreamSynchronize(h->stream));
    dev_free(h, h->adj_ws);
    h->adj_ws = nullptr;
    h->adj_ws_bytes = 0;
    for (; nbuf >= 1 && !h->adj_ws; --nbuf) {
      h->adj_ws = dev_alloc(h, need_for(nbuf));
      if (h->adj_ws) h->adj_ws_bytes = need_for(nbuf);
      else cudaGetLastError();    // clear the failed allocation
    }
    ++nbuf;
    if (!h->adj_ws) return fail(h, PF_ERR_OOM, "adjoint workspace allocation failed");
  }
  char* w = static_cast<char*>(h->adj_ws);
  auto take = [&](size_t b) { char* p = w; w += up(b); return p; };
  std::vector<char*> ck(nseg > 1 ? nseg - 1 : 0);
  for (auto& c : ck) c = take(state_b);
  std::vector<char*> sg[2];
  for (int b = 0; b < nbuf; ++b) {
    sg[b].resize(K);
    for (int i = 0; i < K; ++i) sg[b][i] = take(state_b);
  }
  R* lam[2] = {reinterpret_cast<R*>(take(lam_b)), reinterpret_cast<R*>(take(lam_b))};
  R* ai = reinterpret_cast<R*>(take(ai_b));
  double* partial = reinterpret_cast<double*>(take((size_t)grid * 3 * sizeof(double)));
  double* opart = reinterpret_cast<double*>(take((size_t)oblocks * sizeof(double)));
  auto pop_of = [&](char* st) { return (void*)st; };
  auto aux_of = [&](char* st) { return (void*)(st + up(pop_b)); };
  auto buf_of = [&](int seg) -> std::vector<char*>& { return sg[nbuf == 2 ? (seg & 1) : 0]; };
  const bool fresh = h->steps == 0;
  cudaStream_t A = h->stream;

  // forward sweep: a checkpoint every K steps; the last segment's input
  // states stay in its segment buffer, and its last step writes the handle's
  // state and fields
  const int t_last = (nseg - 1) * K;
  for (int t = 0; t < t_last; ++t) {
    if (t % K == 0) {
      PF_CUDA(h, cudaMemcpyAsync(pop_of(ck[t / K]), h->pop[h->cur], pop_b,
                                 cudaMemcpyDeviceToDevice, A));
      PF_CUDA(h, cudaMemcpyAsync(aux_of(ck[t / K]), h->aux[h->cur], aux_b,
                                 cudaMemcpyDeviceToDevice, A));
    }
    pf_status st = step_t<S, R>(h, false);
    if (st != PF_OK) return st;
  }
  {
    std::vector<char*>& bl = buf_of(nseg - 1);
    const int L = n - t_last;
    PF_CUDA(h, cudaMemcpyAsync(pop_of(bl[0]), h->pop[h->cur], pop_b, cudaMemcpyDeviceToDevice, A));
    PF_CUDA(h, cudaMemcpyAsync(aux_of(bl[0]), h->aux[h->cur], aux_b, cudaMemcpyDeviceToDevice, A));
    for (int j = 0; j < L; ++j) {
      const bool last = j + 1 == L;
      const StepArgs<S, R> a = make_step_args<S, R>(
          h, pop_of(bl[j]), aux_of(bl[j]), last ? h->pop[h->cur ^ 1] : pop_of(bl[j + 1]),
          last ? h->aux[h->cur ^ 1] : aux_of(bl[j + 1]), last);
      pf_status sl = launch_all<S, R>(h, a, A);
      if (sl != PF_OK) return sl;
    }
    h->cur ^= 1;
    h->steps += L;
  }
  // objective J(x_T) and its adjoint lambda_T
  pf_diag dg{};
  pf_status st = pf_reduce(h, 0, nullptr, &dg);
  if (st != PF_OK) return st;
  const double N = (double)dd.nx * dd.ny;
  if (!(dg.gas > 0.0) && obj->w_centroid != 0.0)
    return fail(h, PF_ERR_BAD_ARG, "bubble centroid objective needs gas in the domain");
  const double yc = dg.gas > 0.0 ? dg.gas_y / dg.gas : 0.0;
  const double J = obj->w_solid * dg.sum_hpsi / N + obj->w_centroid * yc / dd.ny;
  PF_CUDA(h, launch_adj_objective<R>(lam[0], dd, (long long)ps, obj->w_solid, obj->w_centroid,
                                     yc, dg.gas > 0.0 ? dg.gas : 1.0, A));
  PF_CUDA(h, cudaMemsetAsync(partial, 0, (size_t)grid * 3 * sizeof(double), A));
  h->launches++;

  // recomputation of segment s < nseg - 1 from its checkpoint into its buffer
  auto recompute = [&](int s, cudaStream_t sx) -> pf_status {
    std::vector<char*>& b = buf_of(s);
    PF_CUDA(h, cudaMemcpyAsync(pop_of(b[0]), pop_of(ck[s]), pop_b, cudaMemcpyDeviceToDevice, sx));
    PF_CUDA(h, cudaMemcpyAsync(aux_of(b[0]), aux_of(ck[s]), aux_b, cudaMemcpyDeviceToDevice, sx));
    for (int j = 0; j + 1 < K; ++j) {
      const StepArgs<S, R> a = make_step_args<S, R>(h, pop_of(b[j]), aux_of(b[j]),
                                                    pop_of(b[j + 1]), aux_of(b[j + 1]), false);
      pf_status sl = launch_all<S, R>(h, a, sx);
      if (sl != PF_OK) return sl;
    }
    return PF_OK;
  };
  // reverse sweep of segment s, on the handle's stream
  const double dfs = 6.0 / (h->p.W_phi * std::sqrt(2.0 * h->p.beta_phi));
  int cl = 0;
  auto reverse = [&](int s) -> pf_status {
    const int t0 = s * K, L = std::min(n, t0 + K) - t0;
    std::vector<char*>& b = buf_of(s);
    for (int j = L - 1; j >= 0; --j) {
      AdjArgs<S, R> aa{};
      aa.step = make_step_args<S, R>(h, pop_of(b[j]), aux_of(b[j]), nullptr, nullptr, false);
      aa.dom = dd;
      aa.lam_in = lam[cl];
      aa.lam_out = lam[cl ^ 1];
      aa.ai = ai;
      aa.partial = partial;
      aa.dfs_dsigma = dfs;
      PF_CUDA(h, launch_adjoint_step<S, R>(aa, grid, A));
      h->launches += ADJ_LAUNCHES_PER_STEP;
      cl ^= 1;
    }
    return PF_OK;
  };
  if (nbuf == 1) {
    for (int s = nseg - 1; s >= 0; --s) {
      if (s < nseg - 1 && (st = recompute(s, A)) != PF_OK) return st;
      if ((st = reverse(s)) != PF_OK) return st;
    }
  } else {
    // Stream B recomputes segment s - 1 while A reverses segment s.  The
    // buffer of segment s - 2 is the one of segment s: B waits for A's
    // reverse of s before it overwrites it, and A waits for B's recompute of
    // a segment before it reverses it.
    if (!h->adj_stream)
      PF_CUDA(h, cudaStreamCreateWithFlags(&h->adj_stream, cudaStreamNonBlocking));
    cudaStream_t B = h->adj_stream;
    struct Events {
      std::vector<cudaEvent_t> ev;
      ~Events() { for (cudaEvent_t e : ev) cudaEventDestroy(e); }
    } evs;
    auto new_event = [&](cudaEvent_t* e) -> pf_status {
      PF_CUDA(h, cudaEventCreateWithFlags(e, cudaEventDisableTiming));
      evs.ev.push_back(*e);
      return PF_OK;
    };
    std::vector<cudaEvent_t> ev_rec(nseg, nullptr), ev_rev(nseg, nullptr);
    cudaEvent_t ev_fwd;
    if ((st = new_event(&ev_fwd)) != PF_OK) return st;
    for (int s = 0; s < nseg; ++s)
      if ((st = new_event(&ev_rec[s])) != PF_OK || (st = new_event(&ev_rev[s])) != PF_OK)
        return st;
    PF_CUDA(h, cudaEventRecord(ev_fwd, A));
    PF_CUDA(h, cudaStreamWaitEvent(B, ev_fwd, 0));
    if ((st = recompute(nseg - 2, B)) != PF_OK) return st;
    PF_CUDA(h, cudaEventRecord(ev_rec[nseg - 2], B));
    for (int s = nseg - 1; s >= 0; --s) {
      if (s < nseg - 1) PF_CUDA(h, cudaStreamWaitEvent(A, ev_rec[s], 0));
      if ((st = reverse(s)) != PF_OK) return st;
      PF_CUDA(h, cudaEventRecord(ev_rev[s], A));
      if (s - 2 >= 0) {
        PF_CUDA(h, cudaStreamWaitEvent(B, ev_rev[s], 0));
        if ((st = recompute(s - 2, B)) != PF_OK) return st;
        PF_CUDA(h, cudaEventRecord(ev_rec[s - 2], B));
      }
    }
  }
  std::vector<double> hp((size_t)grid * 3), ho(oblocks, 0.0);
  if (fresh) {
    // the initial state is checkpoint 0, or the first state of the only segment
    char* x0 = nseg > 1 ? ck[0] : buf_of(0)[0];
    double der[3];
    pf_params_derived(&h->p, der);
    PF_CUDA(h, launch_adj_omega_init<S, R>(lam[cl], (const S*)pop_of(x0), (const R*)aux_of(x0),
                                           dd, (long long)ps, der[0], h->p.k, opart, oblocks, A));
    h->launches++;
    PF_CUDA(h, cudaMemcpyAsync(ho.data(), opart, oblocks * sizeof(double), cudaMemcpyDeviceToHost,
                               A));
  }
  PF_CUDA(h, cudaMemcpyAsync(hp.data(), partial, hp.size() * sizeof(double),
                             cudaMemcpyDeviceToHost, A));
  PF_CUDA(h, cudaStreamSynchronize(A));
  double g[3] = {0.0, 0.0, 0.0};
  for (int b = 0; b < grid; ++b)
    for (int q = 0; q < 3; ++q) g[q] += hp[(size_t)b * 3 + q];
  for (int b = 0; b < oblocks; ++b) g[1] += ho[b];
  if (J_out) *J_out = J;
  for (int q = 0; q < 3; ++q) grad[q] = g[q];
  return PF_OK;
}

extern "C" pf_status pf_adjoint_step(pf_handle* h, int n_steps, const pf_objective* obj,
                                     double* J_out, double grad_out[3]) {
  if (!h) return PF_ERR_BAD_ARG;
  if (!obj || !grad_out || n_steps < 1 || obj->checkpoint_every < 1)
    return fail(h, PF_ERR_BAD_ARG, "need n_steps >= 1, an objective and checkpoint_every >= 1");
  if (h->doms.size() != 1) return fail(h, PF_ERR_BAD_ARG, "the adjoint takes a single-domain handle");
  if (h->prec != PF_FP32 && h->prec != PF_FP64)
    return fail(h, PF_ERR_BAD_ARG, "the adjoint supports the FP32 and FP64 storage forms");
  if (h->thermal)
    return fail(h, PF_ERR_BAD_ARG, "the adjoint covers the isothermal model (thermal = 0) only");
  if (h->any_bc)
    return fail(h, PF_ERR_BAD_ARG, "the adjoint covers periodic domains only");
  if (!h->inited[0]) return fail(h, PF_ERR_STATE, "initialise the domain before the adjoint");
  if (!std::isfinite(obj->w_solid) || !std::isfinite(obj->w_centroid))
    return fail(h, PF_ERR_BAD_ARG, "objective weights must be finite");
  if (h->prec == PF_FP64) return adjoint_t<double, double>(h, n_steps, obj, J_out, grad_out);
  return adjoint_t<float, float>(h, n_steps, obj, J_out, grad_out);
}
