/*
 * pf.h -- C ABI of the GB300 (sm_103a) library for one coupled lattice
 * Boltzmann step of the gas-liquid-dendrite phase-field model of Zhan, Chai,
 * Sun, Shi, Geng and Jiang, "Phase-field modeling of dendritic growth with gas
 * bubbles in the solidification of binary alloys" (arXiv 2407.01651).
 *
 * Conventions (all entry points):
 *  - Every call returns a pf_status; 0 is success, negative values are errors.
 *    Nothing aborts or exits.  pf_last_error() gives a one-line reason.
 *  - Argument errors are reported synchronously.  Errors raised by device work
 *    are reported by the next call that synchronises the stream
 *    (pf_get_fields, pf_get_state, pf_reduce, pf_sync, pf_destroy).
 *  - The handle owns every device buffer it allocates.  When an allocator is
 *    given to pf_create, all device memory comes from it and goes back to it.
 *  - All device work is enqueued on the CUDA stream given to pf_create.  Host
 *    buffers belong to the caller.  A handle is not thread-safe.
 *  - Lattices are periodic, row-major [y][x] with x fastest, in lattice units
 *    (dx = dt = 1).  Host arrays are FP64 regardless of the storage precision.
 */
#ifndef PF_H_
#define PF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PF_OK = 0,
  PF_ERR_BAD_ARG = -1,   /* an argument is out of range or inconsistent        */
  PF_ERR_OOM = -2,       /* device or host allocation failed                   */
  PF_ERR_CUDA = -3,      /* a CUDA call failed (reason in pf_last_error)       */
  PF_ERR_TIMEOUT = -4,   /* a bounded device-side wait gave up                 */
  PF_ERR_NAN = -5,       /* a non-finite value was detected in the fields      */
  PF_ERR_STATE = -6      /* call out of order (e.g. step before init)          */
} pf_status;

/* Storage precision of the populations.  Arithmetic is FP64 for PF_FP64 and
 * FP32 otherwise; the 16-bit forms store populations as offsets from the rest
 * equilibrium. */
typedef enum {
  PF_FP64 = 0,
  PF_FP32 = 1,
  PF_FP16_OFFSET = 2,
  PF_BF16_OFFSET = 3
} pf_precision;

/* Model parameters in the paper's symbols, lattice units.
 *  rho_l, rho_g   liquid / gas density, material interpolation of Section 2.2
 *  nu             kinematic viscosity, mu = rho nu
 *  sigma          gas-liquid surface tension (surface tension force, Sec. 2.2)
 *  W_phi, M_phi   CAC interface width and mobility (Eq. eq-ACE)
 *  beta_phi, beta_psi, beta_inter   double-well / interaction heights
 *                 (Eq. eq-douWell, eq-f3Inter); the paper uses 1/4, 1/4, 3/4
 *  W0, tau0       dendrite interface width and relaxation time (Eq. eq-AnACE)
 *  eps_s          fourfold anisotropy strength (anisotropy function, Sec. 3.3),
 *                 in [0, 0.25); above 1/15 the interface stiffness is negative
 *                 along <11> (corners form)
 *  k              partition coefficient
 *  D              solute diffusivity in the liquid
 *  Omega          solutal undercooling; theta_sys and M c_inf follow from it
 *                 (Eq. eq-Tsys) and F(U) = 1
 *  g              gravity magnitude, acting along -y
 *  grad_eps       regularisation of |grad X| in interface normals
 *  grad_eps_at    regularisation of |grad psi| in the antitrapping direction
 *  s_e, s_eps     free MRT rates of the NS energy moments (default 1)
 * lambda' = 15 lambda / 16 is derived as D tau0 / (a2' W0^2), a2' = 47/75
 * (thin-interface limit, Appendix A).
 * Temperature coupling (Section 2.1, Appendix B), used when thermal = 1:
 *  Le             Lewis number alpha / D; alpha = k_T / (rho_l c_p) is the
 *                 melt's thermal diffusivity, F(U) = 1/Le + M c_inf [1 + (1-k) U]
 *  latent         c_p^s / c_p: theta = H / c_p + latent h(psi)
 *  theta0         uniform initial temperature (pf_set_temperature sets a field)
 *  cp             lattice heat capacity c_p (a numerical constant: the equation
 *                 depends on k_T / c_p only); rho_g * cp >= 2/3 is required
 *                 for the rest population rho H + (w_0 - 1) theta to keep the
 *                 scheme stable in the gas
 *  thermal        0: isothermal closure theta = theta_sys, F = 1 (Eq. eq-Tsys);
 *                 1: temperature lattice (FP32 / FP64 storage, y-march
 *                 traversal; no adjoint)
 *  vin_x, vin_y   velocity at an inlet side (PF_BC_INLET)
 *  reserved       must be 0 */
typedef struct pf_params {
  double rho_l, rho_g, nu, sigma, W_phi, M_phi;
  double beta_phi, beta_psi, beta_inter;
  double W0, tau0, eps_s, k, D, Omega, g;
  double grad_eps, grad_eps_at, s_e, s_eps;
  double Le, latent, theta0, cp;
  double vin_x, vin_y;
  int thermal, reserved;
} pf_params;

/* One periodic domain of an ensemble.  eps_s < 0 uses pf_params.eps_s;
 * otherwise it must be below 0.25. */
typedef struct pf_domain {
  int nx, ny;
  double eps_s;
} pf_domain;

/* Optional device allocator (e.g. a framework's caching allocator). */
typedef struct pf_allocator {
  void *ctx;
  void *(*alloc)(void *ctx, size_t bytes, void *stream);
  void (*free)(void *ctx, void *ptr, void *stream);
} pf_allocator;

/* Initial seeds and bubbles of one domain.  seeds: n_seeds x (x, y, theta),
 * theta the grain orientation; bubbles: n_bubbles x (x, y, R). */
typedef struct pf_init_spec {
  int n_seeds;
  const double *seeds;
  double R_s;
  int n_bubbles;
  const double *bubbles;
} pf_init_spec;

/* FP64 diagnostics of one domain (pf_reduce). */
typedef struct pf_diag {
  double sum_phi;      /* sum phi: conserved by Eq. eq-ACE                    */
  double sum_C;        /* sum C: conserved by the solute equation             */
  double sum_hpsi;     /* sum h(psi) = sum (1+psi)/2; solid fraction x N       */
  double gas;          /* sum (1 - phi)                                       */
  double gas_x, gas_y; /* sum x (1 - phi), sum y (1 - phi): bubble centroid   */
  double p_in_sum, p_in_n, p_out_sum, p_out_n;  /* Laplace probe (Eq. eq-laplace) */
  double max_v;        /* max |v|                                             */
  double nonfinite;    /* number of sites with a non-finite field             */
} pf_diag;

/* Laplace probe: circle centre (xc, yc), radius R, interface width W;
 * inside r < R - 2W, outside r > R + 4W. */
typedef struct pf_probe {
  double xc, yc, R, W;
} pf_probe;

/* Field selection bits for pf_get_fields (order of the output planes). */
enum {
  PF_FIELD_PHI = 1u << 0,  /* bubble order parameter phi                   */
  PF_FIELD_PSI = 1u << 1,  /* dendrite order parameter psi                 */
  PF_FIELD_C = 1u << 2,    /* dimensionless concentration C = c / c_inf     */
  PF_FIELD_U = 1u << 3,    /* supersaturation U                             */
  PF_FIELD_P = 1u << 4,    /* pressure p                                    */
  PF_FIELD_VX = 1u << 5,
  PF_FIELD_VY = 1u << 6,
  PF_FIELD_MU = 1u << 7,   /* chemical potential mu_phi (0 before a step)   */
  PF_FIELD_THETA = 1u << 8 /* temperature theta (theta_sys when isothermal) */
};

/* Number of FP64 planes of the raw state (pf_get_state / pf_set_state):
 * f[9] (NS, post-collision), h[9] (CAC, post-collision), g_pre[5], g_post[5],
 * r = 1/a_s^2, s[5] (solute, post-collision), phi, C, vx, vy, Q_psi of the
 * last step. */
#define PF_STATE_PLANES 39
/* Thermal mode: 6 more planes, e[5] (temperature populations, post-collision)
 * and H of the last step; pf_state_planes() gives the count of a handle. */
#define PF_STATE_PLANES_THERMAL 45

typedef struct pf_handle pf_handle;

/* Default parameters: the 128^2 / 4096^2 benchmark set (rho_l/rho_g = 10,
 * nu = 0.1, sigma = 1e-3, W = 4, eps_s = 0.05, Omega = 0.55, k = 0.15,
 * D = 0.1, g = 1e-6, tau0 = 320 from D tau0 / W0^2 = 2).  Never fails for a
 * non-null pointer. */
pf_status pf_params_default(pf_params *out);

/* Derived coefficients, for inspection: out[0] lambda' (Appendix A),
 * out[1] M c_inf, out[2] theta_sys (Eq. eq-Tsys).  Errors: BAD_ARG (NULL). */
pf_status pf_params_derived(const pf_params *p, double out[3]);

/* Create a handle for n_doms periodic domains (n_doms >= 1, each nx, ny in
 * [4, 65536]; fewer than 2^32 sites in all, each domain padded to a multiple
 * of 64).  cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * alloc may be NULL (cudaMalloc).  Allocates two copies of the 39-plane state
 * (about 2 x 160 B per site in FP32), the field planes and reduction scratch.
 * Errors: BAD_ARG, OOM, CUDA. */
pf_status pf_create(const pf_params *p, const pf_domain *doms, int n_doms,
                    pf_precision prec, void *cuda_stream, const pf_allocator *alloc,
                    pf_handle **out);

/* Initialise domain dom from seeds and bubbles (Eqs. eq-phiEq, eq-psiEq;
 * populations at equilibrium, v = 0, p = 0).  Grain orientation of each site
 * is that of the nearest seed.  Copies the spec to the device (synchronous
 * with respect to the host arrays).  Errors: BAD_ARG, OOM, CUDA. */
pf_status pf_init_fields(pf_handle *h, int dom, const pf_init_spec *spec);

/* Initialise domain dom from macroscopic fields (host, FP64, n = nx*ny each):
 * fields6 = [phi, psi, C, vx, vy, p] planes, one contiguous block of 6 n
 * doubles (page-locked host memory is read by the kernel in place over the
 * CPU-GPU link; other memory is copied to a device staging buffer first); theta (per-site
 * grain angle) may be NULL for 0.  Populations are set to their equilibria.
 * Non-finite values are detected on the device while the equilibria are
 * written: the call then returns BAD_ARG and the domain counts as not
 * initialised until it is set again.  Synchronises the stream.
 * Errors: BAD_ARG, OOM, CUDA. */
pf_status pf_set_fields(pf_handle *h, int dom, const double *fields6, const double *theta,
                        size_t n);

/* Advance every domain by n_steps coupled steps (Section 3 unified LBE and
 * Appendix B).  n_steps >= 0.  Enqueued on the stream; returns without
 * waiting.  Errors: STATE (no init), CUDA. */
pf_status pf_step(pf_handle *h, int n_steps);

/* Traversal of the step kernel (same arithmetic, results identical to
 * rounding order): variant 0 = 2-D tiles of a x b sites (a a multiple of 32,
 * a*b <= 256); variant 1 = column strips of 128 sites marched along y in
 * tiles of a rows (b ignored; the default for FP32/FP64, a = 32); variant 2 =
 * the same strips with their input rows staged in shared memory by bulk
 * copies (b ignored; the default for FP16/BF16 storage, a = 48; needs every
 * domain's nx to be a multiple of 16 bytes of storage: 4 FP32, 8 FP16/BF16,
 * 2 FP64 sites).  Synchronises the stream and rebuilds the tile table.
 * Errors: BAD_ARG. */
pf_status pf_set_step_config(pf_handle *h, int variant, int a, int b);

/* How a step is launched over an ensemble of domains:
 *  per_domain = 0: one launch whose tile list spans every domain (default);
 *               1: one launch per domain, one after the other.
 *  persistent = 1: the grid is the device's resident CTAs of the step kernel,
 *               each looping over tiles; 0: one CTA per tile (default);
 *               2: as 1, and every step of a pf_step call in one cooperative
 *               launch, the resident CTAs meeting at a grid-wide barrier
 *               between steps (y-march traversal over periodic domains, with
 *               per_domain = 0; elsewhere it runs as 1).
 *  graph_steps > 0 (even): pf_step replays CUDA graphs of graph_steps steps
 *               (captured on an internal stream on first use, replayed on the
 *               handle's stream; with persistent = 2 a graph holds one launch
 *               of graph_steps steps); 0 launches step by step (default).
 * Synchronises the stream.  Errors: BAD_ARG (also persistent = 2 without
 * cooperative launch on the device). */
pf_status pf_set_launch(pf_handle *h, int per_domain, int persistent, int graph_steps);

/* Autotuner: times every step traversal and tile height (and persistent or
 * not) on the handle's own domains for trial_steps steps each, starting every
 * candidate from a snapshot of the current state, restores that state and
 * keeps the fastest configuration.  out (may be NULL): variant, a, b,
 * persistent.  Errors: BAD_ARG, STATE, OOM, CUDA. */
pf_status pf_autotune(pf_handle *h, int trial_steps, int out[4]);

/* Current traversal: out[0] variant, out[1] a, out[2] b.  Errors: BAD_ARG
 * (NULL). */
pf_status pf_get_step_config(const pf_handle *h, int out[3]);

/* Copy the fields of the last step of domain dom to host_out (FP64,
 * popcount(mask) planes of nx*ny, in bit order).  n is the capacity of
 * host_out in doubles.  A page-locked host_out is written by the kernel in
 * place over the CPU-GPU link; other memory goes through a device staging
 * buffer.  Synchronises the stream.  Errors: BAD_ARG (domain, mask, NULL,
 * host_out too small), OOM (staging), CUDA, TIMEOUT (a staged step's wait ran
 * out: the fields are invalid). */
pf_status pf_get_fields(pf_handle *h, int dom, uint32_t mask, double *host_out, size_t n);

/* pf_set_fields(h, 0, fields6, NULL, n), pf_step(h, n_steps) and
 * pf_get_fields(h, 0, mask, host_out, n_out) in one call, with the same
 * result bit for bit (Section 3 unified LBE and Appendix B for the steps), for
 * a single-domain handle.  The host copies overlap the steps: the lattice is
 * cut into up to 32 bands of four or more tile rows, each on its own stream, whose
 * copy, equilibria, steps and copy back run as soon as the bands next to it
 * allow (a band's step reads state only from its own band and its two
 * neighbours).  phi is copied first: the buoyancy reference (the mean
 * density) needs all of it before the first step.  fields6: the six planes
 * of pf_set_fields (n = nx*ny each); host_out: popcount(mask) planes as
 * pf_get_fields (n_out doubles).  Page-locked host buffers let the copies run
 * beside the steps; pageable ones work, with less overlap.  The bands' streams
 * are prioritised by distance from the periodic seam (the band pair that
 * waits for everything), so that the middle bands finish first and their
 * copies back overlap the last steps of the rest; with more bands than
 * hardware work queues (CUDA_DEVICE_MAX_CONNECTIONS, 8 unless the process
 * sets it, up to 32) bands that share a queue wait on one another.  Device
 * staging of (6 + popcount(mask)) n doubles is allocated on first use and
 * kept.  The launch mode of pf_set_launch is not used (one launch per band
 * and step).  Runs the three
 * calls one after the other for n_steps = 0, the thermal mode, non-periodic
 * sides or fewer than 12 tile rows.  Non-finite input: BAD_ARG and the domain
 * counts as not initialised, as pf_set_fields.  Synchronises the stream.
 * Errors: BAD_ARG, STATE, OOM, CUDA, TIMEOUT. */
pf_status pf_run(pf_handle *h, const double *fields6, size_t n, int n_steps, uint32_t mask,
                 double *host_out, size_t n_out);

/* Raw state of domain dom (pf_state_planes(h) planes, FP64) to / from the
 * host: checkpoint and restart.  Synchronise the stream.  pf_set_state marks
 * the domain initialised.  Errors: BAD_ARG (domain, NULL, a buffer of the
 * wrong size: at least / exactly planes x nx x ny values), OOM (staging),
 * CUDA; pf_get_state also TIMEOUT (a staged step's wait ran out before the
 * call: the state is invalid), which pf_set_state clears. */
pf_status pf_get_state(pf_handle *h, int dom, double *host_out, size_t n);
pf_status pf_set_state(pf_handle *h, int dom, const double *host_in, size_t n);

/* FP64 reductions of domain dom's last-step fields (conservation of gas and
 * solute, solid fraction, bubble centroid, Laplace pressure jump).  probe may
 * be NULL.  Synchronises the stream.  Errors: BAD_ARG, CUDA. */
pf_status pf_reduce(pf_handle *h, int dom, const pf_probe *probe, pf_diag *out);

/* Final-state objective of the discrete adjoint:
 *   J = w_solid * mean h(psi_T) + w_centroid * y_c(T) / L_y,
 * with h(psi) = (1+psi)/2 the solid fraction and y_c = sum y (1-phi) /
 * sum (1-phi) the bubble centroid height (rows).  The reverse sweep stores a
 * checkpoint every `checkpoint_every` steps and recomputes the steps in
 * between. */
typedef struct pf_objective {
  double w_solid;
  double w_centroid;
  int checkpoint_every;
} pf_objective;

/* Discrete adjoint of the coupled step (reverse mode, hand-written kernels):
 * advances the handle n_steps from its current state exactly as pf_step would
 * (the state afterwards is x_T), evaluates J(x_T) and sweeps back, returning
 * *J_out (may be NULL) and grad_out = dJ/d(eps_s, Omega, sigma) of the whole
 * discrete trajectory.  When the handle has not stepped since its
 * initialisation, the Omega-dependence of the initial lagged Q_psi is
 * included.  Single-domain handles, FP32 or FP64 storage.  Allocates a
 * workspace of (n_steps/K - 1 + 2 K) states plus adjoint planes on first use
 * (n_steps/K - 1 + K states if two segment buffers do not fit; the
 * recomputation of a segment then no longer overlaps the reverse sweep of
 * the next, on an internal second stream).  Synchronises the stream.
 * Errors: BAD_ARG, STATE, OOM, CUDA. */
pf_status pf_adjoint_step(pf_handle *h, int n_steps, const pf_objective *obj, double *J_out,
                          double grad_out[3]);

/* Wait for all enqueued work; reports deferred device errors: CUDA, or
 * TIMEOUT when a bulk copy of the staged step kernel did not arrive within
 * its bounded wait (the state is then invalid until pf_init_fields,
 * pf_set_fields or pf_set_state, which clear the condition). */
pf_status pf_sync(pf_handle *h);

/* Testing only: fault injection for the bounded waits of the staged step
 * kernel (the paper has no counterpart).  on = 1 makes variant 2 skip its
 * bulk copies; each wait then gives up after about one second, the kernel
 * drains and returns, and the next synchronising call reports
 * PF_ERR_TIMEOUT.  No copy is left in flight and the GPU stays usable.
 * on = 0 restores normal copies.  Destroys captured step graphs.
 * Errors: BAD_ARG. */
pf_status pf_test_drop_staged_copies(pf_handle *h, int on);

/* Number of steps taken since the last initialisation; -1 for NULL. */
long long pf_steps_taken(const pf_handle *h);

/* Kernel launches issued by this handle since creation (the library's own
 * kernels only); -1 for NULL. */
long long pf_launch_count(const pf_handle *h);

/* FP64 diagnostics of a field stack without allocating any device memory.
 * The paper has no counterpart: this is a service for callers that cannot
 * allocate device memory, e.g. a plugin inside a host framework that owns the
 * device-memory budget and only hands out buffers it allocated, or a loop
 * that must not call cudaMalloc / cudaFree because they can synchronise the
 * whole device.
 *  fields       device pointer to field planes laid out as in a handle:
 *               plane k (phi, psi, C, U, p, vx, vy, mu_phi in that order)
 *               starts at fields + k * plane_stride elements; the lattice
 *               (nx x ny, row-major) starts at element `offset` of each plane.
 *               Only phi, psi, C, p, vx, vy are read.  Owned by the caller.
 *  fields_fp64  nonzero: planes hold double; zero: float.
 *  probe        Laplace probe or NULL; out: host pf_diag (same quantities and
 *               order as pf_reduce).  cuda_stream: stream for the work.
 * Scratch: a fixed file-scope device array of 1.5 MiB (16384 records of 12
 * doubles) that every GPU loading the library holds until exit; lattices of
 * more than 67,108,864 sites are rejected with PF_ERR_BAD_ARG.  Every call
 * looks up the array's device address in the current context
 * (cudaGetSymbolAddress, no allocation).  Calls share the array: calls that
 * overlap on the GPU (other streams, other threads) race.  Nothing in it needs
 * clearing, since every record read is written by the same call.  The call
 * copies its result to host memory and synchronises the stream, so it cannot
 * be made while the stream is being captured into a CUDA graph.  Errors
 * (message in pf_last_error(NULL)): BAD_ARG, CUDA. */
pf_status pf_reduce_noalloc(const void *fields, int fields_fp64, long long plane_stride,
                            long long offset, int nx, int ny, const pf_probe *probe,
                            pf_diag *out, void *cuda_stream);

/* Boundary types of a domain side (Section 3: half-way bounce-back for no-slip
 * walls and no-flux scalars, the symmetric scheme for symmetry planes;
 * Section 4: far-field Dirichlet values).  Every side sits half-way between
 * the last site and its ghost, except the velocity of PF_BC_INLET_NEE, which is
 * imposed at the ghost node itself. */
enum {
  PF_BC_PERIODIC = 0,   /* wraps to the opposite side (which must be periodic too)   */
  PF_BC_SYMMETRIC = 1,  /* mirror plane: populations reflected, normal velocity flipped */
  PF_BC_WALL = 2,       /* half-way bounce-back on every lattice: no slip, no flux     */
  PF_BC_FARFIELD = 3,   /* bounce-back for the flow and phi; Dirichlet psi = -1, C = 1,
                           theta = theta0 by anti-bounce-back                         */
  PF_BC_INLET = 4,      /* velocity (vin_x, vin_y) by moving-wall bounce-back; liquid
                           phi = 1 and the far-field psi, C, theta by anti-bounce-back */
  PF_BC_OUTLET = 5,     /* pressure p = 0 for the flow (anti-bounce-back); zero gradient
                           for phi, psi, C, theta                                       */
  PF_BC_INLET_NEE = 6   /* velocity (vin_x, vin_y) by non-equilibrium extrapolation
                           (Section 3): the boundary node is the ghost one site beyond
                           the side, its NS populations the equilibrium at vin with the
                           liquid density plus the neighbouring site's non-equilibrium
                           part (pressure extrapolated); phi, psi, C, theta as
                           PF_BC_INLET                                                  */
};

/* Boundary types of domain dom's sides, bc = {x-, x+, y-, y+}, before
 * pf_init_fields / pf_set_fields of that domain (seeds and bubbles then use
 * plain distances along non-periodic axes).  Non-periodic sides need FP32 or
 * FP64 storage and the y-march traversal (selected here); the adjoint takes
 * periodic domains only.  Synchronises the stream.  Errors: BAD_ARG (type out
 * of range, unpaired periodic side, 16-bit storage), STATE (domain already
 * initialised), CUDA. */
pf_status pf_set_boundaries(pf_handle *h, int dom, const int bc[4]);

/* Planes of the raw state of the handle: PF_STATE_PLANES, or
 * PF_STATE_PLANES_THERMAL in thermal mode; -1 for NULL. */
int pf_state_planes(const pf_handle *h);

/* Thermal mode: set the temperature field theta (host, FP64, n = nx*ny) of
 * domain dom after pf_init_fields / pf_set_fields and before the first step.
 * The temperature populations are set to the equilibrium of Appendix B,
 * g^eq(rho H, theta, rho H v) with H = c_p [theta - (c_p^s/c_p) h(psi)] and phi,
 * psi, U, v of the initialisation; the lagged H and the lagged dendrite source
 * Q_psi(theta) / F(U) follow.  Synchronises the stream.  Errors: BAD_ARG (not
 * thermal, bad sizes, non-finite values), STATE (not initialised, or already
 * stepped), CUDA. */
pf_status pf_set_temperature(pf_handle *h, int dom, const double *theta, size_t n);

/* Thermal mode: FP64 totals of domain dom.  out[0] = sum over sites of the
 * five temperature populations (the total of rho H, conserved by the
 * temperature equation of Appendix B on a periodic domain), out[1] = sum theta,
 * out[2] = sum psi.  Synchronises the stream.  Errors: BAD_ARG, CUDA. */
pf_status pf_reduce_thermal(pf_handle *h, int dom, double out[3]);

/* ------------------------------------------------------------------------
 * Three-dimensional dendrite step (Section 2.1 with the anisotropy summed over
 * three axes): psi (anisotropic Allen-Cahn with the a_s^2 time stretch of
 * Appendix B) and C (solute with antitrapping) on D3Q7 lattices (w0 = 1/4,
 * wi = 1/8, c_s^2 = 1/4) in a periodic melt without gas or flow, with one
 * lattice-aligned grain or the grain orientations of pf3_set_orientation.
 * Arrays are [z][y][x], x fastest.
 * Uses the gas and flow parameters of pf_params not at all.  With thermal = 1
 * a D3Q7 temperature lattice (Appendix B at rest: e_0 = rho H - (3/4) theta,
 * e_i = theta/8, k_T = Le D rho_l c_p) is coupled as in 2-D: theta = H / c_p +
 * latent h(psi) enters Q_psi, F(U) = 1/Le + M c_inf [1 + (1-k) U] scales the
 * relaxation of psi, and the source gains W0^2/F^2 grad F . (a_s^2 grad psi +
 * N); Le, latent, theta0, cp and rho_l are read (rho_l cp >= 3/4).
 * ------------------------------------------------------------------------ */
typedef struct pf3_handle pf3_handle;

/* Raw FP64 state planes of pf3_get_state: g_pre[7], g_post[7], r = 1/a_s^2,
 * s[7], Q_psi of the last step (Q_psi / F + the grad F term in thermal mode),
 * then in thermal mode the temperature populations e[7]. */
#define PF3_STATE_PLANES 23
#define PF3_STATE_PLANES_THERMAL 30

/* Handle of an nx x ny x nz lattice (each in [4, 4096]), FP32 or FP64
 * storage, on cuda_stream; allocates two state copies (23 planes each, 30 in
 * thermal mode) and 3 field planes (4 in thermal mode).  Errors: BAD_ARG, OOM. */
pf_status pf3_create(const pf_params *p, int nx, int ny, int nz, pf_precision prec,
                     void *cuda_stream, pf3_handle **out);
/* Spherical seeds n x (x, y, z) of radius R_s: psi = max tanh(sqrt(2 beta_psi)
 * (R_s - r) / W0), C = 1 - (1-k) h(psi), populations at equilibrium (thermal
 * mode: temperature populations at rest at theta0, lagged source Q_psi / F).
 * Synchronises.  Errors: BAD_ARG, OOM, CUDA. */
pf_status pf3_init_seeds(pf3_handle *h, const double *seeds, int n_seeds, double R_s);
/* Initial psi and C fields (host, n = nx*ny*nz each); non-finite values are
 * detected on the device before the state is written and leave it as it
 * was.  Synchronises.  Errors: BAD_ARG (size, non-finite), OOM, CUDA. */
pf_status pf3_set_fields(pf3_handle *h, const double *psi, const double *C, size_t n);
/* Thermal mode: temperature field theta (host, FP64, n = nx*ny*nz) of the
 * initial state, after pf3_init_seeds / pf3_set_fields and before the first
 * step: temperature populations at rest for rho H = rho_l c_p (theta - latent
 * h(psi)), lagged source Q_psi(theta) / F(U).  Synchronises.  Errors: BAD_ARG
 * (not thermal, size, non-finite), STATE (not initialised or already stepped),
 * OOM, CUDA. */
pf_status pf3_set_temperature(pf3_handle *h, const double *theta, size_t n);
/* Grain orientations (the 3-D form of the 2-D grain angle): seeds7 holds
 * n_seeds x (x, y, z, qw, qx, qy, qz); every site takes the rotation R of the
 * nearest seed's quaternion (minimum image, the first seed on an exact tie),
 * and the anisotropy is evaluated on g' = R^T grad psi with N = R N'(g').
 * n_seeds = 0 returns to the lattice-aligned grain.  May be called at any
 * time between steps.  Synchronises.  Errors: BAD_ARG (NULL, non-finite or zero
 * quaternion), OOM, CUDA. */
pf_status pf3_set_orientation(pf3_handle *h, const double *seeds7, int n_seeds);
/* Side types of the six faces x-, x+, y-, y+, z-, z+: 0 periodic, 1 symmetric,
 * 2 wall, 3 far field (psi = -1, C = 1, theta = theta0), each half-way between
 * the last site and its ghost.  On the D3Q7 lattices a symmetric side and a
 * wall are both the half-way bounce-back; a far-field side is the
 * anti-bounce-back to the far values; the stencil ghosts mirror the last site
 * (2 X_far - X across a far-field side).  Opposite sides are both periodic or
 * both not.  Before initialising (seeds then use plain distances along bounded
 * axes).  Errors: BAD_ARG, STATE (already initialised). */
pf_status pf3_set_boundaries(pf3_handle *h, const int bc[6]);
/* Planes per tile of the z-march (default 16).  Errors: BAD_ARG (outside
 * [1, 4096]). */
pf_status pf3_set_chunk(pf3_handle *h, int chunk);
/* Index width of the periodic step: by default sites and plane offsets are
 * indexed in 32 bits while PF3_STATE_PLANES_THERMAL x n < 2^32 (fewer address
 * instructions) and in 64 bits above; on != 0 takes the 64-bit form at any
 * size (results are bit-identical).  Steps with non-periodic sides always
 * index in 64 bits.  Errors: BAD_ARG. */
pf_status pf3_set_index64(pf3_handle *h, int on);
/* Advance n_steps (enqueued; errors of the launch are reported).
 * Errors: BAD_ARG, STATE, CUDA. */
pf_status pf3_step(pf3_handle *h, int n_steps);
/* psi, C, U (and theta in thermal mode) of the last step: pf3_field_planes
 * planes of n.  Synchronises.  Errors: BAD_ARG (out too small), OOM, CUDA. */
pf_status pf3_get_fields(pf3_handle *h, double *out, size_t n);
/* Raw state (pf3_state_planes planes of n).  Synchronises.  Errors: BAD_ARG
 * (NULL, out too small), OOM, CUDA. */
pf_status pf3_get_state(pf3_handle *h, double *out, size_t n);
/* FP64 totals: out[0] = sum C (conserved), out[1] = sum h(psi).  Synchronises.
 * Errors: BAD_ARG (NULL), OOM, CUDA. */
pf_status pf3_reduce(pf3_handle *h, double out[2]);
/* Thermal mode: FP64 totals out[0] = sum of the seven temperature populations
 * (rho H, conserved on the periodic cube), out[1] = sum theta, out[2] = sum
 * psi.  Synchronises.  Errors: BAD_ARG (NULL, not thermal), OOM, CUDA. */
pf_status pf3_reduce_thermal(pf3_handle *h, double out[3]);
/* Field planes (3, or 4 in thermal mode) and raw state planes (23 or 30) of
 * the handle; -1 for NULL. */
int pf3_field_planes(const pf3_handle *h);
int pf3_state_planes(const pf3_handle *h);
/* Kernel launches of the handle; -1 for NULL. */
long long pf3_launch_count(const pf3_handle *h);
/* Last error of the handle, or of the last failed pf3_create for NULL. */
const char *pf3_last_error(const pf3_handle *h);
/* Release the handle (NULL is ignored).  Errors: CUDA (a failed release; the
 * handle is freed all the same). */
pf_status pf3_destroy(pf3_handle *h);

/* ------------------------------------------------------------------------
 * Three-dimensional two-phase step: the coupled step of this library in 3-D.
 * Incompressible Navier-Stokes (pressure-based equilibrium, forcing of
 * surface tension, buoyancy along -y, the mass-flux correction and the
 * diffuse drag v = (1 - h(psi)) v*) and the conservative Allen-Cahn equation
 * on D3Q19 lattices (w0 = 1/3, faces 1/18, edges 1/36, c_s^2 = 1/3) with the
 * MRT of Appendix B in the moment basis of d'Humieres et al. (2002) (NS rates:
 * s_e, s_eps, s_q = 8(2 - s_nu)/(8 - s_nu) on q and m, s_nu on the stresses,
 * 1 elsewhere; CAC: fluxes at s_phi); psi and C on the D3Q7 lattices of the
 * pf3_* step with the gas couplings of Section 2 (f3 in Q_psi, the gas-vacuum
 * flux J) and advection of C.  With thermal = 1 the D3Q7 temperature lattice
 * of the pf3_* step is added with the advective flux rho H v (and d_t(rho H v)
 * through (I - S/2)), theta = H / c_p + latent h(psi) from the local density,
 * F(U) and the grad F source (rho_g cp >= 3/4).  Periodic cube, the
 * lattice-aligned grain or the orientations of pf3f_set_orientation.  Arrays are
 * [z][y][x].
 * ------------------------------------------------------------------------ */
typedef struct pf3f_handle pf3f_handle;

/* Raw FP64 state planes of pf3f_get_state: f[19], h[19], g_pre[7], g_post[7],
 * r = 1/a_s^2, s[7], Q_psi, phi_o, C_o, vx_o, vy_o, vz_o. */
#define PF3F_STATE_PLANES 66
/* Thermal mode: the 66 planes, then e[7] and the lagged H. */
#define PF3F_STATE_PLANES_THERMAL 74
/* Field planes of pf3f_get_fields: phi, psi, C, U, p, vx, vy, vz, mu_phi (and
 * theta in thermal mode: 10). */
#define PF3F_FIELD_PLANES 9

/* Handle of an nx x ny x nz lattice (each in [4, 2048]), FP32 or FP64 storage,
 * on cuda_stream: two state copies of 59 population and 7 auxiliary planes (66
 * and 8 in thermal mode), 9 field planes (10).  Errors: BAD_ARG (sizes,
 * precision, parameters), OOM. */
pf_status pf3f_create(const pf_params *p, int nx, int ny, int nz, pf_precision prec,
                      void *cuda_stream, pf3f_handle **out);
/* Spherical seeds n_seeds x (x, y, z) of radius R_s and bubbles n_bub x (x, y,
 * z, R): psi = max tanh(sqrt(2 beta_psi)(R_s - r)/W0), phi = min [1/2 + 1/2
 * tanh(sqrt(2 beta_phi)(r - R)/(2 W_phi))], C = phi (1 - (1-k) h(psi)), at rest
 * (p = 0); populations at equilibrium.  Sets the buoyancy reference rho_bar
 * from the mean phi.  Synchronises.  Errors: BAD_ARG, OOM, CUDA. */
pf_status pf3f_init_spec(pf3f_handle *h, const double *seeds, int n_seeds, double R_s,
                         const double *bubbles, int n_bub);
/* Initial fields (host, FP64): seven planes of nx*ny*nz in the order phi, psi,
 * C, vx, vy, vz, p (n = 7 nx ny nz); populations at equilibrium, rho_bar from
 * the mean phi.  Non-finite values are detected on the device before the
 * state is written and leave it as it was.  Synchronises.  Errors: BAD_ARG
 * (size, non-finite), OOM, CUDA. */
pf_status pf3f_set_fields(pf3f_handle *h, const double *fields7, size_t n);
/* Buoyancy reference density (after initialisation; replaces the mean).
 * pf3f_set_rho_bar errors: BAD_ARG (NULL, non-finite); pf3f_get_rho_bar
 * returns 0 for NULL. */
pf_status pf3f_set_rho_bar(pf3f_handle *h, double rho_bar);
double pf3f_get_rho_bar(const pf3f_handle *h);
/* Grain orientations as pf3_set_orientation: seeds7 n_seeds x (x, y, z, qw,
 * qx, qy, qz), every site takes the nearest seed's rotation; 0 seeds returns
 * to the lattice-aligned grain.  Synchronises.  Errors: BAD_ARG, OOM, CUDA. */
pf_status pf3f_set_orientation(pf3f_handle *h, const double *seeds7, int n_seeds);
/* Side types of the faces x-, x+, y-, y+, z-, z+ (0 periodic, 1 symmetric, 2
 * wall, 3 far field), half-way between the last site and its ghost: NS and CAC
 * reflect at a symmetric side and bounce back (no slip, no flux) at a wall or a
 * far-field side; psi, C, theta as pf3_set_boundaries; stencil ghosts mirror
 * the last site (the velocity's normal component flipped at a symmetric side,
 * all of it at a wall or far side; 2 X_far - X for psi and U at a far side).
 * Before initialising.  Errors: BAD_ARG, STATE. */
pf_status pf3f_set_boundaries(pf3f_handle *h, const int bc[6]);
/* Planes per tile of the z-march (default 36, the fastest at 256^3 on a
 * 152-SM GPU: the tiles then fill the last wave of one CTA per SM); the state
 * does not depend on it.  Errors: BAD_ARG (outside [1, 2048]). */
pf_status pf3f_set_chunk(pf3f_handle *h, int chunk);
/* Index width of the periodic step: by default sites and plane offsets are
 * indexed in 32 bits while PF3F_STATE_PLANES_THERMAL x n < 2^32 (fewer address
 * instructions) and in 64 bits above; on != 0 takes the 64-bit form at any
 * size (results are bit-identical).  Steps with non-periodic sides always
 * index in 64 bits.  Errors: BAD_ARG. */
pf_status pf3f_set_index64(pf3f_handle *h, int on);
/* Advance n_steps (enqueued).  Errors: BAD_ARG, STATE (not initialised), CUDA. */
pf_status pf3f_step(pf3f_handle *h, int n_steps);
/* Fields of the last step (PF3F_FIELD_PLANES planes of n).  Synchronises.
 * Errors: BAD_ARG (NULL, out too small), OOM, CUDA. */
pf_status pf3f_get_fields(pf3f_handle *h, double *out, size_t n);
/* Raw state (PF3F_STATE_PLANES planes of n).  Synchronises.  Errors: BAD_ARG
 * (NULL, out too small), OOM, CUDA. */
pf_status pf3f_get_state(pf3f_handle *h, double *out, size_t n);
/* FP64 totals of the last fields: out[0] = sum phi, out[1] = sum C (both
 * conserved), out[2] = sum h(psi).  Synchronises.  Errors: BAD_ARG, OOM, CUDA. */
pf_status pf3f_reduce(pf3f_handle *h, double out[3]);
/* Thermal mode: temperature field theta (host, FP64, n = nx*ny*nz) of the
 * initial state, after pf3f_init_spec / pf3f_set_fields (which start at theta0)
 * and before the first step: temperature populations at equilibrium with rho H v,
 * the lagged H and Q_psi(theta) / F(U).  Synchronises.  Errors: BAD_ARG (not
 * thermal, size, non-finite), STATE, OOM, CUDA. */
pf_status pf3f_set_temperature(pf3f_handle *h, const double *theta, size_t n);
/* Thermal mode: FP64 sums out[0] = rho H (the seven temperature populations,
 * conserved on the periodic cube), out[1] = theta, out[2] = psi.  Synchronises.
 * Errors: BAD_ARG (NULL, not thermal), OOM, CUDA. */
pf_status pf3f_reduce_thermal(pf3f_handle *h, double out[3]);
/* Field planes (9, or 10 in thermal mode) and raw state planes (66 or 74) of the
 * handle; -1 for NULL. */
int pf3f_field_planes(const pf3f_handle *h);
int pf3f_state_planes(const pf3f_handle *h);
/* Kernel launches of the handle; -1 for NULL. */
long long pf3f_launch_count(const pf3f_handle *h);
/* Last error of the handle, or of the last failed pf3f_create for NULL. */
const char *pf3f_last_error(const pf3f_handle *h);
/* Release the handle (NULL is ignored).  Errors: CUDA (a failed release; the
 * handle is freed all the same). */
pf_status pf3f_destroy(pf3f_handle *h);

/* Release every resource of the handle (NULL is ignored).  Errors: CUDA (a
 * failed release; the handle is freed all the same). */
pf_status pf_destroy(pf_handle *h);

/* Last error message of the handle, or of the last failed pf_create when h is
 * NULL.  Never NULL. */
const char *pf_last_error(const pf_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* PF_H_ */
