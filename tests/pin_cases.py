"""Measurements shared by the oracle pins and by the test that plants
mistakes in copies of the oracle (tests/test_oracle_mutations.py).

Each function runs one small problem on an oracle library (the oracle's own
build by default, or a copy with a planted mistake) and returns the numbers
its pin bounds.  The reference solutions here are written from the paper's
equations, independently of the oracle's lattice Boltzmann arithmetic.
"""
import functools
import math

import numpy as np

import oracle
from paper_2407_01651_gb300 import workload as wl


# ---------------------------------------------------------------------------
# Time stretch of the dendrite equation.  Eq. eq-AnACE carries
# tau0 a_s^2(n) d psi / dt on its left-hand side; the LB form of Appendix B
# realises the a_s^2 through the time stretch f_i(x + c_i, t + a_s^2 dt).
# For a flat front along <10> of a lattice-aligned grain a_s = 1 + eps_s is
# uniform and N = 0, so the 1-D equation is
#   tau0 a_s^2 d psi/dt = W0^2 a_s^2 psi'' + Q(psi, U),
# with the solute equation d C/dt = d/dx [(1-k) (D q dU/dx - J_at)] and
# J_at built on W_psi = W0 a_s (Section 2.1).
# ---------------------------------------------------------------------------
FRONT_NX, FRONT_W0, FRONT_EPS, FRONT_T = 192, 8.0, 0.05, 1200
STRETCH_TOL = 0.006        # bound on max |psi_LB - psi_FD(tau0 a_s^2)|


def front_params():
    W0 = FRONT_W0
    return dict(wl.BASE_PARAMS, W0=W0, tau0=2 * W0 ** 2 / 0.1, eps_s=FRONT_EPS, g=0.0)


def front_initial():
    p = front_params()
    k = p["k"]
    x = np.arange(FRONT_NX, dtype=float)
    psi0 = np.tanh(math.sqrt(0.5) * (FRONT_NX / 6 - np.abs(x - FRONT_NX / 2))
                   / (FRONT_W0 * (1 + FRONT_EPS)))
    C0 = 0.5 * (1 + k - (1 - k) * psi0)            # U = 0
    return psi0, C0


@functools.lru_cache(maxsize=None)
def front_fd(stretch_power: int):
    """Explicit finite-difference solution (Euler, dt = 0.05, second-order
    central differences, periodic) of the 1-D isothermal equations above with
    tau0 a_s^p on the left: p = 2 is the paper's equation, p = 1 and p = 0
    are plausible mistakes (no or half the stretch)."""
    p = front_params()
    psi0, C0 = front_initial()
    k, W0, tau0, D = p["k"], p["W0"], p["tau0"], p["D"]
    a_s = 1.0 + FRONT_EPS
    lam = D * tau0 / ((47 / 75) * W0 ** 2)          # Appendix A: tau0 D / W0^2 = a2' lambda'
    Mc = 1 - (1 - k) * p["Omega"]                   # Eq. eq-Tsys
    theta = -p["Omega"]
    dt = 0.05

    def ddx(a):
        return (np.roll(a, -1) - np.roll(a, 1)) / 2

    psi, C = psi0.copy(), C0.copy()
    for _ in range(int(round(FRONT_T / dt))):
        U = (2 * C / (1 + k - (1 - k) * psi) - 1) / (1 - k)
        Q = 4 * p["beta_psi"] * psi * (1 - psi ** 2) - lam * (1 - psi ** 2) ** 2 * (theta + Mc * U)
        lap = np.roll(psi, -1) - 2 * psi + np.roll(psi, 1)
        dpsi = (W0 ** 2 * a_s ** 2 * lap + Q) / (tau0 * a_s ** stretch_power)
        g = ddx(psi)
        Jat = (-W0 * a_s / (2 * math.sqrt(2)) * (1 + (1 - k) * U) * dpsi * g
               / np.sqrt(g ** 2 + p["grad_eps_at"] ** 2))
        q = (1 - psi) / 2
        flux = (1 - k) * (D * 0.5 * (q + np.roll(q, -1)) * (np.roll(U, -1) - U)
                          - 0.5 * (Jat + np.roll(Jat, -1)))
        C = C + dt * (flux - np.roll(flux, 1))
        psi = psi + dt * dpsi
    return psi


def front_lb(kind: str = "2d", lib=None):
    """psi along x after FRONT_T steps of the oracle ("2d", "3d" melt or "3f"
    two-phase) from the slab of front_initial, and the largest deviation
    from uniformity across the other axes."""
    p = front_params()
    psi0, C0 = front_initial()
    nx = FRONT_NX
    if kind == "2d":
        o = oracle.Oracle(nx, 4, p, lib=lib)
        o.init_fields(np.ones((4, nx)), np.tile(psi0, (4, 1)), np.tile(C0, (4, 1)))
        o.step(FRONT_T)
        psi = o.fields(("psi",))["psi"]
        return psi[0], float(np.abs(psi - psi[0]).max())
    sh = (4, 4, nx)
    if kind == "3d":
        o = oracle.Oracle3D(nx, 4, 4, {k: p[k] for k in oracle.PARAM_NAMES_3D if k in p},
                            lib=lib)
        o.init_fields(np.broadcast_to(psi0, sh), np.broadcast_to(C0, sh))
    else:
        o = oracle.Oracle3F(nx, 4, 4, {k: p[k] for k in oracle.PARAM_NAMES_3F if k in p},
                            lib=lib)
        o.init_fields(np.ones(sh), np.broadcast_to(psi0, sh), np.broadcast_to(C0, sh))
    o.step(FRONT_T)
    psi = o.fields()["psi"]
    return psi[0, 0], float(np.abs(psi - psi[0, 0]).max())


def stretch_pin_holds(errs) -> bool:
    """The pin: the oracle is within STRETCH_TOL of the paper's equation and
    within a quarter of the distance between the a_s^2 and a_s solutions."""
    gap = float(np.abs(front_fd(2) - front_fd(1)).max())
    return errs[2] < STRETCH_TOL and errs[2] < 0.25 * gap


def stretch_errors(kind: str = "2d", lib=None):
    """max |psi_LB - psi_FD| against the solutions with tau0 a_s^2 (the
    paper's), tau0 a_s and tau0 on the left-hand side."""
    psi, nonuniform = front_lb(kind, lib)
    errs = {pw: float(np.abs(psi - front_fd(pw)).max()) for pw in (2, 1, 0)}
    return errs, nonuniform


# ---------------------------------------------------------------------------
# Mass-consistent momentum flux (Section 2.2): with m = rho v - D (rho_l -
# rho_g) / (phi_l - phi_g), the momentum equation d(rho v)/dt + div(m v) = ...
# keeps a uniform velocity V exactly, because d rho/dt + div m = 0 by the CAC
# equation; with rho v in place of m, mass moved by the diffusive flux D
# arrives without momentum and slows the flow where the density grows.  A
# flat gas layer started at 1.5 times its equilibrium width (so div D != 0
# while it relaxes) in a uniform flow parallel to it (so incompressibility
# does not fix v, unlike a flow normal to a flat layer) measures this.
# ---------------------------------------------------------------------------
MASS_FLUX_V, MASS_FLUX_T = 0.01, 300
MASS_FLUX_TOL = 0.02       # bound on max |v_x - V| / V


def mass_flux_deviation(kind: str = "2d", lib=None):
    """max |v_x - V| / V after MASS_FLUX_T steps, and max |v_y|."""
    W, V = 2.0, MASS_FLUX_V
    ny = 128
    y = np.arange(ny, dtype=float)
    phi1 = 0.5 + 0.5 * np.tanh((np.abs(y - 64.0) - 24.0) / (2 * math.sqrt(2) * W * 1.5))
    p = dict(wl.BASE_PARAMS, g=0.0, sigma=0.0, W_phi=W)
    if kind == "2d":
        phi = np.tile(phi1[:, None], (1, 4))
        one = np.ones_like(phi)
        o = oracle.Oracle(4, ny, p, lib=lib)
        o.init_fields(phi, -one, phi, V * one, 0 * one)
    else:
        phi = np.broadcast_to(phi1[None, :, None], (4, ny, 4)).copy()
        one = np.ones_like(phi)
        o = oracle.Oracle3F(4, ny, 4, {k: p[k] for k in oracle.PARAM_NAMES_3F if k in p},
                            lib=lib)
        o.init_fields(phi, -one, phi, V * one, 0 * one, 0 * one)
    o.step(MASS_FLUX_T)
    f = o.fields()
    return float(np.abs(f["vx"] - V).max() / V), float(np.abs(f["vy"]).max())


# ---------------------------------------------------------------------------
# Dirichlet velocity by non-equilibrium extrapolation (Section 3): the ghost
# node one site beyond the side carries the velocity.
# ---------------------------------------------------------------------------
def nee_couette_holds(lib=None, ny=16, U=0.01) -> bool:
    """Couette flow between a tangential extrapolation inlet (bottom) and a
    no-slip wall (top, half-way): linear through the ghost node, v_x = U (ny -
    1/2 - y) / (ny + 1/2), to 1e-12."""
    p = dict(wl.BASE_PARAMS, g=0.0, vin_x=U, vin_y=0.0, nu=0.5)
    one = np.ones((ny, 4))
    o = oracle.Oracle(4, ny, p, lib=lib)
    o.set_bc(0, 0, 6, 2)
    o.init_fields(one, -one, one, 0 * one, 0 * one, 0 * one)
    o.step(20000)
    v = o.fields(("vx",))["vx"][:, 0]
    y = np.arange(ny)
    return bool(np.abs(v - U * (ny - 0.5 - y) / (ny + 0.5)).max() < 1e-12)


# ---------------------------------------------------------------------------
# Flat gas layer at the equilibrium profile of Eq. (eq-phiEq): a stationary
# state of the CAC equation (Section 2.2).
# ---------------------------------------------------------------------------
FLAT_W, FLAT_NY, FLAT_HALF = 2.0, 96, 24.0


def _tanh_fit(dist, prof, half0, width0):
    from scipy.optimize import curve_fit
    (w, h), _ = curve_fit(lambda d, w, h: np.tanh((h - d) / w), dist, prof, p0=(width0, half0))
    return float(w), float(h)


def flat_layer(lib=None):
    """A gas layer of half-thickness FLAT_HALF started at the tanh profile,
    after 9000 and 10^4 steps: (change over the last 1000 steps, max |v_y|,
    max |v_x|, relative error of the fitted tanh width, position error of the
    fitted interface, max |phi - tanh|)."""
    W, ny = FLAT_W, FLAT_NY
    y = np.arange(ny, dtype=float)
    d = np.abs(y - ny / 2)
    width = 2 * math.sqrt(2) * W
    phi1 = 0.5 + 0.5 * np.tanh((d - FLAT_HALF) / width)
    phi = np.tile(phi1[:, None], (1, 4))
    o = oracle.Oracle(4, ny, dict(wl.BASE_PARAMS, g=0.0, W_phi=W), lib=lib)
    o.init_fields(phi, -np.ones_like(phi), phi * 1.0)
    o.step(9000)
    before = o.fields(("phi",))["phi"][:, 0].copy()
    o.step(1000)
    f = o.fields()
    after = f["phi"][:, 0]
    w, h = _tanh_fit(d, 1.0 - 2.0 * after, FLAT_HALF, width)
    return (float(np.abs(after - before).max()), float(np.abs(f["vy"]).max()),
            float(np.abs(f["vx"]).max()), w / width - 1.0, h - FLAT_HALF,
            float(np.abs(after - phi1).max()))


def flat_layer_3f(lib=None):
    """The flat-layer case of the 3-D two-phase step (NS and CAC on D3Q19): the
    same gas layer, its normal along z on a 4 x 4 x FLAT_NY lattice, after 9000
    and 10^4 steps.  The tuple of flat_layer, with the largest velocity across
    the layer (|v_x|, |v_y|) in the transverse slot."""
    W, n = FLAT_W, FLAT_NY
    z = np.arange(n, dtype=float)
    d = np.abs(z - n / 2)
    width = 2 * math.sqrt(2) * W
    phi1 = 0.5 + 0.5 * np.tanh((d - FLAT_HALF) / width)
    phi = np.broadcast_to(phi1[:, None, None], (n, 4, 4)).copy()
    p3f = {k: wl.BASE_PARAMS[k] for k in oracle.PARAM_NAMES_3F}
    o = oracle.Oracle3F(4, 4, n, dict(p3f, g=0.0, W_phi=W), lib=lib)
    o.init_fields(phi, -np.ones_like(phi), phi * 1.0)
    o.step(9000)
    before = o.fields()["phi"][:, 0, 0].copy()
    o.step(1000)
    f = o.fields()
    after = f["phi"][:, 0, 0]
    w, h = _tanh_fit(d, 1.0 - 2.0 * after, FLAT_HALF, width)
    return (float(np.abs(after - before).max()), float(np.abs(f["vz"]).max()),
            float(max(np.abs(f["vx"]).max(), np.abs(f["vy"]).max())), w / width - 1.0,
            h - FLAT_HALF, float(np.abs(after - phi1).max()))


def flat_layer_holds(m) -> bool:
    drift, vy, vx, dw, dh, dev = m
    return (drift < 1e-7 and vy < 1e-7 and vx < 1e-12 and abs(dw) < 5e-3 and abs(dh) < 1e-5
            and dev < 2.5e-3)
