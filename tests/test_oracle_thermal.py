"""Pins of the FP64 oracle's temperature coupling (Section 2.1, Appendix B).

The thermal mode solves the temperature equation for H = c_p theta -
c_p^s h(psi) with the D2Q5 model of Appendix B, uses the field theta in the
dendrite source, and takes the dendrite equation in its rewritten form with
F(U) = 1/Le + M c_inf [1 + (1-k) U] and the grad F source.  Each test checks
the oracle against something other than its own formulas: the moments the
paper states for the equilibrium, the paper's closed form of F(U) at printed
parameters, an invariant, the textbook variance growth of heat diffusion, the
latent-heat balance of Eq. eq-tem2, and an independent finite-difference
solution of the original (not rewritten) equations.
"""
import json
import functools
import math
import os

import numpy as np

import oracle
from paper_2407_01651_gb300 import workload as wl

CX = np.array([0, 1, 0, -1, 0])
CY = np.array([0, 0, 1, 0, -1])
CS2 = 1 / 3
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def params(**over):
    p = dict(wl.BASE_PARAMS)
    p.update(thermal=1.0, Le=1.0, latent=1.0, theta0=-0.55, cp=10.0)
    p.update(over)
    return p


def test_temperature_equilibrium_moments():
    """Appendix B: sum g^eq = rho H, sum c g^eq = rho H v, and the second
    moment c_s^2 theta I that makes k_T = (1/s - 1/2) c_s^2 the conductivity."""
    rng = np.random.default_rng(1)
    for _ in range(5):
        rhoH, theta, jx, jy = rng.normal(size=4)
        g = oracle.teq_th(rhoH, theta, jx, jy)
        assert math.isclose(g.sum(), rhoH, rel_tol=1e-14, abs_tol=1e-15)
        assert np.allclose([g @ CX, g @ CY], [jx, jy], atol=1e-15)
        assert math.isclose(g @ (CX * CX), CS2 * theta, rel_tol=1e-14)
        assert math.isclose(g @ (CY * CY), CS2 * theta, rel_tol=1e-14)
        assert abs(g @ (CX * CY)) < 1e-15


def test_lewis_function_and_rates():
    """F(U) of Section 2.1 at the paper's printed Le, k, Omega (golden), F = 1
    at U = Omega / (1 - (1-k) Omega) when 1/Le -> 0 (Section 4, below
    Eq. eq-Tsys), and k_T = (1/s - 1/2) c_s^2 with alpha = k_T / (rho_l c_p) =
    Le D (Le = alpha / D)."""
    with open(os.path.join(GOLDEN, "thermal_closure.json")) as fh:
        g = json.load(fh)
    o = oracle.Oracle(4, 4, params(Le=g["Le"], k=g["k"], Omega=g["Omega"]))
    assert math.isclose(o.thermal_coefs(0.0)["F"], g["F_at_U0"], rel_tol=1e-14)
    assert math.isclose(o.thermal_coefs(-1.0 / (1.0 - g["k"]))["F"], g["F_in_gas"],
                        rel_tol=1e-12)
    for Om, k in ((0.55, 0.15), (0.3, 0.5)):
        o = oracle.Oracle(4, 4, params(Le=1e15, Omega=Om, k=k))
        assert math.isclose(o.thermal_coefs(Om / (1 - (1 - k) * Om))["F"], 1.0, rel_tol=1e-13)
    for Le, cp, D in ((1.0, 10.0, 0.1), (50.0, 7.0, 0.05)):
        p = params(Le=Le, cp=cp, D=D)
        c = oracle.Oracle(4, 4, p).thermal_coefs(0.0)
        assert math.isclose((1 / c["s_th"] - 0.5) * CS2, c["kT"], rel_tol=1e-14)
        assert math.isclose(c["kT"] / (p["rho_l"] * cp), Le * D, rel_tol=1e-14)


def test_enthalpy_gas_and_solute_conserved():
    """The temperature equation is in divergence form (Appendix B, rho H
    conserved by the collision and the streaming): with bubbles rising, a
    dendrite growing and latent heat released, the total of rho H is constant
    to rounding, and so are sum phi and sum C."""
    lay = wl.single_seed_bubble(64, 64, R_b=10.0, d_max=24.0)
    o = oracle.Oracle(64, 64, params(Le=2.0))
    o.init_spec(lay.seeds, lay.R_s, lay.bubbles)
    t0, d0 = o.thermal_totals(), o.diag()
    o.step(200)
    t, d = o.thermal_totals(), o.diag()
    assert d["nonfinite"] == 0
    assert abs(t["sum_e"] / t0["sum_e"] - 1) < 1e-13
    assert abs(d["sum_phi"] / d0["sum_phi"] - 1) < 1e-12
    assert abs(d["sum_C"] / d0["sum_C"] - 1) < 1e-12
    assert t["sum_theta"] != t0["sum_theta"]       # the temperature did evolve
    assert o.state().shape[0] == 45


def heat_alpha(Le, cp, lib=None):
    """Measured diffusivity of a temperature Gaussian in the liquid, per axis,
    from the growth of its variance between steps 100 and 150."""
    N, s0 = 96, 4.0
    y, x = np.mgrid[0:N, 0:N].astype(float)
    th = -0.5 + 0.1 * np.exp(-((x - 48) ** 2 + (y - 48) ** 2) / (2 * s0 * s0))
    one = np.ones_like(x)
    o = oracle.Oracle(N, N, params(Le=Le, cp=cp, g=0.0, theta0=-0.5), lib=lib)
    o.init_fields(one, -one, one, theta=th)
    var = []
    for T in (100, 150):
        o.step(T - o.steps)
        w = o.fields(("theta",))["theta"] + 0.5
        var.append((((x - 48) ** 2 * w).sum() / w.sum(), ((y - 48) ** 2 * w).sum() / w.sum()))
    # the variance grows by 2 alpha per step over the 50 steps
    return [(var[1][a] - var[0][a]) / (2 * 50.0) for a in (0, 1)]


def test_heat_gaussian_variance_grows_2_alpha_t():
    """In the liquid (phi = 1, psi = -1, v = 0, no latent heat released) the
    temperature equation reduces to d theta/dt = alpha lap theta with alpha =
    Le D (Eq. eq-tem2): once the populations' flux has relaxed from the
    equilibrium start, a Gaussian's variance grows by 2 alpha per step in each
    direction, whatever the lattice heat capacity c_p."""
    for Le, cp in ((1.0, 10.0), (1.0, 1.0), (0.5, 10.0)):
        alpha = Le * 0.1
        for a in heat_alpha(Le, cp):
            assert math.isclose(a, alpha, rel_tol=1e-4)


def latent_ratio(latent, lib=None):
    """Rise of the mean theta over (latent / 2) times the rise of the mean psi
    while a seed solidifies in a closed melt (300 steps), and the psi rise."""
    N = 48
    o = oracle.Oracle(N, N, params(latent=latent, g=0.0, Le=2.0), lib=lib)
    o.init_spec([(N / 2, N / 2, 0.0)], 6.0, [])
    t0 = o.thermal_totals()
    o.step(300)
    t = o.thermal_totals()
    dpsi = (t["sum_psi"] - t0["sum_psi"]) / (N * N)
    dth = (t["sum_theta"] - t0["sum_theta"]) / (N * N)
    return dth / (0.5 * latent * dpsi), dpsi, o


def test_latent_heat_raises_temperature_by_half_the_psi_change():
    """Eq. eq-tem2: d theta/dt = div(alpha grad theta) + d h(psi)/dt with
    h = (1+psi)/2 scaled by c_p^s / c_p.  In a closed periodic melt without gas
    (rho = 1) the mean temperature therefore rises by (c_p^s/c_p) / 2 times the
    rise of the mean psi while a seed solidifies."""
    for latent in (1.0, 0.5):
        ratio, dpsi, o = latent_ratio(latent)
        assert dpsi > 5e-3                               # the seed did grow
        assert math.isclose(ratio, 1.0, rel_tol=1e-9)
        f = o.fields(("theta",))
        assert f["theta"].max() > -0.55 + 1e-3           # heat released at the front


# ---------------------------------------------------------------------------
# The grad F source of the rewritten dendrite equation (Appendix B), against
# an explicit finite-difference solution of the original equations
# (Eq. eq-AnACE with tau0 a_s^2 F(U) d psi/dt on the left, the solute equation
# with antitrapping, and Eq. eq-tem2) on a 1-D problem.
# ---------------------------------------------------------------------------
def _fd_1d(p, psi0, C0, th0, T, dt, gradF_weight):
    """Plain explicit Euler, second-order central differences, periodic.
    gradF_weight = 1 solves the original equations; 0 gives the rewritten
    equation with its grad F source left out (a plausible mistake)."""
    k, W0, tau0, D = p["k"], p["W0"], p["tau0"], p["D"]
    lam = D * tau0 / ((47 / 75) * W0 ** 2)
    Mc = 1 - (1 - k) * p["Omega"]
    Le, L, alpha = p["Le"], p["latent"], p["Le"] * p["D"]

    def dx(a):
        return (np.roll(a, -1) - np.roll(a, 1)) / 2

    psi, C, th = psi0.copy(), C0.copy(), th0.copy()
    for _ in range(int(round(T / dt))):
        U = (2 * C / (1 + k - (1 - k) * psi) - 1) / (1 - k)
        F = 1 / Le + Mc * (1 + (1 - k) * U)
        Q = 4 * p["beta_psi"] * psi * (1 - psi ** 2) - lam * (1 - psi ** 2) ** 2 * (th + Mc * U)
        lap = np.roll(psi, -1) - 2 * psi + np.roll(psi, 1)
        dpsi = (W0 ** 2 * lap + Q) / (tau0 * F)
        dpsi += (gradF_weight - 1) * W0 ** 2 / (tau0 * F ** 2) * Mc * (1 - k) * dx(U) * dx(psi)
        gp = dx(psi)
        Jat = -W0 / (2 * math.sqrt(2)) * (1 + (1 - k) * U) * dpsi * gp / np.sqrt(
            gp ** 2 + p["grad_eps_at"] ** 2)
        q = (1 - psi) / 2
        flux = (1 - k) * (D * 0.5 * (q + np.roll(q, -1)) * (np.roll(U, -1) - U)
                          - 0.5 * (Jat + np.roll(Jat, -1)))
        C = C + dt * (flux - np.roll(flux, 1))
        th = th + dt * (alpha * (np.roll(th, -1) - 2 * th + np.roll(th, 1)) + 0.5 * L * dpsi)
        psi = psi + dt * dpsi
    return psi, C, th


@functools.lru_cache(maxsize=None)
def _gradF_fd():
    p, psi0, C0, th0, T = _gradF_case()
    psi_fd, C_fd, th_fd = _fd_1d(p, psi0, C0, th0, T, 0.05, 1.0)
    psi_no, _, _ = _fd_1d(p, psi0, C0, th0, T, 0.05, 0.0)
    return psi_fd, C_fd, th_fd, psi_no


def _gradF_case():
    nx, W0 = 192, 8.0
    p = params(W0=W0, tau0=2 * W0 ** 2 / 0.1, eps_s=0.0, Le=50.0, theta0=-0.3, g=0.0)
    k = p["k"]
    x = np.arange(nx, dtype=float)
    psi0 = np.tanh(math.sqrt(0.5) * (nx / 6 - np.abs(x - nx / 2)) / W0)
    U0 = 0.5 * np.sin(4 * math.pi * x / nx)
    C0 = 0.5 * (1 + k - (1 - k) * psi0) * (1 + (1 - k) * U0)
    th0 = np.full(nx, p["theta0"])
    return p, psi0, C0, th0, 1200


def gradF_errors(lib=None):
    """(error of the oracle's psi against the finite-difference solution of
    the original equations, the grad F source's effect in that solution,
    errors of C and theta, the LB fields)."""
    p, psi0, C0, th0, T = _gradF_case()
    nx, ny = len(psi0), 4
    o = oracle.Oracle(nx, ny, p, lib=lib)
    o.init_fields(np.ones((ny, nx)), np.tile(psi0, (ny, 1)), np.tile(C0, (ny, 1)),
                  theta=np.tile(th0, (ny, 1)))
    o.step(T)
    f = o.fields(("psi", "C", "theta", "vx", "vy"))
    psi_fd, C_fd, th_fd, psi_no = _gradF_fd()
    return (float(np.abs(f["psi"][0] - psi_fd).max()), float(np.abs(psi_fd - psi_no).max()),
            float(np.abs(f["C"][0] - C_fd).max()), float(np.abs(f["theta"][0] - th_fd).max()), f)


def gradF_pin_holds(errs) -> bool:
    err, effect, eC, eth, _ = errs
    return effect > 0.03 and err < 0.15 * effect and eC < 0.01 and eth < 0.01


def test_gradF_source_matches_the_original_equation():
    """The rewritten dendrite equation of Appendix B equals Eq. eq-AnACE divided
    by F only with the source + W0^2/(tau0 F^2) grad F . (a_s^2 grad psi + N).
    On a solid slab in an undercooled melt with a sinusoidal supersaturation
    (so F varies in space), the oracle's LB solution agrees with an independent
    finite-difference solution of the original equations far better than that
    solution differs from the one without the grad F source.  W0 = 8 resolves
    the interface well enough for both discretisations."""
    errs = gradF_errors()
    f = errs[4]
    assert np.abs(f["vx"]).max() == 0.0 and np.abs(f["vy"]).max() == 0.0
    for a in ("psi", "C", "theta"):
        assert np.abs(f[a] - f[a][0]).max() < 1e-14          # uniform along y
    p, psi0, C0, th0, T = _gradF_case()
    assert np.abs(_gradF_fd()[0] - psi0).max() > 0.5        # the fronts moved
    assert gradF_pin_holds(errs)
