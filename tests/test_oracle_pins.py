"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage it follows.  None of them retypes an oracle
formula: they check closed forms, invariants, exact special cases and
derivative identities, chosen so that a dropped term, a wrong sign, a wrong
index or a transposed operand in the oracle fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate

import oracle
import pin_cases
from paper_2407_01651_gb300 import workload as wl

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
W5 = np.array([1 / 3] + [1 / 6] * 4)
CS2 = 1 / 3


GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)


def golden_expr(expr, **env):
    return eval(expr, {"__builtins__": {}}, dict(vars(math), **env))


def params(**over):
    p = dict(wl.BASE_PARAMS)
    p.update(over)
    return p


# ---------------------------------------------------------------------------
# Moments of the equilibria and of the forcing (Chapman-Enskog requirements
# of the readings for the cited NS / CAC / solute LB models, Appendix B).
# ---------------------------------------------------------------------------
def test_ns_equilibrium_moments():
    rng = np.random.default_rng(0)
    for _ in range(5):
        p, rho, vx, vy = rng.normal() * 1e-2, 0.1 + rng.random(), *(rng.normal(size=2) * 0.05)
        f = oracle.feq_ns(p, rho, vx, vy)
        # zeroth moment 0, first rho v, second p I + rho v v
        assert abs(f.sum()) < 1e-15
        assert np.allclose([f @ CX, f @ CY], [rho * vx, rho * vy], atol=1e-15)
        assert math.isclose(f @ (CX * CX), p + rho * vx * vx, abs_tol=1e-15)
        assert math.isclose(f @ (CY * CY), p + rho * vy * vy, abs_tol=1e-15)
        assert math.isclose(f @ (CX * CY), rho * vx * vy, abs_tol=1e-15)
        # pressure is carried by the rest population: sum_{i>0} f_i = (1-w0) p/cs2 - rho s_0
        s0 = -W9[0] * (vx * vx + vy * vy) / (2 * CS2)
        assert math.isclose(f[1:].sum(), (1 - W9[0]) * p / CS2 - rho * s0, abs_tol=1e-15)


def test_cac_and_solute_equilibrium_moments():
    h = oracle.heq_cac(0.3, 0.02, -0.01)
    assert math.isclose(h.sum(), 0.3, rel_tol=1e-15)
    assert np.allclose([h @ CX, h @ CY], [0.3 * 0.02, -0.3 * 0.01], atol=1e-16)
    assert np.allclose([h @ (CX * CX), h @ (CY * CY), h @ (CX * CY)], [CS2 * 0.3, CS2 * 0.3, 0],
                       atol=1e-16)
    s = oracle.seq_sol(0.7, 0.011, -0.004)
    cx5, cy5 = CX[:5], CY[:5]
    assert math.isclose(s.sum(), 0.7, rel_tol=1e-15)
    assert np.allclose([s @ cx5, s @ cy5], [0.011, -0.004], atol=1e-16)
    assert np.allclose([s @ (cx5 * cx5), s @ (cy5 * cy5)], [CS2 * 0.7] * 2, atol=1e-16)


# ---------------------------------------------------------------------------
# MRT collision (Appendix B, Lambda = M^-1 S M)
# ---------------------------------------------------------------------------
def test_mrt_equal_rates_is_bgk():
    rng = np.random.default_rng(1)
    for s in (0.3, 1.0, 1.7):
        f, feq, G = rng.normal(size=(3, 9))
        out = oracle.collide9(f, feq, np.full(9, s), G)
        assert np.allclose(out, f - s * (f - feq) + (1 - s / 2) * G, atol=1e-14)
        f5, feq5, G5, F5 = rng.normal(size=(4, 5))
        out5 = oracle.collide5(f5, feq5, np.full(5, s), G5, F5)
        assert np.allclose(out5, f5 - s * (f5 - feq5) + (1 - s / 2) * G5 + F5, atol=1e-14)


def test_mrt_rates_act_on_the_right_moments():
    """Relaxing only the momentum-flux moments of D2Q9 with rate s changes the
    second moment c_x c_y by exactly -s times its non-equilibrium part and
    leaves the zeroth and first moments untouched."""
    rng = np.random.default_rng(2)
    f, feq = rng.normal(size=(2, 9))
    S = np.array([0, 0, 0, 0, 0, 0, 0, 0.6, 0.6])
    out = oracle.collide9(f, feq, S, np.zeros(9))
    for c in (np.ones(9), CX, CY):
        assert math.isclose(out @ c, f @ c, abs_tol=1e-14)
    pxy = CX * CY
    assert math.isclose(out @ pxy, f @ pxy - 0.6 * (f @ pxy - feq @ pxy), abs_tol=1e-14)
    # D2Q5 first moments relax with S[1], S[2]
    f5, feq5 = rng.normal(size=(2, 5))
    out5 = oracle.collide5(f5, feq5, np.array([0, 1.3, 1.3, 0, 0]), np.zeros(5), np.zeros(5))
    assert math.isclose(out5 @ CX[:5], f5 @ CX[:5] - 1.3 * (f5 - feq5) @ CX[:5], abs_tol=1e-14)
    assert math.isclose(out5.sum(), f5.sum(), abs_tol=1e-14)


# ---------------------------------------------------------------------------
# Stencils: the isotropic 9-point forms are exact on quadratics
# ---------------------------------------------------------------------------
def test_stencils_exact_on_quadratics():
    y, x = np.mgrid[0:16, 0:16].astype(float)
    X = 0.3 * x * x - 0.2 * x * y + 0.7 * y * y + 1.1 * x - 0.4 * y + 2.0
    gx, gy, lap = oracle.stencil(X, 7, 9)
    assert math.isclose(gx, 0.6 * 7 - 0.2 * 9 + 1.1, rel_tol=1e-13)
    assert math.isclose(gy, -0.2 * 7 + 1.4 * 9 - 0.4, rel_tol=1e-13)
    assert math.isclose(lap, 0.6 + 1.4, rel_tol=1e-13)


# ---------------------------------------------------------------------------
# Anisotropy a_s and N (Section 2.1 and Section 3.3)
# ---------------------------------------------------------------------------
def test_anisotropy_axis_and_diagonal_values():
    eps = 0.05
    a_axis = oracle.aniso(3.0, 0.0, 0.0, eps)[0]
    a_diag = oracle.aniso(2.0, 2.0, 0.0, eps)[0]
    assert math.isclose(a_axis, 1 + eps, rel_tol=1e-10)     # max along <10>
    assert math.isclose(a_diag, 1 - eps, rel_tol=1e-10)     # min along <11>
    # a grain rotated by pi/4 swaps them
    assert math.isclose(oracle.aniso(3.0, 0.0, math.pi / 4, eps)[0], 1 - eps, rel_tol=1e-10)


def test_anisotropy_vector_is_the_derivative():
    """N_a = |grad psi|^2 a_s d a_s / d(d_a psi) (Section 2.1): checked against a
    central difference of the oracle's own a_s, at random gradients and grain
    angles."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        g = rng.normal(size=2) * rng.choice([1e-2, 0.3, 2.0])
        th, eps = rng.random() * math.pi / 2, 0.01 + 0.08 * rng.random()
        a, Nx, Ny, gm = oracle.aniso(*g, th, eps)
        h = 1e-6 * np.linalg.norm(g)
        da = []
        for e in (np.array([1.0, 0]), np.array([0, 1.0])):
            ap = oracle.aniso(*(g + h * e), th, eps)[0]
            am = oracle.aniso(*(g - h * e), th, eps)[0]
            da.append((ap - am) / (2 * h))
        ref = gm * gm * a * np.array(da)
        assert np.allclose([Nx, Ny], ref, rtol=1e-6, atol=1e-9 * abs(ref).max())


def test_anisotropy_rotates_covariantly():
    rng = np.random.default_rng(4)
    for _ in range(10):
        g = rng.normal(size=2)
        th = rng.random() * math.pi
        c, s = math.cos(th), math.sin(th)
        g_crys = np.array([c * g[0] + s * g[1], -s * g[0] + c * g[1]])
        a, Nx, Ny, _ = oracle.aniso(*g, th, 0.05)
        a0, Nx0, Ny0, _ = oracle.aniso(*g_crys, 0.0, 0.05)
        assert math.isclose(a, a0, rel_tol=1e-13)
        assert np.allclose([Nx, Ny], [c * Nx0 - s * Ny0, s * Nx0 + c * Ny0], atol=1e-13)


# ---------------------------------------------------------------------------
# Thin-interface parameter map (Appendix A) and isothermal closure (Eq. eq-Tsys)
# ---------------------------------------------------------------------------
def test_thin_interface_constants_by_quadrature():
    """a1' = 5 sqrt2/8 and a2' = 47/75 follow from the integrals I, J, K, H of
    Appendix A evaluated on psi0(eta) = -tanh(eta/sqrt2) (beta_psi = 1/4,
    psi_s = 1, psi_l = -1), p'(psi) = 15/16 (1-psi^2)^2, h = (1+psi)/2."""
    psi0 = lambda e: -math.tanh(e / math.sqrt(2))
    dpsi = lambda e: -(1 - psi0(e) ** 2) / math.sqrt(2)
    pprime = lambda s: 15 / 16 * (1 - s * s) ** 2
    h = lambda s: (1 + s) / 2
    L = 40.0
    I = integrate.quad(lambda e: dpsi(e) ** 2, -L, L, limit=200)[0]
    J = -integrate.quad(lambda e: pprime(psi0(e)) * dpsi(e), -L, L, limit=200)[0]
    Hint = lambda e: integrate.quad(lambda z: h(psi0(z)), 0, e, limit=200)[0]
    K = integrate.quad(lambda e: pprime(psi0(e)) * dpsi(e) * Hint(e), -L, L, limit=200)[0]
    H = integrate.quad(lambda e: h(psi0(e)), 0, L, limit=200)[0]   # H+ (= H-)
    g = golden("thin_interface_constants.json")
    env = {k: g[k] for k in ("beta_psi", "psi_s", "psi_l")}
    assert math.isclose(J, g["J"], rel_tol=1e-9)
    assert math.isclose(I, golden_expr(g["I_expr"], **env), rel_tol=1e-9)
    assert math.isclose(H, golden_expr(g["H_expr"], **env), rel_tol=1e-8)
    assert math.isclose(K, golden_expr(g["K_expr"], **env), rel_tol=1e-7)
    a1, a2 = I / J, (K + J * H) / I
    r = g["lambda_prime_over_lambda"]
    assert math.isclose(a1 * r, g["a1_prime"], rel_tol=1e-9)
    assert math.isclose(a2 / r, g["a2_prime"], rel_tol=1e-7)
    assert math.isclose(g["a1_prime"], golden_expr(g["a1_prime_expr"]), rel_tol=1e-15)
    assert math.isclose(g["a2_prime"], golden_expr(g["a2_prime_expr"]), rel_tol=1e-15)
    # the oracle's lambda' obeys tau0 D / W0^2 = a2' lambda'
    o = oracle.Oracle(4, 4, params())
    d = o.derived()
    p = params()
    assert math.isclose(p["tau0"] * p["D"] / p["W0"] ** 2, g["a2_prime"] * d["lambda_p"],
                        rel_tol=1e-14)


def test_isothermal_closure_identity():
    """theta_sys = -M c_inf Omega / (1 - (1-k) Omega) with M c_inf = 1 - (1-k) Omega
    reduces to theta_sys = -Omega, and F(U) = 1 at U = Omega/(1-(1-k)Omega)
    with 1/Le -> 0 (Eq. eq-Tsys)."""
    for Om, k in ((0.55, 0.15), (0.3, 0.5), (0.65, 0.15)):
        o = oracle.Oracle(4, 4, params(Omega=Om, k=k))
        d = o.derived()
        assert math.isclose(d["theta_sys"], -Om, rel_tol=1e-14)
        assert math.isclose(d["Mc_inf"], 1 - (1 - k) * Om, rel_tol=1e-14)
        U = Om / (1 - (1 - k) * Om)
        assert math.isclose(d["Mc_inf"] * (1 + (1 - k) * U), 1.0, rel_tol=1e-14)
    # the paper's printed case: Omega = 0.55, k = 0.15
    g = golden("isothermal_closure.json")
    d = oracle.Oracle(4, 4, params(Omega=g["Omega"], k=g["k"])).derived()
    assert math.isclose(d["Mc_inf"], g["Mc_inf"], rel_tol=1e-14)
    assert math.isclose(d["theta_sys"], g["theta_sys"], rel_tol=1e-14)


def test_supersaturation_and_source_special_values():
    """U = 0 on the equilibrium concentration C = 1 - (1-k) h(psi) (Section 2.1,
    case B), and Q_psi vanishes in the bulk phases psi = +-1 away from gas."""
    o = oracle.Oracle(4, 4, params())
    for psi in (-1.0, -0.3, 0.4, 1.0):
        C = 1 - 0.85 * (1 + psi) / 2
        U, _ = o.pointwise(1.0, psi, C)
        assert abs(U) < 1e-15
    for psi in (-1.0, 1.0):
        _, Q = o.pointwise(1.0, psi, 0.9)
        assert abs(Q) < 1e-15
    # at psi = 0, phi = 1: Q = -lambda' (theta_sys + Mc_inf U) (only the drive is left)
    U, Q = o.pointwise(1.0, 0.0, 0.8)
    d = o.derived()
    assert math.isclose(Q, -d["lambda_p"] * (d["theta_sys"] + d["Mc_inf"] * U), rel_tol=1e-14)
    # gas-solid repulsion: with phi = 0 the interaction term pushes psi down
    _, Qg = o.pointwise(0.0, 0.0, 0.0)
    _, Ql = o.pointwise(1.0, 0.0, 0.0)
    assert math.isclose(Ql - Qg, 2 * 0.75 * 1.0, rel_tol=1e-13)


# ---------------------------------------------------------------------------
# Whole-step invariants and special cases
# ---------------------------------------------------------------------------
def test_conservation_of_gas_and_solute():
    """The CAC equation (Eq. eq-ACE) and the solute equation are in divergence
    form: sum phi and sum C are constant to rounding, with seeds, bubbles,
    gravity and anisotropy all active."""
    lay = wl.random_layout(64, 48, 2, 2, rng_seed=7, R_max=10)
    o = oracle.Oracle(64, 48, lay.params)
    o.init_spec(lay.seeds, lay.R_s, lay.bubbles)
    d0 = o.diag()
    o.step(200)
    d = o.diag()
    assert d["nonfinite"] == 0
    assert abs(d["sum_phi"] / d0["sum_phi"] - 1) < 1e-12
    assert abs(d["sum_C"] / d0["sum_C"] - 1) < 1e-12
    assert d["sum_hpsi"] != d0["sum_hpsi"]          # the dendrites did evolve


def test_single_dendrite_fourfold_symmetry():
    """A single centred seed with a zero grain angle grows with the exact discrete
    D4 symmetry of the square lattice and of a_s (Section 3.3)."""
    N = 48
    o = oracle.Oracle(N, N, params(g=0.0))
    o.init_spec([(N / 2, N / 2, 0.0)], 6.0, [])
    o.step(150)
    f = o.fields()
    psi = f["psi"]
    refl_x = np.roll(psi[:, ::-1], 1, axis=1)
    refl_y = np.roll(psi[::-1, :], 1, axis=0)
    assert np.abs(psi - refl_x).max() < 1e-12
    assert np.abs(psi - refl_y).max() < 1e-12
    assert np.abs(psi - psi.T).max() < 1e-12
    assert np.abs(f["C"] - f["C"].T).max() < 1e-12
    assert psi.max() > 0.5


def test_rotated_grain_breaks_the_axis_symmetry():
    N = 48
    o = oracle.Oracle(N, N, params(g=0.0))
    o.init_spec([(N / 2, N / 2, math.pi / 8)], 6.0, [])
    o.step(150)
    psi = o.fields()["psi"]
    assert np.abs(psi - np.roll(psi[:, ::-1], 1, axis=1)).max() > 1e-6


def _tanh_width(dist, prof, half0, width0):
    from scipy.optimize import curve_fit
    (w, h), _ = curve_fit(lambda d, w, h: np.tanh((h - d) / w), dist, prof, p0=(width0, half0))
    return w, h


def test_flat_cac_interface_is_stationary():
    """A flat gas layer initialised with the equilibrium profile of
    Eq. (eq-phiEq), phi = 1/2 + 1/2 tanh(d / (2 sqrt2 W_phi)), is a stationary
    state of the CAC equation (Section 2.2): after 10^4 steps it no longer
    moves, keeps the tanh width and position and stays at rest.

    The discrete steady profile is not the tanh to 1e-6: the lattice stencils
    and the regularised normal (reading R6) leave 2.1e-3 (measured; the bulk
    phases settle at 2.3e-3 from 0 and 1), so that is bounded at 2.5e-3,
    while the fitted width is held to 0.5 %, which a 1 % error in the
    sharpening coefficient kappa already breaks (-0.76 % and +1.24 % for
    kappa x 1.01 and x 0.99, measured)."""
    m = pin_cases.flat_layer()
    assert pin_cases.flat_layer_holds(m), m
    # a profile of the wrong width (W_phi -> 1.2 W_phi) is clearly excluded
    assert not abs(m[3] - 0.2) < 0.1


def _front_width(angle):
    nx, ny, W0, eps = 128, 4, 4.0, 0.05
    x = np.arange(nx, dtype=float)
    d = np.abs(x - 64.0)
    psi1 = np.tanh((24.0 - d) / (math.sqrt(2) * W0))
    psi = np.tile(psi1[None, :], (ny, 1))
    C = 1 - 0.85 * (1 + psi) / 2
    o = oracle.Oracle(nx, ny, params(g=0.0, Omega=0.0, eps_s=eps))
    o.set_orientation([(64.0, 2.0, angle)])
    o.init_fields(np.ones_like(psi), psi, C)
    o.step(2000)
    return _tanh_width(d, o.fields()["psi"][0], 24.0, math.sqrt(2) * W0)


def test_flat_dendrite_front_has_the_anisotropic_width():
    """With no gas and zero driving force (Omega = 0, so theta_sys + M c_inf U = 0
    on U = 0), a flat solid slab relaxes to psi = tanh(x / (sqrt2 W0 a_s))
    (Eq. eq-psiEq with W_psi = W0 a_s): a_s = 1 + eps for a front along <10>
    and 1 - eps for a grain turned by 45 degrees (Section 3.3)."""
    eps, W0 = 0.05, 4.0
    w_axis, h_axis = _front_width(0.0)
    w_diag, h_diag = _front_width(math.pi / 4)
    assert math.isclose(w_axis, math.sqrt(2) * W0 * (1 + eps), rel_tol=0.02)
    assert math.isclose(w_diag, math.sqrt(2) * W0 * (1 - eps), rel_tol=0.02)
    assert math.isclose(w_axis / w_diag, (1 + eps) / (1 - eps), rel_tol=0.005)
    assert abs(h_axis - 24.0) < 0.1 and abs(h_diag - 24.0) < 0.1


def test_taylor_green_decay():
    """Single-phase liquid (phi = 1, psi = -1, g = 0): the Taylor-Green vortex
    decays as exp(-nu (kx^2 + ky^2) t) (textbook solution of the incompressible
    Navier-Stokes equations of Section 2.2)."""
    N, U0, nu = 48, 1e-3, 0.1
    k = 2 * math.pi / N
    y, x = np.mgrid[0:N, 0:N].astype(float)
    vx = -U0 * np.cos(k * x) * np.sin(k * y)
    vy = U0 * np.sin(k * x) * np.cos(k * y)
    p = -0.25 * U0 * U0 * (np.cos(2 * k * x) + np.cos(2 * k * y))
    one = np.ones_like(x)
    o = oracle.Oracle(N, N, params(g=0.0, nu=nu))
    o.init_fields(one, -one, one, vx, vy, p)
    T = 400
    o.step(T)
    f = o.fields()
    amp = (f["vx"] * vx + f["vy"] * vy).sum() / (vx * vx + vy * vy).sum()
    assert math.isclose(amp, math.exp(-2 * nu * k * k * T), rel_tol=5e-3)


def test_solute_gaussian_spreads_with_variance_2Dt():
    """In the liquid (psi = -1, phi = 1, v = 0) the solute equation reduces to
    dC/dt = D lap C (q = 1, (1-k) U = C - 1): a Gaussian's variance grows by
    2 D t per direction."""
    N, D, s0 = 96, 0.1, 4.0
    y, x = np.mgrid[0:N, 0:N].astype(float)
    r2 = (x - 48) ** 2 + (y - 48) ** 2
    C = 1 + 0.1 * np.exp(-r2 / (2 * s0 * s0))
    one = np.ones_like(x)
    o = oracle.Oracle(N, N, params(g=0.0, D=D))
    o.init_fields(one, -one, C)
    T = 300
    o.step(T)
    c = o.fields()["C"] - 1
    var = ((x - 48) ** 2 * c).sum() / c.sum()
    assert math.isclose(var, s0 * s0 + 2 * D * T, rel_tol=2e-3)


def test_solid_has_zero_velocity():
    """Drag of reading R2: v = (1 - h(psi)) v*, so inside fully solid material
    (psi = 1) the velocity is exactly zero while the melt keeps flowing."""
    N = 48
    y, x = np.mgrid[0:N, 0:N].astype(float)
    psi = np.where((abs(x - 24) < 12) & (abs(y - 24) < 12), 1.0, -1.0)
    one = np.ones_like(x)
    o = oracle.Oracle(N, N, params(g=0.0))
    o.init_fields(one, psi, one - 0.85 * (1 + psi) / 2, 1e-3 * one, 0 * one)
    o.step(5)           # information travels one site per step: the core is untouched
    f = o.fields()
    inner = (abs(x - 24) < 5) & (abs(y - 24) < 5)
    assert np.abs(f["psi"][inner] - 1.0).max() < 1e-14
    assert np.abs(f["vx"][inner]).max() < 1e-15          # v = (1 - h(psi)) v*, h = 1
    assert np.abs(f["vx"][~((abs(x - 24) < 16) & (abs(y - 24) < 16))]).min() > 5e-4


def test_gas_layer_translates_with_uniform_flow():
    """Galilean check of the CAC advection and its dt(phi v) term (Eq. eq-ACE):
    a flat gas layer in a uniform flow normal to it is carried rigidly at that
    speed and the flow stays uniform.  A flow normal to a flat layer is held
    uniform by incompressibility alone, so this check does not involve the
    mass-consistent momentum flux; test_mass_consistent_flux_keeps_a_parallel_
    flow_uniform does."""
    nx, ny, W, V = 4, 128, 2.0, 0.01
    y = np.arange(ny, dtype=float)
    phi1 = 0.5 + 0.5 * np.tanh((np.abs(y - 64.0) - 24.0) / (2 * math.sqrt(2) * W))
    phi = np.tile(phi1[:, None], (1, nx))
    one = np.ones_like(phi)
    o = oracle.Oracle(nx, ny, params(g=0.0, sigma=0.0, W_phi=W))
    o.init_fields(phi, -one, phi, 0 * one, V * one)
    T = 600
    o.step(T)
    f = o.fields()
    # density-contrast start-up waves perturb the flow by a few per cent
    assert np.abs(f["vy"] - V).max() < 0.05 * V
    assert np.abs(f["vx"]).max() == 0.0
    moved = np.roll(phi1, int(V * T))          # 6 lattice units
    assert np.abs(f["phi"][:, 0] - moved).max() < 3e-3
    assert np.abs(f["phi"][:, 0] - phi1).max() > 0.1     # it did move


def test_mass_consistent_flux_keeps_a_parallel_flow_uniform():
    """Section 2.2: with the mass-consistent flux m = rho v - D (rho_l -
    rho_g) / (phi_l - phi_g) in d(rho v)/dt + div(m v), a uniform velocity is
    an exact solution whatever the gas layer does, since d rho/dt + div m = 0
    by the CAC equation.  A flat layer started at 1.5x its equilibrium width
    relaxes (div D != 0) in a uniform flow V parallel to it: the flow stays
    within 2 % of V over 300 steps (measured 0.56 %); with rho v in place of
    m it falls by 15 % where the layer's density grows."""
    dev, vy = pin_cases.mass_flux_deviation("2d")
    assert dev < pin_cases.MASS_FLUX_TOL
    assert vy < 1e-5


def test_time_stretch_follows_the_original_equation():
    """Eq. eq-AnACE has tau0 a_s^2 d psi/dt on its left; the LB form of
    Appendix B carries the a_s^2 by the time stretch t + a_s^2 dt.  A solid
    slab whose fronts lie along <10> (a_s = 1 + eps_s = 1.05, N = 0) grows into
    an undercooled melt for 1200 steps.  The oracle's psi agrees with an
    explicit finite-difference solution of the 1-D original equations to
    0.006 (measured 0.0027), a quarter of the distance between that solution
    and the one with tau0 a_s (0.028): the stretch is there and has its
    square.  Without any stretch the solutions differ by 0.056."""
    errs, nonuniform = pin_cases.stretch_errors("2d")
    psi0, _ = pin_cases.front_initial()
    assert np.abs(pin_cases.front_fd(2) - psi0).max() > 0.5          # the fronts moved
    gap = np.abs(pin_cases.front_fd(2) - pin_cases.front_fd(1)).max()
    assert gap > 0.02
    assert errs[2] < 0.006 and errs[2] < 0.25 * gap
    assert pin_cases.stretch_pin_holds(errs)
    assert errs[1] > 0.02 and errs[0] > 0.04
    assert nonuniform < 1e-12


@pytest.mark.parametrize("N,R,T", [(64, 10.0, 3000), (64, 14.0, 3000), (96, 16.0, 4000),
                                   (96, 24.0, 4000)])
def test_laplace_law_static_bubble(N, R, T):
    """Young-Laplace, Eq. (eq-laplace): a static bubble in a periodic box (no
    solid, no gravity) settles to p_in - p_out = sigma / R (measured within 2 %
    for R = 10 .. 24).  nu = 0.3 damps the start-up pressure waves within the
    run; the residual velocity after these runs, 1.5e-6 .. 7.5e-6, is still
    the decaying start-up transient (see the parasitic-current pin)."""
    W, sigma = 2.0, 1e-3
    o = oracle.Oracle(N, N, params(g=0.0, W_phi=W, nu=0.3, sigma=sigma))
    o.init_spec([], 6.0, [(N / 2, N / 2, R)])
    o.step(T)
    d = o.diag((N / 2, N / 2, R, W))
    dp = d["p_in_sum"] / d["p_in_n"] - d["p_out_sum"] / d["p_out_n"]
    assert math.isclose(dp, sigma / R, rel_tol=0.03)
    assert d["max_v"] < 1e-5


def test_parasitic_current_of_a_static_bubble_below_1e6():
    """The residual velocity around a static bubble (R = 16, W = 2, sigma =
    1e-3, nu = 0.3, no gravity) is a decaying start-up transient: 1.5e-6 after
    4000 steps, 1e-6 after 8000, 4.2e-7 after 16000 (measured).  After 16000
    steps it is below 1e-6 lu, the spurious-current bound for the Laplace
    problem (Section 3.1), with the pressure jump sigma / R to 1 %."""
    N, R, W, sigma = 96, 16.0, 2.0, 1e-3
    o = oracle.Oracle(N, N, params(g=0.0, W_phi=W, nu=0.3, sigma=sigma))
    o.init_spec([], 6.0, [(N / 2, N / 2, R)])
    o.step(16000)
    d = o.diag((N / 2, N / 2, R, W))
    dp = d["p_in_sum"] / d["p_in_n"] - d["p_out_sum"] / d["p_out_n"]
    assert math.isclose(dp, sigma / R, rel_tol=0.01)
    assert d["max_v"] < 1e-6


def _contour_radius(phi, xc, yc, ang, level=0.5):
    """Distance from (xc, yc) along direction ang to the first crossing of
    phi = level (bilinear interpolation, march of 0.05 lu)."""
    def samp(px, py):
        i0, j0 = int(math.floor(px)), int(math.floor(py))
        fx, fy = px - i0, py - j0
        return ((1 - fx) * (1 - fy) * phi[j0, i0] + fx * (1 - fy) * phi[j0, i0 + 1] +
                (1 - fx) * fy * phi[j0 + 1, i0] + fx * fy * phi[j0 + 1, i0 + 1])
    prev, t, dt = samp(xc, yc), 0.0, 0.05
    while t < min(phi.shape) / 2 - 2:
        t += dt
        v = samp(xc + t * math.cos(ang), yc + t * math.sin(ang))
        if v >= level:
            return t - dt + dt * (level - prev) / (v - prev)
        prev = v
    raise AssertionError("no contour crossing")


def test_square_droplet_relaxes_to_circle():
    """Section 3.1: a square of side sqrt(pi) R_eq relaxes under surface
    tension to a circle of radius R_eq, with Delta P = sigma / R_eq
    (Eq. eq-laplace).  The paper's box [-1, 1]^2 with R_eq = 0.5 is scaled to a
    64^2 periodic lattice (R_eq = 16 lu); here the square is a gas region
    (phi = 0 inside) in liquid.  Initially the phi = 1/2 contour lies at
    side/2 = 14.2 lu along the axes and side/sqrt2 = 20.1 lu along the
    diagonals; a wrong sign or size of the surface-tension force leaves it
    square or drives it elsewhere."""
    g = golden("square_droplet.json")
    N = 64
    R_eq = g["R_eq"] / g["box_side"] * N
    side = g["side_over_R_eq"] * R_eq
    W, sigma = 2.0, 5e-3
    o = oracle.Oracle(N, N, params(g=0.0, W_phi=W, nu=0.3, sigma=sigma))
    kap = math.sqrt(2 * 0.25) / W
    y, x = np.mgrid[0:N, 0:N].astype(float)
    xc = yc = N / 2
    dist = np.maximum(abs(x - xc), abs(y - yc)) - side / 2
    phi = 0.5 + 0.5 * np.tanh(kap * dist / 2)
    o.init_fields(phi, -np.ones_like(phi), phi.copy())
    o.step(4000)
    f = o.fields(("phi",))["phi"]
    r_ax = [_contour_radius(f, xc, yc, a) for a in (0, math.pi / 2, math.pi, 1.5 * math.pi)]
    r_dg = [_contour_radius(f, xc, yc, a) for a in (math.pi / 4, 3 * math.pi / 4)]
    assert max(r_ax + r_dg) - min(r_ax + r_dg) < 0.1, (r_ax, r_dg)
    assert math.isclose(np.mean(r_ax + r_dg), R_eq, rel_tol=0.02)
    d = o.diag((xc, yc, R_eq, W))
    dp = d["p_in_sum"] / d["p_in_n"] - d["p_out_sum"] / d["p_out_n"]
    assert math.isclose(dp, sigma / R_eq, rel_tol=0.03)


def test_complex_step_matches_finite_difference():
    """The complex build's derivative equals a central difference of the
    double build (h = 1e-5 relative) for each differentiable parameter."""
    lay = wl.random_layout(32, 32, 1, 1, rng_seed=11, R_max=8)
    base = dict(lay.params, g=1e-5)
    T = 20
    for name in ("eps_s", "Omega", "sigma"):
        oz = oracle.Oracle(32, 32, base, complex_step=True)
        oz.perturb(name, 1e-30)
        oz.init_spec(lay.seeds, lay.R_s, lay.bubbles)
        oz.step(T)
        dj = oz.objective()[1] / 1e-30
        h = 1e-5 * base[name]
        js = []
        for sgn in (1, -1):
            od = oracle.Oracle(32, 32, dict(base, **{name: base[name] + sgn * h}))
            od.init_spec(lay.seeds, lay.R_s, lay.bubbles)
            od.step(T)
            js.append(od.objective()[0])
        fd = (js[0] - js[1]) / (2 * h)
        assert math.isclose(dj, fd, rel_tol=1e-4, abs_tol=1e-9), (name, dj, fd)


def test_diagnostics_and_objective_against_their_definitions():
    """The FP64 diagnostics (S12: totals, gas centroid, Laplace probe means,
    max |v|) and the final-state objective J = mean h(psi) + y_c / L_y
    (readings R16, R17) recomputed with numpy from the oracle's own fields."""
    lay = wl.random_layout(64, 48, 2, 2, rng_seed=13, R_min=4, R_max=8)
    o = oracle.Oracle(lay.nx, lay.ny, dict(lay.params, g=1e-5))
    o.init_spec(lay.seeds, lay.R_s, lay.bubbles)
    o.step(15)
    f = o.fields(("phi", "psi", "C", "p", "vx", "vy"))
    phi, psi, C, p = f["phi"], f["psi"], f["C"], f["p"]
    y, x = np.mgrid[0:lay.ny, 0:lay.nx].astype(float)
    xc, yc, R, W = lay.bubbles[0][0], lay.bubbles[0][1], lay.bubbles[0][2], 4.0

    def mi(d, L):
        return (d + 0.5 * L) % L - 0.5 * L

    r = np.hypot(mi(x - xc, lay.nx), mi(y - yc, lay.ny))
    inside, outside = r < R - 2 * W, r > R + 4 * W
    ref = {"sum_phi": phi.sum(), "sum_C": C.sum(), "sum_hpsi": (0.5 * (1 + psi)).sum(),
           "gas": (1 - phi).sum(), "gas_x": (x * (1 - phi)).sum(), "gas_y": (y * (1 - phi)).sum(),
           "p_in_sum": p[inside].sum(), "p_in_n": inside.sum(), "p_out_sum": p[outside].sum(),
           "p_out_n": outside.sum(), "max_v": np.hypot(f["vx"], f["vy"]).max(), "nonfinite": 0}
    d = o.diag((xc, yc, R, W))
    for k, v in ref.items():
        assert math.isclose(d[k], float(v), rel_tol=1e-12, abs_tol=1e-15), (k, d[k], v)
    J = (0.5 * (1 + psi)).mean() + ((y * (1 - phi)).sum() / (1 - phi).sum()) / lay.ny
    assert math.isclose(o.objective()[0], J, rel_tol=1e-13)
