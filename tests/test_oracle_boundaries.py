"""Pins of the oracle's boundary conditions (Section 3, model parameters:
half-way bounce-back for no-slip and no-flux walls, the symmetric scheme for
symmetry planes; Section 4: far-field Dirichlet values psi = psi_l, C = 1,
theta = -Omega), as read in reading R31.

Each test checks the oracle against something other than its own formulas:
the closed-form decay of a shear wave between no-slip walls, the exact
equivalence of a symmetric side with the mirrored half of a periodic lattice
twice as large, conservation in a closed box, and the Fourier-series solution
of diffusion between a no-flux wall and a Dirichlet side.
"""
import math

import numpy as np

import oracle
import pin_cases
from paper_2407_01651_gb300 import workload as wl

PERIODIC, SYMMETRIC, WALL, FARFIELD = 0, 1, 2, 3


def shear_wave_between_walls_holds(lib=None) -> bool:
    """The lowest shear mode between half-way walls after 600 and 1500 steps:
    its amplitude at exp(-nu (pi/H)^2 t) (1e-3), its shape kept, no v_y."""
    nx, ny, U0 = 4, 32, 1e-3
    p = dict(wl.BASE_PARAMS, g=0.0)
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    mode = np.sin(math.pi * (y + 0.5) / ny)
    one = np.ones_like(x)
    o = oracle.Oracle(nx, ny, p, lib=lib)
    o.set_bc(PERIODIC, PERIODIC, WALL, WALL)
    o.init_fields(one, -one, one, U0 * mode, 0 * one, 0 * one)
    ok = True
    for T in (600, 1500):
        o.step(T - o.steps)
        f = o.fields(("vx", "vy"))
        amp = (f["vx"] * mode).sum() / (mode * mode).sum()
        ok = ok and (math.isclose(amp / U0, math.exp(-p["nu"] * (math.pi / ny) ** 2 * T),
                                  rel_tol=1e-3) and
                     np.abs(f["vx"] - amp * mode).max() < 1e-4 * U0 and
                     np.abs(f["vy"]).max() < 1e-5 * U0)
    return bool(ok)


def test_shear_wave_between_walls_decays_at_the_viscous_rate():
    """v_x = U sin(pi (y + 1/2) / H) between half-way bounce-back walls at
    y = -1/2 and y = H - 1/2 decays as exp(-nu (pi/H)^2 t) with its shape kept:
    the walls sit exactly half-way and carry no slip."""
    assert shear_wave_between_walls_holds()


def mirror_equivalence_holds(axis=0, thermal=False, lib=None) -> bool:
    """The symmetric-side lattice against one half of the mirrored periodic
    lattice of twice its size: every field to 1e-12, with flow present."""
    try:
        _mirror_equivalence(axis, thermal, lib=lib)
    except AssertionError:
        return False
    return True


def _mirror_equivalence(axis, thermal, T=60, lib=None):
    nx, ny = 40, 48
    p = dict(wl.BASE_PARAMS, g=(1e-5 if axis == 0 else 0.0))
    if thermal:
        p.update(wl.THERMAL_PARAMS, Le=2.0)
    a = oracle.Oracle(nx, ny, p, lib=lib)
    a.set_bc(*((SYMMETRIC, SYMMETRIC, PERIODIC, PERIODIC) if axis == 0
               else (PERIODIC, PERIODIC, SYMMETRIC, SYMMETRIC)))
    a.init_spec([(12.3, 20.7, 0.0)], 6.0, [(28.4, 30.2, 9.0)])
    f0 = a.fields(("phi", "psi", "C"))
    if axis == 0:
        NX, NY = 2 * nx, ny
        mir = lambda f: np.concatenate([f, f[:, ::-1]], axis=1)      # noqa: E731
        half = lambda f: f[:, :nx]                                     # noqa: E731
    else:
        NX, NY = nx, 2 * ny
        mir = lambda f: np.concatenate([f, f[::-1, :]], axis=0)      # noqa: E731
        half = lambda f: f[:ny, :]                                     # noqa: E731
    b = oracle.Oracle(NX, NY, p, lib=lib)
    b.set_rho_bar(a.rho_bar)
    b.init_fields(mir(f0["phi"]), mir(f0["psi"]), mir(f0["C"]))
    a.step(T)
    b.step(T)
    fa, fb = a.fields(), b.fields()
    for k in fa:
        scale = max(np.abs(half(fb[k])).max(), 1e-30)
        assert np.abs(fa[k] - half(fb[k])).max() <= 1e-12 * scale, (axis, k)
    assert fa["psi"].max() > 0.5 and np.abs(fa["vx"]).max() > 0.0


def test_symmetric_sides_equal_the_mirrored_periodic_lattice():
    """A lattice with symmetric planes on two opposite sides evolves exactly
    like one half of the periodic lattice of twice its size whose initial
    fields are mirrored (the symmetric scheme reflects populations and the
    normal velocity), with a seed, a bubble, flow and gravity along the
    planes, in the isothermal and thermal models."""
    _mirror_equivalence(0, False)
    _mirror_equivalence(1, False)
    _mirror_equivalence(0, True)


def test_closed_box_conserves_gas_solute_and_enthalpy():
    """Half-way bounce-back on all four sides returns every population to its
    site: sum phi, sum C and sum rho H stay constant with bubbles rising and a
    dendrite growing."""
    lay = wl.random_layout(56, 64, 2, 2, rng_seed=9, R_max=9)
    p = dict(lay.params, g=1e-5, **dict(wl.THERMAL_PARAMS, Le=2.0))
    o = oracle.Oracle(lay.nx, lay.ny, p)
    o.set_bc(WALL, WALL, WALL, WALL)
    o.init_spec(lay.seeds, lay.R_s, lay.bubbles)
    d0, t0 = o.diag(), o.thermal_totals()
    o.step(200)
    d, t = o.diag(), o.thermal_totals()
    assert d["nonfinite"] == 0 and d["max_v"] > 0
    assert abs(d["sum_phi"] / d0["sum_phi"] - 1) < 1e-12
    assert abs(d["sum_C"] / d0["sum_C"] - 1) < 1e-12
    assert abs(t["sum_e"] / t0["sum_e"] - 1) < 1e-12


def _series(v0, vfar, D, t, L, yw):
    """Diffusion on [0, L] with zero flux at 0, u(L) = vfar, u(0, .) = v0."""
    u = np.full_like(yw, vfar)
    for n in range(400):
        k = (n + 0.5) * math.pi / L
        u += (v0 - vfar) * 2 * (-1) ** n / ((n + 0.5) * math.pi) * np.cos(k * yw) * math.exp(
            -D * k * k * t)
    return u


def far_field_series_holds(lib=None) -> bool:
    """C and theta of a melt column between a no-flux wall and a far-field
    side after 1000 steps against the series solution; psi stays psi_l."""
    nx, ny = 4, 40
    p = dict(wl.BASE_PARAMS, g=0.0, **dict(wl.THERMAL_PARAMS, Le=1.0, theta0=-0.55))
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    one = np.ones_like(x)
    o = oracle.Oracle(nx, ny, p, lib=lib)
    o.set_bc(PERIODIC, PERIODIC, WALL, FARFIELD)
    o.init_fields(one, -one, 0.5 * one, theta=-0.3 * one)
    o.step(1000)
    f = o.fields(("C", "theta", "psi"))
    yw = y[:, 0] + 0.5
    return bool(np.abs(f["C"] - _series(0.5, 1.0, p["D"], 1000, ny, yw)[:, None]).max() < 2e-4 and
                np.abs(f["theta"] - _series(-0.3, -0.55, p["D"], 1000, ny, yw)[:, None]).max()
                < 2e-3 and np.abs(f["psi"] + 1).max() < 1e-14)


def test_far_field_dirichlet_against_the_diffusion_series():
    """A melt column between a no-flux wall (y = -1/2) and a far-field side
    (y = H - 1/2) with C = 1 and theta = -Omega there: from uniform C = 0.5 and
    theta = -0.3 both relax like the series solution of the diffusion
    equation (D for C, alpha = Le D for theta); psi stays at psi_l."""
    assert far_field_series_holds()


INLET, OUTLET, INLET_NEE = 4, 5, 6


def test_plug_flow_through_inlet_and_outlet_is_exact():
    """A uniform liquid inflow through a channel with symmetric sides is an
    exact steady state of the inlet (moving-wall bounce-back at u_in) and the
    pressure outlet (p = 0): velocity, pressure and the scalars stay uniform."""
    nx, ny, vin = 8, 40, 0.01
    p = dict(wl.BASE_PARAMS, g=0.0, vin_y=vin)
    one = np.ones((ny, nx))
    o = oracle.Oracle(nx, ny, p)
    o.set_bc(SYMMETRIC, SYMMETRIC, INLET, OUTLET)
    o.init_fields(one, -one, one, 0 * one, vin * one, 0 * one)
    o.step(400)
    f = o.fields(("vx", "vy", "p", "phi", "C", "psi"))
    assert np.abs(f["vy"] / vin - 1).max() < 1e-12
    assert np.abs(f["vx"]).max() < 1e-15 and np.abs(f["p"]).max() < 1e-14
    for k, v in (("phi", 1.0), ("C", 1.0), ("psi", -1.0)):
        assert np.abs(f[k] - v).max() < 1e-14, k


def test_inflow_between_walls_develops_the_poiseuille_profile():
    """Inflow at u_in between two no-slip walls (width W) relaxes downstream to
    the plane Poiseuille profile 6 u_in xi (1 - xi), xi = (x + 1/2) / W, and
    the volume flux W u_in is the same through every row."""
    W, L, vin = 16, 96, 0.01
    p = dict(wl.BASE_PARAMS, g=0.0, vin_y=vin)
    one = np.ones((L, W))
    o = oracle.Oracle(W, L, p)
    o.set_bc(WALL, WALL, INLET, OUTLET)
    o.init_fields(one, -one, one, 0 * one, 0 * one, 0 * one)
    o.step(6000)
    f = o.fields(("vx", "vy"))
    xi = (np.arange(W) + 0.5) / W
    assert np.abs(f["vy"][L - 20] - 6 * vin * xi * (1 - xi)).max() < 5e-3 * 1.5 * vin
    flux = f["vy"].sum(axis=1) / (W * vin)
    assert np.abs(flux - 1).max() < 1e-3
    assert np.abs(f["vx"][L - 20]).max() < 1e-3 * vin


def _forced_convection(vin, T=2500):
    nx, ny = 64, 128
    p = dict(wl.BASE_PARAMS, g=0.0, vin_y=vin)
    cx, cy = -0.5, ny / 2          # seed centred on the symmetry plane x = -1/2
    o = oracle.Oracle(nx, ny, p)
    o.set_bc(SYMMETRIC, SYMMETRIC, INLET, OUTLET)
    phi, psi, C = o.fields_from_spec([(cx, cy, 0.0)], 6.0, [])
    o.set_orientation([(cx, cy, 0.0)])
    o.init_fields(phi, psi, C, 0 * phi, vin * (1 - 0.5 * (1 + psi)), 0 * phi)
    o.step(T)
    f = o.fields(("psi",))["psi"]

    def arm(arr, start, step):        # distance to the psi = 0 crossing
        i = start
        while 0 <= i + step < len(arr) and arr[i + step] > 0:
            i += step
        a, b = arr[i], arr[i + step]
        return abs(i - start) + a / (a - b)
    col, row = f[:, 0], f[int(cy), :]
    return arm(col, int(cy), -1), arm(col, int(cy), +1), arm(row, 0, +1)


def test_forced_convection_favours_the_upstream_arm():
    """Section 3.3 (dendritic growth with an inlet velocity): the arm growing
    against the flow is longer than the normal and the downstream arms.  The
    same growth without inflow is symmetric between up and down."""
    up, down, normal = _forced_convection(0.025)
    assert up > down + 0.3 and up > normal + 0.5
    up0, down0, normal0 = _forced_convection(0.0)
    assert abs(up0 - down0) < 0.05


# ---------------------------------------------------------------------------
# Dirichlet velocity by non-equilibrium extrapolation (Section 3, reading R37):
# the boundary node is the ghost one site beyond the side; its NS populations
# are the equilibrium at u_in plus the non-equilibrium part of the fluid site
# next to it.
# ---------------------------------------------------------------------------
def test_nee_inlet_plug_flow_is_exact():
    """Uniform liquid inflow through a symmetric channel is an exact steady
    state with the extrapolation inlet too: the fluid site's non-equilibrium
    part is the ghost's, so nothing changes."""
    nx, ny, vin = 8, 40, 0.01
    p = dict(wl.BASE_PARAMS, g=0.0, vin_y=vin)
    one = np.ones((ny, nx))
    o = oracle.Oracle(nx, ny, p)
    o.set_bc(SYMMETRIC, SYMMETRIC, INLET_NEE, OUTLET)
    o.init_fields(one, -one, one, 0 * one, vin * one, 0 * one)
    o.step(400)
    f = o.fields(("vx", "vy", "p", "phi", "C", "psi"))
    assert np.abs(f["vy"] / vin - 1).max() < 1e-12
    assert np.abs(f["vx"]).max() < 1e-15 and np.abs(f["p"]).max() < 1e-14
    for k, v in (("phi", 1.0), ("C", 1.0), ("psi", -1.0)):
        assert np.abs(f[k] - v).max() < 1e-14, k


def _couette(bc, ny=16, U=0.01):
    nx = 4
    p = dict(wl.BASE_PARAMS, g=0.0, vin_x=U, vin_y=0.0, nu=0.5)
    one = np.ones((ny, nx))
    o = oracle.Oracle(nx, ny, p)
    o.set_bc(PERIODIC, PERIODIC, bc, WALL)
    o.init_fields(one, -one, one, 0 * one, 0 * one, 0 * one)
    o.step(20000)
    return o.fields(("vx", "vy"))


def test_nee_inlet_is_node_based_in_couette_flow():
    """A tangential velocity U imposed on the bottom side against a no-slip
    wall at the top (half-way, y = ny - 1/2) drives Couette flow, whose
    steady profile is linear between the two boundary positions.  With the
    extrapolation the velocity is imposed at the boundary node y = -1: v_x =
    U (ny - 1/2 - y) / (ny + 1/2) to 1e-12 (measured 4e-14).  The moving-wall
    inlet imposes it half-way, at y = -1/2, and gives U (ny - 1/2 - y) / ny
    instead; the two lines differ by 3 % of U."""
    ny, U = 16, 0.01
    y = np.arange(ny)
    node = U * (ny - 0.5 - y) / (ny + 0.5)
    half = U * (ny - 0.5 - y) / ny
    f = _couette(INLET_NEE, ny, U)
    assert np.abs(f["vx"][:, 0] - node).max() < 1e-12 * U / 1e-2
    assert np.abs(f["vy"]).max() < 1e-15
    assert pin_cases.nee_couette_holds()
    g = _couette(INLET, ny, U)
    assert np.abs(g["vx"][:, 0] - half).max() < 1e-10
    assert np.abs(node - half).max() > 0.02 * U


def test_nee_inflow_between_walls_keeps_one_flux_and_develops_poiseuille():
    """A uniform inflow imposed by extrapolation between no-slip walls: the
    volume flux is the same through every row (to 3e-4; measured 1.7e-4) and
    the profile downstream is plane Poiseuille for that flux to 0.5 %
    (measured 0.2 %).  The flux itself falls short of W u_in by a corner loss
    of about 0.42 lu of width (measured 2.65 % at W = 16 and 1.33 % at W = 32,
    first order), where the imposed uniform velocity meets the walls."""
    W, L, vin = 16, 96, 0.01
    p = dict(wl.BASE_PARAMS, g=0.0, vin_y=vin)
    one = np.ones((L, W))
    o = oracle.Oracle(W, L, p)
    o.set_bc(WALL, WALL, INLET_NEE, OUTLET)
    o.init_fields(one, -one, one, 0 * one, 0 * one, 0 * one)
    o.step(6000)
    f = o.fields(("vx", "vy"))
    Q = f["vy"].sum(axis=1)
    Qm = Q[L // 2]
    assert (Q.max() - Q.min()) / Qm < 3e-4
    xi = (np.arange(W) + 0.5) / W
    assert np.abs(f["vy"][L - 20] - 6 * Qm / W * xi * (1 - xi)).max() < 5e-3 * 1.5 * Qm / W
    assert 0.96 < Qm / (W * vin) < 0.99
    assert np.abs(f["vx"][L - 20]).max() < 1e-3 * vin
