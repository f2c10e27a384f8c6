"""Non-periodic domain sides (symmetric planes, half-way bounce-back walls, far
field; reading R31) of the CUDA path against the FP64 oracle, through the C
ABI.  Tolerances as in test_gpu_parity.py: FP64 within 1e-11 relative per field
over a few steps, FP32 within 1e-5 per step (mu_phi 5e-5, early-flow p and v
up to 30x).
"""
import numpy as np
import pytest

import oracle
from paper_2407_01651_gb300 import pf
from paper_2407_01651_gb300 import workload as wl

pytestmark = pytest.mark.gpu

P, S, W, F = pf.BC_PERIODIC, pf.BC_SYMMETRIC, pf.BC_WALL, pf.BC_FARFIELD
I, O = pf.BC_INLET, pf.BC_OUTLET
N = pf.BC_INLET_NEE
FIELDS = ("phi", "psi", "C", "U", "p", "vx", "vy", "mu", "theta")
FLOOR = {"phi": 1e-9, "psi": 1e-9, "C": 1e-9, "U": 1e-9, "p": 1e-12, "vx": 1e-10,
         "vy": 1e-10, "mu": 1e-3, "theta": 1e-9}
EARLY = {"p": 30.0, "vx": 10.0, "vy": 10.0, "mu": 5.0}


def rel(a, b, floor=1e-300):
    return np.abs(a - b).max() / max(np.abs(b).max(), floor)


def compare(o, sim, tol, dom=0, early=False):
    fo, fg = o.fields(FIELDS), sim.fields(dom, FIELDS)
    errs = {k: rel(fg[k], fo[k], FLOOR[k]) for k in FIELDS}
    fac = EARLY if early else {"mu": 5.0}
    bad = {k: v for k, v in errs.items() if not v <= tol * fac.get(k, 1.0)}
    assert not bad, (bad, errs)


def layout():
    # 150 x 52: two strips (the second ragged), two row tiles; a seed and a
    # bubble touch the left and bottom sides, another seed the top-right corner
    return wl.Layout(150, 52, seeds=[(2.0, 3.0, 0.0), (140.0, 47.0, 0.3)],
                     bubbles=[(40.0, 5.0, 9.0), (100.0, 30.0, 12.0)])


def pair(lay, bc, precision, params):
    o = oracle.Oracle(lay.nx, lay.ny, params)
    o.set_bc(*bc)
    o.init_spec(lay.seeds, lay.R_s, lay.bubbles)
    sim = pf.Simulation([(lay.nx, lay.ny)], params, precision)
    sim.set_boundaries(0, *bc)
    sim.init_fields(0, lay.seeds, lay.R_s, lay.bubbles)
    return o, sim


COMBOS = [(S, S, W, F), (W, W, S, S), (F, F, W, W), (P, P, W, F), (S, W, P, P)]


@pytest.mark.parametrize("bc", COMBOS)
def test_fp64_boundaries_match_oracle(bc):
    lay = layout()
    par = dict(lay.params, g=1e-5)
    o, sim = pair(lay, bc, "fp64", par)
    compare(o, sim, 1e-12)
    for _ in range(4):
        o.step(1)
        sim.step(1)
        compare(o, sim, 1e-11, early=True)


@pytest.mark.parametrize("bc", [(S, S, W, F), (F, F, W, W)])
def test_fp32_boundaries_one_step(bc):
    lay = layout()
    o, sim = pair(lay, bc, "fp32", dict(lay.params, g=1e-5))
    o.step(1)
    sim.step(1)
    compare(o, sim, 1e-5, early=True)


def test_thermal_with_far_field_matches_oracle():
    """The paper's Section-4 arrangement: symmetric sides in x, a no-flux wall
    at the bottom and the far field (psi_l, C = 1, theta = theta0) at the top,
    with the temperature lattice on."""
    lay = layout()
    par = {**lay.params, **wl.THERMAL_PARAMS, "Le": 2.0, "g": 1e-5}
    for prec, tol in (("fp64", 1e-11), ("fp32", 1e-5)):
        o, sim = pair(lay, (S, S, W, F), prec, par)
        o.step(1)
        sim.step(1)
        compare(o, sim, tol, early=True)
        if prec == "fp64":
            o.step(40)
            sim.step(40)
            compare(o, sim, 1e-10)


def test_closed_box_conservation_fp64():
    lay = layout()
    par = {**lay.params, **wl.THERMAL_PARAMS, "Le": 2.0, "g": 1e-5}
    o, sim = pair(lay, (W, W, W, W), "fp64", par)
    d0, t0 = sim.reduce(0), sim.reduce_thermal(0)
    sim.step(200)
    d, t = sim.reduce(0), sim.reduce_thermal(0)
    assert d["nonfinite"] == 0 and d["max_v"] > 0
    assert abs(d["sum_phi"] / d0["sum_phi"] - 1) <= 1e-12
    assert abs(d["sum_C"] / d0["sum_C"] - 1) <= 1e-12
    assert abs(t["sum_e"] / t0["sum_e"] - 1) <= 1e-12
    o.step(200)
    compare(o, sim, 1e-9)


def test_mixed_ensemble_and_launch_modes():
    """A periodic domain and two bounded ones in one handle: each matches its
    own oracle (the periodic one through the boundary-aware kernel), and the
    launch modes (one launch, per domain, persistent, graphs) agree bitwise."""
    lays = [wl.random_layout(64, 40, 1, 1, rng_seed=81, R_max=8),
            wl.random_layout(130, 70, 2, 1, rng_seed=82, R_max=8),
            wl.Layout(33, 45, seeds=[(10.0, 12.0, 0.2)], bubbles=[(22.0, 30.0, 8.0)])]
    bcs = [(P, P, P, P), (S, S, W, F), (W, W, W, W)]
    par = dict(wl.BASE_PARAMS)
    outs = []
    for mode in ((0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 1, 4)):
        sim = pf.Simulation([(l.nx, l.ny) for l in lays], par, "fp64")
        for d, (l, bc) in enumerate(zip(lays, bcs)):
            sim.set_boundaries(d, *bc)
            sim.init_fields(d, l.seeds, l.R_s, l.bubbles)
        sim.set_launch(*mode)
        sim.step(9)
        outs.append(sim)
    for d, (l, bc) in enumerate(zip(lays, bcs)):
        o = oracle.Oracle(l.nx, l.ny, par)
        o.set_bc(*bc)
        o.init_spec(l.seeds, l.R_s, l.bubbles)
        o.step(9)
        compare(o, outs[0], 1e-11, dom=d)
        ref = outs[0].fields(d)
        for sim in outs[1:]:
            f = sim.fields(d)
            for k in FIELDS:
                assert np.array_equal(f[k], ref[k]), (d, k)


def test_boundary_configuration_errors():
    lay = layout()
    sim = pf.Simulation([(lay.nx, lay.ny)], lay.params, "fp32")
    with pytest.raises(pf.PFError) as e:
        sim.set_boundaries(0, P, W, P, P)             # unpaired periodic side
    assert e.value.code == pf.PF_ERR_BAD_ARG
    with pytest.raises(pf.PFError):
        sim.set_boundaries(0, 7, 7, P, P)             # unknown type
    sim.set_boundaries(0, S, S, W, F)
    for variant in (0, 2):
        with pytest.raises(pf.PFError):
            sim.set_step_config(variant, 32, 8)
    sim.init_fields(0, lay.seeds, lay.R_s, lay.bubbles)
    with pytest.raises(pf.PFError) as e:
        sim.set_boundaries(0, W, W, W, W)             # after initialisation
    assert e.value.code == pf.PF_ERR_STATE
    with pytest.raises(pf.PFError):
        sim.adjoint_step(4, 1.0, 0.0, 2)
    s16 = pf.Simulation([(32, 32)], lay.params, "fp16")
    with pytest.raises(pf.PFError):
        s16.set_boundaries(0, W, W, W, W)


@pytest.mark.parametrize("bc,vin", [((S, S, I, O), (0.0, 0.01)), ((W, W, I, O), (0.0, 0.02)),
                                    ((I, O, S, W), (0.015, 0.0)), ((O, I, P, P), (-0.01, 0.0))])
def test_inlet_outlet_match_oracle(bc, vin):
    """Inlet (moving-wall bounce-back at u_in) and pressure outlet (reading R32)
    in several arrangements, with seeds and bubbles, FP64 over 6 steps and
    FP32 for one."""
    lay = layout()
    par = dict(lay.params, g=1e-5, vin_x=vin[0], vin_y=vin[1])
    o, sim = pair(lay, bc, "fp64", par)
    for _ in range(6):
        o.step(1)
        sim.step(1)
        compare(o, sim, 1e-11, early=True)
    o32, s32 = pair(lay, bc, "fp32", par)
    o32.step(1)
    s32.step(1)
    compare(o32, s32, 1e-5, early=True)


@pytest.mark.parametrize("bc,vin", [((S, S, N, O), (0.0, 0.01)), ((W, W, N, O), (0.0, 0.02)),
                                    ((N, O, S, W), (0.015, 0.0)), ((P, P, N, W), (0.01, 0.0)),
                                    ((N, W, S, N), (0.01, -0.005))])
def test_extrapolation_inlet_matches_oracle(bc, vin):
    """Velocity inlet by non-equilibrium extrapolation (Section 3, reading
    R37) in several arrangements, among them a tangential (Couette) inflow,
    two extrapolation sides meeting at a corner and one against a symmetric
    side, with seeds and bubbles: FP64 within 1e-11 of the oracle over 6
    steps, FP32 within 1e-5 after one."""
    lay = layout()
    par = dict(lay.params, g=1e-5, vin_x=vin[0], vin_y=vin[1])
    o, sim = pair(lay, bc, "fp64", par)
    for _ in range(6):
        o.step(1)
        sim.step(1)
        compare(o, sim, 1e-11, early=True)
    o32, s32 = pair(lay, bc, "fp32", par)
    o32.step(1)
    s32.step(1)
    compare(o32, s32, 1e-5, early=True)


def test_extrapolation_inlet_couette_on_the_gpu():
    """FP64 on the CUDA path: a tangential velocity imposed by extrapolation
    on the bottom side against a no-slip wall at the top settles to the
    linear Couette profile through the ghost node, U (ny - 1/2 - y) / (ny +
    1/2); the thermal variant of the same step matches the oracle."""
    nx, ny, U = 64, 16, 0.01
    par = dict(wl.BASE_PARAMS, g=0.0, vin_x=U, vin_y=0.0, nu=0.5)
    one = np.ones((ny, nx))
    sim = pf.Simulation([(nx, ny)], par, "fp64")
    sim.set_boundaries(0, P, P, N, W)
    sim.set_fields(0, one, -one, one)
    sim.step(20000)
    v = sim.fields(0, ("vx",))["vx"]
    y = np.arange(ny)[:, None]
    assert np.abs(v - U * (ny - 0.5 - y) / (ny + 0.5)).max() < 1e-12
    lay = layout()
    part = {**lay.params, **wl.THERMAL_PARAMS, "Le": 2.0, "g": 0.0, "vin_y": 0.0125}
    o, s2 = pair(lay, (S, S, N, O), "fp64", part)
    o.step(20)
    s2.step(20)
    compare(o, s2, 1e-10)


def test_inlet_outlet_thermal_matches_oracle():
    lay = layout()
    par = {**lay.params, **wl.THERMAL_PARAMS, "Le": 2.0, "g": 0.0, "vin_y": 0.0125}
    o, sim = pair(lay, (S, S, I, O), "fp64", par)
    o.step(30)
    sim.step(30)
    compare(o, sim, 1e-10)


def test_forced_convection_upstream_arm_on_the_gpu():
    """Section 3.3 at a larger size on the CUDA path (FP32): a seed on the
    symmetry plane in a melt flowing in from the bottom grows its upstream arm
    longer than its downstream and normal arms."""
    nx, ny, vin = 128, 256, 0.0125
    par = dict(wl.BASE_PARAMS, g=0.0, vin_y=vin)
    cx, cy = -0.5, ny / 2
    o = oracle.Oracle(nx, ny, par)
    o.set_bc(S, S, I, O)
    phi, psi, C = o.fields_from_spec([(cx, cy, 0.0)], 6.0, [])
    sim = pf.Simulation([(nx, ny)], par, "fp32")
    sim.set_boundaries(0, S, S, I, O)
    sim.set_fields(0, phi, psi, C, 0 * phi, vin * (1 - 0.5 * (1 + psi)), 0 * phi)
    sim.step(6000)
    f = sim.fields(0, ("psi",))["psi"]

    def arm(arr, start, step):
        i = start
        while 0 <= i + step < len(arr) and arr[i + step] > 0:
            i += step
        a, b = arr[i], arr[i + step]
        return abs(i - start) + a / (a - b)
    up, down = arm(f[:, 0], int(cy), -1), arm(f[:, 0], int(cy), +1)
    normal = arm(f[int(cy), :], 0, +1)
    assert up > down + 0.5 and up > normal + 0.5, (up, down, normal)
