"""Thermal mode (temperature lattice, finite-Le F(U), grad F source; Section
2.1 and Appendix B) of the CUDA path against the FP64 oracle, through the C ABI.

Tolerances as for the isothermal step: FP64 within 1e-11 relative per field
over a few steps (1e-9 over hundreds), FP32 within 1e-5 per step (mu_phi 5e-5,
early-flow p and v as in test_gpu_parity.py).  The temperature's own scale is
its maximum magnitude (about 0.55).
"""
import numpy as np
import pytest

import oracle
from paper_2407_01651_gb300 import pf
from paper_2407_01651_gb300 import workload as wl

pytestmark = pytest.mark.gpu

FIELDS = ("phi", "psi", "C", "U", "p", "vx", "vy", "mu", "theta")
FLOOR = {"phi": 1e-9, "psi": 1e-9, "C": 1e-9, "U": 1e-9, "p": 1e-12, "vx": 1e-10,
         "vy": 1e-10, "mu": 1e-3, "theta": 1e-9}
EARLY = {"p": 30.0, "vx": 10.0, "vy": 10.0, "mu": 5.0}


def rel(a, b, floor=1e-300):
    return np.abs(a - b).max() / max(np.abs(b).max(), floor)


def thermal(lay, **over):
    return {**lay.params, **wl.THERMAL_PARAMS, **over}


def pair(lay, precision, par):
    o = oracle.Oracle(lay.nx, lay.ny, par)
    o.init_spec(lay.seeds, lay.R_s, lay.bubbles)
    sim = pf.Simulation([(lay.nx, lay.ny)], par, precision)
    sim.init_fields(0, lay.seeds, lay.R_s, lay.bubbles)
    return o, sim


def compare(o, sim, tol, early=False, names=FIELDS):
    fo, fg = o.fields(names), sim.fields(0, names)
    errs = {k: rel(fg[k], fo[k], FLOOR[k]) for k in names}
    fac = EARLY if early else {"mu": 5.0}
    bad = {k: v for k, v in errs.items() if not v <= tol * fac.get(k, 1.0)}
    assert not bad, (bad, errs)
    return errs


def ragged():
    # 150 x 52: two 128-column strips (the second one ragged), partial row tiles
    return wl.random_layout(150, 52, 2, 2, rng_seed=61, R_max=10)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-6)])
def test_thermal_initial_state_matches(precision, tol):
    lay = ragged()
    o, sim = pair(lay, precision, thermal(lay, Le=2.0))
    assert sim.state_planes == pf.STATE_PLANES + 6 == o.state().shape[0]
    compare(o, sim, tol, names=("phi", "psi", "C", "U", "theta"))
    st_o, st_g = o.state(), sim.get_state()
    for p in range(st_o.shape[0]):
        assert rel(st_g[p], st_o[p], 1e-12) <= max(tol, 1e-15), p


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_thermal_steps_match(precision, tol):
    lay = ragged()
    o, sim = pair(lay, precision, thermal(lay, Le=2.0))
    for _ in range(3):
        o.step(1)
        sim.step(1)
        compare(o, sim, tol, early=True)
    st_o, st_g = o.state(), sim.get_state()
    for p in range(39, 45):                  # temperature populations and lagged H
        assert rel(st_g[p], st_o[p], 1e-12) <= tol, p


def test_thermal_fp64_many_steps_and_conservation():
    """Paper's Le = 50 on the 128^2 seed-and-bubble workload: every field within
    1e-9 of the oracle over 300 steps, and the totals of rho H, phi and C
    conserved to 1e-10 in the FP64 reductions."""
    lay = wl.seed_bubble_128()
    o, sim = pair(lay, "fp64", thermal(lay))
    t0, d0 = sim.reduce_thermal(0), sim.reduce(0)
    ot0 = o.thermal_totals()
    assert abs(t0["sum_e"] / ot0["sum_e"] - 1) < 1e-13
    for _ in range(3):
        o.step(100)
        sim.step(100)
        compare(o, sim, 1e-9)
        t, d = sim.reduce_thermal(0), sim.reduce(0)
        assert abs(t["sum_e"] / t0["sum_e"] - 1) <= 1e-10
        assert abs(d["sum_phi"] / d0["sum_phi"] - 1) <= 1e-10
        assert abs(d["sum_C"] / d0["sum_C"] - 1) <= 1e-10
        ot = o.thermal_totals()
        assert abs(t["sum_theta"] / ot["sum_theta"] - 1) <= 1e-10


def test_thermal_fp32_error_and_enthalpy_drift():
    """FP32: per-step error 1e-5 at the first step, bounded over 200 steps, and
    the FP64 total of rho H drifts by less than 1e-6 relative."""
    lay = wl.seed_bubble_128()
    o, sim = pair(lay, "fp32", thermal(lay))
    t0 = sim.reduce_thermal(0)
    o.step(1)
    sim.step(1)
    compare(o, sim, 1e-5, early=True)
    o.step(199)
    sim.step(199)
    compare(o, sim, 1e-3)
    t = sim.reduce_thermal(0)
    assert abs(t["sum_e"] / t0["sum_e"] - 1) <= 1e-6


def test_set_temperature_matches_oracle():
    """A non-uniform initial temperature (pf_set_temperature) with a seed in a
    gas-free melt: same fields as the oracle initialised with that theta."""
    N = 64
    lay = wl.Layout(N, N, seeds=[(N / 2, N / 2, 0.3)], bubbles=[])
    par = thermal(lay, Le=1.0, g=0.0)
    y, x = np.mgrid[0:N, 0:N].astype(float)
    th = -0.55 + 0.05 * np.sin(2 * np.pi * x / N) * np.cos(4 * np.pi * y / N)
    o = oracle.Oracle(N, N, par)
    phi, psi, C = o.fields_from_spec(lay.seeds, lay.R_s, [])
    o.set_orientation(lay.seeds)
    o.init_fields(phi, psi, C, theta=th)
    sim = pf.Simulation([(N, N)], par, "fp64")
    sim.init_fields(0, lay.seeds, lay.R_s, [])
    s0 = sim.get_state(0)
    bad = th.copy()
    bad[5, 9] = np.nan
    with pytest.raises(pf.PFError) as e:
        sim.set_temperature(0, bad)         # found on the device, state untouched
    assert e.value.code == pf.PF_ERR_BAD_ARG and "non-finite" in str(e.value)
    assert np.array_equal(sim.get_state(0), s0)
    sim.set_temperature(0, th)
    compare(o, sim, 1e-12, names=("theta", "psi"))
    o.step(20)
    sim.step(20)
    compare(o, sim, 1e-11)
    with pytest.raises(pf.PFError) as e:
        sim.set_temperature(0, th)          # only before the first step
    assert e.value.code == pf.PF_ERR_STATE


def test_thermal_configuration_errors():
    lay = ragged()
    sim = pf.Simulation([(lay.nx, lay.ny)], thermal(lay), "fp32")
    sim.init_fields(0, lay.seeds, lay.R_s, lay.bubbles)
    for variant in (0, 2):
        with pytest.raises(pf.PFError) as e:
            sim.set_step_config(variant, 32, 8)
        assert e.value.code == pf.PF_ERR_BAD_ARG
    with pytest.raises(pf.PFError) as e:
        sim.adjoint_step(4, 1.0, 0.0, 2)
    assert e.value.code == pf.PF_ERR_BAD_ARG
    iso = pf.Simulation([(16, 16)], wl.BASE_PARAMS, "fp32")
    with pytest.raises(pf.PFError):
        iso.reduce_thermal(0)
    assert iso.state_planes == pf.STATE_PLANES


def test_thermal_ensemble_graphs_and_persistent_are_bitwise_equal():
    """Launch modes of a thermal ensemble: one launch, per-domain launches,
    persistent grid and graph replay all give the same bits."""
    lays = [wl.random_layout(96, 64, 1, 1, rng_seed=71, R_max=8),
            wl.random_layout(130, 40, 2, 1, rng_seed=72, R_max=6)]
    par = dict(wl.BASE_PARAMS, **wl.THERMAL_PARAMS)
    out = []
    for mode in ((0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 1, 4)):
        sim = pf.Simulation([(l.nx, l.ny) for l in lays], par, "fp32")
        for d, l in enumerate(lays):
            sim.init_fields(d, l.seeds, l.R_s, l.bubbles)
        sim.set_launch(*mode)
        sim.step(9)
        out.append([sim.fields(d) for d in range(len(lays))])
    for other in out[1:]:
        for d in range(len(lays)):
            for k in FIELDS:
                assert np.array_equal(other[d][k], out[0][d][k]), (d, k)


def test_thermal_full_size_4096_windows():
    """The thermal 4096^2 workload (64 seeds, 128 bubbles, Le = 50) in the
    launch configuration the benchmark times: after 2 steps, windows around
    seeds, bubbles and the wrap match oracle windows in global coordinates."""
    lay = wl.growth_lattice(4096, 4096)
    par = thermal(lay)
    sim = pf.Simulation([(lay.nx, lay.ny)], par, "fp32")
    sim.init_fields(0, lay.seeds, lay.R_s, lay.bubbles)
    T = 2
    sim.step(T)
    names = ("phi", "psi", "C", "vx", "vy", "p", "theta")
    fg = sim.fields(0, names)
    sim.close()
    nx, ny = lay.nx, lay.ny
    W, M = 24, 2 * T
    probe = oracle.Oracle(4, 4, par, window=(nx, ny, 0, 0))
    rho_bar = par["rho_g"] + probe.mean_phi_global(lay.bubbles) * (par["rho_l"] - par["rho_g"])
    centers = [(int(s[0]) + 5, int(s[1])) for s in lay.seeds[:3]]
    centers += [(int(b[0] + b[2]), int(b[1])) for b in lay.bubbles[:3]]
    centers += [(nx - 3, ny - 3)]
    ref, got = {k: [] for k in names}, {k: [] for k in names}
    for cx, cy in centers:
        x0, y0 = cx - W // 2, cy - W // 2
        o = oracle.Oracle(W, W, par, window=(nx, ny, x0, y0))
        o.set_rho_bar(rho_bar)
        o.init_spec(lay.seeds, lay.R_s, lay.bubbles)
        o.step(T)
        fo = o.fields(names)
        ys = (np.arange(M, W - M) + y0) % ny
        xs = (np.arange(M, W - M) + x0) % nx
        for k in names:
            ref[k].append(fo[k][M:W - M, M:W - M])
            got[k].append(fg[k][np.ix_(ys, xs)])
    for k in names:
        err = rel(np.concatenate(got[k]), np.concatenate(ref[k]), FLOOR[k])
        assert err <= 1e-5 * EARLY.get(k, 1.0), (k, err)
