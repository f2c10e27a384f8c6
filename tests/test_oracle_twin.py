"""The oracle against a literal per-node twin (tests/twin_step.py) on tiny
lattices: the same discrete step written twice, in different forms, must
agree to rounding.

The twin shares no code with the oracle: it relaxes each lattice in
population space with the dense matrix Lambda = M^-1 S M of Appendix B (M^-1
by numerical inversion, M generated from the moment polynomials), evaluates
every term one site at a time in Python, and composes the two passes of the
step (streaming with the time stretch, then stencils, sources and
collisions) from the paper's equations directly.  So a slip in how the oracle
orders the passes, which lagged value feeds which term, or how it builds its
moment matrices shows up here, on inputs no symmetry protects: random fields,
a flow, a pressure field and two rotated grains.
"""
import math

import numpy as np
import pytest

import oracle
import twin_step
from paper_2407_01651_gb300 import workload as wl

STEPS = 3
TOL = 3e-14         # per plane, relative to the plane's maximum (measured <= 1.1e-14)


def _inputs(nx, ny, seed):
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    W = 4.0
    rb = np.hypot(x - 0.37 * nx, y - 0.61 * ny)
    phi = 0.5 + 0.5 * np.tanh((rb - 0.3 * min(nx, ny)) / (2 * math.sqrt(2) * W))
    phi = np.clip(phi + 0.02 * rng.standard_normal(phi.shape), 0.01, 0.99)
    rs = np.hypot(x - 0.7 * nx, y - 0.3 * ny)
    psi = np.tanh((0.25 * min(nx, ny) - rs) / (math.sqrt(2) * W))
    psi = np.clip(psi + 0.05 * rng.standard_normal(psi.shape), -0.99, 0.99)
    C = phi * (1 - 0.85 * 0.5 * (1 + psi)) * (1 + 0.05 * rng.standard_normal(phi.shape))
    vx = 2e-3 * rng.standard_normal(phi.shape)
    vy = 2e-3 * rng.standard_normal(phi.shape)
    p = 1e-4 * rng.standard_normal(phi.shape)
    theta = -0.55 + 0.05 * rng.standard_normal(phi.shape)
    # two grains, each site taking the angle of the nearer seed (minimum
    # image; the positions leave no exact ties)
    seeds = [(0.21 * nx, 0.33 * ny, 0.4), (0.73 * nx, 0.81 * ny, 1.1)]
    angle = np.zeros_like(phi)
    best = np.full_like(phi, np.inf)
    for sx, sy, a in seeds:
        dx = (x - sx + nx / 2) % nx - nx / 2
        dy = (y - sy + ny / 2) % ny - ny / 2
        d2 = dx * dx + dy * dy
        angle = np.where(d2 < best, a, angle)
        best = np.minimum(best, d2)
    return dict(phi=phi, psi=psi, C=C, vx=vx, vy=vy, p=p, theta=theta, angle=angle,
                seeds=seeds)


@pytest.mark.parametrize("nx,ny", [(8, 8), (12, 10)])
@pytest.mark.parametrize("thermal", [False, True])
def test_oracle_equals_the_per_node_twin(nx, ny, thermal):
    par = dict(wl.BASE_PARAMS, sigma=1e-2, g=1e-3, eps_s=0.05)
    if thermal:
        par.update(wl.THERMAL_PARAMS, cp=10.0)
    inp = _inputs(nx, ny, seed=nx * 100 + ny + (7 if thermal else 0))
    o = oracle.Oracle(nx, ny, par)
    o.set_orientation(inp["seeds"])
    o.init_fields(inp["phi"], inp["psi"], inp["C"], inp["vx"], inp["vy"], inp["p"],
                  inp["theta"] if thermal else None)
    t = twin_step.Twin(nx, ny, par)
    t.init(inp["phi"], inp["psi"], inp["C"], inp["vx"], inp["vy"], inp["p"], inp["angle"],
           inp["theta"] if thermal else None)
    s0 = o.state()
    assert np.abs(s0 - t.state()).max() <= 1e-15 * np.abs(s0).max()
    for _ in range(STEPS):
        o.step(1)
        t.step()
        so, st = o.state(), t.state()
        assert so.shape == st.shape
        for q in range(so.shape[0]):
            scale = max(np.abs(so[q]).max(), 1e-12)
            err = np.abs(so[q] - st[q]).max() / scale
            assert err <= TOL, (q, err)
        fo = o.fields()
        for nm in oracle.FIELDS:
            if nm == "theta" and not thermal:
                continue
            scale = max(np.abs(fo[nm]).max(), 1e-12)
            err = np.abs(fo[nm] - t.fields[nm]).max() / scale
            assert err <= TOL, (nm, err)
    # the flow, the pressure and both grains took part
    assert np.abs(fo["vx"]).max() > 1e-4 and np.abs(fo["p"]).max() > 1e-6
    assert len(np.unique(inp["angle"])) == 2


def twin_error(lib=None, nx=8, ny=8, thermal=False):
    """Largest per-plane relative difference of the state over 3 steps
    between an oracle library (its own build, or a copy with a planted
    mistake) and the twin."""
    par = dict(wl.BASE_PARAMS, sigma=1e-2, g=1e-3, eps_s=0.05)
    if thermal:
        par.update(wl.THERMAL_PARAMS, cp=10.0)
    inp = _inputs(nx, ny, seed=nx * 100 + ny + (7 if thermal else 0))
    o = oracle.Oracle(nx, ny, par, lib=lib)
    o.set_orientation(inp["seeds"])
    o.init_fields(inp["phi"], inp["psi"], inp["C"], inp["vx"], inp["vy"], inp["p"],
                  inp["theta"] if thermal else None)
    t = twin_step.Twin(nx, ny, par)
    t.init(inp["phi"], inp["psi"], inp["C"], inp["vx"], inp["vy"], inp["p"], inp["angle"],
           inp["theta"] if thermal else None)
    worst = 0.0
    for _ in range(STEPS):
        o.step(1)
        t.step()
        so, st = o.state(), t.state()
        for q in range(so.shape[0]):
            worst = max(worst, float(np.abs(so[q] - st[q]).max() / max(np.abs(so[q]).max(), 1e-12)))
    return worst
