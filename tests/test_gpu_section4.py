"""The paper's Section-4 problem on the CUDA path: a 200 x 400 domain with
symmetric sides in x, a no-flux wall at the bottom and the far field (psi_l,
C = 1, theta = -Omega) at the top, the temperature lattice on (Le = 50), a gas
bubble of diameter 40 centred on the symmetry plane at y = Ly/5 and two seeds
of radius 10 at the bottom corners.  The first steps match the FP64 oracle;
over 6000 FP32 steps the bubble rises, the seeds grow and the gas is
conserved."""
import numpy as np
import pytest

import oracle
from paper_2407_01651_gb300 import pf
from paper_2407_01651_gb300 import workload as wl

pytestmark = pytest.mark.gpu

NX, NY = 200, 400
SIDES = (pf.BC_SYMMETRIC, pf.BC_SYMMETRIC, pf.BC_WALL, pf.BC_FARFIELD)
SEEDS = [(-0.5, -0.5, 0.0), (NX - 0.5, -0.5, 0.0)]
BUBBLE = [(-0.5, NY / 5, 20.0)]
PAR = dict(wl.BASE_PARAMS, **wl.THERMAL_PARAMS, g=1e-5)
FIELDS = ("phi", "psi", "C", "U", "p", "vx", "vy", "theta")
FLOOR = {"phi": 1e-9, "psi": 1e-9, "C": 1e-9, "U": 1e-9, "p": 1e-12, "vx": 1e-10,
         "vy": 1e-10, "theta": 1e-9}


def sim_of(precision):
    sim = pf.Simulation([(NX, NY)], PAR, precision)
    sim.set_boundaries(0, *SIDES)
    sim.init_fields(0, SEEDS, 10.0, BUBBLE)
    return sim


def test_section4_first_steps_match_oracle():
    o = oracle.Oracle(NX, NY, PAR)
    o.set_bc(*SIDES)
    o.init_spec(SEEDS, 10.0, BUBBLE)
    sim = sim_of("fp64")
    o.step(20)
    sim.step(20)
    fo, fg = o.fields(FIELDS), sim.fields(0, FIELDS)
    for k in FIELDS:
        err = np.abs(fg[k] - fo[k]).max() / max(np.abs(fo[k]).max(), FLOOR[k])
        assert err <= 1e-10, (k, err)


def test_section4_bubble_rises_and_seeds_grow():
    sim = sim_of("fp32")
    d0 = sim.reduce(0)
    yc0 = d0["gas_y"] / d0["gas"]
    sim.step(6000)
    d = sim.reduce(0)
    assert d["nonfinite"] == 0
    assert d["gas_y"] / d["gas"] > yc0 + 5.0             # the bubble rose
    assert d["sum_hpsi"] > 2.0 * d0["sum_hpsi"]          # the seeds grew
    assert abs(d["sum_phi"] / d0["sum_phi"] - 1) < 1e-5  # no gas is lost or gained
    theta = sim.fields(0, ("theta",))["theta"]
    assert theta.max() > -0.55 + 1e-3                     # latent heat at the fronts
    assert np.abs(theta[-1, :] + 0.55).max() < 0.05      # near the far-field value on top
