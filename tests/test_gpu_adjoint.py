"""Discrete adjoint (pf_adjoint_step) against the oracle's complex-step
derivative of the same discrete map, against central differences, and its
bookkeeping (checkpoint interval, final state, argument errors, autograd)."""
import math

import numpy as np
import pytest

import oracle
from paper_2407_01651_gb300 import pf
from paper_2407_01651_gb300 import workload as wl

pytestmark = pytest.mark.gpu

NAMES = ("eps_s", "Omega", "sigma")


def oracle_gradient(lay, par, T, w_s=1.0, w_c=1.0):
    out = []
    J = None
    for name in NAMES:
        o = oracle.Oracle(lay.nx, lay.ny, par, complex_step=True)
        o.perturb(name, 1e-30)
        o.init_spec(lay.seeds, lay.R_s, lay.bubbles)
        o.step(T)
        re, im = o.objective()
        J = re
        out.append(im / 1e-30)
    return J, np.array(out)


@pytest.mark.parametrize("shape,T,K", [((48, 40), 30, 7), ((64, 64), 50, 10)])
def test_fp64_adjoint_equals_oracle_complex_step(shape, T, K):
    """Both are exact derivatives of the same discrete trajectory (the oracle by
    the complex-step method), so they agree to rounding."""
    nx, ny = shape
    lay = wl.random_layout(nx, ny, 1, 1, rng_seed=11, R_max=8)
    par = dict(lay.params, g=1e-5)
    sim = pf.Simulation([(nx, ny)], par, "fp64")
    sim.init_fields(0, lay.seeds, lay.R_s, lay.bubbles)
    J, g = sim.adjoint_step(T, 1.0, 1.0, K)
    Jo, go = oracle_gradient(lay, par, T)
    assert math.isclose(J, Jo, rel_tol=1e-12)
    assert np.allclose(g, go, rtol=1e-10, atol=0), (g, go)


def test_adjoint_does_not_depend_on_the_checkpoint_interval():
    lay = wl.random_layout(48, 40, 1, 1, rng_seed=12, R_max=8)
    res = []
    for K in (1, 7, 30):
        sim = pf.Simulation([(lay.nx, lay.ny)], lay.params, "fp64")
        sim.init_fields(0, lay.seeds, lay.R_s, lay.bubbles)
        res.append(sim.adjoint_step(30, 1.0, 1.0, K))
    for J, g in res[1:]:
        assert J == res[0][0]
        assert np.array_equal(g, res[0][1])


def test_fp32_adjoint_against_central_differences():
    """FP32 adjoint vs FP64 central differences (h = 1e-4 relative, the step the
    benchmark recipe names) on a 128^2 layout over 200 steps."""
    lay = wl.random_layout(128, 128, 2, 2, rng_seed=4, R_max=16)
    T = 200
    sim = pf.Simulation([(128, 128)], lay.params, "fp32")
    sim.init_fields(0, lay.seeds, lay.R_s, lay.bubbles)
    _, g32 = sim.adjoint_step(T, 1.0, 1.0, 50)
    fd = []
    for name in NAMES:
        h = 1e-4 * lay.params[name]
        Js = []
        for sgn in (1, -1):
            s = pf.Simulation([(128, 128)], dict(lay.params, **{name: lay.params[name] + sgn * h}),
                              "fp64")
            s.init_fields(0, lay.seeds, lay.R_s, lay.bubbles)
            Js.append(s.adjoint_step(T, 1.0, 1.0, T)[0])
        fd.append((Js[0] - Js[1]) / (2 * h))
    assert np.allclose(g32, fd, rtol=5e-4), (g32, fd)


def test_adjoint_leaves_the_final_state():
    lay = wl.random_layout(64, 48, 2, 1, rng_seed=13, R_max=8)
    a = pf.Simulation([(lay.nx, lay.ny)], lay.params, "fp32")
    b = pf.Simulation([(lay.nx, lay.ny)], lay.params, "fp32")
    for s in (a, b):
        s.init_fields(0, lay.seeds, lay.R_s, lay.bubbles)
    a.adjoint_step(25, 1.0, 0.5, 10)
    b.step(25)
    fa, fb = a.fields(), b.fields()
    for k in ("phi", "psi", "C", "p", "vx", "vy"):
        assert np.array_equal(fa[k], fb[k]), k
    assert a.steps == b.steps == 25


def test_adjoint_argument_errors():
    lay = wl.random_layout(32, 32, 1, 1, rng_seed=14, R_max=6)
    multi = pf.Simulation([(32, 32), (32, 32)], lay.params, "fp32")
    for d in (0, 1):
        multi.init_fields(d, lay.seeds, lay.R_s, lay.bubbles)
    with pytest.raises(pf.PFError) as e:
        multi.adjoint_step(5)
    assert e.value.code == pf.PF_ERR_BAD_ARG
    half = pf.Simulation([(32, 32)], lay.params, "fp16")
    half.init_fields(0, lay.seeds, lay.R_s, lay.bubbles)
    with pytest.raises(pf.PFError):
        half.adjoint_step(5)
    one = pf.Simulation([(32, 32)], lay.params, "fp32")
    with pytest.raises(pf.PFError) as e:
        one.adjoint_step(5)
    assert e.value.code == pf.PF_ERR_STATE
    one.init_fields(0, lay.seeds, lay.R_s, lay.bubbles)
    with pytest.raises(pf.PFError):
        one.adjoint_step(5, checkpoint_every=0)


def test_autograd_function_returns_the_adjoint_gradient():
    import torch
    from paper_2407_01651_gb300.autograd import final_state_objective

    lay = wl.random_layout(48, 40, 1, 1, rng_seed=11, R_max=8)
    lay.params = dict(lay.params, g=1e-5)
    theta = torch.tensor([lay.params[n] for n in NAMES], dtype=torch.float64, requires_grad=True)
    J = final_state_objective(theta, lay, 30, checkpoint_every=7, precision="fp64")
    (g,) = torch.autograd.grad(2.0 * J, theta)
    Jo, go = oracle_gradient(lay, lay.params, 30)
    assert math.isclose(J.item(), Jo, rel_tol=1e-12)
    assert np.allclose(g.numpy(), 2.0 * go, rtol=1e-10)
