"""pf_run: fields in, n steps, fields out in one call, with the host copies
overlapped with the steps in row bands.  It must give bit for bit what
pf_set_fields, pf_step and pf_get_fields give one after the other."""
import numpy as np
import pytest

from paper_2407_01651_gb300 import pf
from paper_2407_01651_gb300 import workload as wl

pytestmark = pytest.mark.gpu

NAMES6 = ("phi", "psi", "C", "vx", "vy", "p")


def developed_fields(lay, precision, steps=30):
    """Six input planes of a state with flow, from a few steps of the GPU path."""
    sim = pf.Simulation([(lay.nx, lay.ny)], lay.params, precision)
    sim.init_fields(0, lay.seeds, lay.R_s, lay.bubbles)
    sim.step(steps)
    f = sim.fields(0, NAMES6)
    sim.close()
    return np.ascontiguousarray(np.stack([f[n] for n in NAMES6]))


def one_after_the_other(lay, precision, cfg, f6, n):
    sim = pf.Simulation([(lay.nx, lay.ny)], lay.params, precision)
    sim.set_step_config(*cfg)
    sim.set_fields_stack(0, f6)
    sim.step(n)
    out = sim.fields(0, pf.FIELDS)
    state = sim.get_state(0)
    sim.close()
    return out, state


def banded(lay, precision, cfg, f6, n, out=None):
    sim = pf.Simulation([(lay.nx, lay.ny)], lay.params, precision)
    sim.set_step_config(*cfg)
    res = sim.run(f6, n, pf.FIELDS, out=out)
    state = sim.get_state(0)
    steps = sim.steps
    sim.close()
    return res, state, steps


@pytest.mark.parametrize("precision,cfg,n", [
    ("fp32", (1, 8, 0), 7),      # 48 tile rows: 8 bands
    ("fp32", (1, 32, 0), 4),     # 12 tile rows: 3 bands
    ("fp64", (1, 16, 0), 5),
    ("fp16", (2, 16, 0), 6),     # staged traversal
    ("bf16", (2, 24, 0), 3),
    ("fp32", (0, 32, 8), 5),     # 2-D tiles
])
def test_run_equals_set_step_get(precision, cfg, n):
    lay = wl.random_layout(256, 384, 3, 4, rng_seed=5, R_max=20)
    f6 = developed_fields(lay, precision)
    ref, ref_state = one_after_the_other(lay, precision, cfg, f6, n)
    got, got_state, steps = banded(lay, precision, cfg, f6, n)
    assert steps == n
    for nm in pf.FIELDS:
        assert np.array_equal(got[nm], ref[nm]), nm
    assert np.array_equal(got_state, ref_state)


def test_run_with_page_locked_buffers():
    torch = pytest.importorskip("torch")
    lay = wl.random_layout(192, 256, 2, 3, rng_seed=6, R_max=16)
    f6 = developed_fields(lay, "fp32")
    pin_in = torch.empty(f6.shape, dtype=torch.float64, pin_memory=True).numpy()
    pin_in[...] = f6
    pin_out = torch.empty(len(pf.FIELDS) * f6[0].size, dtype=torch.float64,
                          pin_memory=True).numpy()
    ref, _ = one_after_the_other(lay, "fp32", (1, 8, 0), f6, 9)
    got, _, _ = banded(lay, "fp32", (1, 8, 0), pin_in, 9, out=pin_out)
    for nm in pf.FIELDS:
        assert np.array_equal(got[nm], ref[nm]), nm


def test_run_small_lattice_and_zero_steps_run_the_calls_in_turn():
    lay = wl.random_layout(64, 40, 1, 1, rng_seed=7, R_max=8)
    f6 = developed_fields(lay, "fp32", 5)
    for n in (0, 3):
        ref, ref_state = one_after_the_other(lay, "fp32", (1, 32, 0), f6, n)
        got, got_state, _ = banded(lay, "fp32", (1, 32, 0), f6, n)
        for nm in pf.FIELDS:
            assert np.array_equal(got[nm], ref[nm]), (n, nm)
        assert np.array_equal(got_state, ref_state)


def test_run_rejects_non_finite_input_and_bad_arguments():
    lay = wl.random_layout(128, 256, 1, 2, rng_seed=8, R_max=12)
    f6 = developed_fields(lay, "fp32", 5)
    bad = f6.copy()
    bad[4, 200, 17] = np.nan
    sim = pf.Simulation([(lay.nx, lay.ny)], lay.params, "fp32")
    sim.set_step_config(1, 8, 0)
    with pytest.raises(pf.PFError, match="non-finite"):
        sim.run(bad, 4)
    with pytest.raises(pf.PFError):
        sim.step(1)          # the domain counts as not initialised
    sim.run(f6, 2)           # and a good call sets it again
    with pytest.raises(ValueError):
        sim.run(f6[:, :-1].copy(), 2)
    sim.close()
    two = pf.Simulation([(64, 64), (64, 64)], lay.params, "fp32")
    with pytest.raises(ValueError):
        two.run(np.zeros((6, 64, 64)), 1)
    two.close()


def test_run_beside_graphs_and_the_one_launch_mode():
    """pf_run ignores the launch mode (one launch per band and step) and may
    leave the state in the other buffer; steps taken after it under the
    one-launch mode with captured graphs give what plain steps give."""
    lay = wl.random_layout(256, 384, 3, 4, rng_seed=9, R_max=20)
    f6 = developed_fields(lay, "fp32")
    states = []
    for mode in ((0, 0, 0), (0, 2, 4)):
        sim = pf.Simulation([(lay.nx, lay.ny)], lay.params, "fp32")
        sim.set_step_config(1, 8, 0)
        sim.set_launch(*mode)
        sim.init_fields(0, lay.seeds, lay.R_s, lay.bubbles)
        sim.step(4)                  # graphs captured before the call (mode 2)
        sim.run(f6, 5)               # odd: the state ends in the other buffer
        sim.step(9)
        states.append(sim.get_state(0))
        sim.close()
    assert np.array_equal(states[0], states[1])


@pytest.mark.parametrize("shape,cfg", [((200, 385), (1, 32, 0)), ((136, 300), (2, 16, 0))])
def test_run_ragged_lattices(shape, cfg):
    """Lattices whose last tile row is ragged (385 = 12 x 32 + 1 rows) and whose
    width is not a multiple of the strip: pf_run still equals the three calls."""
    nx, ny = shape
    lay = wl.random_layout(nx, ny, 2, 3, rng_seed=10, R_max=14)
    prec = "fp16" if cfg[0] == 2 else "fp32"
    f6 = developed_fields(lay, prec, 10)
    ref, ref_state = one_after_the_other(lay, prec, cfg, f6, 7)
    got, got_state, _ = banded(lay, prec, cfg, f6, 7)
    for nm in pf.FIELDS:
        assert np.array_equal(got[nm], ref[nm]), nm
    assert np.array_equal(got_state, ref_state)
