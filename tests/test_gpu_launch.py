"""Launch machinery of the step: one launch over all domains vs one per
domain, persistent grids, CUDA-graph replay, and the autotuner.  The
arithmetic per site is the same in every mode, so results are bitwise equal
(same traversal) or agree to rounding (different traversal)."""
import numpy as np
import pytest

from paper_2407_01651_gb300 import pf
from paper_2407_01651_gb300 import workload as wl

pytestmark = pytest.mark.gpu

NAMES = ("phi", "psi", "C", "U", "p", "vx", "vy", "mu")


def ensemble(n=5, seed=3):
    lays = []
    for i in range(n):
        nx, ny = [(64, 48), (96, 96), (40, 72), (128, 64), (33, 45)][i % 5]
        lay = wl.random_layout(nx, ny, 1 + i % 2, 1 + i % 3, rng_seed=seed + i, R_min=4,
                               R_max=6)
        lay.params = dict(lay.params, eps_s=0.02 + 0.01 * i)
        lays.append(lay)
    return lays


def make(lays, precision="fp32"):
    sim = pf.Simulation([(l.nx, l.ny, l.params["eps_s"]) for l in lays], wl.BASE_PARAMS,
                        precision)
    for d, l in enumerate(lays):
        sim.init_fields(d, l.seeds, l.R_s, l.bubbles)
    return sim


def fields_all(sim, n):
    return [sim.fields(d) for d in range(n)]


def test_launch_modes_and_graphs_are_bitwise_identical():
    lays = ensemble()
    ref = make(lays)
    ref.step(21)
    fr = fields_all(ref, len(lays))
    for per_domain, persistent, graph in ((1, 0, 0), (0, 1, 0), (0, 0, 8), (1, 1, 4), (0, 1, 2),
                                          (0, 2, 0), (0, 2, 4)):
        sim = make(lays)
        sim.set_launch(per_domain, persistent, graph)
        sim.step(10)
        sim.step(11)      # second call starts from the other buffer parity
        assert sim.steps == 21
        fs = fields_all(sim, len(lays))
        for d in range(len(lays)):
            for k in NAMES:
                assert np.array_equal(fs[d][k], fr[d][k]), (per_domain, persistent, graph, d, k)


def test_changing_the_tiles_drops_captured_graphs():
    """A graph captured before pf_set_step_config or pf_autotune changed the
    tiles is dropped and captured again: the steps after the change give the
    same bits as a handle that never used graphs (every y-march chunk gives
    the same per-site arithmetic)."""
    lays = ensemble(3)
    ref = make(lays)
    ref.step(18)
    fr = fields_all(ref, len(lays))
    ref.step(9)
    fr27 = fields_all(ref, len(lays))
    for persistent in (0, 2):
        sim = make(lays)
        sim.set_launch(0, persistent, 4)
        sim.step(9)
        sim.set_step_config(1, 16)
        sim.step(9)
        fs = fields_all(sim, len(lays))
        for d in range(len(lays)):
            for k in NAMES:
                assert np.array_equal(fs[d][k], fr[d][k]), (persistent, d, k)
        # the autotuner may pick another traversal (same arithmetic, its own
        # rounding order): agreement to FP32 rounding
        sim.autotune(3)
        sim.set_launch(0, persistent, 4)
        sim.step(9)
        fs = fields_all(sim, len(lays))
        for d in range(len(lays)):
            for k in NAMES:
                scale = max(np.abs(fr27[d][k]).max(), 1e-9)
                assert np.abs(fs[d][k] - fr27[d][k]).max() <= 1e-5 * scale, (persistent, d, k)


def test_graph_replay_counts_launches():
    lays = ensemble(3)
    sim = make(lays)
    sim.set_launch(0, 0, 8)
    l0 = sim.launches
    sim.step(17)
    sim.sync()
    assert sim.launches - l0 == 17


def test_autotune_restores_the_state_and_keeps_a_valid_config():
    lays = ensemble()
    a = make(lays)
    cfg = a.autotune(3)
    assert a.steps == 0
    b = make(lays)
    b.set_step_config(cfg[0], cfg[1], cfg[2])
    b.set_launch(0, cfg[3], 0)
    a.step(9)
    b.step(9)
    fa, fb = fields_all(a, len(lays)), fields_all(b, len(lays))
    for d in range(len(lays)):
        for k in NAMES:
            assert np.array_equal(fa[d][k], fb[d][k]), (cfg, d, k)


def test_set_launch_rejects_bad_arguments():
    sim = make(ensemble(2))
    for args in ((2, 0, 0), (0, 3, 0), (1, 2, 0), (0, 0, 3), (0, 0, -2)):
        with pytest.raises(pf.PFError) as e:
            sim.set_launch(*args)
        assert e.value.code == pf.PF_ERR_BAD_ARG


def test_staged_copy_timeout_is_reported_and_recoverable():
    """Failure detection of the staged kernel's bounded waits: with its bulk
    copies dropped (host-side injection) every wait gives up after about a
    second, the kernel drains and returns, and the host reads PF_ERR_TIMEOUT.
    The GPU stays usable: re-initialising clears the condition and the same
    handle then steps to the same state as a fresh one."""
    lay = wl.random_layout(256, 48, 1, 1, rng_seed=7, R_min=4, R_max=6)
    sim = pf.Simulation([(lay.nx, lay.ny)], lay.params, "fp16")
    sim.init_fields(0, lay.seeds, lay.R_s, lay.bubbles)
    assert sim.step_config()[0] == 2
    sim.test_drop_staged_copies(True)
    sim.step(1)
    with pytest.raises(pf.PFError) as e:
        sim.sync()
    assert e.value.code == pf.PF_ERR_TIMEOUT
    sim.test_drop_staged_copies(False)
    sim.init_fields(0, lay.seeds, lay.R_s, lay.bubbles)
    sim.step(3)
    sim.sync()
    ref = pf.Simulation([(lay.nx, lay.ny)], lay.params, "fp16")
    ref.init_fields(0, lay.seeds, lay.R_s, lay.bubbles)
    ref.step(3)
    fa, fb = sim.fields(), ref.fields()
    for k in NAMES:
        assert np.array_equal(fa[k], fb[k]), k


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_one_launch_per_call_is_bitwise_identical_and_counts_one_launch(precision):
    """persistent = 2: every step of a pf_step call in one cooperative launch
    of the resident grid (a grid-wide barrier between steps), also when a
    graph replays such launches; the same bits as one launch per step, and
    one kernel launch per call (per graph replay)."""
    lays = ensemble()
    ref = make(lays, precision)
    ref.step(17)
    fr = fields_all(ref, len(lays))
    sim = make(lays, precision)
    sim.set_launch(0, 2, 0)
    l0 = sim.launches
    sim.step(17)
    assert sim.launches - l0 == 1 and sim.steps == 17
    fs = fields_all(sim, len(lays))
    for d in range(len(lays)):
        for k in NAMES:
            assert np.array_equal(fs[d][k], fr[d][k]), (d, k)
    sim = make(lays, precision)
    sim.set_launch(0, 2, 8)
    l0 = sim.launches
    sim.step(17)          # two replays of an 8-step launch, then one launch of 1 step
    assert sim.launches - l0 == 3 and sim.steps == 17
    fs = fields_all(sim, len(lays))
    for d in range(len(lays)):
        for k in NAMES:
            assert np.array_equal(fs[d][k], fr[d][k]), (d, k)
    with pytest.raises(pf.PFError):
        sim.set_launch(1, 2, 0)          # one launch per domain excludes it
