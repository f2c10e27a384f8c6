"""The flop count per lattice update of the step as the oracle writes it,
from the instrumented-scalar build of the oracle (oracle/counting.h).

The count is exact: every addition, multiplication, division and square
root on the step's values is tallied.  It is the same at every site of a
periodic lattice (the step has no data-dependent branches there), so the
counts of two lattice sizes differ by exactly the per-site count times the
difference in sites, plus nothing; the few operations done once per step
(derived coefficients) cancel in the difference.  The instrumented build
computes the same values as the double build, bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_2407_01651_gb300 import workload as wl


def _per_site(params):
    lay_a = wl.random_layout(48, 40, 2, 1, rng_seed=3, R_max=8)
    lay_b = wl.random_layout(64, 48, 2, 1, rng_seed=3, R_max=8)
    ca = oracle.count_step_ops(dict(lay_a.params, **params), lay_a.nx, lay_a.ny, lay_a.seeds,
                               lay_a.R_s, lay_a.bubbles)
    cb = oracle.count_step_ops(dict(lay_b.params, **params), lay_b.nx, lay_b.ny, lay_b.seeds,
                               lay_b.R_s, lay_b.bubbles)
    dn = lay_b.nx * lay_b.ny - lay_a.nx * lay_a.ny
    per = {}
    for k in ca:
        d = cb[k] - ca[k]
        assert d % dn == 0, (k, d, dn)      # uniform per site
        per[k] = d // dn
        # what is left over is the once-per-step part, the same for both
        assert ca[k] - per[k] * lay_a.nx * lay_a.ny == cb[k] - per[k] * lay_b.nx * lay_b.ny
    return per


@pytest.mark.parametrize("thermal", [False, True])
def test_flops_per_lattice_update(thermal):
    per = _per_site(wl.THERMAL_PARAMS if thermal else {})
    total = sum(per.values())
    print(f"\n{'thermal' if thermal else 'isothermal'} flops per LU: {per}, total {total}")
    # dense D2Q9 and D2Q5 moment transforms dominate: a few thousand per site
    assert 2000 < total < 5000
    assert per["sqrt"] == 4 and per["div"] > 50


def test_counting_build_computes_the_same_values():
    lay = wl.random_layout(48, 40, 2, 1, rng_seed=3, R_max=8)
    for params in ({}, wl.THERMAL_PARAMS):
        par = dict(lay.params, **params)
        a = oracle.Oracle(lay.nx, lay.ny, par)
        b = oracle.Oracle(lay.nx, lay.ny, par, lib=oracle.counting_lib())
        for o in (a, b):
            o.init_spec(lay.seeds, lay.R_s, lay.bubbles)
            o.step(3)
        assert np.array_equal(a.state(), b.state())
        assert all(np.array_equal(a.fields()[k], b.fields()[k]) for k in oracle.FIELDS)
