"""The 3-D dendrite step (psi and C on D3Q7, reading R33) of the CUDA path
against the FP64 3-D oracle, through the C ABI.  Tolerances as for the 2-D
step: FP64 within 1e-11 relative per field over a few steps (1e-9 over
hundreds), FP32 within 1e-5 per step."""
import numpy as np
import pytest

import oracle
from paper_2407_01651_gb300 import pf
from paper_2407_01651_gb300 import workload as wl

pytestmark = pytest.mark.gpu

P3 = {k: wl.BASE_PARAMS[k] for k in oracle.PARAM_NAMES_3D}
# Without gas, U starts at exactly 0 (C = 1 - (1-k) h(psi)) and grows slowly
# from solute rejection: its scale is that of the supersaturation the
# undercooling sets, O(Omega) = O(0.1), not its tiny early maximum (FP32
# computes 2C/A - 1 from C rounded to ~6e-8).
FLOOR = {"psi": 1e-9, "C": 1e-9, "U": 0.1}


def rel(a, b, floor):
    return np.abs(a - b).max() / max(np.abs(b).max(), floor)


def pair(shape, seeds, R_s, precision, params=P3):
    nx, ny, nz = shape
    o = oracle.Oracle3D(nx, ny, nz, params)
    o.init_spec(seeds, R_s)
    sim = pf.Simulation3D(shape, dict(wl.BASE_PARAMS, **params), precision)
    sim.init_seeds(seeds, R_s)
    return o, sim


def compare(o, sim, tol):
    fo, fg = o.fields(), sim.fields()
    errs = {k: rel(fg[k], fo[k], FLOOR[k]) for k in fg}      # the oracle adds theta
    assert all(v <= tol for v in errs.values()), errs
    return errs


RAGGED = (40, 19, 13)          # two column tiles in x (one ragged), three in y, chunks in z
SEEDS = [(10.3, 9.1, 6.2), (33.0, 4.0, 11.5)]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_3d_initial_state(precision, tol):
    o, sim = pair(RAGGED, SEEDS, 5.0, precision)
    compare(o, sim, tol)
    so, sg = o.state(), sim.get_state()
    for p in range(pf.PF3_STATE_PLANES):
        assert rel(sg[p], so[p], 1e-12) <= max(tol, 1e-15), p


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_3d_steps_match_oracle(precision, tol):
    o, sim = pair(RAGGED, SEEDS, 5.0, precision)
    sim.set_chunk(5)
    for _ in range(3):
        o.step(1)
        sim.step(1)
        compare(o, sim, tol)
    so, sg = o.state(), sim.get_state()
    for p in range(pf.PF3_STATE_PLANES):
        assert rel(sg[p], so[p], 1e-12) <= tol * 10, p


def test_3d_fp64_many_steps_symmetry_and_conservation():
    """A centred seed over 150 steps: within 1e-9 of the oracle, with the
    symmetry of the cube and sum C conserved to 1e-12 in FP64."""
    n = 28
    o, sim = pair((n, n, n), [(n / 2, n / 2, n / 2)], 8.0, "fp64")
    c0 = sim.reduce()["sum_C"]
    o.step(150)
    sim.step(150)
    compare(o, sim, 1e-9)
    psi = sim.fields()["psi"]
    for t in (psi.transpose(0, 2, 1), psi.transpose(2, 1, 0),
              np.roll(np.flip(psi, axis=2), 1, axis=2)):
        assert np.abs(psi - t).max() < 1e-12
    assert abs(sim.reduce()["sum_C"] / c0 - 1) <= 1e-12


def test_3d_fp32_drift_and_bounded_error():
    n = 32
    o, sim = pair((n, n, n), [(10.0, 12.0, 16.0), (24.0, 20.0, 8.0)], 7.0, "fp32")
    c0 = sim.reduce()["sum_C"]
    o.step(200)
    sim.step(200)
    compare(o, sim, 1e-3)
    assert abs(sim.reduce()["sum_C"] / c0 - 1) <= 1e-6


def test_3d_full_size_windows():
    """The 256^3 workload (64 seeds) in the benchmark's launch configuration:
    after 2 steps, 24^3 windows around seeds and across the periodic corner
    match oracle windows placed in global coordinates."""
    n = 256
    seeds, R_s = wl.growth_3d(n)
    sim = pf.Simulation3D((n, n, n), wl.BASE_PARAMS, "fp32")
    sim.init_seeds(seeds, R_s)
    T = 2
    sim.step(T)
    fg = sim.fields()
    sim.close()
    W, M = 24, 2 * T
    centres = [(int(s[0]) + 7, int(s[1]), int(s[2])) for s in seeds[:3]] + [(n - 2, n - 2, n - 2)]
    ref, got = {k: [] for k in fg}, {k: [] for k in fg}
    for cx, cy, cz in centres:
        x0, y0, z0 = cx - W // 2, cy - W // 2, cz - W // 2
        o = oracle.Oracle3D(W, W, W, P3, window=(n, n, n, x0, y0, z0))
        o.init_spec(seeds, R_s)
        o.step(T)
        fo = o.fields()
        idx = [(np.arange(M, W - M) + c0) % n for c0 in (z0, y0, x0)]
        for k in fg:
            ref[k].append(fo[k][M:W - M, M:W - M, M:W - M].ravel())
            got[k].append(fg[k][np.ix_(*idx)].ravel())
    for k in fg:
        err = rel(np.concatenate(got[k]), np.concatenate(ref[k]), FLOOR[k])
        assert err <= 1e-5, (k, err)


def test_3d_configuration_errors():
    with pytest.raises(pf.PFError):
        pf.Simulation3D((3, 8, 8), wl.BASE_PARAMS, "fp32")
    with pytest.raises(pf.PFError):
        pf.Simulation3D((8, 8, 8), wl.BASE_PARAMS, "fp16")
    sim = pf.Simulation3D((8, 8, 8), wl.BASE_PARAMS, "fp32")
    with pytest.raises(pf.PFError) as e:
        sim.step(1)                        # not initialised
    assert e.value.code == pf.PF_ERR_STATE
    # non-finite input is rejected on the device and leaves the state as it was
    psi = np.full((8, 8, 8), -1.0)
    C = np.ones((8, 8, 8))
    sim.set_fields(psi, C)
    s0 = sim.get_state()
    for bad in (np.nan, np.inf):
        C2 = C.copy()
        C2[3, 5, 7] = bad
        with pytest.raises(pf.PFError) as e:
            sim.set_fields(psi, C2)
        assert e.value.code == pf.PF_ERR_BAD_ARG and "non-finite" in str(e.value)
    assert np.array_equal(sim.get_state(), s0)


# ---------------------------------------------------------------------------
# thermal mode: D3Q7 temperature lattice, F(U) and the grad F source
# ---------------------------------------------------------------------------
T3 = dict(P3, thermal=1, Le=2.0, latent=1.0, theta0=-0.55, cp=10.0, rho_l=1.0)
FLOOR_T = dict(FLOOR, theta=1e-9)


def compare_t(o, sim, tol):
    fo, fg = o.fields(), sim.fields()
    assert set(fg) == set(fo) == {"psi", "C", "U", "theta"}
    errs = {k: rel(fg[k], fo[k], FLOOR_T[k]) for k in fo}
    assert all(v <= tol for v in errs.values()), errs
    return errs


def theta_field(shape):
    """A smooth non-uniform temperature: a gradient along x and a bump."""
    nx, ny, nz = shape
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx].astype(float)
    return -0.55 + 0.05 * np.sin(2 * np.pi * x / nx) + \
        0.08 * np.exp(-((x - nx / 3) ** 2 + (y - ny / 2) ** 2 + (z - nz / 2) ** 2) / 20.0)


def pair_t(shape, seeds, R_s, precision, theta=None, params=T3):
    o, sim = pair(shape, seeds, R_s, precision, params)
    if theta is not None:
        o.init_fields(o.fields()["psi"], o.fields()["C"], theta)
        sim.set_temperature(theta)
    return o, sim


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_3d_thermal_initial_state(precision, tol):
    o, sim = pair_t(RAGGED, SEEDS, 5.0, precision, theta_field(RAGGED))
    compare_t(o, sim, tol)
    so, sg = o.state(), sim.get_state()
    assert sg.shape[0] == pf.PF3_STATE_PLANES_THERMAL == so.shape[0]
    for p in range(pf.PF3_STATE_PLANES_THERMAL):
        assert rel(sg[p], so[p], 1e-12) <= max(tol, 1e-15), p


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_3d_thermal_steps_match_oracle(precision, tol):
    o, sim = pair_t(RAGGED, SEEDS, 5.0, precision, theta_field(RAGGED))
    sim.set_chunk(5)
    for _ in range(3):
        o.step(1)
        sim.step(1)
        compare_t(o, sim, tol)
    so, sg = o.state(), sim.get_state()
    for p in range(pf.PF3_STATE_PLANES_THERMAL):
        assert rel(sg[p], so[p], 1e-12) <= tol * 10, p


def test_3d_thermal_fp64_many_steps_conservation_and_latent_heat():
    """A centred seed over 150 steps in FP64: within 1e-9 of the oracle, the
    cube's symmetry, sum rho H constant to 1e-13 and the mean theta rising by
    (latent/2) x the mean psi rise."""
    n = 28
    o, sim = pair_t((n, n, n), [(n / 2, n / 2, n / 2)], 8.0, "fp64")
    t0 = sim.reduce_thermal()
    o.step(150)
    sim.step(150)
    compare_t(o, sim, 1e-9)
    psi = sim.fields()["psi"]
    for t in (psi.transpose(0, 2, 1), psi.transpose(2, 1, 0)):
        assert np.abs(psi - t).max() < 1e-12
    t1 = sim.reduce_thermal()
    assert abs(t1["sum_e"] / t0["sum_e"] - 1) < 1e-13
    dpsi, dth = t1["sum_psi"] - t0["sum_psi"], t1["sum_theta"] - t0["sum_theta"]
    assert dpsi > 0.05 * n ** 3 and abs(dth / (0.5 * dpsi) - 1) < 1e-9


def test_3d_thermal_fp32_drift_and_bounded_error():
    n = 32
    shape = (n, n, n)
    o, sim = pair_t(shape, [(10.0, 12.0, 16.0), (24.0, 20.0, 8.0)], 7.0, "fp32", theta_field(shape))
    t0, c0 = sim.reduce_thermal(), sim.reduce()["sum_C"]
    o.step(200)
    sim.step(200)
    compare_t(o, sim, 1e-3)
    assert abs(sim.reduce_thermal()["sum_e"] / t0["sum_e"] - 1) <= 1e-6
    assert abs(sim.reduce()["sum_C"] / c0 - 1) <= 1e-6


def test_3d_thermal_full_size_windows():
    """The 256^3 thermal workload (64 seeds, theta0 everywhere, Le 50) in the
    benchmark's launch configuration: after 2 steps, 24^3 windows match
    oracle windows placed in global coordinates."""
    n = 256
    seeds, R_s = wl.growth_3d(n)
    sim = pf.Simulation3D((n, n, n), dict(wl.BASE_PARAMS, **wl.THERMAL_PARAMS), "fp32")
    sim.init_seeds(seeds, R_s)
    T = 2
    sim.step(T)
    fg = sim.fields()
    sim.close()
    W, M = 24, 2 * T
    centres = [(int(s[0]) + 7, int(s[1]), int(s[2])) for s in seeds[:2]] + [(n - 2, n - 2, n - 2)]
    ref, got = {k: [] for k in fg}, {k: [] for k in fg}
    for cx, cy, cz in centres:
        x0, y0, z0 = cx - W // 2, cy - W // 2, cz - W // 2
        o = oracle.Oracle3D(W, W, W, dict(T3, **wl.THERMAL_PARAMS), window=(n, n, n, x0, y0, z0))
        o.init_spec(seeds, R_s)
        o.step(T)
        fo = o.fields()
        idx = [(np.arange(M, W - M) + c0) % n for c0 in (z0, y0, x0)]
        for k in fg:
            ref[k].append(fo[k][M:W - M, M:W - M, M:W - M].ravel())
            got[k].append(fg[k][np.ix_(*idx)].ravel())
    for k in fg:
        err = rel(np.concatenate(got[k]), np.concatenate(ref[k]), FLOOR_T[k])
        assert err <= 1e-5, (k, err)


def test_3d_thermal_configuration_errors():
    with pytest.raises(pf.PFError):
        pf.Simulation3D((8, 8, 8), dict(wl.BASE_PARAMS, **dict(T3, cp=0.5)), "fp32")
    iso = pf.Simulation3D((8, 8, 8), wl.BASE_PARAMS, "fp32")
    iso.init_seeds([(4, 4, 4)], 2.0)
    with pytest.raises(pf.PFError):
        iso.set_temperature(np.zeros((8, 8, 8)))          # not thermal
    with pytest.raises(pf.PFError):
        iso.reduce_thermal()
    sim = pf.Simulation3D((8, 8, 8), dict(wl.BASE_PARAMS, **T3), "fp32")
    with pytest.raises(pf.PFError) as e:
        sim.set_temperature(np.zeros((8, 8, 8)))          # not initialised
    assert e.value.code == pf.PF_ERR_STATE
    sim.init_seeds([(4, 4, 4)], 2.0)
    s0 = sim.get_state()
    th = np.full((8, 8, 8), -0.5)
    th[2, 3, 4] = np.nan
    with pytest.raises(pf.PFError) as e:
        sim.set_temperature(th)                            # found on the device
    assert e.value.code == pf.PF_ERR_BAD_ARG and "non-finite" in str(e.value)
    assert np.array_equal(sim.get_state(), s0)
    sim.step(1)
    with pytest.raises(pf.PFError) as e:
        sim.set_temperature(np.zeros((8, 8, 8)))          # already stepped
    assert e.value.code == pf.PF_ERR_STATE


@pytest.mark.parametrize("shape", [(4, 4, 4), (5, 7, 6), (33, 9, 17)])
@pytest.mark.parametrize("thermal", [False, True])
def test_3d_small_and_ragged_lattices(shape, thermal):
    """The smallest lattice, odd sizes, and ragged tiles and chunks, with and
    without the temperature lattice: FP64 within 1e-11 over 4 steps."""
    nx, ny, nz = shape
    params = T3 if thermal else P3
    o, sim = pair(shape, [(nx / 3, ny / 2, nz / 2)], 1.5, "fp64", params)
    sim.set_chunk(3)
    o.step(4)
    sim.step(4)
    (compare_t if thermal else compare)(o, sim, 1e-11)


# ---------------------------------------------------------------------------
# grain orientations (ROT template): each site takes the nearest seed's rotation
# ---------------------------------------------------------------------------
ROT = [(10.3, 9.1, 6.2, 0.9, 0.2, -0.3, 0.1), (33.0, 4.0, 11.5, 0.7, -0.1, 0.4, 0.6)]


@pytest.mark.parametrize("thermal", [False, True])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_3d_rotated_grains_match_oracle(precision, tol, thermal):
    params = T3 if thermal else P3
    o, sim = pair(RAGGED, [s[:3] for s in ROT], 5.0, precision, params)
    o.set_orientation(ROT)
    sim.set_orientation(ROT)
    sim.set_chunk(5)
    for _ in range(3):
        o.step(1)
        sim.step(1)
        (compare_t if thermal else compare)(o, sim, tol)


def test_3d_rotated_grains_fp64_many_steps():
    n = 28
    seeds7 = [(9.0, 10.0, 14.0, 0.9, 0.2, -0.3, 0.1), (20.0, 18.0, 12.0, 0.3, 0.5, 0.2, -0.8)]
    o, sim = pair((n, n, n), [s[:3] for s in seeds7], 6.0, "fp64")
    o.set_orientation(seeds7)
    sim.set_orientation(seeds7)
    c0 = sim.reduce()["sum_C"]
    o.step(120)
    sim.step(120)
    compare(o, sim, 1e-9)
    assert abs(sim.reduce()["sum_C"] / c0 - 1) <= 1e-12


def test_3d_identity_orientation_is_the_aligned_grain():
    """The identity rotation takes the ROT template through exactly the
    arithmetic of the aligned grain (bit for bit), and an empty orientation
    list returns to the aligned kernel."""
    seeds = [s[:3] for s in ROT]
    ident = [tuple(s) + (1.0, 0.0, 0.0, 0.0) for s in seeds]
    out = []
    for orient in (None, ident, "reset"):
        sim = pf.Simulation3D(RAGGED, dict(wl.BASE_PARAMS, **P3), "fp32")
        sim.init_seeds(seeds, 5.0)
        if orient == "reset":
            sim.set_orientation(ROT)
            sim.set_orientation([])
        elif orient is not None:
            sim.set_orientation(orient)
        sim.step(5)
        out.append(sim.fields())
    for f in out[1:]:
        for k in out[0]:
            assert np.array_equal(f[k], out[0][k]), k
    with pytest.raises(pf.PFError):
        sim.set_orientation([(1.0, 1.0, 1.0, 0.0, 0.0, 0.0, 0.0)])      # zero quaternion


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("thermal", [False, True])
@pytest.mark.parametrize("rotated", [False, True])
def test_3d_index_widths_are_bit_identical(precision, thermal, rotated):
    """The periodic melt step indexes sites and plane offsets in 32 bits while
    they fit and in 64 bits above: both forms run the same arithmetic, so the
    whole state after several steps agrees bit for bit (the 64-bit form forced
    on a small ragged lattice)."""
    seeds = [s[:3] for s in ROT]
    states = []
    for wide in (False, True):
        sim = pf.Simulation3D(RAGGED, dict(wl.BASE_PARAMS, **(T3 if thermal else P3)), precision)
        sim.init_seeds(seeds, 5.0)
        if thermal:
            sim.set_temperature(theta_field(RAGGED))
        if rotated:
            sim.set_orientation(ROT)
        sim.set_chunk(5)
        sim.set_index64(wide)
        sim.step(5)
        states.append(sim.get_state())
    assert states[0].shape == states[1].shape
    assert np.array_equal(states[0], states[1])


# ---------------------------------------------------------------------------
# non-periodic sides (BC template)
# ---------------------------------------------------------------------------
SIDES = [(1, 1, 2, 2, 3, 3), (3, 3, 0, 0, 1, 1), (2, 2, 3, 3, 0, 0)]


def pair_bc(shape, sides, precision, params, seeds=SEEDS, R_s=5.0):
    nx, ny, nz = shape
    o = oracle.Oracle3D(nx, ny, nz, params)
    o.set_bc(sides)
    o.init_spec(seeds, R_s)
    sim = pf.Simulation3D(shape, dict(wl.BASE_PARAMS, **params), precision)
    sim.set_boundaries(sides)
    sim.init_seeds(seeds, R_s)
    return o, sim


@pytest.mark.parametrize("sides", SIDES)
@pytest.mark.parametrize("thermal", [False, True])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_3d_sides_match_oracle(sides, thermal, precision, tol):
    params = T3 if thermal else P3
    o, sim = pair_bc(RAGGED, sides, precision, params)
    (compare_t if thermal else compare)(o, sim, tol)
    sim.set_chunk(5)
    for _ in range(3):
        o.step(1)
        sim.step(1)
        (compare_t if thermal else compare)(o, sim, tol)


def test_3d_sides_fp64_many_steps_with_rotated_grains():
    """Walls, symmetric planes and a far-field pair with rotated grains and the
    temperature lattice: FP64 within 1e-9 of the oracle over 120 steps; with
    walls and symmetric planes only, sum C and sum rho H are conserved."""
    n = 24
    seeds7 = [(4.0, 12.0, 12.0, 0.9, 0.2, -0.3, 0.1), (18.0, 6.0, 20.0, 0.3, 0.5, 0.2, -0.8)]
    for sides, conserving in (((1, 1, 2, 2, 1, 1), True), ((2, 2, 1, 1, 3, 3), False)):
        o, sim = pair_bc((n, n, n), sides, "fp64", T3, [s[:3] for s in seeds7], 5.0)
        o.set_orientation(seeds7)
        sim.set_orientation(seeds7)
        t0, c0 = sim.reduce_thermal(), sim.reduce()["sum_C"]
        o.step(120)
        sim.step(120)
        compare_t(o, sim, 1e-9)
        if conserving:
            assert abs(sim.reduce_thermal()["sum_e"] / t0["sum_e"] - 1) < 1e-12
            assert abs(sim.reduce()["sum_C"] / c0 - 1) < 1e-12


def test_3d_sides_configuration_errors():
    sim = pf.Simulation3D((8, 8, 8), wl.BASE_PARAMS, "fp32")
    with pytest.raises(pf.PFError):
        sim.set_boundaries((0, 1, 0, 0, 0, 0))      # periodic opposite a symmetric side
    with pytest.raises(pf.PFError):
        sim.set_boundaries((4, 4, 0, 0, 0, 0))      # no inlet in 3-D
    sim.init_seeds([(4, 4, 4)], 2.0)
    with pytest.raises(pf.PFError) as e:
        sim.set_boundaries((1, 1, 0, 0, 0, 0))      # after initialisation
    assert e.value.code == pf.PF_ERR_STATE
