"""The 3-D two-phase step (NS and CAC on D3Q19, psi and C on D3Q7, reading
R34) of the CUDA path against the FP64 3-D two-phase oracle, through the C
ABI.  FP64 within 1e-11 relative per field over a few steps (1e-9 over a
hundred); FP32 within 1e-5 per step for phi, psi, C, U and within 5e-5 for
v and p of a developed flow (their populations carry the rounding of O(0.05)
values into O(1e-3) differences) and 1e-4 for mu_phi (W_phi^2 times the
18-neighbour Laplacian amplifies the storage rounding of phi)."""
import numpy as np
import pytest

import oracle
from paper_2407_01651_gb300 import pf
from paper_2407_01651_gb300 import workload as wl

pytestmark = pytest.mark.gpu

P3F = {k: wl.BASE_PARAMS[k] for k in oracle.PARAM_NAMES_3F}
FLOOR = {"phi": 1e-9, "psi": 1e-9, "C": 1e-9, "U": 0.1, "p": 1e-4, "vx": 1e-3, "vy": 1e-3,
         "vz": 1e-3, "mu": 1e-3, "theta": 1e-9}
TOL32 = {"phi": 1e-5, "psi": 1e-5, "C": 1e-5, "U": 1e-5, "p": 5e-5, "vx": 5e-5, "vy": 5e-5,
         "vz": 5e-5, "mu": 1e-4, "theta": 1e-5}

RAGGED = (40, 19, 13)
SEEDS = [(10.3, 9.1, 6.2), (33.0, 4.0, 11.5)]
BUBBLES = [(25.0, 12.0, 7.0, 5.0), (6.0, 15.0, 3.0, 3.5)]


def rel(a, b, floor):
    return np.abs(a - b).max() / max(np.abs(b).max(), floor)


def flow_fields(shape, seeds, R_s, bubbles, amp=1e-3):
    """Spec fields plus a smooth velocity and pressure (a developed flow)."""
    nx, ny, nz = shape
    o = oracle.Oracle3F(nx, ny, nz, P3F)
    f = o.fields_from_spec(seeds, R_s, bubbles)
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx].astype(float)
    kx, ky, kz = 2 * np.pi / nx, 2 * np.pi / ny, 2 * np.pi / nz
    vx = amp * np.sin(ky * y + 0.3) * np.cos(kz * z)
    vy = amp * np.sin(kz * z + 1.1) * np.cos(kx * x)
    vz = amp * np.sin(kx * x + 0.7) * np.cos(ky * y)
    p = 0.1 * amp * np.cos(kx * x) * np.sin(ky * y + kz * z)
    return f["phi"], f["psi"], f["C"], vx, vy, vz, p


def pair(shape, precision, seeds=SEEDS, R_s=5.0, bubbles=BUBBLES, params=P3F, amp=1e-3):
    nx, ny, nz = shape
    planes = flow_fields(shape, seeds, R_s, bubbles, amp)
    o = oracle.Oracle3F(nx, ny, nz, params)
    o.init_fields(*planes)
    sim = pf.Simulation3F(shape, dict(wl.BASE_PARAMS, **params), precision)
    sim.set_fields(*planes)
    return o, sim


def compare(o, sim, tol):
    fo, fg = o.fields(), sim.fields()
    errs = {k: rel(fg[k], fo[k], FLOOR[k]) for k in fg}
    lim = {k: (tol[k] if isinstance(tol, dict) else tol) for k in fg}
    assert all(errs[k] <= lim[k] for k in fg), errs
    return errs


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_3f_initial_state(precision, tol):
    o, sim = pair(RAGGED, precision)
    assert abs(sim.rho_bar / o.rho_bar - 1) < 1e-7
    so, sg = o.state(), sim.get_state()
    assert sg.shape[0] == pf.PF3F_STATE_PLANES == so.shape[0]
    for p in range(pf.PF3F_STATE_PLANES):
        assert rel(sg[p], so[p], 1e-12) <= max(tol, 1e-15), p


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", TOL32)])
def test_3f_steps_match_oracle(precision, tol):
    o, sim = pair(RAGGED, precision)
    o.set_rho_bar(sim.rho_bar)
    sim.set_chunk(5)
    for _ in range(3):
        o.step(1)
        sim.step(1)
        compare(o, sim, tol)
    if precision == "fp64":
        so, sg = o.state(), sim.get_state()
        for p in range(pf.PF3F_STATE_PLANES):
            assert rel(sg[p], so[p], 1e-12) <= 1e-10, p


def test_3f_fp64_many_steps_and_conservation():
    """100 FP64 steps with gravity, a bubble and a seed: within 1e-9 of the
    oracle; sum phi and sum C constant to 1e-12."""
    n = 24
    params = dict(P3F, g=1e-5)
    o, sim = pair((n, n, n), "fp64", [(8.0, 12.0, 12.0)], 5.0, [(16.5, 11.0, 12.5, 4.5)], params)
    o.set_rho_bar(sim.rho_bar)
    r0 = sim.reduce()
    o.step(100)
    sim.step(100)
    compare(o, sim, 1e-9)
    r1 = sim.reduce()
    assert abs(r1["sum_phi"] / r0["sum_phi"] - 1) < 1e-12
    assert abs(r1["sum_C"] / r0["sum_C"] - 1) < 1e-12


def test_3f_fp32_drift_and_bounded_error():
    n = 32
    o, sim = pair((n, n, n), "fp32", [(10.0, 12.0, 16.0)], 6.0,
                  [(22.0, 20.0, 10.0, 6.0), (8.0, 26.0, 24.0, 4.0)])
    o.set_rho_bar(sim.rho_bar)
    r0 = sim.reduce()
    o.step(200)
    sim.step(200)
    compare(o, sim, 2e-3)
    r1 = sim.reduce()
    assert abs(r1["sum_phi"] / r0["sum_phi"] - 1) <= 1e-6
    assert abs(r1["sum_C"] / r0["sum_C"] - 1) <= 1e-6


def test_3f_full_size_windows():
    """The 256^3 two-phase workload (32 seeds, 64 bubbles) in the benchmark's
    launch configuration: after 2 steps, 24^3 windows around seeds, bubbles
    and across the periodic corner match oracle windows placed in global
    coordinates with the global buoyancy reference."""
    n = 256
    seeds, R_s, bubbles = wl.flow_3d(n)
    sim = pf.Simulation3F((n, n, n), wl.BASE_PARAMS, "fp32")
    sim.init_spec(seeds, R_s, bubbles)
    T = 2
    sim.step(T)
    fg = sim.fields()
    sim.close()
    W, M = 24, 2 * T
    centres = ([(int(s[0]) + 7, int(s[1]), int(s[2])) for s in seeds[:2]] +
               [(int(b[0]) + int(b[3]), int(b[1]), int(b[2])) for b in bubbles[:2]] +
               [(n - 2, n - 2, n - 2)])
    ref, got = {k: [] for k in fg}, {k: [] for k in fg}
    rho_bar = None
    for cx, cy, cz in centres:
        x0, y0, z0 = cx - W // 2, cy - W // 2, cz - W // 2
        o = oracle.Oracle3F(W, W, W, P3F, window=(n, n, n, x0, y0, z0))
        if rho_bar is None:
            rho_bar = P3F["rho_g"] + o.mean_phi_global(bubbles) * (P3F["rho_l"] - P3F["rho_g"])
        o.set_rho_bar(rho_bar)
        o.init_spec(seeds, R_s, bubbles)
        o.step(T)
        fo = o.fields()
        idx = [(np.arange(M, W - M) + c0) % n for c0 in (z0, y0, x0)]
        for k in fg:
            ref[k].append(fo[k][M:W - M, M:W - M, M:W - M].ravel())
            got[k].append(fg[k][np.ix_(*idx)].ravel())
    for k in fg:
        err = rel(np.concatenate(got[k]), np.concatenate(ref[k]), FLOOR[k])
        assert err <= TOL32[k], (k, err)


def test_3f_configuration_errors():
    with pytest.raises(pf.PFError):
        pf.Simulation3F((3, 8, 8), wl.BASE_PARAMS, "fp32")
    with pytest.raises(pf.PFError):
        pf.Simulation3F((8, 8, 8), wl.BASE_PARAMS, "fp16")
    with pytest.raises(pf.PFError):
        pf.Simulation3F((8, 8, 8), dict(wl.BASE_PARAMS, thermal=2), "fp32")
    sim = pf.Simulation3F((8, 8, 8), wl.BASE_PARAMS, "fp32")
    with pytest.raises(pf.PFError) as e:
        sim.step(1)                        # not initialised
    assert e.value.code == pf.PF_ERR_STATE
    with pytest.raises(pf.PFError):
        sim.set_fields(*[np.full((8, 8, 8), np.nan)] * 3)
    # one non-finite value anywhere is found on the device; the state is kept
    one = np.ones((8, 8, 8))
    sim.set_fields(one, -one, one)
    s0 = sim.get_state()
    vz = np.zeros((8, 8, 8))
    vz[1, 2, 3] = np.inf
    with pytest.raises(pf.PFError) as e:
        sim.set_fields(one, -one, one, vz=vz)
    assert e.value.code == pf.PF_ERR_BAD_ARG and "non-finite" in str(e.value)
    assert np.array_equal(sim.get_state(), s0)


def test_3f_free_rates_and_gravity():
    """Free MRT rates of the energy moments away from 1 (s_e = 1.2, s_eps =
    0.9) and gravity on: the e and eps rows of the NS collision enter, FP64
    within 1e-11 of the oracle over 3 steps."""
    params = dict(P3F, s_e=1.2, s_eps=0.9, g=2e-5)
    o, sim = pair(RAGGED, "fp64", params=params)
    o.set_rho_bar(sim.rho_bar)
    for _ in range(3):
        o.step(1)
        sim.step(1)
        compare(o, sim, 1e-11)


@pytest.mark.parametrize("shape", [(4, 4, 4), (5, 7, 6), (33, 9, 17)])
def test_3f_small_and_ragged_lattices(shape):
    """The smallest lattice (one site more than the stencil reach on each
    side), odd sizes, and tiles ragged in x and y with chunks ragged in z."""
    nx, ny, nz = shape
    seeds = [(nx / 3, ny / 2, nz / 2)]
    bubbles = [(2 * nx / 3, ny / 3, nz / 3, 1.5)]
    o, sim = pair(shape, "fp64", seeds=seeds, R_s=1.5, bubbles=bubbles)
    o.set_rho_bar(sim.rho_bar)
    sim.set_chunk(3)
    o.step(4)
    sim.step(4)
    compare(o, sim, 1e-11)


ROT = [(10.3, 9.1, 6.2, 0.9, 0.2, -0.3, 0.1), (33.0, 4.0, 11.5, 0.7, -0.1, 0.4, 0.6)]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", TOL32)])
def test_3f_rotated_grains_match_oracle(precision, tol):
    """Grain orientations in the two-phase step (each site takes the nearest
    seed's rotation): the oracle with the same orientations over 3 steps."""
    o, sim = pair(RAGGED, precision, seeds=[s[:3] for s in ROT])
    o.set_orientation(ROT)
    sim.set_orientation(ROT)
    o.set_rho_bar(sim.rho_bar)
    sim.set_chunk(5)
    for _ in range(3):
        o.step(1)
        sim.step(1)
        compare(o, sim, tol)


def test_3f_identity_orientation_is_the_aligned_grain():
    seeds = [s[:3] for s in ROT]
    out = []
    for orient in (None, [tuple(s) + (1.0, 0.0, 0.0, 0.0) for s in seeds]):
        sim = pf.Simulation3F(RAGGED, wl.BASE_PARAMS, "fp32")
        sim.init_spec(seeds, 5.0, BUBBLES)
        if orient is not None:
            sim.set_orientation(orient)
        sim.step(4)
        out.append(sim.fields())
    for k in out[0]:
        assert np.array_equal(out[1][k], out[0][k]), k


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("thermal", [False, True])
@pytest.mark.parametrize("rotated", [False, True])
def test_3f_index_widths_are_bit_identical(precision, thermal, rotated):
    """The periodic step indexes sites and plane offsets in 32 bits while they
    fit and in 64 bits above: both forms run the same arithmetic, so the whole
    state after several steps agrees bit for bit (the 64-bit form forced on a
    small ragged lattice)."""
    params = dict(T3F if thermal else P3F)
    seeds = [s[:3] for s in ROT]
    states = []
    for wide in (False, True):
        sim = pf.Simulation3F(RAGGED, dict(wl.BASE_PARAMS, **params), precision)
        sim.init_spec(seeds, 5.0, BUBBLES)
        if thermal:
            sim.set_temperature(theta_field(RAGGED))
        if rotated:
            sim.set_orientation(ROT)
        sim.set_chunk(5)
        sim.set_index64(wide)
        sim.step(4)
        states.append(sim.get_state())
    assert states[0].shape == states[1].shape
    assert np.array_equal(states[0], states[1])



# ---------------------------------------------------------------------------
# thermal mode (TH template): advected temperature lattice, F(U), grad F source
# ---------------------------------------------------------------------------
T3F = dict(P3F, thermal=1, Le=2.0, latent=1.0, theta0=-0.55, cp=10.0)


def theta_field(shape):
    nx, ny, nz = shape
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx].astype(float)
    return -0.55 + 0.05 * np.sin(2 * np.pi * x / nx) * np.cos(2 * np.pi * z / nz) + \
        0.03 * np.exp(-((y - ny / 2) ** 2) / 8.0)


def pair_t(shape, precision, params=T3F, **kw):
    o, sim = pair(shape, precision, params=params, **kw)
    th = theta_field(shape)
    o.set_temperature(th)
    sim.set_temperature(th)
    o.set_rho_bar(sim.rho_bar)
    return o, sim


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", TOL32)])
def test_3f_thermal_steps_match_oracle(precision, tol):
    o, sim = pair_t(RAGGED, precision)
    assert set(sim.fields()) == set(oracle.FIELDS_3F)
    sim.set_chunk(5)
    for _ in range(3):
        o.step(1)
        sim.step(1)
        compare(o, sim, tol)
    if precision == "fp64":
        so, sg = o.state(), sim.get_state()
        assert sg.shape[0] == pf.PF3F_STATE_PLANES_THERMAL == so.shape[0]
        for p in range(pf.PF3F_STATE_PLANES_THERMAL):
            assert rel(sg[p], so[p], 1e-12) <= 1e-10, p


def test_3f_thermal_fp64_many_steps_and_conservation():
    """100 FP64 steps with gravity, a bubble, a rotated seed and the
    temperature lattice: within 1e-9 of the oracle; sum rho H, sum phi and
    sum C constant to 1e-12."""
    n = 24
    params = dict(T3F, g=1e-5)
    seeds7 = [(8.0, 12.0, 12.0, 0.9, 0.2, -0.3, 0.1)]
    o, sim = pair_t((n, n, n), "fp64", params=params, seeds=[s[:3] for s in seeds7], R_s=5.0,
                    bubbles=[(16.5, 11.0, 12.5, 4.5)])
    o.set_orientation(seeds7)
    sim.set_orientation(seeds7)
    t0, r0 = sim.reduce_thermal(), sim.reduce()
    o.step(100)
    sim.step(100)
    compare(o, sim, 1e-9)
    t1, r1 = sim.reduce_thermal(), sim.reduce()
    assert abs(t1["sum_e"] / t0["sum_e"] - 1) < 1e-12
    assert abs(r1["sum_phi"] / r0["sum_phi"] - 1) < 1e-12
    assert abs(r1["sum_C"] / r0["sum_C"] - 1) < 1e-12


def test_3f_thermal_fp32_drift_and_bounded_error():
    n = 32
    o, sim = pair_t((n, n, n), "fp32", seeds=[(10.0, 12.0, 16.0)], R_s=6.0,
                    bubbles=[(22.0, 20.0, 10.0, 6.0), (8.0, 26.0, 24.0, 4.0)])
    t0 = sim.reduce_thermal()
    o.step(200)
    sim.step(200)
    compare(o, sim, 2e-3)
    assert abs(sim.reduce_thermal()["sum_e"] / t0["sum_e"] - 1) <= 1e-6


def test_3f_thermal_full_size_windows():
    """The 256^3 thermal two-phase workload (32 seeds, 64 bubbles, Le 50,
    theta0 everywhere) in the benchmark's launch configuration: after 2 steps,
    24^3 windows match oracle windows in global coordinates."""
    n = 256
    seeds, R_s, bubbles = wl.flow_3d(n)
    params = dict(P3F, **wl.THERMAL_PARAMS)
    sim = pf.Simulation3F((n, n, n), dict(wl.BASE_PARAMS, **wl.THERMAL_PARAMS), "fp32")
    sim.init_spec(seeds, R_s, bubbles)
    T = 2
    sim.step(T)
    fg = sim.fields()
    sim.close()
    W, M = 24, 2 * T
    centres = ([(int(s[0]) + 7, int(s[1]), int(s[2])) for s in seeds[:2]] +
               [(int(b[0]) + int(b[3]), int(b[1]), int(b[2])) for b in bubbles[:2]])
    ref, got = {k: [] for k in fg}, {k: [] for k in fg}
    rho_bar = None
    for cx, cy, cz in centres:
        x0, y0, z0 = cx - W // 2, cy - W // 2, cz - W // 2
        o = oracle.Oracle3F(W, W, W, params, window=(n, n, n, x0, y0, z0))
        if rho_bar is None:
            rho_bar = P3F["rho_g"] + o.mean_phi_global(bubbles) * (P3F["rho_l"] - P3F["rho_g"])
        o.set_rho_bar(rho_bar)
        o.init_spec(seeds, R_s, bubbles)
        o.step(T)
        fo = o.fields()
        idx = [(np.arange(M, W - M) + c0) % n for c0 in (z0, y0, x0)]
        for k in fg:
            ref[k].append(fo[k][M:W - M, M:W - M, M:W - M].ravel())
            got[k].append(fg[k][np.ix_(*idx)].ravel())
    for k in fg:
        err = rel(np.concatenate(got[k]), np.concatenate(ref[k]), FLOOR[k])
        assert err <= TOL32[k], (k, err)


def test_3f_thermal_configuration_errors():
    with pytest.raises(pf.PFError):
        pf.Simulation3F((8, 8, 8), dict(wl.BASE_PARAMS, **dict(T3F, cp=5.0)), "fp32")  # rho_g cp < 3/4
    iso = pf.Simulation3F((8, 8, 8), wl.BASE_PARAMS, "fp32")
    iso.init_spec([(4, 4, 4)], 2.0, [])
    with pytest.raises(pf.PFError):
        iso.set_temperature(np.zeros((8, 8, 8)))
    with pytest.raises(pf.PFError):
        iso.reduce_thermal()
    sim = pf.Simulation3F((8, 8, 8), dict(wl.BASE_PARAMS, **T3F), "fp32")
    sim.init_spec([(4, 4, 4)], 2.0, [])
    s0 = sim.get_state()
    th = np.full((8, 8, 8), -0.5)
    th[7, 0, 1] = np.inf
    with pytest.raises(pf.PFError) as e:
        sim.set_temperature(th)                            # found on the device
    assert e.value.code == pf.PF_ERR_BAD_ARG and "non-finite" in str(e.value)
    assert np.array_equal(sim.get_state(), s0)
    sim.step(1)
    with pytest.raises(pf.PFError) as e:
        sim.set_temperature(np.zeros((8, 8, 8)))
    assert e.value.code == pf.PF_ERR_STATE


def test_3f_thermal_long_fp32_run():
    """2000 FP32 steps of the thermal two-phase step with gravity, bubbles and
    rotated grains on 64^3: every field stays finite, sum phi and sum rho H stay
    put, the solid grows and the released latent heat warms the melt."""
    n = 64
    seeds, R_s, bub = wl.flow_3d(n, 4, 6, rng_seed=7)
    par = dict(wl.BASE_PARAMS, **wl.THERMAL_PARAMS, g=1e-5)
    sim = pf.Simulation3F((n, n, n), par, "fp32")
    sim.init_spec(seeds, R_s, bub)
    sim.set_orientation([tuple(s) + (0.9, 0.1 * i, -0.2, 0.3) for i, s in enumerate(seeds)])
    r0, t0 = sim.reduce(), sim.reduce_thermal()
    sim.step(2000)
    f, r, t = sim.fields(), sim.reduce(), sim.reduce_thermal()
    assert all(np.isfinite(v).all() for v in f.values())
    assert abs(r["sum_phi"] / r0["sum_phi"] - 1) < 1e-8
    assert abs(r["sum_C"] / r0["sum_C"] - 1) < 1e-6
    assert abs(t["sum_e"] / t0["sum_e"] - 1) < 1e-6
    assert r["sum_hpsi"] > 1.5 * r0["sum_hpsi"]
    assert f["theta"].mean() > wl.THERMAL_PARAMS["theta0"]


# ---------------------------------------------------------------------------
# non-periodic sides (BC template)
# ---------------------------------------------------------------------------
SIDES = [(1, 1, 2, 2, 3, 3), (2, 2, 0, 0, 1, 1), (3, 3, 1, 1, 0, 0)]


def pair_bc(shape, sides, precision, params=P3F, seeds=SEEDS, R_s=5.0, bubbles=BUBBLES):
    nx, ny, nz = shape
    o = oracle.Oracle3F(nx, ny, nz, params)
    o.set_bc(sides)
    o.init_spec(seeds, R_s, bubbles)
    sim = pf.Simulation3F(shape, dict(wl.BASE_PARAMS, **params), precision)
    sim.set_boundaries(sides)
    sim.init_spec(seeds, R_s, bubbles)
    o.set_rho_bar(sim.rho_bar)
    return o, sim


@pytest.mark.parametrize("sides", SIDES)
@pytest.mark.parametrize("thermal", [False, True])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", TOL32)])
def test_3f_sides_match_oracle(sides, thermal, precision, tol):
    o, sim = pair_bc(RAGGED, sides, precision, dict(T3F if thermal else P3F, g=2e-5))
    sim.set_chunk(5)
    for _ in range(3):
        o.step(1)
        sim.step(1)
        compare(o, sim, tol)


def test_3f_sides_fp64_many_steps():
    """Symmetric planes and walls with gravity, a bubble, a rotated seed and
    the temperature lattice: FP64 within 1e-9 of the oracle over 100 steps,
    sum phi, sum C and sum rho H constant to 1e-12."""
    n = 24
    seeds7 = [(6.0, 12.0, 12.0, 0.9, 0.2, -0.3, 0.1)]
    o, sim = pair_bc((n, n, n), (1, 1, 2, 2, 1, 1), "fp64", dict(T3F, g=2e-5),
                     [s[:3] for s in seeds7], 5.0, [(16.0, 10.0, 12.0, 4.5)])
    o.set_orientation(seeds7)
    sim.set_orientation(seeds7)
    r0, t0 = sim.reduce(), sim.reduce_thermal()
    o.step(100)
    sim.step(100)
    compare(o, sim, 1e-9)
    r1, t1 = sim.reduce(), sim.reduce_thermal()
    assert abs(r1["sum_phi"] / r0["sum_phi"] - 1) < 1e-12
    assert abs(r1["sum_C"] / r0["sum_C"] - 1) < 1e-12
    assert abs(t1["sum_e"] / t0["sum_e"] - 1) < 1e-12


def test_3f_sides_configuration_errors():
    sim = pf.Simulation3F((8, 8, 8), wl.BASE_PARAMS, "fp32")
    with pytest.raises(pf.PFError):
        sim.set_boundaries((0, 2, 0, 0, 0, 0))
    sim.init_spec([(4, 4, 4)], 2.0, [])
    with pytest.raises(pf.PFError) as e:
        sim.set_boundaries((1, 1, 0, 0, 0, 0))
    assert e.value.code == pf.PF_ERR_STATE


# ---------------------------------------------------------------------------
# z-tile length: the march recomputes its ring at each tile start, so the
# tiling of z must not change a single bit of the state
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("kind", ["periodic", "thermal", "sides"])
def test_3f_z_tile_length_does_not_change_the_state(precision, kind):
    """80 planes in z: the default tile (36: tiles of 36, 36 and a ragged 8),
    tiles of 5, 7 (ragged 3) and one tile over all of z give the same state
    bit for bit after several steps, periodic, with the temperature lattice
    and with walls and symmetric planes."""
    shape = (40, 24, 80)
    params = dict(T3F if kind == "thermal" else P3F, g=2e-5)
    seeds = [(10.3, 9.1, 6.2), (33.0, 14.0, 40.5), (20.0, 4.0, 74.0)]
    bubbles = [(25.0, 12.0, 36.0, 5.0), (6.0, 15.0, 78.0, 3.5)]
    states = []
    for chunk in (None, 5, 7, 80):
        sim = pf.Simulation3F(shape, dict(wl.BASE_PARAMS, **params), precision)
        if kind == "sides":
            sim.set_boundaries((1, 1, 2, 2, 3, 3))
        sim.init_spec(seeds, 5.0, bubbles)
        if kind == "thermal":
            sim.set_temperature(theta_field(shape))
        if chunk is not None:
            sim.set_chunk(chunk)
        sim.step(5)
        states.append(sim.get_state())
        sim.close()
    for s in states[1:]:
        assert np.array_equal(s, states[0])
