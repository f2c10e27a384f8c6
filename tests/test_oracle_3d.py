"""Pins of the three-dimensional dendrite oracle (oracle/pf_oracle3d.c): the
anisotropic Allen-Cahn and solute equations of Section 2.1 on D3Q7 lattices,
with the anisotropy summed over three axes, in a melt without gas or flow
(reading R33).  Closed forms, exact symmetries, invariants, textbook special
cases and the reduction to the 2-D stencil."""
import math

import numpy as np
import pytest

import oracle
import pin_cases
from test_oracle_pins import _tanh_width

P3 = dict(beta_psi=0.25, W0=4.0, tau0=320.0, eps_s=0.05, k=0.15, D=0.1, Omega=0.55,
          grad_eps=1e-3, grad_eps_at=1e-2)
C7 = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]])
W7 = np.array([0.25] + [0.125] * 6)


def test_d3q7_collision_reduces_to_bgk_and_keeps_the_moments():
    """Equal rates give the BGK update f - s (f - f_eq) + (1 - s/2) G + Fd; with
    the flux rate apart, the zeroth moment is conserved (plus the source) and
    the flux relaxes at its own rate (Appendix B, Lambda = M^-1 S M)."""
    rng = np.random.default_rng(3)
    f, feq, G, Fd = rng.normal(size=(4, 7))
    G -= G.mean() * 0      # arbitrary forcing vector
    s = 0.7
    out = oracle.collide7(f, feq, np.full(7, s), G, Fd)
    assert np.allclose(out, f - s * (f - feq) + (1 - s / 2) * G + Fd, atol=1e-14)
    S = np.array([1.0, s, s, s, 1.0, 1.0, 1.0])
    out = oracle.collide7(f, feq, S, 0 * G, 0 * Fd)
    assert math.isclose(out.sum(), feq.sum(), abs_tol=1e-14)
    for a in range(3):
        j, jeq, jo = f @ C7[:, a], feq @ C7[:, a], out @ C7[:, a]
        assert math.isclose(jo, j - s * (j - jeq), abs_tol=1e-14)


def test_gradient_stencil_is_exact_on_quadratics_and_reduces_to_2d():
    """The D3Q19-weighted 18-neighbour gradient is exact on quadratic fields,
    and on a field that does not vary along z it equals the isotropic 9-point
    D2Q9 gradient of the 2-D model (reading R5)."""
    n = 8
    z, y, x = np.mgrid[0:n, 0:n, 0:n].astype(float)
    X = 0.3 * x * x - 0.2 * x * y + 0.1 * z * z + 0.5 * y - 0.7 * z
    g = oracle.grad3(X, 3, 4, 2)
    assert np.allclose(g, [0.6 * 3 - 0.2 * 4, -0.2 * 3 + 0.5, 0.2 * 2 - 0.7], atol=1e-13)
    rng = np.random.default_rng(4)
    F2 = rng.normal(size=(n, n))
    F3 = np.repeat(F2[None, :, :], 5, axis=0)
    for (xx, yy) in ((0, 0), (3, 5), (7, 2)):
        g3 = oracle.grad3(F3, xx, yy, 2)
        g2 = oracle.stencil(F2, xx, yy)
        assert np.allclose(g3[:2], g2[:2], atol=1e-14) and abs(g3[2]) < 1e-14


def anisotropy_closed_forms_hold(lib=None) -> bool:
    """a_s along the cube's axes, face and body diagonals, and N against
    central differences of a_s."""
    eps = 0.05
    ok = True
    for g, a in (((1.0, 0, 0), 1 + eps), ((1.0, 1.0, 0), 1 - eps),
                 ((1.0, 1.0, 1.0), 1 - 5 * eps / 3), ((0, 0, -2.0), 1 + eps)):
        out = oracle.aniso3(np.array(g) * 0.1, eps, 1e-12, lib)
        ok = ok and math.isclose(out[0], a, rel_tol=1e-9)
    rng = np.random.default_rng(5)
    for _ in range(5):
        g = rng.normal(size=3) * 0.1
        geps = 1e-3
        a, Nx, Ny, Nz, m = oracle.aniso3(g, eps, geps, lib)
        for ax, Nv in zip(range(3), (Nx, Ny, Nz)):
            h = 1e-7
            gp, gm_ = g.copy(), g.copy()
            gp[ax] += h
            gm_[ax] -= h
            da = (oracle.aniso3(gp, eps, geps, lib)[0] - oracle.aniso3(gm_, eps, geps, lib)[0]) / (2 * h)
            ok = ok and math.isclose(Nv, m * m * a * da, rel_tol=1e-6, abs_tol=1e-12)
    return bool(ok)


def test_anisotropy_closed_forms_in_three_dimensions():
    """a_s = 1 + eps (4 sum n^4 - 3): 1 + eps along <100>, 1 - eps along
    <110>, 1 - 5 eps / 3 along <111>; N = |g|^2 a_s d a_s / d g (Section 2.1)
    by central differences."""
    assert anisotropy_closed_forms_hold()


def test_single_seed_keeps_the_cubic_symmetry_and_solute_is_conserved():
    """A centred seed grows with the symmetry of the cube (axis permutations
    and reflections) to rounding, and sum C is constant."""
    n = 28
    o = oracle.Oracle3D(n, n, n, P3)
    o.init_spec([(n / 2, n / 2, n / 2)], 8.0)
    f0 = o.fields()
    C0, solid0 = f0["C"].sum(), (1 + f0["psi"]).sum()
    o.step(100)
    f = o.fields()
    psi = f["psi"]                       # [z][y][x]
    sh = lambda a, ax: np.roll(np.flip(a, axis=ax), 1, axis=ax)   # noqa: E731  x -> n - x
    for t in (psi.transpose(0, 2, 1), psi.transpose(2, 1, 0), psi.transpose(1, 0, 2),
              sh(psi, 0), sh(psi, 1), sh(psi, 2)):
        assert np.abs(psi - t).max() < 1e-12
    assert (1 + psi).sum() > 1.2 * solid0              # the seed grew
    assert abs(f["C"].sum() / C0 - 1) < 1e-12


def test_solute_gaussian_in_3d_spreads_with_variance_2Dt():
    """In the liquid (psi = -1) the solute equation is dC/dt = D lap C: a 3-D
    Gaussian's variance grows by 2 D per step along each axis (D3Q7, flux rate
    from D = (1/s - 1/2) c_s^2, c_s^2 = 1/4)."""
    n, s0, D = 48, 3.0, 0.1
    z, y, x = np.mgrid[0:n, 0:n, 0:n].astype(float)
    C = 1 + 0.1 * np.exp(-((x - 24) ** 2 + (y - 24) ** 2 + (z - 24) ** 2) / (2 * s0 * s0))
    o = oracle.Oracle3D(n, n, n, dict(P3, D=D))
    o.init_fields(-np.ones_like(C), C)
    var = []
    for T in (30, 90):
        o.step(T - (0 if T == 30 else 30))
        c = o.fields()["C"] - 1
        var.append([((q - 24) ** 2 * c).sum() / c.sum() for q in (x, y, z)])
    for a in range(3):
        assert math.isclose((var[1][a] - var[0][a]) / 60.0, 2 * D, rel_tol=2e-3)


def _front_width_3d(diagonal):
    N, W0, eps = 96, 4.0, 0.05
    x = np.arange(N, dtype=float)
    if diagonal:        # slab normal to <110>: s = x + y (mod N), distance |s - N/2| / sqrt 2
        s = (x[None, :] + x[:, None]) % N
        d = np.abs(s - N / 2) / math.sqrt(2)
    else:
        d = np.abs(x[None, :] - N / 2) * np.ones((N, 1))
    psi2 = np.tanh((22.0 - d) / (math.sqrt(2) * W0))
    psi = np.repeat(psi2[None, :, :], 2, axis=0)
    C = 1 - 0.85 * (1 + psi) / 2
    o = oracle.Oracle3D(N, N, 2, dict(P3, Omega=0.0, eps_s=eps))
    o.init_fields(psi, C)
    o.step(2000)
    row = o.fields()["psi"][0, 0, :]          # y = 0: s = x
    dd = np.abs(x - N / 2) / (math.sqrt(2) if diagonal else 1.0)
    return _tanh_width(dd, row, 22.0, math.sqrt(2) * W0)


def test_flat_fronts_have_the_3d_anisotropic_widths():
    """With zero driving force a flat slab relaxes to tanh(x / (sqrt2 W0 a_s)):
    a_s = 1 + eps for a front along <100> and 1 - eps along <110> (here a
    front that runs diagonally across the lattice, so the lattice's own
    anisotropy enters the width at the 1-2 % level)."""
    eps, W0 = 0.05, 4.0
    w100, h100 = _front_width_3d(False)
    w110, h110 = _front_width_3d(True)
    assert math.isclose(w100, math.sqrt(2) * W0 * (1 + eps), rel_tol=0.02)
    assert math.isclose(w110, math.sqrt(2) * W0 * (1 - eps), rel_tol=0.02)
    assert math.isclose(w100 / w110, (1 + eps) / (1 - eps), rel_tol=0.02)
    assert not math.isclose(w100 / w110, 1.0, rel_tol=0.05)    # anisotropy is there


# ---------------------------------------------------------------------------
# temperature coupling in 3-D (thermal mode: D3Q7 temperature lattice, F(U)
# and the grad F source of Appendix B; readings R28-R30, R33)
# ---------------------------------------------------------------------------
T3 = dict(P3, thermal=1, Le=2.0, latent=1.0, theta0=-0.55, cp=10.0, rho_l=1.0)


def enthalpy_latent_holds(lib=None) -> bool:
    """A centred seed solidifying for 150 steps, latent factor 1 and 1/2:
    sum rho H constant, mean theta rise (c_p^s/c_p)/2 x the mean psi rise."""
    n = 28
    ok = True
    for latent in (1.0, 0.5):
        o = oracle.Oracle3D(n, n, n, dict(T3, latent=latent), lib=lib)
        o.init_spec([(n / 2, n / 2, n / 2)], 8.0)
        t0, f0 = o.thermal_totals(), o.fields()
        o.step(150)
        t1, f1 = o.thermal_totals(), o.fields()
        dpsi = (f1["psi"].sum() - f0["psi"].sum()) / n ** 3
        dth = (t1["sum_theta"] - t0["sum_theta"]) / n ** 3
        ok = ok and (abs(t1["sum_e"] / t0["sum_e"] - 1) < 1e-13 and dpsi > 0.05 and
                     math.isclose(dth, 0.5 * latent * dpsi, rel_tol=1e-9))
    return bool(ok)


def test_3d_enthalpy_conserved_and_latent_heat_balance():
    """sum rho H is constant, and the mean temperature rises by (c_p^s/c_p)/2
    times the rise of the mean psi while a seed solidifies (Eq. eq-tem2)."""
    assert enthalpy_latent_holds()


def heat_variance_holds(lib=None) -> bool:
    """A temperature Gaussian in the liquid: its variance grows 2 Le D per
    step along each axis (Le = 1.5)."""
    m, Le = 56, 1.5
    z, y, x = np.mgrid[0:m, 0:m, 0:m].astype(float)
    th = -0.5 + 0.1 * np.exp(-((x - 28) ** 2 + (y - 28) ** 2 + (z - 28) ** 2) / 18.0)
    o = oracle.Oracle3D(m, m, m, dict(T3, Le=Le, theta0=-0.5), lib=lib)
    o.init_fields(-np.ones_like(th), np.ones_like(th), th)
    var = []
    for T in (40, 100):
        o.step(T - (0 if T == 40 else 40))
        w = o.fields()["theta"] + 0.5
        var.append([((q - 28) ** 2 * w).sum() / w.sum() for q in (x, y, z)])
    return all(math.isclose((var[1][a] - var[0][a]) / 60.0, 2 * Le * T3["D"], rel_tol=3e-3)
               for a in range(3))


def test_3d_heat_gaussian_variance():
    """In the liquid the temperature diffuses with alpha = Le D: a 3-D
    Gaussian's variance grows 2 alpha per step per axis."""
    assert heat_variance_holds()


def test_3d_gradF_source_matches_the_original_equation():
    """The planar problem of the 2-D grad F pin on a 192 x 4 x 4 lattice: the
    3-D scheme (D3Q7) follows the finite-difference solution of the original
    equations far better than that solution differs from the one without the
    grad F source."""
    from test_oracle_thermal import _fd_1d
    nx, W0 = 192, 8.0
    base = dict(beta_psi=0.25, W0=W0, tau0=2 * W0 ** 2 / 0.1, eps_s=0.0, k=0.15, D=0.1,
                Omega=0.55, grad_eps=1e-3, grad_eps_at=1e-2, thermal=1, Le=50.0, latent=1.0,
                theta0=-0.3, cp=10.0, rho_l=1.0)
    k = base["k"]
    x = np.arange(nx, dtype=float)
    psi0 = np.tanh(math.sqrt(0.5) * (nx / 6 - np.abs(x - nx / 2)) / W0)
    U0 = 0.5 * np.sin(4 * math.pi * x / nx)
    C0 = 0.5 * (1 + k - (1 - k) * psi0) * (1 + (1 - k) * U0)
    th0 = np.full(nx, base["theta0"])
    T = 1200
    o = oracle.Oracle3D(nx, 4, 4, base)
    tile = lambda a: np.tile(a, (4, 4, 1))          # noqa: E731  [z][y][x]
    o.init_fields(tile(psi0), tile(C0), tile(th0))
    o.step(T)
    f = o.fields()
    for a in ("psi", "C", "theta"):
        assert np.abs(f[a] - f[a][0, 0]).max() < 1e-13          # planar
    psi_fd, C_fd, th_fd = _fd_1d(base, psi0, C0, th0, T, 0.05, 1.0)
    psi_no, _, _ = _fd_1d(base, psi0, C0, th0, T, 0.05, 0.0)
    effect = np.abs(psi_fd - psi_no).max()
    assert effect > 0.03
    assert np.abs(f["psi"][0, 0] - psi_fd).max() < 0.15 * effect
    assert np.abs(f["C"][0, 0] - C_fd).max() < 0.01
    assert np.abs(f["theta"][0, 0] - th_fd).max() < 0.01


# ---------------------------------------------------------------------------
# grain orientations in 3-D (reading R10 for d = 3: crystal frame g' = R^T g,
# N = R N'(g'), each site takes the rotation of the nearest seed)
# ---------------------------------------------------------------------------
def _quat(axis, angle):
    q = [math.cos(angle / 2), 0.0, 0.0, 0.0]
    q[1 + axis] = math.sin(angle / 2)
    return q


def orientation_nearest_holds(lib=None) -> bool:
    """40 random sites: each carries the rotation of its nearest seed
    (minimum image), as scipy's rotation of that seed's quaternion."""
    from scipy.spatial.transform import Rotation
    n = 12
    seeds7 = [(2.0, 3.0, 4.0) + tuple(_quat(2, 0.3)), (9.5, 8.0, 10.0, 0.9, 0.2, -0.3, 0.1)]
    o = oracle.Oracle3D(n, n, n, P3, lib=lib)
    o.set_orientation(seeds7)
    rng = np.random.default_rng(3)
    ok = True
    for site in rng.integers(0, n ** 3, 40):
        x, y, z = site % n, (site // n) % n, site // (n * n)
        d2 = []
        for s in seeds7:
            dd = (np.array([x, y, z], float) - np.array(s[:3]) + n / 2) % n - n / 2
            d2.append((dd ** 2).sum())
        s = seeds7[int(np.argmin(d2))]
        want = Rotation.from_quat([s[4], s[5], s[6], s[3]]).as_matrix()
        ok = ok and np.abs(o.orientation(int(site)) - want).max() < 1e-14
    return bool(ok)


def test_3d_orientation_follows_the_nearest_seed():
    """Every site carries the rotation of the nearest seed (minimum image);
    the rotation is the one the quaternion defines (checked against scipy's)."""
    assert orientation_nearest_holds()


def test_3d_orientation_identity_and_cubic_symmetry():
    """The identity orientation reproduces the unoriented step bit for bit; a
    quarter turn about any axis maps the cubic anisotropy onto itself, so the
    grains grow exactly as unrotated (to rounding)."""
    n, seeds = 24, [(9.3, 11.0, 12.5), (17.0, 6.0, 5.0)]
    base = oracle.Oracle3D(n, n, n, P3)
    base.init_spec(seeds, 5.0)
    base.step(60)
    fb = base.fields()
    for q, tol in (([1.0, 0.0, 0.0, 0.0], 0.0), (_quat(0, math.pi / 2), 1e-12),
                   (_quat(1, math.pi / 2), 1e-12), (_quat(2, -math.pi / 2), 1e-12)):
        o = oracle.Oracle3D(n, n, n, P3)
        o.init_spec(seeds, 5.0)
        o.set_orientation([tuple(s) + tuple(q) for s in seeds])
        o.step(60)
        fo = o.fields()
        for k in ("psi", "C"):
            assert np.abs(fo[k] - fb[k]).max() <= tol * np.abs(fb[k]).max(), (q, k)


def _rotated_front_width(axis_front, q):
    N, W0, eps = 96, 4.0, 0.05
    x = np.arange(N, dtype=float)
    d1 = np.abs(x - N / 2)
    psi1 = np.tanh((22.0 - d1) / (math.sqrt(2) * W0))
    if axis_front == 0:
        psi = np.broadcast_to(psi1[None, None, :], (2, N, N)).copy()
    else:
        psi = np.broadcast_to(psi1[None, :, None], (2, N, N)).copy()
    o = oracle.Oracle3D(N, N, 2, dict(P3, Omega=0.0, eps_s=eps))
    o.init_fields(psi, 1 - 0.85 * (1 + psi) / 2)
    o.set_orientation([(N / 2, N / 2, 1.0) + tuple(q)])
    o.step(2000)
    f = o.fields()["psi"]
    row = f[0, 0, :] if axis_front == 0 else f[0, :, 0]
    return _tanh_width(d1, row, 22.0, math.sqrt(2) * W0)[0]


def test_3d_rotated_grain_front_widths():
    """A lattice-aligned flat front takes the width sqrt2 W0 a_s of the
    crystal direction it faces: turned by pi/4 about z, a front normal to x
    faces <110> (a_s = 1 - eps); turned by pi/4 about x, a front normal to y
    faces <011> (1 - eps) while one normal to x still faces <100> (1 + eps)."""
    W0, eps = 4.0, 0.05
    w_z = _rotated_front_width(0, _quat(2, math.pi / 4))
    w_xy = _rotated_front_width(1, _quat(0, math.pi / 4))
    w_xx = _rotated_front_width(0, _quat(0, math.pi / 4))
    # the lattice itself adds about 1 % to both widths (as for the unrotated fronts)
    assert math.isclose(w_z, math.sqrt(2) * W0 * (1 - eps), rel_tol=0.02)
    assert math.isclose(w_xy, math.sqrt(2) * W0 * (1 - eps), rel_tol=0.02)
    assert math.isclose(w_xx, math.sqrt(2) * W0 * (1 + eps), rel_tol=0.02)
    assert math.isclose(w_xx / w_z, (1 + eps) / (1 - eps), rel_tol=0.01)
    assert abs(w_xy / w_z - 1) < 1e-9        # the same crystal direction, two rotations


# ---------------------------------------------------------------------------
# non-periodic sides of the melt step (reading R35: on D3Q7 a symmetric side
# and a wall are both the half-way bounce-back; a far-field side the
# anti-bounce-back to psi = -1, C = 1, theta = theta0; stencil ghosts mirror)
# ---------------------------------------------------------------------------
def _mirror_fields(n_small, ny, nz, seed_x, thermal):
    """Fields on an n_small-wide box and on the 2 n_small periodic box made of it
    and its mirror image."""
    z, y, x = np.mgrid[0:nz, 0:ny, 0:2 * n_small].astype(float)
    xs = np.where(x < n_small, x, 2 * n_small - 1 - x)
    r = np.sqrt((xs - seed_x) ** 2 + (y - ny / 2) ** 2 + (z - nz / 3) ** 2)
    psi = np.tanh(math.sqrt(0.5) * (5.0 - r) / 4.0)
    C = 1 - 0.85 * (1 + psi) / 2 + 0.02 * np.cos(2 * np.pi * y / ny)
    th = -0.55 + 0.03 * np.sin(2 * np.pi * z / nz) if thermal else None
    return psi, C, th


@pytest.mark.parametrize("side,thermal", [(1, False), (2, False), (1, True)])
def test_3d_symmetric_sides_are_mirror_planes(side, thermal):
    """A box with symmetric (or wall) sides in x evolves exactly as the left
    half of the periodic box twice as wide that holds the box and its mirror
    image (both side types act on D3Q7 as the half-way bounce-back)."""
    n, ny, nz = 12, 10, 8
    psi, C, th = _mirror_fields(n, ny, nz, 3.5, thermal)
    params = dict(P3, **(dict(thermal=1, Le=2.0, theta0=-0.55) if thermal else {}))
    big = oracle.Oracle3D(2 * n, ny, nz, params)
    big.init_fields(psi, C, th)
    small = oracle.Oracle3D(n, ny, nz, params)
    small.set_bc([side, side, 0, 0, 0, 0])
    small.init_fields(psi[:, :, :n], C[:, :, :n], None if th is None else th[:, :, :n])
    big.step(60)
    small.step(60)
    fb, fs = big.fields(), small.fields()
    for k in ("psi", "C", "U") + (("theta",) if thermal else ()):
        half = fb[k][:, :, :n]
        assert np.abs(fs[k] - half).max() <= 1e-12 * max(np.abs(half).max(), 1e-3), k
        assert np.abs(fb[k][:, :, n:] - half[:, :, ::-1]).max() <= 1e-12 * max(np.abs(half).max(), 1e-3)


def test_3d_walls_conserve_solute_and_enthalpy():
    """Walls on all six sides: no flux leaves, so sum C and sum rho H stay
    constant to rounding while a seed grows against a side."""
    n = 20
    o = oracle.Oracle3D(n, n, n, dict(P3, thermal=1, Le=2.0, theta0=-0.55))
    o.set_bc([2, 2, 2, 2, 2, 2])
    o.init_spec([(3.0, 10.0, 10.0)], 5.0)
    c0, t0 = o.fields()["C"].sum(), o.thermal_totals()
    o.step(150)
    assert abs(o.fields()["C"].sum() / c0 - 1) < 1e-13
    assert abs(o.thermal_totals()["sum_e"] / t0["sum_e"] - 1) < 1e-13
    assert o.fields()["psi"].max() > 0.5


def test_3d_far_field_sides_are_half_way_dirichlet():
    """Far-field sides at x = -1/2 and x = nx - 1/2 hold C = 1: in a liquid
    (psi = -1) a uniform deficit 1 - C relaxes as the slowest Dirichlet mode,
    decaying at D (pi / nx)^2 per step (D_C = D in the liquid)."""
    nx, D = 32, 0.1
    one = np.ones((4, 4, nx))
    o = oracle.Oracle3D(nx, 4, 4, dict(P3, D=D))
    o.set_bc([3, 3, 0, 0, 0, 0])
    o.init_fields(-one, 0.8 * one)
    o.step(1000)                      # the higher odd modes have died out
    a0 = 1 - o.fields()["C"][0, 0, nx // 2]
    o.step(1000)
    a1 = 1 - o.fields()["C"][0, 0, nx // 2]
    rate = math.log(a0 / a1) / 1000
    assert math.isclose(rate, D * (math.pi / nx) ** 2, rel_tol=0.01)
    assert np.abs(o.fields()["psi"] + 1).max() < 1e-12


def test_3d_time_stretch_follows_the_original_equation():
    """The 3-D melt step carries Eq. eq-AnACE's tau0 a_s^2 d psi/dt by the
    time stretch of Appendix B, as in 2-D.  A slab with fronts along <100>
    (a_s = 1 + eps_s) on a 192 x 4 x 4 lattice follows the finite-difference
    solution of the 1-D original equations to 0.006 (measured 0.0023), a
    quarter of its distance to the solution with tau0 a_s; without the stretch
    the solutions differ by 0.055."""
    errs, nonuniform = pin_cases.stretch_errors("3d")
    gap = np.abs(pin_cases.front_fd(2) - pin_cases.front_fd(1)).max()
    assert errs[2] < 0.006 and errs[2] < 0.25 * gap
    assert pin_cases.stretch_pin_holds(errs)
    assert errs[1] > 0.02 and errs[0] > 0.04
    assert nonuniform < 1e-12
