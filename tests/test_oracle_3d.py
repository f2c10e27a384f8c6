"""Pins of the three-dimensional dendrite oracle (oracle/pf_oracle3d.c): the
anisotropic Allen-Cahn and solute equations of Section 2.1 on D3Q7 lattices,
with the anisotropy summed over three axes, in a melt without gas or flow
(reading R33).  Closed forms, exact symmetries, invariants, textbook special
cases and the reduction to the 2-D stencil."""
import math

import numpy as np

import oracle
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


def test_anisotropy_closed_forms_in_three_dimensions():
    """a_s = 1 + eps (4 sum n^4 - 3): 1 + eps along <100>, 1 - eps along
    <110>, 1 - 5 eps / 3 along <111>; N = |g|^2 a_s d a_s / d g (Section 2.1)
    by central differences."""
    eps = 0.05
    for g, a in (((1.0, 0, 0), 1 + eps), ((1.0, 1.0, 0), 1 - eps),
                 ((1.0, 1.0, 1.0), 1 - 5 * eps / 3), ((0, 0, -2.0), 1 + eps)):
        out = oracle.aniso3(np.array(g) * 0.1, eps, 1e-12)
        assert math.isclose(out[0], a, rel_tol=1e-9)
    rng = np.random.default_rng(5)
    for _ in range(5):
        g = rng.normal(size=3) * 0.1
        geps = 1e-3
        a, Nx, Ny, Nz, m = oracle.aniso3(g, eps, geps)
        for ax, Nv in zip(range(3), (Nx, Ny, Nz)):
            h = 1e-7
            gp, gm_ = g.copy(), g.copy()
            gp[ax] += h
            gm_[ax] -= h
            da = (oracle.aniso3(gp, eps, geps)[0] - oracle.aniso3(gm_, eps, geps)[0]) / (2 * h)
            assert math.isclose(Nv, m * m * a * da, rel_tol=1e-6, abs_tol=1e-12)


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
