"""Mistakes planted in copies of the oracle, each of which a pin must catch.

The oracle's own builds are never touched: oracle.mutant() copies a source,
applies one text edit and compiles the copy into a temporary directory.  Each
case names the passage the edit breaks and the pin measurement that catches
it (tests/pin_cases.py).  A pin that a plausible mistake survives is not a
pin, so these cases keep the pins honest as the oracle changes.
"""
import pytest

import oracle
import pin_cases
import test_oracle_boundaries as bnd
import test_oracle_3d as t3d
import test_oracle_3f as t3f
import test_oracle_thermal as th
from test_oracle_twin import TOL as TWIN_TOL
from test_oracle_twin import twin_error

# 2-D oracle (pf_oracle.c)
STRETCH_2D = "st->gS[i][idx] = gold + (gsrc - gold) * st->rr[src];"
RATE_2D = "st->nrr[idx] = 1.0 / as2;"
FM_2D = ("const real_t Fmx = (rl - rg) * (divD * vxo + Dx * dvxx + Dy * dvxy);\n"
         "      const real_t Fmy = (rl - rg) * (divD * vyo + Dx * dvyx + Dy * dvyy);")
# 3-D oracles (pf_oracle3d.c): the melt step and the two-phase step each
# carry their own stretch, told apart by the lines around them
STRETCH_3D = ("/* far field: anti-bounce-back -f*_opp + 2 w_i X_far (psi -1, C 1) */\n"
              "          const real gsrc = mode == 2 ? -st->gpost[q][src] + 2.0 * W7[i] * (-1.0)"
              " : st->gpost[q][src];\n"
              "          st->gS[i][id] = gold + (gsrc - gold) * st->rr[src];")
RATE_3D = ("(tau0 * CS2_7) + 0.5);\n"
           "          const real S[7] = {1, s1, s1, s1, 1, 1, 1};\n"
           "          collide7(gg, geq, S, G, Fd, out);\n"
           "          for (int i = 0; i < 7; ++i) { st->ngpost[i][id] = out[i];"
           " st->ngpre[i][id] = gg[i]; }\n"
           "          st->nrr[id] = 1.0 / as2;")
STRETCH_3F = ("          if (refl) src = idx3f(st, x, y, z);\n"
              "          const real gold = st->gpre[i][id];\n"
              "          const real gsrc = mode == 2 ? -st->gpost[q][src] + 2.0 * W7[i] * (-1.0)"
              " : st->gpost[q][src];\n"
              "          st->gS[i][id] = gold + (gsrc - gold) * st->rr[src];")
FM_3F = ("const double Fm = (rl - rg) * (divD * vo[a] + Dm[0] * dv[a][0] + Dm[1] * dv[a][1]"
         " + Dm[2] * dv[a][2]);")

NEE_2D = "st->fS[i][idx] = st->f[q][src] + st->par[P_RHO_L] * sb - rho_f * sf;"

CASES = {
    # Appendix B time stretch t + a_s^2 dt (Eq. eq-AnACE: tau0 a_s^2 d psi/dt)
    "2d: no time stretch": ("pf_oracle.c", [(STRETCH_2D, STRETCH_2D.replace(
        " * st->rr[src]", " * 1.0"))], "stretch", "2d"),
    "2d: stretch a_s instead of a_s^2": ("pf_oracle.c", [(RATE_2D, RATE_2D.replace(
        "/ as2", "/ as"))], "stretch", "2d"),
    "3d melt: no time stretch": ("pf_oracle3d.c", [(STRETCH_3D, STRETCH_3D.replace(
        " * st->rr[src]", " * 1.0"))], "stretch", "3d"),
    "3d melt: stretch a_s instead of a_s^2": ("pf_oracle3d.c", [(RATE_3D, RATE_3D.replace(
        "/ as2;", "/ sqrt(as2);"))], "stretch", "3d"),
    "3d two-phase: no time stretch": ("pf_oracle3d.c", [(STRETCH_3F, STRETCH_3F.replace(
        " * st->rr[src]", " * 1.0"))], "stretch", "3f"),
    # Section 2.2 mass-consistent momentum flux m = rho v - D (rho_l - rho_g)
    "2d: no mass-flux correction": ("pf_oracle.c", [(FM_2D, FM_2D.replace(
        "(rl - rg) *", "0.0 *"))], "mass_flux", "2d"),
    "2d: mass-flux correction without (div D) v": ("pf_oracle.c", [(FM_2D, FM_2D.replace(
        "(divD * vxo", "(0.0 * vxo").replace("(divD * vyo", "(0.0 * vyo"))], "mass_flux", "2d"),
    "2d: mass-flux correction of the wrong sign": ("pf_oracle.c", [(FM_2D, FM_2D.replace(
        "= (rl - rg) *", "= -(rl - rg) *"))], "mass_flux", "2d"),
    "3d two-phase: no mass-flux correction": ("pf_oracle3d.c", [(FM_3F, FM_3F.replace(
        "(rl - rg) *", "0.0 *"))], "mass_flux", "3f"),
    # Section 3: Dirichlet velocity by non-equilibrium extrapolation
    "2d: extrapolation inlet without the equilibrium difference": ("pf_oracle.c", [(
        NEE_2D, "st->fS[i][idx] = st->f[q][src];")], "couette", "2d"),
    # reading R31: symmetric, wall and far-field sides
    "2d: symmetric side keeps the ghost's normal velocity": ("pf_oracle.c", [(
        "if (t == BC_SYMMETRIC) return normal ? -v : v;", "if (t == BC_SYMMETRIC) return v;")],
        "mirror", "2d"),
    "2d: wall bounce-back into the same direction": ("pf_oracle.c", [(
        "if (bounce) { *src = y * nx + x; *q = OPP[i]; return bounce; }",
        "if (bounce) { *src = y * nx + x; *q = i; return bounce; }")], "walls", "2d"),
    "2d: far-field anti-bounce-back without its sign": ("pf_oracle.c", [(
        "st->sS[i][idx] = (mode == 2 || mode == 3) ? -st->s[q][src] + 2.0 * W5[i] * C_FAR",
        "st->sS[i][idx] = (mode == 2 || mode == 3) ? st->s[q][src] + 2.0 * W5[i] * C_FAR")],
        "farfield", "2d"),
    # Appendix B temperature coupling and the rewritten dendrite equation
    "thermal: grad F source of the wrong sign": ("pf_oracle.c", [(
        "Qeff = Q / Fu + par[P_W0] * par[P_W0] / (Fu * Fu) * (dFx * Xx + dFy * Xy);",
        "Qeff = Q / Fu - par[P_W0] * par[P_W0] / (Fu * Fu) * (dFx * Xx + dFy * Xy);")],
        "gradF", "2d"),
    "thermal: latent heat of the wrong sign": ("pf_oracle.c", [(
        "theta = rhoH / (rho * par[P_CP]) + par[P_LATENT] * 0.5 * (1.0 + psi);",
        "theta = rhoH / (rho * par[P_CP]) - par[P_LATENT] * 0.5 * (1.0 + psi);")],
        "latent", "2d"),
    "thermal: c_p left out of the conductivity": ("pf_oracle.c", [(
        "d.kT = p[P_LE] * p[P_D] * p[P_RHO_L] * p[P_CP];",
        "d.kT = p[P_LE] * p[P_D] * p[P_RHO_L];")], "heat", "2d"),
    # Section 2.2 CAC sharpening flux M kappa phi (1 - phi) n
    "2d: sharpening coefficient kappa 1 % too large": ("pf_oracle.c", [(
        "const real_t aphi = d.kappa * phi * (1.0 - phi);",
        "const real_t aphi = 1.01 * d.kappa * phi * (1.0 - phi);")], "flat", "2d"),
    "2d: sharpening flux of the wrong sign": ("pf_oracle.c", [(
        "const real_t aphi = d.kappa * phi * (1.0 - phi);",
        "const real_t aphi = -d.kappa * phi * (1.0 - phi);")], "flat", "2d"),
    "3d two-phase: sharpening coefficient kappa 1 % too large": ("pf_oracle3d.c", [(
        "const double aphi = kappa * phi * (1.0 - phi);",
        "const double aphi = 1.01 * kappa * phi * (1.0 - phi);")], "flat", "3f"),
    "3d two-phase: sharpening flux of the wrong sign": ("pf_oracle3d.c", [(
        "const double aphi = kappa * phi * (1.0 - phi);",
        "const double aphi = -kappa * phi * (1.0 - phi);")], "flat", "3f"),
    # reading R33: the 3-D anisotropy (sums over three axes) and grain orientations
    "3d melt: fourth powers of the normal summed over two axes": ("pf_oracle3d.c", [(
        "s4 += n[a] * n[a] * n[a] * n[a];", "s4 += (a < 2) * n[a] * n[a] * n[a] * n[a];")],
        "aniso", "3d"),
    "3d melt: orientation of the farthest seed": ("pf_oracle3d.c", [(
        "if (s2 == 0 || r2 < bd) { bd = r2; best = s2; }",
        "if (s2 == 0 || r2 > bd) { bd = r2; best = s2; }")], "nearest", "3d"),
    # reading R33 with R28-R30: the 3-D temperature lattice
    "3d melt: latent heat counted twice in theta": ("pf_oracle3d.c", [(
        "theta = rhoH / (p[Q_RHO_L] * p[Q_CP]) + p[Q_LATENT] * 0.5 * (1.0 + psi);",
        "theta = rhoH / (p[Q_RHO_L] * p[Q_CP]) + p[Q_LATENT] * 1.0 * (1.0 + psi);")],
        "latent3d", "3d"),
    "3d melt: Le left out of the conductivity": ("pf_oracle3d.c", [(
        "const double kT = p[Q_LE] * p[Q_D] * p[Q_RHO_L] * p[Q_CP];",
        "const double kT = p[Q_D] * p[Q_RHO_L] * p[Q_CP];")], "heat3d", "3d"),
    # reading R34: the 3-D two-phase step's forces, couplings and lattice
    "3d two-phase: surface tension of the wrong sign": ("pf_oracle3d.c", [(
        "const double Fs = fs_coef * mu * gp[a];",
        "const double Fs = -fs_coef * mu * gp[a];")], "laplace", "3f"),
    "3d two-phase: Laplacian over two axes": ("pf_oracle3d.c", [(
        "    a += W19[i] * (field3f(st, X, x + C19[i][0], y + C19[i][1], z + C19[i][2], kind) - c);",
        "    a += (C19[i][2] == 0) * W19[i] * (field3f(st, X, x + C19[i][0], y + C19[i][1],"
        " z + C19[i][2], kind) - c);")], "laplace", "3f"),
    "3d two-phase: no CAC advection": ("pf_oracle3d.c", [(
        "heq19(phi, v, heq);", "heq19(phi, (const double[3]){0.0, 0.0, 0.0}, heq);")],
        "advection", "3f"),
    "3d two-phase: no solute advection": ("pf_oracle3d.c", [(
        "Jq[a] = C * v[a] - E * gs[a]", "Jq[a] = 0.0 * v[a] - E * gs[a]")], "advection", "3f"),
    "3d two-phase: gravity of the wrong sign": ("pf_oracle3d.c", [(
        "const double Fb = a == 1 ? -(rho - st->rho_bar) * p[F3_G] : 0.0;",
        "const double Fb = a == 1 ? (rho - st->rho_bar) * p[F3_G] : 0.0;")], "bubble", "3f"),
    "3d two-phase: no drag in the solid": ("pf_oracle3d.c", [(
        "v[a] = (1.0 - chi) * vs[a];", "v[a] = vs[a];")], "solid", "3f"),
    "3d two-phase: wrong D3Q19 edge weight": ("pf_oracle3d.c", [(
        "W19[j] = c2 == 0 ? 1.0 / 3.0 : (c2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);",
        "W19[j] = c2 == 0 ? 1.0 / 3.0 : (c2 == 1 ? 1.0 / 18.0 : 1.0 / 35.0);")], "lattice", "3f"),
    # mistakes in how the step is composed, caught by the per-node twin
    "2d: stretch factor taken at the destination": ("pf_oracle.c", [(STRETCH_2D, STRETCH_2D.replace(
        "st->rr[src]", "st->rr[idx]"))], "twin", "2d"),
    "2d: mass-flux correction without (D . grad) v": ("pf_oracle.c", [(FM_2D, FM_2D.replace(
        " + Dx * dvxx + Dy * dvxy", "").replace(" + Dx * dvyx + Dy * dvyy", ""))], "twin", "2d"),
    "2d: previous psi from the streamed populations": ("pf_oracle.c", [(
        "psio += gold;", "psio += st->gS[i][idx];")], "twin", "2d"),
    "2d: drag force on v instead of v*": ("pf_oracle.c", [(
        "const real_t Fx = Fpx - 2.0 * chi * rho * vsx,",
        "const real_t Fx = Fpx - 2.0 * chi * rho * vx,")], "twin", "2d"),
    "2d: CAC time derivative with the current velocity twice": ("pf_oracle.c", [(
        "const real_t G1x = (phi * vx - phio * vxo)",
        "const real_t G1x = (phi * vx - phio * vx)")], "twin", "2d"),
}


@pytest.fixture(scope="module")
def mutant_dir(tmp_path_factory):
    return str(tmp_path_factory.mktemp("oracle_mutants"))


@pytest.mark.parametrize("case", sorted(CASES))
def test_planted_mistake_fails_its_pin(case, mutant_dir):
    source, edits, pin, kind = CASES[case]
    lib = oracle.mutant(source, edits, mutant_dir)
    if pin == "stretch":
        errs, _ = pin_cases.stretch_errors(kind, lib)
        assert not pin_cases.stretch_pin_holds(errs), errs
    elif pin == "gradF":
        assert not th.gradF_pin_holds(th.gradF_errors(lib)), case
    elif pin == "latent":
        ratio, dpsi, _ = th.latent_ratio(1.0, lib)
        assert not abs(ratio - 1.0) < 1e-9, (case, ratio)
    elif pin == "heat":
        alphas = th.heat_alpha(1.0, 10.0, lib)
        assert not all(abs(a / 0.1 - 1.0) < 1e-4 for a in alphas), (case, alphas)
    elif pin == "couette":
        assert not pin_cases.nee_couette_holds(lib), case
    elif pin == "flat":
        m = pin_cases.flat_layer(lib) if kind == "2d" else pin_cases.flat_layer_3f(lib)
        assert not pin_cases.flat_layer_holds(m), (case, m)
    elif pin == "twin":
        err = twin_error(lib)
        assert not err <= TWIN_TOL, err
    elif pin == "laplace":
        assert not t3f.laplace_cylinder_holds(lib), case
    elif pin == "advection":
        m = t3f.gas_layer_advection(lib)
        assert not t3f.gas_layer_advection_holds(m), (case, m)
    elif pin == "bubble":
        assert not t3f.bubble_rise_holds(lib), case
    elif pin == "solid":
        assert not t3f.solid_velocity_holds(lib), case
    elif pin == "lattice":
        assert not t3f.lattice_isotropy_holds(lib), case
    elif pin == "mirror":
        assert not bnd.mirror_equivalence_holds(0, False, lib), case
    elif pin == "walls":
        assert not bnd.shear_wave_between_walls_holds(lib), case
    elif pin == "farfield":
        assert not bnd.far_field_series_holds(lib), case
    elif pin == "aniso":
        assert not t3d.anisotropy_closed_forms_hold(lib), case
    elif pin == "nearest":
        assert not t3d.orientation_nearest_holds(lib), case
    elif pin == "latent3d":
        assert not t3d.enthalpy_latent_holds(lib), case
    elif pin == "heat3d":
        assert not t3d.heat_variance_holds(lib), case
    else:
        dev, _ = pin_cases.mass_flux_deviation(kind, lib)
        assert not dev < pin_cases.MASS_FLUX_TOL, dev


def test_the_unmodified_copy_passes():
    """The copy-and-compile route itself changes nothing: a copy with an
    edit that leaves the text as it is passes the pins (of the 2-D oracle, and
    the quick ones of the 3-D two-phase oracle)."""
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        lib = oracle.mutant("pf_oracle.c", [(STRETCH_2D, STRETCH_2D)], d)
        errs, _ = pin_cases.stretch_errors("2d", lib)
        assert pin_cases.stretch_pin_holds(errs)
        dev, _ = pin_cases.mass_flux_deviation("2d", lib)
        assert dev < pin_cases.MASS_FLUX_TOL
        assert twin_error(lib) <= TWIN_TOL
        assert pin_cases.flat_layer_holds(pin_cases.flat_layer(lib))
        lib3 = oracle.mutant("pf_oracle3d.c", [(STRETCH_3F, STRETCH_3F)], d)
        assert t3f.lattice_isotropy_holds(lib3)
        assert t3f.gas_layer_advection_holds(t3f.gas_layer_advection(lib3))
        assert t3f.solid_velocity_holds(lib3)
