"""A literal, per-node twin of one coupled lattice Boltzmann step, written
from the paper's equations and this library's readings of them, for the
brute-force check of the oracle on tiny lattices.

TEST INFRASTRUCTURE.  It imports nothing from ``oracle/`` and nothing from
the library: constants, lattices, moment matrices, equilibria and the step
are written here again, in a different form.  Where the oracle transforms to
moment space, relaxes and transforms back (m* = m - S(m - m_eq) + (I - S/2)MG
+ M F_d), this twin relaxes in population space with the dense collision
matrix Lambda = M^-1 S M of Appendix B, M^-1 taken by numerical inversion:

    f* = f - Lambda (f - f_eq) + (I - Lambda / 2) G + F_d.

Every equation is evaluated one site at a time and one lattice at a time, in
plain Python loops over the sites: slow, and small enough to read against the
paper.  Periodic lattices only.

The model (Section 2, Appendix B) with the readings it needs:
  NS      D2Q9, pressure-based equilibrium, drag v = (1 - h(psi)) v*,
          surface tension, buoyancy about the mean density, mass-flux force
  CAC     D2Q9, h_eq = w phi (1 + c.v / cs2), anti-diffusion and d(phi v)/dt
          through (I - Lambda / 2)
  psi     D2Q5, time stretch t + a_s^2 dt by interpolation in time, flux rate
          from W0^2 a_s^2 / tau0, source Q / tau0 + 1/2 dQ/dt / tau0
  solute  D2Q5, C conserved and diffused with D_C = 2 D q / A, the rest of
          (1-k) D q grad U, the flow and the antitrapping and gas fluxes in
          the equilibrium flux
  heat    (thermal mode) D2Q5 for H = c_p theta - c_p^s h(psi), F(U) and the
          grad F source in the psi equation
"""
import math

import numpy as np

# D2Q9 velocities in the order rest, +x, +y, -x, -y, (+,+), (-,+), (-,-), (+,-)
C9 = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
W9 = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4
C5 = C9[:5]
W5 = [1 / 3] + [1 / 6] * 4          # D2Q5 weights (the paper gives none)
CS2 = 1 / 3


def _m9():
    """Lallemand-Luo rows: rho, e, eps, jx, qx, jy, qy, pxx, pxy."""
    rows = []
    for cx, cy in C9:
        c2 = cx * cx + cy * cy
        rows.append([1, -4 + 3 * c2, 4 - 21 * c2 / 2 + 9 * c2 * c2 / 2, cx, (-5 + 3 * c2) * cx,
                     cy, (-5 + 3 * c2) * cy, cx * cx - cy * cy, cx * cy])
    return np.array(rows, dtype=float).T


def _m5():
    """Rows: zeroth, jx, jy, 5|c|^2 - 4, cx^2 - cy^2."""
    rows = []
    for cx, cy in C5:
        c2 = cx * cx + cy * cy
        rows.append([1, cx, cy, 5 * c2 - 4, cx * cx - cy * cy])
    return np.array(rows, dtype=float).T


M9, M5 = _m9(), _m5()
M9INV, M5INV = np.linalg.inv(M9), np.linalg.inv(M5)


def collide(f, feq, S, G, Fd=None):
    """f* = f - Lambda (f - f_eq) + (I - Lambda/2) G + F_d, Lambda = M^-1 S M."""
    q = len(f)
    M, Minv = (M9, M9INV) if q == 9 else (M5, M5INV)
    Lam = Minv @ np.diag(S) @ M
    out = f - Lam @ (f - feq) + (np.eye(q) - 0.5 * Lam) @ G
    if Fd is not None:
        out = out + Fd
    return out


def feq_ns(p, rho, vx, vy):
    v2 = vx * vx + vy * vy
    out = np.empty(9)
    for i, (cx, cy) in enumerate(C9):
        cu = cx * vx + cy * vy
        out[i] = W9[i] * p / CS2 + rho * W9[i] * (cu / CS2 + cu * cu / (2 * CS2 * CS2)
                                                  - v2 / (2 * CS2))
    out[0] -= p / CS2
    return out


def heq_cac(phi, vx, vy):
    return np.array([W9[i] * phi * (1 + (cx * vx + cy * vy) / CS2)
                     for i, (cx, cy) in enumerate(C9)])


def flux_eq5(X, jx, jy):
    """w_i X + w_i c_i . j / cs2 on D2Q5."""
    return np.array([W5[i] * X + W5[i] * (cx * jx + cy * jy) / CS2
                     for i, (cx, cy) in enumerate(C5)])


def heat_eq5(rhoH, theta, jx, jy):
    out = np.array([W5[i] * theta + W5[i] * (cx * jx + cy * jy) / CS2
                    for i, (cx, cy) in enumerate(C5)])
    out[0] = rhoH + (W5[0] - 1) * theta
    return out


class Twin:
    """State of a periodic nx x ny lattice: per site f[9], h[9], g_pre[5],
    g_post[5], r = 1/a_s^2, s[5], lagged phi, C, vx, vy, Q; thermal mode adds
    e[5] and the lagged H.  Arrays are [y][x]."""

    def __init__(self, nx, ny, par):
        self.nx, self.ny, self.p = nx, ny, dict(par)
        p = self.p
        self.thermal = bool(p.get("thermal", 0))
        self.lam = p["D"] * p["tau0"] / ((47 / 75) * p["W0"] ** 2)          # Appendix A
        self.Mc = 1 - (1 - p["k"]) * p["Omega"]                             # Eq. eq-Tsys
        self.theta_sys = -self.Mc * p["Omega"] / (1 - (1 - p["k"]) * p["Omega"])
        self.kappa = math.sqrt(2 * p["beta_phi"]) / p["W_phi"]
        self.s_nu = 1 / (3 * p["nu"] + 0.5)
        self.s_q = 8 * (2 - self.s_nu) / (8 - self.s_nu)
        self.s_phi = 1 / (3 * p["M_phi"] + 0.5)
        self.kT = p.get("Le", 1.0) * p["D"] * p["rho_l"] * p.get("cp", 1.0)
        self.s_T = 1 / (self.kT / CS2 + 0.5)

    # -- pointwise model functions -----------------------------------------
    def U_of(self, C, psi):
        k = self.p["k"]
        return (2 * C / (1 + k - (1 - k) * psi) - 1) / (1 - k)

    def Q_of(self, phi, psi, U, theta):
        p = self.p
        return (4 * p["beta_psi"] * psi * (1 - psi * psi)
                - 2 * p["beta_inter"] * (1 - phi) ** 2 * (1 + psi)
                - self.lam * (1 - psi * psi) ** 2 * (theta + self.Mc * U))

    def F_of(self, U):
        return 1 / self.p["Le"] + self.Mc * (1 + (1 - self.p["k"]) * U)

    def rho_of(self, phi):
        return self.p["rho_g"] + phi * (self.p["rho_l"] - self.p["rho_g"])

    # -- initial state (equilibria at the given fields) ----------------------
    def init(self, phi, psi, C, vx, vy, pr, angle, theta=None):
        p = self.p
        ny, nx = self.ny, self.nx
        self.angle = np.array(angle, dtype=float)
        self.f = np.zeros((9, ny, nx)); self.h = np.zeros((9, ny, nx))
        self.gpre = np.zeros((5, ny, nx)); self.gpost = np.zeros((5, ny, nx))
        self.r = np.ones((ny, nx)); self.s = np.zeros((5, ny, nx))
        self.e = np.zeros((5, ny, nx)); self.Ho = np.zeros((ny, nx))
        self.phio = np.array(phi, dtype=float); self.Co = np.array(C, dtype=float)
        self.vxo = np.array(vx, dtype=float); self.vyo = np.array(vy, dtype=float)
        self.Qo = np.zeros((ny, nx))
        for y in range(ny):
            for x in range(nx):
                ph, ps, c = phi[y][x], psi[y][x], C[y][x]
                ux, uy = vx[y][x], vy[y][x]
                rho = self.rho_of(ph)
                self.f[:, y, x] = feq_ns(pr[y][x], rho, ux, uy)
                self.h[:, y, x] = heq_cac(ph, ux, uy)
                for i in range(5):
                    self.gpre[i, y, x] = self.gpost[i, y, x] = W5[i] * ps
                self.s[:, y, x] = flux_eq5(c, c * ux, c * uy)
                U = self.U_of(c, ps)
                if self.thermal:
                    th = theta[y][x]
                    H = p["cp"] * (th - p["latent"] * 0.5 * (1 + ps))
                    self.e[:, y, x] = heat_eq5(rho * H, th, rho * H * ux, rho * H * uy)
                    self.Ho[y, x] = H
                    self.Qo[y, x] = self.Q_of(ph, ps, U, th) / self.F_of(U)
                else:
                    self.Qo[y, x] = self.Q_of(ph, ps, U, self.theta_sys)
        self.rho_bar = self.rho_of(float(np.mean(phi)))

    # -- one step ------------------------------------------------------------
    def _grad(self, X, x, y):
        gx = gy = 0.0
        for i in range(1, 9):
            cx, cy = C9[i]
            v = X[(y + cy) % self.ny, (x + cx) % self.nx]
            gx += W9[i] * cx * v
            gy += W9[i] * cy * v
        return gx / CS2, gy / CS2

    def _lap(self, X, x, y):
        a = 0.0
        for i in range(1, 9):
            cx, cy = C9[i]
            a += W9[i] * (X[(y + cy) % self.ny, (x + cx) % self.nx] - X[y, x])
        return 2 * a / CS2

    def step(self):
        p = self.p
        nx, ny = self.nx, self.ny
        drho = p["rho_l"] - p["rho_g"]
        eps, k = p["eps_s"], p["k"]
        # streaming (pull) and zeroth moments
        fS = np.zeros_like(self.f); hS = np.zeros_like(self.h)
        gS = np.zeros_like(self.gpre); sS = np.zeros_like(self.s); eS = np.zeros_like(self.e)
        for y in range(ny):
            for x in range(nx):
                for i, (cx, cy) in enumerate(C9):
                    sy, sx = (y - cy) % ny, (x - cx) % nx
                    fS[i, y, x] = self.f[i, sy, sx]
                    hS[i, y, x] = self.h[i, sy, sx]
                    if i < 5:
                        sS[i, y, x] = self.s[i, sy, sx]
                        eS[i, y, x] = self.e[i, sy, sx]
                        # t + a_s^2 dt: the population moves the fraction
                        # 1/a_s^2 (taken where it was emitted) of the way
                        gS[i, y, x] = (self.gpre[i, y, x] + self.r[sy, sx]
                                       * (self.gpost[i, sy, sx] - self.gpre[i, y, x]))
        phi = hS.sum(axis=0)
        psi = gS.sum(axis=0)
        C = sS.sum(axis=0)
        psio = self.gpre.sum(axis=0)
        U = self.U_of(C, psi)
        nf = np.zeros_like(self.f); nh = np.zeros_like(self.h)
        ngpost = np.zeros_like(self.gpost); nr = np.zeros_like(self.r)
        ns = np.zeros_like(self.s); ne = np.zeros_like(self.e)
        nphio = np.zeros_like(phi); nCo = np.zeros_like(phi)
        nvxo = np.zeros_like(phi); nvyo = np.zeros_like(phi); nQo = np.zeros_like(phi)
        nHo = np.zeros_like(phi)
        fields = {nm: np.zeros_like(phi) for nm in ("phi", "psi", "C", "U", "p", "vx", "vy",
                                                     "mu", "theta")}
        for y in range(ny):
            for x in range(nx):
                ph, ps, c = phi[y, x], psi[y, x], C[y, x]
                pho, co = self.phio[y, x], self.Co[y, x]
                vxo, vyo = self.vxo[y, x], self.vyo[y, x]
                gpx, gpy = self._grad(phi, x, y)
                lphi = self._lap(phi, x, y)
                gsx, gsy = self._grad(psi, x, y)
                dvxx, dvxy = self._grad(self.vxo, x, y)
                dvyx, dvyy = self._grad(self.vyo, x, y)
                # gas-liquid interface
                rho = self.rho_of(ph)
                grx, gry = drho * gpx, drho * gpy
                gnorm = math.sqrt(gpx * gpx + gpy * gpy + p["grad_eps"] ** 2)
                nfx, nfy = gpx / gnorm, gpy / gnorm
                mu = (2 * p["beta_phi"] * ph * (1 - ph) * (1 - 2 * ph)
                      - 2 * p["beta_inter"] * (1 - ph) * (1 + ps) ** 2
                      - p["W_phi"] ** 2 * lphi)
                cs = 6 * p["sigma"] / (p["W_phi"] * math.sqrt(2 * p["beta_phi"]))
                Fsx, Fsy = cs * mu * gpx, cs * mu * gpy
                Fbx, Fby = 0.0, -(rho - self.rho_bar) * p["g"]
                sharp = self.kappa * ph * (1 - ph)
                Dx = p["M_phi"] * (gpx - sharp * nfx)
                Dy = p["M_phi"] * (gpy - sharp * nfy)
                divD = (ph - pho) + vxo * gpx + vyo * gpy
                Fmx = drho * (divD * vxo + Dx * dvxx + Dy * dvxy)
                Fmy = drho * (divD * vyo + Dx * dvyx + Dy * dvyy)
                f = fS[:, y, x]
                jx = sum(C9[i][0] * f[i] for i in range(9))
                jy = sum(C9[i][1] * f[i] for i in range(9))
                Fpx, Fpy = Fsx + Fbx + Fmx, Fsy + Fby + Fmy
                vsx, vsy = (jx + 0.5 * Fpx) / rho, (jy + 0.5 * Fpy) / rho
                chi = 0.5 * (1 + ps)
                vx, vy = (1 - chi) * vsx, (1 - chi) * vsy
                Fx, Fy = Fpx - 2 * chi * rho * vsx, Fpy - 2 * chi * rho * vsy
                pr = CS2 / (1 - W9[0]) * (sum(f[1:]) + 0.5 * (vx * grx + vy * gry)
                                          - W9[0] * rho * (vx * vx + vy * vy) / (2 * CS2))
                # dendrite geometry in the grain frame
                th = self.angle[y, x]
                ct, sn = math.cos(th), math.sin(th)
                gnm = math.sqrt(gsx * gsx + gsy * gsy + p["grad_eps"] ** 2)
                nx_, ny_ = -gsx / gnm, -gsy / gnm
                nxr, nyr = ct * nx_ + sn * ny_, -sn * nx_ + ct * ny_
                n2 = nxr * nxr + nyr * nyr
                s4 = nxr ** 4 + nyr ** 4
                a_s = 1 + eps * (4 * s4 - 3 * n2 * n2)
                iso = s4 + 0.75 * n2 * (1 - n2)
                Nxr = -16 * eps * a_s * gnm * nxr * (nxr * nxr - iso)
                Nyr = -16 * eps * a_s * gnm * nyr * (nyr * nyr - iso)
                Nx, Ny = ct * Nxr - sn * Nyr, sn * Nxr + ct * Nyr
                u = U[y, x]
                theta = self.theta_sys
                if self.thermal:
                    rhoH = eS[:, y, x].sum()
                    theta = rhoH / (rho * p["cp"]) + p["latent"] * 0.5 * (1 + ps)
                Q = self.Q_of(ph, ps, u, theta)
                at = (-(1 / (2 * math.sqrt(2))) * p["W0"] * a_s * (1 + (1 - k) * u) * (ps - psio[y, x])
                      / math.sqrt(gsx * gsx + gsy * gsy + p["grad_eps_at"] ** 2))
                Jatx, Jaty = at * gsx, at * gsy
                qf = 0.5 * (1 - ps)
                jv = p["D"] * qf * c * self.kappa * (1 - ph)
                Jx, Jy = jv * nfx, jv * nfy
                # NS
                G = np.array([W9[i] * ((cx * Fx + cy * Fy) / CS2
                                       + (cx * vx + cy * vy) * (cx * grx + cy * gry) / CS2)
                              for i, (cx, cy) in enumerate(C9)])
                S = [1, p["s_e"], p["s_eps"], 1, self.s_q, 1, self.s_q, self.s_nu, self.s_nu]
                nf[:, y, x] = collide(f, feq_ns(pr, rho, vx, vy), S, G)
                # CAC
                G1x = (ph * vx - pho * vxo) + CS2 * sharp * nfx
                G1y = (ph * vy - pho * vyo) + CS2 * sharp * nfy
                G = np.array([W9[i] * (cx * G1x + cy * G1y) / CS2 for i, (cx, cy) in enumerate(C9)])
                S = [1, 1, 1, self.s_phi, 1, self.s_phi, 1, 1, 1]
                nh[:, y, x] = collide(hS[:, y, x], heq_cac(ph, vx, vy), S, G)
                # psi
                Fu, Qeff = 1.0, Q
                if self.thermal:
                    Fu = self.F_of(u)
                    gux, guy = self._grad(U, x, y)
                    dFx, dFy = self.Mc * (1 - k) * gux, self.Mc * (1 - k) * guy
                    Qeff = Q / Fu + p["W0"] ** 2 / Fu ** 2 * (dFx * (a_s * a_s * gsx + Nx)
                                                             + dFy * (a_s * a_s * gsy + Ny))
                G = np.array([-W5[i] * (cx * Nx + cy * Ny) / (a_s * a_s)
                              for i, (cx, cy) in enumerate(C5)])
                Fd = np.array([W5[i] * Qeff / p["tau0"] + 0.5 * W5[i] * (Qeff - self.Qo[y, x])
                               / p["tau0"] for i in range(5)])
                s1 = 1 / (p["W0"] ** 2 * a_s * a_s / (p["tau0"] * Fu * CS2) + 0.5)
                ngpost[:, y, x] = collide(gS[:, y, x], np.array([W5[i] * ps for i in range(5)]),
                                          [1, s1, s1, 1, 1], G, Fd)
                nr[y, x] = 1 / (a_s * a_s)
                # solute
                A = 1 + k - (1 - k) * ps
                DC = 2 * p["D"] * qf / A
                E = 2 * (1 - k) * p["D"] * qf * c / (A * A)
                jex = c * vx - E * gsx + (1 - k) * (Jatx + Jx)
                jey = c * vy - E * gsy + (1 - k) * (Jaty + Jy)
                Gx, Gy = c * vx - co * vxo, c * vy - co * vyo
                G = np.array([W5[i] * (cx * Gx + cy * Gy) / CS2 for i, (cx, cy) in enumerate(C5)])
                sc = 1 / (DC / CS2 + 0.5)
                ns[:, y, x] = collide(sS[:, y, x], flux_eq5(c, jex, jey), [1, sc, sc, 1, 1], G)
                # heat
                if self.thermal:
                    rho_o = self.rho_of(pho)
                    hx, hy = rhoH * vx, rhoH * vy
                    Gx = hx - rho_o * self.Ho[y, x] * vxo
                    Gy = hy - rho_o * self.Ho[y, x] * vyo
                    G = np.array([W5[i] * (cx * Gx + cy * Gy) / CS2
                                  for i, (cx, cy) in enumerate(C5)])
                    ne[:, y, x] = collide(eS[:, y, x], heat_eq5(rhoH, theta, hx, hy),
                                          [1, self.s_T, self.s_T, 1, 1], G)
                    nHo[y, x] = rhoH / rho
                nphio[y, x], nCo[y, x] = ph, c
                nvxo[y, x], nvyo[y, x], nQo[y, x] = vx, vy, Qeff
                for nm, v in (("phi", ph), ("psi", ps), ("C", c), ("U", u), ("p", pr),
                              ("vx", vx), ("vy", vy), ("mu", mu), ("theta", theta)):
                    fields[nm][y, x] = v
        self.f, self.h, self.gpre, self.gpost, self.r, self.s = nf, nh, gS, ngpost, nr, ns
        self.phio, self.Co, self.vxo, self.vyo, self.Qo = nphio, nCo, nvxo, nvyo, nQo
        if self.thermal:
            self.e, self.Ho = ne, nHo
        self.fields = fields

    def state(self):
        """Planes in the order f[9], h[9], g_pre[5], g_post[5], r, s[5],
        phi_o, C_o, vx_o, vy_o, Q (+ e[5], H_o in thermal mode)."""
        planes = [*self.f, *self.h, *self.gpre, *self.gpost, self.r, *self.s,
                  self.phio, self.Co, self.vxo, self.vyo, self.Qo]
        if self.thermal:
            planes += [*self.e, self.Ho]
        return np.array(planes)
