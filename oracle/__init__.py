"""Plain FP64 CPU oracle of the coupled gas-liquid-dendrite LB step.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The library path
(``paper_2407_01651_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``pf_oracle.c`` (one site at a time, dense moment
matrices, two passes per step).  This module only compiles it with gcc and
marshals arrays through ctypes.  Two builds of the same source exist:
``liboracle_d.so`` (double) and ``liboracle_z.so`` (double complex, the
complex-step derivative with respect to one parameter).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")

# Order of the oracle's parameter vector (enum in pf_oracle.c).
PARAM_NAMES = (
    "rho_l", "rho_g", "nu", "sigma", "W_phi", "M_phi", "beta_phi", "beta_psi",
    "beta_inter", "W0", "tau0", "eps_s", "k", "D", "Omega", "g", "grad_eps",
    "s_e", "s_eps", "grad_eps_at", "thermal", "Le", "latent", "theta0", "cp", "vin_x", "vin_y",
)
# Defaults of the temperature-coupling parameters: isothermal closure
# (Eq. eq-Tsys), so a parameter dict without them runs the isothermal model.
THERMAL_DEFAULTS = dict(thermal=0.0, Le=1.0, latent=1.0, theta0=-0.55, cp=10.0, vin_x=0.0,
                        vin_y=0.0)
# Field order of or_get_fields.
FIELDS = ("phi", "psi", "C", "U", "p", "vx", "vy", "mu", "theta")
N_STATE_PLANES = 39          # isothermal; thermal mode adds e[5] and H_o

_lock = threading.Lock()
_libs: dict[str, ctypes.CDLL] = {}


_SRC3 = os.path.join(_HERE, "pf_oracle3d.c")


def build(force: bool = False) -> None:
    """Compile both oracle builds and the 3-D oracle with gcc: -O3, no
    fast-math and no FMA contraction (IEEE round-to-nearest in the written
    order), OpenMP over lattice rows.  No -march=native: the same source must
    build, and give the same results, on x86-64 and Arm hosts."""
    os.makedirs(_BUILD, exist_ok=True)
    for tag, extra, src in (("d", [], _SRC), ("z", ["-DPF_ORACLE_Z"], _SRC), ("3d", [], _SRC3)):
        out = os.path.join(_BUILD, f"liboracle_{tag}.so")
        if (not force and os.path.exists(out)
                and os.path.getmtime(out) >= os.path.getmtime(src)):
            continue
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c11", "-O3", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", *extra, src, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    # the flop-counting build: the same source as C++ with an instrumented
    # scalar (counting.h); single-threaded, used only to count operations
    out = os.path.join(_BUILD, "liboracle_count.so")
    hdr = os.path.join(_HERE, "counting.h")
    if (force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC)
            or os.path.getmtime(out) < os.path.getmtime(hdr)):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-x", "c++", "-std=c++17", "-O2", "-fPIC", "-shared",
                        "-ffp-contract=off", "-DPF_ORACLE_COUNT", f"-I{_HERE}", _SRC, "-o", tmp],
                       check=True)
        os.replace(tmp, out)


def _setup_2d(lib: ctypes.CDLL) -> ctypes.CDLL:
    """Argument and result types of the 2-D oracle's C functions."""
    P = ctypes.c_void_p
    D = ctypes.POINTER(ctypes.c_double)
    lib.or_new.restype = P
    lib.or_new.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.or_free.argtypes = [P]
    lib.or_set_params.argtypes = [P, D]
    lib.or_perturb_param.argtypes = [P, ctypes.c_int, ctypes.c_double]
    lib.or_set_window.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.or_set_rho_bar.argtypes = [P, ctypes.c_double]
    lib.or_get_rho_bar.restype = ctypes.c_double
    lib.or_get_rho_bar.argtypes = [P]
    lib.or_init_from_fields.argtypes = [P, D, D, D, D, D, D, D]
    lib.or_set_orientation.argtypes = [P, D, ctypes.c_int]
    lib.or_fields_from_spec.argtypes = [P, D, ctypes.c_int, ctypes.c_double, D,
                                        ctypes.c_int, D, D, D]
    lib.or_init_spec.restype = ctypes.c_int
    lib.or_init_spec.argtypes = [P, D, ctypes.c_int, ctypes.c_double, D, ctypes.c_int]
    lib.or_step.argtypes = [P, ctypes.c_int]
    lib.or_get_fields.argtypes = [P, ctypes.c_uint, D]
    lib.or_get_fields_im.argtypes = [P, ctypes.c_uint, D]
    lib.or_get_state.argtypes = [P, D]
    lib.or_diag.argtypes = [P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                            ctypes.c_double, D]
    lib.or_objective.argtypes = [P, D, D]
    lib.or_aniso.argtypes = [ctypes.c_double] * 5 + [D]
    lib.or_feq_ns.argtypes = [ctypes.c_double] * 4 + [D]
    lib.or_heq_cac.argtypes = [ctypes.c_double] * 3 + [D]
    lib.or_seq_sol.argtypes = [ctypes.c_double] * 3 + [D]
    lib.or_collide9.argtypes = [D] * 5
    lib.or_collide5.argtypes = [D] * 6
    lib.or_stencil.argtypes = [D, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                               ctypes.c_int, D]
    lib.or_derived.argtypes = [P, D]
    lib.or_pointwise.argtypes = [P, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, D]
    lib.or_mean_phi_global.restype = ctypes.c_double
    lib.or_mean_phi_global.argtypes = [P, D, ctypes.c_int]
    lib.or_get_steps.restype = ctypes.c_long
    lib.or_get_steps.argtypes = [P]
    lib.or_set_bc.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.or_state_planes.restype = ctypes.c_int
    lib.or_state_planes.argtypes = [P]
    lib.or_teq_th.argtypes = [ctypes.c_double] * 4 + [D]
    lib.or_thermal_coefs.argtypes = [P, ctypes.c_double, D]
    lib.or_thermal_totals.argtypes = [P, D]
    return lib


def _lib(tag: str) -> ctypes.CDLL:
    with _lock:
        if tag in _libs:
            return _libs[tag]
        build()
        lib = _setup_2d(ctypes.CDLL(os.path.join(_BUILD, f"liboracle_{tag}.so")))
        _libs[tag] = lib
        return lib


def mutant(source: str, edits, tmpdir: str) -> ctypes.CDLL:
    """A copy of one oracle source with a mistake planted in it, compiled
    like the oracle itself, for tests that check that a pin catches that
    mistake.  source: "pf_oracle.c" or "pf_oracle3d.c"; edits: (old, new)
    text pairs, each old text present exactly once; tmpdir: where the copy
    and its library go.  Returns the library with the argument types of the
    source's functions set; pass it as ``lib=`` to Oracle / Oracle3D /
    Oracle3F.  The oracle's own builds are never modified."""
    with open(os.path.join(_HERE, source)) as fh:
        text = fh.read()
    for old, new in edits:
        if text.count(old) != 1:
            raise ValueError(f"edit target must occur exactly once in {source}: {old!r}")
        text = text.replace(old, new)
    # one file name per planted text: the loader caches libraries by path
    import hashlib
    tag = hashlib.sha256(text.encode()).hexdigest()[:16]
    src = os.path.join(tmpdir, f"mutant_{tag}_{source}")
    with open(src, "w") as fh:
        fh.write(text)
    out = src[:-2] + ".so"
    subprocess.run(["gcc", "-std=c11", "-O3", "-fPIC", "-shared", "-fopenmp",
                    "-ffp-contract=off", src, "-o", out, "-lm"], check=True)
    lib = ctypes.CDLL(out)
    if source == "pf_oracle.c":
        return _setup_2d(lib)
    return _setup_3f(_setup_3d(lib))


def counting_lib() -> ctypes.CDLL:
    """The flop-counting build of the 2-D oracle (same values as the double
    build; or_count_reset / or_count_get read the operation tally)."""
    with _lock:
        if "count" in _libs:
            return _libs["count"]
        build()
        lib = _setup_2d(ctypes.CDLL(os.path.join(_BUILD, "liboracle_count.so")))
        lib.or_count_get.argtypes = [ctypes.POINTER(ctypes.c_ulonglong)]
        lib.or_count_reset.argtypes = []
        _libs["count"] = lib
        return lib


def count_step_ops(lay_params: dict, nx: int, ny: int, seeds, R_s: float, bubbles,
                   warm: int = 2) -> dict:
    """Operations of one oracle step over an nx x ny lattice (after `warm`
    steps), counted by the instrumented scalar: additions (and subtractions),
    multiplications, divisions and square roots, in total."""
    lib = counting_lib()
    o = Oracle(nx, ny, lay_params, lib=lib)
    o.init_spec(seeds, R_s, bubbles)
    o.step(warm)
    lib.or_count_reset()
    o.step(1)
    c = (ctypes.c_ulonglong * 4)()
    lib.or_count_get(c)
    return dict(zip(("add", "mul", "div", "sqrt"), [int(v) for v in c]))


def _dp(a: np.ndarray | None):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class Oracle:
    """One periodic lattice (or a window of one) advanced by the FP64 oracle.

    Arrays are row-major ``[y][x]``.  ``params`` is a dict keyed by
    ``PARAM_NAMES``.  ``complex_step=True`` selects the complex build.
    """

    def __init__(self, nx: int, ny: int, params: dict, complex_step: bool = False,
                 window: tuple[int, int, int, int] | None = None, lib: ctypes.CDLL | None = None):
        self.lib = lib if lib is not None else _lib("z" if complex_step else "d")
        self.nx, self.ny = int(nx), int(ny)
        self.h = self.lib.or_new(self.nx, self.ny)
        if not self.h:
            raise MemoryError("oracle allocation failed")
        pv = _f64([float(params[k] if k in params else THERMAL_DEFAULTS[k])
                   for k in PARAM_NAMES])
        self.lib.or_set_params(self.h, _dp(pv))
        self._pv = pv
        if window is not None:
            NX, NY, x0, y0 = window
            self.lib.or_set_window(self.h, NX, NY, x0, y0)
        self.NY = window[1] if window is not None else self.ny

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.or_free(h)
            self.h = None

    # -- set-up --------------------------------------------------------------
    def perturb(self, name: str, h: float) -> None:
        self.lib.or_perturb_param(self.h, PARAM_NAMES.index(name), float(h))

    def set_bc(self, xm: int, xp: int, ym: int, yp: int) -> None:
        """Boundary types of the sides x-, x+, y-, y+: 0 periodic, 1 symmetric,
        2 wall (half-way bounce-back), 3 far field (wall for the flow and phi,
        Dirichlet psi = -1, C = 1, theta = theta0), 4 inlet (velocity
        (vin_x, vin_y), liquid phi = 1, far-field scalars), 5 outlet (zero
        gradient), 6 inlet whose velocity is imposed by non-equilibrium
        extrapolation at the ghost node (the scalars as 4).  Set before
        initialising."""
        self.lib.or_set_bc(self.h, int(xm), int(xp), int(ym), int(yp))

    def set_rho_bar(self, rho_bar: float) -> None:
        self.lib.or_set_rho_bar(self.h, float(rho_bar))

    @property
    def rho_bar(self) -> float:
        return self.lib.or_get_rho_bar(self.h)

    def init_spec(self, seeds, R_s: float, bubbles) -> None:
        s = _f64(seeds).reshape(-1, 3) if len(seeds) else np.zeros((0, 3))
        b = _f64(bubbles).reshape(-1, 3) if len(bubbles) else np.zeros((0, 3))
        s = np.ascontiguousarray(s)
        b = np.ascontiguousarray(b)
        rc = self.lib.or_init_spec(self.h, _dp(s), len(s), float(R_s), _dp(b), len(b))
        if rc != 0:
            raise MemoryError("oracle init failed")

    def fields_from_spec(self, seeds, R_s, bubbles):
        s = np.ascontiguousarray(_f64(seeds).reshape(-1, 3))
        b = np.ascontiguousarray(_f64(bubbles).reshape(-1, 3))
        n = self.nx * self.ny
        phi, psi, C = (np.empty(n), np.empty(n), np.empty(n))
        self.lib.or_fields_from_spec(self.h, _dp(s), len(s), float(R_s), _dp(b), len(b),
                                     _dp(phi), _dp(psi), _dp(C))
        shp = (self.ny, self.nx)
        return phi.reshape(shp), psi.reshape(shp), C.reshape(shp)

    def mean_phi_global(self, bubbles) -> float:
        b = np.ascontiguousarray(_f64(bubbles).reshape(-1, 3))
        return self.lib.or_mean_phi_global(self.h, _dp(b), len(b))

    def set_orientation(self, seeds) -> None:
        s = np.ascontiguousarray(_f64(seeds).reshape(-1, 3))
        self.lib.or_set_orientation(self.h, _dp(s), len(s))

    def init_fields(self, phi, psi, C, vx=None, vy=None, p=None, theta=None) -> None:
        arrs = [_f64(a).ravel() if a is not None else None
                for a in (phi, psi, C, vx, vy, p, theta)]
        self._keep = arrs
        self.lib.or_init_from_fields(self.h, *[_dp(a) for a in arrs])

    # -- run -----------------------------------------------------------------
    def step(self, n: int = 1) -> None:
        self.lib.or_step(self.h, int(n))

    # -- outputs -------------------------------------------------------------
    def fields(self, names=FIELDS, imag: bool = False) -> dict[str, np.ndarray]:
        mask = 0
        for nm in names:
            mask |= 1 << FIELDS.index(nm)
        sel = [nm for nm in FIELDS if mask & (1 << FIELDS.index(nm))]
        out = np.empty(len(sel) * self.nx * self.ny)
        fn = self.lib.or_get_fields_im if imag else self.lib.or_get_fields
        fn(self.h, mask, _dp(out))
        out = out.reshape(len(sel), self.ny, self.nx)
        return {nm: out[i] for i, nm in enumerate(sel)}

    def state(self) -> np.ndarray:
        npl = self.lib.or_state_planes(self.h)
        out = np.empty(npl * self.nx * self.ny)
        self.lib.or_get_state(self.h, _dp(out))
        return out.reshape(npl, self.ny, self.nx)

    def thermal_coefs(self, U: float) -> dict[str, float]:
        """F(U), k_T and the temperature flux rate s_th."""
        out = np.zeros(3)
        self.lib.or_thermal_coefs(self.h, float(U), _dp(out))
        return dict(zip(("F", "kT", "s_th"), out.tolist()))

    def thermal_totals(self) -> dict[str, float]:
        """Sum of the temperature populations (total rho H), sum theta, sum psi."""
        out = np.zeros(3)
        self.lib.or_thermal_totals(self.h, _dp(out))
        return dict(zip(("sum_e", "sum_theta", "sum_psi"), out.tolist()))

    def diag(self, probe=(0.0, 0.0, 0.0, 0.0)) -> dict[str, float]:
        out = np.zeros(12)
        xc, yc, R, W = probe
        self.lib.or_diag(self.h, float(xc), float(yc), float(R), float(W), _dp(out))
        keys = ("sum_phi", "sum_C", "sum_hpsi", "gas", "gas_x", "gas_y", "p_in_sum",
                "p_in_n", "p_out_sum", "p_out_n", "max_v", "nonfinite")
        return dict(zip(keys, out.tolist()))

    def derived(self) -> dict[str, float]:
        out = np.zeros(8)
        self.lib.or_derived(self.h, _dp(out))
        keys = ("lambda_p", "Mc_inf", "theta_sys", "kappa", "fs_coef", "s_nu", "s_q", "s_phi")
        return dict(zip(keys, out.tolist()))

    def pointwise(self, phi, psi, C) -> tuple[float, float]:
        """(U, Q_psi) at one site."""
        out = np.zeros(2)
        self.lib.or_pointwise(self.h, float(phi), float(psi), float(C), _dp(out))
        return float(out[0]), float(out[1])

    @property
    def steps(self) -> int:
        return self.lib.or_get_steps(self.h)

    def objective(self) -> tuple[float, float]:
        re = ctypes.c_double()
        im = ctypes.c_double()
        self.lib.or_objective(self.h, ctypes.byref(re), ctypes.byref(im))
        return re.value, im.value


# -- pointwise pieces (double build), used by the pin tests ------------------
def aniso(gx, gy, theta, eps, geps=1e-6):
    """(a_s, Nx, Ny, |grad psi|_reg) at gradient (gx, gy) for a grain at theta."""
    out = np.zeros(4)
    _lib("d").or_aniso(float(gx), float(gy), float(theta), float(eps), float(geps), _dp(out))
    return out


def feq_ns(p, rho, vx, vy):
    out = np.zeros(9)
    _lib("d").or_feq_ns(float(p), float(rho), float(vx), float(vy), _dp(out))
    return out


def heq_cac(phi, vx, vy):
    out = np.zeros(9)
    _lib("d").or_heq_cac(float(phi), float(vx), float(vy), _dp(out))
    return out


def seq_sol(C, jx, jy):
    out = np.zeros(5)
    _lib("d").or_seq_sol(float(C), float(jx), float(jy), _dp(out))
    return out


def teq_th(rhoH, theta, jx, jy):
    out = np.zeros(5)
    _lib("d").or_teq_th(float(rhoH), float(theta), float(jx), float(jy), _dp(out))
    return out


def collide9(f, feq, S, G):
    args = [_f64(a) for a in (f, feq, S, G)]
    out = np.zeros(9)
    _lib("d").or_collide9(*[_dp(a) for a in args], _dp(out))
    return out


def collide5(f, feq, S, G, Fd):
    args = [_f64(a) for a in (f, feq, S, G, Fd)]
    out = np.zeros(5)
    _lib("d").or_collide5(*[_dp(a) for a in args], _dp(out))
    return out


def stencil(X, x, y):
    """(d_x X, d_y X, lap X) of a periodic [ny][nx] array at site (x, y)."""
    X = _f64(X)
    ny, nx = X.shape
    out = np.zeros(3)
    _lib("d").or_stencil(_dp(X), nx, ny, int(x), int(y), _dp(out))
    return out


# -- the three-dimensional dendrite oracle (pf_oracle3d.c) ---------------------
PARAM_NAMES_3D = ("beta_psi", "W0", "tau0", "eps_s", "k", "D", "Omega", "grad_eps",
                  "grad_eps_at", "thermal", "Le", "latent", "theta0", "cp", "rho_l")
_lib3 = None


def _setup_3d(lib: ctypes.CDLL) -> ctypes.CDLL:
    """Argument and result types of the 3-D melt oracle's C functions."""
    P, D, I = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
    lib.or3_new.restype = P
    lib.or3_new.argtypes = [I, I, I]
    lib.or3_free.argtypes = [P]
    lib.or3_set_params.argtypes = [P, D]
    lib.or3_init.argtypes = [P, D, I, ctypes.c_double]
    lib.or3_init_fields.argtypes = [P, D, D]
    lib.or3_step.argtypes = [P, I]
    lib.or3_fields.argtypes = [P, D]
    lib.or3_state.argtypes = [P, D]
    lib.or3_aniso.argtypes = [D, ctypes.c_double, ctypes.c_double, D]
    lib.or3_collide7.argtypes = [D] * 6
    lib.or3_grad.argtypes = [D, I, I, I, I, I, I, D]
    lib.or3_set_window.argtypes = [P, I, I, I, I, I, I]
    lib.or3_init_fields.argtypes = [P, D, D, D]
    lib.or3_state_planes.restype = I
    lib.or3_state_planes.argtypes = [P]
    lib.or3_thermal_totals.argtypes = [P, D]
    lib.or3_set_orientation.argtypes = [P, D, I]
    lib.or3_set_orientation.restype = I
    lib.or3_set_bc.argtypes = [P, ctypes.POINTER(ctypes.c_int)]
    lib.or3_orientation.argtypes = [P, I, D]
    return lib


def _l3() -> ctypes.CDLL:
    global _lib3
    with _lock:
        if _lib3 is None:
            build()
            _lib3 = _setup_3d(ctypes.CDLL(os.path.join(_BUILD, "liboracle_3d.so")))
    return _lib3


class Oracle3D:
    """Periodic nx x ny x nz lattice of the 3-D dendrite model (psi and C on
    D3Q7, no gas, no flow).  Arrays are [z][y][x]."""

    def __init__(self, nx: int, ny: int, nz: int, params: dict, window=None,
                 lib: ctypes.CDLL | None = None):
        self.lib = lib if lib is not None else _l3()
        self.shape = (int(nz), int(ny), int(nx))
        self.h = self.lib.or3_new(int(nx), int(ny), int(nz))
        if not self.h:
            raise MemoryError("oracle allocation failed")
        dflt = dict(THERMAL_DEFAULTS, rho_l=1.0)
        pv = _f64([float(params[k] if k in params else dflt[k]) for k in PARAM_NAMES_3D])
        self.lib.or3_set_params(self.h, _dp(pv))
        if window is not None:           # (NX, NY, NZ, x0, y0, z0)
            self.lib.or3_set_window(self.h, *[int(v) for v in window])

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.or3_free(h)
            self.h = None

    def init_spec(self, seeds, R_s: float) -> None:
        s = np.ascontiguousarray(_f64(seeds).reshape(-1, 3))
        self.lib.or3_init(self.h, _dp(s), len(s), float(R_s))

    def set_orientation(self, seeds7) -> None:
        """Grain orientations: n x (x, y, z, qw, qx, qy, qz); each site takes the
        rotation of the nearest seed."""
        s = np.ascontiguousarray(_f64(seeds7).reshape(-1, 7))
        if self.lib.or3_set_orientation(self.h, _dp(s), len(s)) != 0:
            raise MemoryError("oracle allocation failed")

    def set_bc(self, bc) -> None:
        """Side types x-, x+, y-, y+, z-, z+: 0 periodic, 1 symmetric, 2 wall,
        3 far field (opposite sides both periodic or both not)."""
        arr = (ctypes.c_int * 6)(*[int(b) for b in bc])
        self.lib.or3_set_bc(self.h, arr)

    def orientation(self, site: int) -> np.ndarray:
        out = np.zeros(9)
        self.lib.or3_orientation(self.h, int(site), _dp(out))
        return out.reshape(3, 3)

    def init_fields(self, psi, C, theta=None) -> None:
        self._keep = [_f64(psi).ravel(), _f64(C).ravel(),
                      None if theta is None else _f64(theta).ravel()]
        self.lib.or3_init_fields(self.h, *[_dp(a) for a in self._keep])

    def step(self, n: int = 1) -> None:
        self.lib.or3_step(self.h, int(n))

    def fields(self) -> dict:
        out = np.empty(4 * int(np.prod(self.shape)))
        self.lib.or3_fields(self.h, _dp(out))
        out = out.reshape((4,) + self.shape)
        return {"psi": out[0], "C": out[1], "U": out[2], "theta": out[3]}

    def state(self) -> np.ndarray:
        npl = self.lib.or3_state_planes(self.h)
        out = np.empty(npl * int(np.prod(self.shape)))
        self.lib.or3_state(self.h, _dp(out))
        return out.reshape((npl,) + self.shape)

    def thermal_totals(self) -> dict:
        out = np.zeros(2)
        self.lib.or3_thermal_totals(self.h, _dp(out))
        return {"sum_e": out[0], "sum_theta": out[1]}


def aniso3(g, eps, geps=1e-3, lib: ctypes.CDLL | None = None):
    out = np.zeros(5)
    gg = _f64(g)
    (lib if lib is not None else _l3()).or3_aniso(_dp(gg), float(eps), float(geps), _dp(out))
    return out


def collide7(f, feq, S, G, Fd):
    args = [_f64(a) for a in (f, feq, S, G, Fd)]
    out = np.zeros(7)
    _l3().or3_collide7(*[_dp(a) for a in args], _dp(out))
    return out


def grad3(X, x, y, z):
    X = _f64(X)
    nz, ny, nx = X.shape
    out = np.zeros(3)
    _l3().or3_grad(_dp(X), nx, ny, nz, int(x), int(y), int(z), _dp(out))
    return out


# -- the three-dimensional two-phase oracle (pf_oracle3d.c, or3f_*) ----------
PARAM_NAMES_3F = ("rho_l", "rho_g", "nu", "sigma", "W_phi", "M_phi", "beta_phi", "beta_psi",
                  "beta_inter", "W0", "tau0", "eps_s", "k", "D", "Omega", "g", "grad_eps",
                  "grad_eps_at", "s_e", "s_eps", "thermal", "Le", "latent", "theta0", "cp")
FIELDS_3F = ("phi", "psi", "C", "U", "p", "vx", "vy", "vz", "mu", "theta")
_lib3f = None


def _setup_3f(lib: ctypes.CDLL) -> ctypes.CDLL:
    """Argument and result types of the 3-D two-phase oracle's C functions."""
    P, D, I = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
    lib.or3f_new.restype = P
    lib.or3f_new.argtypes = [I, I, I]
    lib.or3f_free.argtypes = [P]
    lib.or3f_set_params.argtypes = [P, D]
    lib.or3f_set_window.argtypes = [P, I, I, I, I, I, I]
    lib.or3f_set_rho_bar.argtypes = [P, ctypes.c_double]
    lib.or3f_get_rho_bar.argtypes = [P]
    lib.or3f_get_rho_bar.restype = ctypes.c_double
    lib.or3f_init_fields.argtypes = [P, D, D, D, D, D, D, D]
    lib.or3f_fields_from_spec.argtypes = [P, D, I, ctypes.c_double, D, I, D, D, D]
    lib.or3f_mean_phi_global.argtypes = [P, D, I]
    lib.or3f_mean_phi_global.restype = ctypes.c_double
    lib.or3f_init_spec.argtypes = [P, D, I, ctypes.c_double, D, I]
    lib.or3f_step.argtypes = [P, I]
    lib.or3f_fields.argtypes = [P, D]
    lib.or3f_state.argtypes = [P, D]
    lib.or3f_totals.argtypes = [P, D]
    lib.or3f_basis.argtypes = [D, D, ctypes.POINTER(ctypes.c_int)]
    lib.or3f_collide19.argtypes = [D] * 5
    lib.or3f_feq.argtypes = [ctypes.c_double, ctypes.c_double, D, D]
    lib.or3f_set_orientation.argtypes = [P, D, I]
    lib.or3f_set_orientation.restype = I
    lib.or3f_set_temperature.argtypes = [P, D]
    lib.or3f_set_bc.argtypes = [P, ctypes.POINTER(ctypes.c_int)]
    lib.or3f_thermal_totals.argtypes = [P, D]
    lib.or3f_state_planes.argtypes = [P]
    lib.or3f_state_planes.restype = I
    return lib


def _l3f() -> ctypes.CDLL:
    global _lib3f
    lib = _l3()                          # takes the module lock itself
    with _lock:
        if _lib3f is None:
            _lib3f = _setup_3f(lib)
    return _lib3f


class Oracle3F:
    """Periodic nx x ny x nz lattice of the 3-D two-phase step: NS and CAC on
    D3Q19, psi and C on D3Q7, coupled as in 2-D.  Arrays are [z][y][x]; seeds
    are (x, y, z), bubbles (x, y, z, R)."""

    def __init__(self, nx: int, ny: int, nz: int, params: dict, window=None,
                 lib: ctypes.CDLL | None = None):
        self.lib = lib if lib is not None else _l3f()
        self.shape = (int(nz), int(ny), int(nx))
        self.h = self.lib.or3f_new(int(nx), int(ny), int(nz))
        if not self.h:
            raise MemoryError("oracle allocation failed")
        dflt = dict(THERMAL_DEFAULTS, s_e=1.0, s_eps=1.0)
        pv = _f64([float(params[k] if k in params else dflt[k]) for k in PARAM_NAMES_3F])
        self.lib.or3f_set_params(self.h, _dp(pv))
        if window is not None:           # (NX, NY, NZ, x0, y0, z0)
            self.lib.or3f_set_window(self.h, *[int(v) for v in window])

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.or3f_free(h)
            self.h = None

    def set_rho_bar(self, rho_bar: float) -> None:
        self.lib.or3f_set_rho_bar(self.h, float(rho_bar))

    def set_bc(self, bc) -> None:
        """Side types x-, x+, y-, y+, z-, z+: 0 periodic, 1 symmetric, 2 wall,
        3 far field."""
        arr = (ctypes.c_int * 6)(*[int(b) for b in bc])
        self.lib.or3f_set_bc(self.h, arr)

    @property
    def rho_bar(self) -> float:
        return self.lib.or3f_get_rho_bar(self.h)

    def fields_from_spec(self, seeds, R_s, bubbles):
        s = np.ascontiguousarray(_f64(seeds).reshape(-1, 3))
        b = np.ascontiguousarray(_f64(bubbles).reshape(-1, 4))
        n = int(np.prod(self.shape))
        out = np.empty(3 * n)
        self.lib.or3f_fields_from_spec(self.h, _dp(s), len(s), float(R_s), _dp(b), len(b),
                                       _dp(out[:n]), _dp(out[n:2 * n]), _dp(out[2 * n:]))
        out = out.reshape((3,) + self.shape)
        return {"phi": out[0], "psi": out[1], "C": out[2]}

    def mean_phi_global(self, bubbles) -> float:
        b = np.ascontiguousarray(_f64(bubbles).reshape(-1, 4))
        return self.lib.or3f_mean_phi_global(self.h, _dp(b), len(b))

    def init_spec(self, seeds, R_s: float, bubbles) -> None:
        s = np.ascontiguousarray(_f64(seeds).reshape(-1, 3))
        b = np.ascontiguousarray(_f64(bubbles).reshape(-1, 4))
        self.lib.or3f_init_spec(self.h, _dp(s), len(s), float(R_s), _dp(b), len(b))

    def init_fields(self, phi, psi, C, vx=None, vy=None, vz=None, p=None) -> None:
        self._keep = [None if a is None else _f64(a).ravel() for a in (phi, psi, C, vx, vy, vz, p)]
        self.lib.or3f_init_fields(self.h, *[_dp(a) for a in self._keep])

    def set_orientation(self, seeds7) -> None:
        """Grain orientations: n x (x, y, z, qw, qx, qy, qz); each site takes the
        rotation of the nearest seed."""
        s = np.ascontiguousarray(_f64(seeds7).reshape(-1, 7))
        if self.lib.or3f_set_orientation(self.h, _dp(s), len(s)) != 0:
            raise MemoryError("oracle allocation failed")

    def step(self, n: int = 1) -> None:
        self.lib.or3f_step(self.h, int(n))

    def fields(self) -> dict:
        k = len(FIELDS_3F)
        out = np.empty(k * int(np.prod(self.shape)))
        self.lib.or3f_fields(self.h, _dp(out))
        return dict(zip(FIELDS_3F, out.reshape((k,) + self.shape)))

    def state(self) -> np.ndarray:
        npl = self.lib.or3f_state_planes(self.h)
        out = np.empty(npl * int(np.prod(self.shape)))
        self.lib.or3f_state(self.h, _dp(out))
        return out.reshape((npl,) + self.shape)

    def set_temperature(self, theta) -> None:
        """Thermal mode: initial temperature field after init_spec / init_fields."""
        self._theta = _f64(theta).ravel()
        self.lib.or3f_set_temperature(self.h, _dp(self._theta))

    def thermal_totals(self) -> dict:
        out = np.zeros(2)
        self.lib.or3f_thermal_totals(self.h, _dp(out))
        return {"sum_e": out[0], "sum_theta": out[1]}

    def totals(self) -> dict:
        out = np.zeros(5)
        self.lib.or3f_totals(self.h, _dp(out))
        return {"sum_phi": out[0], "sum_C": out[1], "j": out[2:5].copy()}


def basis19(lib: ctypes.CDLL | None = None):
    """(M, w, c) of the D3Q19 lattice: moment rows, weights, velocities."""
    M, W = np.zeros((19, 19)), np.zeros(19)
    C = np.zeros(57, dtype=np.int32)
    (lib if lib is not None else _l3f()).or3f_basis(_dp(M), _dp(W), C.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return M, W, C.reshape(19, 3)


def collide19(f, feq, S, G):
    args = [_f64(a) for a in (f, feq, S, G)]
    out = np.zeros(19)
    _l3f().or3f_collide19(*[_dp(a) for a in args], _dp(out))
    return out


def feq19(p, rho, v):
    out = np.zeros(19)
    vv = _f64(v)
    _l3f().or3f_feq(float(p), float(rho), _dp(vv), _dp(out))
    return out
