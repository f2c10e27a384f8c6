"""Thin ctypes binding of the C ABI in ``include/pf.h``.

Argument marshalling only: every step of the method runs in the CUDA kernels
of ``_build/libpf.so``.  PyTorch supplies the CUDA stream and, optionally, the
device memory (its caching allocator is handed to ``pf_create``).  There is
no CPU fallback: if the library is missing this module raises on first use.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpf.so")

PF_OK, PF_ERR_BAD_ARG, PF_ERR_OOM, PF_ERR_CUDA, PF_ERR_TIMEOUT, PF_ERR_NAN, PF_ERR_STATE = (
    0, -1, -2, -3, -4, -5, -6)
PF_FP64, PF_FP32, PF_FP16_OFFSET, PF_BF16_OFFSET = 0, 1, 2, 3
PRECISIONS = {"fp64": PF_FP64, "fp32": PF_FP32, "fp16": PF_FP16_OFFSET, "bf16": PF_BF16_OFFSET}
BC_PERIODIC, BC_SYMMETRIC, BC_WALL, BC_FARFIELD, BC_INLET, BC_OUTLET = 0, 1, 2, 3, 4, 5
BC_INLET_NEE = 6
FIELDS = ("phi", "psi", "C", "U", "p", "vx", "vy", "mu", "theta")
STATE_PLANES = 39            # PF_STATE_PLANES; thermal handles have 45

_PARAM_FIELDS = ("rho_l", "rho_g", "nu", "sigma", "W_phi", "M_phi", "beta_phi", "beta_psi",
                 "beta_inter", "W0", "tau0", "eps_s", "k", "D", "Omega", "g", "grad_eps",
                 "grad_eps_at", "s_e", "s_eps", "Le", "latent", "theta0", "cp", "vin_x", "vin_y")
_PARAM_INTS = ("thermal", "reserved")


class pf_params(ctypes.Structure):
    _fields_ = ([(n, ctypes.c_double) for n in _PARAM_FIELDS] +
                [(n, ctypes.c_int) for n in _PARAM_INTS])


class pf_domain(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("eps_s", ctypes.c_double)]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class pf_allocator(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("alloc", _ALLOC_FN), ("free", _FREE_FN)]


class pf_init_spec(ctypes.Structure):
    _fields_ = [("n_seeds", ctypes.c_int), ("seeds", ctypes.POINTER(ctypes.c_double)),
                ("R_s", ctypes.c_double), ("n_bubbles", ctypes.c_int),
                ("bubbles", ctypes.POINTER(ctypes.c_double))]


_DIAG_FIELDS = ("sum_phi", "sum_C", "sum_hpsi", "gas", "gas_x", "gas_y", "p_in_sum", "p_in_n",
                "p_out_sum", "p_out_n", "max_v", "nonfinite")


class pf_diag(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in _DIAG_FIELDS]


class pf_objective(ctypes.Structure):
    _fields_ = [("w_solid", ctypes.c_double), ("w_centroid", ctypes.c_double),
                ("checkpoint_every", ctypes.c_int)]


class pf_probe(ctypes.Structure):
    _fields_ = [("xc", ctypes.c_double), ("yc", ctypes.c_double), ("R", ctypes.c_double),
                ("W", ctypes.c_double)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libpf.so (built by ``build()``); raise if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(LIB_PATH)
    P, D, I, S = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_size_t
    L.pf_params_default.argtypes = [ctypes.POINTER(pf_params)]
    L.pf_params_derived.argtypes = [ctypes.POINTER(pf_params), D]
    L.pf_create.argtypes = [ctypes.POINTER(pf_params), ctypes.POINTER(pf_domain), I, I, P,
                            ctypes.POINTER(pf_allocator), ctypes.POINTER(P)]
    L.pf_init_fields.argtypes = [P, I, ctypes.POINTER(pf_init_spec)]
    L.pf_set_fields.argtypes = [P, I, D, D, S]
    L.pf_step.argtypes = [P, I]
    L.pf_get_fields.argtypes = [P, I, ctypes.c_uint32, D, S]
    L.pf_run.argtypes = [P, D, S, I, ctypes.c_uint32, D, S]
    L.pf_get_state.argtypes = [P, I, D, S]
    L.pf_set_state.argtypes = [P, I, D, S]
    L.pf_reduce.argtypes = [P, I, ctypes.POINTER(pf_probe), ctypes.POINTER(pf_diag)]
    L.pf_set_step_config.argtypes = [P, I, I, I]
    L.pf_get_step_config.argtypes = [P, ctypes.POINTER(ctypes.c_int)]
    L.pf_reduce_noalloc.argtypes = [P, I, ctypes.c_longlong, ctypes.c_longlong, I, I,
                                    ctypes.POINTER(pf_probe), ctypes.POINTER(pf_diag), P]
    L.pf_adjoint_step.argtypes = [P, I, ctypes.POINTER(pf_objective), D, D]
    L.pf_set_launch.argtypes = [P, I, I, I]
    L.pf_autotune.argtypes = [P, I, ctypes.POINTER(ctypes.c_int)]
    L.pf_sync.argtypes = [P]
    L.pf_test_drop_staged_copies.argtypes = [P, I]
    L.pf_steps_taken.argtypes = [P]
    L.pf_steps_taken.restype = ctypes.c_longlong
    L.pf_launch_count.argtypes = [P]
    L.pf_launch_count.restype = ctypes.c_longlong
    L.pf_destroy.argtypes = [P]
    L.pf_last_error.argtypes = [P]
    L.pf_last_error.restype = ctypes.c_char_p
    L.pf_state_planes.argtypes = [P]
    L.pf_state_planes.restype = ctypes.c_int
    L.pf_set_temperature.argtypes = [P, I, D, S]
    L.pf_reduce_thermal.argtypes = [P, I, D]
    L.pf_set_boundaries.argtypes = [P, I, ctypes.POINTER(ctypes.c_int)]
    L.pf3_create.argtypes = [ctypes.POINTER(pf_params), I, I, I, I, P, ctypes.POINTER(P)]
    L.pf3_init_seeds.argtypes = [P, D, I, ctypes.c_double]
    L.pf3_set_fields.argtypes = [P, D, D, S]
    L.pf3_set_chunk.argtypes = [P, I]
    L.pf3_set_index64.argtypes = [P, I]
    L.pf3_step.argtypes = [P, I]
    L.pf3_get_fields.argtypes = [P, D, S]
    L.pf3_get_state.argtypes = [P, D, S]
    L.pf3_reduce.argtypes = [P, D]
    L.pf3_set_temperature.argtypes = [P, D, S]
    L.pf3_set_orientation.argtypes = [P, D, I]
    L.pf3_set_boundaries.argtypes = [P, ctypes.POINTER(ctypes.c_int)]
    L.pf3_reduce_thermal.argtypes = [P, D]
    L.pf3_field_planes.argtypes = [P]
    L.pf3_state_planes.argtypes = [P]
    L.pf3_launch_count.argtypes = [P]
    L.pf3_launch_count.restype = ctypes.c_longlong
    L.pf3_last_error.argtypes = [P]
    L.pf3_last_error.restype = ctypes.c_char_p
    L.pf3_destroy.argtypes = [P]
    L.pf3f_create.argtypes = [ctypes.POINTER(pf_params), I, I, I, I, P, ctypes.POINTER(P)]
    L.pf3f_init_spec.argtypes = [P, D, I, ctypes.c_double, D, I]
    L.pf3f_set_fields.argtypes = [P, D, S]
    L.pf3f_set_rho_bar.argtypes = [P, ctypes.c_double]
    L.pf3f_get_rho_bar.argtypes = [P]
    L.pf3f_get_rho_bar.restype = ctypes.c_double
    L.pf3f_set_chunk.argtypes = [P, I]
    L.pf3f_set_index64.argtypes = [P, I]
    L.pf3f_set_orientation.argtypes = [P, D, I]
    L.pf3f_set_boundaries.argtypes = [P, ctypes.POINTER(ctypes.c_int)]
    L.pf3f_set_temperature.argtypes = [P, D, S]
    L.pf3f_reduce_thermal.argtypes = [P, D]
    L.pf3f_field_planes.argtypes = [P]
    L.pf3f_state_planes.argtypes = [P]
    L.pf3f_step.argtypes = [P, I]
    L.pf3f_get_fields.argtypes = [P, D, S]
    L.pf3f_get_state.argtypes = [P, D, S]
    L.pf3f_reduce.argtypes = [P, D]
    L.pf3f_launch_count.argtypes = [P]
    L.pf3f_launch_count.restype = ctypes.c_longlong
    L.pf3f_last_error.argtypes = [P]
    L.pf3f_last_error.restype = ctypes.c_char_p
    L.pf3f_destroy.argtypes = [P]
    for name in ("pf_params_default", "pf_params_derived", "pf_create", "pf_init_fields",
                 "pf_set_fields", "pf_step", "pf_get_fields", "pf_run", "pf_get_state",
                 "pf_set_state", "pf_reduce", "pf_sync", "pf_destroy", "pf_set_step_config",
                 "pf_get_step_config", "pf_reduce_noalloc", "pf_adjoint_step",
                 "pf_set_launch", "pf_autotune", "pf_set_temperature", "pf_reduce_thermal",
                 "pf_set_boundaries", "pf3_create", "pf3_init_seeds", "pf3_set_fields",
                 "pf3_set_chunk", "pf3_set_index64", "pf3_step", "pf3_get_fields", "pf3_get_state", "pf3_reduce",
                 "pf3_destroy", "pf3_set_temperature", "pf3_reduce_thermal", "pf3_set_orientation",
                 "pf3_set_boundaries",
                 "pf3f_create",
                 "pf3f_init_spec", "pf3f_set_fields", "pf3f_set_rho_bar", "pf3f_set_chunk",
                 "pf3f_set_index64",
                 "pf3f_step", "pf3f_get_fields", "pf3f_get_state", "pf3f_reduce", "pf3f_destroy",
                 "pf3f_set_orientation", "pf3f_set_temperature", "pf3f_reduce_thermal",
                 "pf3f_set_boundaries"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


class PFError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"pf error {code}: {msg}")
        self.code = code


def _check(code: int, handle=None) -> None:
    if code != PF_OK:
        msg = lib().pf_last_error(handle).decode(errors="replace")
        raise PFError(code, msg)


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def params_from_dict(d: dict | None = None) -> pf_params:
    p = pf_params()
    _check(lib().pf_params_default(ctypes.byref(p)))
    for k, v in (d or {}).items():
        if k in _PARAM_FIELDS:
            setattr(p, k, float(v))
        elif k in _PARAM_INTS:
            setattr(p, k, int(v))
    return p


def pf_params_derived(d: dict) -> tuple[float, float, float]:
    out = np.zeros(3)
    _check(lib().pf_params_derived(ctypes.byref(params_from_dict(d)), _dp(out)))
    return tuple(out.tolist())


def pf_reduce_noalloc(fields_ptr: int, fp64: bool, plane_stride: int, offset: int, nx: int,
                      ny: int, probe=None, stream: int = 0) -> dict:
    """FP64 diagnostics of caller-owned device field planes; the library
    allocates no device memory for it (see include/pf.h)."""
    d = pf_diag()
    pr = pf_probe(*probe) if probe is not None else None
    _check(lib().pf_reduce_noalloc(ctypes.c_void_p(fields_ptr), int(bool(fp64)),
                                   int(plane_stride), int(offset), int(nx), int(ny),
                                   ctypes.byref(pr) if pr else None, ctypes.byref(d),
                                   ctypes.c_void_p(stream)))
    return {k: getattr(d, k) for k in _DIAG_FIELDS}


def torch_allocator(device=None):
    """A pf_allocator backed by PyTorch's caching allocator."""
    import torch

    dev = torch.cuda.current_device() if device is None else device

    def _alloc(ctx, nbytes, stream):
        return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream or 0)

    def _free(ctx, ptr, stream):
        torch.cuda.caching_allocator_delete(ptr)

    a = pf_allocator(None, _ALLOC_FN(_alloc), _FREE_FN(_free))
    return a


class Simulation:
    """Handle of ``n`` periodic domains; methods mirror the C ABI."""

    def __init__(self, domains, params: dict | None = None, precision: str = "fp32",
                 stream=None, use_torch_allocator: bool = False):
        L = lib()
        doms = (pf_domain * len(domains))()
        for i, dm in enumerate(domains):
            nx, ny = dm[0], dm[1]
            eps = dm[2] if len(dm) > 2 and dm[2] is not None else -1.0
            doms[i] = pf_domain(int(nx), int(ny), float(eps))
        self.domains = [(int(d.nx), int(d.ny)) for d in doms]
        self.params = params_from_dict(params)
        self._alloc = torch_allocator() if use_torch_allocator else None
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream
            except Exception:
                stream = 0
        self.stream = stream
        h = ctypes.c_void_p()
        code = L.pf_create(ctypes.byref(self.params), doms, len(domains), PRECISIONS[precision],
                           ctypes.c_void_p(stream),
                           ctypes.byref(self._alloc) if self._alloc else None, ctypes.byref(h))
        _check(code, None)
        self.h = h
        self.precision = precision

    def close(self) -> None:
        if getattr(self, "h", None):
            code = lib().pf_destroy(self.h)
            self.h = None
            _check(code)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- initialisation --------------------------------------------------------
    def set_boundaries(self, dom: int, xm: int, xp: int, ym: int, yp: int) -> None:
        """Side types x-, x+, y-, y+ of a domain before its initialisation:
        BC_PERIODIC, BC_SYMMETRIC, BC_WALL, BC_FARFIELD, BC_INLET, BC_OUTLET or
        BC_INLET_NEE."""
        bc = (ctypes.c_int * 4)(int(xm), int(xp), int(ym), int(yp))
        _check(lib().pf_set_boundaries(self.h, int(dom), bc), self.h)

    def init_fields(self, dom: int, seeds, R_s: float, bubbles) -> None:
        s = np.ascontiguousarray(np.asarray(seeds, dtype=np.float64).reshape(-1, 3))
        b = np.ascontiguousarray(np.asarray(bubbles, dtype=np.float64).reshape(-1, 3))
        spec = pf_init_spec(len(s), _dp(s), float(R_s), len(b), _dp(b))
        _check(lib().pf_init_fields(self.h, dom, ctypes.byref(spec)), self.h)

    def set_fields(self, dom: int, phi, psi, C, vx=None, vy=None, p=None, theta=None) -> None:
        """Initialise a domain from its macroscopic fields ([ny][nx] each;
        vx, vy, p default to 0).  Separate arrays are stacked into one block
        first; set_fields_stack passes a ready block without that copy."""
        nx, ny = self.domains[dom]
        z = np.zeros((ny, nx))
        f6 = np.ascontiguousarray(np.stack([np.asarray(a if a is not None else z, dtype=np.float64)
                                            .reshape(ny, nx) for a in (phi, psi, C, vx, vy, p)]))
        self.set_fields_stack(dom, f6, theta)

    def set_fields_stack(self, dom: int, f6: np.ndarray, theta=None) -> None:
        """Initialise a domain from one C-contiguous float64 block of shape
        (6, ny, nx) holding phi, psi, C, vx, vy, p.  The block's memory is
        handed to pf_set_fields as it is (no copy on the host), so a block in
        page-locked memory is copied to the device at full link speed."""
        nx, ny = self.domains[dom]
        if (not isinstance(f6, np.ndarray) or f6.dtype != np.float64 or f6.shape != (6, ny, nx)
                or not f6.flags["C_CONTIGUOUS"]):
            raise ValueError(f"f6 must be a C-contiguous float64 array of shape (6, {ny}, {nx})")
        th = None if theta is None else np.ascontiguousarray(
            np.broadcast_to(np.asarray(theta, dtype=np.float64), (ny, nx)))
        _check(lib().pf_set_fields(self.h, dom, _dp(f6), _dp(th) if th is not None else None,
                                   nx * ny), self.h)

    # -- stepping --------------------------------------------------------------
    def step(self, n: int = 1) -> None:
        _check(lib().pf_step(self.h, int(n)), self.h)

    def set_step_config(self, variant: int, a: int, b: int = 0) -> None:
        """variant 0: 2-D tiles a x b; variant 1: y-march strips, a rows per tile;
        variant 2: y-march strips with the input rows staged in shared memory by
        bulk copies, a rows per tile (needs nx a multiple of 16 bytes of storage
        in every domain)."""
        _check(lib().pf_set_step_config(self.h, int(variant), int(a), int(b)), self.h)

    def set_launch(self, per_domain: bool = False, persistent: int = 0,
                   graph_steps: int = 0) -> None:
        """per_domain: one launch per domain; persistent 1: resident grid
        looping over the tiles, 2: and every step of a call in one cooperative
        launch; graph_steps > 0 (even): replay CUDA graphs of that many steps."""
        _check(lib().pf_set_launch(self.h, int(per_domain), int(persistent), int(graph_steps)),
               self.h)

    def autotune(self, trial_steps: int = 20) -> tuple[int, int, int, int]:
        """Pick the fastest step traversal for these domains (state unchanged)."""
        out = (ctypes.c_int * 4)()
        _check(lib().pf_autotune(self.h, int(trial_steps), out), self.h)
        return tuple(out)

    def step_config(self) -> tuple[int, int, int]:
        out = (ctypes.c_int * 3)()
        _check(lib().pf_get_step_config(self.h, out), self.h)
        return tuple(out)

    def test_drop_staged_copies(self, on: bool) -> None:
        """Testing only: make the staged step kernel skip its bulk copies, so
        that its bounded waits time out and the next synchronising call
        raises PFError(PF_ERR_TIMEOUT)."""
        _check(lib().pf_test_drop_staged_copies(self.h, int(bool(on))), self.h)

    def sync(self) -> None:
        _check(lib().pf_sync(self.h), self.h)

    @property
    def steps(self) -> int:
        return lib().pf_steps_taken(self.h)

    @property
    def launches(self) -> int:
        return lib().pf_launch_count(self.h)

    # -- outputs ---------------------------------------------------------------
    def fields(self, dom: int = 0, names=FIELDS, out: np.ndarray | None = None) -> dict:
        mask = 0
        for nm in names:
            mask |= 1 << FIELDS.index(nm)
        sel = [nm for nm in FIELDS if mask & (1 << FIELDS.index(nm))]
        nx, ny = self.domains[dom]
        if out is None:
            out = np.empty(len(sel) * nx * ny)
        _check(lib().pf_get_fields(self.h, dom, mask, _dp(out), out.size), self.h)
        out = out[: len(sel) * nx * ny].reshape(len(sel), ny, nx)
        return {nm: out[i] for i, nm in enumerate(sel)}

    def run(self, f6: np.ndarray, n_steps: int, names=FIELDS,
            out: np.ndarray | None = None) -> dict:
        """pf_run: set the fields of the single domain from f6 (C-contiguous
        float64, shape (6, ny, nx): phi, psi, C, vx, vy, p), advance n_steps
        and return the named fields of the last step, with the host copies
        overlapped with the steps (page-locked f6 and out let them run beside
        the kernels).  out: optional float64 buffer of at least
        len(names) * nx * ny values."""
        if len(self.domains) != 1:
            raise ValueError("run takes a single-domain handle")
        nx, ny = self.domains[0]
        if (not isinstance(f6, np.ndarray) or f6.dtype != np.float64 or f6.shape != (6, ny, nx)
                or not f6.flags["C_CONTIGUOUS"]):
            raise ValueError(f"f6 must be a C-contiguous float64 array of shape (6, {ny}, {nx})")
        mask = 0
        for nm in names:
            mask |= 1 << FIELDS.index(nm)
        sel = [nm for nm in FIELDS if mask & (1 << FIELDS.index(nm))]
        if out is None:
            out = np.empty(len(sel) * nx * ny)
        _check(lib().pf_run(self.h, _dp(f6), nx * ny, int(n_steps), mask, _dp(out), out.size),
               self.h)
        out = out[: len(sel) * nx * ny].reshape(len(sel), ny, nx)
        return {nm: out[i] for i, nm in enumerate(sel)}

    @property
    def state_planes(self) -> int:
        return lib().pf_state_planes(self.h)

    def get_state(self, dom: int = 0) -> np.ndarray:
        nx, ny = self.domains[dom]
        npl = self.state_planes
        out = np.empty(npl * nx * ny)
        _check(lib().pf_get_state(self.h, dom, _dp(out), out.size), self.h)
        return out.reshape(npl, ny, nx)

    def set_temperature(self, dom: int, theta) -> None:
        """Thermal mode: temperature field theta ([ny][nx]) before the first step."""
        nx, ny = self.domains[dom]
        a = np.ascontiguousarray(np.broadcast_to(np.asarray(theta, dtype=np.float64), (ny, nx)))
        _check(lib().pf_set_temperature(self.h, dom, _dp(a), nx * ny), self.h)

    def reduce_thermal(self, dom: int = 0) -> dict:
        """Thermal mode: FP64 sum of the temperature populations (total rho H),
        sum theta and sum psi."""
        out = np.zeros(3)
        _check(lib().pf_reduce_thermal(self.h, dom, _dp(out)), self.h)
        return dict(zip(("sum_e", "sum_theta", "sum_psi"), out.tolist()))

    def set_state(self, dom: int, state: np.ndarray) -> None:
        a = np.ascontiguousarray(np.asarray(state, dtype=np.float64)).ravel()
        _check(lib().pf_set_state(self.h, dom, _dp(a), a.size), self.h)

    def adjoint_step(self, n_steps: int, w_solid: float = 1.0, w_centroid: float = 1.0,
                     checkpoint_every: int = 100) -> tuple[float, np.ndarray]:
        """Run n_steps forward with checkpoints, then the discrete adjoint:
        returns (J, dJ/d(eps_s, Omega, sigma))."""
        obj = pf_objective(float(w_solid), float(w_centroid), int(checkpoint_every))
        J = ctypes.c_double()
        g = np.zeros(3)
        _check(lib().pf_adjoint_step(self.h, int(n_steps), ctypes.byref(obj), ctypes.byref(J),
                                     _dp(g)), self.h)
        return J.value, g

    def reduce(self, dom: int = 0, probe=None) -> dict:
        d = pf_diag()
        pr = pf_probe(*probe) if probe is not None else None
        _check(lib().pf_reduce(self.h, dom, ctypes.byref(pr) if pr else None, ctypes.byref(d)),
               self.h)
        return {k: getattr(d, k) for k in _DIAG_FIELDS}


PF3_STATE_PLANES = 23
PF3_STATE_PLANES_THERMAL = 30


def _check3(code: int, handle=None) -> None:
    if code != PF_OK:
        raise PFError(code, lib().pf3_last_error(handle).decode(errors="replace"))


class Simulation3D:
    """Handle of the 3-D dendrite step (psi and C on D3Q7, periodic
    nx x ny x nz, no gas or flow); arrays are [z][y][x]."""

    def __init__(self, shape, params: dict | None = None, precision: str = "fp32", stream=None):
        nx, ny, nz = (int(v) for v in shape)
        self.shape = (nz, ny, nx)
        self.params = params_from_dict(params)
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream
            except Exception:
                stream = 0
        h = ctypes.c_void_p()
        _check3(lib().pf3_create(ctypes.byref(self.params), nx, ny, nz, PRECISIONS[precision],
                                 ctypes.c_void_p(stream), ctypes.byref(h)))
        self.h = h
        self.n = nx * ny * nz

    def close(self) -> None:
        if getattr(self, "h", None):
            code = lib().pf3_destroy(self.h)
            self.h = None
            _check3(code)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_seeds(self, seeds, R_s: float) -> None:
        s = np.ascontiguousarray(np.asarray(seeds, dtype=np.float64).reshape(-1, 3))
        _check3(lib().pf3_init_seeds(self.h, _dp(s), len(s), float(R_s)), self.h)

    def set_fields(self, psi, C) -> None:
        a = np.ascontiguousarray(np.asarray(psi, dtype=np.float64).reshape(self.shape))
        b = np.ascontiguousarray(np.asarray(C, dtype=np.float64).reshape(self.shape))
        _check3(lib().pf3_set_fields(self.h, _dp(a), _dp(b), self.n), self.h)

    def set_boundaries(self, bc) -> None:
        """Side types x-, x+, y-, y+, z-, z+ (BC_PERIODIC, BC_SYMMETRIC, BC_WALL,
        BC_FARFIELD), before initialising."""
        arr = (ctypes.c_int * 6)(*[int(b) for b in bc])
        _check3(lib().pf3_set_boundaries(self.h, arr), self.h)

    def set_orientation(self, seeds7) -> None:
        """Grain orientations: n x (x, y, z, qw, qx, qy, qz); each site takes the
        rotation of the nearest seed (empty: the lattice-aligned grain)."""
        s = np.ascontiguousarray(np.asarray(seeds7, dtype=np.float64).reshape(-1, 7))
        _check3(lib().pf3_set_orientation(self.h, _dp(s), len(s)), self.h)

    def set_temperature(self, theta) -> None:
        """Thermal mode: temperature field of the initial state ([z][y][x])."""
        a = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).reshape(self.shape))
        _check3(lib().pf3_set_temperature(self.h, _dp(a), self.n), self.h)

    def set_chunk(self, chunk: int) -> None:
        _check3(lib().pf3_set_chunk(self.h, int(chunk)), self.h)

    def set_index64(self, on: bool = True) -> None:
        """Take the 64-bit index form of the periodic step at any size
        (otherwise 32-bit while the state planes fit; results are identical)."""
        _check3(lib().pf3_set_index64(self.h, int(bool(on))), self.h)

    def step(self, n: int = 1) -> None:
        _check3(lib().pf3_step(self.h, int(n)), self.h)

    def fields(self, out: np.ndarray | None = None) -> dict:
        """psi, C, U (and theta in thermal mode), [z][y][x]; out: optional
        float64 buffer of at least field_planes * n values (e.g. page-locked)."""
        k = lib().pf3_field_planes(self.h)
        if out is None:
            out = np.empty(k * self.n)
        _check3(lib().pf3_get_fields(self.h, _dp(out), out.size), self.h)
        out = out.reshape(-1)[: k * self.n].reshape((k,) + self.shape)
        return dict(zip(("psi", "C", "U", "theta"), out))

    @property
    def field_planes(self) -> int:
        return lib().pf3_field_planes(self.h)

    def get_state(self) -> np.ndarray:
        k = lib().pf3_state_planes(self.h)
        out = np.empty(k * self.n)
        _check3(lib().pf3_get_state(self.h, _dp(out), out.size), self.h)
        return out.reshape((k,) + self.shape)

    def reduce(self) -> dict:
        out = np.zeros(2)
        _check3(lib().pf3_reduce(self.h, _dp(out)), self.h)
        return {"sum_C": out[0], "sum_hpsi": out[1]}

    def reduce_thermal(self) -> dict:
        """Thermal mode: FP64 sums of rho H (the seven populations), theta, psi."""
        out = np.zeros(3)
        _check3(lib().pf3_reduce_thermal(self.h, _dp(out)), self.h)
        return {"sum_e": out[0], "sum_theta": out[1], "sum_psi": out[2]}

    @property
    def launches(self) -> int:
        return lib().pf3_launch_count(self.h)


PF3F_STATE_PLANES = 66
PF3F_STATE_PLANES_THERMAL = 74
FIELDS_3F = ("phi", "psi", "C", "U", "p", "vx", "vy", "vz", "mu", "theta")


def _check3f(code: int, handle=None) -> None:
    if code != PF_OK:
        raise PFError(code, lib().pf3f_last_error(handle).decode(errors="replace"))


class Simulation3F:
    """Handle of the 3-D two-phase step (NS and CAC on D3Q19, psi and C on
    D3Q7, periodic nx x ny x nz); arrays are [z][y][x]; seeds (x, y, z),
    bubbles (x, y, z, R)."""

    def __init__(self, shape, params: dict | None = None, precision: str = "fp32", stream=None):
        nx, ny, nz = (int(v) for v in shape)
        self.shape = (nz, ny, nx)
        self.params = params_from_dict(params)
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream
            except Exception:
                stream = 0
        h = ctypes.c_void_p()
        _check3f(lib().pf3f_create(ctypes.byref(self.params), nx, ny, nz, PRECISIONS[precision],
                                   ctypes.c_void_p(stream), ctypes.byref(h)))
        self.h = h
        self.n = nx * ny * nz

    def close(self) -> None:
        if getattr(self, "h", None):
            code = lib().pf3f_destroy(self.h)
            self.h = None
            _check3f(code)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_spec(self, seeds, R_s: float, bubbles) -> None:
        s = np.ascontiguousarray(np.asarray(seeds, dtype=np.float64).reshape(-1, 3))
        b = np.ascontiguousarray(np.asarray(bubbles, dtype=np.float64).reshape(-1, 4))
        _check3f(lib().pf3f_init_spec(self.h, _dp(s), len(s), float(R_s), _dp(b), len(b)), self.h)

    def set_fields(self, phi, psi, C, vx=None, vy=None, vz=None, p=None) -> None:
        planes = [phi, psi, C] + [np.zeros(self.shape) if a is None else a for a in (vx, vy, vz, p)]
        a = np.ascontiguousarray(np.stack([np.asarray(q, dtype=np.float64).reshape(self.shape)
                                           for q in planes]))
        self.set_fields_stack(a)

    def set_fields_stack(self, f7: np.ndarray) -> None:
        """Initial fields from one C-contiguous float64 block of shape
        (7, nz, ny, nx) holding phi, psi, C, vx, vy, vz, p, passed to
        pf3f_set_fields without a copy on the host."""
        if (not isinstance(f7, np.ndarray) or f7.dtype != np.float64
                or f7.shape != (7,) + tuple(self.shape) or not f7.flags["C_CONTIGUOUS"]):
            raise ValueError(f"f7 must be a C-contiguous float64 array of shape (7, {self.shape})")
        _check3f(lib().pf3f_set_fields(self.h, _dp(f7), f7.size), self.h)

    @property
    def rho_bar(self) -> float:
        return lib().pf3f_get_rho_bar(self.h)

    def set_rho_bar(self, rho_bar: float) -> None:
        _check3f(lib().pf3f_set_rho_bar(self.h, float(rho_bar)), self.h)

    def set_boundaries(self, bc) -> None:
        """Side types x-, x+, y-, y+, z-, z+ (BC_PERIODIC, BC_SYMMETRIC, BC_WALL,
        BC_FARFIELD), before initialising."""
        arr = (ctypes.c_int * 6)(*[int(b) for b in bc])
        _check3f(lib().pf3f_set_boundaries(self.h, arr), self.h)

    def set_orientation(self, seeds7) -> None:
        """Grain orientations: n x (x, y, z, qw, qx, qy, qz) (empty: aligned)."""
        s = np.ascontiguousarray(np.asarray(seeds7, dtype=np.float64).reshape(-1, 7))
        _check3f(lib().pf3f_set_orientation(self.h, _dp(s), len(s)), self.h)

    def set_chunk(self, chunk: int) -> None:
        _check3f(lib().pf3f_set_chunk(self.h, int(chunk)), self.h)

    def set_index64(self, on: bool = True) -> None:
        """Take the 64-bit index form of the periodic step at any size
        (otherwise 32-bit while the state planes fit; results are identical)."""
        _check3f(lib().pf3f_set_index64(self.h, int(bool(on))), self.h)

    def step(self, n: int = 1) -> None:
        _check3f(lib().pf3f_step(self.h, int(n)), self.h)

    def fields(self, out: np.ndarray | None = None) -> dict:
        """FIELDS_3F planes, [z][y][x]; out: optional float64 buffer of at
        least field_planes * n values (e.g. page-locked)."""
        k = lib().pf3f_field_planes(self.h)
        if out is None:
            out = np.empty(k * self.n)
        _check3f(lib().pf3f_get_fields(self.h, _dp(out), out.size), self.h)
        return dict(zip(FIELDS_3F, out.reshape(-1)[: k * self.n].reshape((k,) + self.shape)))

    @property
    def field_planes(self) -> int:
        return lib().pf3f_field_planes(self.h)

    def get_state(self) -> np.ndarray:
        k = lib().pf3f_state_planes(self.h)
        out = np.empty(k * self.n)
        _check3f(lib().pf3f_get_state(self.h, _dp(out), out.size), self.h)
        return out.reshape((k,) + self.shape)

    def set_temperature(self, theta) -> None:
        """Thermal mode: temperature field of the initial state ([z][y][x])."""
        a = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).reshape(self.shape))
        _check3f(lib().pf3f_set_temperature(self.h, _dp(a), self.n), self.h)

    def reduce_thermal(self) -> dict:
        """Thermal mode: FP64 sums of rho H (the seven populations), theta, psi."""
        out = np.zeros(3)
        _check3f(lib().pf3f_reduce_thermal(self.h, _dp(out)), self.h)
        return {"sum_e": out[0], "sum_theta": out[1], "sum_psi": out[2]}

    def reduce(self) -> dict:
        out = np.zeros(3)
        _check3f(lib().pf3f_reduce(self.h, _dp(out)), self.h)
        return {"sum_phi": out[0], "sum_C": out[1], "sum_hpsi": out[2]}

    @property
    def launches(self) -> int:
        return lib().pf3f_launch_count(self.h)
