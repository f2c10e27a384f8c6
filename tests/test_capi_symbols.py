"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/pf.h declares.  Host-only entry points are called; nothing here
touches a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pf.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w]+\s*\**\s*(pf3?f?_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpf():
    from paper_2407_01651_gb300 import build as b
    b.build()
    return ctypes.CDLL(b.LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pf_create", "pf_init_fields", "pf_step", "pf_get_fields", "pf_destroy",
                     "pf_reduce", "pf_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libpf):
    missing = [n for n in declared_functions() if not hasattr(libpf, n)]
    assert not missing, missing


def test_binding_uses_the_same_names():
    from paper_2407_01651_gb300 import pf
    src = open(pf.__file__).read()
    for n in declared_functions():
        assert n in src, n


def test_host_only_parameter_map(libpf):
    from paper_2407_01651_gb300 import pf
    d = dict(Omega=0.55, k=0.15, D=0.1, tau0=320.0, W0=4.0)
    lam, mc, th = pf.pf_params_derived(d)
    assert abs(th + 0.55) < 1e-15
    assert abs(mc - (1 - 0.85 * 0.55)) < 1e-15
    assert abs(lam * (47 / 75) * 16 - 0.1 * 320) < 1e-12


def test_defaults_match_the_workload_parameters(libpf):
    from paper_2407_01651_gb300 import pf, workload
    p = pf.params_from_dict({})
    for k, v in workload.BASE_PARAMS.items():
        assert getattr(p, k) == v, k


def test_thermal_parameters_are_checked_before_any_device_work(libpf):
    """Thermal mode: rho_g c_p below 2/3 (unstable rest population), non-positive
    Le, or 16-bit storage are rejected by pf_create before it touches a GPU."""
    from paper_2407_01651_gb300 import pf
    doms = (pf.pf_domain * 1)(pf.pf_domain(16, 16, -1.0))
    h = ctypes.c_void_p()
    L = pf.lib()
    for over, prec in ((dict(thermal=1, cp=1.0), pf.PF_FP32),
                       (dict(thermal=1, Le=0.0), pf.PF_FP32),
                       (dict(thermal=2), pf.PF_FP32),
                       (dict(thermal=1), pf.PF_FP16_OFFSET),
                       (dict(thermal=1), pf.PF_BF16_OFFSET)):
        p = pf.params_from_dict(over)
        code = L.pf_create(ctypes.byref(p), doms, 1, prec, None, None, ctypes.byref(h))
        assert code == pf.PF_ERR_BAD_ARG, over
        assert L.pf_last_error(None)
    assert L.pf_state_planes(None) == -1


def test_every_entry_point_states_its_error_behaviour():
    """Each declaration of the header sits under a comment (its own, or the one
    over its group of declarations) that says what the call returns on bad
    input or failure: an Errors list, a NULL rule or a never-fails note."""
    text = open(HEADER).read()
    stated = re.compile(r"Errors|errors|BAD_ARG|NULL|[Nn]ever fails|-1 for")
    missing = []
    last_comment = ""
    for tok in re.finditer(r"/\*.*?\*/|^[^\n/#]*\b(pf3?f?_\w+)\s*\(", text, flags=re.S | re.M):
        if tok.group(0).startswith("/*"):
            last_comment = tok.group(0)
        elif tok.group(1) and not stated.search(last_comment):
            missing.append(tok.group(1))
    assert not missing, missing
