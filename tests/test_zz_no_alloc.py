"""pf_reduce_noalloc: the FP64 diagnostics for callers that cannot allocate
device memory (a plugin whose host framework owns the device-memory budget, a
loop that must not call cudaMalloc / cudaFree).  The field planes are device
memory owned by the caller (here: a PyTorch tensor); the library uses only
its fixed, file-scope scratch.  Checked against pf_reduce on the same fields,
twice in a row (the scratch keeps the previous call's contents), and checked
not to take any device memory.

Collected last on purpose: if it fails, a stop-at-first-failure run has
already run every other test."""
import gc
import math

import numpy as np
import pytest

from paper_2407_01651_gb300 import pf
from paper_2407_01651_gb300 import workload as wl

pytestmark = pytest.mark.gpu

EXACT = ("p_in_n", "p_out_n", "nonfinite", "max_v")


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_noalloc_reduce_matches_pf_reduce_twice(precision):
    import torch

    lay = wl.random_layout(96, 80, 2, 2, rng_seed=77, R_max=10)
    sim = pf.Simulation([(lay.nx, lay.ny)], lay.params, precision)
    sim.init_fields(0, lay.seeds, lay.R_s, lay.bubbles)
    sim.step(5)
    b = lay.bubbles[0]
    probe = (b[0], b[1], b[2], lay.params["W_phi"])
    ref = sim.reduce(0, probe)
    f = sim.fields(0)
    dtype = torch.float64 if precision == "fp64" else torch.float32
    # the eight planes of the documented field stack (phi .. mu_phi)
    planes = torch.tensor(np.stack([f[k] for k in pf.FIELDS[:8]]), dtype=dtype, device="cuda")
    n = lay.nx * lay.ny
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    for call in range(2):
        if call == 1:
            # The second call, after the kernels are loaded, allocates nothing:
            # the device's free memory does not shrink and torch's allocator
            # does not move.  The garbage collector is held off meanwhile, so
            # that an earlier test's handle cannot be freed in the middle.
            gc.collect()
            gc.disable()
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            torch_bytes0 = torch.cuda.memory_allocated()
        try:
            got = pf.pf_reduce_noalloc(planes.data_ptr(), precision == "fp64", n, 0, lay.nx,
                                       lay.ny, probe, stream)
            if call == 1:
                assert torch.cuda.mem_get_info()[0] >= free0
                assert torch.cuda.memory_allocated() == torch_bytes0
        finally:
            if call == 1:
                gc.enable()
        for k, v in ref.items():
            if k in EXACT:
                assert got[k] == v, k
            else:
                # same values, different summation order
                assert math.isclose(got[k], v, rel_tol=1e-12, abs_tol=1e-12), (k, got[k], v)
    # a second field stack placed at an offset in a wider plane stride
    wide = torch.zeros((8, n + 100), dtype=dtype, device="cuda")
    wide[:, 37:37 + n] = planes.reshape(8, n)
    got = pf.pf_reduce_noalloc(wide.data_ptr(), precision == "fp64", n + 100, 37, lay.nx,
                               lay.ny, None, stream)
    for k in ("sum_phi", "sum_C", "gas_y"):
        assert math.isclose(got[k], ref[k], rel_tol=1e-12), k
    sim.close()


def test_noalloc_rejects_lattices_beyond_its_scratch():
    import torch

    t = torch.zeros(8, dtype=torch.float32, device="cuda")
    with pytest.raises(pf.PFError) as e:
        pf.pf_reduce_noalloc(t.data_ptr(), False, 10**9, 0, 9000, 8000)
    assert e.value.code == pf.PF_ERR_BAD_ARG
    assert "capacity" in pf.lib().pf_last_error(None).decode()
