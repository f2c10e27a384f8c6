"""The hand-written reverse of the per-site update (pf_local.cuh, the core of
the discrete-adjoint kernel) agrees with central differences of the same
forward: compiled for the host with g++ and checked on 200 random sites for
random output adjoints, input directions and the three parameters."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_local_reverse_matches_central_differences(tmp_path):
    exe = tmp_path / "lac"
    subprocess.run(["g++", "-std=c++17", "-O1", "-o", str(exe),
                    os.path.join(HERE, "host", "local_adjoint_check.cpp")], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    lines = out.stdout.strip().splitlines()
    assert lines[-1] == "bad 0", out.stdout[-2000:]
    worst = [max(float(l.split()[k]) for l in lines[:-1]) for k in range(1, 5)]
    assert worst[0] < 1e-6      # inputs
    assert max(worst[1:]) < 1e-5  # eps_s, Omega, sigma
