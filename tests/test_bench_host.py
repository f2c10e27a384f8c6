"""Host-side logic of the benchmark line (no GPU): the roofline arithmetic and
the rule that a recorded DRAM traffic figure is reported only while the
kernel sources keep the hash it was captured on."""
import json
import os

import pytest


def _bench():
    import bench          # imported here: it sets CUDA_DEVICE_MAX_CONNECTIONS on import
    return bench


def test_roofline_arithmetic():
    b = _bench()
    peak, _ = b.measured_peaks()
    r = b.roofline(276, 4096 ** 2, 0.8627, "k", traffic=5.0e9, state_bpl=313)
    achieved = 276 * 4096 ** 2 / 0.8627e-3 / 1e9
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(achieved, rel=1e-12)
    assert r["frac"] == pytest.approx(achieved / peak, rel=1e-12)
    assert r["frac_at_state_bytes"] == pytest.approx(313 / 276 * achieved / peak, rel=1e-12)
    assert r["traffic"] == 5.0e9


@pytest.mark.parametrize("kind,key,size,sources", [
    ("step", "fp32", 4096, "KERNEL_SOURCES"),
    ("step", "fp16", 4096, "KERNEL_SOURCES"),
    ("step", "thermal_fp32", 4096, "KERNEL_SOURCES"),
    ("step3f", "fp32", 256, "KERNEL_SOURCES_3F"),
    ("step3f", "thermal_fp32", 256, "KERNEL_SOURCES_3F"),
])
def test_recorded_traffic_follows_the_source_hash(kind, key, size, sources, monkeypatch):
    b = _bench()
    src = getattr(b, sources)
    path = os.path.join(b.ROOT, "profiles", f"{kind}_{key}_{size}_traffic.json")
    with open(path) as fh:
        rec = json.load(fh)
    got = b.recorded_traffic(key, size, kind, src)
    if rec["kernel_hash"] == b.kernel_hash(src):
        assert got == rec["dram_bytes_per_launch"]
    else:
        assert got is None
    # a changed source (another hash) turns the figure off
    monkeypatch.setattr(b, "kernel_hash", lambda sources=None: "0" * 16)
    assert b.recorded_traffic(key, size, kind, src) is None
    # the record is per launch: bytes per site times the sites of one launch
    sites = size ** 2 if kind == "step" else size ** 3
    assert rec["dram_bytes_per_launch"] == pytest.approx(rec["bytes_per_site_measured"] * sites,
                                                         rel=1e-3)


def test_missing_record_gives_no_traffic():
    b = _bench()
    assert b.recorded_traffic("fp32", 123, "step3f", b.KERNEL_SOURCES_3F) is None


def test_reference_arm_other_ranks_exit_without_work():
    """Under torchrun only rank 0 runs and prints the reference arm; any other
    rank exits 0 at once and prints nothing."""
    import subprocess
    import sys
    b = _bench()
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(b.ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True,
                       text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
