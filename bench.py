#!/usr/bin/env python
"""Throughput of the coupled gas-liquid-dendrite LB step on GB300.

Workload: the 4096 x 4096 periodic lattice with 64 dendrite seeds (R = 6,
orientation uniform in [0, pi/2)) and 128 non-overlapping bubbles (R uniform
in [8, 40]), FP32, the paper's Section-4 problem restated periodically
(``workload.growth_lattice``).  A step is one coupled LB step of every site.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on a bounded window of the same workload instead.

Multi-GPU: the path is run as independent replicas (one lattice per rank, no
data-path collective); value = all sites updated by all ranks / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os

# pf_run (the end-to-end measurement) gives each row band of the lattice its
# own stream; with the default 8 hardware work queues, streams share queues
# and the bands wait on one another in submission order.  Read when the CUDA
# context is created, so it is set before anything initialises CUDA.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coupled-step MLUPS at 4096² and % of HBM roofline; adjoint/forward time ratio"
# Algorithmic HBM bytes per lattice update of the step kernel: 39 planes read
# + 39 planes written (9 NS, 9 CAC, 5+5+1 dendrite, 5 solute, 5 lagged scalars)
# and 1 byte of grain id read.
# The 16-bit forms store the 33 population planes in 2 bytes and keep 7 lagged
# scalars (with psi) in FP32.
BYTES_PER_LU = {"fp32": 39 * 4 * 2 + 1, "fp64": 39 * 8 * 2 + 1,
                "fp16": (33 * 2 + 7 * 4) * 2 + 1, "bf16": (33 * 2 + 7 * 4) * 2 + 1}
DTYPE = {"fp32": "f32", "fp64": "f64", "fp16": "f16-storage/f32", "bf16": "bf16-storage/f32"}
# The strict algorithmic bytes per lattice update of the coupled step: 28
# populations and 6 temporal scalars read and written, and a 4-byte grain
# angle read (FP32 276 B); populations in 16 bits with FP32 scalars about 164
# B.  The library stores the time stretch's pre-collision populations and
# 1/a_s^2 besides (BYTES_PER_LU): the roofline's achieved rate takes the strict
# figure and the line also gives the fraction at the stored bytes.
STRICT_BYTES_PER_LU = {"fp32": 276, "fp16": 164, "bf16": 164, "fp64": 2 * 276 - 4}
# Thermal mode adds 5 temperature populations and the lagged H: 45 planes.
BYTES_PER_LU_THERMAL = {"fp32": 45 * 4 * 2 + 1, "fp64": 45 * 8 * 2 + 1}
KERNEL_SOURCES = ("paper_2407_01651_gb300/csrc/pf_step.cu",
                  "paper_2407_01651_gb300/csrc/pf_device.cuh",
                  "paper_2407_01651_gb300/csrc/pf_model.cuh",
                  "paper_2407_01651_gb300/csrc/pf_pull.cuh",
                  "paper_2407_01651_gb300/csrc/pf_site.cuh",
                  "paper_2407_01651_gb300/csrc/pf_v2.cuh",
                  "paper_2407_01651_gb300/csrc/pf_step_staged.cu")
# the 3-D two-phase step (its kernel, launch and default z-tile length)
KERNEL_SOURCES_3F = ("paper_2407_01651_gb300/csrc/pf_step3f.cuh",
                     "paper_2407_01651_gb300/csrc/pf_step3f.cu",
                     "paper_2407_01651_gb300/csrc/pf_d3.cuh",
                     "paper_2407_01651_gb300/csrc/pf_device.cuh")


def kernel_hash(sources=KERNEL_SOURCES) -> str:
    h = hashlib.sha256()
    for f in sources:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks() -> tuple[float, str]:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def recorded_traffic(precision: str, size: int, kind: str = "step", sources=KERNEL_SOURCES):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source."""
    path = os.path.join(ROOT, "profiles", f"{kind}_{precision}_{size}_traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
        if rec.get("kernel_hash") == kernel_hash(sources):
            return rec["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = None
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        idx = str(gpu_index)
        if vis:
            parts = [p.strip() for p in vis.split(",") if p.strip()]
            if gpu_index < len(parts):
                idx = parts[gpu_index]
        self.idx = idx

    def start(self, wait_s: float = 10.0):
        """Start sampling and wait for the first sample, so that nvidia-smi's
        own start-up (NVML initialisation) happens before the timed region."""
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", self.idx], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        t0 = time.time()
        while time.time() - t0 < wait_s:
            if self.proc.poll() is not None:
                break
            try:
                if os.path.getsize(self.path) > 0:
                    break
            except OSError:
                pass
            time.sleep(0.05)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        with open(self.path) as fh:
            for line in fh:
                cols = [c.strip() for c in line.split(",")]
                if len(cols) < 9:
                    continue
                try:
                    sm.append(float(cols[1]))
                    mx.append(float(cols[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, cols[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def workload_config(size: int, precision: str) -> dict:
    """The lattice workload both arms measure (growth_lattice at size^2)."""
    return {"workload": f"{size}x{size} periodic lattice, 64 seeds (R=6, theta~U[0,pi/2)), "
                        "128 bubbles (R~U[8,40]), seed 2",
            "lattice": [size, size], "precision": precision}


def cpu_oracle_sample(steps_hint: int, target_s: float, side: int | None = None,
                      cores: int | None = None, warm: int = 1) -> dict:
    """Time the FP64 oracle (test infrastructure, run as a child process) on a
    window of the 4096^2 workload (global coordinates, so the window holds the
    same seeds and bubbles); all host cores unless `cores` is given."""
    cores = cores or os.cpu_count() or 1
    code = f"""
import json, sys, time
sys.path.insert(0, {ROOT!r})
import oracle
from paper_2407_01651_gb300 import workload as wl
lay = wl.growth_lattice()
def make(s):
    o = oracle.Oracle(s, s, lay.params, window=(lay.nx, lay.ny, 1024, 1024))
    o.init_spec(lay.seeds, lay.R_s, lay.bubbles)
    return o
side = {side if side else 0}
if not side:
    o = make(256); t = time.perf_counter(); o.step(2); dt = (time.perf_counter() - t) / 2
    rate = 256 * 256 / dt
    side = int(min(2048, max(128, (rate * {target_s} / max({steps_hint}, 1)) ** 0.5)) // 32 * 32)
o = make(side)
o.step({warm})
t = time.perf_counter(); o.step({steps_hint}); dt = time.perf_counter() - t
small = wl.random_layout(48, 40, 2, 1, rng_seed=3, R_max=8)
ca = oracle.count_step_ops(lay.params, 48, 40, small.seeds, small.R_s, small.bubbles)
cb = oracle.count_step_ops(lay.params, 64, 40, small.seeds, small.R_s, small.bubbles)
flops = sum(cb.values()) - sum(ca.values())
print(json.dumps(dict(side=side, steps={steps_hint}, seconds=dt, flops_per_lu=flops / (16 * 40))))
"""
    env = dict(os.environ, OMP_NUM_THREADS=str(cores))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         check=True)
    rec = json.loads(out.stdout.strip().splitlines()[-1])
    mlups = rec["side"] ** 2 * rec["steps"] / rec["seconds"] / 1e6
    return {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle (gcc -O3, OpenMP over rows), {rec['side']}x{rec['side']} "
                      f"window at (1024, 1024) of the 4096^2 layout, {rec['steps']} steps "
                      f"after {warm}, in {rec['seconds']:.1f} s",
            "window": rec["side"], "steps": rec["steps"], "seconds": rec["seconds"],
            "flops_per_lu": rec["flops_per_lu"],
            "gflops": mlups * rec["flops_per_lu"] / 1e3,
            "flops_def": "operations of the oracle's step per lattice update (dense moment "
                         "transforms), counted by its instrumented-scalar build"}


def cpu_oracle_variant(kind: str, steps: int = 0) -> dict:
    """Time the FP64 oracle (a child process, all host cores) on a bounded
    sample of a variant workload: 'thermal' (a 768^2 window of the thermal
    4096^2 lattice), 'bounded' (a 768^2 lattice of the same recipe with the
    Section-4 sides, thermal), '3d' (a 96^3 melt with 8 seeds), '3d_thermal'
    (the same with the temperature lattice)."""
    cores = os.cpu_count() or 1
    steps = steps or {"thermal": 60, "bounded": 60, "3d": 120, "3d_thermal": 300,
                      "3d_flow": 160, "3d_flow_thermal": 140, "precision": 60,
                      "ensemble": 200}[kind]  # about 10 s of CPU work
    code = f"""
import json, sys, time
sys.path.insert(0, {ROOT!r})
import oracle
from paper_2407_01651_gb300 import workload as wl
kind = {kind!r}
if kind in ("3d_flow", "3d_flow_thermal"):
    n = 64
    seeds, R_s, bub = wl.flow_3d(n, 4, 8)
    p = {{k: wl.BASE_PARAMS[k] for k in oracle.PARAM_NAMES_3F}}
    if kind == "3d_flow_thermal":
        p.update(wl.THERMAL_PARAMS)
    o = oracle.Oracle3F(n, n, n, p)
    o.init_spec(seeds, R_s, bub)
    sites = n ** 3
    what = f"{{n}}^3 melt with 4 seeds and 8 bubbles (3-D two-phase oracle{{', thermal' if p['thermal'] else ''}})"
elif kind in ("3d", "3d_thermal"):
    n = 96
    seeds, R_s = wl.growth_3d(n, 8)
    p = {{k: wl.BASE_PARAMS[k] for k in oracle.PARAM_NAMES_3D}}
    if kind == "3d_thermal":
        p.update(wl.THERMAL_PARAMS)
    o = oracle.Oracle3D(n, n, n, p)
    o.init_spec(seeds, R_s)
    sites = n ** 3
    what = f"{{n}}^3 melt with 8 seeds (3-D oracle{{', thermal' if p['thermal'] else ''}})"
elif kind == "precision":
    lay = wl.single_seed_bubble(8192, 4096, rng_seed=1)
    s = 768
    o = oracle.Oracle(s, s, lay.params, window=(lay.nx, lay.ny, 4096 - s // 2, 2048 - s // 2))
    o.set_rho_bar(lay.params["rho_g"] + o.mean_phi_global(lay.bubbles) * (lay.params["rho_l"] - lay.params["rho_g"]))
    o.init_spec(lay.seeds, lay.R_s, lay.bubbles)
    sites = s * s
    what = f"{{s}}x{{s}} window around the seed of the 8192x4096 layout"
elif kind == "ensemble":
    lays = wl.ensemble_96()
    pick = [lays[0], lays[32], lays[64]]
    os_ = []
    for l in pick:
        oo = oracle.Oracle(l.nx, l.ny, dict(wl.BASE_PARAMS, eps_s=l.params["eps_s"]))
        oo.init_spec(l.seeds, l.R_s, l.bubbles)
        os_.append(oo)
    class _All:
        def step(self, n):
            for oo in os_:
                oo.step(n)
    o = _All()
    sites = sum(l.nx * l.ny for l in pick)
    what = "3 of the 96 domains (256^2, 512x384, 1024x512)"
else:
    lay = wl.growth_lattice()
    par = dict(lay.params, **wl.THERMAL_PARAMS)
    s = 768
    if kind == "thermal":
        o = oracle.Oracle(s, s, par, window=(lay.nx, lay.ny, 1024, 1024))
        what = f"{{s}}x{{s}} window of the thermal 4096^2 layout"
    else:
        lay = wl.random_layout(s, s, 3, 6, rng_seed=2)
        o = oracle.Oracle(s, s, par)
        o.set_bc(1, 1, 2, 3)
        what = f"{{s}}x{{s}} lattice, 3 seeds, 6 bubbles, Section-4 sides, thermal"
    o.init_spec(lay.seeds, lay.R_s, lay.bubbles)
    sites = s * s
o.step(1)
t = time.perf_counter(); o.step({steps}); dt = time.perf_counter() - t
print(json.dumps(dict(sites=sites, steps={steps}, seconds=dt, what=what)))
"""
    env = dict(os.environ, OMP_NUM_THREADS=str(cores))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         check=True)
    rec = json.loads(out.stdout.strip().splitlines()[-1])
    return {"value": rec["sites"] * rec["steps"] / rec["seconds"] / 1e6, "unit": "MLUPS",
            "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle (gcc -O3, OpenMP over rows), {rec['what']}, "
                      f"{rec['steps']} steps after 1, in {rec['seconds']:.1f} s"}


def timed_region(torch, stream, step, n: int, local: int, no_clocks: bool):
    """Time n steps with CUDA events on the launching stream, synchronised
    on both sides, with nvidia-smi clock samples taken during the region."""
    clocks = ClockSampler(local)
    if not no_clocks:
        clocks.start()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    step(n)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), clocks.stop()


def roofline(bpl: int, sites: int, ms_per_step: float, kernel: str, traffic=None,
             state_bpl: int | None = None) -> dict:
    """HBM roofline of the dominant kernel: algorithmic bytes per launch over
    the average launch time, against the measured copy bandwidth.  With
    state_bpl, the fraction at the bytes the library's state moves too."""
    peak, peak_kind = measured_peaks()
    achieved = bpl * sites / (ms_per_step / 1e3) / 1e9
    r = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
         "bytes_per_lu": bpl, "kernel": kernel}
    if state_bpl is not None:
        r["state_bytes_per_lu"] = state_bpl
        r["frac_at_state_bytes"] = state_bpl * sites / (ms_per_step / 1e3) / 1e9 / peak
    return r


def _pinned(torch, shape):
    return torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()


def e2e_2d(torch, sim, doms, steps: int, thermal: bool = False) -> dict:
    """End to end through the public API, every domain of the handle: the
    six fields (phi, psi, C, vx, vy, p; and theta in thermal mode) in from
    page-locked FP64 host memory (pf_set_fields, pf_set_temperature),
    pf_step(steps), the same fields back to page-locked host memory
    (pf_get_fields); host wall clock.  doms: [(dom, nx, ny)]."""
    names = ("phi", "psi", "C", "vx", "vy", "p")
    ins, ths, outs = [], [], []
    for d, nx, ny in doms:
        f = sim.fields(d, names + (("theta",) if thermal else ()))
        a = _pinned(torch, (6, ny, nx))
        for i, nm in enumerate(names):
            a[i] = f[nm]
        ins.append(a)
        if thermal:
            t = _pinned(torch, (ny, nx))
            t[...] = f["theta"]
            ths.append(t)
        outs.append(_pinned(torch, (6 * nx * ny,)))
    sites = sum(nx * ny for _, nx, ny in doms)
    one = len(doms) == 1 and not thermal
    if one:
        sim.run(ins[0], 2, ("phi", "psi", "C", "p", "vx", "vy"), out=outs[0])
    else:
        # touch the fresh page-locked outputs once, untimed (see e2e_3d)
        for k, (d, nx, ny) in enumerate(doms):
            sim.fields(d, ("phi", "psi", "C", "p", "vx", "vy"), out=outs[k])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if one:
        # pf_run: the three calls in one, the copies overlapped with the steps
        # (timed after one untimed call that sets up its streams and staging)
        sim.run(ins[0], steps, ("phi", "psi", "C", "p", "vx", "vy"), out=outs[0])
    else:
        for k, (d, nx, ny) in enumerate(doms):
            sim.set_fields_stack(d, ins[k])
            if thermal:
                sim.set_temperature(d, ths[k])
        sim.step(steps)
        for k, (d, nx, ny) in enumerate(doms):
            sim.fields(d, ("phi", "psi", "C", "p", "vx", "vy"), out=outs[k])
    e_s = time.perf_counter() - t0
    nb = (7 if thermal else 6) * 8 * sites
    what = ("pf_run: the FP64 host fields from page-locked memory, K steps and the fields back "
            "to page-locked memory in one call, the copies overlapped with the steps in row "
            "bands" if one else
            "pf_set_fields" + (" and pf_set_temperature" if thermal else "") +
            " from page-locked FP64 host fields, pf_step(K), pf_get_fields to page-locked "
            "FP64 host memory (written once before, untimed)")
    return {"value": sites * steps / e_s / 1e6, "unit": "MLUPS",
            "h2d_bytes_per_step": nb / steps, "d2h_bytes_per_step": 6 * 8 * sites / steps,
            "seconds": e_s,
            "what": what + "; host wall clock; grain angles are not re-sent (theta = 0)"}


def e2e_3d(torch, sim, steps: int, flow: bool, thermal: bool = False) -> dict:
    """End to end through the 3-D API: the initial fields in from page-locked
    FP64 host memory (pf3_set_fields: psi, C; pf3f_set_fields: phi, psi, C,
    vx, vy, vz, p; and the temperature in thermal mode), pf3[f]_step(steps),
    every field plane back to page-locked host memory; host wall clock."""
    f = sim.fields()
    shape = tuple(sim.shape)
    n = int(np.prod(shape))
    theta = None
    if thermal:
        theta = _pinned(torch, shape)
        theta[...] = f["theta"]
    if flow:
        names = ("phi", "psi", "C", "vx", "vy", "vz", "p")
        src = _pinned(torch, (7,) + shape)
        for i, nm in enumerate(names):
            src[i] = f[nm]
    else:
        psi, C = _pinned(torch, shape), _pinned(torch, shape)
        psi[...] = f["psi"]
        C[...] = f["C"]
    k = sim.field_planes
    out = _pinned(torch, (k * n,))
    # the first copy into freshly page-locked memory costs several times a
    # later one (the pages are mapped then): touch the output once, untimed
    sim.fields(out=out)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if flow:
        sim.set_fields_stack(src)
    else:
        sim.set_fields(psi, C)
    if thermal:
        sim.set_temperature(theta)
    sim.step(steps)
    sim.fields(out=out)
    e_s = time.perf_counter() - t0
    nin = (7 if flow else 2) + (1 if thermal else 0)
    return {"value": n * steps / e_s / 1e6, "unit": "MLUPS",
            "h2d_bytes_per_step": nin * 8 * n / steps, "d2h_bytes_per_step": k * 8 * n / steps,
            "seconds": e_s,
            "what": ("pf3f_set_fields" if flow else "pf3_set_fields") +
                    (" and the temperature" if thermal else "") +
                    " from page-locked FP64 host fields, step(K), every field plane to "
                    "page-locked FP64 host memory (written once before, untimed); host wall "
                    "clock"}


def run_reference(args) -> None:
    """The reference arm: the FP64 oracle itself, timed on the host cores on a
    bounded window of the 4096^2 workload (the paper publishes no code).  Each
    timed step is one oracle step of that window; value and ms_per_step are
    the window's own measurements."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    base = cpu_oracle_sample(steps_hint=args.steps, target_s=60.0, warm=args.warmup)
    side = base["window"]
    line = {
        "impl": "reference", "metric": METRIC, "value": base["value"], "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": base["seconds"] / base["steps"] * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{side}x{side} window at (1024, 1024) of the 4096x4096 periodic "
                               "lattice (64 seeds, 128 bubbles, seed 2), global coordinates",
                   "lattice": [side, side], "precision": "fp64",
                   "sample": f"{base['steps']} oracle steps of the window, after {args.warmup}"},
        "cpu_baseline": base,
        "e2e": {"value": base["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_adjoint_ratio(torch, pf, wl, stream, n_adj: int, K: int = 100) -> dict:
    """Adjoint / forward cost per step on the differentiation workload.
    ratio = time of pf_adjoint_step per step (its forward sweep, the
    recomputation from checkpoints and the reverse sweep) / time of pf_step
    per step.  kernel_only_ratio = reverse-step kernels per step / forward
    step per step, from an adjoint call over a single checkpoint segment (K
    steps: a forward sweep that keeps every state, no recomputation, the
    reverse sweep) minus its forward sweep."""
    lay4 = wl.growth_512()
    s4 = pf.Simulation([(lay4.nx, lay4.ny)], lay4.params, "fp32", stream=stream.cuda_stream)
    s4.init_fields(0, lay4.seeds, lay4.R_s, lay4.bubbles)
    cfg = s4.autotune(10)
    s4.set_launch(0, cfg[3], 0)
    s4.step(20)
    s4.sync()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    ev[0].record(stream)
    s4.step(n_adj)
    ev[1].record(stream)
    J, g = s4.adjoint_step(n_adj, 1.0, 1.0, K)
    ev[2].record(stream)
    s4.adjoint_step(K, 1.0, 1.0, K)
    ev[3].record(stream)
    s4.step(K)
    ev[4].record(stream)
    torch.cuda.synchronize()
    t_f = ev[0].elapsed_time(ev[1]) / n_adj
    t_a = ev[1].elapsed_time(ev[2]) / n_adj
    t_seg = ev[2].elapsed_time(ev[3]) / K
    t_f2 = ev[3].elapsed_time(ev[4]) / K
    s4.close()
    return {"workload": f"512x512, 4 seeds, 8 bubbles, FP32, {n_adj} steps, checkpoint every {K}",
            "forward_step_config": list(cfg),
            "forward_ms_per_step": t_f,
            "adjoint_call_ms_per_step": t_a,
            "ratio": t_a / t_f,
            "ratio_def": "pf_adjoint_step time per step (forward sweep, recomputation, reverse "
                         "sweep) / pf_step time per step",
            "reverse_ms_per_step": t_seg - t_f2,
            "kernel_only_ratio": (t_seg - t_f2) / t_f2,
            "kernel_only_def": "(adjoint call over one checkpoint segment - its forward sweep) "
                               "per step / forward step",
            "grad": g.tolist()}


def _time_steps(torch, sim, stream, n):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sim.sync()
    e0.record(stream)
    sim.step(n)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def run_ensemble(args) -> None:
    """96 independent domains of uneven size (32 each of 256^2, 512x384,
    1024x512; 1-4 seeds, 1-6 bubbles, eps_s ~ U[0.02, 0.07]) in one handle:
    one launch per domain per step vs one batched launch per step vs the
    autotuned batched launch replayed as CUDA graphs vs (the headline) the
    autotuned tiles with 64 steps in one persistent cooperative launch,
    replayed from a CUDA graph.  Under
    torchrun the domains are split across ranks (shard.shard_domains) with no
    collective on the data path; the job time is the slowest rank's."""
    import torch

    from paper_2407_01651_gb300 import pf
    from paper_2407_01651_gb300 import shard
    from paper_2407_01651_gb300 import workload as wl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    lays_all = wl.ensemble_96()
    sizes = [l.nx * l.ny for l in lays_all]
    parts = shard.shard_domains(sizes, world)
    lays = [lays_all[d] for d in parts[rank]]
    stream = torch.cuda.current_stream()
    sim = pf.Simulation([(l.nx, l.ny, l.params["eps_s"]) for l in lays], wl.BASE_PARAMS, "fp32",
                        stream=stream.cuda_stream)
    for d, l in enumerate(lays):
        sim.init_fields(d, l.seeds, l.R_s, l.bubbles)
    units = [sum(sizes[d] for d in p) for p in parts]
    my_sites = units[rank]

    def timed(clk=False):
        if dist is not None:
            dist.barrier()
        ms, c = timed_region(torch, stream, sim.step, args.steps, local, args.no_clocks or not clk)
        if dist is not None:
            dist.barrier()
        return shard.max_over_ranks(ms, dist, device="cuda"), c

    res, ms_mode = {}, {}
    sim.set_launch(1, 0, 0)
    sim.step(args.warmup)
    ms, _ = timed()
    res["sequential_per_domain"] = shard.job_rate(units, args.steps, ms / 1e3) / 1e6
    ms_mode["sequential_per_domain"] = ms / args.steps
    sim.set_launch(0, 0, 0)
    sim.step(args.warmup)
    ms, _ = timed()
    res["batched_one_launch"] = shard.job_rate(units, args.steps, ms / 1e3) / 1e6
    ms_mode["batched_one_launch"] = ms / args.steps
    cfg = sim.autotune(10)
    sim.set_launch(0, cfg[3], 64)
    sim.step(args.warmup)
    ms, _ = timed()
    res["batched_autotuned_graph"] = shard.job_rate(units, args.steps, ms / 1e3) / 1e6
    ms_mode["batched_autotuned_graph"] = ms / args.steps
    # the headline: every 64 steps in one persistent cooperative launch,
    # replayed from a CUDA graph, with the y-march chunk timed in that mode
    best = None
    for chunk in (16, 24, 32, 48, 64):
        sim.set_step_config(1, chunk, 0)
        sim.set_launch(0, 2, 0)
        sim.step(2)
        t_ms, _ = timed_region(torch, stream, sim.step, 20, local, True)
        if best is None or t_ms < best[0]:
            best = (t_ms, chunk)
    cfg_one = [1, best[1], 0, 2]
    sim.set_step_config(1, best[1], 0)
    sim.set_launch(0, 2, 64)
    sim.step(args.warmup)
    launches0 = sim.launches
    ms, clk = timed(clk=True)
    launches = sim.launches - launches0
    res["one_persistent_launch_graph"] = shard.job_rate(units, args.steps, ms / 1e3) / 1e6
    ms_mode["one_persistent_launch_graph"] = ms / args.steps
    e2e = None
    if not args.no_e2e:
        e2e = e2e_2d(torch, sim, [(d, l.nx, l.ny) for d, l in enumerate(lays)], args.steps)
        if dist is not None:
            t = torch.tensor([e2e["seconds"]], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e["value"] = sum(units) * args.steps / float(t.item()) / 1e6
    if rank == 0:
        cpu = None if (args.no_cpu_baseline or world > 1) else cpu_oracle_variant("ensemble")
        print(json.dumps({
            "metric": "ensemble aggregate MLUPS (96 uneven domains)",
            "value": res["one_persistent_launch_graph"],
            "unit": "MLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "96 domains: 32 x 256^2, 32 x 512x384, 32 x 1024x512, seed 5",
                       "sites": sum(sizes), "autotuned": list(cfg), "graph_steps": 64,
                       "launch": "64 steps per persistent cooperative launch, graph replay",
                       "autotuned_one_launch": cfg_one,
                       "parallelism": f"domains sharded over {world} rank(s)",
                       "l2": f"{313 * my_sites / 1e9:.1f} GB read+written per step > L2 "
                             "(no flush)"},
            "roofline": roofline(STRICT_BYTES_PER_LU["fp32"], my_sites, ms / args.steps,
                                 "k_step_ymarch_steps (64 steps per cooperative launch, every "
                                 "domain's tiles)", state_bpl=BYTES_PER_LU["fp32"]),
            "modes": res, "ms_per_step_modes": ms_mode,
            "speedup_vs_sequential": res["one_persistent_launch_graph"] /
            res["sequential_per_domain"],
            "speedup_vs_one_launch_per_step": res["one_persistent_launch_graph"] /
            res["batched_one_launch"],
            "gpu_launches": launches, "clocks": clk, "e2e": e2e, "cpu_baseline": cpu}))
    sim.close()
    if dist is not None:
        dist.destroy_process_group()


def run_precision(args) -> None:
    """8192 x 4096 seeded like the 128^2 case (one seed, one bubble): the
    16-bit offset storage forms against FP32, each timed over the same steps.
    The headline is the FP16 form."""
    import torch

    from paper_2407_01651_gb300 import pf
    from paper_2407_01651_gb300 import workload as wl

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    lay = wl.single_seed_bubble(8192, 4096, rng_seed=1)
    stream = torch.cuda.current_stream()
    sites = lay.nx * lay.ny
    out, clk, e2e = {}, None, None
    for prec in ("fp32", "bf16", "fp16"):
        sim = pf.Simulation([(lay.nx, lay.ny)], lay.params, prec, stream=stream.cuda_stream)
        sim.init_fields(0, lay.seeds, lay.R_s, lay.bubbles)
        sim.step(args.warmup)
        launches0 = sim.launches
        ms, c = timed_region(torch, stream, sim.step, args.steps, local,
                             args.no_clocks or prec != "fp16")
        bpl = BYTES_PER_LU[prec]
        out[prec] = {"mlups": sites * args.steps / ms / 1e3,
                     "ms_per_step": ms / args.steps,
                     "algorithmic_gbs": bpl * sites * args.steps / ms / 1e6,
                     "bytes_per_lu": bpl, "gpu_launches": sim.launches - launches0,
                     "step_config": list(sim.step_config())}
        if prec == "fp16":
            clk = c
            if not args.no_e2e:
                e2e = e2e_2d(torch, sim, [(0, lay.nx, lay.ny)], args.steps)
        sim.close()
        torch.cuda.empty_cache()
    f16 = out["fp16"]
    print(json.dumps({
        "metric": "precision-form MLUPS at 8192x4096", "value": f16["mlups"],
        "unit": "MLUPS", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": f16["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE["fp16"], "data": "synthetic",
        "config": {"workload": "8192x4096, one seed + one R=16 bubble (seed 1)",
                   "lattice": [lay.nx, lay.ny], "precision": "fp16",
                   "l2": f"{(BYTES_PER_LU['fp16'] - 1) * sites / 1e9:.1f} GB read+written per "
                         "step > L2 (no flush)"},
        "roofline": roofline(STRICT_BYTES_PER_LU["fp16"], sites, f16["ms_per_step"],
                             "k_step_staged<__half,float> (one launch per step)",
                             recorded_traffic("fp16", 4096) and
                             recorded_traffic("fp16", 4096) * sites / 4096 ** 2,
                             state_bpl=BYTES_PER_LU["fp16"]),
        "forms": out, "speedup_fp16_vs_fp32": f16["mlups"] / out["fp32"]["mlups"],
        "speedup_bf16_vs_fp32": out["bf16"]["mlups"] / out["fp32"]["mlups"],
        "gpu_launches": f16["gpu_launches"], "clocks": clk, "e2e": e2e,
        "cpu_baseline": None if args.no_cpu_baseline else cpu_oracle_variant("precision")}))


def _thermal_like(args, mode: str) -> None:
    """The 4096^2 lattice with the temperature lattice on (Le = 50, c_p^s /
    c_p = 1, theta0 = -Omega, Section 4 of the paper), periodic ('thermal') or
    with the paper's Section-4 sides ('bounded': symmetric in x, a no-flux wall
    at the bottom, the far field at the top), against the periodic isothermal
    (for 'thermal') or thermal (for 'bounded') step in the same process."""
    import torch

    from paper_2407_01651_gb300 import pf
    from paper_2407_01651_gb300 import workload as wl

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    prec = args.precision if args.precision in BYTES_PER_LU_THERMAL else "fp32"
    lay = wl.growth_lattice(args.size, args.size)
    par = dict(lay.params, **wl.THERMAL_PARAMS)
    stream = torch.cuda.current_stream()
    sites = lay.nx * lay.ny
    sides = (pf.BC_SYMMETRIC, pf.BC_SYMMETRIC, pf.BC_WALL, pf.BC_FARFIELD)
    if mode == "thermal":
        runs = (("thermal", par, None, BYTES_PER_LU_THERMAL[prec]),
                ("isothermal", lay.params, None, BYTES_PER_LU[prec]))
    else:
        runs = (("bounded", par, sides, BYTES_PER_LU_THERMAL[prec]),
                ("periodic", par, None, BYTES_PER_LU_THERMAL[prec]))
    res, clk, e2e = {}, None, None
    for name, p_, bc, bpl in runs:
        head = name == runs[0][0]
        sim = pf.Simulation([(lay.nx, lay.ny)], p_, prec, stream=stream.cuda_stream)
        if bc:
            sim.set_boundaries(0, *bc)
        sim.init_fields(0, lay.seeds, lay.R_s, lay.bubbles)
        th = p_.get("thermal", 0)
        d0 = sim.reduce(0)
        t0 = sim.reduce_thermal(0) if th else None
        sim.step(args.warmup)
        launches0 = sim.launches
        ms, c = timed_region(torch, stream, sim.step, args.steps, local,
                             args.no_clocks or not head)
        launches = sim.launches - launches0
        d = sim.reduce(0)
        if d["nonfinite"]:
            raise SystemExit(f"{name}: non-finite fields after the timed run")
        r = {"mlups": sites * args.steps / ms / 1e3, "ms_per_step": ms / args.steps,
             "bytes_per_lu": bpl, "algorithmic_gbs": bpl * sites * args.steps / ms / 1e6,
             "gpu_launches": launches,
             "sum_phi_rel_drift": d["sum_phi"] / d0["sum_phi"] - 1.0,
             "sum_C_rel_drift": d["sum_C"] / d0["sum_C"] - 1.0}
        if t0 is not None:
            t = sim.reduce_thermal(0)
            r["sum_rhoH_rel_drift"] = t["sum_e"] / t0["sum_e"] - 1.0
            r["mean_theta"] = t["sum_theta"] / sites
        if head:
            clk = c
            if not args.no_e2e:
                e2e = e2e_2d(torch, sim, [(0, lay.nx, lay.ny)], args.steps, thermal=True)
        res[name] = r
        sim.close()
        torch.cuda.empty_cache()
    h = res[runs[0][0]]
    if mode == "thermal":
        metric = "thermal coupled-step MLUPS at 4096² and % of HBM roofline"
        kernel = "k_step_ymarch<thermal> (one launch per step)"
        traffic = recorded_traffic(f"thermal_{prec}", args.size)
        extra = {"thermal_cost_vs_isothermal": res["isothermal"]["mlups"] / h["mlups"]}
        cfg = dict(workload_config(lay.nx, prec), thermal=wl.THERMAL_PARAMS)
    else:
        metric = "bounded thermal coupled-step MLUPS at 4096² and % of HBM roofline"
        kernel = ("k_step_ymarch<thermal> on interior tiles + k_step_ymarch_bc<thermal> on edge "
                  "tiles (side stream)")
        traffic = None
        extra = {}
        cfg = dict(workload_config(lay.nx, prec), thermal=wl.THERMAL_PARAMS,
                   boundaries="x: symmetric | y-: wall | y+: far field")
    cfg["l2"] = f"{(h['bytes_per_lu'] - 1) * sites / 1e9:.1f} GB read+written per step > L2 (no flush)"
    print(json.dumps({
        "metric": metric, "value": h["mlups"], "unit": "MLUPS", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": h["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[prec],
        "data": "synthetic", "config": cfg,
        "roofline": roofline(h["bytes_per_lu"], sites, h["ms_per_step"], kernel, traffic),
        "modes": res, **extra, "gpu_launches": h["gpu_launches"], "clocks": clk, "e2e": e2e,
        "cpu_baseline": None if args.no_cpu_baseline else cpu_oracle_variant(mode)}))


def run_bounded(args) -> None:
    _thermal_like(args, "bounded")


def run_thermal(args) -> None:
    _thermal_like(args, "thermal")


def run_3d(args) -> None:
    """The 3-D dendrite step (psi and C on D3Q7, no gas or flow) on a periodic
    256^3 melt with 64 seeds: MLUPS and the HBM roofline at 184 B/LU (FP32: 23
    planes read and written, g_pre[7], g_post[7], r, s[7], Q_psi); with the
    temperature lattice ('3d_thermal') 240 B/LU (30 planes, e[7] added)."""
    import torch

    from paper_2407_01651_gb300 import pf
    from paper_2407_01651_gb300 import workload as wl

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    n = args.size if args.size != 4096 else 256
    seeds, R_s = wl.growth_3d(n)
    stream = torch.cuda.current_stream()
    prec = args.precision if args.precision in ("fp32", "fp64") else "fp32"
    thermal = args.workload == "3d_thermal"
    params = dict(wl.BASE_PARAMS, **wl.THERMAL_PARAMS) if thermal else wl.BASE_PARAMS
    sim = pf.Simulation3D((n, n, n), params, prec, stream=stream.cuda_stream)
    sim.init_seeds(seeds, R_s)
    if args.chunk:
        sim.set_chunk(args.chunk)
    d0 = sim.reduce()
    t0 = sim.reduce_thermal() if thermal else None
    sim.step(args.warmup)
    l0 = sim.launches
    ms, clk = timed_region(torch, stream, sim.step, args.steps, local, args.no_clocks)
    launches = sim.launches - l0
    d = sim.reduce()
    sites = n ** 3
    planes = 30 if thermal else 23
    bpl = planes * 2 * (4 if prec == "fp32" else 8)
    extra = {}
    if thermal:
        t1 = sim.reduce_thermal()
        extra = {"sum_rhoH_rel_drift": t1["sum_e"] / t0["sum_e"] - 1.0,
                 "mean_theta": t1["sum_theta"] / sites}
    e2e = None if args.no_e2e else e2e_3d(torch, sim, args.steps, flow=False, thermal=thermal)
    print(json.dumps({
        "metric": ("3-D thermal dendrite-step" if thermal else "3-D dendrite-step") +
                  " MLUPS at 256³ and % of HBM roofline",
        "value": sites * args.steps / ms / 1e3, "unit": "MLUPS", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[prec], "data": "synthetic",
        "config": {"workload": f"{n}^3 periodic melt, 64 seeds (R=8) at uniform positions, seed 4"
                               + (", temperature lattice (Le 50, theta0 -0.55)" if thermal else ""),
                   "lattice": [n, n, n], "precision": prec,
                   "l2": f"{bpl * sites / 1e9:.1f} GB read+written per step > L2 (no flush)"},
        "roofline": roofline(bpl, sites, ms / args.steps, "k_step3d (one launch per step)"),
        "sum_C_rel_drift": d["sum_C"] / d0["sum_C"] - 1.0,
        "solid_fraction": d["sum_hpsi"] / sites, **extra,
        "gpu_launches": launches, "clocks": clk, "e2e": e2e,
        "cpu_baseline": None if args.no_cpu_baseline else
        cpu_oracle_variant("3d_thermal" if thermal else "3d")}))
    sim.close()


def run_3d_flow(args) -> None:
    """The 3-D two-phase step (NS and CAC on D3Q19, psi and C on D3Q7) on a
    periodic 256^3 melt with 32 seeds and 64 bubbles: MLUPS and the HBM
    roofline at 528 B/LU (FP32: 66 planes read and written, f[19], h[19],
    g_pre[7], g_post[7], s[7], r, Q_psi, phi_o, C_o, v_o[3])."""
    import torch

    from paper_2407_01651_gb300 import pf
    from paper_2407_01651_gb300 import workload as wl

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    n = args.size if args.size != 4096 else 256
    seeds, R_s, bubbles = wl.flow_3d(n)
    stream = torch.cuda.current_stream()
    prec = args.precision if args.precision in ("fp32", "fp64") else "fp32"
    thermal = args.workload == "3d_flow_thermal"
    params = dict(wl.BASE_PARAMS, **wl.THERMAL_PARAMS) if thermal else wl.BASE_PARAMS
    sim = pf.Simulation3F((n, n, n), params, prec, stream=stream.cuda_stream)
    sim.init_spec(seeds, R_s, bubbles)
    if args.chunk:
        sim.set_chunk(args.chunk)
    d0 = sim.reduce()
    t0 = sim.reduce_thermal() if thermal else None
    sim.step(args.warmup)
    l0 = sim.launches
    ms, clk = timed_region(torch, stream, sim.step, args.steps, local, args.no_clocks)
    launches = sim.launches - l0
    d = sim.reduce()
    extra = {}
    if thermal:
        t1 = sim.reduce_thermal()
        extra = {"sum_rhoH_rel_drift": t1["sum_e"] / t0["sum_e"] - 1.0}
    sites = n ** 3
    bpl = (74 if thermal else 66) * 2 * (4 if prec == "fp32" else 8)
    e2e = None if args.no_e2e else e2e_3d(torch, sim, args.steps, flow=True, thermal=thermal)
    print(json.dumps({
        "metric": ("3-D thermal two-phase" if thermal else "3-D two-phase") +
                  " coupled-step MLUPS at 256³ and % of HBM roofline",
        "value": sites * args.steps / ms / 1e3, "unit": "MLUPS", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[prec], "data": "synthetic",
        "config": {"workload": f"{n}^3 periodic melt, 32 seeds (R=8) and 64 bubbles "
                               "(R~U[6,14]) at uniform positions, seed 5" +
                               (", temperature lattice (Le 50, theta0 -0.55)" if thermal else ""),
                   "lattice": [n, n, n], "precision": prec,
                   "l2": f"{bpl * sites / 1e9:.1f} GB read+written per step > L2 (no flush)"},
        "roofline": roofline(bpl, sites, ms / args.steps, "k_step3f (one launch per step)",
                             recorded_traffic(("thermal_" if thermal else "") + prec, n, "step3f",
                                              KERNEL_SOURCES_3F)),
        "sum_phi_rel_drift": d["sum_phi"] / d0["sum_phi"] - 1.0,
        "sum_C_rel_drift": d["sum_C"] / d0["sum_C"] - 1.0,
        "solid_fraction": d["sum_hpsi"] / sites, **extra,
        "gpu_launches": launches, "clocks": clk, "e2e": e2e,
        "cpu_baseline": None if args.no_cpu_baseline else
        cpu_oracle_variant("3d_flow_thermal" if thermal else "3d_flow")}))
    sim.close()


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--precision", default="fp32", choices=("fp32", "fp64", "fp16", "bf16"))
    ap.add_argument("--size", type=int, default=4096)
    ap.add_argument("--variant", type=int, default=None, help="step kernel traversal")
    ap.add_argument("--chunk", type=int, default=None, help="rows per y-march tile / tile a")
    ap.add_argument("--tile-b", type=int, default=0)
    ap.add_argument("--workload", default="lattice",
                    choices=("lattice", "ensemble", "precision", "thermal", "bounded", "3d",
                             "3d_thermal", "3d_flow", "3d_flow_thermal"),
                    help="lattice: the 4096^2 headline; ensemble: 96 uneven domains; "
                         "precision: 8192x4096 in FP32 / FP16 / BF16 storage; "
                         "thermal: the 4096^2 lattice with the temperature lattice on; "
                         "bounded: the same with the paper's Section-4 boundaries; "
                         "3d: the 3-D dendrite step on a 256^3 melt; "
                         "3d_thermal: the same with the temperature lattice; "
                         "3d_flow: the 3-D two-phase step (flow, bubbles, dendrites) on 256^3; "
                         "3d_flow_thermal: the same with the temperature lattice")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--adjoint-steps", type=int, default=2000)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "ensemble":
        run_ensemble(args)
        return
    if args.workload == "precision":
        run_precision(args)
        return
    if args.workload == "thermal":
        run_thermal(args)
        return
    if args.workload == "bounded":
        run_bounded(args)
        return
    if args.workload in ("3d", "3d_thermal"):
        run_3d(args)
        return
    if args.workload in ("3d_flow", "3d_flow_thermal"):
        run_3d_flow(args)
        return

    import numpy as np
    import torch

    from paper_2407_01651_gb300 import pf
    from paper_2407_01651_gb300 import workload as wl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    lay = wl.growth_lattice(args.size, args.size)
    stream = torch.cuda.current_stream()
    sim = pf.Simulation([(lay.nx, lay.ny)], lay.params, args.precision,
                        stream=stream.cuda_stream)
    sim.init_fields(0, lay.seeds, lay.R_s, lay.bubbles)
    if args.variant is not None:
        sim.set_step_config(args.variant, args.chunk or 64, args.tile_b)
    sites = lay.nx * lay.ny
    d_init = sim.reduce(0)
    sim.step(args.warmup)
    sim.sync()

    clocks = ClockSampler(local)
    if not args.no_clocks:
        clocks.start()
    barrier()
    torch.cuda.synchronize()
    launches0 = sim.launches
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    sim.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1)
    launches = sim.launches - launches0
    clk = clocks.stop()
    ms_max = ms
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
    d = sim.reduce(0)
    if d["nonfinite"]:
        raise SystemExit(f"non-finite fields after the timed run: {d['nonfinite']}")
    conservation = {"steps": args.warmup + args.steps,
                    "sum_phi_rel_drift": d["sum_phi"] / d_init["sum_phi"] - 1.0,
                    "sum_C_rel_drift": d["sum_C"] / d_init["sum_C"] - 1.0,
                    "reductions": "FP64 on the GPU"}

    ms_per_step = ms_max / args.steps
    value = world * sites * args.steps / (ms_max / 1e3) / 1e6
    bpl = BYTES_PER_LU[args.precision]
    roof = roofline(STRICT_BYTES_PER_LU[args.precision], sites, ms / args.steps,
                    "k_step (one launch per step; average over the timed region)",
                    recorded_traffic(args.precision, args.size), state_bpl=bpl)

    # end to end through the public API: fields in from pinned host memory,
    # steps, fields out to pinned host memory
    e2e = None
    if not args.no_e2e:
        names = ("phi", "psi", "C", "vx", "vy", "p")
        init = sim.fields(0, names)
        host_in = torch.empty((6, lay.ny, lay.nx), dtype=torch.float64, pin_memory=True)
        for i, nm in enumerate(names):
            host_in[i].copy_(torch.from_numpy(init[nm]))
        host_out = torch.empty(6 * sites, dtype=torch.float64, pin_memory=True)
        out_np = host_out.numpy()
        in_np = host_in.numpy()
        out_names = ("phi", "psi", "C", "p", "vx", "vy")
        # one untimed call sets up pf_run's band streams and device staging
        sim.run(in_np, 2, out_names, out=out_np)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.run(in_np, args.steps, out_names, out=out_np)
        t1 = time.perf_counter()
        e_s = t1 - t0
        if dist is not None:
            t = torch.tensor([e_s], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e_s = float(t.item())
        e2e = {"value": world * sites * args.steps / e_s / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": 6 * 8 * sites / args.steps,
               "d2h_bytes_per_step": 6 * 8 * sites / args.steps,
               "what": "pf_run: FP64 host fields in from pinned memory, K steps, the fields of "
                       "the last step out to pinned memory, the host copies overlapped with the "
                       "steps in row bands (one untimed call before); host wall clock"}

    # adjoint / forward cost on the differentiation workload (512^2, 4 seeds,
    # 8 bubbles, FP32, checkpoint every 100 steps), with the forward in its
    # autotuned traversal (the adjoint's forward and recomputation use it too)
    adj = None
    if not args.no_adjoint and rank == 0:
        adj = run_adjoint_ratio(torch, pf, wl, stream, args.adjoint_steps)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(steps_hint=40, target_s=20.0)
        one = cpu_oracle_sample(steps_hint=10, target_s=8.0, cores=1)
        cpu["one_core"] = {"value": one["value"], "unit": "MLUPS", "cores": 1,
                           "sample": one["sample"]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": dict(workload_config(lay.nx, args.precision),
                           parallelism=f"replicas x{world}",
                           l2=f"inputs {(bpl - 1) * sites / 1e9:.1f} GB read+written per step "
                              "> L2 (no flush)"),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "step_config": list(sim.step_config()),
            "adjoint": adj,
            "conservation": conservation,
            "clocks": clk,
        }
        print(json.dumps(line))
    sim.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
