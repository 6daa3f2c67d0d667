#!/usr/bin/env python
"""Throughput of the hybrid LBM / FENE-P time step on one GB300.

Workload (default): the weakly confined matrix-viscoelastic droplet,
192 x 96 x 80 lattice (W = 80, R = 16, 2R/W = 0.4, lambda = 1, De = 1,
L^2 = 100, eta_P/eta_M = 0.4, Ca = 0.2), FP32.  One bench step is one
lattice time step over the whole box (every population and conformation
component read and written once).  The state (about 0.6 GB) is larger than
the 129 MB L2, so no flush is needed between steps.

Printed JSON line: MLUPS (whole job), roofline of the step kernels against
the measured HBM bandwidth, the end-to-end MLUPS through the C ABI with the
initial densities copied from pinned host memory and the observables read
back inside the timed region, the FP64 CPU oracle timed on the host cores,
clocks sampled during the timed region and the kernel-launch count.

``--impl reference`` times the CPU oracle itself (the reference arm of this
method, which has no other implementation) on a bounded sample of the same
workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# per lattice update, each value read and written once: FP32 2x19 populations
# (304 B) + 6 conformation components (48 B); the reduced forms store the
# populations in 2 bytes (152 B) and keep the cell's two offset densities in
# FP32 (16 B)
ALGO_BYTES = {0: 352, 1: 216, 2: 216}
DTYPE = {0: "f32", 1: "f16-store/f32", 2: "bf16-store/f32"}
METRIC = "MLUPS"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="matrix_ve_192x96x80",
                    choices=["matrix_ve_192x96x80", "droplet_ve_256x128x64", "box_32cubed", "batched_64"])
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--precision", choices=["fp32", "fp16", "bf16"], default="fp32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--advection", choices=["upwind1", "upwind2"], default="upwind1",
                    help="u.grad C scheme: first-order upwind, or second-order minmod-limited upwind")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the sub-records of the other storage forms, config 3 and the 64-instance batch")
    ap.add_argument("--_oracle-timing", dest="oracle_timing", default=None, help=argparse.SUPPRESS)
    return ap.parse_args()


def workload(name: str, precision: int, advection: int = 0):
    """Instances (list of Params) and their initial densities."""
    from dataclasses import replace
    from paper_1411_2181_gb300 import configs
    if name == "batched_64":
        inst = configs.config4(64, seed=4)
        return ([replace(p, precision=precision, advection=advection) for p, _ in inst],
                [configs.config4_densities(p, sd) for p, sd in inst])
    if name == "matrix_ve_192x96x80":
        p, rho, _ = configs.config2(0.2)
    elif name == "droplet_ve_256x128x64":
        p, rho, _ = configs.config3()
    else:
        p, rho, _ = configs.config1()
    return [replace(p, precision=precision, advection=advection)], [rho]


def config_dict(name, ps):
    cells = sum(p.N for p in ps)
    if len(ps) > 1:
        return {"workload": name, "instances": len(ps), "cells": cells,
                "Lx_range": [min(p.Lx for p in ps), max(p.Lx for p in ps)],
                "W_range": [min(p.Lz for p in ps), max(p.Lz for p in ps)],
                "l2_policy": "state (>20 GB) larger than L2; no flush"}
    p = ps[0]
    return {"workload": name, "lattice": [p.Lx, p.Ly, p.Lz], "cells": cells, "W": p.Lz, "R": p.R,
            "visco_phase": ["newtonian", "droplet", "matrix"][p.visco_phase], "lambda": p.lambda_,
            "L2": p.L2, "Uw": p.Uw, "advection": ["upwind1", "upwind2"][p.advection],
            "l2_policy": "state (>0.5 GB) larger than L2; no flush"}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """SM clock and clock-event reasons of the benchmark's GPU while the
    timed region runs: read through NVML (read-only queries) on entry, every
    0.5 ms and on exit, the GPU found by its UUID; where NVML cannot be loaded, nvidia-smi every
    200 ms from 0.3 s before the region to 0.25 s after it."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # NVML clock-event reason bits
    REASON_BITS = ((0x4, "sw_power_cap"), (0x8, "hw_slowdown"), (0x20, "sw_thermal_slowdown"),
                   (0x40, "hw_thermal_slowdown"), (0x80, "hw_power_brake_slowdown"))

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.nvml = None
        self.samples = []
        self.max_mhz = None
        self.stop = threading.Event()

    def _nvml_open(self):
        import ctypes as ct
        import torch
        lib = ct.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            return None
        uuid = "GPU-" + str(torch.cuda.get_device_properties(self.idx).uuid)
        dev = ct.c_void_p()
        if lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ct.byref(dev)) != 0:
            return None
        mx = ct.c_uint()
        if lib.nvmlDeviceGetMaxClockInfo(dev, 1, ct.byref(mx)) == 0:   # 1: NVML_CLOCK_SM
            self.max_mhz = float(mx.value)
        reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        return lib, dev, reasons

    def _nvml_sample(self):
        import ctypes as ct
        lib, dev, reasons = self.nvml
        clk, bits = ct.c_uint(), ct.c_ulonglong()
        if lib.nvmlDeviceGetClockInfo(dev, 1, ct.byref(clk)) == 0 and reasons(dev, ct.byref(bits)) == 0:
            self.samples.append((float(clk.value), int(bits.value)))

    def _nvml_loop(self):
        while not self.stop.is_set():
            self._nvml_sample()
            time.sleep(0.0005)

    def __enter__(self):
        try:
            self.nvml = self._nvml_open()
        except Exception:
            self.nvml = None
        if self.nvml:
            self._nvml_sample()
            self.t = threading.Thread(target=self._nvml_loop, daemon=True)
            self.t.start()
            return self
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.nvml:
            self.stop.set()
            self.t.join(1.0)
            try:
                self._nvml_sample()
            except Exception:
                pass
            return False
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(2)
            except Exception:
                self.proc.kill()
        return False

    def summary(self):
        if self.nvml is not None:
            if not self.samples:
                return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["unsampled"], "samples": 0,
                        "sampler": "nvml"}
            reasons = {nm for bit, nm in self.REASON_BITS for _, b in self.samples if b & bit}
            return {"sm_mhz": statistics.median(c for c, _ in self.samples), "sm_max_mhz": self.max_mhz,
                    "reasons": sorted(reasons), "samples": len(self.samples), "sampler": "nvml, 0.5 ms"}
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm), "sampler": "nvidia-smi, 200 ms"}


# ---------------------------------------------------------------- roofline inputs
def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# sources of the step kernels (device code and their launch code); a
# profile summary stays valid while these are unchanged
STEP_SOURCES = ("lbfe_internal.cuh", "lbfe_step.cuh", "lbfe_fused.cu", "lbfe_fused2.cu")


def kernel_source_hash():
    """Hash of the step-kernel sources with comments and layout removed, so
    that a profile summary survives edits to comments only."""
    h = hashlib.sha256()
    for fn in STEP_SOURCES:
        src = open(os.path.join(ROOT, "paper_1411_2181_gb300", "csrc", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update(re.sub(r"\s+", " ", src).strip().encode())
    return h.hexdigest()[:16]


def profiled_traffic(workload_name: str, precision: int, advection: int = 0):
    """DRAM bytes per lattice update of the step from the committed ncu
    summary, if it was taken on the current kernel sources."""
    suffix = "_upwind2" if advection else ""
    fn = os.path.join(ROOT, "profiles",
                      f"step_{workload_name}_{['fp32', 'fp16', 'bf16'][precision]}{suffix}.md")
    if not os.path.exists(fn):
        return None, None
    txt = open(fn).read()
    m_h = re.search(r"kernel source hash:\s*`?([0-9a-f]{16})", txt)
    m_b = re.search(r"dram bytes per lattice update:\s*([0-9.]+)", txt)
    if not m_h or not m_b or m_h.group(1) != kernel_source_hash():
        return None, fn
    return float(m_b.group(1)), fn


# ---------------------------------------------------------------- CPU oracle
def oracle_timing_child(spec: str):
    """Run in a child process (its OpenMP thread count fixed by the
    environment): time the FP64 oracle, as it stands, on one case and print
    one JSON line."""
    import numpy as np
    from oracle import oracle as O
    d = json.loads(spec)
    ps, rhos = workload(d["workload"], 0)
    p, rho = ps[0], rhos[0]
    dz = min(p.Lz, int(d["planes"])) if d.get("planes") else p.Lz
    o = O.Oracle(dict(p.oracle_dict(), Lz=dz), np.ascontiguousarray(rho[:, :dz]))
    o.step(1)
    t = time.perf_counter()
    o.step(int(d["steps"]))
    dt = time.perf_counter() - t
    print(json.dumps({"mlups": p.Lx * p.Ly * dz * int(d["steps"]) / dt / 1e6, "seconds": dt,
                      "lattice": [p.Lx, p.Ly, dz]}))


def oracle_timings(cores: int):
    """The FP64 oracle on the host cores, single-threaded and on all cores:
    config 1 (32^3, 500 steps) and a 200-step slice of config 2 (the full
    192 x 96 plane over a z-slab of the box; a single thread takes about a
    minute per million cells, so the slab keeps that leg to seconds)."""
    cases = [("box_32cubed", 500, None), ("matrix_ve_192x96x80", 200, 4)]
    out = []
    for name, steps, planes in cases:
        for threads in (1, cores):
            env = dict(os.environ, OMP_NUM_THREADS=str(threads))
            spec = json.dumps({"workload": name, "steps": steps, "planes": planes})
            r = subprocess.run([sys.executable, os.path.abspath(__file__), "--_oracle-timing", spec],
                               capture_output=True, text=True, env=env, timeout=900)
            if r.returncode != 0:
                out.append({"workload": name, "threads": threads, "error": r.stderr.strip()[-300:]})
                continue
            d = json.loads(r.stdout.strip().splitlines()[-1])
            out.append({"workload": name, "steps": steps, "lattice": d["lattice"], "threads": threads,
                        "value": round(d["mlups"], 4), "unit": METRIC, "seconds": round(d["seconds"], 2)})
    return out


def cpu_baseline_record():
    """cpu_baseline of the JSON line: the all-core config-2 slice as the
    headline value, with all four timings beside it."""
    cores = os.cpu_count() or 1
    runs = oracle_timings(cores)
    head = next((r for r in runs if r.get("workload") == "matrix_ve_192x96x80" and r.get("threads") == cores
                 and "value" in r), None)
    return {"value": head["value"] if head else None, "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": ("FP64 oracle as it stands, OpenMP threads = 1 and = all host cores: config 1 "
                       "(32^3, 500 steps) and 200 steps of config 2 on its full 192 x 96 plane over a "
                       "4-plane z-slab (walls at both ends); value = the all-core config-2 slice"),
            "runs": runs}


# ---------------------------------------------------------------- ours
def reduce_max_ms(ms: float, device=None) -> float:
    """The timed region's duration as the max over ranks (replicas run the
    same work; the slowest sets the whole-job time).  One rank: unchanged."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return ms
    tt = torch.tensor([ms], dtype=torch.float64, device=device)
    tdist.all_reduce(tt, op=tdist.ReduceOp.MAX)
    return float(tt.item())


def whole_job_mlups(cells_per_rank: int, steps: int, t_max_ms: float, world: int) -> float:
    """Lattice updates of all ranks per second (weak scaling: every rank
    advances its own replica of the workload)."""
    return cells_per_rank * steps / (t_max_ms / 1e3) / 1e6 * world


def timed_steps(s, stream, steps: int, warmup: int, dist=False):
    """Warm-up, then `steps` steps bracketed by CUDA events on the solver's
    stream (barrier + synchronize on both sides); returns ms."""
    import torch
    for _ in range(warmup):
        s.step(1)
    torch.cuda.synchronize()
    if dist:
        import torch.distributed as tdist
        tdist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    s.step(steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        tdist.barrier()
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1)


def roofline_record(prec: int, ncell: int, ms_per_step: float, workload_name: str, advection: int):
    peak, peak_kind = measured_peak()
    algo = ALGO_BYTES[prec]
    achieved = algo * ncell / (ms_per_step / 1e3) / 1e9
    traffic_per_lup, prof_file = profiled_traffic(workload_name, prec, advection)
    return {"bound": "hbm", "kernel": "k_fused (whole time step in one kernel)",
            "achieved": round(achieved, 1), "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "algorithmic_bytes_per_lup": algo,
            "traffic": (round(traffic_per_lup * ncell) if traffic_per_lup else None),
            "traffic_source": os.path.relpath(prof_file, ROOT) if (prof_file and traffic_per_lup) else None}


def time_form(name: str, prec: int, steps: int, warmup: int, device: str, autotune_on: bool):
    """One sub-record: the workload `name` in storage form `prec`, autotuned,
    timed on its own stream with CUDA events (state resident in HBM)."""
    import torch
    from paper_1411_2181_gb300 import lbfe, autotune
    ps, rhos = workload(name, prec)
    ncell = sum(p.N for p in ps)
    shape = autotune.tune(ps, device=device, rho=rhos) if autotune_on else None
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = lbfe.Solver(ps, device=device, stream=stream)
        if shape:
            s.tune(shape["tile_y"], shape["z_chunk"], shape.get("kernel", 0))
        for k, r in enumerate(rhos):
            s.init(k, r)
        ms = timed_steps(s, stream, steps, warmup)
        st = s.check()
        launch = s.launch_config()
        s.close()
    del s
    torch.cuda.empty_cache()
    msps = ms / steps
    roof = roofline_record(prec, ncell, msps, name, 0)
    return {"workload": name, "dtype": DTYPE[prec], "cells": ncell, "steps": steps,
            "value": round(ncell * steps / (ms / 1e3) / 1e6, 2), "unit": METRIC, "ms_per_step": round(msps, 5),
            "roofline": {k: roof[k] for k in ("achieved", "peak", "unit", "frac", "algorithmic_bytes_per_lup",
                                              "traffic")},
            "launch": launch, "status": lbfe._lib.lbfe_status_str(st).decode()}


# the other forms of the metric: FP16 / BF16 storage beside FP32 on the
# headline lattice, the strongly confined 256 x 128 x 64 droplet in all three
# forms, and the 64-instance uneven batch in one persistent launch per step
FORMS = [("matrix_ve_192x96x80", 1), ("matrix_ve_192x96x80", 2),
         ("droplet_ve_256x128x64", 0), ("droplet_ve_256x128x64", 1), ("droplet_ve_256x128x64", 2),
         ("batched_64", 0), ("batched_64", 1)]


def run_ours(a):
    import numpy as np
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = world > 1
    if dist:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1411_2181_gb300 import build
    if rank == 0 or not dist:
        build.build()
    if dist:
        tdist.barrier()
    from paper_1411_2181_gb300 import lbfe, autotune
    prec = {"fp32": 0, "fp16": 1, "bf16": 2}[a.precision]
    adv = 1 if a.advection == "upwind2" else 0
    ps, rhos = workload(a.workload, prec, adv)
    ncell = sum(p.N for p in ps)
    shape = None
    if not a.no_autotune:
        shape = autotune.tune(ps, device=f"cuda:{local}", rho=rhos)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = lbfe.Solver(ps, device=f"cuda:{local}", stream=stream)
        if shape:
            s.tune(shape["tile_y"], shape["z_chunk"], shape.get("kernel", 0))
        for k, r in enumerate(rhos):
            s.init(k, r)
        with ClockSampler(local) as clk:
            ms = timed_steps(s, stream, a.steps, a.warmup, dist)
        st = s.check()
        launch = s.launch_config()
        launches = s.launches_per_step() * a.steps
        status = lbfe._lib.lbfe_status_str(st).decode()
        s.close()
    t_max = reduce_max_ms(ms, device=f"cuda:{local}")
    ms_per_step = t_max / a.steps
    value = whole_job_mlups(ncell, a.steps, t_max, world)

    # end to end through the C ABI: H2D of the initial densities from pinned
    # memory, the steps, and the observables read back, all timed
    e2e = None
    if not a.no_e2e:
        hosts = [torch.from_numpy(np.ascontiguousarray(r, dtype=np.float64)).pin_memory() for r in rhos]
        with torch.cuda.stream(stream):
            s2 = lbfe.Solver(ps, device=f"cuda:{local}", stream=stream)
            if shape:
                s2.tune(shape["tile_y"], shape["z_chunk"], shape.get("kernel", 0))
            for k, hbuf in enumerate(hosts):
                s2.init_from_host_ptr(k, hbuf.data_ptr())
            s2.step(2)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for k, hbuf in enumerate(hosts):
                s2.init_from_host_ptr(k, hbuf.data_ptr())
            s2.step(a.steps)
            for k in range(len(ps)):
                s2.observables(k)
            t1 = time.perf_counter()
            s2.close()
        e2e_mlups = ncell * a.steps / (t1 - t0) / 1e6 * world
        obs_bytes = sum(6 * p.Lx * 8 + 2 * 8 + 4 for p in ps)
        e2e = {"value": round(e2e_mlups, 2), "unit": METRIC,
               "h2d_bytes_per_step": int(sum(h.numel() for h in hosts) * 8 / a.steps),
               "d2h_bytes_per_step": int(obs_bytes / a.steps),
               "timed": "lbfe_init (pinned H2D of rho[2][N] float64) + lbfe_step(K) + lbfe_observables"}
    torch.cuda.empty_cache()

    roof = roofline_record(prec, ncell, ms_per_step, a.workload, adv)

    # the other forms, each timed on its own (one GPU only: the scaling runs
    # time the headline alone)
    forms = None
    if not a.no_forms and world == 1 and a.workload == "matrix_ve_192x96x80" and adv == 0:
        forms = []
        for name, fprec in FORMS:
            if (name, fprec) == (a.workload, prec):
                continue
            fsteps = max(3, a.steps // 20) if name == "batched_64" else a.steps
            try:
                forms.append(time_form(name, fprec, fsteps, max(3, a.warmup), f"cuda:{local}",
                                       not a.no_autotune))
            except Exception as e:   # recorded, not fatal: the headline stands on its own
                forms.append({"workload": name, "dtype": DTYPE[fprec], "error": str(e)[:300]})

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = cpu_baseline_record()

    if rank == 0:
        out = {"metric": METRIC, "value": round(value, 2), "unit": METRIC, "n_gpus": world,
               "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(ms_per_step, 5),
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": DTYPE[prec], "data": "synthetic (seeded droplet, NumPy PCG64)",
               "config": dict(config_dict(a.workload, ps), launch=launch), "roofline": roof, "cpu_baseline": cpu,
               "e2e": e2e, "clocks": clk.summary(), "gpu_launches": launches,
               "autotune": autotune_summary(shape), "forms": forms,
               "status": status,
               "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}
        print(json.dumps(out))
    if dist:
        tdist.destroy_process_group()


def autotune_summary(shape):
    """Fastest measured step time (ms) of each kernel variant and tile height
    over the z-chunks the autotuner tried on this GPU."""
    if not shape:
        return None
    best = {}
    for kern, ty, _zc, ms in shape.get("trials", []):
        key = f"{'pair' if kern else 'cell'}_32x{ty}"
        best[key] = round(min(ms, best.get(key, ms)), 5)
    return {"best_ms_per_step": best}


# ---------------------------------------------------------------- reference arm
def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    from oracle import oracle as O
    O.build()
    prec = {"fp32": 0, "fp16": 1, "bf16": 2}[a.precision]
    from paper_1411_2181_gb300 import configs
    ps, rhos = workload(a.workload, prec, 1 if a.advection == "upwind2" else 0)
    p, rho = ps[0], rhos[0]
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    d = p.oracle_dict()
    # each timed step: one oracle step on a z-slab of the box, sized so the
    # whole run stays within about two minutes
    probe = O.Oracle(dict(d, Lz=4), np.ascontiguousarray(rho[:, :4]))
    t = time.perf_counter(); probe.step(1); rate = p.Lx * p.Ly * 4 / (time.perf_counter() - t)
    per_step_s = 100.0 / max(1, a.steps + a.warmup)
    dz = int(max(2, min(p.Lz, rate * per_step_s / (p.Lx * p.Ly))))
    o = O.Oracle(dict(d, Lz=dz), np.ascontiguousarray(rho[:, :dz]))
    for _ in range(a.warmup):
        o.step(1)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        o.step(1)
    dt = time.perf_counter() - t0
    mlups = p.Lx * p.Ly * dz * a.steps / dt / 1e6
    sample = f"one FP64 oracle step per bench step on a {p.Lx}x{p.Ly}x{dz} slab of the workload"
    out = {"impl": "reference", "metric": METRIC, "value": round(mlups, 4), "unit": METRIC, "n_gpus": a.gpus,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(dt / a.steps * 1e3, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded droplet, NumPy PCG64)", "config": config_dict(a.workload, ps),
           "cpu_baseline": {"value": round(mlups, 4), "unit": METRIC, "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(mlups, 4), "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    args = parse()
    if args.oracle_timing:
        oracle_timing_child(args.oracle_timing)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)
