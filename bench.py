"""Benchmark: electron particle-steps/s of the batched FP32-split PIC/MCC step.

Workload (default): 64 independent helium discharges advanced together, gaps
U(0.3, 2) mm at 150..2000 cells, 1e4..2e6 electrons each (log-uniform),
100..400 V, drift-diffusion or full-fluid ions, FP32 particles with FP64 field
solves; one bench step = one 100-step chunk (one CUDA graph).  Inputs are
seeded and synthetic.

One JSON line on rank 0.  --impl reference runs the FP64 CPU oracle on the
same workload instead (one PIC step over all discharges per bench step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading

import numpy as np
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_SPLIT = 48   # per particle-step: read c,o,v,id (28 B) + write c,o,v (20 B)
BYTES_FP64 = 72    # read z,v,id (40 B) + write z,v (32 B)
CHUNK = 100
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal
TUNE_KEYS = ("lanes", "sort_interval", "blocks_per_sm", "field_threads", "field_cluster", "electron_threads",
             "particles_per_thread")
METRIC = "electron particle-steps/s, FP32-batched vs FP64 plain, 1 GB300; p50/p99 latency"


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def source_hash(text):
    """First 16 hex digits of the sha256 of CUDA source text with its comments
    and blank space removed (a comment edit leaves the compiled kernel, and so
    a profile of it, unchanged)."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    text = " ".join(text.split())
    return hashlib.sha256(text.encode()).hexdigest()[:16]


def kernel_hash():
    """source_hash of what the electron kernel is compiled from: its file, the
    device headers it includes, and the nvcc flags (without paths)."""
    sys.path.insert(0, ROOT)
    from paper_1508_02892_gb300 import build
    csrc = os.path.join(ROOT, "paper_1508_02892_gb300", "csrc")
    parts = []
    for name in ("hyb_electron.cu", "hyb_internal.cuh", "hyb_device.cuh"):
        with open(os.path.join(csrc, name)) as f:
            parts.append(f.read())
    flags = [t for t in build._flags() if not os.path.isabs(t)]
    return source_hash("\n".join(parts) + "\nnvcc " + " ".join(flags))


def electron_profile_value(key):
    """A per-push figure (`dram_bytes_per_push`, `warp_instructions_per_push`)
    of the electron kernel from the committed ncu summary, if it was taken on
    the current kernel source."""
    path = os.path.join(ROOT, "profiles", "electron_split_config3_ncu.txt")
    try:
        kv = {}
        with open(path) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = (v.split() or [""])[0]
        if kv.get("kernel_source_sha256_16") != kernel_hash():
            return None
        return float(kv[key])
    except Exception:
        return None


def traffic_per_push():
    """DRAM bytes per particle push of the electron kernel (committed ncu summary)."""
    return electron_profile_value("dram_bytes_per_push")


def issue_roofline(per_launch, avg_ms, sm_mhz):
    """The electron kernel against its instruction-issue ceiling: warp
    instructions per push (committed ncu summary) x pushes per launch / launch
    time, against every SM sub-partition issuing one warp instruction per cycle
    at the median SM clock sampled during the timed region."""
    import torch
    ipp = electron_profile_value("warp_instructions_per_push")
    if ipp is None or not sm_mhz:
        return None
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    peak = sms * 4 * sm_mhz * 1e6
    achieved = ipp * per_launch / (avg_ms / 1e3)
    return {"bound": "alu", "unit": "warp instructions/s", "warp_instructions_per_push": ipp,
            "achieved": achieved, "peak": peak, "frac": achieved / peak,
            "peak_note": f"{sms} SMs x 4 sub-partitions x 1 warp instruction per cycle x {sm_mhz:.0f} MHz"}


def workload(rank=0, n_inst=64, scale=1.0):
    from paper_1508_02892_gb300 import shard, workloads as W
    return W.config3_instances(n=n_inst, seed=shard.instance_seed(rank), scale=scale)


def _oracle_worker(conn, plist):
    """One host core's share of the discharges: build their oracles, then on
    each request step all of them by one PIC step and report (particle-steps,
    seconds)."""
    import oracle
    sims = [oracle.Oracle(p) for p in plist]
    conn.send("ready")
    while True:
        msg = conn.recv()
        if msg is None:
            break
        n = 0
        t0 = time.perf_counter()
        for o in sims:
            n += o.n_particles
            o.step(1)
        conn.send((n, time.perf_counter() - t0))
    for o in sims:
        o.close()


class OraclePool:
    """The oracle, as it stands, on the host cores: the discharges are dealt to
    one process per core (largest first, to the least loaded), each process
    steps its own, and a step of the pool is one PIC step of every discharge.
    Processes are started with `spawn` (never forked from a process that has
    used the GPU)."""

    def __init__(self, params, cores):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        cores = max(1, min(cores, len(params)))
        shares, load = [[] for _ in range(cores)], [0] * cores
        for p in sorted(params, key=lambda q: -q["n_particles"]):
            k = load.index(min(load))
            shares[k].append(p)
            load[k] += p["n_particles"]
        self.conns, self.procs = [], []
        for sh in shares:
            a, b = ctx.Pipe()
            pr = ctx.Process(target=_oracle_worker, args=(b, sh), daemon=True)
            pr.start()
            self.conns.append(a)
            self.procs.append(pr)
        for c in self.conns:
            if c.recv() != "ready":
                raise RuntimeError("oracle worker failed to start")
        self.cores = len(self.procs)

    def step(self):
        t0 = time.perf_counter()
        for c in self.conns:
            c.send(1)
        n = sum(c.recv()[0] for c in self.conns)
        return n, time.perf_counter() - t0

    def close(self):
        for c in self.conns:
            c.send(None)
        for pr in self.procs:
            pr.join(timeout=60)


def cpu_baseline_all_cores(params_list, window=6):
    """The oracle on every host core: all discharges of the workload, `window`
    lockstep PIC steps (the processes' start and the initial loads are not
    timed)."""
    cores = os.cpu_count() or 1
    pool = OraclePool(params_list, cores)
    n, t = 0, 0.0
    for _ in range(window):
        dn, dt = pool.step()
        n += dn
        t += dt
    pool.close()
    return {"value": n / t, "unit": "particle-steps/s", "cores": pool.cores, "kind": "oracle",
            "sample": f"all {len(params_list)} discharges of the workload, {window} steps, {n} particle-steps "
                      f"in {t:.1f} s on {pool.cores} processes"}


def cpu_baseline(params_list, budget_s=12.0, window=6):
    """The FP64 oracle as it stands, single thread, on the first discharges of
    the workload, `window` steps each, until `budget_s` of stepping."""
    import oracle
    pushes = 0
    t_used = 0.0
    used = []
    for i, p in enumerate(params_list):
        o = oracle.Oracle(p)
        for _ in range(window):
            n = o.n_particles
            t0 = time.perf_counter()
            o.step(1)
            t_used += time.perf_counter() - t0
            pushes += n
        used.append(i)
        o.close()
        if t_used >= budget_s:
            break
    return {"value": pushes / t_used, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
            "sample": f"discharges {used[0]}..{used[-1]} of the workload, {window} steps each, "
                      f"{pushes} particle-steps in {t_used:.1f} s"}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on the same workload, on every host
    core (one process per core, each stepping its share of the discharges)."""
    params = workload(0, args.instances, args.scale)
    pool = OraclePool(params, os.cpu_count() or 1)
    step = pool.step
    for _ in range(args.warmup):
        step()
    tot_n, tot_t, lat = 0, 0.0, []
    for _ in range(args.steps):
        n, t = step()
        tot_n += n
        tot_t += t
        lat.append(t * 1e3)
    pool.close()
    v = tot_n / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "particle-steps/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_t / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.instances} batched He discharges (config 3 ranges), one PIC step "
                                   f"over all of them per bench step", "instances": args.instances,
                       "particles": sum(p["n_particles"] for p in params)},
            "cpu_baseline": {"value": v, "unit": "particle-steps/s", "cores": pool.cores, "kind": "oracle",
                             "sample": f"all {args.instances} discharges, {args.steps} timed PIC steps on "
                                       f"{pool.cores} processes"},
            "e2e": {"value": v, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_fp64_plain(params, chunks=2, steps=20):
    """The plain FP64 path: one discharge at a time (the largest of the mix)."""
    import torch

    from paper_1508_02892_gb300 import hybrid, workloads as W
    p = dict(max(params, key=lambda q: q["n_particles"]))
    p["precision"] = W.FP64
    stream = torch.cuda.current_stream()
    d = hybrid.Discharge(p, stream=stream.cuda_stream)
    d.advance(steps)
    d.sync()
    c0 = d.counters()["pushes"]
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = 0.0
    for _ in range(chunks):
        s.record(stream)
        d.advance(steps)
        e.record(stream)
        e.synchronize()
        ms += s.elapsed_time(e)
    n = d.counters()["pushes"] - c0
    d.close()
    return {"value": n / (ms / 1e3), "unit": "particle-steps/s", "particles": int(p["n_particles"]),
            "steps": chunks * steps, "dtype": "f64"}


def _oracle_rate(p, steps):
    """The oracle as it stands on one host core: particle-steps/s of `steps`
    PIC steps of discharge p (its construction and initial load not timed)."""
    import oracle
    o = oracle.Oracle(p)
    n = 0
    t = 0.0
    for _ in range(steps):
        k = o.n_particles
        t0 = time.perf_counter()
        o.step(1)
        t += time.perf_counter() - t0
        n += k
    o.close()
    return n / t, n, t


def single_config_load(name, p, stream, flush, chunks=3, oracle_particles=200000, oracle_steps=5, tuning=None,
                       tune_steps=0):
    """One discharge of a single-instance workload as a one-slot batch, its
    launch layout from the library's autotuner (`tune_steps`-step trials on a
    scratch copy of the discharge) or fixed (`tuning`; default one lane, sort
    every 100 steps): whole-step particle-steps/s over `chunks` graph chunks (CUDA
    events), the electron kernel's fraction of the HBM roofline from one
    profiled chunk, and the oracle on one host core on a bounded sample: the
    same discharge with `oracle_particles` electrons (weight scaled to keep the
    density), `oracle_steps` steps."""
    import torch

    from paper_1508_02892_gb300 import hybrid
    if tune_steps > 0 and not tuning:
        # tune on a scratch copy of the discharge, so that the timed run starts
        # from the workload's initial state like a fixed-layout run
        bt = hybrid.Batch(1, p["precision"], stream=stream.cuda_stream)
        bt.admit(p)
        chosen = bt.autotune(tune_steps)
        bt.close()
        tuning_used = {k: chosen[k] for k in TUNE_KEYS}
    else:
        tuning_used = dict({"lanes": 1, "sort_interval": 100}, **(tuning or {}))
    b = hybrid.Batch(1, p["precision"], stream=stream.cuda_stream)
    s = b.admit(p)
    chosen = b.set_tuning(**tuning_used)
    b.advance(CHUNK)
    torch.cuda.synchronize()
    c0 = b.counters(s)["pushes"]
    ms = 0.0
    for _ in range(chunks):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.advance(CHUNK)
        e1.record(stream)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
    n = b.counters(s)["pushes"] - c0
    b.set_profiling(True)
    b.profile(reset=True)
    q0 = b.counters(s)["pushes"]
    flush.zero_()
    b.advance(CHUNK)
    torch.cuda.synchronize()
    prof = b.profile()
    nq = b.counters(s)["pushes"] - q0
    b.set_profiling(False)
    status = b.counters(s)["status"]
    b.close()
    peak, peak_kind = peaks()
    per_launch = nq / max(prof["n_electron"], 1)
    avg_ms = prof["ms_electron"] / max(prof["n_electron"], 1)
    bpu = BYTES_SPLIT if p["precision"] == 1 else BYTES_FP64
    achieved = bpu * per_launch / (avg_ms / 1e3) / 1e9
    q = dict(p)
    q["weight"] = p["n0_m3"] * p["gap_m"] / p["n_particles"] if not p.get("weight") else p["weight"]
    q["weight"] *= p["n_particles"] / oracle_particles
    q["n_particles"] = oracle_particles
    orate, on, ot = _oracle_rate(q, oracle_steps) if oracle_steps > 0 else (None, 0, 0.0)
    return {"workload": name, "value": n / (ms / 1e3), "unit": "particle-steps/s", "particles": int(p["n_particles"]),
            "tuning": {k: chosen[k] for k in TUNE_KEYS},
            "cells": int(p["n_cells"]), "steps_timed": chunks * CHUNK, "status": int(status),
            "kernel_ms_per_step": {"electron": prof["ms_electron"] / max(prof["n_electron"], 1),
                                   "field": prof["ms_field"] / max(prof["n_field"], 1)},
            "roofline": {"kernel": "k_electron", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind, "bytes_per_unit": bpu,
                         "units_per_launch": per_launch, "avg_launch_ms": avg_ms},
            "cpu_oracle": None if orate is None else
            {"value": orate, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
             "sample": f"the same discharge with {oracle_particles} electrons (density kept), "
                       f"{oracle_steps} steps, {on} particle-steps in {ot:.1f} s"}}


def config1_full(stream):
    """Config 1 as stated: FP64 plain method, one discharge, 2000 steps, on the
    GPU (CUDA events around the whole run) and in the oracle on one host core,
    both in full."""
    import torch

    from paper_1508_02892_gb300 import hybrid, workloads as W
    p = W.config1(precision=W.FP64)
    d = hybrid.Discharge(p, stream=stream.cuda_stream)
    d.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    d.advance(2000)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    c = d.counters()
    d.close()
    orate, on, ot = _oracle_rate(p, 2000)
    return {"workload": "config 1: He 0.5 mm / 200 cells, 2e4 electrons, DD constant mobility, FP64, 2000 steps",
            "gpu": {"value": c["pushes"] / (ms / 1e3), "unit": "particle-steps/s", "ms": ms, "pushes": c["pushes"]},
            "cpu_oracle": {"value": orate, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
                           "sample": f"the whole run: 2000 steps, {on} particle-steps in {ot:.1f} s"}}


def accuracy_load(params, stream, n=8, n_e=30000, steps=300):
    """The split path against the FP64 oracle on discharges of the benchmarked
    mix: the first n discharges with n_e electrons each (weight scaled to
    keep the density), `steps` steps, as one split batch and in the oracle
    (spawned processes).  L2-relative error of each time-averaged moment, the
    largest and the mean over the discharges."""
    import oracle
    from paper_1508_02892_gb300 import hybrid
    plist = []
    for p in params[:n]:
        q = dict(p)
        q["weight"] = p["n0_m3"] * p["gap_m"] / n_e
        q["n_particles"] = n_e
        plist.append(q)
    orc = oracle.run_ensemble(plist, steps)
    b = hybrid.Batch(len(plist), hybrid.HYB_FP32_SPLIT, stream=stream.cuda_stream)
    slots = [b.admit(q, steps) for q in plist]
    b.advance(steps)
    gpu = [b.moments(s) for s in slots]
    b.close()
    out = {}
    for k in ("ne", "ni", "ebar", "gamma", "eedf"):
        errs = [float(np.linalg.norm(g[k] - o[k]) / max(np.linalg.norm(o[k]), 1e-300)) for g, o in zip(gpu, orc)]
        out[k] = {"max_l2": max(errs), "mean_l2": sum(errs) / len(errs)}
    return {"sample": f"first {len(plist)} discharges of the mix, {n_e} electrons each, {steps} steps, split batch "
                      f"vs the FP64 oracle (same random numbers)", "l2": out}


def serve_load(args, stream, rank=0, world=1, tuning=None, n_requests=None, rate_hz=20.0):
    """Config-4 serving: Poisson arrivals (20/s) of discharges from the batched
    ranges, 1e4..4e6 electrons, each advanced by `serve_steps` steps, admitted
    under a 120 GB HBM cap into one resident batch (continuous batching);
    requests are dealt to ranks round-robin.  A higher rate_hz keeps the
    queue full (the server's capacity rather than the offered load)."""
    from paper_1508_02892_gb300 import hybrid, workloads as W
    from paper_1508_02892_gb300.serve import Server, summarize
    from paper_1508_02892_gb300 import shard
    n_req = args.serve_requests if n_requests is None else n_requests
    reqs = shard.rank_share(W.config4_requests(n_requests=n_req, rate_hz=rate_hz, steps=args.serve_steps), rank,
                            world)
    srv = Server(max_slots=64, hbm_cap_bytes=120e9, precision=hybrid.HYB_FP32_SPLIT, stream=stream.cuda_stream,
                 tuning=tuning, pipelined=args.serve_mode == "pipelined")
    t0 = time.perf_counter()
    out = srv.run(reqs, keep=("counters",))
    wall = time.perf_counter() - t0
    srv.close()
    s = summarize(out, wall)
    offered = sum(r["steps"] * r["params"]["n_particles"] for r in reqs) / max(reqs[-1]["arrival_s"], 1e-9)
    s.update({"mode": args.serve_mode, "rate_hz": rate_hz, "steps_per_request": args.serve_steps, "hbm_cap_gb": 120,
              "offered_particle_steps_per_s": offered,
              "peak_admitted_gb": srv.max_bytes / 1e9, "failed": sum(1 for r in out if r["status"] != 0)})
    return s


def swarm_load(n_fields=64, n_ions=65536, n_steps=20000):
    """Auxiliary ion swarm (Sec. II.C) at the size a mobility table is built:
    64 field values up to 5 MV/m, He+ in He at 1 atm; FP32 and FP64 device
    time (CUDA events around the call, which includes its small copies), and
    the oracle on one core for a bounded sample."""
    import torch

    import oracle
    from paper_1508_02892_gb300 import hybrid, workloads as W
    fields = W.swarm_fields(n_fields, 5e6)
    out = {"fields": n_fields, "ions_per_field": n_ions, "steps": n_steps,
           "unit": "ion-steps/s", "data": "synthetic: He+/He cross-section fits quoted with Tables 2/3"}
    s = torch.cuda.current_stream()
    for prec, name in ((W.FP32_SPLIT, "fp32"), (W.FP64, "fp64")):
        # the FP64 build (the parity path) runs on a sixteenth of the ions
        ni = n_ions if prec == W.FP32_SPLIT else max(256, n_ions // 16)
        p = W.swarm_params(n_ions=ni, n_steps=n_steps, n_relax=n_steps // 5, precision=prec)
        hybrid.swarm_run(dict(p, n_steps=200, n_relax=100), fields[:2])      # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        res, rc = hybrid.swarm_run(p, fields)
        e1.record(s)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        out[name] = {"value": n_fields * ni * n_steps / (ms / 1e3), "ms": ms, "rc": rc, "ions_per_field": ni,
                     "mobility_at_5MV_m": res[-1]["mobility"]}
    p = W.swarm_params(n_ions=200, n_steps=2000, n_relax=400)
    t0 = time.perf_counter()
    oracle.swarm_run(p, 1e6)
    dt = time.perf_counter() - t0
    out["cpu_baseline"] = {"value": 200 * 2000 / dt, "cores": 1, "kind": "oracle",
                           "sample": "200 ions x 2000 steps at 1 MV/m"}
    return out


def variants_load(params, stream, flush, n_inst=16, chunks=3, only=None):
    """The widened paths on the first `n_inst` discharges of the batched
    workload (FP32 split electrons, one lane, per-kernel CUDA events): the
    plain step; recombination with metastables, Penning and pooling (the
    electron kernel's chemistry variant and the metastable field step);
    power control (Eq. 2.9); and fully kinetic ions (split-mode ions: the
    electron kernel's ion-birth variant, k_ion and the ion sort), whose k_ion
    is measured against the HBM roofline at 48 algorithmic bytes per ion-step
    (read cell, offset, velocity and id, 28 B; write cell, offset and
    velocity, 20 B), as the electrons.
    Electron particle-steps/s over `chunks` timed chunks (L2 flushed between
    them), and the device time per step of each kernel interval."""
    import torch

    from paper_1508_02892_gb300 import hybrid, workloads as W
    sub = [dict(p) for p in params[:n_inst]]
    mods = {
        "plain": {},
        "recombination_metastables": dict(xs_rec=W.recombination_table(1e-8),
                                          **W.metastable_params(met_n0_m3=1e19, gamma_met=0.05)),
        "power_control": dict(power_w_m2=2e5, power_alpha=0.1),
        "kinetic_ions": dict(ion_model=W.ION_KINETIC),
    }
    peak, peak_kind = peaks()
    out = {"instances": n_inst, "chunks": chunks, "chunk_steps": CHUNK, "unit": "particle-steps/s",
           "initial_particles": sum(p["n_particles"] for p in sub)}
    for name, mod in mods.items():
        if only and name not in only:
            continue
        b = hybrid.Batch(n_inst, hybrid.HYB_FP32_SPLIT, stream=stream.cuda_stream)
        slots = [b.admit(dict(p, capacity_factor=2.5, **mod)) for p in sub]
        b.set_tuning(lanes=1)
        b.advance(CHUNK)                       # warm-up (graph capture)
        b.set_profiling(True)
        b.advance(CHUNK)
        torch.cuda.synchronize()
        b.profile(reset=True)
        c0 = [b.counters(s) for s in slots]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = 0.0
        for _ in range(chunks):
            flush.zero_()
            e0.record(stream)
            b.advance(CHUNK)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
        prof = b.profile()
        c1 = [b.counters(s) for s in slots]
        n = sum(y["pushes"] - x["pushes"] for x, y in zip(c0, c1))
        steps = chunks * CHUNK
        r = {"value": n / (ms / 1e3), "ms_per_step": ms / steps,
             "electron_ms_per_step": prof["ms_electron"] / steps, "field_ms_per_step": prof["ms_field"] / steps,
             "sort_ms_per_step": prof["ms_sort"] / steps,
             "status": max(c["status"] for c in c1)}
        if name == "recombination_metastables":
            r["events"] = {k: sum(y[k] - x[k] for x, y in zip(c0, c1))
                           for k in ("recombinations", "births_penning", "births_pooling")}
        if name == "kinetic_ions":
            ni = sum(y["ion_pushes"] - x["ion_pushes"] for x, y in zip(c0, c1))
            avg = prof["ms_ion"] / max(prof["n_ion"], 1)
            ach = 48.0 * ni / max(prof["n_ion"], 1) / (avg / 1e3) / 1e9
            r["ion_steps_per_s"] = ni / (ms / 1e3)
            r["ion_roofline"] = {"kernel": "k_ion_prefix + k_ion<FP32_SPLIT>", "bound": "hbm", "bytes_per_unit": 48,
                                 "units_per_launch": ni / max(prof["n_ion"], 1), "avg_launch_ms": avg,
                                 "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                                 "peak_kind": peak_kind}
        # the oracle beside it: one host core, the four smallest of these
        # discharges with the same change, three steps each
        import oracle
        small = sorted(sub, key=lambda q: q["n_particles"])[:4]
        n_o, t_o = 0, 0.0
        for q in small:
            o = oracle.Oracle(dict(q, capacity_factor=2.5, **mod))
            for _ in range(3):
                n_o += o.n_particles
                t0 = time.perf_counter()
                o.step(1)
                t_o += time.perf_counter() - t0
            o.close()
        r["cpu_baseline"] = {"value": n_o / t_o, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
                             "sample": f"the 4 smallest of the {n_inst} discharges, 3 steps each, {n_o} particle-steps"}
        out[name] = r
        b.close()
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist

    import __graft_entry__ as G
    G.build()
    from paper_1508_02892_gb300 import hybrid, workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    params = workload(rank, args.instances, args.scale)
    # one non-default stream for the library, the L2 flush and the timing events
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    b = hybrid.Batch(args.instances, hybrid.HYB_FP32_SPLIT, stream=stream.cuda_stream)
    slots = [b.admit(p) for p in params]
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def pushes():
        return sum(b.counters(s)["pushes"] for s in slots)

    # launch configuration picked by the library's autotuner on this workload
    # (its trial chunks are real steps of the runs and count as warm-up)
    if args.lanes > 0:
        fixed = {"lanes": args.lanes}
        if args.sort_interval > 0:
            fixed["sort_interval"] = args.sort_interval
        if args.field_cluster >= 0:
            fixed["field_cluster"] = args.field_cluster
        if args.electron_threads > 0:
            fixed["electron_threads"] = args.electron_threads
        if args.particles_per_thread > 0:
            fixed["particles_per_thread"] = args.particles_per_thread
        tuning = b.set_tuning(**fixed)
    elif args.tune_steps > 0:
        tuning = b.autotune(args.tune_steps)
    else:
        tuning = b.tuning()
    for _ in range(args.warmup):
        b.advance(CHUNK)
    torch.cuda.synchronize()
    prof0 = b.profile()
    p0 = pushes()
    clocks = Clocks(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()                         # L2 flush outside the timed interval
        ev_s[k].record(stream)
        b.advance(CHUNK)
        ev_e[k].record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    lat = [ev_s[k].elapsed_time(ev_e[k]) for k in range(args.steps)]
    ms_local = sum(lat)
    prof1 = b.profile()
    n_local = pushes() - p0
    from paper_1508_02892_gb300 import shard
    ms_tot, n_tot = shard.aggregate(ms_local, n_local, device="cuda")
    value = n_tot / (ms_tot / 1e3)

    # roofline of the dominant kernel (electron step), timed alone: one lane,
    # CUDA events around every kernel of a few more chunks
    b.set_tuning(lanes=1)
    b.set_profiling(True)
    b.advance(CHUNK)
    torch.cuda.synchronize()
    b.profile(reset=True)
    q0 = pushes()
    rchunks = max(1, min(args.steps, 5))
    for _ in range(rchunks):
        flush.zero_()
        b.advance(CHUNK)
    torch.cuda.synchronize()
    prof = b.profile()
    n_roof = pushes() - q0
    b.set_profiling(False)
    b.set_tuning(lanes=tuning["lanes"])
    n_launch = prof["n_electron"]
    ms_e = prof["ms_electron"]
    per_launch = n_roof / max(n_launch, 1)
    avg_ms = ms_e / max(n_launch, 1)
    peak, peak_kind = peaks()
    achieved = BYTES_SPLIT * per_launch / (avg_ms / 1e3) / 1e9
    tpp = traffic_per_push()
    shares = {"electron": ms_e, "field": prof["ms_field"], "sort": prof["ms_sort"],
              "chunks": rchunks, "lanes": 1}

    # end to end through the public API: admit from host parameters, chunks
    # with a host read of every discharge's moments, evict
    e2e = None
    if rank == 0 and not args.no_e2e:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b2 = hybrid.Batch(args.instances, hybrid.HYB_FP32_SPLIT, stream=stream.cuda_stream)
        b2.set_tuning(**{k: tuning[k] for k in TUNE_KEYS})
        s2 = [b2.admit(p) for p in params]
        h2d = 0
        for p in params:
            h2d += sum(p[k].nbytes for k in ("xs_ev", "xs_el", "xs_exc", "xs_ion", "tab_eon_td", "tab_mu", "tab_nu"))
            h2d += 8 * (p["n_cells"] + 1)
        d2h = 0

        def read_all():
            # every discharge's moments as of the snapshot queued last, read
            # while the chunk queued after it runs
            n = 0
            for s in s2:
                m = b2.snapshot_read_moments(s)
                n += sum(m[k].nbytes for k in ("ne", "ni", "gamma", "ebar", "eedf"))
            return n

        for i in range(args.steps):
            b2.advance(CHUNK)
            if i > 0:
                d2h += read_all()
            b2.snapshot_moments()
        d2h += read_all()
        n2 = sum(b2.counters(s)["pushes"] for s in s2)
        for s in s2:
            b2.evict(s)
        torch.cuda.synchronize()
        t2 = time.perf_counter() - t0
        b2.close()
        e2e = {"value": n2 / t2, "unit": "particle-steps/s", "h2d_bytes_per_step": h2d // args.steps,
               "d2h_bytes_per_step": d2h // args.steps,
               "note": "admission from host parameters and tables (pageable), per-chunk host read of all "
                       "moments (a stream-ordered snapshot of each chunk, read while the next chunk runs), "
                       "eviction, all inside the wall-clock region"}

    variants = None
    if rank == 0 and not args.no_variants:
        variants = variants_load(params, stream, flush)

    configs = None
    accuracy = None
    if rank == 0 and not args.no_configs:
        from paper_1508_02892_gb300 import workloads as W
        configs = {"config1_fp64_full": config1_full(stream),
                   "config2": single_config_load("config 2: He 1 mm / 1000 cells, 2e6 electrons, full fluid, "
                                                 "gamma 0.1, FP32 split", W.config2(), stream, flush,
                                                 oracle_particles=200000, oracle_steps=20,
                                                 tune_steps=min(args.tune_steps, 200)),
                   "config5": single_config_load("config 5: Ar 1 mm / 4000 cells, 5e7 electrons, full fluid, "
                                                 "gamma 0.15, dt 1e-13 s, FP32 split", W.config5(), stream, flush,
                                                 oracle_particles=500000, oracle_steps=20,
                                                 tune_steps=min(args.tune_steps, 200))}
        accuracy = accuracy_load(params, stream)

    swarm = None
    if rank == 0 and not args.no_swarm:
        swarm = swarm_load(n_ions=args.swarm_ions, n_steps=args.swarm_steps)

    serving = None
    if args.serve_requests > 0:
        # every rank serves its round-robin share of the requests on its GPU
        barrier()
        serving = serve_load(args, stream, rank, world,
                             tuning={k: tuning[k] for k in TUNE_KEYS})
        wall_ms, steps_all = shard.aggregate(serving["wall_s"] * 1e3, serving["particle_steps"], device="cuda")
        serving["throughput_all_ranks"] = steps_all / (wall_ms / 1e3)
        serving["latency_ranks"] = "rank 0's requests" if world > 1 else "all requests"
        if args.serve_saturated > 0:
            # arrivals faster than the GPU serves them: the queue stays full
            sat = serve_load(args, stream, rank, world, tuning={k: tuning[k] for k in TUNE_KEYS},
                             n_requests=args.serve_saturated, rate_hz=200.0)
            wall_ms, steps_all = shard.aggregate(sat["wall_s"] * 1e3, sat["particle_steps"], device="cuda")
            sat["throughput_all_ranks"] = steps_all / (wall_ms / 1e3)
            serving["saturated"] = sat

    fp64 = None
    if rank == 0 and not args.no_fp64:
        fp64 = run_fp64_plain(params)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        single = cpu_baseline(params, budget_s=args.cpu_budget)
        cpu = cpu_baseline_all_cores(params)
        cpu["single_core"] = single

    total_particles = sum(p["n_particles"] for p in params)
    lat_sorted = sorted(lat)
    line = {
        "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 particles / f64 grids", "data": "synthetic",
        "config": {"workload": f"{args.instances} batched He discharges (gap 0.3-2 mm, 150-2000 cells, "
                               f"1e4-2e6 electrons log-uniform, 100-400 V, DD/full ions), FP32 split, "
                               f"{CHUNK}-step CUDA-graph chunks", "instances": args.instances,
                   "initial_particles_per_gpu": total_particles, "chunk_steps": CHUNK,
                   "tuning": {k: tuning[k] for k in TUNE_KEYS},
                   "l2": "256 MB buffer written between timed chunks; particle store > L2"},
        "p50_ms_per_chunk": lat_sorted[len(lat) // 2], "p99_ms_per_chunk": lat_sorted[min(len(lat) - 1,
                                                                                           int(0.99 * len(lat)))],
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": peak_kind,
                     "traffic": (tpp * per_launch if tpp is not None else None),
                     "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                     "issue": issue_roofline(per_launch, avg_ms, (clk or {}).get("sm_mhz")),
                     "kernel": "k_electron<FP32_SPLIT>", "bytes_per_unit": BYTES_SPLIT,
                     "units_per_launch": per_launch, "avg_launch_ms": avg_ms,
                     "timed": f"electron kernel alone (1 lane), CUDA events around each launch of "
                              f"{rchunks} chunks after the headline region"},
        "kernel_ms": shares,
        "gpu_launches": prof1["kernel_launches"] - prof0["kernel_launches"],
        "clocks": clk,
    }
    if fp64:
        line["fp64_plain"] = fp64
        line["speedup_vs_fp64_plain"] = value / world / fp64["value"]
    if e2e:
        line["e2e"] = e2e
    if serving:
        line["serving"] = serving
    if swarm:
        line["swarm"] = swarm
    if variants:
        line["variants"] = variants
    if configs:
        line["configs"] = configs
    if accuracy:
        line["accuracy"] = accuracy
    if cpu:
        line["cpu_baseline"] = cpu
    line["device_index_guards"] = hybrid.debug_checks()
    b.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--instances", type=int, default=64)
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--tune-steps", type=int, default=500)
    ap.add_argument("--lanes", type=int, default=0, help="fixed lane count instead of the autotuner's")
    ap.add_argument("--sort-interval", type=int, default=0, help="with --lanes: fixed sort interval")
    ap.add_argument("--field-cluster", type=int, default=-1, help="with --lanes: fixed field cluster size (0: auto)")
    ap.add_argument("--electron-threads", type=int, default=0, help="with --lanes: electron block size (128/256/512)")
    ap.add_argument("--particles-per-thread", type=int, default=0, help="with --lanes: electron particles per thread (2/4)")
    ap.add_argument("--serve-requests", type=int, default=1000, help="config-4 serving requests (0: none)")
    ap.add_argument("--serve-saturated", type=int, default=300,
                    help="requests of a second serving run at 200/s (queue kept full; 0: none)")
    ap.add_argument("--serve-mode", default="pipelined", choices=["pipelined", "plain"],
                    help="request loop: one chunk queued ahead of the one being read (pipelined), or not")
    ap.add_argument("--serve-steps", type=int, default=5000)
    ap.add_argument("--no-swarm", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="skip the widened-path measurements")
    ap.add_argument("--only-variants", default="", help="run and print the widened-path measurements alone: "
                                                         "'all' or a comma list of plain, recombination_metastables, "
                                                         "power_control, kinetic_ions")
    ap.add_argument("--swarm-ions", type=int, default=65536, help="ions per field of the swarm run")
    ap.add_argument("--swarm-steps", type=int, default=20000)
    ap.add_argument("--only-swarm", action="store_true", help="run and print the ion-swarm measurement alone")
    ap.add_argument("--only-config", type=int, default=0, choices=[0, 2, 5],
                    help="run and print one single-instance workload alone (2: He 1000 cells, 2e6 electrons; "
                         "5: Ar 4000 cells, 5e7 electrons)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip configs 1, 2, 5 and the accuracy check")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        if int(os.environ.get("RANK", "0")) != 0:
            return
        import oracle
        oracle.build()
        run_reference(args)
        return
    if args.only_swarm:
        import torch

        import __graft_entry__ as G
        G.build()
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        print(json.dumps({"swarm": swarm_load(n_ions=args.swarm_ions, n_steps=args.swarm_steps)}), flush=True)
        return
    if args.only_config:
        import torch

        import __graft_entry__ as G
        from paper_1508_02892_gb300 import workloads as W
        G.build()
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        stream = torch.cuda.Stream()
        torch.cuda.set_stream(stream)
        flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
        p = W.config2() if args.only_config == 2 else W.config5()
        tuning = {}
        if args.sort_interval > 0:
            tuning["sort_interval"] = args.sort_interval
        if args.field_cluster >= 0:
            tuning["field_cluster"] = args.field_cluster
        if args.electron_threads > 0:
            tuning["electron_threads"] = args.electron_threads
        if args.particles_per_thread > 0:
            tuning["particles_per_thread"] = args.particles_per_thread
        out = single_config_load(f"config {args.only_config}", p, stream, flush, chunks=max(args.steps // CHUNK, 1),
                                 oracle_particles=200000, oracle_steps=0 if args.no_cpu else 20, tuning=tuning,
                                 tune_steps=min(args.tune_steps, 200))
        print(json.dumps({f"config{args.only_config}": out}), flush=True)
        return
    if args.only_variants:
        import torch

        import __graft_entry__ as G
        G.build()
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        stream = torch.cuda.Stream()
        torch.cuda.set_stream(stream)
        flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
        only = args.only_variants.split(",") if args.only_variants != "all" else None
        print(json.dumps({"variants": variants_load(workload(0, args.instances, args.scale), stream, flush,
                                                    only=only)}), flush=True)
        return
    run_ours(args)


if __name__ == "__main__":
    main()
