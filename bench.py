#!/usr/bin/env python
"""Benchmark of the LBE and DUGKS time steps on GB300 (one JSON line on stdout).

Workload (per GPU): decaying homogeneous isotropic turbulence on a periodic
256^3 box, D3Q19, FP32 storage, seeded initial field with k0 = 8, Ma = 0.15,
Re_lambda = 70 (viscosity from the field).  One bench step advances an MRT-LBE
simulation by one step (dt = 1) and a DUGKS simulation by one step (dt = 0.5);
E and eps of both are read back every 10 steps and E(k) every 200 steps (the
logging cadence of the 128^3 run).  value = cell updates of all ranks / the
slowest rank's time, in MLUPS.  The state (2 x 1.27 GB per scheme) is far
larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (a smaller box from the same recipe) on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "LBE/DUGKS MLUPS at 256^3 FP32, % HBM roofline; ensemble p50/p99 latency"
BYTES_PER_CELL = {"f32": 152, "f16": 76, "bf16": 76, "f64": 304}  # 19 loads + 19 stores
K0, MA, RE_LAMBDA = 8.0, 0.15, 70.0
STATS_EVERY, SPECTRUM_EVERY = 10, 200
# The MRT-LBE run of this field goes non-finite after about 70 steps (a
# stability result, reported under "stability"); every timed segment therefore
# restarts both schemes from the seeded field, outside the timed region.
SEGMENT = 50
STABILITY_STEPS = 300


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=400)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--N", type=int, default=256)
    p.add_argument("--storage", choices=["f32", "f16", "bf16", "f64"], default="f32")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-stability", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the ensemble, serving and reduced-precision reports")
    p.add_argument("--serving-seconds", type=float, default=15.0)
    p.add_argument("--record-counters", nargs="+", metavar="NCU_CSV",
                   help="write the counters record from ncu --csv logs of one fused DUGKS launch and exit")
    p.add_argument("--record-command", default="", help="the ncu command line, for the counters record")
    return p.parse_args()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _sm_max_mhz():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["sm_max_mhz"])
    except Exception:
        return 2070.0


# The fused DUGKS kernel's translation unit, its headers and the build flags:
# DRAM traffic and instruction counts recorded from an ncu capture hold only
# while these are unchanged.
KERNEL_SOURCES = ("dugks_fused.cu", "dugks_tile.cuh", "dugks_face.cuh", "pair_math.cuh", "kin_common.cuh",
                  "kin_internal.h")
COUNTERS_RECORD = "profiles/dugks_fused_kernel_256_f32_counters.md"
SMS, SCHEDULERS = 152, 4  # GB300: streaming multiprocessors, warp schedulers per SM


def kernel_source_hash() -> str:
    from paper_1601_03815_gb300 import build as b

    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(b.CSRC, name), "rb") as fh:
            h.update(name.encode() + b"\0" + fh.read() + b"\0")
    h.update(" ".join(b.NVCC_FLAGS[:4] + b.ARCH).encode())
    return h.hexdigest()[:16]


def read_counters(path=COUNTERS_RECORD) -> dict:
    """`key = value` lines of the fenced block of a counters record."""
    out = {}
    try:
        with open(os.path.join(ROOT, path)) as fh:
            inside = False
            for line in fh:
                if line.startswith("```"):
                    inside = not inside
                    continue
                if inside and "=" in line:
                    k, v = (t.strip() for t in line.split("=", 1))
                    out[k] = v
    except OSError:
        pass
    return out


def record_counters(csv_paths, workload: str, command: str, path=COUNTERS_RECORD) -> None:
    """Write the counters record from ncu --csv logs of one launch of the fused
    DUGKS kernel (dram__bytes_read/write.sum, smsp__inst_executed.sum)."""
    import csv

    vals = {}
    for p in csv_paths:
        with open(p) as fh:
            rows = [r for r in csv.reader(fh) if len(r) > 10]
        hdr = rows[0]
        for r in rows[1:]:
            d = dict(zip(hdr, r))
            if "dugks_fused" in d.get("Kernel Name", ""):
                vals[d["Metric Name"]] = int(float(d["Metric Value"].replace(",", "")))
    lines = ["kernel_sources_sha256 = %s" % kernel_source_hash(),
             "workload = %s" % workload,
             "dram_bytes_read = %d" % vals["dram__bytes_read.sum"],
             "dram_bytes_write = %d" % vals["dram__bytes_write.sum"],
             "warp_instructions = %d" % vals["smsp__inst_executed.sum"]]
    with open(os.path.join(ROOT, path), "w") as fh:
        fh.write("# Counters of one fused DUGKS launch, 256^3 FP32 (read by bench.py)\n\n")
        fh.write("Command (GB300; each ncu run is one pass, checked on a 128^3 capture of the same metric\n"
                 "group first; the plain command exited 0 before it):\n\n    %s\n\n" % command)
        fh.write("bench.py reports `traffic` = read + write and the issue roof from these values\n"
                 "while the kernel sources hash to the recorded value, and null otherwise.\n\n")
        fh.write("```\n%s\n```\n" % "\n".join(lines))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms while the
    timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(self.rows)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def bench_config(N: int, storage: str, world: int) -> dict:
    bpc = BYTES_PER_CELL[storage]
    return {"workload": "DHIT %d^3 D3Q19: one MRT-LBE step (dt=1) + one DUGKS step (dt=0.5) "
                        "per bench step; k0=8, Ma=0.15, Re_lambda=70; E, eps every %d steps, "
                        "E(k) every %d" % (N, STATS_EVERY, SPECTRUM_EVERY),
            "N": N, "storage": storage,
            "l2": "inputs larger than L2 (one copy of f is %.2f GB), no flush" % (N ** 3 * bpc / 2 / 1e9),
            "parallelism": "replicas" if world > 1 else "single"}


def max_over_ranks(value: float, dist, device=None) -> float:
    """Largest `value` over all ranks (identity without a process group)."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(cells_per_rank: int, steps: int, world: int, tmax: float) -> float:
    """Cell updates of all ranks over the slowest rank's time (weak scaling)."""
    return world * cells_per_rank * steps / tmax / 1e6


def cpu_model() -> str:
    """The host CPU's model name (lscpu), else what Python reports."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


def cpu_baseline_sample(steps: int = 1):
    """The FP64 oracle (as it stands) on the host cores, on the 128^3
    workloads of the CPU-baseline plan: C2 (k0 = 8, Ma = 0.1, Re_lambda = 25,
    seed 1200) and the paper-parity P1 (the Table I field of Sec. IV.A, u' = 0.032,
    nu = 1.2395e-2 of Table I), `steps` MRT-LBE and `steps` DUGKS (dt = 0.5)
    steps each, with all host cores and with 16 threads (the paper's 16 MPI
    cores).  The headline value is C2 with all cores."""
    import kin_inputs as ki
    import oracle

    oracle.build()
    n = 128
    nproc = os.cpu_count() or 1
    cases = {}
    u, info = ki.dhit_velocity(n, 1200, 8.0, 0.1, return_info=True)
    cases["C2"] = (u, ki.nu_from_re_lambda(info["u_prime"], info["omega"], 25.0))
    u, _ = ki.dhit_velocity(n, 1700, math.sqrt(2.0 / 0.14), 0.032 / math.sqrt(1.0 / 3.0), return_info=True)
    cases["P1"] = (u, 1.2395e-2)
    threads = sorted({nproc, 16})
    runs = {}
    for name, (u, nu) in cases.items():
        f = oracle.equilibrium_field(u)
        for th in threads:
            oracle.set_num_threads(th)
            rec = {}
            for scheme, dt in (("lbe", 1.0), ("dugks", 0.5)):
                g = oracle.step(scheme, f, nu, dt)  # warm (page-in, thread start)
                t0 = time.perf_counter()
                for _ in range(steps):
                    g = oracle.step(scheme, g, nu, dt)
                rec[scheme + "_mlups"] = steps * n ** 3 / (time.perf_counter() - t0) / 1e6
            runs["%s_%dthreads" % (name, th)] = rec
        del f
    oracle.set_num_threads(nproc)
    head = runs["C2_%dthreads" % nproc]
    # one LBE + one DUGKS step per bench step: cell updates over both times
    value = 2.0 / (1.0 / head["lbe_mlups"] + 1.0 / head["dugks_mlups"])
    return {"value": value, "unit": "MLUPS", "cores": nproc, "kind": "oracle", "cpu": cpu_model(),
            "nproc": nproc,
            "sample": "FP64 oracle, 128^3: C2 (k0=8, Ma=0.1, Re_lambda=25) and P1 (Table I field, "
                      "u'=0.032, nu=1.2395e-2), %d MRT-LBE + %d DUGKS steps each, at %s threads; value = "
                      "C2 at all %d cores, one LBE + one DUGKS step per update pair" % (
                          steps, steps, " and ".join(str(t) for t in threads), nproc),
            "runs": runs,
            "paper": {"lbe_mlups": 128 ** 3 / 0.666 / 1e6, "dugks_mlups": 128 ** 3 / 0.911 / 1e6,
                      "hardware": "16 CPU cores, MPI (Sec. IV.E)"}}


def extras(args) -> dict:
    """Batched ensemble, serving and reduced-precision reports (one GPU)."""
    from paper_1601_03815_gb300 import ensemble as ens_mod
    from paper_1601_03815_gb300 import precision as prec_mod
    from paper_1601_03815_gb300 import serving as srv_mod

    out = {}
    out["ensemble"] = ens_mod.measure(steps=500)
    # the same seeded arrival trace through both serving backends; the first
    # (per-simulation streams) is the serving loop's default
    for key, name in (("serving", "streams"), ("serving_ensemble_backend", "ensemble")):
        reqs = srv_mod.poisson_requests(4.0, args.serving_seconds, seed=2024)
        backend = srv_mod.BACKENDS[name]()
        _, rep = srv_mod.Server(backend, 64 * 2 ** 30, 64, 50).run(reqs)
        backend.close()
        rep["backend"] = name
        rep["arrival_window_s"] = args.serving_seconds
        rep["rate_per_s"] = 4.0
        out[key] = rep
    out["precision"] = prec_mod.study(args.N, 1000)
    return out


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    import kin_inputs as ki
    import oracle

    oracle.build()
    # size the per-step sample so W + K steps take about two minutes
    probe_n = 24
    u, info = ki.dhit_velocity(probe_n, 1300, min(K0, probe_n / 4), MA, return_info=True)
    f = oracle.equilibrium_field(u)
    t0 = time.perf_counter()
    oracle.lbe_step(f, 0.01)
    oracle.dugks_step(f, 0.01, 0.5)
    per_cell = (time.perf_counter() - t0) / probe_n ** 3
    budget = 120.0 / max(1, args.steps + args.warmup)
    n = int((budget / per_cell) ** (1.0 / 3.0)) // 2 * 2
    n = max(16, min(128, n))
    u, info = ki.dhit_velocity(n, 1300, min(K0, n / 4), MA, return_info=True)
    nu = ki.nu_from_re_lambda(info["u_prime"], info["omega"], RE_LAMBDA)
    fl = oracle.equilibrium_field(u)
    fd = fl.copy()
    for _ in range(args.warmup):
        fl = oracle.lbe_step(fl, nu)
        fd = oracle.dugks_step(fd, nu, 0.5)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        fl = oracle.lbe_step(fl, nu)
        fd = oracle.dugks_step(fd, nu, 0.5)
    elapsed = time.perf_counter() - t0
    value = 2 * args.steps * n ** 3 / elapsed / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * elapsed / max(1, args.steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(args.N, args.storage, world),
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": oracle.num_threads(),
                         "kind": "oracle",
                         "sample": "each bench step: one MRT-LBE + one DUGKS oracle step (FP64) on a "
                                   "%d^3 box of the same recipe (k0=%g, Ma=0.15, Re_lambda=70), %d steps"
                                   % (n, min(K0, n / 4), args.steps)},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    import paper_1601_03815_gb300 as kin

    world, rank, local = _dist()
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    kin.load()
    st = {"f32": kin.F32, "f16": kin.F16, "bf16": kin.BF16, "f64": kin.F64}[args.storage]
    N = args.N
    stream = torch.cuda.Stream()
    seed = 1300 + rank
    lbe = kin.Sim(N, kin.LBE_MRT, 0.01, MA, 1.0, st, stream=stream)
    dug = kin.Sim(N, kin.DUGKS, 0.01, MA, 0.5, st, stream=stream)
    lbe.init_field(seed, K0, RE_LAMBDA)
    dug.init_field(seed, K0, RE_LAMBDA)

    def bench_step(k, record=None):
        """One step of each scheme; True if the DUGKS step was bracketed by
        events (a statistics step runs it inside kin_step_stats instead)."""
        if record is not None:
            record[0].record(stream)
        lbe.step(1)
        if record is not None:
            record[1].record(stream)
        if (k + 1) % STATS_EVERY == 0:
            spec = (k + 1) % SPECTRUM_EVERY == 0
            # the DUGKS step also writes the velocity its statistics need
            dug.step_stats(1, spectrum=spec)
            lbe.stats(spectrum=spec)
            return False
        dug.step(1)
        if record is not None:
            record[2].record(stream)
        return True

    def reinit():
        lbe.init_field(seed, K0, RE_LAMBDA)
        dug.init_field(seed, K0, RE_LAMBDA)

    reinit()
    for k in range(args.warmup):
        bench_step(k)
    # one E(k) of each scheme: the FFT plans are made on a simulation's first
    # spectrum, a one-time cost that stays out of the timed steps
    lbe.stats(spectrum=True)
    dug.stats(spectrum=True)
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    seg_ev = []
    launches0 = lbe.kernel_launches + dug.kernel_launches
    clocks = ClockSampler(local)
    clocks.start()
    done = 0
    elapsed = 0.0
    dug_timed = []  # steps whose DUGKS step has its own events
    while done < args.steps:
        n = min(SEGMENT, args.steps - done)
        reinit()  # untimed: every segment starts from the seeded field
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for j in range(n):
            if bench_step(done + j, evs[done + j]):
                dug_timed.append(done + j)
        stop.record(stream)
        torch.cuda.synchronize()
        elapsed += start.elapsed_time(stop) / 1000.0
        seg_ev.append(n)
        done += n
    clocks.stop()
    launches = lbe.kernel_launches + dug.kernel_launches - launches0
    t_lbe = sum(e[0].elapsed_time(e[1]) for e in evs) / args.steps / 1000.0
    t_dug = sum(evs[k][1].elapsed_time(evs[k][2]) for k in dug_timed) / max(1, len(dug_timed)) / 1000.0
    tmax = max_over_ranks(elapsed, dist, "cuda")
    if dist:
        dist.barrier()
    cells = N ** 3
    value = whole_job_mlups(2 * cells, args.steps, world, tmax)

    # end to end through the C ABI: the initial field from pinned host memory,
    # then per step one step of each scheme and a read-back of E and eps
    e2e = None
    if not args.no_e2e:
        import kin_inputs as ki

        u0 = ki.dhit_velocity(N, seed, K0, MA)
        pinned = torch.empty(u0.shape, dtype=torch.float64, pin_memory=True)
        pinned.numpy()[...] = u0
        hu = pinned.numpy()
        k_e2e = max(10, min(args.steps, SEGMENT))
        # the two schemes as a user would run two independent simulations,
        # each on its own stream, monitoring E and eps every step: the
        # statistics of step k are copied to page-locked host memory
        # asynchronously and read (checked) once step k + 1 is enqueued
        sl, sd = torch.cuda.Stream(), torch.cuda.Stream()
        lbe_e = kin.Sim(N, kin.LBE_MRT, lbe.nu, MA, 1.0, st, stream=sl)
        dug_e = kin.Sim(N, kin.DUGKS, dug.nu, MA, 0.5, st, stream=sd)
        res = torch.zeros((k_e2e, 2, 2), dtype=torch.float64, pin_memory=True).numpy()
        done = [(torch.cuda.Event(), torch.cuda.Event()) for _ in range(k_e2e)]

        def e2e_steps(n):
            for k in range(n):
                lbe_e.step(1)
                lbe_e.stats_async(res[k, 0])
                # the fused DUGKS step also writes the velocity its statistics need
                dug_e.step_stats_async(1, res[k, 1])
                done[k][0].record(sl)
                done[k][1].record(sd)
                if k > 0:
                    for ev in done[k - 1]:
                        ev.synchronize()
                    if not np.all(np.isfinite(res[k - 1])):
                        raise RuntimeError("non-finite statistics at end-to-end step %d" % (k - 1))
            lbe_e.sync()
            dug_e.sync()
            if not np.all(np.isfinite(res[n - 1])):
                raise RuntimeError("non-finite statistics at end-to-end step %d" % (n - 1))

        lbe_e.set_velocity(hu)
        dug_e.set_velocity(hu)
        e2e_steps(2)
        # three timed runs of the whole sequence (upload included); the median
        # is reported, so that one host stall in a ~0.1 s run does not decide it
        samples = []
        for _ in range(3):
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lbe_e.set_velocity(hu)
            dug_e.set_velocity(hu)
            e2e_steps(k_e2e)
            torch.cuda.synchronize()
            te = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
            samples.append(whole_job_mlups(2 * cells, k_e2e, world, te))
        lbe_e.close()
        dug_e.close()
        e2e = {"value": sorted(samples)[1], "unit": "MLUPS", "samples": samples,
               "h2d_bytes_per_step": int(2 * u0.nbytes / k_e2e), "d2h_bytes_per_step": 2 * 2 * 8,
               "steps": k_e2e,
               "what": "kin_set_velocity from pinned host memory for both schemes, then per step "
                       "kin_step(1) + kin_stats_async of the LBE run and kin_step_stats_async(1) of "
                       "the DUGKS run, each simulation on its own stream; E and eps of both copied "
                       "to page-locked host memory every step and checked one step later; host "
                       "wall clock, median of three runs"}

    # stability probe (untimed): first check at which E is non-finite, every 5
    # steps up to STABILITY_STEPS, from the seeded field
    stability = {}
    for name, sim in (() if args.no_stability else (("lbe", lbe), ("dugks", dug))):
        sim.init_field(seed, K0, RE_LAMBDA)
        bad = None
        for n in range(0, STABILITY_STEPS + 1, 5):
            try:
                sim.stats()
            except kin.KinError as exc:
                if exc.code != kin.KIN_ENONFINITE:
                    raise
                bad = n
                break
            sim.step(5)
        stability[name] = {"nonfinite_at_step": bad, "checked_through_step": STABILITY_STEPS,
                           "nu": sim.nu}

    peak, peak_kind = _peaks()
    bpc = BYTES_PER_CELL[args.storage]
    per = {}
    for name, t, sim in [("lbe", t_lbe, lbe), ("dugks", t_dug, dug)]:
        gbs = bpc * cells / t / 1e9
        per[name] = {"mlups": cells / t / 1e6, "ms_per_step": 1000 * t, "gbs": gbs,
                     "frac_of_%s_hbm" % peak_kind: gbs / peak, "launches_per_step": sim.step_launches}
    dom = "dugks" if t_dug >= t_lbe else "lbe"
    t_dom = t_dug if dom == "dugks" else t_lbe
    achieved = bpc * cells / t_dom / 1e9
    # DRAM traffic and warp instructions of one launch of the fused DUGKS
    # kernel on this workload, from the counters record, while the kernel's
    # sources are the ones it was captured from
    traffic, issue, traffic_source = None, None, None
    if dom == "dugks" and args.storage == "f32" and N == 256:
        rec = read_counters()
        if rec and rec.get("kernel_sources_sha256") == kernel_source_hash():
            traffic = int(rec["dram_bytes_read"]) + int(rec["dram_bytes_write"])
            traffic_source = "%s (kernel sources sha256 %s)" % (COUNTERS_RECORD, rec["kernel_sources_sha256"])
            inst = int(rec["warp_instructions"])
            peak_issue = SMS * SCHEDULERS * _sm_max_mhz() * 1e6
            issue = {"bound": "issue", "achieved": inst / t_dom, "peak": peak_issue,
                     "peak_kind": "nominal: %d SMs x %d schedulers x 1 warp instruction per cycle x %.0f MHz"
                                  % (SMS, SCHEDULERS, _sm_max_mhz()),
                     "unit": "warp inst/s", "frac": inst / t_dom / peak_issue,
                     "warp_instructions_per_launch": inst}
        else:
            traffic_source = "none: the kernel sources differ from those of %s" % COUNTERS_RECORD
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tmax / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.storage,
        "data": "synthetic",
        "config": bench_config(N, args.storage, world),
        "per_scheme": per,
        "roofline": {"bound": "hbm", "kernel": "%s step" % dom, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "traffic_source": traffic_source,
                     "algorithmic_bytes_per_launch": bpc * cells, "issue": issue},
        "clocks": clocks.summary(),
        "gpu_launches": launches * world,
        "e2e": e2e,
        "stability": stability,
        "timing": "%d segments of up to %d steps, each from the seeded field; per-scheme times from "
                  "events around each step (DUGKS: the %d steps without statistics; on a statistics "
                  "step its step runs inside kin_step_stats)" % (len(seg_ev), SEGMENT, len(dug_timed)),
    }
    for sim in (lbe, dug):
        sim.close()
    if world == 1 and not args.no_extras:
        line.update(extras(args))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample()
    elif rank == 0:
        line["cpu_baseline"] = None
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.record_counters:
        record_counters(args.record_counters, "256^3 FP32 fused DUGKS step (bench.py default workload)",
                        args.record_command)
        return 0
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
