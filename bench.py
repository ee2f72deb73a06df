"""Benchmark: SU(3) checkerboard heatbath link updates per second on GB300.

Workload (the paper's own timing workload, Berg & Wu Sec. 2.1, Table 1, 32^4
column): a 32^4 periodic lattice at beta = 5.7, hot start from Philox seed 7,
FP64 links; one step = 2 full checkerboard sweeps (4 * 32^4 * 2 link updates)
with no measurement inside the step, start-configuration creation outside the
timed region (Sec. 2).  The FP32-mixed form of the same workload is reported
under "variants".

Timing: W untimed warm-up steps, then K steps between a barrier and a device
synchronise, CUDA events on the library's stream around every sweep graph,
maximum over ranks.  The link store (604 MB FP64, 201 MB FP32-mixed) exceeds
the 129 MB L2, so no flush is needed between steps.

Multi-GPU: replicas only -- each rank runs its own lattice (weak scaling), no
collective on the data path; value = all ranks' link updates / slowest rank's
time.

--impl reference times the FP64 CPU oracle on every host core (spawned
processes on disjoint site subsets) on a bounded sample of the same workload
(one half-sweep of the 32^4 lattice per step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SU(3) link updates/s at 32^4 (FP64 vs FP32-mixed vs batched); % HBM roofline"
UNIT = "link updates/s"
DIMS = (32, 32, 32, 32)
BETA = 5.7
SEED = 7
SWEEPS_PER_STEP = 2
# Paper, Table 1: 32^4, 2 sweeps, non-MPI program on one 2 GHz Intel E5405 core: 48.9 s.
PAPER_UPS = 4 * 32 ** 4 * 2 / 48.9
# Table 1, first row (non-MPI program, one core), per column 8^4 x 512, 12^4 x 101, 16^4 x 32, 32^4 x 2.
PAPER_TABLE1_SECONDS = [48.2, 48.3, 48.7, 48.9]

# Algorithmic cost per link update of one half-sweep (mu, parity): the V/2
# updated links, the V/2 opposite-parity links of direction mu and the 3V links
# of the other directions are read once, the V/2 updated links written once:
# 9 links moved per update.
BYTES_PER_UPDATE = {"fp64": 9 * 18 * 8, "fp32_mixed": 9 * 12 * 4}
# FP64 floating-point operations per link update of the FP64 kernel as written
# (an FMA counts 2; transcendental calls, square roots and divisions are not
# counted):
#   staple 2070: 6 paths x 2 products of rows 0,1 (or columns 0,1) = 12 x 144,
#     first path's row completion 42, 5 accumulations with the row completion
#     fused in, 60 each;
#   three SU(2) steps 254 + 254 + 212 = 720: projection 100, |r|^2 and
#     1/alpha 8, uniforms 6, Kennedy-Pendleton proposal and test 8, a0 and the
#     direction 8, quaternions 8, SU(2) matrix 32, rotation of rows (i, j) 84
#     (42 in the last step, whose row 2 is rebuilt by Gram-Schmidt);
#   Gram-Schmidt 84 and row completion 42.
FP64_FLOP_PER_UPDATE = 2070 + 720 + 126


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# dominant kernel of each line, from one ncu capture: the bytes, the command
# that captured them (after the same command ran without ncu), and the SHA-256
# of the kernel's code at capture time (kernel_sources_sha: the translation
# units that define and launch the kernel and every csrc/*.cuh, comments
# stripped).  A line reports the figure only while that code still hashes the
# same; otherwise its traffic is null and the line says why.
_U_F64, _U_F32, _U_BATCH = ("su3_kernels.cu",), ("su3_kernels.cu", "su3_kernels_pair.cu"), ("su3_batch.cu",)
_SHA_F64 = "885129abed2f07dcf526279300c7e616b6ab6d05d7f194316ac183375be7f880"
_SHA_F32 = "b69b3efb95b8c7b71cd98f8e15af6aec0aaf08bce33ea207b3a093f079754790"
_SHA_BATCH = "d9029b824bda46a252b5670089d82c5b7d10b27581aefd95730e21efa98e8ad2"
_NCU_METRICS = "ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum --clock-control none"
NCU_TRAFFIC = {
    # one launch of the default 32^4 FP32 sweep = one chained half-sweep; the mean of the eight launches of
    # the second sweep
    "fp32_mixed": {"bytes": 208961760 + 12656192, "units": _U_F32, "sources_sha256": _SHA_F32,
                   "capture": _NCU_METRICS + " -k regex:k_half_sweep_f32_chain -s 8 -c 8 python bench.py --profile "
                                             "fp32_mixed"},
    "fp32_eft": {"bytes": 208966496 + 13336640, "units": _U_F32, "sources_sha256": _SHA_F32,
                 "capture": _NCU_METRICS + " -k regex:k_half_sweep_f32_chain -s 8 -c 8 python bench.py --profile "
                                           "fp32_eft"},
    "fp32_mixed_phases": {"bytes": 207816192 + 15345664, "units": _U_F32, "sources_sha256": _SHA_F32,
                          "capture": _NCU_METRICS + " -k regex:k_half_sweep -s 8 -c 1 python bench.py --profile "
                                                    "fp32_mixed_phases"},
    "fp32_eft_phases": {"bytes": 207962880 + 15926528, "units": _U_F32, "sources_sha256": _SHA_F32,
                        "capture": _NCU_METRICS + " -k regex:k_half_sweep -s 8 -c 1 python bench.py --profile "
                                                  "fp32_eft_phases"},
    "fp64": {"bytes": 624059904 + 64907520, "units": _U_F64, "sources_sha256": _SHA_F64,
             "capture": _NCU_METRICS + " -k regex:k_half_sweep -s 8 -c 1 python bench.py --profile fp64"},
    "batched": {"bytes": 2830772736 + 442051584, "units": _U_BATCH, "sources_sha256": _SHA_BATCH,
                "capture": _NCU_METRICS + " -k regex:k_batch_sweep -s 4 -c 4 python bench.py --profile batched "
                                          "(the four launches of the second sweep, summed)"},
    "batched_eft": {"bytes": 2829066240 + 442415616, "units": _U_BATCH, "sources_sha256": _SHA_BATCH,
                    "capture": _NCU_METRICS + " -k regex:k_batch_sweep -s 4 -c 4 python bench.py --profile batched_eft "
                                              "(the four launches of the second sweep, summed)"},
}


def _code_only(text):
    """C/C++ source without comments and with whitespace runs collapsed, so
    that the provenance hash below changes with the code, not with its prose."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def kernel_sources_sha(units=None):
    """sha256 of the code (comments stripped) of the translation units `units`
    (csrc/*.cu names; None = all) and of every csrc/*.cuh, sorted by name."""
    import hashlib
    d = os.path.join(ROOT, "paper_0904_1179_gb300", "csrc")
    h = hashlib.sha256()
    for fn in sorted(os.listdir(d)):
        if fn.endswith(".cuh") or (fn.endswith(".cu") and (units is None or fn in units)):
            with open(os.path.join(d, fn), encoding="utf-8") as f:
                h.update(fn.encode() + b"\0" + _code_only(f.read()).encode())
    return h.hexdigest()


def traffic_of(variant):
    """(bytes or None, provenance) of a line's ncu DRAM traffic figure."""
    rec = NCU_TRAFFIC.get(variant)
    if rec is None:
        return None, "no ncu capture recorded for this kernel"
    if rec["sources_sha256"] != kernel_sources_sha(rec["units"]):
        return None, "kernel sources changed since the ncu capture (%s)" % rec["capture"]
    return rec["bytes"], "ncu capture: %s; code sha256 of %s and csrc/*.cuh: %s" % (
        rec["capture"], ", ".join(rec["units"]), rec["sources_sha256"][:16])

# FP64 peak of GB300 from unit counts and clock: 152 SMs x 2 FP64 FMA per
# clock (1/64 of the 128 FP32 lanes) x 2 flop x 2.070 GHz = 1.2586 TFLOP/s
# (the nominal 1.25).  An FMA-loop probe reached 1.006 TFLOP/s (0.80 of it);
# both are reported.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
FP64_PROBE_TFLOPS = 1.006


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(local)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max_sum(world, seconds, units, device):
    """Slowest rank's time and the sum of all ranks' units (host logic shared with the CPU tests)."""
    if world == 1:
        return seconds, units
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def time_sweeps(lat, stream, steps, warmup, sweeps_per_step, world, sampler=None):
    """W warm-up steps, then K steps; CUDA events on the lattice's stream around every sweep graph."""
    import torch
    for _ in range(warmup):
        lat.sweep(sweeps_per_step)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    n = steps * sweeps_per_step
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(n + 1)]
    if sampler:
        sampler.start()
    evs[0].record(stream)
    for i in range(n):
        lat.sweep(1)
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    barrier(world)
    total_ms = evs[0].elapsed_time(evs[-1])
    sweep_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(n)]
    return total_ms, sweep_ms, clocks


def time_e2e(su3, L, prec, steps, warmup, sweeps_per_step):
    """End to end through the public API with page-locked host buffers: per step, copy the
    configuration in (su3_links_set), run the sweeps -- the last one measuring the plaquette
    inside the sweep (su3_sweep_measured) -- read the plaquette back, copy the configuration
    out (su3_links_get)."""
    import numpy as np
    import torch
    shape = su3.links_shape(L)
    host_in = torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
    host_out = torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
    stream = torch.cuda.Stream()
    with su3.Lattice(L, BETA, SEED, start=su3.SU3_HOT, precision=prec, stream=stream.cuda_stream) as lat:
        lat.get_links(host_in)  # the host-side start configuration
        for _ in range(warmup):
            lat.set_links(host_in)
            lat.sweep(sweeps_per_step - 1)
            lat.sweep_measured(1)
            lat.get_links(host_out)
        # events around the sweeps split each step into device sweep time and the rest
        # (host copies and layout conversion); they do not change what is timed
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        t0 = time.perf_counter()
        for e0, e1 in ev:
            lat.set_links(host_in)
            e0.record(stream)
            lat.sweep(sweeps_per_step - 1)
            lat.sweep_measured(1)
            e1.record(stream)
            lat.get_links(host_out)
        dt = time.perf_counter() - t0
        sweeps_ms = sum(e0.elapsed_time(e1) for e0, e1 in ev) / steps
    ups = 4 * int(np.prod(L)) * sweeps_per_step * steps / dt
    return {"value": ups, "unit": UNIT, "h2d_bytes_per_step": int(host_in.nbytes),
            "d2h_bytes_per_step": int(host_out.nbytes) + 8, "ms_per_step": dt / steps * 1e3,
            "sweeps_ms_per_step": sweeps_ms, "transfer_and_host_ms_per_step": dt / steps * 1e3 - sweeps_ms,
            "step": "su3_links_set(host) + %d sweeps, the last with the fused plaquette (su3_sweep_measured) "
                    "+ su3_links_get(host)" % sweeps_per_step}


# --- the oracle on every host core -------------------------------------------
# The links of one checkerboard half-sweep never enter each other's staples, so
# disjoint site subsets of a half-sweep can be updated in place by separate
# processes running the unchanged oracle.  The configuration lives in a
# file-backed shared mapping; the pool is spawned (never forked).
_POOL_U = None


def _pool_attach(path, shape):
    global _POOL_U
    import numpy as np
    _POOL_U = np.memmap(path, dtype=np.float64, mode="r+", shape=shape)


def _pool_update(job):
    import oracle
    L, beta, seed, t, mu, sites = job
    oracle.update_links(L, beta, seed, t, mu, sites, _POOL_U)
    return len(sites)


class OraclePool:
    """The oracle's half-sweep split over `procs` spawned single-thread processes."""

    def __init__(self, L, U0, procs=None):
        import concurrent.futures as cf
        import multiprocessing as mp
        import tempfile
        import numpy as np
        self.L = tuple(L)
        self.procs = procs or os.cpu_count() or 1
        fd, self.path = tempfile.mkstemp(prefix="su3_oracle_links_", suffix=".bin")
        os.close(fd)
        U = np.memmap(self.path, dtype=np.float64, mode="w+", shape=U0.shape)
        U[...] = U0
        U.flush()
        self.U = U
        s = np.arange(int(np.prod(L)), dtype=np.int64)
        x0 = s % L[0]
        r = s // L[0]
        par = (x0 + r % L[1] + (r // L[1]) % L[2] + r // (L[1] * L[2])) & 1
        self.sites = [np.array_split(s[par == p], self.procs) for p in (0, 1)]
        self.ex = cf.ProcessPoolExecutor(max_workers=self.procs, mp_context=mp.get_context("spawn"),
                                         initializer=_pool_attach, initargs=(self.path, U0.shape))

    def half_sweep(self, beta, seed, t, mu, p):
        jobs = [(self.L, beta, seed, t, mu, c) for c in self.sites[p]]
        return sum(self.ex.map(_pool_update, jobs))

    def close(self):
        self.ex.shutdown()
        del self.U
        os.remove(self.path)


def host_cpu_model():
    """Host CPU model as the OS reports it (lscpu, else /proc/cpuinfo, else platform)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def cpu_baseline_sample(f32):
    """The oracle as it stands on the same 32^4 workload: on every host core (spawned
    processes on disjoint site subsets of each half-sweep, two full sweeps), and on one
    core (one full sweep)."""
    import oracle
    oracle.build()
    U = oracle.hot_start(DIMS, SEED, f32=f32)
    pool = OraclePool(DIMS, U)
    try:
        pool.half_sweep(BETA, SEED, 0, 0, 0)  # start the workers, load the library
        t0 = time.perf_counter()
        n = 0
        for t in range(1, 3):
            for mu in range(4):
                for p in range(2):
                    n += pool.half_sweep(BETA, SEED, t, mu, p)
        dt_all = time.perf_counter() - t0
        procs = pool.procs
    finally:
        pool.close()
    t0 = time.perf_counter()
    oracle.sweep(DIMS, BETA, SEED, 0, 1, U, f32=f32)
    dt = time.perf_counter() - t0
    one = 4 * 32 ** 4 / dt
    return {"value": n / dt_all, "unit": UNIT, "cores": procs, "kind": "oracle", "cpu_model": host_cpu_model(),
            "sample": "two full sweeps (2*4*32^4 link updates) of the 32^4 beta=5.7 hot-start lattice, %s, "
                      "%d single-thread processes on disjoint site subsets of each half-sweep, %.1f s"
                      % ("FP32-mixed reading" if f32 else "FP64", procs, dt_all),
            "one_core": {"value": one, "cores": 1, "us_per_update": dt / (4 * 32 ** 4) * 1e6,
                         "sample": "one full sweep, single thread, %.1f s" % dt}}


def run_reference(args):
    """The reference arm: the oracle as it stands on every host core (spawned
    single-thread processes on disjoint site subsets); one step = one checkerboard
    half-sweep of the 32^4 lattice."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    pool = OraclePool(DIMS, oracle.hot_start(DIMS, SEED))
    phases = [(mu, p) for mu in range(4) for p in range(2)]
    try:
        for i in range(args.warmup):
            mu, p = phases[i % 8]
            pool.half_sweep(BETA, SEED, i // 8, mu, p)
        t0 = time.perf_counter()
        n = 0
        for i in range(args.steps):
            mu, p = phases[(args.warmup + i) % 8]
            n += pool.half_sweep(BETA, SEED, (args.warmup + i) // 8, mu, p)
        dt = time.perf_counter() - t0
        procs = pool.procs
    finally:
        pool.close()
    ups = n / dt
    line = {"impl": "reference", "metric": METRIC, "value": ups, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": ups / PAPER_UPS, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "32^4 beta=5.7 hot start seed 7, FP64 checkerboard heatbath; reference step = "
                                   "one half-sweep (V/2 link updates) of the FP64 CPU oracle",
                       "lattice": list(DIMS), "beta": BETA},
            "cpu_baseline": {"value": ups, "unit": UNIT, "cores": procs, "kind": "oracle",
                             "cpu_model": host_cpu_model(),
                             "sample": "one checkerboard half-sweep of the 32^4 lattice per step, %d single-thread "
                                       "processes on disjoint site subsets" % procs},
            "e2e": {"value": ups, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def variant_fp32(su3, stream, steps, warmup, world, hbm_peak, peak_kind, precision=None, schedule=None):
    """The FP32 sweep of the 32^4 lattice.  schedule: None = the library's
    default (at 32^4 the eight chained half-sweep kernels), or another
    su3.SU3_SCHED_* form.  The events
    bracket each sweep's graph (counter reset, sweep kernels, sweep-counter
    increment), so the kernel time below slightly overstates the kernels' own."""
    import numpy as np
    if precision is None:
        precision = su3.SU3_FP32_MIXED
    eft = precision == su3.SU3_FP32_EFT
    with su3.Lattice(DIMS, BETA, SEED, start=su3.SU3_HOT, precision=precision,
                     stream=stream.cuda_stream) as lat:
        if schedule is not None:
            lat.set_schedule(schedule)
        sched = lat.schedule
        total_ms, sweep_ms, _ = time_sweeps(lat, stream, steps, warmup, SWEEPS_PER_STEP, world)
        plaq = lat.plaquette()
    V = int(np.prod(DIMS))
    ups = 4 * V * SWEEPS_PER_STEP * steps / (total_ms * 1e-3)
    # launches per sweep, traffic key suffix, kernel, description of each form
    forms = {
        su3.SU3_SCHED_PERSISTENT: (1, "_onelaunch", "k_sweep_f32_pair<-1> (site-paired FP32 sweep: the eight "
                                   "half-sweeps in one launch)", "one persistent kernel per sweep"),
        su3.SU3_SCHED_PER_DIRECTION: (4, "_perdir", "k_sweep_f32_pair<mu> (site-paired FP32 sweep of one direction: "
                                      "two half-sweeps per launch, four chained launches per sweep)",
                                      "one persistent kernel per direction"),
        su3.SU3_SCHED_CHAINED: (8, "", "k_half_sweep_f32_chain<mu> (site-paired FP32 half-sweep, eight chained "
                                "launches per sweep)", "eight chained half-sweep kernels per sweep"),
        su3.SU3_SCHED_PHASES: (8, "_phases", "k_half_sweep_f32_pair (site-paired FP32 half-sweep, eight launches "
                               "per sweep)", "eight half-sweep kernels per sweep"),
    }
    launches, suffix, kernel, form = forms[sched]
    kernel_ms = statistics.mean(sweep_ms) / launches
    bytes_per_launch = BYTES_PER_UPDATE["fp32_mixed"] * (V // 2) * (8 // launches)
    achieved = bytes_per_launch / (kernel_ms * 1e-3) / 1e9
    gs = ("Gram-Schmidt coefficients as compensated FP32 sums (error-free transformations, ~2^-47)" if eft
          else "FP64 Gram-Schmidt coefficients")
    traffic, provenance = traffic_of(("fp32_eft" if eft else "fp32_mixed") + suffix)
    return {"workload": "32^4 beta=5.7 hot start seed 7, FP32-mixed (12-real FP32 links, FP32 staple and "
                        "heatbath, %s), 2 sweeps/step, %s" % (gs, form),
            "value": ups, "unit": UNIT, "ms_per_step": total_ms / steps,
            "dtype": "f32 (compensated-f32 reunitarisation)" if eft else "f32 (f64 reunitarisation)",
            "plaquette_after": plaq,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "peak_kind": peak_kind,
                         "traffic": traffic, "traffic_source": provenance,
                         "kernel": kernel, "bytes_per_launch": bytes_per_launch, "kernel_ms": kernel_ms}}


def variant_measured(su3, stream, steps, warmup, precision):
    """Sweeps that also measure the plaquette after every sweep: fused into the
    update kernels (su3_sweep_measured) against a separate su3_plaquette pass
    after each sweep; both timed with CUDA events on the lattice's stream."""
    import numpy as np
    import torch
    V = int(np.prod(DIMS))
    n = steps * SWEEPS_PER_STEP
    out = {}
    with su3.Lattice(DIMS, BETA, SEED, start=su3.SU3_HOT, precision=precision,
                     stream=stream.cuda_stream) as lat:
        lat.sweep_measured(warmup * SWEEPS_PER_STEP)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fused = lat.sweep_measured(n)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out["fused"] = {"value": 4 * V * n / (ms * 1e-3), "ms_per_sweep": ms / n}
        e0.record(stream)
        sep = []
        for _ in range(n):
            lat.sweep(1)
            sep.append(lat.plaquette())
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out["separate"] = {"value": 4 * V * n / (ms * 1e-3), "ms_per_sweep": ms / n}
    out.update({"unit": UNIT, "plaquettes_fused_last": float(fused[-1]), "plaquettes_separate_last": sep[-1],
                "workload": "32^4 beta=5.7 hot start seed 7, %s, plaquette after every sweep"
                            % ("FP64" if precision == su3.SU3_FP64 else "FP32-mixed")})
    return out


def run_profile_case(case):
    import paper_0904_1179_gb300 as su3
    if case in ("batched", "batched_eft"):
        from paper_0904_1179_gb300.workloads import batch_96
        dims, betas, seeds = batch_96()
        prec = su3.SU3_FP32_EFT if case == "batched_eft" else su3.SU3_FP32_MIXED
        with su3.Batch(dims, betas, seeds, start=su3.SU3_HOT, precision=prec) as b:
            b.config(256, 0, 48)  # the autotuner's usual choice on GB300
            b.sweep(3)
            p = b.plaquettes()
        print(json.dumps({"profile_case": case, "replicas": len(dims), "sweeps": 3, "plaquette_0": p[0]}))
        return 0
    if case == "decomp16":
        with su3.Lattice(DIMS, BETA, SEED, start=su3.SU3_HOT, precision=su3.SU3_FP32_MIXED, decomp=(4, 2, 1)) as lat:
            lat.sweep(3)
            print(json.dumps({"profile_case": case, "lattice": list(DIMS), "decomp": [4, 2, 1],
                              "halo_links_per_sweep": lat.decomp_info()[4], "plaquette": lat.plaquette()}))
        return 0
    dims, beta = (DIMS, BETA)
    schedule = None
    if case.endswith("_phases"):  # the eight half-sweep kernels instead of the persistent sweep
        schedule, case = su3.SU3_SCHED_PHASES, case[:-7]
    elif case.endswith("_perdir"):  # one persistent launch per direction
        schedule, case = su3.SU3_SCHED_PER_DIRECTION, case[:-7]
    elif case.endswith("_onelaunch"):  # the whole sweep in one persistent launch
        schedule, case = su3.SU3_SCHED_PERSISTENT, case[:-10]
    if case.endswith("_64"):
        dims, beta, case = (64, 64, 64, 64), 6.0, case[:-3]
    elif case.endswith("_64s"):  # 64^3 x 16: the x3 lines of 64^4 in 805 MB (FP32)
        dims, beta, case = (64, 64, 64, 16), 6.0, case[:-4]
    elif case.endswith("_48"):
        dims, case = (48, 48, 48, 48), case[:-3]
    elif case.endswith("_8"):
        dims, case = (8, 8, 8, 8), case[:-2]
    prec = {"fp64": su3.SU3_FP64, "fp32_mixed": su3.SU3_FP32_MIXED, "fp32_eft": su3.SU3_FP32_EFT}[case]
    with su3.Lattice(dims, beta, SEED, start=su3.SU3_HOT, precision=prec) as lat:
        if schedule is not None:
            lat.set_schedule(schedule)
        lat.sweep(3)
        print(json.dumps({"profile_case": case, "lattice": list(dims), "sweeps": 3, "schedule": lat.schedule,
                          "plaquette": lat.plaquette()}))
    return 0


_BATCH_KERNEL = "k_batch_sweep_c<mu> (one block per work item; four per-direction launches per sweep)"
_BATCH_NOTE = ("the four launches of a sweep run back to back (launches 1-3 programmatic dependent launches), "
               "so the unit here is one sweep of all replicas: its algorithmic bytes over its duration "
               "(the counter reset included), and its DRAM traffic summed over the four launches")


def variant_batched_eft(su3, stream, steps, warmup, hbm_peak, peak_kind):
    """The same 96 replicas in the FP32-EFT precision (compensated-FP32 Gram-Schmidt
    coefficients), four chained per-direction launches per sweep, autotuned."""
    import torch
    from paper_0904_1179_gb300.workloads import batch_96, updates_per_sweep
    dims, betas, seeds = batch_96()
    ups = updates_per_sweep(dims)
    with su3.Batch(dims, betas, seeds, start=su3.SU3_HOT, precision=su3.SU3_FP32_EFT,
                   stream=stream.cuda_stream) as b:
        cfg = b.autotune()
        for _ in range(warmup):
            b.sweep(1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.sweep(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        b.status()
        sweep_ms = e0.elapsed_time(e1) / steps
    achieved = BYTES_PER_UPDATE["fp32_mixed"] * ups / (sweep_ms * 1e-3) / 1e9
    traffic, provenance = traffic_of("batched_eft")
    return {"workload": "the 96 replicas of variant 'batched' in FP32-EFT", "value": ups / (sweep_ms * 1e-3),
            "unit": UNIT, "ms_per_step": sweep_ms, "dtype": "f32 (compensated-f32 reunitarisation)",
            "autotuned": {"threads": cfg[0], "blocks_per_sm": cfg[1], "window": cfg[2]},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "peak_kind": peak_kind, "traffic": traffic,
                         "traffic_source": provenance, "kernel": _BATCH_KERNEL,
                         "bytes_per_launch": BYTES_PER_UPDATE["fp32_mixed"] * ups, "kernel_ms": sweep_ms,
                         "note": _BATCH_NOTE}}


def variant_batched(su3, stream, steps, warmup, hbm_peak, peak_kind):
    """96 uneven FP32-mixed replicas, four chained per-direction launches per sweep in one graph
    (autotuned outside the timed region), against the same replicas swept one by one."""
    import torch
    from paper_0904_1179_gb300.workloads import batch_96, updates_per_sweep
    dims, betas, seeds = batch_96()
    ups = updates_per_sweep(dims)
    with su3.Batch(dims, betas, seeds, start=su3.SU3_HOT, precision=su3.SU3_FP32_MIXED,
                   stream=stream.cuda_stream) as b:
        cfg = b.autotune()
        for _ in range(warmup):
            b.sweep(1)
        torch.cuda.synchronize()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        evs[0].record(stream)
        for i in range(steps):
            b.sweep(1)
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
        b.status()
        total_ms = evs[0].elapsed_time(evs[-1])
    value = ups * steps / (total_ms * 1e-3)
    # the same 96 lattices, one handle each, swept one after the other
    lats = [su3.Lattice(L, be, s, start=su3.SU3_HOT, precision=su3.SU3_FP32_MIXED, stream=stream.cuda_stream)
            for L, be, s in zip(dims, betas, seeds)]
    try:
        for _ in range(warmup):
            for lat in lats:
                lat.sweep(1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            for lat in lats:
                lat.sweep(1)
        e1.record(stream)
        torch.cuda.synchronize()
        one_by_one = ups * steps / (e0.elapsed_time(e1) * 1e-3)
    finally:
        for lat in lats:
            lat.close()
    sweep_ms = total_ms / steps
    achieved = BYTES_PER_UPDATE["fp32_mixed"] * ups / (sweep_ms * 1e-3) / 1e9
    traffic, provenance = traffic_of("batched")
    return {"workload": "96 replicas (32x 8^4, 32x 12^4, 16x 16^4, 16x 8^3x16), beta in [5.5, 6.2], hot starts "
                        "seed 1000+r, FP32-mixed; step = 1 sweep of every replica = four chained launches",
            "value": value, "unit": UNIT, "ms_per_step": sweep_ms, "dtype": "f32 (f64 reunitarisation)",
            "updates_per_step": ups, "autotuned": {"threads": cfg[0], "blocks_per_sm": cfg[1], "window": cfg[2]},
            "one_by_one": {"value": one_by_one, "unit": UNIT, "speedup": value / one_by_one},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "peak_kind": peak_kind, "traffic": traffic,
                         "traffic_source": provenance, "kernel": _BATCH_KERNEL,
                         "bytes_per_launch": BYTES_PER_UPDATE["fp32_mixed"] * ups, "kernel_ms": sweep_ms,
                         "note": _BATCH_NOTE}}


def binned_mean(x, nbins=20):
    import numpy as np
    x = np.asarray(x, dtype=np.float64)
    b = x[: (x.size // nbins) * nbins].reshape(nbins, -1).mean(axis=1)
    return float(b.mean()), float(b.std(ddof=1) / np.sqrt(nbins))


def tau_int(x, c=6.0):
    """Integrated autocorrelation time with the self-consistent window W >= c tau
    (Madras and Sokal, J. Stat. Phys. 50 (1988) 109), from the FFT autocovariance."""
    import numpy as np
    x = np.asarray(x, dtype=np.float64) - np.mean(x)
    n = x.size
    f = np.fft.rfft(x, 2 * n)
    acf = np.fft.irfft(f * np.conj(f))[:n] / np.arange(n, 0, -1)
    acf /= acf[0]
    tau = 0.5
    for w in range(1, n // 4):
        tau += acf[w]
        if w >= c * tau:
            break
    return float(tau)


def run_chains(args):
    """Plaquette chains of the precision study: 32^4 and 48^4 at beta 5.7 and 6.0, hot start,
    thermalisation then measured sweeps with the plaquette after every sweep (fused into the
    sweep), in FP64, FP32-mixed and FP32-EFT from the same Philox seed; prints one JSON line
    per (lattice, beta) with the means, errors from 20 bins (each bin many autocorrelation
    times long), the integrated autocorrelation time, and the deviations of the FP32 chains
    from the FP64 chain."""
    import numpy as np
    import paper_0904_1179_gb300 as su3
    cases = [((32, 32, 32, 32), 5.7), ((32, 32, 32, 32), 6.0), ((48, 48, 48, 48), 5.7), ((48, 48, 48, 48), 6.0)]
    if args.chains_small:
        cases = [((8, 8, 8, 8), 5.7)]
    if args.chains_case:
        ext, b = args.chains_case.split(":")
        cases = [((int(ext),) * 4, float(b))]
    seed = args.chains_seed
    precs = [("fp64", su3.SU3_FP64), ("fp32_mixed", su3.SU3_FP32_MIXED), ("fp32_eft", su3.SU3_FP32_EFT)]
    for L, beta in cases:
        big = int(np.prod(L)) > 32 ** 4
        ntherm = args.chains_therm if not big else max(args.chains_therm * 3 // 5, 1)
        nmeas = args.chains_meas if not big else max(args.chains_meas * 5 // 16, 20)
        res = {}
        for name, prec in precs:
            t0 = time.perf_counter()
            with su3.Lattice(L, beta, seed, start=su3.SU3_HOT, precision=prec) as lat:
                lat.sweep(ntherm)
                plaq = lat.sweep_measured(nmeas)
                lat.set_stats(True)
                lat.sweep(10)
                acc, prop = lat.stats()
            m, e = binned_mean(plaq)
            _, e40 = binned_mean(plaq, 40)
            tau = tau_int(plaq)
            res[name] = {"mean": m, "err": e, "err_40bins": e40, "tau_int": tau,
                         "err_tau": float(np.std(plaq, ddof=1) * np.sqrt(2 * tau / len(plaq))),
                         "acceptance": acc / prop, "seconds": time.perf_counter() - t0}
        out = {"chains": True, "lattice": list(L), "beta": beta, "therm": ntherm, "measured": nmeas, "seed": seed,
               "start": "hot", "bins": 20, **res}
        for name in ("fp32_mixed", "fp32_eft"):
            d = res[name]["mean"] - res["fp64"]["mean"]
            sig = (res[name]["err"] ** 2 + res["fp64"]["err"] ** 2) ** 0.5
            out["delta_" + name] = {"value": d, "sigma": sig, "n_sigma": d / sig}
        print(json.dumps(out), flush=True)
    return 0


def run_table1(args):
    """The paper's Table 1 workloads in full, FP64 on the GPU: 8^4 x 512, 12^4 x 101,
    16^4 x 32 and 32^4 x 2 sweeps at beta 5.7 from the seed-7 hot start (each column
    the same 8.39 M link updates).  CUDA events around the n sweeps of each column
    (the sweep graph built beforehand, the start configuration restored).  With the
    CPU baseline on, the oracle runs the four columns in full at the same time, one
    spawned single-thread process per column."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import numpy as np
    from paper_0904_1179_gb300.workloads import TABLE1, HEADLINE_SEED
    pool = futs = None
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        pool = cf.ProcessPoolExecutor(max_workers=len(TABLE1), mp_context=mp.get_context("spawn"))
        futs = [pool.submit(oracle.hot_chain, L, BETA, HEADLINE_SEED, n) for L, n in TABLE1]
    import torch
    import paper_0904_1179_gb300 as su3
    stream = torch.cuda.Stream()
    cols = []
    for (L, n), paper_s in zip(TABLE1, PAPER_TABLE1_SECONDS):
        V = int(np.prod(L))
        row = {"lattice": list(L), "sweeps": n, "updates": 4 * V * n, "paper_1core_s": paper_s}
        for prec, name in ((su3.SU3_FP64, "fp64"), (su3.SU3_FP32_MIXED, "fp32_mixed")):
            with su3.Lattice(L, BETA, HEADLINE_SEED, start=su3.SU3_HOT, precision=prec,
                             stream=stream.cuda_stream) as lat:
                U0 = lat.get_links()
                lat.sweep(1)  # builds the sweep graph
                lat.set_links(U0)
                lat.sweep_count = 0
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                lat.sweep(n)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                row[name] = {"seconds": ms * 1e-3, "value": 4 * V * n / (ms * 1e-3), "plaquette": lat.plaquette()}
        cols.append(row)
    if futs:
        for row, f in zip(cols, futs):
            _, plaq, _, secs = f.result()
            row["oracle_1core"] = {"seconds": secs, "us_per_update": secs / row["updates"] * 1e6,
                                   "plaquette": float(plaq[-1])}
        pool.shutdown()
    print(json.dumps({"mode": "table1", "unit": UNIT, "beta": BETA, "seed": HEADLINE_SEED, "columns": cols,
                      "note": "paper: non-MPI Fortran program on one 2 GHz Intel E5405 core (Table 1, first row); "
                              "oracle: plain C FP64 program, one host core per column, four columns at once"}))
    return 0


def run_oracle_configs(args):
    """The oracle timed on the other workloads, in microseconds per link update: one
    full sweep of 48^4 (beta 5.7) and of 64^4 (beta 6.0) on every host core (spawned
    processes on disjoint site subsets, as the CPU baseline; the configuration is an
    oracle hot start of a 12^4 / 8^4 cell repeated), and one sweep of one replica of
    each lattice size of the 96-replica batch on one core."""
    import numpy as np
    import oracle
    from paper_0904_1179_gb300.workloads import batch_96
    oracle.build()
    out = {"mode": "oracle_configs", "unit": "us per link update", "kind": "oracle", "rows": []}
    for L, beta, cell in (((48, 48, 48, 48), 5.7, 12), ((64, 64, 64, 64), 6.0, 8)):
        # an oracle hot start on a small cell, repeated: a full hot start of 64^4
        # would take the oracle longer than the sweep being timed
        r = L[0] // cell
        U = np.tile(oracle.hot_start((cell,) * 4, SEED), (r, r, r, r, 1, 1, 1, 1))
        pool = OraclePool(L, U)
        del U
        try:
            pool.half_sweep(beta, SEED, 0, 0, 0)  # start the workers
            t0 = time.perf_counter()
            n = 0
            for mu in range(4):
                for p in range(2):
                    n += pool.half_sweep(beta, SEED, 1, mu, p)
            dt = time.perf_counter() - t0
            procs = pool.procs
        finally:
            pool.close()
        out["rows"].append({"lattice": list(L), "beta": beta, "sample": "one sweep", "cores": procs,
                            "seconds": dt, "core_us_per_update": dt * procs / n * 1e6,
                            "value": n / dt})
    dims, betas, seeds = batch_96()
    seen = {}
    for L, b, sd in zip(dims, betas, seeds):
        if tuple(L) in seen:
            continue
        U = oracle.hot_start(L, sd, f32=True)
        t0 = time.perf_counter()
        oracle.sweep(L, b, sd, 0, 1, U, f32=True)
        dt = time.perf_counter() - t0
        n = 4 * int(np.prod(L))
        seen[tuple(L)] = True
        out["rows"].append({"lattice": list(L), "beta": b, "sample": "one sweep of the first replica of this size, "
                            "FP32-mixed reading", "cores": 1, "seconds": dt, "core_us_per_update": dt / n * 1e6,
                            "value": n / dt})
    print(json.dumps(out))
    return 0


def run_decomp(args):
    """Table 1's structure on one GPU: each column (8^4 x 512 ... 32^4 x 2 sweeps, FP64,
    beta 5.7) undivided and cut like the paper's rows -- ndmpi = 1 with one sublattice and
    the boundary exchange on ("1"), then np = 2, 4, 8, 16 (ndmpi 1..4, mpifactor 2).  CUDA
    events around the n sweeps of each run (sweep graph built and sublattices filled by one
    sweep beforehand).  Each row's time is given against the undivided lattice in its
    one-thread-per-update form (vs_plain) and against the "1F" row (vs_1F): one sublattice
    with the exchange off runs the same sublattice kernel as the cut rows, so vs_1F is the
    cost of the cut and the exchange alone."""
    import numpy as np
    import torch
    import paper_0904_1179_gb300 as su3
    from paper_0904_1179_gb300.workloads import TABLE1, HEADLINE_SEED
    rows = [("plain", None), ("1F", (1, 1, 0)), ("1", (1, 1, 1)), ("2", (1, 2, 1)), ("4", (2, 2, 1)),
            ("8", (3, 2, 1)), ("16", (4, 2, 1))]
    stream = torch.cuda.Stream()
    precs = [(su3.SU3_FP64, "fp64"), (su3.SU3_FP32_MIXED, "fp32_mixed")]
    out = []
    for L, n in TABLE1:
        V = int(np.prod(L))
        col = {"lattice": list(L), "sweeps": n, "rows": {}}
        for prec, pname in precs:
            base = base1f = None
            for name, dec in rows:
                with su3.Lattice(L, BETA, HEADLINE_SEED, start=su3.SU3_HOT, precision=prec, decomp=dec,
                                 stream=stream.cuda_stream) as lat:
                    if dec is None:
                        lat.set_lanes(1)  # the sublattices run one thread per update too
                    lat.sweep(1)
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    lat.sweep(n)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    sec = e0.elapsed_time(e1) * 1e-3
                    info = lat.decomp_info()
                if base is None:
                    base = sec
                if name == "1F":
                    base1f = sec
                link_bytes = 144 if prec == su3.SU3_FP64 else 48
                col["rows"].setdefault(name, {})[pname] = {
                    "seconds": sec, "value": 4 * V * n / sec, "vs_plain": sec / base,
                    "vs_1F": sec / base1f if base1f else None,
                    "np": info[3], "halo_links_per_sweep": info[4],
                    "halo_bytes_per_sweep": 2 * info[4] * link_bytes}
        out.append(col)
    print(json.dumps({"mode": "decomp", "unit": UNIT, "beta": BETA, "columns": out,
                      "note": "rows as in Table 1: plain = the undivided lattice, one thread per update "
                              "(FP32: per link pair where L3 is a multiple of 4); 1F = one sublattice, "
                              "exchange off; 1 = one sublattice exchanging with itself; 2..16 = np sublattices "
                              "(ndmpi 1..4, mpifactor 2); vs_1F compares runs of the same sublattice kernel; "
                              "halo bytes count the read and the write of every copied link"}))
    return 0


def run_large(args):
    """64^4 at beta 6.0, hot start seed 7, 100 sweeps: FP64 against FP32-mixed side by side."""
    import numpy as np
    import torch
    import paper_0904_1179_gb300 as su3
    L = (64, 64, 64, 64)
    V = int(np.prod(L))
    nsw = args.large_sweeps
    out = {"large": True, "lattice": list(L), "beta": 6.0, "sweeps": nsw}
    for name, prec in (("fp32_mixed", su3.SU3_FP32_MIXED), ("fp32_eft", su3.SU3_FP32_EFT), ("fp64", su3.SU3_FP64)):
        stream = torch.cuda.Stream()
        with su3.Lattice(L, 6.0, 7, start=su3.SU3_HOT, precision=prec, stream=stream.cuda_stream) as lat:
            total_ms, sweep_ms, _ = time_sweeps(lat, stream, nsw, 3, 1, 1)
            p = lat.plaquette()
        ups = 4 * V * nsw / (total_ms * 1e-3)
        bpu = BYTES_PER_UPDATE["fp64" if prec == su3.SU3_FP64 else "fp32_mixed"]
        out[name] = {"value": ups, "unit": UNIT, "ms_per_sweep": total_ms / nsw, "plaquette_after": p,
                     "algorithmic_GBps": bpu * ups / 1e9}
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--chains", action="store_true", help="precision study: FP64 vs FP32 plaquette chains")
    ap.add_argument("--chains-small", action="store_true", help="one small chain (8^4) instead of 32^4/48^4")
    ap.add_argument("--chains-seed", type=int, default=11)
    ap.add_argument("--chains-case", help="one case only, extent:beta, e.g. 48:5.7")
    ap.add_argument("--chains-therm", type=int, default=500, help="thermalisation sweeps (48^4: 3/5 of it)")
    ap.add_argument("--chains-meas", type=int, default=8000, help="measured sweeps (48^4: 5/16 of it)")
    ap.add_argument("--large", action="store_true", help="64^4 beta 6.0, FP64 vs FP32-mixed")
    ap.add_argument("--oracle-configs", action="store_true",
                    help="the oracle's microseconds per update on 48^4, 64^4 and the batch's lattice sizes")
    ap.add_argument("--decomp", action="store_true",
                    help="Table 1's rows on one GPU: the domain decomposition emulated, exchange cost measured")
    ap.add_argument("--table1", action="store_true",
                    help="the paper's Table 1 columns in full (FP64 and FP32-mixed), with the oracle beside them")
    ap.add_argument("--large-sweeps", type=int, default=100)
    ap.add_argument("--profile", choices=["fp64", "fp32_mixed", "fp32_eft", "batched", "batched_eft", "fp64_64", "fp32_mixed_64", "decomp16",
                             "fp64_8", "fp32_mixed_64s", "fp32_eft_64s", "fp32_mixed_48", "fp32_eft_48",
                             "fp32_mixed_phases", "fp32_eft_phases", "fp32_mixed_onelaunch", "fp32_eft_onelaunch",
                             "fp32_mixed_perdir", "fp32_eft_perdir"],
                    help="small case for ncu: create the 32^4 lattice (or the 96-replica batch) and run 3 graphed "
                         "sweeps, nothing else")
    args = ap.parse_args()
    if args.profile:
        return run_profile_case(args.profile)
    if args.chains:
        return run_chains(args)
    if args.large:
        return run_large(args)
    if args.table1:
        return run_table1(args)
    if args.decomp:
        return run_decomp(args)
    if args.oracle_configs:
        return run_oracle_configs(args)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import paper_0904_1179_gb300 as su3

    rank, world, local = dist_setup()
    device = torch.device("cuda", local)
    hbm_peak, peak_kind = peaks()
    stream = torch.cuda.Stream(device=device)
    V = int(np.prod(DIMS))

    with su3.Lattice(DIMS, BETA, SEED + rank, start=su3.SU3_HOT, precision=su3.SU3_FP64,
                     stream=stream.cuda_stream) as lat:
        sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
        total_ms, sweep_ms, clocks = time_sweeps(lat, stream, args.steps, args.warmup, SWEEPS_PER_STEP, world, sampler)
        plaq = lat.plaquette()
    units = 4.0 * V * SWEEPS_PER_STEP * args.steps
    secs, all_units = reduce_max_sum(world, total_ms * 1e-3, units, device)
    value = all_units / secs
    kernel_ms = statistics.mean(sweep_ms) / 8
    flop_per_launch = FP64_FLOP_PER_UPDATE * (V // 2)
    achieved_tf = flop_per_launch / (kernel_ms * 1e-3) / 1e12

    if rank != 0:
        barrier(world)
        return 0

    variants = {}
    if not args.no_variants:
        variants["fp32_mixed"] = variant_fp32(su3, stream, args.steps, args.warmup, 1, hbm_peak, peak_kind)
        variants["fp32_eft"] = variant_fp32(su3, stream, args.steps, args.warmup, 1, hbm_peak, peak_kind,
                                            su3.SU3_FP32_EFT)
        # like for like: the same sweeps as eight half-sweep kernels
        variants["fp32_mixed_phases"] = variant_fp32(su3, stream, args.steps, args.warmup, 1, hbm_peak, peak_kind,
                                                     schedule=su3.SU3_SCHED_PHASES)
        variants["fp32_eft_phases"] = variant_fp32(su3, stream, args.steps, args.warmup, 1, hbm_peak, peak_kind,
                                                   su3.SU3_FP32_EFT, schedule=su3.SU3_SCHED_PHASES)
        variants["batched"] = variant_batched(su3, stream, args.steps, args.warmup, hbm_peak, peak_kind)
        variants["batched_eft"] = variant_batched_eft(su3, stream, args.steps, args.warmup, hbm_peak, peak_kind)
        variants["measured_fp64"] = variant_measured(su3, stream, args.steps, args.warmup, su3.SU3_FP64)
        variants["measured_fp32_mixed"] = variant_measured(su3, stream, args.steps, args.warmup, su3.SU3_FP32_MIXED)
    e2e = time_e2e(su3, DIMS, su3.SU3_FP64, max(3, args.steps // 4), 3, SWEEPS_PER_STEP)
    cpu = None if args.no_cpu_baseline else cpu_baseline_sample(False)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": value / PAPER_UPS, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "32^4 periodic lattice, beta=5.7, hot start (Haar, Philox seed 7), FP64 links, "
                               "checkerboard Cabibbo-Marinari one-hit heatbath; step = 2 sweeps (paper Table 1 "
                               "32^4 column)",
                   "lattice": list(DIMS), "beta": BETA, "seed": SEED, "sweeps_per_step": SWEEPS_PER_STEP,
                   "precision": "fp64", "parallelism": "replicas" if world > 1 else "single",
                   "l2": "no flush: the 604 MB link store exceeds the 129 MB L2",
                   "plaquette_after": plaq},
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": args.steps * SWEEPS_PER_STEP * 9,
        "gpu_launches_note": "headline timed region: per sweep 8 half-sweep kernels + 1 sweep-counter kernel",
        "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved_tf / FP64_PEAK_TFLOPS, "traffic": traffic_of("fp64")[0],
                     "traffic_source": traffic_of("fp64")[1],
                     "peak_kind": "derived: 152 SMs x 2 FP64 FMA/clock x 2 flop x 2.070 GHz",
                     "probe_peak": FP64_PROBE_TFLOPS, "frac_of_probe": achieved_tf / FP64_PROBE_TFLOPS,
                     "kernel": "k_half_sweep_f64", "flop_per_launch": flop_per_launch, "kernel_ms": kernel_ms,
                     "hbm_frac": BYTES_PER_UPDATE["fp64"] * (V // 2) / (kernel_ms * 1e-3) / 1e9 / hbm_peak,
                     "hbm_peak": hbm_peak, "hbm_peak_kind": peak_kind},
        "cpu_baseline": cpu,
        "variants": variants,
    }
    print(json.dumps(line))
    barrier(world)
    return 0


if __name__ == "__main__":
    sys.exit(main())
