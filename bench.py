"""Throughput of the two-timescale multicomponent LB step on GB300.

Workload (default): charged ternary mixture (solvent, cation z=+1, anion
z=-1), D3Q19, 128^3 periodic, ion number fractions 0.01 +/- U(1e-3) seeded,
Bjerrum length 0.7, Poisson solved every step to a relative residual of
1e-8 (spectral solver; the multigrid solver is timed beside it), Sc = 1,
FP32.  One step = charge density + Poisson solve + fused
stream/collide of all species, each step one CUDA-graph replay (the
library's LBM_FLAG_STEP_GRAPH; --host-steps drives the steps from the host
instead).  Metric: species-site MLUPS (S * N * steps / time / 1e6), with
the stream/collide kernel's fraction of the measured HBM roofline and the
Poisson iterations per step.  A host-stepped run of the same workload
gives the per-phase CUDA-event times (phase_ms_per_step, host_steps).
Each Poisson solve starts from the extrapolation of the three previous
potentials (--no-extrapolation: from the previous one).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the only other implementation:
the paper ships no code) on bounded samples of the same workload, one
single-threaded instance per host core.
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
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "species-site MLUPS & % HBM roofline; Poisson iters/step, learned vs plain"
UNIT = "species-site MLUPS"
BYTES_PER_SPECIES_SITE = {"fp32": 152, "fp16": 76, "bf16": 76}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    # the benchmark's protocol: 100 timed steps after 10 warm-up steps (the
    # bulk charge relaxes over the run; later steps need fewer Poisson
    # applications, so longer runs would flatter the rate)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--schmidt", type=float, default=1.0)
    ap.add_argument("--storage", default="fp32", choices=["fp32", "fp16", "bf16"])
    ap.add_argument("--poisson", default="fft", choices=["mg", "sor", "fft"])
    ap.add_argument("--no-alt", action="store_true", help="skip the multigrid comparison run")
    ap.add_argument("--only", choices=["batched", "learned", "slit", "conductivity", "slit_transport",
                                       "multigrid", "porous"], default=None,
                    help="run one extra measurement alone and print it")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched-slit and learned-guess measurements")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--host-steps", action="store_true",
                    help="headline with host-driven steps instead of CUDA-graph steps")
    ap.add_argument("--no-extrapolation", action="store_true",
                    help="spectral solves start from the previous potential, not its "
                         "extrapolation in time")
    ap.add_argument("--charge-pass", action="store_true",
                    help="charge density by a separate pass over the charged populations "
                         "(LBM_FLAG_CHARGE_PASS), not scattered by the previous stream/collide")
    return ap.parse_args()


def dist_env():
    from paper_1507_04891_gb300 import replicas
    return replicas.env()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def collide_source_hash():
    """Hash of the stream/collide kernel's source: the kernel unit and the
    device helpers it includes, with comments and blank space removed (a
    comment edit leaves the counters of a profile valid)."""
    import re
    csrc = os.path.join(ROOT, "paper_1507_04891_gb300", "csrc")
    text = "".join(open(os.path.join(csrc, f)).read() for f in ("lbm_lattice.cuh", "lbm_collide.cu"))
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    text = " ".join(text.split())
    return hashlib.sha256(text.encode()).hexdigest()[:16]


def kernel_traffic(storage="fp32", variant=""):
    """DRAM bytes per stream/collide launch from the committed ncu summary,
    valid only while the kernel source is unchanged (hash recorded there)."""
    path = os.path.join(ROOT, "profiles", "stream_collide_ternary_128_%s%s.md" % (storage, variant))
    try:
        h = collide_source_hash()
        rec = {}
        for line in open(path):
            if line.startswith("- ") and ":" in line:
                k, v = line[2:].split(":", 1)
                rec[k.strip()] = v.strip().strip("`")
        if rec.get("kernel_source_sha256_16") != h:
            return None
        return float(rec["dram_bytes_per_launch"])
    except Exception:
        return None


class NvmlClockSampler:
    """SM clock and throttle reasons read through NVML (the driver's
    libnvidia-ml, via ctypes; read-only queries) every 2 ms from a thread
    while the timed steps run, so that even a 30 ms timed window holds
    samples.  Bits of the reasons mask from the public nvml.h: SW power cap
    0x4, HW slowdown 0x8, SW thermal 0x20, HW thermal 0x40."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown"}

    def __init__(self, index=0):
        import ctypes
        import threading
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        if self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(self.h)) != 0:
            raise RuntimeError("no NVML handle")
        self.reasons_fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        mx = ctypes.c_uint(0)
        self.lib.nvmlDeviceGetMaxClockInfo(self.h, ctypes.c_int(1), ctypes.byref(mx))
        self.max_mhz = float(mx.value)
        self.rows = []
        self.t0 = self.t1 = None
        self.stop_flag = threading.Event()
        self.thread = threading.Thread(target=self._run, daemon=True)

    def _run(self):
        ct = self.ct
        clk, bits = ct.c_uint(0), ct.c_ulonglong(0)
        while not self.stop_flag.is_set():
            t = time.time()
            ok = self.lib.nvmlDeviceGetClockInfo(self.h, ct.c_int(1), ct.byref(clk)) == 0
            ok = ok and self.reasons_fn(self.h, ct.byref(bits)) == 0
            if ok:
                self.rows.append((t, float(clk.value), int(bits.value)))
            time.sleep(0.002)

    def start(self):
        self.thread.start()

    def begin(self):
        self.t0 = time.time()

    def end(self):
        self.t1 = time.time()

    def stop(self):
        self.stop_flag.set()
        self.thread.join(timeout=5)
        try:
            self.lib.nvmlShutdown()
        except Exception:
            pass
        inside = [r for r in self.rows if self.t0 is not None and self.t1 is not None
                  and self.t0 <= r[0] <= self.t1]
        if not inside:
            return None
        reasons = sorted({n for r in inside for b, n in self.REASONS.items() if r[2] & b})
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": self.max_mhz,
                "reasons": reasons, "samples": len(inside), "source": "nvml",
                "window_s": round(self.t1 - self.t0, 3)}


def clock_sampler(index=0):
    """NVML sampler when the driver library loads, else nvidia-smi."""
    try:
        return NvmlClockSampler(index)
    except Exception:
        return ClockSampler(index)


class ClockSampler:
    """nvidia-smi samples (every 50 ms, timestamped) of the SM clock and the
    throttle reasons; stop() keeps the samples taken inside the window given
    by begin() / end() (host wall clock), or the one nearest to it when the
    window is shorter than the sampling interval."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, index=0):
        self.proc = None
        self.index = index
        self.path = os.path.join(tempfile.gettempdir(), "lbm_bench_clocks_%d.csv" % os.getpid())
        self.t0 = self.t1 = None

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # wait for the first sample so that the window is covered from its start
        deadline = time.time() + 5.0
        while time.time() < deadline and self.proc.poll() is None:
            try:
                if os.path.getsize(self.path) > 0:
                    break
            except OSError:
                pass
            time.sleep(0.02)

    def begin(self):
        self.t0 = time.time()

    def end(self):
        self.t1 = time.time()

    @staticmethod
    def _epoch(ts):
        from datetime import datetime
        return datetime.strptime(ts.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.06)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                t = self._epoch(parts[0])
                sm, mx = float(parts[1]), float(parts[2])
            except ValueError:
                continue
            rows.append((t, sm, mx, [n for n, v in zip(self.NAMES, parts[3:7]) if v.lower() == "active"]))
        if not rows:
            return None
        inside = rows
        if self.t0 is not None and self.t1 is not None:
            inside = [r for r in rows if self.t0 <= r[0] <= self.t1]
            if not inside:
                mid = 0.5 * (self.t0 + self.t1)
                inside = [min(rows, key=lambda r: abs(r[0] - mid))]
        reasons = sorted({n for r in inside for n in r[3]})
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": inside[-1][2],
                "reasons": reasons, "samples": len(inside), "source": "nvidia-smi",
                "window_s": None if self.t0 is None or self.t1 is None else round(self.t1 - self.t0, 3)}


def cpu_oracle_sample(n_sample=24, budget_s=12.0, schmidt=1.0):
    """Times the FP64 oracle in this process on a bounded sample of the
    workload: the same charged ternary physics on an n_sample^3 periodic
    lattice (the oracle's cost per node does not depend on the lattice size
    except through the Poisson solve).  Its sparse LU solve may use several
    BLAS threads: `cores` counts the threads available to it."""
    import oracle as O
    from paper_1507_04891_gb300 import workloads as WL

    wl = WL.ternary_bulk(shape=(n_sample,) * 3, seed=1235, schmidt=schmidt)
    p = O.Params(wl.omega_visc, O.omega_drag_for_schmidt(wl.omega_visc, schmidt), wl.mass,
                 wl.valence, bjerrum=wl.bjerrum)
    o = O.Oracle(p, wl.shape)
    o.initialise(wl.n0)
    o.step()
    t0 = time.perf_counter()
    steps = 0
    while steps < 3 or time.perf_counter() - t0 < budget_s:
        o.step()
        steps += 1
    dt = time.perf_counter() - t0
    mlups = 3 * wl.sites * steps / dt / 1e6
    return {"value": mlups, "unit": UNIT, "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
            "sample": "FP64 numpy oracle in one process (BLAS threads not limited), same charged "
                      "ternary physics (Sc=%g, l_B=0.7, Poisson each step) on a %d^3 periodic "
                      "lattice, %d timed steps after 1 untimed, %.1f s" % (schmidt, n_sample, steps, dt)}


def _oracle_proc(task, barrier, out):
    """One single-threaded oracle instance in a spawned process: builds its
    charged ternary sample (own seed), takes `warm` untimed steps, waits for
    all instances, then times `steps` steps; puts (updates, start, end) or
    the error text on `out`."""
    try:
        n_sample, seed, schmidt, warm, steps = task
        import oracle as O
        from paper_1507_04891_gb300 import workloads as WL
        wl = WL.ternary_bulk(shape=(n_sample,) * 3, seed=seed, schmidt=schmidt)
        p = O.Params(wl.omega_visc, O.omega_drag_for_schmidt(wl.omega_visc, schmidt), wl.mass,
                     wl.valence, bjerrum=wl.bjerrum)
        o = O.Oracle(p, wl.shape)
        o.initialise(wl.n0)
        for _ in range(warm):
            o.step()
        barrier.wait(timeout=180)
        t0 = time.time()
        for _ in range(steps):
            o.step()
        t1 = time.time()
        out.put((3 * wl.sites * steps, t0, t1))
    except Exception as ex:  # reported by the parent
        out.put(repr(ex))


def cpu_oracle_instances(procs, n_sample=24, warm=1, steps=40, schmidt=1.0):
    """The oracle as `procs` independent single-threaded instances (spawned
    processes with one BLAS thread each, distinct seeds), started together
    after their set-up and timed over the common interval from the first
    start to the last end of their timed loops.  The oracle itself is
    unchanged; the instances share no work."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    # one thread per instance: the children read these when numpy loads
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        barrier, out = ctx.Barrier(procs), ctx.Queue()
        ps = [ctx.Process(target=_oracle_proc,
                          args=((n_sample, 1235 + k, schmidt, warm, steps), barrier, out))
              for k in range(procs)]
        for q in ps:
            q.start()
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    try:
        res = [out.get(timeout=300) for _ in range(procs)]
    finally:
        for q in ps:
            q.join(timeout=30)
            if q.is_alive():
                q.terminate()
    bad = [r for r in res if not isinstance(r, tuple)]
    if bad:
        raise RuntimeError(bad[0])
    updates = sum(r[0] for r in res)
    wall = max(r[2] for r in res) - min(r[1] for r in res)
    return {"value": updates / wall / 1e6, "unit": UNIT, "cores": procs, "kind": "oracle",
            "ms_per_step": wall / steps * 1e3,
            "sample": "%d single-threaded FP64 oracle instance(s), one per core, each %d steps "
                      "after %d untimed on a %d^3 charged ternary sample (Sc=%g, l_B=0.7, Poisson "
                      "each step; seeds from 1235), started together, %.1f s from the first "
                      "start to the last end" % (procs, steps, warm, n_sample, schmidt, wall)}


def cpu_baseline(schmidt=1.0):
    """One core (one single-threaded instance), and every core beside it;
    the in-process sample if spawned processes are not available."""
    try:
        one = cpu_oracle_instances(1, steps=250, schmidt=schmidt)   # ~10 s on a GB300 host core
    except Exception as ex:
        one = cpu_oracle_sample(schmidt=schmidt)
        one["spawn_failed"] = repr(ex)
        return one
    one.pop("ms_per_step", None)
    try:
        allc = cpu_oracle_instances(len(os.sched_getaffinity(0)), steps=100, schmidt=schmidt)
        allc.pop("kind", None)
        one["all_cores"] = allc
    except Exception as ex:  # reported, never required
        one["all_cores"] = {"value": None, "sample": "failed: %s" % ex}
    return one


def run_reference(args, rank, world):
    """The oracle on the host cores: one single-threaded instance per core,
    each K timed steps after W untimed of a 24^3 sample of the workload;
    the in-process sample if spawned processes are not available."""
    if rank != 0:
        return 0
    steps = max(1, args.steps)
    warm = max(0, args.warmup)
    try:
        cb = cpu_oracle_instances(len(os.sched_getaffinity(0)), warm=warm, steps=steps,
                                  schmidt=args.schmidt)
        value, ms = cb.pop("value"), cb.pop("ms_per_step")
    except Exception as ex:
        cb = cpu_oracle_sample(schmidt=args.schmidt, budget_s=10.0)
        cb["spawn_failed"] = repr(ex)
        value = cb.pop("value")
        ms = 3 * 24 ** 3 / (value * 1e6) * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": steps, "warmup": warm, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "ternary_bulk_%d^3" % args.n, "sc": args.schmidt,
                       "bjerrum": 0.7, "poisson_tol": 1e-8},
            "cpu_baseline": dict(value=value, **cb),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_batched(lbm, WL, steps=40, local=0, extrapolate=True):
    """Batched slit sweep (64 channels, widths U{16..128}, 32x32, Sc
    log-uniform 1..1000, wall charge U[-0.02,-0.002]).  Three arms, each
    graph-stepped, so that each ratio changes one thing: the channels
    stacked in one lattice with FP16 storage (the batched form), the same
    stack with FP32 storage, and the 64 channels stepped one after another
    as separate FP32 lattices."""
    import torch
    insts = WL.batched_slits()
    S = 3
    sites = sum(int(np.prod(w.shape)) for w in insts)

    def timed_steps(lat, warm):
        lat.step(warm)
        lat.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        stream = torch.cuda.ExternalStream(lat.stream)
        lat.set_timing(True)
        t0.record(stream)
        lat.step(steps)
        t1.record(stream)
        lat.synchronize()
        iters = lat.get_timing()["poisson_iters"]
        lat.set_timing(False)
        return t0.elapsed_time(t1), iters

    arms = {}
    tune = None
    for storage in ("fp16", "fp32"):
        lat, _ = lbm.stack_slits(insts, storage=storage, step_graph=True, device=local,
                                 extrapolate=extrapolate)
        t = lat.autotune()
        if storage == "fp16":
            tune = t
        tb, iters = timed_steps(lat, 3)
        arms["stacked_" + storage] = {
            "value": S * sites * steps / (tb / 1e3) / 1e6, "ms_per_step": tb / steps,
            "poisson_iters_per_step": iters / steps,
            "poisson_residual_last": lat.diagnostics()["poisson_residual"],
            "collide_threads": t["collide_threads"]}
        lat.destroy()
    total, iters_tot = 0.0, 0
    for w in insts:
        one = lbm.Lattice(w.shape[2], w.shape[1], w.shape[0], 3, omega_visc=w.omega_visc,
                          omega_drag=lbm.omega_drag_for_schmidt(w.omega_visc, w.schmidt),
                          bjerrum=w.bjerrum, e_ext=w.e_ext, storage="fp32", poisson="fft",
                          step_graph=True, device=local, extrapolate=extrapolate)
        one.set_walls(w.solid, w.sigma)
        for s in range(3):
            one.set_species(s, 1.0, w.valence[s], np.where(w.solid, 1.0, w.n0[s]))
        t, it = timed_steps(one, 3)
        total += t
        iters_tot += it
        one.destroy()
    arms["sequential_fp32"] = {"value": S * sites * steps / (total / 1e3) / 1e6,
                               "ms_per_step": total / steps,
                               "poisson_iters_per_step": iters_tot / (steps * len(insts))}
    head = arms["stacked_fp16"]
    return {"workload": "64 slit channels 32x32xW, W~U{16..128} (seed 1237), %d nodes" % sites,
            "storage": "fp16", "step_graph": True, "autotune": tune,
            "autotune_space": "CTA size of the stream/collide and charge kernels: 64, 128, 256",
            "value": head["value"], "unit": UNIT, "ms_per_step": head["ms_per_step"],
            "poisson_iters_per_step": head["poisson_iters_per_step"],
            "extrapolated_start": extrapolate, "arms": arms,
            "speedup_stacked_vs_sequential_fp32": total / (arms["stacked_fp32"]["ms_per_step"] * steps),
            "speedup_fp16_vs_fp32_stacked": arms["stacked_fp32"]["ms_per_step"] / head["ms_per_step"]}


def run_learned(lbm, WL, n=64, steps=20, warm=20, local=0, train=None):
    """Learned Poisson initial guess on the charged ternary porous box
    (spheres of radius 4..12 up to 20% solid, surface charge +/-0.01),
    multigrid to 1e-8 every step.  The network (two 3x3x3 layers) is trained
    on the GPU on the residuals the solver's own starts leave (16 steps of a
    training run), then three arms step the same trajectory from the same
    initial state: each solve from the previous potential (plain), from the
    history start (history), and from the history start corrected by the
    network (learned).  Returns V-cycles and Poisson time per step and the
    start residuals of each arm, and the trained parameters."""
    import torch
    wl = WL.porous_spheres(n=n, seed=1238)
    od = lbm.omega_drag_for_schmidt(1.0, 1.0)

    def make(extrapolate=True):
        lat = lbm.Lattice(n, n, n, 3, omega_drag=od, bjerrum=0.7, poisson="mg", poisson_maxit=200,
                          device=local, extrapolate=extrapolate)
        lat.set_walls(wl.solid, wl.sigma)
        for s in range(3):
            lat.set_species(s, 1.0, wl.valence[s], np.where(wl.solid, 1.0, wl.n0[s]))
        return lat

    out = {"workload": "porous_%d^3 ternary, solid %.3f, multigrid, Sc 1" % (n, wl.meta["solid_fraction"]),
           "steps": steps, "warmup": warm}
    if train is None:
        base = make()
        base.step(4)
        base.nn_init(hidden=8, seed=3)
        base.nn_collect(16)
        base.step(16)
        t = time.perf_counter()
        losses = base.nn_train(epochs=40, lr=5e-3)
        train_s = time.perf_counter() - t
        params = base.nn_params()
        base.destroy()
        out["training"] = {"fields": 16, "epochs": 40, "loss_first": float(losses[0]),
                           "loss_last": float(losses[-1]), "seconds": train_s,
                           "params": int(params.size), "lattice": "%d^3" % n}
    else:
        params = train
    for arm in ("plain", "history", "learned"):
        lat = make(extrapolate=arm != "plain")
        if arm == "learned":
            lat.nn_init(hidden=8, seed=3)
            lat.nn_params(params)
            lat.nn_use(True)
        lat.step(warm)
        lat.synchronize()
        stream = torch.cuda.ExternalStream(lat.stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        lat.set_timing(True)
        e0.record(stream)
        lat.step(steps)
        e1.record(stream)
        lat.synchronize()
        t_ms = e0.elapsed_time(e1)
        tm = lat.get_timing()
        ps = lat.poisson_stats()
        st = lat.nn_stats() if arm == "learned" else None
        out[arm] = {"vcycles_per_step": tm["poisson_iters"] / steps,
                    "poisson_ms_per_step": tm["poisson_ms"] / steps,
                    "ms_per_step": t_ms / steps,
                    "value": 3 * wl.sites * steps / (t_ms / 1e3) / 1e6,
                    "start_residual_geomean": ps["start_residual_geomean"],
                    "residual_ratio_after_guess": st["mean_ratio"] if st else None,
                    "guesses_kept": ("%d/%d" % (st["kept"], st["tried"])) if st else None,
                    "final_residual": lat.diagnostics()["poisson_residual"]}
        lat.destroy()
    out["params"] = params
    return out


def run_porous(lbm, WL, steps=20, warm=5, local=0, n=256, params=None):
    """The charged ternary porous box at full size (256^3, seeded spheres of
    radius 4..12 up to 20% solid, surface charge +/-0.01 per surface node),
    Sc = 1, the multigrid Poisson solve every step to 1e-8: whole-step rate,
    V-cycles per step and the phase times, for each solve's start from the
    previous potential (plain), from the history start (history) and, given
    trained parameters, from the history start corrected by the network."""
    import torch
    t0 = time.perf_counter()
    wl = WL.porous_spheres(n=n, seed=1238)
    gen_s = time.perf_counter() - t0
    od = lbm.omega_drag_for_schmidt(1.0, 1.0)
    nfluid = int((~wl.solid).sum())
    out = {"workload": "porous_%d^3 ternary, solid %.3f, multigrid, Sc 1" % (n, wl.meta["solid_fraction"]),
           "steps": steps, "warmup": warm, "input_seconds": gen_s}
    arms = ("plain", "history") + (("learned",) if params is not None else ())
    for arm in arms:
        t0 = time.perf_counter()
        lat = lbm.Lattice(n, n, n, 3, omega_drag=od, bjerrum=wl.bjerrum, poisson="mg",
                          poisson_tol=1e-8, poisson_maxit=200, device=local,
                          extrapolate=arm != "plain")
        lat.set_walls(wl.solid, wl.sigma)
        for s in range(3):
            lat.set_species(s, 1.0, wl.valence[s], np.where(wl.solid, 1.0, wl.n0[s]))
        if arm == "learned":
            # the network trained on the 64^3 box (a convolution: it applies
            # at any size)
            lat.nn_init(hidden=8, seed=3)
            lat.nn_params(params)
            lat.nn_use(True)
        setup_s = time.perf_counter() - t0
        lat.step(warm)
        lat.synchronize()
        stream = torch.cuda.ExternalStream(lat.stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        lat.set_timing(True)
        e0.record(stream)
        lat.step(steps)
        e1.record(stream)
        lat.synchronize()
        t_ms = e0.elapsed_time(e1)
        tm = lat.get_timing()
        ps = lat.poisson_stats()
        lat.set_timing(False)
        d = lat.diagnostics()
        out[arm] = {"value": 3 * wl.sites * steps / (t_ms / 1e3) / 1e6, "unit": UNIT,
                    "start_residual_geomean": ps["start_residual_geomean"],
                    "ms_per_step": t_ms / steps,
                    "vcycles_per_step": tm["poisson_iters"] / steps,
                    "poisson_ms_per_step": tm["poisson_ms"] / steps,
                    "charge_ms_per_step": tm["charge_ms"] / steps,
                    "collide_ms_per_step": tm["collide_ms"] / steps,
                    # stream/collide roofline: 152 B per fluid species-node
                    "collide_frac_of_measured_hbm": 152.0 * 3 * nfluid / (tm["collide_ms"] / steps * 1e-3)
                    / 1e9 / measured_peaks()[0],
                    "poisson_residual_last": d["poisson_residual"], "setup_seconds": setup_s}
        lat.destroy()
    return out


# Fine-box bytes of one V(2,2) cycle per fine cell, in units of N (cells):
# pre-smoothing 4 half-sweeps of 6.5 (other colour 2 + own residual 2 + own
# mask 0.5 + own correction 2; the first one writes zeros to the other colour
# instead of reading it), restriction 9.5 (e 4, r 4, mask 1, coarse 0.5),
# prolongation 10 (e read and write 8, mask 1, coarse 1), post-smoothing 26
# plus the potential update of the last half-sweep 16.5 (psi in 8, psi out 8,
# mask 0.5), residual 25 (psi 8, source 8, component label 4, mask 1,
# residual 4).
MG_BYTES_PER_CELL = 26 + 9.5 + 10 + 26 + 16.5 + 25


def run_multigrid(lbm, WL, n=256, steps=20, warm=5, local=0):
    """Standalone measure of the multigrid V-cycle on the porous box (n^3,
    seeded spheres, charged walls) with one weakly charged species (the
    solvent of the porous workload with valence 0.01, so that the lattice
    itself stays small and the run stable): each step solves from the
    previous potential to 1e-8.  Reports the solve time per V-cycle and the
    fine-box bytes of a cycle over that time (every coarse level's time
    included)."""
    import torch
    wl = WL.porous_spheres(n=n, seed=1238)
    lat = lbm.Lattice(n, n, n, 1, bjerrum=wl.bjerrum, poisson="mg", poisson_tol=1e-8,
                      poisson_maxit=200, device=local, extrapolate=False)
    lat.set_walls(wl.solid, wl.sigma)
    lat.set_species(0, 1.0, 0.01, np.where(wl.solid, 1.0, wl.n0[0]))
    lat.step(warm)
    lat.synchronize()
    lat.set_timing(True)
    stream = torch.cuda.ExternalStream(lat.stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat.step(steps)
    e1.record(stream)
    lat.synchronize()
    tm = lat.get_timing()
    lat.set_timing(False)
    d = lat.diagnostics()
    lat.destroy()
    cycles = tm["poisson_iters"]
    ms_cycle = tm["poisson_ms"] / max(1, cycles)
    nb = wl.sites  # fine cells (the box is periodic in z: no planes trimmed)
    gbs = MG_BYTES_PER_CELL * nb / (ms_cycle * 1e-3) / 1e9
    peak, src = measured_peaks()
    return {"workload": "porous_%d^3, one species of valence 0.01, charged walls, multigrid from "
                        "the previous potential to 1e-8" % n,
            "steps": steps, "warmup": warm, "vcycles_per_step": cycles / steps,
            "poisson_ms_per_step": tm["poisson_ms"] / steps, "ms_per_vcycle": ms_cycle,
            "step_ms": e0.elapsed_time(e1) / steps,
            "fine_bytes_per_vcycle": MG_BYTES_PER_CELL * nb,
            "fine_bytes_per_cell": MG_BYTES_PER_CELL,
            "achieved_gbs": gbs, "peak_gbs": peak, "peak_source": src, "frac": gbs / peak,
            "poisson_residual_last": d["poisson_residual"]}


def run_conductivity(lbm, WL, n=64, local=0):
    """Bulk conductivity (Sec. 4, current against D; Eq. Drude): a uniform
    neutral ternary electrolyte (ion fractions 0.01) in a field 1e-3 along
    x, n^3 periodic, graph steps, spectral Poisson, FP32, at Sc 1 ... 1000.
    Each run lasts until the species velocities have relaxed (they relax by
    |1 - omega_drag| per step); the measured current J = sum z n u over the
    box is compared with the Drude-Lorentz value (D / c_s^2) sum z^2 n E,
    D = c_s^2 (1/omega_drag - 1/2)."""
    import torch
    cs2, e, fraction = 1.0 / 3.0, 1e-3, 0.01
    out = []
    for sc in (1.0, 3.0, 10.0, 30.0, 100.0, 300.0, 1000.0):
        wl = WL.bulk_conductivity(n=n, e_field=e, schmidt=sc, fraction=fraction)
        od = lbm.omega_drag_for_schmidt(wl.omega_visc, sc)
        q = abs(1.0 - od)
        steps = 200 if q < 1e-3 else 200 + int(math.log(1e-9) / math.log(q))
        lat = lbm.Lattice(n, n, n, 3, omega_visc=wl.omega_visc, omega_drag=od, bjerrum=wl.bjerrum,
                          e_ext=wl.e_ext, poisson="fft", step_graph=True, device=local)
        for s in range(3):
            lat.set_species(s, 1.0, wl.valence[s], wl.n0[s])
        lat.step(3)
        lat.synchronize()
        st = torch.cuda.ExternalStream(lat.stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        lat.step(steps)
        e1.record(st)
        lat.synchronize()
        ms = e0.elapsed_time(e1)
        J = 0.0
        for s in range(3):
            ns, us = lat.get_moments(s)
            J += float(wl.valence[s] * (ns * us[0]).mean())
        D = cs2 * (1.0 / od - 0.5)
        jd = D / cs2 * 2 * fraction * e
        out.append({"sc": sc, "omega_drag": od, "D": D, "steps": steps, "current": J,
                    "drude": jd, "current_over_drude": J / jd,
                    "value": 3 * wl.sites * steps / (ms / 1e3) / 1e6,
                    "poisson_residual_last": lat.diagnostics()["poisson_residual"]})
        lat.destroy()
    return {"workload": "bulk conductivity %d^3, ion fractions 0.01, E 1e-3 along x" % n,
            "runs": out}


def slit_theory(e, sigma, debye, width, nu):
    """Helmholtz-Smoluchowski mass flow and Debye-Hueckel convective current
    of a slit of `width` fluid planes (h = width / 2), wall charge `sigma`
    per wall node, k = 1 / debye (unit density, derived from the model:
    u_x = E (psi - psi_w) / (4 pi l_B nu), psi = psi_w cosh(k z) / cosh(k h),
    psi_w = 4 pi l_B sigma / (k tanh(k h)))."""
    k, h = 1.0 / debye, 0.5 * width
    kh = k * h
    im = (e * sigma / nu) * (2.0 / k ** 2) * (1.0 - kh / math.tanh(kh))
    ieo = -(e * sigma ** 2 / (nu * k * math.tanh(kh) ** 2)) * (
        (kh + 0.5 * math.sinh(2 * kh)) / math.cosh(kh) ** 2 - 2.0 * math.tanh(kh))
    return im, ieo


def run_slit_transport(lbm, WL, local=0, relax=20000):
    """Slit transport sweep (Sec. 4, Figs. of I_m, I, I_eo against
    lambda_D / L_z and omega_drag): 32 x 8 x (50 + 2 walls), wall charge
    -1e-4 per wall node (the paper's Sigma Lx Ly = -0.04 on a 40 x 10 wall),
    field 1e-4 along x, lambda_D / L_z = 0.4, 0.2, 0.1, Sc = 1, 10, 100, 1000.
    The double layer is formed at Sc = 1 (ion diffusion over lambda_D^2 / D
    is 10^3 times slower at Sc = 1000); each Sc then sets the drag frequency
    of every plane and runs `relax` steps (flow: L^2 / (pi^2 nu) ~ 1500 steps
    per e-fold; drift: |1 - omega_drag| per step) before the currents are
    read.  The steady state does not depend on the path."""
    import torch
    from paper_1507_04891_gb300 import transport
    W, sigma, e = 50, -1e-4, 1e-4
    nu = (1.0 / 3.0) * (1.0 / 1.0 - 0.5)
    out = []
    for ratio in (0.4, 0.2, 0.1):
        debye = ratio * W
        wl = WL.slit(nx=32, ny=8, width=W, sigma=sigma, debye=debye, e_field=e, schmidt=1.0)
        lat = lbm.Lattice(32, 8, W + 2, 3, omega_drag=lbm.omega_drag_for_schmidt(1.0, 1.0),
                          bjerrum=wl.bjerrum, e_ext=wl.e_ext, poisson="fft", step_graph=True,
                          device=local)
        lat.set_walls(wl.solid, wl.sigma)
        for s in range(3):
            lat.set_species(s, 1.0, wl.valence[s], np.where(wl.solid, 1.0, wl.n0[s]))
        im_th, ieo_th = slit_theory(e, sigma, debye, W, nu)
        for sc in (1.0, 10.0, 100.0, 1000.0):
            od = lbm.omega_drag_for_schmidt(1.0, sc)
            lat.set_plane_omega_drag(np.full(W + 2, od))
            st = torch.cuda.ExternalStream(lat.stream)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            lat.step(relax)
            e1.record(st)
            lat.synchronize()
            ms = e0.elapsed_time(e1)
            c = transport.slit_currents(lat, wl.valence, wl.solid)
            c.update({"lambda_D_over_Lz": ratio, "sc": sc, "omega_drag": od,
                      "I_m_theory_HS": im_th, "I_m_over_theory": c["I_m"] / im_th,
                      "I_eo_theory_DH": ieo_th, "I_eo_over_theory": c["I_eo"] / ieo_th,
                      "value": 3 * wl.sites * relax / (ms / 1e3) / 1e6,
                      "poisson_residual_last": lat.diagnostics()["poisson_residual"]})
            out.append(c)
        lat.destroy()
    return {"workload": "slit 32x8x(50+2), sigma -1e-4 per wall node, E 1e-4, %d steps per Sc "
                        "after the Sc = 1 run" % relax, "runs": out}


def run_slit(lbm, WL, steps=2000, local=0):
    """Charged slit 64x64x(64 + 2 walls), wall charge -0.01 per node, Debye
    length 8, field 1e-4 along x: FP32, FP16 and BF16 storage at Sc 1 ... 1000
    (graph steps, spectral Poisson): throughput, the 16-bit fields against
    FP32, and the electro-osmotic mass flow rate I_m = sum_z rho u_x."""
    import torch
    out = []
    for sc in (1.0, 10.0, 100.0, 1000.0):
        wl = WL.slit(nx=64, ny=64, width=64, sigma=-0.01, debye=8.0, e_field=1e-4, schmidt=sc)
        od = lbm.omega_drag_for_schmidt(1.0, sc)
        fields = {}
        row = {"sc": sc, "omega_drag": od}
        for storage in ("fp32", "fp16", "bf16"):
            lat = lbm.Lattice(64, 64, 66, 3, omega_drag=od, bjerrum=wl.bjerrum, e_ext=wl.e_ext,
                              storage=storage, poisson="fft", step_graph=True, device=local)
            lat.set_walls(wl.solid, wl.sigma)
            for s in range(3):
                lat.set_species(s, 1.0, wl.valence[s], np.where(wl.solid, 1.0, wl.n0[s]))
            lat.step(3)
            lat.synchronize()
            st = torch.cuda.ExternalStream(lat.stream)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            lat.step(steps)
            e1.record(st)
            lat.synchronize()
            ms = e0.elapsed_time(e1)
            mom = [lat.get_moments(s) for s in range(3)]
            n = np.stack([m[0] for m in mom])
            j = np.stack([m[0][None] * m[1] for m in mom])
            fields[storage] = (n, j)
            jx = j[:, 0].sum(0)  # mixture momentum density along x
            im = float(jx[1:-1].mean(axis=(1, 2)).sum())
            row[storage] = {"value": 3 * wl.sites * steps / (ms / 1e3) / 1e6,
                            "ms_per_step": ms / steps, "mass_flow_rate": im,
                            "poisson_residual_last": lat.diagnostics()["poisson_residual"]}
            lat.destroy()
        fl = ~wl.solid
        n32, j32 = fields["fp32"]
        for storage in ("fp16", "bf16"):
            n16, j16 = fields[storage]
            row[storage]["max_rel_density_error_vs_fp32"] = float(
                (np.abs(n16 - n32)[:, fl] / n32[:, fl]).max())
            row[storage]["max_momentum_error_vs_fp32"] = float(
                (np.abs(j16 - j32)[:, :, fl] / (n32[:, None, fl] / math.sqrt(3.0))).max())
        out.append(row)
    return {"workload": "slit 64x64x66, sigma -0.01, Debye 8, E 1e-4, %d steps" % steps,
            "runs": out}


def run_ours(args, rank, world, local):
    import torch

    from paper_1507_04891_gb300 import lbm
    from paper_1507_04891_gb300 import workloads as WL
    from paper_1507_04891_gb300.build import build_library

    from paper_1507_04891_gb300 import replicas

    build_library()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    replicas.init(world, backend="nccl", device=dev)
    n = args.n
    wl = WL.ternary_bulk(n=n, seed=1235 + rank, schmidt=args.schmidt)
    S, N = wl.nspecies, wl.sites
    od = lbm.omega_drag_for_schmidt(wl.omega_visc, args.schmidt)
    warm = max(3, args.warmup)
    K = args.steps

    def make(poisson, graph=False, omega_drag=None, storage=None, charge_pass=False):
        return lbm.Lattice(n, n, n, S, omega_visc=wl.omega_visc,
                           omega_drag=od if omega_drag is None else omega_drag, bjerrum=wl.bjerrum,
                           storage=storage or args.storage, poisson=poisson, poisson_tol=1e-8,
                           poisson_maxit=500, device=local, step_graph=graph,
                           extrapolate=not args.no_extrapolation,
                           charge_pass=charge_pass or args.charge_pass)

    def barrier():
        replicas.barrier(world)
        torch.cuda.synchronize()

    def max_over_ranks(x):
        return replicas.max_over_ranks(x, world, device="cuda")

    def timed(poisson, sample_clocks, graph=False, omega_drag=None, storage=None, keep=False,
              charge_pass=False):
        """W warm-up steps, then K steps timed with CUDA events on the
        library's stream; phase times from the library's own events."""
        lat = make(poisson, graph, omega_drag, storage, charge_pass)
        for s in range(S):
            lat.set_species(s, 1.0, wl.valence[s], wl.n0[s])
        stream = torch.cuda.ExternalStream(lat.stream, device=dev)
        lat.step(warm)
        lat.synchronize()
        clocks = clock_sampler(local) if sample_clocks else None
        barrier()
        lat.set_timing(True)
        if clocks:
            clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        if clocks:
            clocks.begin()
        e0.record(stream)
        lat.step(K)
        e1.record(stream)
        lat.synchronize()
        if clocks:
            clocks.end()
        barrier()
        clk = clocks.stop() if clocks else None
        t_ms = max_over_ranks(e0.elapsed_time(e1))
        tm = lat.get_timing()
        lat.set_timing(False)
        diag = lat.diagnostics()
        if keep:
            return t_ms, tm, diag, clk, lat
        lat.destroy()
        return t_ms, tm, diag, clk

    def rate(t_ms):
        return world * S * N * K / (t_ms / 1e3) / 1e6

    # headline: every step one CUDA-graph replay (spectral solver); the
    # host-stepped run beside it gives the per-phase CUDA-event times
    graph_head = args.poisson == "fft" and not args.host_steps
    t_ms, tm_head, diag, clk, lat_head = timed(args.poisson, True, graph=graph_head, keep=True)
    value = rate(t_ms)
    if graph_head:
        t_host, tm, _, _ = timed(args.poisson, False, graph=False)
        host_run = {"value": rate(t_host), "ms_per_step": t_host / K,
                    "poisson_iters_per_step": tm["poisson_iters"] / K}
    else:
        tm, host_run = tm_head, None
    collide_ms = tm["collide_ms"] / max(1, tm["collide_launches"])
    bpl = BYTES_PER_SPECIES_SITE[args.storage] * S * N
    # with the charge scatter (FP32, x rows of whole warps, no walls) the
    # stream/collide also adds the next step's 8-byte source per node
    scatter = args.storage == "fp32" and n % 32 == 0 and not args.charge_pass
    bpl_head = bpl + (8 * N if scatter else 0)
    peak, peak_kind = measured_peaks()
    achieved = bpl_head / (collide_ms / 1e3) / 1e9
    traffic = kernel_traffic(args.storage, "" if scatter else "_charge_pass") if n == 128 else None

    # the same workload with 16-bit shifted storage (FP32 arithmetic), graph
    # steps for the rate and host steps for the kernel time; the fields after
    # the same steps against the FP32 headline run
    storage_lines = {}
    if args.storage == "fp32" and not args.no_alt:
        ref = [lat_head.get_moments(s) for s in range(S)]
        for st in ("fp16", "bf16"):
            ts, tms, _, _, lat16 = timed(args.poisson, False, graph=graph_head, storage=st, keep=True)
            en = ej = 0.0
            for s in range(S):
                n16, u16 = lat16.get_moments(s)
                n32, u32 = ref[s]
                en = max(en, float((np.abs(n16 - n32) / n32).max()))
                ej = max(ej, float((np.abs(n16 * u16 - n32 * u32) / (n32 / math.sqrt(3.0))).max()))
            lat16.destroy()
            th, tmh, _, _ = timed(args.poisson, False, graph=False, storage=st)
            cms = tmh["collide_ms"] / max(1, tmh["collide_launches"])
            b16 = BYTES_PER_SPECIES_SITE[st] * S * N
            storage_lines[st] = {
                "value": rate(ts), "ms_per_step": ts / K,
                "poisson_iters_per_step": tms["poisson_iters"] / K,
                "speedup_vs_fp32": t_ms / ts,
                "max_rel_density_diff_vs_fp32": en, "max_momentum_diff_vs_fp32_over_n_cs": ej,
                "accuracy": "fields after %d steps against the FP32 run (the GPU tests hold "
                            "16-bit storage within 1e-3 of the FP64 oracle per node)" % (warm + K),
                "roofline": {"kernel": "k_stream_collide", "bound": "hbm",
                             "achieved": b16 / (cms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                             "frac": b16 / (cms / 1e3) / 1e9 / peak, "peak_source": peak_kind,
                             "algorithmic_bytes_per_launch": b16, "collide_ms": cms,
                             "traffic": kernel_traffic(st) if n == 128 else None}}
    lat_head.destroy()

    # the same workload with the charge density from a separate pass over
    # the charged populations (LBM_FLAG_CHARGE_PASS) instead of the
    # previous stream/collide's scatter: whole steps, and the stream/collide
    # without the scatter against its roofline
    charge_pass = None
    if scatter and not args.no_alt:
        tc, tmc, _, _ = timed(args.poisson, False, graph=graph_head, charge_pass=True)
        th, tmh, _, _ = timed(args.poisson, False, graph=False, charge_pass=True)
        cms = tmh["collide_ms"] / max(1, tmh["collide_launches"])
        charge_pass = {
            "value": rate(tc), "ms_per_step": tc / K, "poisson_iters_per_step": tmc["poisson_iters"] / K,
            "phase_ms_per_step": {"charge": tmh["charge_ms"] / K, "poisson": tmh["poisson_ms"] / K,
                                  "stream_collide": tmh["collide_ms"] / K},
            "roofline": {"kernel": "k_stream_collide (no scatter)", "bound": "hbm",
                         "achieved": bpl / (cms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": bpl / (cms / 1e3) / 1e9 / peak, "peak_source": peak_kind,
                         "algorithmic_bytes_per_launch": bpl, "collide_ms": cms,
                         "traffic": kernel_traffic("fp32", "_charge_pass") if n == 128 else None}}

    # the same workload with the multigrid solver, for comparison
    alt = None
    if args.poisson != "mg" and not args.no_alt:
        ta, tma, _, _ = timed("mg", False)
        alt = {"poisson": "mg", "value": rate(ta), "ms_per_step": ta / K,
               "poisson_iters_per_step": tma["poisson_iters"] / K,
               "poisson_ms_per_step": tma["poisson_ms"] / K}

    # the benchmark's second Schmidt number, Sc = 100, same configuration
    sc100 = None
    if args.schmidt == 1.0 and not args.no_alt:
        od100 = lbm.omega_drag_for_schmidt(wl.omega_visc, 100.0)
        t100, tm100, _, _ = timed(args.poisson, False, graph=graph_head, omega_drag=od100)
        sc100 = {"sc": 100.0, "omega_drag": od100, "value": rate(t100), "ms_per_step": t100 / K,
                 "poisson_iters_per_step": tm100["poisson_iters"] / K}

    batched = learned = porous = None
    if rank == 0 and world == 1 and not args.no_extras:
        batched = run_batched(lbm, WL, local=local, extrapolate=not args.no_extrapolation)
        learned = run_learned(lbm, WL, local=local)
        porous = run_porous(lbm, WL, steps=K, warm=warm, local=local, params=learned.pop("params"))

    # end to end through the C ABI: the initial densities copied from pinned
    # host memory to device buffers and handed over with lbm_set_species_dev
    # (a fresh start: potential from zero, empty solve history), every
    # step's FP64 diagnostics read back (the step's metric; lbm_step_record
    # queues each step's copy behind it), and at the end the moments of every
    # species (lbm_get_moments_dev) copied to pinned host memory -- all inside
    # the timed region.  The lattice object was created and stepped through
    # the same warm-up before (the step graphs exist, as in the device-timed
    # run).
    lat2 = make(args.poisson, graph_head)
    for s in range(S):
        lat2.set_species(s, 1.0, wl.valence[s], wl.n0[s])
    lat2.step(warm)
    lat2.synchronize()
    pin_in = [torch.from_numpy(np.ascontiguousarray(wl.n0[s])).pin_memory() for s in range(S)]
    dev_in = [torch.empty(N, dtype=torch.float64, device=dev) for _ in range(S)]
    pin_n = [torch.empty(N, dtype=torch.float64).pin_memory() for _ in range(S)]
    pin_u = [torch.empty(3 * N, dtype=torch.float64).pin_memory() for _ in range(S)]
    # a stream of our own: the copies, the library's work queued on it and the
    # read-back are ordered on it (the library's own stream does not wait for
    # the legacy default stream)
    cur = torch.cuda.Stream(dev)
    barrier()
    t0 = time.perf_counter()
    with torch.cuda.stream(cur):
        for s in range(S):
            dev_in[s].copy_(pin_in[s].view(-1), non_blocking=True)
            lat2.set_species_dev(s, 1.0, wl.valence[s], dev_in[s].data_ptr(), stream=cur.cuda_stream)
        e2e_rows = lat2.step_record(K, stream=cur.cuda_stream)
        for s in range(S):
            # the gather writes the pinned host buffers directly
            lat2.get_moments_dev(s, pin_n[s].data_ptr(), pin_u[s].data_ptr(), stream=cur.cuda_stream)
    torch.cuda.synchronize(dev)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e_value = world * S * N * K / e2e_s / 1e6
    e2e_mass = float(pin_n[1].sum())
    lat2.destroy()

    iters = tm_head["poisson_iters"]
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cpu = cpu_baseline(schmidt=args.schmidt)
        except Exception as ex:  # the baseline is reported, never required
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": "failed: %s" % ex}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": warm, "ms_per_step": t_ms / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "fp16": "f16 storage, f32 arithmetic",
                      "bf16": "bf16 storage, f32 arithmetic"}[args.storage],
            "data": "synthetic",
            "config": {"workload": "ternary_bulk_%d^3" % n, "species": S, "sc": args.schmidt,
                       "omega_visc": wl.omega_visc, "omega_drag": od, "bjerrum": wl.bjerrum,
                       "poisson": args.poisson, "poisson_tol": 1e-8, "storage": args.storage,
                       "poisson_start": ("previous psi" if args.no_extrapolation
                                         else "history projection (5 source differences)"),
                       "charge_density": ("scattered by the previous stream/collide" if scatter
                                          else "separate pass over the charged populations"),
                       "l2": "not flushed: inputs larger than L2 (2 x %.0f MB population lattices)"
                             % (BYTES_PER_SPECIES_SITE[args.storage] / 2 * S * N / 1e6),
                       "steps": "cuda_graph" if graph_head else "host",
                       "parallelism": "replicas" if world > 1 else "single"},
            "poisson_iters_per_step": iters / K,
            "phase_ms_per_step": {"charge": tm["charge_ms"] / K,
                                  "poisson": tm["poisson_ms"] / K,
                                  "stream_collide": tm["collide_ms"] / K},
            "roofline": {"kernel": "k_stream_collide" + (" (with the charge scatter)" if scatter else ""),
                         "bound": "hbm", "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_source": peak_kind,
                         "algorithmic_bytes_per_launch": bpl_head, "collide_ms": collide_ms,
                         "traffic": traffic},
            "clocks": clk,
            "gpu_launches": tm_head["kernel_launches"],
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": 8 * S * N / K,
                    "d2h_bytes_per_step": 8 * (9 + 2) + 8 * 4 * S * N / K,
                    "api": "lbm_set_species_dev from pinned host memory (fresh start), "
                           "lbm_step_record (every step's FP64 diagnostics written to pinned host "
                           "memory behind it), lbm_get_moments_dev of every species straight "
                           "into pinned host memory at the end",
                    "steps_recorded": int(e2e_rows.shape[0]),
                    "final_cation_mass": e2e_mass},
            "storage_variants": storage_lines or None,
            "charge_pass": charge_pass,
            "poisson_alternative": alt,
            "sc100": sc100,
            "host_steps": host_run,
            "batched": batched,
            "learned_vs_plain": learned,
            "porous_256": porous,
            "diagnostics": {"mass": list(map(float, diag["mass"])),
                            "poisson_residual_last": diag["poisson_residual"]},
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    replicas.finish(world)
    return 0


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.only:
        from paper_1507_04891_gb300 import lbm
        from paper_1507_04891_gb300 import workloads as WL
        from paper_1507_04891_gb300.build import build_library
        build_library()
        if args.only == "batched":
            res = run_batched(lbm, WL, steps=max(1, args.steps), extrapolate=not args.no_extrapolation)
        elif args.only == "slit":
            res = run_slit(lbm, WL, steps=max(1, args.steps))
        elif args.only == "slit_transport":
            res = run_slit_transport(lbm, WL)
        elif args.only == "conductivity":
            res = run_conductivity(lbm, WL, n=args.n if args.n != 128 else 64)
        elif args.only == "porous":
            res = run_porous(lbm, WL, steps=max(1, args.steps), warm=max(1, args.warmup), n=args.n)
        elif args.only == "multigrid":
            res = run_multigrid(lbm, WL, n=args.n,
                                steps=min(max(1, args.steps), 50), warm=max(1, args.warmup))
        else:
            res = run_learned(lbm, WL)
            res["porous_256"] = run_porous(lbm, WL, params=res.pop("params"))
        print(json.dumps({"metric": METRIC, "only": args.only, **res}), flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
