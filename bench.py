#!/usr/bin/env python3
"""Benchmark: FIRE site-updates/s of the fused force + FIRE step on the 512^3
lattice (four homeotropic colloids, planar-degenerate walls, three-constant
elasticity), in the FP32-bulk / FP64-reduction form (``value``) and the FP64
form, with the HBM roofline of the step kernel.

  python bench.py [--gpus N --steps K --warmup W] [--impl ours|reference]

One JSON line on stdout (rank 0).  Under torchrun (N > 1) every rank runs an
independent replica of the lattice on its own GPU (the path is single-GPU;
replicas only) and the value is the sum over ranks divided by the slowest
rank's time.  ``--impl reference`` times the CPU oracle on a bounded sample
of the same workload instead.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1911_07045_b300 import synth  # noqa: E402

METRIC = "FIRE site-updates/s at 512^3 (FP32 vs FP64), % HBM peak; served p50/p99 latency"
UNIT = "site-updates/s"
# algorithmic bytes per site-update: the FIRE state that must persist, q and
# v (5 components each), read and written, plus the 1-byte site mask
ALG_BYTES = {"fp32": 4 * 5 * 4 + 1, "fp64": 4 * 5 * 8 + 1}
# bytes the stored-force design moves: q, v, F read and written + mask
DESIGN_BYTES = {"fp32": 6 * 5 * 4 + 1, "fp64": 6 * 5 * 8 + 1}
# DRAM bytes per site-update of the step kernel, dram__bytes_read.sum +
# dram__bytes_write.sum from one ncu capture of the same kernel on the 256^3
# case of this workload, divided by its 16,777,216 sites (the traffic of a
# launch grows with the sites it updates); the bench scales it to its lattice.
# The FP64 one-constant form moves the same state bytes as the three-constant
# one and takes its figure.
DRAM_BYTES_PER_SITE = {"fp32": (1.073290e9 + 0.960306176e9) / 256 ** 3,
                       "fp64": (2.260472e9 + 1.955142e9) / 256 ** 3,
                       "fp32_1c": (1.059682e9 + 0.95704064e9) / 256 ** 3}
# DRAM bytes per site-update of the batched leg's launch (64 lattices, 32x4
# tiles, z chunk 128; ncu, mean of three launches): re-reads around the
# colloids lift it above the single-lattice figure
DRAM_BYTES_PER_SITE_BATCH = (4.677079040e9 + 2.734580736e9) / 46252032
# FP64 form: bound by the FP64 pipe (2 FP64 operations per clock per SM).
# FP64 arithmetic operations per site-update of the regular three-constant
# site, counted from the kernel's arithmetic: stencil 94 (second
# differences 15 x 2, the site's central differences D_y, D_z 10, mixed
# differences from them 13, shared partial sums 12, one- and three-constant
# combinations 29, which start from the bulk force: no separate sum), bulk
# force 33, drift 10, mixing and kick 15, reductions 18 (ring sites' drift
# and central differences are not counted)
FP64_OPS_PER_SITE = 170
# the same for a one-constant site: the stencil is 15 second differences (add
# + FMA), 10 adds for the three-axis sums and 8 scalings (48 instead of 94)
FP64_OPS_PER_SITE_1C = 124
FP64_OPS_PER_CLK_SM = 2
N_SM = 148


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6400.0), "measured"
    return 6400.0, "fallback"


# ---- distributed plumbing ------------------------------------------------------

class Dist:
    def __init__(self, backend=None):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            if backend is None:
                import torch
                backend = "nccl" if torch.cuda.is_available() else "gloo"
            dist.init_process_group(backend)
            self.pg = dist
            self.backend = backend

    def barrier(self):
        if self.pg:
            if self.backend == "nccl":
                import torch
                self.pg.barrier(device_ids=[self.local])
            else:
                self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        dev = f"cuda:{self.local}" if self.backend == "nccl" else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        dev = f"cuda:{self.local}" if self.backend == "nccl" else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def aggregate(dist: Dist, units: float, seconds: float):
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    tmax = dist.max(seconds)
    total = dist.sum(units)
    return total / tmax, tmax


# ---- clocks during the timed region ---------------------------------------------

class ClockSampler:
    """SM clocks and throttle reasons of one GPU, sampled while a timed
    region runs: through the driver's NVML library (ctypes) every 2 ms where
    it loads (a 20-step region of the 512^3 workload lasts under 100 ms),
    else through ``nvidia-smi -lms 200``.  Only reads the GPU's state."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    BITS = [0x8, 0x40, 0x20, 0x4]      # nvmlClocksEventReason* of nvml.h, in NAMES order
    NVML_CLOCK_SM = 1

    def __init__(self, gpu_index: int, interval_s: float = 0.002):
        self.gpu = gpu_index
        self.interval = interval_s
        self.proc = None
        self.nvml = None
        self.lines = []
        self.samples = []          # NVML: (sm MHz, max sm MHz, reason names)
        self.stop = threading.Event()

    def _nvml_open(self):
        import ctypes as C
        lib = C.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit")
        dev = C.c_void_p()
        # the CUDA device's PCI address names the same GPU in NVML whatever
        # CUDA_VISIBLE_DEVICES hides; the index is the fallback
        rc = -1
        try:
            import torch
            pr = torch.cuda.get_device_properties(self.gpu)
            bus = f"{pr.pci_domain_id:08X}:{pr.pci_bus_id:02X}:{pr.pci_device_id:02X}.0".encode()
            rc = lib.nvmlDeviceGetHandleByPciBusId_v2(C.c_char_p(bus), C.byref(dev))
        except Exception:
            rc = -1
        if rc != 0 and lib.nvmlDeviceGetHandleByIndex_v2(C.c_uint(self.gpu), C.byref(dev)) != 0:
            lib.nvmlShutdown()
            raise RuntimeError("nvmlDeviceGetHandleByIndex")
        reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        mx = C.c_uint()
        lib.nvmlDeviceGetMaxClockInfo(dev, self.NVML_CLOCK_SM, C.byref(mx))
        clk, rs = C.c_uint(), C.c_ulonglong()

        def read():
            if lib.nvmlDeviceGetClockInfo(dev, self.NVML_CLOCK_SM, C.byref(clk)) != 0:
                return None
            if reasons_fn(dev, C.byref(rs)) != 0:
                return None
            return (float(clk.value), float(mx.value),
                    [n for n, b in zip(self.NAMES, self.BITS) if rs.value & b])
        if read() is None:
            lib.nvmlShutdown()
            raise RuntimeError("nvml clock query")
        return lib, read

    def __enter__(self):
        try:
            lib, read = self._nvml_open()

            def poll():
                while True:
                    smp = read()
                    if smp is not None:
                        self.samples.append(smp)
                    if self.stop.wait(self.interval):
                        break
            self.nvml = lib
            self.t = threading.Thread(target=poll, daemon=True)
            self.t.start()
            return self
        except Exception:
            self.nvml = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.nvml is not None:
            self.stop.set()
            self.t.join(timeout=2)
            self.nvml.nvmlShutdown()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        for f_sm, f_mx, names in self.samples:
            sm.append(f_sm)
            mx = f_mx
            reasons.update(names)
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, val in zip(self.NAMES, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm), "source": "nvml 2 ms" if self.samples else "nvidia-smi 200 ms"}


# ---- our arm ------------------------------------------------------------------------

def run_form(precision: str, L: int, steps: int, warmup: int, dist: Dist, sampler_gpu: int,
             staging: int = 0):
    """One precision form on the L^3 workload; a "_1c" suffix runs the same
    geometry with one-constant elasticity (L2 = L3 = 0), a "_chiral" suffix
    adds the chiral term L4 = 0.05 and "_cubic" also the cubic term L6 = 0.3
    (the kernel form with the chiral and cubic terms)."""
    import torch
    from paper_1911_07045_b300 import lqmin
    cfg = synth.config_large(L)
    if precision.endswith("_1c"):
        cfg = dict(cfg, L2=0.0, L3=0.0)
    stream = torch.cuda.Stream()
    prec = lqmin.LQ_FP32_BULK_FP64_RED if precision.startswith("fp32") else lqmin.LQ_FP64
    if precision.endswith("_chiral") or precision.endswith("_cubic"):
        s = lqmin.Solver(cfg["shape"], synth.A_5CB, synth.B_5CB, synth.C_5CB, cfg["L1"], cfg["L2"],
                         cfg["L3"], precision=prec, stream=stream.cuda_stream, L4=0.05,
                         L6=0.3 if precision.endswith("_cubic") else 0.0)
        s.add_objects(cfg["objects"])
    else:
        s = lqmin.solver_for(cfg, precision=prec, stream=stream.cuda_stream)
    if staging and prec == lqmin.LQ_FP32_BULK_FP64_RED and cfg.get("L2", 0.0) != 0.0 \
            and not (precision.endswith("_chiral") or precision.endswith("_cubic")):
        s.set_staging(staging)
    nsim, nrec = s.geometry_info()
    s.init_random_uniaxial(cfg["seed"])
    # fixed-step run: a tolerance of 0 never converges, so every step is done
    p = lqmin.fire_params(**dict(synth.FIRE_DEFAULTS, max_iter=10 ** 12, force_tol=0.0))
    r = s.step(p, warmup)
    assert r.fire_status == lqmin.FIRE_RUNNING, r.as_dict()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(sampler_gpu) as clk:
        e0.record(stream)
        r = s.step(p, steps)
        e1.record(stream)
        torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3
    ok = r.fire_status == lqmin.FIRE_RUNNING and r.iterations == warmup + steps
    N = L ** 3
    value, tmax = aggregate(dist, N * steps, sec)
    per_launch = sec / steps
    out = dict(value=value, ms_per_step=tmax / steps * 1e3, per_launch_s=per_launch, ok=ok,
               clocks=clk.summary(), nsim=nsim, nanchored=nrec, N=N,
               max_force=r.max_force, launches=steps)
    # end to end through the C interface with host buffers: upload q0 from
    # pinned memory, read the FIRE residual back after every step, download q
    q_host = torch.empty((5, N), dtype=torch.float64, pin_memory=True).numpy()
    s.init_random_uniaxial(cfg["seed"])
    s._ck(s.lib.lq_get_q(s.h, lqmin._ptr(q_host)))   # the start state, in pinned memory
    k_e2e = max(3, min(steps, 20))
    dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.set_q(q_host)
    for j in range(k_e2e):
        r = s.step(p, 1)        # returns the residual (max |F|) to the host
        if j == 0:
            ta = time.perf_counter()
    tb = time.perf_counter()
    s._ck(s.lib.lq_get_q(s.h, lqmin._ptr(q_host)))
    t1 = time.perf_counter()
    dist.barrier()
    e2e_val, _ = aggregate(dist, N * k_e2e, t1 - t0)
    out["e2e"] = dict(value=e2e_val, unit=UNIT, steps=k_e2e,
                      h2d_bytes_per_step=int(5 * N * 8 / k_e2e),
                      d2h_bytes_per_step=int((5 * N * 8) / k_e2e + 160),
                      # where the time goes: the upload with the first step,
                      # the other steps (each with its residual read), the download
                      upload_and_first_step_s=round(ta - t0, 4), steps_s=round(tb - ta, 4),
                      download_s=round(t1 - tb, 4))
    s.close()
    return out


def run_batch(steps: int, tile=None):
    """64 uneven lattices (edges 32..128, 0-3 colloids, one constant, FP32
    form) advanced by the persistent batch kernel; the tiling is autotuned,
    or ``tile`` = (width, height, z chunk) when given (for profiling)."""
    from paper_1911_07045_b300 import lqmin
    cfgs = synth.config_batch()
    solvers = []
    for c in cfgs:
        s = lqmin.solver_for(c, precision=lqmin.LQ_FP32_BULK_FP64_RED)
        s.init_random_uniaxial(c["seed"])
        solvers.append(s)
    sites = sum(int(np.prod(c["shape"])) for c in cfgs)
    batch = lqmin.Batch(solvers)
    p = lqmin.fire_params(**dict(synth.FIRE_DEFAULTS, max_iter=10 ** 12, force_tol=0.0))
    if tile:
        (tx, ty, zc), tuned_ms = tile, None
        batch.set_tile(tx, ty, zc)
    else:
        (tx, ty, zc), tuned_ms = batch.autotune(p, launches=12)
    batch.step(p, 3)                                  # warm-up
    t0 = time.perf_counter(); batch.step(p, steps); t1 = time.perf_counter()
    batch.step(p, 2 * steps); t2 = time.perf_counter()
    sec = (t2 - t1) - (t1 - t0)                       # host overhead of a call cancels
    peak, peak_kind = measured_peaks()
    ach = ALG_BYTES["fp32"] * sites / (sec / steps) / 1e9
    out = {"workload": f"{len(cfgs)} cubic lattices, edges {{32,48,64,96,128}}, 0-3 colloids "
                       f"R~U[6,16] (W=5.3), one constant, FP32 form",
           "sites": sites, "steps": steps, "value": sites * steps / sec, "unit": UNIT,
           "ms_per_step": sec / steps * 1e3, "tiling": {"tile": f"{tx}x{ty}", "zchunk": zc},
           "autotune_ms_per_step": tuned_ms, "autotune_launches_per_candidate": 12 if not tile else 0,
           "launches_per_step": 1,
           # algorithmic bytes (q, v read + written, mask) of every lattice
           # per launch over the time per launch (host-timed graph launches)
           "roofline": {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                        "frac": round(ach / peak, 4),
                        "traffic": round(DRAM_BYTES_PER_SITE_BATCH * sites) if sites == 46252032 else None,
                        "dram_frac": round(DRAM_BYTES_PER_SITE_BATCH * sites / (sec / steps) / 1e9 / peak, 4)
                        if sites == 46252032 else None,
                        "alg_bytes_per_site": ALG_BYTES["fp32"],
                        "peak_kind": peak_kind + " (HBM copy)"}}
    batch.close()
    for s in solvers:
        s.close()
    return out


SERVING_FIRE = dict(synth.FIRE_DEFAULTS, max_iter=200000, force_tol=1e-6)


def serve_stream(rate: float, window_s, extra_s: float, max_requests: int = 2000,
                 max_active: int = 8, budget_gb: float = 120.0, seed: int = 5, sample_s: float = 5.0):
    """Serve the seeded request stream of the serving workload (Poisson
    arrivals, edges 48..192, half patterned substrate + homeotropic top wall,
    half 1-2 colloids, one constant, FP32 form, max|F| < 1e-6) in real time
    on a continuous-batching server with an HBM budget: submit every request
    that arrives within ``window_s`` seconds (None: the first
    ``max_requests``), keep serving ``extra_s`` seconds after the last
    arrival, then stop (the server drops what is left).  Reports the requests
    completed, in flight and queued at the end, the queue over time, the
    sustained site-updates/s (site updates the server issued to the GPU, and
    those of completed solves alone), and p50/p99 time-to-converged of the
    completed requests."""
    from paper_1911_07045_b300 import lqmin
    p = lqmin.fire_params(**SERVING_FIRE)
    sv = lqmin.Server(int(budget_gb * (1 << 30)), max_active=max_active)
    pending, done, timeline = {}, [], []
    t0 = time.perf_counter()
    nxt = [0.0]

    def collect():
        for t in list(pending):
            got = sv.poll(t)
            if got is not None:
                code, res, _ = got
                L, kind = pending.pop(t)
                done.append(dict(latency=res.seconds, iterations=int(res.iterations), L=L, kind=kind,
                                 converged=bool(code == lqmin.LQ_OK and
                                                res.fire_status == lqmin.FIRE_CONVERGED)))

    def tick(force=False):
        now = time.perf_counter() - t0
        if force or now >= nxt[0]:
            collect()
            st = sv.stats()
            timeline.append(dict(t=round(now, 1), queued=st["queued"], active=st["active"],
                                 completed=st["completed"], issued=st["site_updates_issued"]))
            nxt[0] = now + sample_s
        return now

    submitted = 0
    last_arrival = 0.0
    for r in synth.iter_serving_requests(seed=seed, count=max_requests, rate=rate):
        if window_s is not None and r["t_arrival"] > window_s:
            break
        while True:
            now = tick()
            if now >= r["t_arrival"]:
                break
            time.sleep(min(r["t_arrival"] - now, 0.05))
        t = sv.submit(r, p, seed=r["seed"])
        pending[t] = (r["shape"][0], r["kind"])
        submitted += 1
        last_arrival = r["t_arrival"]
    end = (window_s if window_s is not None else last_arrival) + extra_s
    while pending and tick() < end:
        time.sleep(0.05)
    wall = tick(force=True)
    st = sv.stats()
    sv.close()
    lat = np.array([d["latency"] for d in done]) if done else np.array([np.nan])
    # sustained rate: issued site updates between the first sample with work
    # on the GPU and the end
    first = next((x for x in timeline if x["issued"] > 0), timeline[-1])
    span = max(1e-9, timeline[-1]["t"] - first["t"])
    by_edge = {}
    for d in done:
        if d["converged"]:
            by_edge.setdefault(d["L"], []).append(d["iterations"])
    return {"rate_per_s": rate, "arrival_window_s": window_s if window_s is not None else last_arrival,
            "extra_s": extra_s,
            "max_active": max_active, "hbm_budget_gb": budget_gb, "submitted": submitted,
            "completed": len(done), "converged": sum(d["converged"] for d in done),
            "in_flight_at_end": int(st["active"]), "queued_at_end": int(st["queued"]),
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_iterations_completed": float(np.mean([d["iterations"] for d in done])) if done else None,
            "iterations_by_edge": {str(k): float(np.median(v)) for k, v in sorted(by_edge.items())},
            "site_updates_per_s": (timeline[-1]["issued"] - first["issued"]) / span,
            "completed_site_updates_per_s": st["site_updates"] / wall, "wall_s": round(wall, 1),
            "queue_over_time": [[x["t"], x["queued"], x["active"], x["completed"]]
                                for x in timeline[:: max(1, len(timeline) // 24)] + [timeline[-1]]]}


# FIRE iterations to max|F| < 1e-6 of the serving stream's requests by cubic
# edge: the mean over the first five requests of each edge in the seeded
# stream, each minimised alone on a B300 (FP32 form, `bench.py
# --serving-calibrate`; requests that stop at the 200 000-iteration limit
# count with that limit).  The mean work per request from it, 1.70e11 site
# updates, is what the first 64 requests of the stream cost when served (the
# capacity needs the mean, not a typical request); the scaled-rate stream
# takes its arrival rate from these and the measured throughput
SERVING_ITERS_BY_EDGE = {"48": 30886, "64": 34999, "80": 43593, "96": 72288, "112": 78296, "128": 77236,
                         "144": 49290, "160": 94536, "176": 43122, "192": 78535}


def serving_capacity(rate_site_updates: float, iters_by_edge: dict) -> float:
    """Requests per second one GPU finishes at ``rate_site_updates``: the
    stream's edges are uniform over {48, 64, ..., 192}, so the mean work per
    request is the mean over edges of L^3 x iterations(L)."""
    edges = list(range(48, 193, 16))
    known = sorted((int(k), v) for k, v in iters_by_edge.items())
    if not known:
        return float("nan")
    xs = np.array([k for k, _ in known], dtype=float)
    ys = np.array([v for _, v in known], dtype=float)
    work = np.mean([L ** 3 * float(np.interp(L, xs, ys)) for L in edges])
    return rate_site_updates / work


def serving_calibrate(count: int = 5):
    """Minimise the first ``count`` requests of each edge of the seeded
    stream alone (FP32 form, the serving FIRE parameters): iterations and
    seconds of each."""
    from paper_1911_07045_b300 import lqmin
    p = lqmin.fire_params(**SERVING_FIRE)
    seen, out = {}, {}
    for r in synth.iter_serving_requests(count=2000):
        L = r["shape"][0]
        if seen.get(L, 0) >= count:
            continue
        seen[L] = seen.get(L, 0) + 1
        s = lqmin.solver_for(r, precision=lqmin.LQ_FP32_BULK_FP64_RED)
        s.init_random_uniaxial(r["seed"])
        st, res = s.minimize(p)
        out.setdefault(str(L), []).append(dict(iterations=int(res.iterations), seconds=round(res.seconds, 2),
                                               kind=r["kind"], converged=bool(res.fire_status == 1)))
        s.close()
        if len(seen) == 10 and all(v >= count for v in seen.values()):
            break
    return out


def _trace(s, p, seconds, thresholds=(1e-2, 1e-3, 1e-4)):
    """Run one minimiser for about ``seconds`` of wall clock in growing
    chunks of steps: a trace of (time, iterations, |F|/sqrt(N), energy) and
    the time at which |F|/sqrt(N) first fell below each threshold."""
    r = s.step(p, 1)
    t0 = time.perf_counter()
    trace, reach = [], {}
    chunk, it = 16, 1
    while True:
        r = s.step(p, chunk)
        it += chunk
        t = time.perf_counter() - t0
        rms = r.rms_force
        trace.append([round(t, 3), it, rms, s.energy()[0]])
        for thr in thresholds:
            if rms < thr and str(thr) not in reach:
                reach[str(thr)] = round(t, 3)
        if t > seconds or r.fire_status != 0 or not np.isfinite(rms):
            break
        chunk = min(chunk * 2, 1024)
    return trace, reach, it, int(r.fire_status)


def run_objects(L: int, seconds: float):
    """Fig. 3: FIRE against gradient descent on the paper's three object
    geometries (two colloids between plates, a droplet interior, a
    spherocylinder between planar plates) at L^3 from a random start, each
    for the same wall-clock budget on the FP32 form.  The energy is reported
    relative to the lowest energy any run reached on that geometry."""
    from paper_1911_07045_b300 import lqmin
    runs = {
        "fire": lqmin.fire_params(**dict(synth.FIRE_DEFAULTS, max_iter=10 ** 12, force_tol=0.0)),
        # homeotropic anchoring (6 W = 32 on the stiffest boundary mode) adds to
        # the bulk's ~84: eta lam < 2 needs eta < 0.017 here, 0.02 diverges
        "gd_eta_0.015": lqmin.descent_params(lqmin.LQ_MIN_GD, 0.015, max_iter=10 ** 12,
                                             force_tol=0.0),
    }
    out = {"workload": f"Fig. 3 geometries at {L}^3, one constant, random directors (seed 1), "
                       f"FP32 form, {seconds} s per method", "geometries": {}}
    for gname, cfg in synth.config_fig3(L).items():
        res = {}
        for name, p in runs.items():
            s = lqmin.solver_for(cfg, precision=lqmin.LQ_FP32_BULK_FP64_RED)
            s.init_random_uniaxial(1)
            trace, reach, it, status = _trace(s, p, seconds)
            res[name] = dict(trace=trace, reach=reach, iterations=it, status=status)
            s.close()
        e_min = min(min(t[3] for t in r["trace"]) for r in res.values())
        g = {}
        for name, r in res.items():
            tr = [[t, i, rms, e - e_min] for t, i, rms, e in r["trace"]]
            g[name] = {"seconds_to_rms_force": r["reach"], "iterations": r["iterations"],
                       "status": r["status"], "final_rms_force": tr[-1][2],
                       "final_energy_above_min": tr[-1][3],
                       "trace_t_it_rms_dE": tr[:: max(1, len(tr) // 12)] + [tr[-1]]}
        out["geometries"][gname] = {"energy_min": e_min, "methods": g}
    return out


def run_step_scaling(sizes, tol: float, seeds=(1, 2, 3)):
    """Minimisation steps to a force tolerance against the linear size
    (section IV.A: about L steps without boundaries, about L^1.5 with a
    colloid): FIRE from random starts on a periodic one-constant bulk and on
    the same box with a centred homeotropic colloid of radius L/8, FP32
    form, until the largest site force is below ``tol``; the median over
    seeds at each L and the fitted exponent of that median against L."""
    from paper_1911_07045_b300 import lqmin
    hom = (0, synth.W_HOMEOTROPIC, (0.0, 0.0, 1.0))
    p = lqmin.fire_params(**dict(synth.FIRE_DEFAULTS, max_iter=400000, force_tol=tol))
    out = {"workload": f"periodic L^3, one constant, random directors (seeds {list(seeds)}), "
                       f"FP32 form, FIRE to max site force < {tol}", "families": {}}
    for fam in ("bulk", "colloid"):
        rows = []
        for L in sizes:
            objs = [] if fam == "bulk" else [dict(type="sphere", c=((L - 1) / 2.0,) * 3, R=L / 8.0,
                                                  anchor=hom)]
            its, secs, conv = [], [], True
            for seed in seeds:
                s = lqmin.solver_for(dict(shape=(L, L, L), L1=synth.L1_5CB, L2=0.0, L3=0.0,
                                          objects=objs), precision=lqmin.LQ_FP32_BULK_FP64_RED)
                s.init_random_uniaxial(seed)
                st, r = s.minimize(p)
                its.append(int(r.iterations))
                secs.append(round(r.seconds, 3))
                conv = conv and r.fire_status == 1
                s.close()
            rows.append(dict(L=L, iterations=its, median=float(np.median(its)), seconds=secs,
                             converged=conv))
        ok = [w for w in rows if w["converged"]]
        slope = None
        if len(ok) >= 3:
            slope = float(np.polyfit(np.log([w["L"] for w in ok]),
                                     np.log([w["median"] for w in ok]), 1)[0])
        out["families"][fam] = {"runs": rows, "fitted_exponent": slope}
    return out


def run_precision_check(max_iter: int = 400000):
    """The FP32-bulk / FP64-reduction form against the plain FP64 path on the
    same GPU, at the accuracy the precision form must keep (final energy
    within 1e-6 relative, per-site order parameter within 1e-4): the 128^3
    colloid slab (homeotropic walls, centred colloid R = 20, three
    constants) from a smooth start -- a uniform director tilted slightly
    from z, so that both forms settle in the same basin (from a random start
    they may reach different defect arrangements) -- minimised by FIRE to a
    largest site force of 1e-7 (FP64) and 1e-6 (FP32 form)."""
    from paper_1911_07045_b300 import lqmin
    cfg = synth.config_colloid_slab()
    n = np.array([0.1, 0.05, 1.0])
    n /= np.linalg.norm(n)
    N = int(np.prod(cfg["shape"]))
    q0 = np.repeat(synth.uniaxial_q(n[:, None], synth.s0_closed_form(synth.A_5CB, synth.B_5CB,
                                                                      synth.C_5CB)), N, axis=1)
    out = {"workload": "128^3 slab, homeotropic walls z=0,127 and colloid R=20 (W=5.3), "
                       "L1/L2/L3=2.32/0.5/0.3, smooth start (director (0.1, 0.05, 1))"}
    res = {}
    for form, prec, tol in (("fp64", lqmin.LQ_FP64, 1e-7), ("fp32", lqmin.LQ_FP32_BULK_FP64_RED, 1e-6)):
        s = lqmin.solver_for(cfg, precision=prec)
        s.set_q(q0)
        st, r = s.minimize(lqmin.fire_params(**dict(synth.FIRE_DEFAULTS, max_iter=max_iter,
                                                    force_tol=tol)))
        sim = (s.mask() & 1).astype(bool)
        res[form] = dict(energy=r.energy, S=s.order_field()[sim], iterations=int(r.iterations),
                         status=int(r.fire_status), seconds=round(r.seconds, 3), tol=tol)
        s.close()
    e64, e32 = res["fp64"]["energy"], res["fp32"]["energy"]
    out.update({f: {k: v for k, v in r.items() if k != "S"} for f, r in res.items()})
    out["energy_rel_diff"] = abs(e32 - e64) / abs(e64)
    out["max_S_diff"] = float(np.abs(res["fp32"]["S"] - res["fp64"]["S"]).max())
    out["within_tolerance"] = bool(out["energy_rel_diff"] <= 1e-6 and out["max_S_diff"] <= 1e-4)
    return out


def run_minimizers(L: int, seconds: float):
    """FIRE against gradient descent and Nesterov's accelerated gradient on a
    periodic one-constant bulk from a random start (the comparison of Fig. 2,
    at L^3), each for the same wall-clock budget on the FP32 form: the
    residual |F|/sqrt(N) and the energy against time, and the time each
    method needs to bring |F|/sqrt(N) below 1e-2, 1e-3, 1e-4."""
    from paper_1911_07045_b300 import lqmin
    cfg = dict(shape=(L, L, L), L1=synth.L1_5CB, L2=0.0, L3=0.0, objects=[])
    runs = {
        "fire": lqmin.fire_params(**dict(synth.FIRE_DEFAULTS, max_iter=10 ** 12, force_tol=0.0)),
        "fire_dtmax_0.05": lqmin.fire_params(**dict(synth.FIRE_DEFAULTS, dt_max=0.05,
                                                    max_iter=10 ** 12, force_tol=0.0)),
        # steps near the stability limit of the stiffest mode: eta lam < 2
        # (GD), < 2 (1 + mu) / (1 + 2 mu) (Nesterov), lam ~ 3 L1 x 12 = 84
        "gd_eta_0.02": lqmin.descent_params(lqmin.LQ_MIN_GD, 0.02, max_iter=10 ** 12, force_tol=0.0),
        "nesterov_eta_0.012_mu_0.9": lqmin.descent_params(lqmin.LQ_MIN_NESTEROV, 0.012, momentum=0.9,
                                                          max_iter=10 ** 12, force_tol=0.0),
    }
    out = {"workload": f"{L}^3 periodic bulk, one constant, random directors (seed 1), FP32 form, "
                       f"{seconds} s each", "methods": {}}
    for name, p in runs.items():
        s = lqmin.solver_for(cfg, precision=lqmin.LQ_FP32_BULK_FP64_RED)
        s.init_random_uniaxial(1)
        trace, reach, it, status = _trace(s, p, seconds)
        out["methods"][name] = {"seconds_to_rms_force": reach, "iterations": it,
                                "status": status,
                                "final_rms_force": trace[-1][2], "final_energy": trace[-1][3],
                                "trace": trace[:: max(1, len(trace) // 12)] + [trace[-1]]}
        s.close()
    return out


def _oracle_fire_rate(L_sample, steps, threads=None):
    """FIRE iterations of the FP64 oracle on an L_sample^3 lattice with the
    bench workload's structure; site-updates/s and the threads it used."""
    import oracle
    oracle.build()
    if threads is not None:
        oracle.set_num_threads(threads)
    cfg = synth.config_large(L_sample)
    o = oracle.Oracle(cfg["shape"], synth.A_5CB, synth.B_5CB, synth.C_5CB, cfg["L1"], cfg["L2"],
                      cfg["L3"], objects=cfg["objects"])
    q = synth.random_uniaxial_q(cfg["shape"], cfg["seed"])
    params = dict(synth.FIRE_DEFAULTS, max_iter=10 ** 9, force_tol=0.0)
    q, v, F, st = o.fire(q, params, 0)           # initial force, not timed
    t0 = time.perf_counter()
    q, v, F, st = o.fire(q, params, steps, state=st, v=v, F=F)
    dt = time.perf_counter() - t0
    return o.N * steps / dt, oracle.num_threads(), dt


def cpu_baseline(L_sample=128, steps=16):
    """The oracle as it stands, on the host cores: FIRE iterations on a
    L_sample^3 lattice with the same structure (colloids scaled by L/512,
    planar walls, three constants), on every host core; then on one thread
    (a 64^3 sample of 3 iterations)."""
    import oracle
    all_cores = os.cpu_count() or 1
    val, cores, dt = _oracle_fire_rate(L_sample, steps, threads=all_cores)
    v1, _, dt1 = _oracle_fire_rate(64, 3, threads=1)
    oracle.set_num_threads(all_cores)
    return {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{steps} FIRE iterations of the FP64 oracle on a {L_sample}^3 lattice with the "
                      f"same structure (4 colloids scaled by {L_sample}/512, planar walls, 3 constants)",
            "seconds": dt, "cpu_model": _cpu_model(),
            "single_thread": {"value": v1, "unit": UNIT, "cores": 1, "seconds": dt1,
                              "sample": "3 FIRE iterations of the FP64 oracle on a 64^3 lattice with the "
                                        "same structure"}}


def _cpu_model() -> str:
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def run_baselines():
    """The CPU-baseline plan next to the GPU forms, on the workloads the
    oracle can finish: config 1 (32^3 periodic bulk, one constant, random
    start seed 1, FIRE to max site |F| < 1e-9) minimised in full by the
    oracle on every host core, by the FP64 form and by the FP32 form (to
    1e-6, the FP32 form's tolerance); config 2 (128^3 colloid slab, three
    constants, seed 2, tol 1e-8) minimised in full by the FP64 form and the
    FP32 form (1e-6), with the oracle's rate on it from 4 iterations on
    every core and 1 on one thread (a full oracle minimisation of config 2
    takes hours)."""
    import oracle
    from paper_1911_07045_b300 import lqmin
    oracle.build()
    all_cores = os.cpu_count() or 1
    out = {"host": {"cpu_model": _cpu_model(), "cores": all_cores}}
    # config 1
    c1 = synth.config_small_periodic()
    q0 = synth.random_uniaxial_q(c1["shape"], c1["seed"])
    N1 = int(np.prod(c1["shape"]))
    oracle.set_num_threads(all_cores)
    o = oracle.Oracle(c1["shape"], synth.A_5CB, synth.B_5CB, synth.C_5CB, c1["L1"], 0.0, 0.0)
    params = dict(synth.FIRE_DEFAULTS, max_iter=10 ** 6, force_tol=c1["tol"])
    t0 = time.perf_counter()
    q, v, F, st = o.fire(q0, params, 10 ** 6)
    dt = time.perf_counter() - t0
    e_orc = o.energy(q)[0]
    res = {"oracle_fp64": dict(iterations=int(st["iter"]), seconds=round(dt, 2),
                               converged=bool(st["status"] == 1), energy=e_orc,
                               site_updates_per_s=N1 * st["iter"] / dt, cores=oracle.num_threads())}
    for form, prec, tol in (("gpu_fp64", lqmin.LQ_FP64, c1["tol"]),
                            ("gpu_fp32", lqmin.LQ_FP32_BULK_FP64_RED, 1e-6)):
        s = lqmin.solver_for(c1, precision=prec)
        s.set_q(q0)
        code, r = s.minimize(lqmin.fire_params(**dict(synth.FIRE_DEFAULTS, max_iter=10 ** 6,
                                                       force_tol=tol)))
        res[form] = dict(iterations=int(r.iterations), seconds=round(r.seconds, 3), tol=tol,
                         converged=bool(r.fire_status == 1), energy=r.energy,
                         energy_rel_diff_vs_oracle=abs(r.energy - e_orc) / abs(e_orc),
                         site_updates_per_s=N1 * r.iterations / r.seconds)
        s.close()
    out["config1_32cube"] = res
    # config 2
    c2 = synth.config_colloid_slab()
    N2 = int(np.prod(c2["shape"]))
    q0 = synth.random_uniaxial_q(c2["shape"], c2["seed"])
    res = {}
    for form, prec, tol in (("gpu_fp64", lqmin.LQ_FP64, c2["tol"]),
                            ("gpu_fp32", lqmin.LQ_FP32_BULK_FP64_RED, 1e-6)):
        s = lqmin.solver_for(c2, precision=prec)
        s.set_q(q0)
        code, r = s.minimize(lqmin.fire_params(**dict(synth.FIRE_DEFAULTS, max_iter=400000,
                                                       force_tol=tol)))
        res[form] = dict(iterations=int(r.iterations), seconds=round(r.seconds, 3), tol=tol,
                         converged=bool(r.fire_status == 1), energy=r.energy,
                         site_updates_per_s=N2 * r.iterations / r.seconds)
        s.close()
    o2 = oracle.Oracle(c2["shape"], synth.A_5CB, synth.B_5CB, synth.C_5CB, c2["L1"], c2["L2"], c2["L3"],
                       objects=c2["objects"])
    p2 = dict(synth.FIRE_DEFAULTS, max_iter=10 ** 9, force_tol=0.0)
    for key, threads, steps in (("oracle_fp64_all_cores", all_cores, 4), ("oracle_fp64_1_thread", 1, 1)):
        oracle.set_num_threads(threads)
        q, v, F, st = o2.fire(q0, p2, 0)
        t0 = time.perf_counter()
        o2.fire(q, p2, steps, state=st, v=v, F=F)
        dt = time.perf_counter() - t0
        res[key] = dict(iterations=steps, seconds=round(dt, 2), cores=threads,
                        site_updates_per_s=N2 * steps / dt)
    oracle.set_num_threads(all_cores)
    out["config2_128cube"] = res
    # the oracle on one thread on config 1's lattice too
    oracle.set_num_threads(1)
    q, v, F, st = o.fire(synth.random_uniaxial_q(c1["shape"], c1["seed"]), params, 0)
    t0 = time.perf_counter()
    o.fire(q, dict(params, force_tol=0.0), 20, state=st, v=v, F=F)
    dt = time.perf_counter() - t0
    out["config1_32cube"]["oracle_fp64_1_thread_rate"] = dict(iterations=20, seconds=round(dt, 2),
                                                             site_updates_per_s=N1 * 20 / dt)
    oracle.set_num_threads(all_cores)
    return out


def main_ours(args, dist: Dist):
    import torch
    torch.cuda.set_device(dist.local)
    t_start = time.perf_counter()
    legs = {}
    peak, peak_kind = measured_peaks()
    forms = {}
    for prec in args.precision.split(","):
        # the FP64 form is ~13x slower: a tenth of the steps, but at least 10
        # (half a second at 512^3), keeps its timed region long enough to time
        k = args.steps if prec.startswith("fp32") else max(10, args.steps // 10)
        forms[prec] = run_form(prec, args.size, k, args.warmup, dist, dist.local, args.staging)
    legs["forms"] = round(time.perf_counter() - t_start, 1)
    fp64_rate = None
    if any(not k.startswith("fp32") for k in forms):
        from paper_1911_07045_b300 import lqmin
        fp64_rate = lqmin.fp64_fma_rate() / 1e9      # measured, G FP64 op/s
    head = "fp32" if "fp32" in forms else next(iter(forms))
    h = forms[head]
    # roofline of the step kernel: algorithmic bytes per launch over the
    # device time per launch (CUDA events around the timed launches)
    rl = {}
    for k, f in forms.items():
        base = k.split("_")[0]    # the one-constant forms move the same state bytes
        traffic = DRAM_BYTES_PER_SITE.get(k, DRAM_BYTES_PER_SITE[base]) * f["N"]
        if base == "fp32":
            ach = ALG_BYTES[base] * f["N"] / f["per_launch_s"] / 1e9
            rl[k] = {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(ach / peak, 4), "traffic": round(traffic),
                     "dram_gbs": round(traffic / f["per_launch_s"] / 1e9, 1),
                     "dram_frac": round(traffic / f["per_launch_s"] / 1e9 / peak, 4),
                     "design_bytes_per_site": DESIGN_BYTES[base], "alg_bytes_per_site": ALG_BYTES[base],
                     "peak_kind": peak_kind + " (HBM copy)"}
            if k not in DRAM_BYTES_PER_SITE:
                rl[k]["traffic_from"] = "three-constant capture (same state bytes)"
        else:
            # FP64 pipe: the measured fused multiply-add rate (lq_fp64_fma_rate);
            # the figure derived from 148 SMs x 2 FP64 ops/clock x max SM clock
            # is kept beside it
            derived = N_SM * FP64_OPS_PER_CLK_SM * (f["clocks"].get("sm_max_mhz") or 2032.0) * 1e6 / 1e9
            ops = FP64_OPS_PER_SITE if k == base else FP64_OPS_PER_SITE_1C
            ach = ops * f["N"] / f["per_launch_s"] / 1e9
            rl[k] = {"bound": "alu", "achieved": round(ach, 1), "peak": round(fp64_rate, 1),
                     "unit": "G FP64 op/s", "frac": round(ach / fp64_rate, 4),
                     "traffic": round(traffic), "ops_per_site": ops,
                     "hbm_frac": round(traffic / f["per_launch_s"] / 1e9 / peak, 4),
                     "peak_kind": "measured: FP64 fused multiply-add chains on every SM "
                                  "(lq_fp64_fma_rate), CUDA events",
                     "derived_peak": round(derived, 1)}
            if k not in DRAM_BYTES_PER_SITE:
                rl[k]["traffic_from"] = "three-constant capture (same state bytes)"
    line = {
        "metric": METRIC, "value": h["value"], "unit": UNIT, "n_gpus": dist.world,
        "steps": h["launches"], "warmup": args.warmup, "ms_per_step": h["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if head == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.size), "form": head, "sites_per_gpu": h["N"], "simulated_sites": h["nsim"],
                   "anchored_sites": h["nanchored"],
                   "parallelism": f"replicas x{dist.world}" if dist.world > 1 else "1 GPU",
                   "l2": "inputs larger than L2 (state > 126 MB)"},
        "roofline": rl[head],
        "forms": {k: {"value": f["value"], "ms_per_step": f["ms_per_step"], "steps": f["launches"],
                      "roofline": rl[k], "clocks": f["clocks"], "valid": f["ok"]}
                  for k, f in forms.items()},
        "e2e": h["e2e"],
        "gpu_launches": sum(f["launches"] for f in forms.values()),
        "clocks": h["clocks"],
    }
    def leg(name, fn, *a):
        t = time.perf_counter()
        line[name] = fn(*a)
        legs[name] = round(time.perf_counter() - t, 1)
    if dist.world == 1 and args.batch_steps > 0:
        leg("batched", run_batch, args.batch_steps,
            tuple(int(v) for v in args.batch_tile.split("x")) if args.batch_tile else None)
    if dist.world == 1 and args.serving_window > 0:
        leg("served", run_served, args)
    if dist.world == 1 and not args.no_precision_check:
        leg("precision_check", run_precision_check)
    if dist.world == 1 and args.minimizers > 0:
        leg("minimizers", run_minimizers, args.minimizer_size, args.minimizers)
    if dist.world == 1 and args.objects > 0:
        leg("objects_fig3", run_objects, args.minimizer_size, args.objects)
    if dist.world == 1 and args.step_scaling:
        leg("step_scaling", run_step_scaling, [int(v) for v in args.step_scaling.split(",")],
            args.step_scaling_tol)
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        leg("cpu_baseline", cpu_baseline)
    legs["total"] = round(time.perf_counter() - t_start, 1)
    line["wall_seconds_by_leg"] = legs
    if not all(f["ok"] for f in forms.values()):
        line["invalid"] = "FIRE stopped before all timed steps ran"
    return line


def run_served(args):
    """The serving workload: (1) the seeded stream at its own rate (20/s) for
    ``--serving-window`` seconds of arrivals -- far above what one GPU serves,
    so the queue grows and the latencies are those of the requests that
    finished; (2) the scaled-rate deviation: ``--serving-scaled`` requests of
    the same stream at about 0.8 of the measured capacity (arrival rate from
    the per-edge steps-to-converge and the throughput of stream 1)."""
    out = {"workload": "seeded serving stream (seed 5): Poisson arrivals, cubic edges 48..192 step 16, "
                       "half patterned substrate + homeotropic top wall, half 1-2 colloids, one constant, "
                       "FP32 form, FIRE to max|F| < 1e-6, HBM budget 120 GB"}
    a = serve_stream(args.serving_rate, args.serving_window, args.serving_extra,
                     max_active=args.serving_max_active)
    out["stream"] = a
    if args.serving_scaled > 0:
        table = SERVING_ITERS_BY_EDGE or a["iterations_by_edge"]
        cap = serving_capacity(a["site_updates_per_s"], table)
        if np.isfinite(cap) and cap > 0:
            rate = args.serving_utilisation * cap
            # the first --serving-scaled requests of the stream at this rate,
            # then a drain of a fraction of their expected arrival span
            b = serve_stream(rate, None, args.serving_scaled_extra * args.serving_scaled / rate,
                             max_requests=args.serving_scaled, max_active=args.serving_max_active)
            b["capacity_req_per_s"] = cap
            b["target_utilisation"] = args.serving_utilisation
            b["iterations_table"] = "committed calibration" if SERVING_ITERS_BY_EDGE else "stream 1 completions"
            out["scaled_rate"] = b
    p50, p99 = out.get("scaled_rate", a)["p50_s"], out.get("scaled_rate", a)["p99_s"]
    out.update(p50_s=p50, p99_s=p99, site_updates_per_s=a["site_updates_per_s"])
    return out


def workload_name(size: int) -> str:
    return (f"{size}^3 lattice, 4 homeotropic colloids (W=5.3), planar walls z=0,{size - 1} (W=1), "
            f"L1/L2/L3=2.32/0.5/0.3, random uniaxial start (seed 3)")


def main_reference(args, dist: Dist):
    """CPU oracle as the reference arm: each step is one FIRE iteration of
    the oracle on a bounded 96^3 sample of the workload."""
    if dist.rank != 0:
        return None
    import oracle
    oracle.build()
    Ls = 96
    cfg = synth.config_large(Ls)
    o = oracle.Oracle(cfg["shape"], synth.A_5CB, synth.B_5CB, synth.C_5CB, cfg["L1"], cfg["L2"],
                      cfg["L3"], objects=cfg["objects"])
    q = synth.random_uniaxial_q(cfg["shape"], cfg["seed"])
    params = dict(synth.FIRE_DEFAULTS, max_iter=10 ** 9, force_tol=0.0)
    q, v, F, st = o.fire(q, params, 0)
    q, v, F, st = o.fire(q, params, args.warmup, state=st, v=v, F=F)
    t0 = time.perf_counter()
    q, v, F, st = o.fire(q, params, args.steps, state=st, v=v, F=F)
    sec = time.perf_counter() - t0
    val = o.N * args.steps / sec
    sample = (f"each step = 1 FIRE iteration of the FP64 oracle on a {Ls}^3 lattice with the same "
              f"structure (colloids scaled by {Ls}/512, planar walls, 3 constants)")
    return {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": dist.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(args.size), "form": "fp64 oracle",
                       "sample": f"{Ls}^3 lattice with the same structure",
                       "parallelism": f"1 process, {oracle.num_threads()} host threads"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=512)
    ap.add_argument("--precision", default="fp32,fp64,fp32_1c,fp64_1c")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--staging", type=int, default=0, choices=[0, 1, 2],
                    help="plane staging of the FP32 three-constant step: 0 automatic, 1 per-thread "
                         "loads, 2 tensor copies (lq_set_staging)")
    ap.add_argument("--batch-steps", type=int, default=50)
    ap.add_argument("--batch-tile", default="",
                    help="WxHxZ: run the batched leg with this tiling instead of autotuning it")
    ap.add_argument("--serving-window", type=float, default=100.0,
                    help="seconds of arrivals of the served stream (0: skip serving)")
    ap.add_argument("--serving-extra", type=float, default=10.0,
                    help="seconds of serving after the last arrival before stopping")
    ap.add_argument("--serving-rate", type=float, default=20.0)
    ap.add_argument("--serving-max-active", type=int, default=8)
    ap.add_argument("--serving-scaled", type=int, default=32,
                    help="requests of the scaled-rate stream (0: skip); at 0.8 of capacity (0.1 "
                         "requests/s) the first 32 arrive over 331 s, the first 64 over 757 s")
    ap.add_argument("--serving-utilisation", type=float, default=0.8)
    ap.add_argument("--serving-scaled-extra", type=float, default=0.25,
                    help="drain time of the scaled-rate stream as a fraction of its arrival window")
    ap.add_argument("--baselines", action="store_true",
                    help="only run the CPU-baseline plan: full minimisations of the 32^3 and 128^3 "
                         "workloads next to the oracle, and print them")
    ap.add_argument("--serving-calibrate", action="store_true",
                    help="only minimise the first requests of each edge of the served stream alone and "
                         "print them with the median and mean iterations per edge")
    ap.add_argument("--serving-calibrate-count", type=int, default=5,
                    help="requests per edge of --serving-calibrate")
    ap.add_argument("--minimizers", type=float, default=0.0,
                    help="seconds per method of the FIRE / GD / Nesterov comparison (0: skip)")
    ap.add_argument("--minimizer-size", type=int, default=250)
    ap.add_argument("--no-precision-check", action="store_true",
                    help="skip the FP32-form-against-FP64 minimisation of the 128^3 slab")
    ap.add_argument("--objects", type=float, default=0.0,
                    help="seconds per method of the Fig. 3 object-geometry comparison (0: skip)")
    ap.add_argument("--step-scaling", default="",
                    help="comma-separated edges L of the steps-to-tolerance study (empty: skip)")
    ap.add_argument("--step-scaling-tol", type=float, default=1e-5)
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    if args.baselines:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"baselines": run_baselines()}), flush=True)
        return
    if args.serving_calibrate:
        import torch
        torch.cuda.set_device(0)
        cal = serving_calibrate(args.serving_calibrate_count)
        med = {L: int(np.median([x["iterations"] for x in v])) for L, v in cal.items()}
        mean = {L: int(np.mean([x["iterations"] for x in v])) for L, v in cal.items()}
        print(json.dumps({"serving_calibration": cal, "median_iterations_by_edge": med,
                          "mean_iterations_by_edge": mean}), flush=True)
        return
    dist = Dist(backend="gloo" if args.impl == "reference" else None)
    try:
        line = main_reference(args, dist) if args.impl == "reference" else main_ours(args, dist)
        if dist.rank == 0 and line is not None:
            print(json.dumps(line), flush=True)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
