"""Benchmark of the relativistic lattice Boltzmann step on GB300.

Workload (N = 1): the 4096 x 4096 periodic random flow (m/T = 1, tau = 0.8,
stencil G5,G12,G14,G17,G21,G26 folded to Q = 58), FP32 population storage.
One step = one fused pull-stream / moments / Landau / EOS / equilibrium /
Anderson-Witting update of every site.  Metric: MLUPS (million lattice-site
updates per second) and the fraction of the measured HBM roofline, where the
algorithmic bytes of a site update are the populations read and written
(2 Q sizeof(storage)).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--dtype f32|f64]
  python bench.py --impl reference      # the FP64 CPU oracle on host cores

With N > 1 (torchrun) every rank advances its own independent lattice of the
same size (weak scaling, no data-path collective); value = all sites updated
by all ranks / max-over-ranks time.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "MLUPS and % HBM roofline on 1 GB300, FP32/BF16 vs FP64 at stated error"
WORKLOAD = "random_flow_4096: 4096x4096 periodic random flow, n,T = 1+0.01 g, u = 0.05 g (g Gaussian-smoothed, width 8), m/T=1, tau=0.8, stencil G5,G12,G14,G17,G21,G26 (Q=58 folded), v0=0.23342"
N_SIDE = 4096
TAU = 0.8


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class _NVMLClocks:
    """Read-only NVML queries through ctypes (SM clock, its maximum and the
    clock-event reasons); the device is matched to the CUDA device by PCI bus
    id when torch reports it, else by index."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, gpu_index):
        import ctypes
        self.C = ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        h = ctypes.c_void_p()
        bus = None
        try:
            import torch
            pr = torch.cuda.get_device_properties(gpu_index)
            bus = ("%08X:%02X:%02X.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)).encode()
        except Exception:
            bus = None
        if not (bus and lib.nvmlDeviceGetHandleByPciBusId_v2(bus, ctypes.byref(h)) == 0):
            if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(gpu_index), ctypes.byref(h)) != 0:
                raise RuntimeError("no NVML handle")
        self.lib, self.h = lib, h
        self.reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        mx = ctypes.c_uint()
        self.max_mhz = float(mx.value) if lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0 else None

    def sample(self):
        C = self.C
        mhz, rs = C.c_uint(), C.c_ulonglong()
        if self.lib.nvmlDeviceGetClockInfo(self.h, 1, C.byref(mhz)) != 0:
            return None
        if self.reasons_fn(self.h, C.byref(rs)) != 0:
            return None
        return float(mhz.value), [nm for bit, nm in self.REASONS.items() if rs.value & bit]


class ClockSampler:
    """SM clock samples during the timed region (read-only queries): NVML
    polled every 2 ms from a thread where libnvidia-ml is loadable, else
    nvidia-smi every 20 ms.  Started before the region and stopped after it."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.rows = []          # (sm_mhz, max_mhz, [reasons])
        self.proc = None
        self.nvml = None
        self.stop = threading.Event()
        self.source = None

    def __enter__(self):
        try:
            self.nvml = _NVMLClocks(self.idx)
            self.source = "nvml, 2 ms"
            self.t = threading.Thread(target=self._poll, daemon=True)
            self.t.start()
            return self
        except Exception:
            self.nvml = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.source = "nvidia-smi, 20 ms"
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)     # the first query row is out before the region starts
        except Exception:
            self.proc = None
        return self

    def _poll(self):
        while not self.stop.is_set():
            r = self.nvml.sample()
            if r:
                self.rows.append((r[0], self.nvml.max_mhz, r[1]))
            time.sleep(0.002)

    def _read(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.proc.stdout:
            r = [c.strip() for c in line.split(",")]
            try:
                self.rows.append((float(r[1]), float(r[2]),
                                  [nm for k, nm in enumerate(names) if r[5 + k].lower().startswith("active")]))
            except Exception:
                continue

    def __exit__(self, *exc):
        self.stop.set()
        if self.nvml:
            self.t.join(timeout=1)
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm = [r[0] for r in self.rows]
        mx = next((r[1] for r in reversed(self.rows) if r[1]), None)
        reasons = sorted({nm for r in self.rows for nm in r[2]})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": reasons, "samples": len(sm), "source": self.source}


def cpu_baseline(seconds=12.0, side=96, procs=None):
    """The FP64 oracle as it stands on the host cores: `procs` independent
    processes (default: one per core), each with one thread, each advancing its
    own side x side lattice drawn by the same generator (same smoothing,
    amplitudes and seed) for about `seconds` of CPU time.  Value = the site
    updates of all processes / wall time."""
    procs = procs or os.cpu_count() or 1
    w0 = time.perf_counter()
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = (
        "import sys, time, json; sys.path.insert(0, %r)\n"
        "from paper_1703_04605_gb300 import workloads as W\n"
        "from oracle import lattice as L\n"
        "f = W.random_flow(%d)\n"
        "st = W.STENCIL_M1\n"
        "lat = L.make_lattice(st['groups'], st['m'], st['v0'], %r, (%d, %d))\n"
        "lat.init(f['n'], f['ux'], f['uy'], f['T'])\n"
        "t0 = time.process_time(); w0 = time.time(); k = 0\n"
        "while time.process_time() - t0 < %r:\n"
        "    lat.step(1); k += 1\n"
        "dt = time.time() - w0\n"
        "print(json.dumps({'steps': k, 'seconds': dt}))\n"
    ) % (ROOT, side, TAU, side, side, seconds)
    ps = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                           text=True, env=env) for _ in range(procs)]
    res, errs = [], []
    for p in ps:
        out, err = p.communicate()
        if p.returncode == 0:
            res.append(json.loads(out.strip().splitlines()[-1]))
        else:
            errs.append(err.strip().splitlines()[-1] if err.strip() else "failed")
    if not res:
        return {"value": None, "unit": "MLUPS", "cores": procs, "kind": "oracle", "sample": "failed: " + errs[0]}
    mlups = sum(side * side * r["steps"] / r["seconds"] for r in res) / 1e6
    return {"value": mlups, "unit": "MLUPS", "cores": len(res), "kind": "oracle",
            "wall_ms": (time.perf_counter() - w0) * 1e3,
            "site_updates": sum(side * side * r["steps"] for r in res),
            "sample": "%d processes x one %dx%d lattice of the same generator, %d-%d steps each in %.1f s wall, "
                      "1 thread each" % (len(res), side, side, min(r["steps"] for r in res),
                                         max(r["steps"] for r in res), max(r["seconds"] for r in res))}


def cpu_baseline3d(seconds=10.0, side=12, procs=None):
    """The FP64 oracle's 3D lattice on the host cores: one process per core,
    each advancing its own side^3 lattice of the 3D random-flow recipe (same
    stencil, m, tau) for about `seconds` of CPU time."""
    procs = procs or os.cpu_count() or 1
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = (
        "import sys, time, json; sys.path.insert(0, %r)\n"
        "from paper_1703_04605_gb300 import workloads as W\n"
        "from oracle import lattice as L\n"
        "f = W.random_flow3d(%d)\n"
        "st = W.STENCIL_M1\n"
        "lat = L.make_lattice(st['groups'], st['m'], st['v0'], %r, (%d, %d, %d), two_d=False)\n"
        "lat.init(f['n'], f['ux'], f['uy'], f['T'], uz=f['uz'])\n"
        "t0 = time.process_time(); w0 = time.time(); k = 0\n"
        "while time.process_time() - t0 < %r:\n"
        "    lat.step(1); k += 1\n"
        "print(json.dumps({'steps': k, 'seconds': time.time() - w0}))\n"
    ) % (ROOT, side, TAU, side, side, side, seconds)
    ps = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                           text=True, env=env) for _ in range(procs)]
    res = []
    for p in ps:
        out, _ = p.communicate()
        if p.returncode == 0:
            res.append(json.loads(out.strip().splitlines()[-1]))
    if not res:
        return {"value": None, "unit": "MLUPS", "cores": procs, "kind": "oracle", "sample": "failed"}
    return {"value": sum(side ** 3 * r["steps"] / r["seconds"] for r in res) / 1e6, "unit": "MLUPS",
            "cores": len(res), "kind": "oracle",
            "sample": "%d processes x one %d^3 lattice of the 3D recipe, %d-%d steps each, 1 thread each" % (
                len(res), side, min(r["steps"] for r in res), max(r["steps"] for r in res))}


def cpu_baseline_o3(seconds=10.0, side=24, procs=None):
    """The FP64 oracle's third-order lattice on the host cores: one process
    per core, each advancing its own side^2 lattice of the random-flow recipe
    with the third-order stencil (same m, tau) for about `seconds` of CPU time."""
    procs = procs or os.cpu_count() or 1
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = (
        "import sys, time, json; sys.path.insert(0, %r)\n"
        "from paper_1703_04605_gb300 import workloads as W\n"
        "from oracle import lattice as L\n"
        "f = W.random_flow(%d)\n"
        "st = W.STENCIL_O3\n"
        "lat = L.make_lattice(st['groups'], st['m'], st['v0'], %r, (%d, %d))\n"
        "lat.init(f['n'], f['ux'], f['uy'], f['T'])\n"
        "t0 = time.process_time(); w0 = time.time(); k = 0\n"
        "while time.process_time() - t0 < %r:\n"
        "    lat.step(1); k += 1\n"
        "print(json.dumps({'steps': k, 'seconds': time.time() - w0}))\n"
    ) % (ROOT, side, TAU, side, side, seconds)
    ps = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                           text=True, env=env) for _ in range(procs)]
    res = []
    for p in ps:
        out, _ = p.communicate()
        if p.returncode == 0:
            res.append(json.loads(out.strip().splitlines()[-1]))
    if not res:
        return {"value": None, "unit": "MLUPS", "cores": procs, "kind": "oracle", "sample": "failed"}
    return {"value": sum(side ** 2 * r["steps"] / r["seconds"] for r in res) / 1e6, "unit": "MLUPS",
            "cores": len(res), "kind": "oracle",
            "sample": "%d processes x one %d^2 lattice of the random-flow recipe, third-order stencil, "
                      "%d-%d steps each, 1 thread each" % (
                          len(res), side, min(r["steps"] for r in res), max(r["steps"] for r in res))}


# FP64 paths are bound by the FP64 pipe.  FLOPs per site of the FP64 step
# kernels on the benchmarked stencils, from ncu's FP64 instruction counts
# (profiles/fp64_kernels_alu_1024.md).  The peak is measured (fp64_peak); GB300's
# nominal FP64 rate is reported beside it and used only if the probe fails.
FP64_PEAK_TFLOPS = 1.25
FP64_FLOP_PER_SITE = {"step_f64_kernel/5,12,14,17,21,26": 3271.0,
                      "step_o3_kernel/1,2,5,6,7,9,10,11,12,13,15": 7352.0}


_FP64_PEAK = []


def fp64_peak():
    """(TFLOP/s, kind): the FP64 FMA rate measured on this GPU by the
    library's own probe (rlbm_fp64_fma_rate, CUDA events), once per process;
    the nominal figure if the probe fails."""
    if not _FP64_PEAK:
        import ctypes as C
        from paper_1703_04605_gb300 import _abi as A
        v = C.c_double()
        ok = A.load().rlbm_fp64_fma_rate(None, C.byref(v)) == A.RLBM_OK and v.value > 0
        _FP64_PEAK.append((v.value, "measured (rlbm_fp64_fma_rate: FMA chains on register operands, best of 5, CUDA events)")
                          if ok else (FP64_PEAK_TFLOPS, "nominal"))
    return _FP64_PEAK[0]


def fp64_alu(mlups, key):
    flop = FP64_FLOP_PER_SITE.get(key)
    if flop is None:
        return None
    achieved = mlups * 1e6 * flop / 1e12
    peak, kind = fp64_peak()
    return {"bound": "alu", "unit": "TFLOP/s", "achieved": achieved, "peak": peak,
            "peak_kind": kind, "frac": achieved / peak, "flop_per_site": flop,
            "nominal_peak": FP64_PEAK_TFLOPS,
            "flop_source": "ncu FP64 instruction counts (profiles/fp64_kernels_alu_1024.md)"}


def kernel_name(dtype, variant):
    stencil = {1: "5,12,14,17,21,26", 2: "1,2,3,4,5,6", 3: "1,14,49,51,60,70", 4: "3,9,10,14,17,21"}.get(variant)
    if dtype == "f64":
        return "step_f64_kernel<64>"
    if stencil is None:
        return "step_f32_kernel<64>"
    return "fused_f32_kernel<StencilDef<%s>, %s>" % (stencil, "true" if dtype == "bf16dev" else "false")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(value, pg, device):
    """Max over ranks of a per-rank time (identity without a process group)."""
    if pg is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


REJECTING_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")


def clocks_rejected(summary, low=0.85):
    """True when a timed region's clock record disqualifies its number: a
    hardware or thermal slowdown was active, or the median SM clock sat well
    below the maximum with no reason given (a clock lock left behind).
    sw_power_cap is kept (normal under a dense load on a power-capped part)."""
    if not summary:
        return False
    if any(r in REJECTING_REASONS for r in summary.get("reasons", [])):
        return True
    sm, mx = summary.get("sm_mhz"), summary.get("sm_max_mhz")
    return bool(sm and mx and sm < low * mx and not summary.get("reasons"))


def whole_job_mlups(sites_per_rank, world_size, ms_per_step_max):
    """Weak scaling: every rank updates its own lattice; the job's throughput
    is all ranks' site updates over the slowest rank's time."""
    return world_size * float(sites_per_rank) / (ms_per_step_max / 1e3) / 1e6


def emit(line, rank):
    """The one JSON line, printed by rank 0 only."""
    if rank == 0:
        print(json.dumps(line), flush=True)


def _source_hash(files):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


O3_SOURCES = ["paper_1703_04605_gb300/csrc/rlbm_fused_o3.cu", "paper_1703_04605_gb300/csrc/rlbm_o3.cuh",
              "paper_1703_04605_gb300/csrc/rlbm_fused.cuh",
              "paper_1703_04605_gb300/csrc/rlbm_internal.h", "paper_1703_04605_gb300/csrc/rlbm_stencils.h",
              "paper_1703_04605_gb300/csrc/rlbm_kernels.cuh"]
F3D_SOURCES = ["paper_1703_04605_gb300/csrc/rlbm_fused3d.cu", "paper_1703_04605_gb300/csrc/rlbm_fused.cuh",
               "paper_1703_04605_gb300/csrc/rlbm_internal.h", "paper_1703_04605_gb300/csrc/rlbm_stencils.h",
               "paper_1703_04605_gb300/csrc/rlbm_kernels.cuh"]
FUSED_SOURCES = ["paper_1703_04605_gb300/csrc/rlbm_fused.cuh", "paper_1703_04605_gb300/csrc/rlbm_internal.h",
                 "paper_1703_04605_gb300/csrc/rlbm_stencils.h", "paper_1703_04605_gb300/csrc/rlbm_kernels.cuh",
                 "paper_1703_04605_gb300/csrc/rlbm_fused_m1.cu"]

FUSED_E5_SOURCES = FUSED_SOURCES[:4] + ["paper_1703_04605_gb300/csrc/rlbm_fused_e5.cu"]


def profiled_traffic(profile, sources):
    """DRAM bytes per launch recorded in a committed ncu summary, or None when
    the kernel sources changed since the counters were taken.  The summary
    carries two lines 'traffic_bytes_per_launch: B' and 'source_hash: H'."""
    try:
        with open(os.path.join(ROOT, "profiles", profile)) as fh:
            txt = fh.read()
    except OSError:
        return None
    rec = {}
    for line in txt.splitlines():
        line = line.strip().strip("`")
        for key in ("traffic_bytes_per_launch", "source_hash"):
            if line.startswith(key + ":"):
                rec[key] = line.split(":", 1)[1].strip()
    if rec.get("source_hash") != _source_hash(sources) or "traffic_bytes_per_launch" not in rec:
        return None
    return float(rec["traffic_bytes_per_launch"])


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    vals = []
    side = 64
    for _ in range(args.warmup):
        cpu_baseline(seconds=1.0, side=side)
    for _ in range(args.steps):
        vals.append(cpu_baseline(seconds=5.0, side=side))
    v = float(np.mean([d["value"] for d in vals]))
    ms = float(np.mean([d["wall_ms"] for d in vals]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "dtype": "f64",
            "data": "synthetic", "scaling": "weak",
            "config": {"workload": WORKLOAD,
                       "sample": "each bench step is one bounded sample of the workload: %s (%.1f M site updates "
                                 "on average); value = the sum over the processes of their site-update rates"
                                 % (vals[-1]["sample"], float(np.mean([d["site_updates"] for d in vals])) / 1e6),
                       "ms_per_step": "wall time of one such sample (process start to last result), "
                                      "not a %dx%d step" % (N_SIDE, N_SIDE)},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": vals[-1]["cores"], "kind": "oracle",
                             "sample": vals[-1]["sample"]},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "vs_baseline": None}
    emit(line, rank)


def batch_error_vs_f64(specs, lats, nsteps, stream):
    """Untimed: every lattice of the batch advanced nsteps on the FP64 path
    from the same fields, against the batched FP32 result.  n and T: max
    relative error; u: max |du| over the larger of the lattice's largest FP64
    velocity and its initial velocity scale (u0 for a vortex, 0.05 for a
    tube, whose flow can die out within the run)."""
    from paper_1703_04605_gb300 import Lattice, stencils, workloads as W
    worst = {"n": 0.0, "T": 0.0, "u": 0.0}
    where = {}
    over = 0
    listed = []
    for i, (s, lat) in enumerate(zip(specs, lats)):
        groups, mu = stencils.choose(s["m"])
        f = W.batch_fields(s)
        got = lat.moments()
        with Lattice(groups, mu, s["tau"], s["L"], s["L"], dtype="f64", v0=lat.info()["v0"],
                     stream=stream.cuda_stream) as ref:
            ref.init(f["n"], f["ux"], f["uy"], f["T"])
            ref.step(nsteps)
            rm = ref.moments()
        scale = max(np.abs(rm["ux"]).max(), np.abs(rm["uy"]).max(), s.get("u0", 0.05))
        e = {"n": float(np.max(np.abs(got["n"] / rm["n"] - 1))),
             "T": float(np.max(np.abs(got["T"] / rm["T"] - 1))),
             "u": float(max(np.abs(got["ux"] - rm["ux"]).max(), np.abs(got["uy"] - rm["uy"]).max()) / scale)}
        if max(e.values()) > 1e-5:
            over += 1
            listed.append([i, s["kind"], s["L"], round(s["m"], 3), round(s["tau"], 3),
                           float("%.2g" % e["n"]), float("%.2g" % e["T"]), float("%.2g" % e["u"])])
        for k in worst:
            if e[k] > worst[k]:
                worst[k] = e[k]
                where[k] = {"lattice": i, "kind": s["kind"], "L": s["L"], "m": round(s["m"], 3),
                            "tau": round(s["tau"], 3)}
    return dict(worst, steps=nsteps, lattices=len(specs), lattices_over_1e_5=over, worst_at=where,
                over_1e_5=listed, against="FP64 path of this library, every lattice")


def run_batch(args):
    """256 independent periodic lattices (sides log-uniform in 64..1024, m/T
    log-uniform in 0.1..10 mapped onto the stencil library, tau in 0.6..1.5,
    Sod tubes and Taylor-Green vortices), FP32.  Batched arm: one batched call
    of K steps (replays of one CUDA graph holding every lattice's chain of
    step kernels) after a warm-up call that runs the autotuner.
    One-at-a-time arm: a second, freshly initialised copy of the
    same lattices, each advanced K steps by its own rlbm_step calls."""
    import torch
    from paper_1703_04605_gb300 import (Lattice, batch_engine, batch_step, build, set_batch_options, stencils,
                                        workloads as W)
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    build.build()
    stream = torch.cuda.Stream()
    specs = W.batch_specs(256)
    names = {1: "M1", 2: "G16", 3: "E5", 4: "S2"}

    def make_set():
        lats = []
        for s in specs:
            groups, mu = stencils.choose(s["m"])
            f = W.batch_fields(s)
            lat = Lattice(groups, mu, s["tau"], s["L"], s["L"], dtype="f32", v0=0.0, stream=stream.cuda_stream)
            lat.init(f["n"], f["ux"], f["uy"], f["T"])
            lats.append(lat)
        return lats

    def timed(fn, clk=None):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        if clk:
            clk.__enter__()
        e0.record(stream)
        fn()
        e1.record(stream)
        stream.synchronize()
        if clk:
            clk.__exit__(None, None, None)
        return e0.elapsed_time(e1)

    lats = make_set()
    sites = sum(s["L"] * s["L"] for s in specs)
    nbytes = sum(lat.info()["bytes_per_site"] * s["L"] * s["L"] for lat, s in zip(lats, specs))
    kinds = {}
    for lat in lats:
        k = names.get(lat.info()["kernel"], "?")
        kinds[k] = kinds.get(k, 0) + 1
    warm = max(args.warmup, 72)                # the first call also autotunes (66 steps)
    set_batch_options("auto")
    batch_step(lats, warm)
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    ms_b = timed(lambda: batch_step(lats, args.steps), clk)
    for lat in lats:
        lat.sync()                             # every lattice still physical
    tune = batch_engine(lats)
    check = None
    if args.check_f64:
        check = batch_error_vs_f64(specs, lats, warm + args.steps, stream)
    for lat in lats:
        lat.close()

    # the engine the autotuner did not pick, timed the same way
    other = "graph" if tune["engine"] == "persistent" else "persistent"
    set_batch_options(other)
    lats = make_set()
    batch_step(lats, warm)
    ms_o = timed(lambda: batch_step(lats, args.steps))
    other_tune = batch_engine(lats)
    for lat in lats:
        lat.sync()
        lat.close()
    set_batch_options("auto")

    lats = make_set()
    for lat in lats:
        lat.step(args.warmup)
    ms_1 = timed(lambda: [lat.step(args.steps) for lat in lats])
    for lat in lats:
        lat.sync()
        lat.close()

    value = sites * args.steps / (ms_b / 1e3) / 1e6
    peak = _peaks()
    achieved = nbytes / (ms_b / args.steps / 1e3) / 1e9
    line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
            "warmup": warm, "ms_per_step": ms_b / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch_256: 256 periodic lattices, sides log-uniform 64..1024, m/T log-uniform "
                                   "0.1..10 on the stencil library (clamped to 0.36..10), tau 0.6..1.5, half Sod "
                                   "(T in units of the mean of the pair, ratio capped at 2), half Taylor-Green",
                       "sites": sites, "lattices_per_stencil": kinds, "autotuned": tune,
                       "l2": "inputs larger than L2 (%.1f GB of populations)" % (nbytes / 1e9)},
            "one_at_a_time": {"MLUPS": sites * args.steps / (ms_1 / 1e3) / 1e6, "ms_per_step": ms_1 / args.steps},
            "batched_over_one_at_a_time": ms_1 / ms_b,
            "engines": {tune["engine"]: {"MLUPS": value, "ms_per_step": ms_b / args.steps, "chosen": True,
                                         "param": tune["param"]},
                        other: {"MLUPS": sites * args.steps / (ms_o / 1e3) / 1e6,
                                "ms_per_step": ms_o / args.steps, "chosen": False,
                                "param": other_tune["param"]}},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak[0], "unit": "GB/s",
                         "frac": achieved / peak[0], "peak_kind": peak[1], "traffic": None},
            "error_vs_f64": check,
            "gpu_launches": (tune["launches"] * args.steps if tune["engine"] == "graph" else tune["launches"]),
            "clocks": clk.summary()}
    emit(line, rank)


def run_blast(args):
    """The near-massless blast: 8192 x 8192, disc of radius 512 at T = 2 in a
    T = 1 background, tau = 0.7, BF16-deviation storage, m/T = 0.01 requested,
    run at m/T_R = 0.36 on the 133-velocity stencil (the smallest covered
    mass).  Reports MLUPS, the roofline, the equation of state of the
    read-out (e/(3nT) - 1 and its residual against (zeta/3) K1/K2) and the
    error against the FP32 path after the same steps."""
    import torch
    from scipy import special as sp
    from paper_1703_04605_gb300 import Lattice, build, workloads as W
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    build.build()
    st = W.STENCIL_E5
    # --side: a smaller copy with the disc radius scaled with the side (profiling)
    N = 8192 if args.side == N_SIDE else args.side
    R, tau = max(1, 512 * N // 8192), 0.7
    f = W.blast(N, R)
    stream = torch.cuda.Stream()
    sites = float(N) * N
    peak, peak_kind = _peaks()

    def run(dtype, clk=None):
        lat = Lattice(st["groups"], st["m"], tau, N, N, dtype=dtype, v0=st["v0"], stream=stream.cuda_stream)
        lat.init(f["n"], f["ux"], f["uy"], f["T"])
        lat.step(args.warmup)
        lat.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        if clk:
            clk.__enter__()
        e0.record(stream)
        lat.step(args.steps)
        e1.record(stream)
        stream.synchronize()
        if clk:
            clk.__exit__(None, None, None)
        lat.sync()
        info = lat.info()
        mom = lat.moments()
        lat.close()
        return e0.elapsed_time(e1) / args.steps, info, mom

    clk = ClockSampler(local)
    ms, info, mb = run("bf16dev", clk)
    z = st["m"] / mb["T"]
    dev = mb["e"] / (3 * mb["n"] * mb["T"]) - 1
    resid = np.abs(dev - z * (sp.kve(1, z) / sp.kve(2, z)) / 3)
    err = None
    if not args.no_extra:
        _, _, m32 = run("f32")
        umax = max(np.abs(m32["ux"]).max(), np.abs(m32["uy"]).max())
        err = {"n": float(np.max(np.abs(mb["n"] / m32["n"] - 1))), "T": float(np.max(np.abs(mb["T"] / m32["T"] - 1))),
               "u": float(max(np.abs(mb["ux"] - m32["ux"]).max(), np.abs(mb["uy"] - m32["uy"]).max()) / umax),
               "steps": args.warmup + args.steps,
               "against": "FP32 path (within 1e-4 of FP64 on the 1024^2, r=64 copy of this workload)"}
    achieved = info["bytes_per_site"] * sites / (ms / 1e3) / 1e9
    line = {"metric": METRIC, "value": sites / (ms / 1e3) / 1e6, "unit": "MLUPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "blast_%d: %dx%d periodic, disc r=%d at T=2 in T=1 (T_R = their mean), " % (N, N, N, R) +
                                   "n=1, u=0, tau=0.7, "
                                   "m/T=0.01 requested, run at m/T_R=0.36 (smallest covered), stencil "
                                   "G1,G14,G49,G51,G60,G70 (Q=73 folded), v0=0.1488232",
                       "sites": int(sites), "Q": info["Q"], "m_over_T_used": st["m"],
                       "l2": "inputs larger than L2"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "traffic": (profiled_traffic("fused_bf16_kernel_blast_8192.md", FUSED_E5_SOURCES)
                                     if N == 8192 and info["kernel"] == 3 else None),
                         "kernel": kernel_name("bf16dev", info["kernel"]),
                         "bytes_per_site": info["bytes_per_site"],
                         "frac_incl_coefficients": (info["bytes_per_site"] + info["extra_bytes_per_site"]) * sites
                         / (ms / 1e3) / 1e9 / peak},
            "eos": {"e_over_3nT_minus_1": [float(dev.min()), float(dev.max())],
                    "residual_vs_zeta_K1_over_3K2": float(resid.max())},
            "error_vs_f32": err, "gpu_launches": args.steps, "clocks": clk.summary()}
    emit(line, rank)


def run_random3d(args):
    """Native 3D: the random-flow recipe on a 256^3 periodic lattice with the
    unfolded stencil G5,G12,G14,G17,G21,G26 (Q = 96), m/T = 1, tau = 0.8, FP32
    storage (the compiled 3D kernel); FP64 timed on fewer steps; FP32 error
    against the FP64 path after the same steps; the oracle's 3D lattice on the
    host cores."""
    import torch
    from paper_1703_04605_gb300 import Lattice3D, build, workloads as W
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    build.build()
    st = W.STENCIL_M1
    N = 256 if args.side == N_SIDE else args.side
    f = W.random_flow3d(N)
    stream = torch.cuda.Stream()
    sites = float(N) ** 3
    peak, peak_kind = _peaks()

    def run(dtype, steps, clk=None):
        lat = Lattice3D(st["groups"], st["m"], TAU, N, N, N, dtype=dtype, v0=st["v0"], stream=stream.cuda_stream)
        lat.init(f["n"], f["ux"], f["uy"], f["uz"], f["T"])
        lat.step(args.warmup)
        lat.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        if clk:
            clk.__enter__()
        e0.record(stream)
        lat.step(steps)
        e1.record(stream)
        stream.synchronize()
        if clk:
            clk.__exit__(None, None, None)
        lat.sync()
        info = lat.info()
        mom = lat.moments()
        lat.close()
        return e0.elapsed_time(e1) / steps, info, mom

    clk = ClockSampler(local)
    ms, info, m32 = run("f32", args.steps, clk)
    k64 = max(5, args.steps // 10)
    ms64, info64, _ = run("f64", k64)
    err = None
    if not args.no_extra:
        # FP64 after the same number of steps as the FP32 run
        with Lattice3D(st["groups"], st["m"], TAU, N, N, N, dtype="f64", v0=st["v0"],
                       stream=stream.cuda_stream) as ref:
            ref.init(f["n"], f["ux"], f["uy"], f["uz"], f["T"])
            ref.step(args.warmup + args.steps)
            m64 = ref.moments()
        umax = max(np.abs(m64[k]).max() for k in ("ux", "uy", "uz"))
        err = {"n": float(np.max(np.abs(m32["n"] / m64["n"] - 1))),
               "T": float(np.max(np.abs(m32["T"] / m64["T"] - 1))),
               "u": float(max(np.abs(m32[k] - m64[k]).max() for k in ("ux", "uy", "uz")) / umax),
               "steps": args.warmup + args.steps, "against": "FP64 3D path (parity-tested vs the oracle)"}
    achieved = info["bytes_per_site"] * sites / (ms / 1e3) / 1e9
    line = {"metric": METRIC, "value": sites / (ms / 1e3) / 1e6, "unit": "MLUPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "random_flow3d_%d: %d^3 periodic random flow (n,T = 1+0.01 g, u = 0.05 g, " % (N, N) +
                                   "g Gaussian-smoothed width 8), m/T=1, tau=0.8, unfolded stencil "
                                   "G5,G12,G14,G17,G21,G26 (Q=96), v0=0.23342",
                       "sites": int(sites), "Q": info["Q"], "l2": "inputs larger than L2"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "traffic": (profiled_traffic("fused3d_kernel_random_flow3d_256.md", F3D_SOURCES)
                                     if N == 256 and info["kernel"] == 1 else None),
                         "kernel": ("fused3d_kernel<Stencil3Def<5,12,14,17,21,26>>" if info["kernel"] == 1
                                    else "step3d_kernel<float>"),
                         "bytes_per_site": info["bytes_per_site"]},
            "f64": {"MLUPS": sites / (ms64 / 1e3) / 1e6, "ms_per_step": ms64, "steps": k64,
                    "frac_hbm": info64["bytes_per_site"] * sites / (ms64 / 1e3) / 1e9 / peak},
            "error_vs_f64": err, "gpu_launches": args.steps, "clocks": clk.summary()}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline3d()
    emit(line, rank)


def run_third_order(args):
    """Third order: the random-flow recipe on a 4096^2 lattice (--side for a
    smaller one) at m/T_R = 5 with the eleven-group stencil
    G1,G2,G5,G6,G7,G9,G10,G11,G12,G13,G15 (Q = 100 folded), tau = 0.8, FP32
    storage; FP64 timed on fewer steps; FP32 error against the FP64 path after
    the same steps; the oracle's third-order lattice on the host cores."""
    import torch
    from paper_1703_04605_gb300 import Lattice, build, workloads as W
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    build.build()

    def barrier():
        if pg:
            pg.barrier()
        torch.cuda.synchronize()

    if args.mass is None:
        st = W.STENCIL_O3
    else:
        from paper_1703_04605_gb300 import quadrature_window, stencils
        groups, mb = stencils.choose(args.mass, order=3)
        lo, hi, _ = quadrature_window(groups, mb)
        st = dict(groups=groups, m=mb, v0=0.5 * (lo + hi))
    N = args.side
    f = W.random_flow(N)
    stream = torch.cuda.Stream()
    sites = float(N) ** 2
    peak, peak_kind = _peaks()

    def run(dtype, steps, clk=None):
        lat = Lattice(st["groups"], st["m"], TAU, N, N, dtype=dtype, v0=st["v0"], stream=stream.cuda_stream)
        lat.init(f["n"], f["ux"], f["uy"], f["T"])
        lat.step(args.warmup)
        lat.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        barrier()
        if clk:
            clk.__enter__()
        e0.record(stream)
        lat.step(steps)
        e1.record(stream)
        stream.synchronize()
        if clk:
            clk.__exit__(None, None, None)
        barrier()
        lat.sync()
        info = lat.info()
        mom = lat.moments()
        lat.close()
        return reduce_max(e0.elapsed_time(e1) / steps, pg, "cuda:%d" % local), info, mom

    clk = ClockSampler(local)
    ms, info, m32 = run("f32", args.steps, clk)
    k64 = max(5, args.steps // 10)
    ms64, info64, _ = run("f64", k64)
    err = None
    if not args.no_extra:
        with Lattice(st["groups"], st["m"], TAU, N, N, dtype="f64", v0=st["v0"], stream=stream.cuda_stream) as ref:
            ref.init(f["n"], f["ux"], f["uy"], f["T"])
            ref.step(args.warmup + args.steps)
            m64 = ref.moments()
        umax = max(np.abs(m64[k]).max() for k in ("ux", "uy"))
        err = {"n": float(np.max(np.abs(m32["n"] / m64["n"] - 1))),
               "T": float(np.max(np.abs(m32["T"] / m64["T"] - 1))),
               "u": float(max(np.abs(m32[k] - m64[k]).max() for k in ("ux", "uy")) / umax),
               "steps": args.warmup + args.steps, "against": "FP64 third-order path (parity-tested vs the oracle)"}
    achieved = info["bytes_per_site"] * sites / (ms / 1e3) / 1e9
    line = {"metric": METRIC, "value": ws * sites / (ms / 1e3) / 1e6, "unit": "MLUPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "random_flow_o3_%d: %d^2 periodic random flow (n,T = 1+0.01 g, u = 0.05 g, " % (N, N) +
                                   "g Gaussian-smoothed width 8), m/T_R=%g, tau=0.8, third-order stencil " % st["m"] +
                                   "G" + ",G".join(str(g) for g in st["groups"]) +
                                   " (Q=%d folded), v0=%.6g" % (info["Q"], st["v0"]),
                       "sites": int(sites), "Q": info["Q"], "order": info["order"], "l2": "inputs larger than L2"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "traffic": (profiled_traffic("fused_o3_kernel_random_flow_o3_4096.md", O3_SOURCES)
                                     if info["kernel"] == 5 and N == N_SIDE and args.mass is None else None),
                         "kernel": ("fused_o3_kernel<StencilO3Def<%s>>" % ",".join(str(g) for g in sorted(st["groups"]))
                                    if info["kernel"] >= 5 else "step_o3_kernel<float>"),
                         "bytes_per_site": info["bytes_per_site"]},
            "f64": {"MLUPS": sites / (ms64 / 1e3) / 1e6, "ms_per_step": ms64, "steps": k64,
                    "frac_hbm": info64["bytes_per_site"] * sites / (ms64 / 1e3) / 1e9 / peak,
                    "alu": fp64_alu(sites / (ms64 / 1e3) / 1e6,
                                    "step_o3_kernel/" + ",".join(str(g) for g in sorted(st["groups"])))},
            "error_vs_f64": err, "gpu_launches": args.steps, "clocks": clk.summary()}
    if not args.no_cpu_baseline and rank == 0:
        line["cpu_baseline"] = cpu_baseline_o3()
    emit(line, rank)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64", "bf16dev"])
    ap.add_argument("--side", type=int, default=N_SIDE,
                    help="random_flow: time a side x side crop of the 4096^2 field; random3d: a side^3 lattice "
                         "instead of 256^3; blast: a side^2 copy with the disc radius scaled "
                         "(profiling of small cases)")
    ap.add_argument("--mass", type=float, default=None,
                    help="third_order only: m/T_R of the stencil library's set to time (default: the m/T_R = 5 set)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the accuracy check and the other dtypes")
    ap.add_argument("--check-f64", action="store_true",
                    help="batch only: compare every lattice with the FP64 path after the run (untimed, minutes)")
    ap.add_argument("--workload", default="random_flow", choices=["random_flow", "batch", "blast", "random3d", "third_order"],
                    help="random_flow: the headline 4096^2 lattice; batch: 256 independent lattices; "
                         "blast: the 8192^2 near-massless blast in BF16-deviation storage; "
                         "random3d: a 256^3 lattice with the unfolded stencil")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "blast":
        return run_blast(args)
    if args.workload == "third_order":
        return run_third_order(args)
    if args.workload == "random3d":
        return run_random3d(args)

    import torch
    from paper_1703_04605_gb300 import Lattice, build, workloads as W

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    build.build()

    def barrier():
        if pg:
            pg.barrier()
        torch.cuda.synchronize()

    st = W.STENCIL_M1
    side = args.side
    f = W.random_flow(N_SIDE) if side == N_SIDE else W.random_flow_crop(N_SIDE, side)
    stream = torch.cuda.Stream()
    sites = float(side) * side
    peak, peak_kind = _peaks()

    def measure(dtype, steps, warmup, sample_clocks=False):
        lat = Lattice(st["groups"], st["m"], TAU, side, side, dtype=dtype, v0=st["v0"],
                      stream=stream.cuda_stream)
        info = lat.info()
        lat.init(f["n"], f["ux"], f["uy"], f["T"])
        lat.step(warmup)
        lat.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        clk = ClockSampler(local) if sample_clocks else None
        if clk:
            clk.__enter__()
        barrier()
        e0.record(stream)
        lat.step(steps)
        e1.record(stream)
        stream.synchronize()
        barrier()
        if clk:
            clk.__exit__(None, None, None)
        lat.sync()
        ms = reduce_max(e0.elapsed_time(e1), pg, "cuda")
        return lat, info, ms / steps, clk

    lat, info, ms_step, clk = measure(args.dtype, args.steps, args.warmup, sample_clocks=True)
    # a disqualified clock record on any rank: time the region once more
    rejected_clocks = None
    if reduce_max(float(clocks_rejected(clk.summary())), pg, "cuda") > 0:
        rejected_clocks = clk.summary()
        lat.close()
        lat, info, ms_step, clk = measure(args.dtype, args.steps, args.warmup, sample_clocks=True)
    value = whole_job_mlups(sites, ws, ms_step)
    bytes_launch = info["bytes_per_site"] * sites
    achieved = bytes_launch / (ms_step / 1e3) / 1e9

    def errs(got, rm):
        umax = max(np.abs(rm["ux"]).max(), np.abs(rm["uy"]).max())
        return {"n": float(np.max(np.abs(got["n"] / rm["n"] - 1))),
                "T": float(np.max(np.abs(got["T"] / rm["T"] - 1))),
                "u": float(max(np.abs(got["ux"] - rm["ux"]).max(), np.abs(got["uy"] - rm["uy"]).max()) / umax)}

    # accuracy against the FP64 path on the same input and step count (untimed),
    # and the other storage types on the same workload
    err = None
    by_dtype = {}
    if rank == 0 and not args.no_extra:
        got = lat.moments()
        nsteps = args.warmup + args.steps
        with Lattice(st["groups"], st["m"], TAU, side, side, dtype="f64", v0=st["v0"]) as ref:
            ref.init(f["n"], f["ux"], f["uy"], f["T"])
            ref.step(nsteps)
            rm = ref.moments()
        if args.dtype != "f64":
            err = dict(errs(got, rm), steps=nsteps, against="FP64 path of this library (parity-tested vs oracle)")
        for dt, k in (("bf16dev", args.steps), ("f64", 10), ("f32", args.steps)):
            if dt == args.dtype:
                continue
            l2, i2, m2, _ = measure(dt, k, args.warmup if dt != "f64" else 3)
            rec = {"MLUPS": sites / (m2 / 1e3) / 1e6, "ms_per_step": m2, "bytes_per_site": i2["bytes_per_site"],
                   "frac_hbm": i2["bytes_per_site"] * sites / (m2 / 1e3) / 1e9 / peak,
                   "frac_hbm_incl_extra": (i2["bytes_per_site"] + i2["extra_bytes_per_site"]) * sites
                   / (m2 / 1e3) / 1e9 / peak, "steps": k}
            if dt != "f64":
                l2.step(nsteps - (args.warmup + k))
                rec["error_vs_f64"] = dict(errs(l2.moments(), rm), steps=nsteps)
            else:
                rec["alu"] = fp64_alu(rec["MLUPS"], "step_f64_kernel/" + ",".join(str(g) for g in st["groups"]))
            by_dtype[dt] = rec
            l2.close()

    # end to end through the C ABI: pinned host fields in, K steps with the
    # status word read back every step, macroscopic fields out
    e2e = None
    if rank == 0:
        pin = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in f.items()}
        hostf = {k: v.numpy() for k, v in pin.items()}
        mask = 0x1F                                   # n, u_x, u_y, T, e
        pout = torch.empty(lat.moments_size(mask), dtype=torch.float64, pin_memory=True).numpy()
        ke = max(10, args.steps)          # the device-timed region's step count
        runs = []
        for _ in range(3):                # the host link and cores are shared: median of three
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lat.init(hostf["n"], hostf["ux"], hostf["uy"], hostf["T"])
            t1 = time.perf_counter()
            for _ in range(ke):
                lat.step(1)
                lat.sync()
            t2 = time.perf_counter()
            out = lat.moments(mask, out=pout)
            t3 = time.perf_counter()
            assert np.isfinite(out["n"]).all()
            runs.append((t3 - t0, t1 - t0, t2 - t1, t3 - t2))
        runs.sort()
        tt, ti, ts, tr = runs[1]
        e2e = {"value": sites * ke / tt / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": int(4 * 8 * sites / ke),
               "d2h_bytes_per_step": int(4 + 5 * 8 * sites / ke),
               "steps": ke,
               "breakdown_ms": {"init": ti * 1e3, "steps": ts * 1e3, "readout": tr * 1e3},
               "runs_ms": [round(r[0] * 1e3, 3) for r in runs],
               "region": "median of 3 runs of: rlbm_init from pinned host fields (upload, device check of "
                         "the copy, init kernel), %d steps with the status word read back after each, "
                         "rlbm_moments of n, u_x, u_y, T, e written by the read-out kernel into a pinned "
                         "host buffer" % ke}
    lat.close()

    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"bf16dev": "bf16"}.get(args.dtype, args.dtype), "data": "synthetic",
        "config": {"workload": WORKLOAD if side == N_SIDE else "%dx%d crop of: %s" % (side, side, WORKLOAD),
                   "sites": int(sites), "Q": info["Q"], "parallelism": "independent lattice per rank",
                   "l2": "inputs larger than L2 (%.1f GB of populations per step)" % (2 * bytes_launch / 2 / 1e9)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": (profiled_traffic("fused_f32_kernel_random_flow_4096.md", FUSED_SOURCES)
                                 if args.dtype == "f32" and side == N_SIDE else None),
                     "kernel": kernel_name(args.dtype, info["kernel"]), "peak_kind": peak_kind,
                     "bytes_per_site": info["bytes_per_site"]},
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
        "error_vs_f64": err,
        "by_dtype": by_dtype,
        "e2e": e2e,
    }
    if rejected_clocks:
        line["clocks"]["remeasured_after"] = rejected_clocks
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    emit(line, rank)
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
