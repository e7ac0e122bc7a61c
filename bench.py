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


class ClockSampler:
    """nvidia-smi samples during the timed region (read-only queries)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(nm)
            except Exception:
                continue
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(seconds=12.0, side=96):
    """The FP64 oracle as it stands, one thread, on a side x side lattice drawn
    by the same generator (same smoothing, amplitudes and seed), for about
    `seconds` of CPU time."""
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
        "print(json.dumps({'steps': k, 'seconds': dt, 'mlups': %d * %d * k / dt / 1e6}))\n"
    ) % (ROOT, side, TAU, side, side, seconds, side, side)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        return {"value": None, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                "sample": "failed: " + r.stderr.strip().splitlines()[-1] if r.stderr else "failed"}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": d["mlups"], "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "sample": "%dx%d lattice of the same generator, %d steps in %.1f s wall, 1 thread" % (
                side, side, d["steps"], d["seconds"])}


def kernel_name(dtype, variant):
    stencil = {1: "5,12,14,17,21,26", 2: "1,2,3,4,5,6", 3: "1,14,49,51,60,70"}.get(variant)
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


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    vals = []
    side = 64
    for _ in range(args.warmup):
        cpu_baseline(seconds=2.0, side=side)
    for _ in range(args.steps):
        vals.append(cpu_baseline(seconds=6.0, side=side))
    v = float(np.mean([d["value"] for d in vals]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "f64",
            "data": "synthetic", "scaling": "weak",
            "config": {"workload": WORKLOAD, "sample": "%dx%d lattice of the same generator per step" % (side, side)},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                             "sample": vals[-1]["sample"]},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "vs_baseline": None}
    print(json.dumps(line), flush=True)


def run_batch(args):
    """256 independent periodic lattices (sides log-uniform in 64..1024, m/T
    log-uniform in 0.1..10 mapped onto the stencil library, tau in 0.6..1.5,
    Sod tubes and Taylor-Green vortices), FP32.  Batched arm: one batched call
    of K steps (graph-captured launches) after a warm-up call that runs the
    autotuner.  One-at-a-time arm: a second, freshly initialised copy of the
    same lattices, each advanced K steps by its own rlbm_step calls."""
    import torch
    from paper_1703_04605_gb300 import Lattice, batch_step, batch_tuning, build, stencils, workloads as W
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
    warm = max(args.warmup, 16)                # the first call also autotunes (12 steps)
    batch_step(lats, warm)
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    ms_b = timed(lambda: batch_step(lats, args.steps), clk)
    for lat in lats:
        lat.sync()                             # every lattice still physical
    tune = batch_tuning(lats)
    for lat in lats:
        lat.close()

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
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak[0], "unit": "GB/s",
                         "frac": achieved / peak[0], "peak_kind": peak[1], "traffic": None},
            "gpu_launches": tune["launches"] * args.steps,
            "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the accuracy check and the other dtypes")
    ap.add_argument("--workload", default="random_flow", choices=["random_flow", "batch"],
                    help="random_flow: the headline 4096^2 lattice; batch: 256 independent lattices")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)

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
    f = W.random_flow(N_SIDE)
    stream = torch.cuda.Stream()
    sites = float(N_SIDE) * N_SIDE
    peak, peak_kind = _peaks()

    def measure(dtype, steps, warmup, sample_clocks=False):
        lat = Lattice(st["groups"], st["m"], TAU, N_SIDE, N_SIDE, dtype=dtype, v0=st["v0"],
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
        ms = e0.elapsed_time(e1)
        if pg:
            t = torch.tensor([ms], device="cuda")
            pg.all_reduce(t, op=pg.ReduceOp.MAX)
            ms = float(t.item())
        return lat, info, ms / steps, clk

    lat, info, ms_step, clk = measure(args.dtype, args.steps, args.warmup, sample_clocks=True)
    value = ws * sites / (ms_step / 1e3) / 1e6
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
        with Lattice(st["groups"], st["m"], TAU, N_SIDE, N_SIDE, dtype="f64", v0=st["v0"]) as ref:
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
            by_dtype[dt] = rec
            l2.close()

    # end to end through the C ABI: pinned host fields in, K steps with the
    # status word read back every step, macroscopic fields out
    e2e = None
    if rank == 0:
        pin = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in f.items()}
        hostf = {k: v.numpy() for k, v in pin.items()}
        ke = max(10, args.steps // 4)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat.init(hostf["n"], hostf["ux"], hostf["uy"], hostf["T"])
        for _ in range(ke):
            lat.step(1)
            lat.sync()
        out = lat.moments()
        t1 = time.perf_counter()
        assert np.isfinite(out["n"]).all()
        e2e = {"value": sites * ke / (t1 - t0) / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": int(4 * 8 * sites / ke),
               "d2h_bytes_per_step": int(4 + 5 * 8 * sites / ke),
               "steps": ke}
    lat.close()

    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": WORKLOAD, "sites": int(sites), "Q": info["Q"], "parallelism": "independent lattice per rank",
                   "l2": "inputs larger than L2 (%.1f GB of populations per step)" % (2 * bytes_launch / 2 / 1e9)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": kernel_name(args.dtype, info["kernel"]), "peak_kind": peak_kind,
                     "bytes_per_site": info["bytes_per_site"]},
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
        "error_vs_f64": err,
        "by_dtype": by_dtype,
        "e2e": e2e,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
