#!/usr/bin/env python
"""Throughput of the full two-fluid FlIC/Godunov step on the 256^3 head-on
two-galaxy collision (synthetic, seeded), through libflic's C ABI.

One bench step = one full time step: FFT Poisson solve (Sec. 2.3), CFL step,
gas and Boltzmann-moment Eulerian + Lagrangian stages, kappa, energy balance and
diagnostics (Sec. 2.1-2.4).  The headline path is the float32-bulk ("mixed")
path; the float64 path is measured beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU runs (torchrun, one rank per GPU) are independent replicas of the
same workload (weak scaling; no data-path collective).  ``--impl reference``
times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cell-updates/s per full step at 256^3 (% HBM peak), mixed vs FP64, L1<=1e-4"
UNIT = "cell-updates/s"
# compulsory HBM bytes per cell of one launch: fields read (+ Phi) and written
ALG_WORDS = {"gas": 7 + 6, "bme": 17 + 16, "poisson": 2 + 1}


def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=300)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", choices=("ours", "reference"), default="ours")
    p.add_argument("--config", default="head-on-256",
                   choices=("head-on-256", "ensemble-64", "off-axis-512", "disc-128", "sphere-32"),
                   help="workload; the default is the headline 256^3 head-on collision")
    p.add_argument("--n", type=int, default=256, help="grid size of the head-on collision")
    p.add_argument("--precision", choices=("mixed", "fp64"), default="mixed")
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--fp64-steps", type=int, default=10)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-compare", action="store_true")
    p.add_argument("--compare-steps", type=int, default=10,
                   help="steps after which the mixed path is compared with the FP64 path (10 and 200 at 256^3)")
    p.add_argument("--tiles", default="auto",
                   help="launch shapes of the fluid kernels: 'auto' (the tuner times every compiled shape) or "
                        "'G,B' (indices of the gas and moment shapes, e.g. 0,0 for the defaults)")
    return p.parse_args(argv)


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def aggregate(local: dict, world: int) -> dict:
    """Max of the timed durations and sum of the cells over ranks (gloo, CPU)."""
    if world == 1:
        return {"max_s": local["seconds"], "cells": local["cells"]}
    import torch
    import torch.distributed as dist
    t = torch.tensor([local["seconds"]], dtype=torch.float64)
    c = torch.tensor([float(local["cells"])], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return {"max_s": float(t.item()), "cells": float(c.item())}


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.samples = []
        self.proc = None
        self.thread = None
        self.marks = {}

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "10"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.perf_counter(), line.strip()))

    def mark(self, name):
        self.marks[name] = time.perf_counter()

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        t0, t1 = self.marks.get("t0", 0.0), self.marks.get("t1", 1e30)
        inside = [s for t, s in self.samples if t0 <= t <= t1]
        window = "timed region"
        if len(inside) < 3:   # short timed region: widen to the warm-up + timed window
            w0 = self.marks.get("w0", t0)
            inside = [s for t, s in self.samples if w0 <= t <= t1]
            window = "warm-up + timed region"
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in inside:
            parts = [x.strip() for x in s.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "window": window}


# ---------------------------------------------------------------------------
# the oracle on the host cores
# ---------------------------------------------------------------------------
def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_full_steps(setup, nsteps: int, warmup: int = 0, workers=None):
    """Times full oracle steps of the whole grid on the host cores.

    Each step is the oracle's own step (whole-grid Poisson solve and CFL step,
    then the update slab by slab over ``workers`` processes, default all host
    cores: ``oracle.slab_pool``).  Returns per-step seconds and the worker count."""
    import oracle as O
    from oracle.slab_pool import SlabPool
    prm = O.Params(h=setup.h, gamma=setup.gamma)
    with SlabPool(setup.shape, workers=workers) as pool:
        pool.load(setup.state)
        for _ in range(warmup):
            pool.step(prm)
        secs = []
        for _ in range(nsteps):
            t = time.perf_counter()
            pool.step(prm)
            secs.append(time.perf_counter() - t)
        return secs, pool.workers


def oracle_one_core_sample(setup, budget_s: float):
    """The oracle on one core, on a bounded sample: the whole-grid Poisson solve
    and CFL step, plus the update of a slab of S z-planes (S sized to
    ``budget_s``), scaled to the full grid as t_poisson + t_cfl + N t_slab / S."""
    import oracle as O
    st = setup.state
    N = setup.shape[0]
    prm = O.Params(h=setup.h, gamma=setup.gamma)
    t = time.perf_counter()
    phi = O.solve_poisson(st, prm)
    tau = O.cfl_dt(st, prm)
    t_serial = time.perf_counter() - t
    t = time.perf_counter()
    O.advance_window(st, phi, tau, prm, zslab=(0, 2))
    t_plane = (time.perf_counter() - t) / 2
    S = int(max(2, min(N, (budget_s - t_serial) / max(t_plane, 1e-6))))
    t = time.perf_counter()
    O.advance_window(st, phi, tau, prm, zslab=(N // 2, N // 2 + S))
    t_slab = time.perf_counter() - t
    est = t_serial + N * t_slab / S
    return {"value": N ** 3 / est, "seconds_per_step_estimate": est, "planes": S}


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1311_0861_gb300 import inputs
    setup = inputs.head_on(args.n)
    # every step is a full oracle step of the whole grid on all host cores
    secs, workers = oracle_full_steps(setup, args.steps, warmup=args.warmup)
    total = float(np.sum(secs))
    value = args.n ** 3 * args.steps / total
    sample = (f"oracle (numpy FP64) on the {args.n}^3 head-on collision: {args.steps} full steps timed after "
              f"{args.warmup} untimed ones; each step is the whole-grid Poisson solve and CFL step in one process "
              f"and the update in z-slabs over {workers} worker processes; CPU: {cpu_model()}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"head-on two-galaxy collision {args.n}^3", "n": args.n,
                       "precision": "fp64 (CPU oracle)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model(), "host_cores": os.cpu_count()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def make_workload(args, rank):
    """(setup, poisson, name) of a single-grid configuration."""
    from paper_1311_0861_gb300 import inputs
    if args.config == "head-on-256":
        n = args.n
        setup = inputs.head_on(n) if rank == 0 else inputs.collision(n, seed=3 + 1000 * rank)
        return setup, "periodic", f"head-on two-galaxy collision {n}^3 (seeded synthetic)"
    if args.config == "off-axis-512":
        return inputs.off_axis(512), "isolated", "off-axis two-galaxy collision 512^3, isolated gravity"
    if args.config == "disc-128":
        return inputs.disc(128), "periodic", "rotating disc galaxy 128^3"
    if args.config == "sphere-32":
        return inputs.sphere(32), "periodic", "self-gravitating sphere 32^3"
    raise ValueError(args.config)


TRAFFIC_SOURCES = ("paper_1311_0861_gb300/csrc/flic_stencil.cuh", "paper_1311_0861_gb300/csrc/flic_stencil_launch.cuh",
                   "paper_1311_0861_gb300/csrc/flic_stencil_gas32.cu", "paper_1311_0861_gb300/csrc/flic_stencil_bme32.cu")


def traffic_key_hash() -> str:
    """Hash of the sources that define the float32 fluid kernels and their shapes."""
    import hashlib
    h = hashlib.sha256()
    for rel in TRAFFIC_SOURCES:
        h.update(open(os.path.join(ROOT, rel), "rb").read())
    return h.hexdigest()[:16]


def roofline_entry(kern, stage_ms, steps, cells, esz, precision, N, cand=None):
    avg_s = stage_ms[kern] / steps / 1e3
    alg_bytes = ALG_WORDS[kern] * esz * cells
    peak, peak_kind = peaks()
    achieved = alg_bytes / avg_s / 1e9
    r = {"bound": "hbm", "kernel": f"fluid_step_kernel<{'Bme' if kern == 'bme' else 'Gas'}Phys>",
         "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
         "peak_kind": peak_kind, "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": avg_s * 1e3}
    # ncu DRAM bytes per launch, recorded for a given kernel source and launch
    # shape: used only while the sources are unchanged
    traffic_file = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(traffic_file) and N is not None and cand is not None:
        try:
            rec = json.load(open(traffic_file))
            if rec.get("sha256_16") == traffic_key_hash():
                r["traffic"] = rec.get(f"{kern}-{precision}-{N}-shape{cand}")
        except Exception:
            pass
    return r


def run_single(args, rank, world, stream, clocks):
    import torch
    from paper_1311_0861_gb300 import flic, inputs
    setup, poisson, name = make_workload(args, rank)
    N = setup.shape[0]
    esz = 4 if args.precision == "mixed" else 8
    g = flic.Grid(N, precision=args.precision, gamma=setup.gamma, poisson=poisson, stream=stream.cuda_stream)
    g.set_state(setup.state)
    if args.tiles == "auto":
        tune = g.autotune(reps=5)
        chosen_by = ("cached launch-shape tuner" if tune["cached"] else
                     "launch-shape tuner (every compiled shape timed on this GPU)")
    else:
        gi, bi = (int(v) for v in args.tiles.split(","))
        g.set_tile_config(gi, bi)
        chosen_by = f"fixed on the command line ({args.tiles})"
    tiles = g.tile_config()["text"]
    launches = g.launches_per_step()
    clocks.start()
    time.sleep(0.2)
    clocks.mark("w0")
    g.run(args.warmup, sync=True)
    # ---- timed region: K steps, CUDA events per stage on the launching stream ----
    barrier(world)
    torch.cuda.synchronize()
    clocks.mark("t0")
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    stage_ms, _ = g.profile(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks.mark("t1")
    barrier(world)
    clocks.stop()
    elapsed_ms = ev0.elapsed_time(ev1)
    agg = aggregate({"seconds": elapsed_ms / 1e3, "cells": N ** 3 * args.steps}, world)
    value = agg["cells"] / agg["max_s"]
    d = g.step_diagnostics()
    kern = max(("gas", "bme"), key=lambda k: stage_ms[k])
    tcfg = g.tile_config()
    roofline = roofline_entry(kern, stage_ms, args.steps, N ** 3, esz, args.precision, N, cand=tcfg[kern])

    # ---- end to end through the public API with pinned host buffers ----
    e2e = None
    if args.e2e_steps > 0:
        host_in = torch.empty((22, N, N, N), dtype=torch.float64, pin_memory=True)
        host_out = torch.empty((22, N, N, N), dtype=torch.float64, pin_memory=True)
        host_in.numpy()[...] = inputs.stack(setup.state)
        ins = [host_in[i] for i in range(22)]
        outs = [host_out[i] for i in range(22)]
        barrier(world)
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(args.e2e_steps):
            g.set_state(ins)
            g.step(wait=False)
            g.get_state(outs)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t
        aggE = aggregate({"seconds": e2e_s, "cells": N ** 3 * args.e2e_steps}, world)
        e2e = {"value": aggE["cells"] / aggE["max_s"], "unit": UNIT,
               "h2d_bytes_per_step": 22 * 8 * N ** 3, "d2h_bytes_per_step": 22 * 8 * N ** 3,
               "steps": args.e2e_steps,
               "what": "per step: set_state from pinned host float64 arrays, step, get_state to pinned host"}
        del host_in, host_out

    # ---- float64 path and mixed-vs-float64 accuracy on the same input ----
    compare = None
    if not args.no_compare and args.precision == "mixed":
        K = args.compare_steps
        g.set_state(setup.state)
        m0 = g.diagnostics()
        g.run(K, sync=True)
        m1 = g.diagnostics()
        mixedK = g.get_state()
        g.close()
        g64 = flic.Grid(N, precision="fp64", gamma=setup.gamma, poisson=poisson, stream=stream.cuda_stream)
        g64.set_state(setup.state)
        g64.autotune(reps=2)
        g64.run(2, sync=True)
        st64, tot64 = g64.profile(args.fp64_steps)
        v64 = N ** 3 * args.fp64_steps / (tot64 / 1e3)
        g64.set_state(setup.state)
        d0 = g64.diagnostics()
        g64.run(K, sync=True)
        d1 = g64.diagnostics()
        fp64K = g64.get_state()
        g64.close()
        l1 = {f: float(np.sum(np.abs(mixedK[f] - fp64K[f])) / np.sum(np.abs(fp64K[f]))) for f in flic.FIELDS}

        def drift(a, b):
            e_a = a["ekin_gas"] + a["eint_gas"] + a["ekin_bme"] + a["etherm_bme"] + a["epot"]
            e_b = b["ekin_gas"] + b["eint_gas"] + b["ekin_bme"] + b["etherm_bme"] + b["epot"]
            return {"mass_gas": (b["mass_gas"] - a["mass_gas"]) / a["mass_gas"],
                    "mass_bme": (b["mass_bme"] - a["mass_bme"]) / a["mass_bme"],
                    "energy": (e_b - e_a) / abs(e_a)}
        compare = {"fp64_value": v64 * world, "fp64_ms_per_step": tot64 / args.fp64_steps,
                   "mixed_over_fp64": value / (v64 * world), "steps": K,
                   f"rel_l1_mixed_vs_fp64_after_{K}_steps": l1,
                   "drift_mixed": drift(m0, m1), "drift_fp64": drift(d0, d1)}
    else:
        g.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and poisson == "periodic":
        # two full oracle steps of the whole grid on all host cores (bounded: a
        # few seconds each at 256^3), and a one-core sample scaled to a step
        secs, workers = oracle_full_steps(setup, 2)
        one = oracle_one_core_sample(setup, 10.0)
        cpu = {"value": N ** 3 * len(secs) / float(np.sum(secs)), "unit": UNIT, "cores": workers, "kind": "oracle",
               "sample": (f"numpy FP64 oracle: {len(secs)} full {N}^3 steps (whole-grid Poisson solve and CFL "
                          f"step, then the update in z-slabs over {workers} worker processes), "
                          f"{float(np.mean(secs)):.2f} s per step"),
               "cpu_model": cpu_model(), "host_cores": os.cpu_count(),
               "one_core": {"value": one["value"], "cores": 1,
                            "sample": (f"whole-grid Poisson solve and CFL step + update of {one['planes']} of {N} "
                                       f"z-planes on one core, scaled to one full step")}}
    line = {"value": value, "ms_per_step": agg["max_s"] * 1e3 / args.steps,
            "config": {"workload": name, "n": N, "precision": args.precision,
                       "poisson": f"{poisson} FFT", "tiles": tiles, "tiles_chosen_by": chosen_by,
                       "l2": f"inputs larger than L2 (state {22 * esz * N ** 3 / 2 ** 30:.2f} GiB)"
                       if 22 * esz * N ** 3 > 2 ** 27 else "state smaller than L2; no flush",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches * args.steps,
            "stages_ms_per_step": {k: v / args.steps for k, v in stage_ms.items()},
            "compare": compare, "status": "ok" if not d["nonphysical"] else "nonphysical"}
    return line


def run_ensemble(args, rank, world, stream, clocks):
    """64 independent collisions of uneven sizes advanced by one batched launch per stage."""
    import torch
    from paper_1311_0861_gb300 import flic, inputs
    members = [inputs.ensemble_member(r) for r in range(64)]
    sizes = [m.shape[0] for m in members]
    cells = sum(n ** 3 for n in sizes)
    esz = 4 if args.precision == "mixed" else 8
    ens = flic.Ensemble(sizes, precision=args.precision, stream=stream.cuda_stream)
    for r, m in enumerate(members):
        ens.set_state(r, m.state)
    ens.autotune(reps=2)
    tiles = ens.tile_config()["text"]
    launches = ens.launches_per_step()
    clocks.start()
    time.sleep(0.2)
    clocks.mark("w0")
    ens.step(args.warmup)
    barrier(world)
    torch.cuda.synchronize()
    clocks.mark("t0")
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    stage_ms, _ = ens.profile(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks.mark("t1")
    barrier(world)
    clocks.stop()
    elapsed_ms = ev0.elapsed_time(ev1)
    agg = aggregate({"seconds": elapsed_ms / 1e3, "cells": cells * args.steps}, world)
    value = agg["cells"] / agg["max_s"]
    bad = any(ens.diagnostics(r)["nonphysical"] for r in range(len(sizes)))
    kern = max(("gas", "bme"), key=lambda k: stage_ms[k])
    roofline = roofline_entry(kern, stage_ms, args.steps, cells, esz, args.precision, None)
    # the same runs one after another, each a single-grid handle
    seq_ms, seq_steps = 0.0, max(1, min(args.steps, 10))
    for m in members:
        with flic.Grid(m.shape[0], precision=args.precision, gamma=m.gamma, stream=stream.cuda_stream) as g:
            g.set_state(m.state)
            g.autotune(reps=2)
            g.run(2, sync=True)
            _, tot = g.profile(seq_steps)
            seq_ms += tot
    seq_value = cells * seq_steps / (seq_ms / 1e3)
    # end to end: every run's state from host, one step, every state back
    e2e = None
    if args.e2e_steps > 0:
        # page-locked host copies of every run's state, filled before the timed region
        pin_in, pin_out = [], []
        for m, n in zip(members, sizes):
            a = torch.empty((22, n, n, n), dtype=torch.float64, pin_memory=True)
            a.numpy()[...] = inputs.stack(m.state)
            pin_in.append([a[i] for i in range(22)])
            b = torch.empty((22, n, n, n), dtype=torch.float64, pin_memory=True)
            pin_out.append([b[i] for i in range(22)])
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(args.e2e_steps):
            for r in range(len(sizes)):
                ens.set_state(r, pin_in[r])
            ens.step(1, sync=False)
            for r in range(len(sizes)):
                ens.get_state(r, pin_out[r])
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t
        e2e = {"value": cells * args.e2e_steps / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": 22 * 8 * cells, "d2h_bytes_per_step": 22 * 8 * cells,
               "steps": args.e2e_steps,
               "what": "per step: every run's state from pinned host float64 arrays, one step, every state back"}
        del pin_in, pin_out
    ens.close()
    counts = {n: sizes.count(n) for n in sorted(set(sizes))}
    return {"value": value, "ms_per_step": agg["max_s"] * 1e3 / args.steps,
            "config": {"workload": "64-run collision ensemble, uneven grids " +
                       ", ".join(f"{c}x{n}^3" for n, c in counts.items()),
                       "cells_per_step": cells, "precision": args.precision, "poisson": "periodic FFT",
                       "tiles": tiles, "tiles_chosen_by": "launch-shape tuner (every compiled shape and chunk cap "
                                                         "timed over the ensemble's work list on this GPU)",
                       "l2": f"state {22 * esz * cells / 2 ** 30:.2f} GiB",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": roofline, "cpu_baseline": None, "e2e": e2e,
            "gpu_launches": launches * args.steps,
            "stages_ms_per_step": {k: v / args.steps for k, v in stage_ms.items()},
            "compare": {"sequential_value": seq_value, "batched_over_sequential": value / seq_value},
            "status": "ok" if not bad else "nonphysical"}


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return reference_arm(args)
    rank, world, local = dist_env()
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    from paper_1311_0861_gb300 import flic
    if not os.path.exists(flic.LIB_PATH):
        from paper_1311_0861_gb300 import build
        build.build()
    stream = torch.cuda.Stream()
    clocks = ClockSampler(torch.cuda.current_device())
    if args.config == "ensemble-64":
        res = run_ensemble(args, rank, world, stream, clocks)
    else:
        res = run_single(args, rank, world, stream, clocks)
    if rank == 0:
        line = {"metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": res["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if args.precision == "mixed" else "f64", "data": "synthetic",
                "config": res["config"], "roofline": res["roofline"], "cpu_baseline": res["cpu_baseline"],
                "e2e": res["e2e"], "gpu_launches": res["gpu_launches"], "clocks": clocks.summary(),
                "stages_ms_per_step": res["stages_ms_per_step"], "compare": res["compare"],
                "status": res["status"]}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
