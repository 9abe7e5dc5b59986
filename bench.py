#!/usr/bin/env python3
"""Benchmark: collision-handled steps/sec of the two-way method on GB300.

Workload (default): two stacked 256 x 256 cloth grids (2 m side, 1 cm apart,
the top one spinning at 6 rad/s with N(0, 0.3 m/s) noise), dt = 1/30 s, FP64.
A "step" is one full collision-handling call (Algorithm 1 from x^t and x~ to
x^{t+1}).  The chain of inputs (x^t, x~) is produced once, untimed, by running
the chain; the timed region then replays W warm-up and K timed steps with
their inputs already resident in HBM, flushing L2 between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun), every rank runs its own replica of the workload (the
method has no cross-scene exchange) and value = all ranks' steps / the
slowest rank's time.  --impl reference times the CPU FP64 oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "collision-handled steps/sec + contact pairs/sec (served/batched vs plain); p50/p99 step ms"
L2_FLUSH_BYTES = 256 << 20


def workload(name: str):
    from paper_2211_04045_gb300 import scenes
    if name == "two_cloths":
        return scenes.two_cloths(n=256, side=2.0, sep=0.01, omega=6.0, noise=0.3, seed=0), "two_cloths_256x256"
    if name == "cloth_sphere":
        return scenes.cloth_over_sphere(n=32), "cloth32_sphere3"
    if name == "tets":
        return scenes.tet_bodies(), "tets64x8"
    if name == "knot":
        return scenes.tube_knot(), "knot2x64x561"
    if name == "normal_flow":
        return scenes.normal_flow_torus(), "normal_flow_torus384x64"
    if name == "hair_sand":
        return scenes.hair_sand(), "hair10000x32_sand100000"
    if name == "rotating_sphere":
        return scenes.cloth_on_rotating_sphere(n=64, side=1.0, sphere_subdiv=4, sphere_r=0.3), \
            "cloth64_rotating_sphere4_friction"
    raise SystemExit(f"unknown config {name}")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def csrc_hash(files=None) -> str:
    """Hash of the CUDA sources (all of them, or the named files that define a
    kernel): a recorded ncu traffic figure is used only while it matches."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2211_04045_gb300", "csrc")
    for f in sorted(files or os.listdir(d)):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

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
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=2)
        except Exception:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) >= 9:
                for k, nm in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _ranks(dev):
    import torch
    d = torch.distributed
    return d if (d.is_available() and d.is_initialized() and d.get_world_size() > 1) else None


def slowest(x: float, dev) -> float:
    """The job's time is its slowest rank's: max over ranks (x itself on one rank)."""
    import torch
    d = _ranks(dev)
    if d is None:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    d.all_reduce(t, op=d.ReduceOp.MAX)
    return float(t.item())


def job_total(x: float, dev) -> float:
    """Units processed by the whole job: sum over ranks."""
    import torch
    d = _ranks(dev)
    if d is None:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    d.all_reduce(t, op=d.ReduceOp.SUM)
    return float(t.item())


def oracle_sample(sc, x_t, x_tilde, budget_s: float, solver: int = 0, step_rule: int = 0):
    """Times the oracle, as it stands, on the first iterations of one step.
    Returns (seconds per iteration, iterations timed, pairs evaluated)."""
    import oracle
    osc = oracle.OracleScene(sc)
    prm = oracle.params_for(sc, max_iters=0, solver=solver, step_rule=step_rule)
    t0 = time.perf_counter()
    _, st, _ = oracle.handle_step(osc, prm, x_t, x_tilde)
    t1 = time.perf_counter() - t0
    m = int(max(1, min(64, budget_s / max(t1, 1e-6))))
    if m > 1:
        prm = oracle.params_for(sc, max_iters=m - 1, solver=solver, step_rule=step_rule)
        t0 = time.perf_counter()
        _, st, _ = oracle.handle_step(osc, prm, x_t, x_tilde)
        t1 = time.perf_counter() - t0
    return t1 / st["iterations"], st["iterations"], st["pairs_evaluated"]


def _oracle_worker(job):
    cfg, x_t, x_tilde, budget_s, solver, step_rule = job
    sc, _ = workload(cfg)
    return oracle_sample(sc, x_t, x_tilde, budget_s, solver, step_rule)


def oracle_samples(cfg, x_t, x_tilde, budget_s: float, cores: int, solver: int = 0, step_rule: int = 0, pool=None):
    """oracle_sample on `cores` host cores at once: one single-threaded oracle
    per core (processes started by spawn), each on the same bounded sample of
    the workload, as a CPU serving independent requests would run.  Returns
    the list of (seconds per iteration, iterations timed, pairs evaluated)."""
    if cores <= 1 and pool is None:
        sc, _ = workload(cfg)
        return [oracle_sample(sc, x_t, x_tilde, budget_s, solver, step_rule)]
    jobs = [(cfg, x_t, x_tilde, budget_s, solver, step_rule)] * cores
    if pool is not None:
        return pool.map(_oracle_worker, jobs)
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(cores) as p:
        return p.map(_oracle_worker, jobs)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def serving_mix():
    """Resident scenes of the serving workload: the paper's scene kinds (cloth
    over a sphere, two cloth layers, volumetric bodies, tightening tubes,
    hair and sand), each at a small and a large size, from about 2K to 150K
    triangles (hair and sand: primitives)."""
    from paper_2211_04045_gb300 import scenes
    return [scenes.cloth_over_sphere(n=24, side=0.5, sphere_subdiv=3, sphere_r=0.15, noise=0.5, seed=11),
            scenes.cloth_over_sphere(n=256, side=1.5, sphere_subdiv=4, sphere_r=0.4, noise=0.5, seed=12),
            scenes.two_cloths(n=32, side=0.25, sep=0.01, omega=6.0, noise=0.3, seed=13),
            scenes.two_cloths(n=190, side=1.5, sep=0.01, omega=6.0, noise=0.3, seed=14),
            scenes.tet_bodies(n_bodies=8, n=6, side=0.2, box=0.8, seed=15),
            scenes.tet_bodies(n_bodies=125, n=10, side=0.2, box=1.75, seed=16),
            scenes.tube_knot(around=16, rings=65, r=0.004, helix_r=0.0055, pitch=0.03, ring_dz=0.002),
            scenes.tube_knot(),
            scenes.hair_sand(n_strands=100, segs=16, n_points=1000, grain_r=0.002, bowl_r=0.15, bowl_subdiv=3,
                             seg_len=0.005, seed=17),
            scenes.hair_sand(n_strands=4000, segs=32, n_points=40000, grain_r=0.002, bowl_r=0.4, bowl_subdiv=5,
                             seed=18)]


def prims(sc):
    return int(len(sc.tris) + len(sc.edges) + len(sc.points)) if len(sc.tris) < 1000 else int(len(sc.tris))


def smooth_displacement(sc, rng):
    """A displacement of every movable vertex by a random smooth field: per
    axis a sinusoid of x with a random direction, wavelength between a third
    of the scene's extent and its extent, and phase, with an amplitude drawn
    log-uniformly from 0.05 to 1 mm (a time step of 1/100 s at up to 10 cm/s)."""
    x = sc.x0
    ext = float(np.ptp(x, axis=0).max())
    amp = float(np.exp(rng.uniform(np.log(5e-5), np.log(1e-3))))
    d = np.zeros_like(x)
    for a in range(3):
        k = rng.normal(0.0, 1.0, 3)
        k *= rng.uniform(1.0, 3.0) / (np.linalg.norm(k) * ext)
        d[:, a] = amp * np.sin(2.0 * np.pi * (x @ k) + rng.uniform(0.0, 2.0 * np.pi))
    return d * (sc.inv_mass > 0)[:, None]


def serve_compare(dev, requests: int, rate: float, max_active: int, precisions=("mixed", "fp64"), group: int = 8):
    """Poisson request stream served with continuous batching, against the
    same requests run one at a time in plain FP64 (each on its own resident
    scene).  Returns the comparison as a dict."""
    import torch
    from paper_2211_04045_gb300 import cch, scenes
    scs = serving_mix()
    rng = np.random.default_rng(0)
    N = requests
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=N))
    which = rng.integers(0, len(scs), size=N)
    inputs = []
    for i in range(N):
        # a seeded random (x^t, x~) pair: the scene's start and a target
        # moved by a smooth random displacement field (one time step of a
        # simulator: neighbouring vertices move alike)
        sc = scs[which[i]]
        x = sc.x0
        xt = x + smooth_displacement(sc, rng)
        inputs.append((torch.tensor(x, device=dev), torch.tensor(xt, device=dev)))
    out = {"requests": N, "rate_per_s": rate, "max_active": max_active, "budget_bytes": 80 << 30,
           "scene_prims": [prims(sc) for sc in scs]}
    # plain: one request at a time, FP64, one resident scene per kind
    # every scene with its own physical parameters (Table 2 values, or the
    # scene's: the tubes take delta = 0.5 mm)
    plain = [cch.Scene(sc, cch.params_for(sc, iters_per_launch=group)) for sc in scs]
    for g, sc in zip(plain, scs):  # warm-up: builds and graph capture
        x, xt, _ = scenes.initial(sc)
        g.step(torch.tensor(x, device=dev), torch.tensor(xt, device=dev))
    torch.cuda.synchronize()
    # the same Poisson stream served one request at a time, in arrival order:
    # a request waits for its arrival and for the one before it; latency runs
    # from arrival to completion, as for the served requests
    t0 = time.perf_counter()
    plain_lat, plain_svc, plain_out, plain_it = [], [], [], []
    for i in range(N):
        delay = arrivals[i] - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        a = time.perf_counter()
        o, st = plain[which[i]].step(inputs[i][0], inputs[i][1])
        b = time.perf_counter()
        plain_svc.append(1000.0 * (b - a))
        plain_lat.append(1000.0 * (b - t0 - arrivals[i]))
        plain_out.append(o)
        plain_it.append(st["iterations"])
    plain_s = time.perf_counter() - t0
    for g in plain:
        g.close()
    plain_svc, plain_it = np.array(plain_svc), np.array(plain_it)
    plain_cap = N / (float(np.sum(plain_svc)) / 1000.0)
    out["plain_fp64"] = {"value": N / plain_s, "unit": "steps/s", "p50_ms": float(np.percentile(plain_lat, 50)),
                         "p99_ms": float(np.percentile(plain_lat, 99)), "capacity": plain_cap,
                         "service_p50_ms": float(np.percentile(plain_svc, 50)),
                         "per_scene": [{"requests": int(np.sum(which == k)),
                                        "mean_ms": round(float(np.mean(plain_svc[which == k])), 2) if np.any(which == k) else None,
                                        "max_iterations": int(np.max(plain_it[which == k])) if np.any(which == k) else None}
                                       for k in range(len(scs))]}
    for prec in precisions:
        prm = cch.params_for(scs[0], precision=1 if prec == "mixed" else 0, iters_per_launch=group)
        sv = cch.Server(80 << 30, prm, max_active=max_active)
        ids = [sv.add_scene(sc, cch.params_for(sc)) for sc in scs]
        for k, sc in enumerate(scs):  # one warm request per scene (pool build, graph capture)
            x, xt, _ = scenes.initial(sc)
            o = torch.empty((sc.n_verts, 3), dtype=torch.float64, device=dev)
            sv.wait(sv.submit(ids[k], torch.tensor(x, device=dev), torch.tensor(xt, device=dev), o))
        outs = [torch.empty((scs[which[i]].n_verts, 3), dtype=torch.float64, device=dev) for i in range(N)]
        tickets = []
        t0 = time.perf_counter()
        for i in range(N):
            delay = arrivals[i] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            tickets.append(sv.submit(ids[which[i]], inputs[i][0], inputs[i][1], outs[i]))
        lat, iters = [], []
        for tk in tickets:
            st, ms = sv.wait(tk)
            lat.append(ms)
            iters.append(st["iterations"])
        served_s = time.perf_counter() - t0
        # FP64 served results equal the plain ones bitwise; mixed: max deviation
        dev_max = max(float((o - p).abs().max().item()) for o, p in zip(outs, plain_out))
        # capacity: the whole stream submitted at once
        t0 = time.perf_counter()
        tickets = [sv.submit(ids[which[i]], inputs[i][0], inputs[i][1], outs[i]) for i in range(N)]
        for tk in tickets:
            sv.wait(tk)
        cap = N / (time.perf_counter() - t0)
        sv.close()
        out[f"served_{prec}"] = {"value": N / served_s, "unit": "steps/s", "p50_ms": float(np.percentile(lat, 50)),
                                 "p99_ms": float(np.percentile(lat, 99)), "speedup_vs_plain": plain_s / served_s,
                                 "capacity": cap, "capacity_vs_plain": cap / plain_cap,
                                 "iterations_per_step": float(np.mean(iters)),
                                 "max_abs_diff_vs_plain_m": dev_max}
    return out


def run_serving(args):
    """The serving workload on its own: one JSON line."""
    import torch
    dev = torch.device("cuda:0")
    r = serve_compare(dev, args.requests, args.rate, args.max_active, precisions=(args.precision,),
                      group=args.serve_group)
    srv = r[f"served_{args.precision}"]
    out = {"metric": METRIC, "value": srv["value"], "unit": "steps/s", "n_gpus": 1, "steps": args.requests,
           "warmup": len(r["scene_prims"]), "ms_per_step": 1000.0 / srv["value"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
           "config": {"workload": f"serving_mix_{args.precision}", "requests": args.requests,
                      "rate_per_s": args.rate, "scene_prims": r["scene_prims"], "max_active": args.max_active,
                      "budget_bytes": 80 << 30},
           "p50_ms": srv["p50_ms"], "p99_ms": srv["p99_ms"], "plain_fp64": r["plain_fp64"],
           "speedup_vs_plain": srv["speedup_vs_plain"], "iterations_per_step": srv["iterations_per_step"]}
    print(json.dumps(out), flush=True)
    return 0


def batch_mix(n: int = 64, seed: int = 0):
    """64 uneven volumetric scenes: one tet cube each (5 to 8 vertices per
    side, 0.2 m, random orientation, N(0, 2 m/s) velocity and N(0, 4 rad/s)
    spin), the bodies of the 64-body workload as scenes of their own."""
    from paper_2211_04045_gb300 import scenes
    rng = np.random.default_rng(seed)
    return [scenes.tet_bodies(n_bodies=1, n=int(rng.integers(5, 9)), side=0.2, box=0.4, seed=1000 + b)
            for b in range(n)]


def batch_compare(dev, stream, n_scenes: int, reps: int, flush):
    """n_scenes uneven scenes handled in one batched launch sequence against
    the plain loop of one call per scene (FP64; each scene's result is the
    same in both, bitwise)."""
    import torch
    from paper_2211_04045_gb300 import cch, scenes
    scs = batch_mix(n_scenes)
    xs = [[torch.tensor(a, device=dev) for a in scenes.initial(sc)[:2]] for sc in scs]
    prm = cch.params_for(scs[0])
    batch = cch.Scene(scs, prm, stream=stream.cuda_stream)
    singles = [cch.Scene(sc, prm, stream=stream.cuda_stream) for sc in scs]
    outs_b, _ = batch.batch_step([a for a, _ in xs], [b for _, b in xs])  # warm-up
    outs_s = [g.step(a, b)[0] for g, (a, b) in zip(singles, xs)]
    same = all(torch.equal(p, q) for p, q in zip(outs_b, outs_s))
    torch.cuda.synchronize(dev)
    tb = []
    for _ in range(reps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        _, sts = batch.batch_step([a for a, _ in xs], [b for _, b in xs], outs_b)
        tb.append(time.perf_counter() - t0)
    ts = []
    for _ in range(reps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for g, (a, b), o in zip(singles, xs, outs_s):
            g.step(a, b, out=o)
        ts.append(time.perf_counter() - t0)
    batch.close()
    for g in singles:
        g.close()
    its = [s["iterations"] for s in sts]
    return {"scenes": n_scenes, "verts": [sc.n_verts for sc in scs][:8] + ["..."],
            "batched": {"value": n_scenes / min(tb), "unit": "scene-steps/s", "ms": 1000.0 * min(tb)},
            "plain_loop": {"value": n_scenes / min(ts), "unit": "scene-steps/s", "ms": 1000.0 * min(ts)},
            "speedup": min(ts) / min(tb), "same_results": bool(same),
            "iterations_min_max": [int(min(its)), int(max(its))]}


def sec8d_bytes(st, n, T, E, NL, fp=8):
    """Algorithmic bytes of one step by kernel group, counted as the method
    must move them (FP64 sizes unless fp = 4 for the mixed projection):
    forward step 96 N per iteration plus 8 N for D_i; distance refresh
    16 |P| + 24 N_P per refresh iteration (N_P distinct vertices of P); a
    search 24 N + 12 T + 8 E + 16 |P|; contacts |A| (16 + 12 fp + fp) +
    9 fp N_A (x and y read, y written, once per distinct contact vertex);
    edge-length constraints 8 C_e + 6 fp N per sweep; the colouring reads 16
    bytes of vertex ids and writes a 4-byte colour per contact."""
    it, se = st["iterations"], st["searches"]
    P, A = st["pairs_evaluated"], st["active_contacts"]
    NA, NP = st["contact_vertices"], st["pair_vertices"]
    per_search_pairs = P / max(1, it)
    sweeps = st.get("gs_sweeps", 1)
    return {
        "forward": it * 104.0 * n,
        "refresh": 16.0 * P * (it - se) / max(1, it) + 24.0 * NP * (it - se) / max(1, it),
        "search": se * (24.0 * n + 12.0 * T + 8.0 * E + 16.0 * per_search_pairs),
        "assemble": A * (16.0 + 12 * fp + fp) + 3 * fp * NA,
        "sweep": sweeps * (A * (16.0 + 12 * fp + fp) + 9 * fp * NA + it * (8.0 * NL + 6 * fp * n)),
        "colour": A * 20.0,
    }


def chain_target(sc, dyn, g):
    """x~ of the next step of the chain on the GPU: the stand-in dynamics, or
    the library's pre-pass kernels for the normal-flow and friction
    workloads."""
    def target(x, v):
        if sc.flow is not None:
            f = sc.flow
            return g.normal_flow_target(x, f["beta"], f["alpha"], f["sign"], f["iters"])
        if sc.friction is not None:
            f = sc.friction
            y = dyn.predict_frictionless(x, v)
            return g.friction_filter(x, y, f["mu"], f["reach"], f["sep"], out=y)
        return dyn.predict(x, v)
    return target


def run_reference(args):
    """CPU oracle as the reference arm (rank 0 only)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2211_04045_gb300 import scenes
    sc, wname = workload(args.config)
    x, xt, v = scenes.initial(sc)
    L = int(dict(sc.params).get("max_iters", 2048))
    cores = args.ref_cores or host_cores()
    per_step = []
    budget = max(2.0, args.ref_budget / max(1, args.steps + args.warmup))
    pool = None
    if cores > 1:
        import multiprocessing as mp
        pool = mp.get_context("spawn").Pool(cores)
    try:
        for s in range(args.warmup + args.steps):
            res = oracle_samples(args.config, x, xt, budget, cores, pool=pool)
            if s >= args.warmup:
                # the cores' steps run side by side: steps per second add up
                per_step.append(1.0 / sum(1.0 / (spi * (L + 1)) for spi, _, _ in res))
    finally:
        if pool is not None:
            pool.close()
            pool.join()
    tot = float(np.sum(per_step))
    val = len(per_step) / tot
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "steps/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * tot / len(per_step),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"{wname}_fp64", "verts": sc.n_verts, "tris": len(sc.tris), "dt": sc.dt},
           "cpu_baseline": {"value": val, "unit": "steps/s", "cores": cores, "kind": "oracle",
                            "sample": f"per step and core ({cores} single-threaded oracles side by side, their "
                                      "steps per second added): the oracle's first iterations of the workload's "
                                      f"first step (about {budget:.0f} s), seconds per iteration times L + 1 = "
                                      f"{L + 1} iterations, "
                                      "the count every step of this chain takes (it runs to L on the GPU, and the "
                                      "oracle takes the GPU's iteration count on every scene the parity tests "
                                      "compare)"},
           "e2e": {"value": val, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def variant_compare(sc, kw, inputs, refs, dev, stream, flush, tune_iters, log, name):
    """A variant of the step (mixed precision: FP32 distances and projection,
    FP64 forward step, CCD and acceptance; or the greedy colouring) timed on
    the same step inputs as the headline run; its position difference from
    the headline results is reported per step."""
    import torch
    from paper_2211_04045_gb300 import cch
    g = cch.Scene(sc, cch.params_for(sc, accept_check=1, **kw), stream=stream.cuda_stream)
    g.step(inputs[0][0], inputs[0][1])  # warm-up: graph capture
    if tune_iters:
        g.autotune(inputs[0][0], inputs[0][1], probe_iters=tune_iters)
    ms, errs, its, isect, unc = [], [], [], 0, 0
    for (x, xt), ref in zip(inputs, refs):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out, st = g.step(x, xt)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms.append(e0.elapsed_time(e1))
        errs.append(float(torch.linalg.norm(out - ref, dim=1).max().item()))
        its.append(st["iterations"])
        isect += st["intersections"]
        unc += st["uncertain"]
    g.close()
    log(f"{name}: {', '.join(f'{m:.0f} ms' for m in ms)}; max |x - x_headline| per step "
        + ", ".join(f"{e:.2e}" for e in errs))
    return {"value": len(ms) / (sum(ms) / 1000.0), "unit": "steps/s", "steps": len(ms),
            "p50_ms": float(np.percentile(ms, 50)), "iterations_per_step": float(np.mean(its)),
            "max_abs_diff_vs_headline_m": max(errs), "intersections": int(isect), "uncertain": int(unc)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="two_cloths")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--solver", default="gs", choices=["gs", "jacobi"],
                    help="backward step: projected Gauss-Seidel (the paper's) or projected Jacobi (omega 0.5)")
    ap.add_argument("--cpu-budget", type=float, default=15.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--ref-budget", type=float, default=60.0, help="seconds of oracle work for --impl reference")
    ap.add_argument("--ref-cores", type=int, default=0,
                    help="host cores of the oracle runs (reference arm, cpu_baseline); 0: all")
    ap.add_argument("--gap", action="store_true", help="gap contact constraints instead of the volume-based ones")
    ap.add_argument("--colouring", type=int, default=1, choices=[0, 1],
                    help="randomized colouring of the Gauss-Seidel sweep: 1 level (default), 0 greedy")
    ap.add_argument("--step-rule", default="distance", choices=["distance", "ccd"],
                    help="forward step size: the distance bound (Eq. forward2) or the CCD-based scheme of Sec. 5.1")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the launch-configuration autotuner")
    ap.add_argument("--tune-iters", type=int, default=48, help="iterations of the autotuner's probe step")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the comparisons (mixed precision, batched, served) after the headline")
    ap.add_argument("--mixed-steps", type=int, default=3, help="timed steps of the mixed-precision comparison")
    ap.add_argument("--batch-scenes", type=int, default=64, help="scenes of the batching comparison")
    ap.add_argument("--requests", type=int, default=None, help="serving: requests in the stream (512)")
    ap.add_argument("--rate", type=float, default=200.0, help="serving: mean arrivals per second")
    ap.add_argument("--max-active", type=int, default=16, help="serving: requests batched at once")
    ap.add_argument("--serve-group", type=int, default=8, help="serving: iterations per graph launch (both arms)")
    ap.add_argument("--ncu-warm", type=int, default=0, help="full chain steps before the --ncu-case step")
    ap.add_argument("--ncu-case", type=int, default=0,
                    help="profiling aid: run one step of the workload capped at this many iterations and exit "
                         "(prints no bench line)")
    args = ap.parse_args()
    if args.requests is None:
        args.requests = 512
    if args.impl == "reference":
        return run_reference(args)
    if args.config == "serve":
        return run_serving(args)

    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)

    from paper_2211_04045_gb300 import cch, scenes
    sc, wname = workload(args.config)
    gs = args.solver == "gs"
    prm = cch.params_for(sc, precision=1 if args.precision == "mixed" else 0,
                         solver=0 if gs else 1, constraint_form=1 if args.gap else 0,
                         step_rule=1 if args.step_rule == "ccd" else 0, accept_check=1, colouring=args.colouring)
    if args.ncu_case:
        x0, xt0, v0 = scenes.initial(sc)
        x, xt, v = (torch.tensor(a, device=dev) for a in (x0, xt0, v0))
        if args.ncu_warm:
            dyn = scenes.TorchDynamics(sc, dev)
            gw = cch.Scene(sc, prm)
            target = chain_target(sc, dyn, gw)
            for _ in range(args.ncu_warm):
                out, _ = gw.step(x, xt)
                v = dyn.next_velocity(out, x)
                x, xt = out, target(out, v)
            gw.close()
        prm.max_iters = args.ncu_case
        g = cch.Scene(sc, prm)
        torch.cuda.synchronize(dev)
        torch.cuda.profiler.start()  # captures with --profile-from-start off cover this step only
        _, st = g.step(x, xt)
        torch.cuda.synchronize(dev)
        torch.cuda.profiler.stop()
        torch.cuda.synchronize(dev)
        sys.stderr.write(f"[bench] ncu case: {st['iterations']} iterations, {st['kernel_launches']} launches, "
                         f"{st['pairs_evaluated'] / st['iterations']:.0f} pairs/iter, "
                         f"{st['active_contacts'] / st['iterations']:.0f} contacts/iter, "
                         f"{st['max_vertex_contacts']} contacts at one vertex, {st['contact_colours']} contact "
                         f"and {st['edge_colours']} edge colours\n")
        g.close()
        return 0
    stream = torch.cuda.current_stream(dev)
    gpu = cch.Scene(sc, prm, stream=stream.cuda_stream)
    n = sc.n_verts
    W, K = args.warmup, args.steps

    def log(msg):
        if rank == 0:
            sys.stderr.write(f"[bench] {msg}\n")
            sys.stderr.flush()

    # ---- warm-up: the first W steps of the chain ----
    dyn = scenes.TorchDynamics(sc, dev)
    target = chain_target(sc, dyn, gpu)
    x0, xt0, v0 = scenes.initial(sc)
    x = torch.tensor(x0, device=dev)
    xt = torch.tensor(xt0, device=dev)
    v = torch.tensor(v0, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    outbuf = torch.empty((n, 3), dtype=torch.float64, device=dev)
    for s in range(W):
        t0 = time.perf_counter()
        _, st = gpu.step(x, xt, out=outbuf)
        v = dyn.next_velocity(outbuf, x)
        x = outbuf.clone()
        xt = target(x, v)
        log(f"warm-up step {s}: {st['iterations']} iterations, {time.perf_counter() - t0:.2f} s")
    torch.cuda.synchronize(dev)
    timed_inputs = (x.clone(), xt.clone())
    tune = None
    if not args.no_tune:
        tune = gpu.autotune(x, xt, probe_iters=args.tune_iters)
        log(f"autotune: {tune}")

    # ---- timed region: K further steps of the chain, each with the exact
    # acceptance test of x^{t+1} ----
    keep = 0 if args.no_compare else max(0, min(args.mixed_steps, K))
    kept_in, kept_out = [], []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    clocks = ClockSampler(torch.cuda.current_device() if world == 1 else local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    stats = []
    for k in range(K):
        flush.zero_()
        if k < keep:
            kept_in.append((x.clone(), xt.clone()))
        ev[k][0].record(stream)
        _, st = gpu.step(x, xt, out=outbuf)
        ev[k][1].record(stream)
        stats.append(st)
        if k < keep:
            kept_out.append(outbuf.clone())
        v = dyn.next_velocity(outbuf, x)
        x = outbuf.clone()
        xt = target(x, v)
    t_end.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    step_ms = np.array([a.elapsed_time(b) for a, b in ev])
    log(f"timed {K} steps in {total_ms / 1000:.2f} s: " + ", ".join(f"{m:.0f} ms" for m in step_ms))
    log("per step: iterations " + ", ".join(str(s["iterations"]) for s in stats) + "; final ||r|| "
        + ", ".join(f"{s['final_r_inf']:.3g}" for s in stats) + "; frozen "
        + ", ".join(str(s["frozen_vertices"]) for s in stats) + "; searches "
        + ", ".join(str(s["searches"]) for s in stats))
    total_ms = slowest(total_ms, dev)

    iters = np.array([s["iterations"] for s in stats])
    pairs = job_total(float(np.sum([s["pairs_evaluated"] for s in stats])), dev)
    launches = int(job_total(float(np.sum([s["kernel_launches"] for s in stats])), dev))
    steps_per_s = job_total(float(K), dev) / (total_ms / 1000.0)

    # ---- per-kernel timing (events on the launching stream, no graphs) ----
    gpu.set_profiling(True)
    flush.zero_()
    prof_out, pst = gpu.step(timed_inputs[0], timed_inputs[1])
    prof = gpu.profile()
    gpu.set_profiling(False)
    deterministic = pst["iterations"] == stats[0]["iterations"] and pst["pairs_evaluated"] == stats[0]["pairs_evaluated"]
    log(f"profiled one step: {pst['iterations']} iterations")

    T, E, NL = len(sc.tris), len(sc.edges), len(sc.len_edges)
    fp = 8 if args.precision == "fp64" else 4
    pst = dict(pst, gs_sweeps=prm.gs_sweeps)
    algo = sec8d_bytes(pst, n, T, E, NL, fp)
    groups_of = {"search": ("refit", "query_vt", "query_ee", "query_vv", "finalize")}
    gms = {g: (sum(prof[h][0] for h in groups_of.get(g, (g,))), max(prof[h][1] for h in groups_of.get(g, (g,))))
           for g in algo}
    dominant = max(prof, key=lambda g: prof[g][0])
    peak, peak_kind = peaks()
    dms, dcount = prof[dominant]
    roof = {"kernel": dominant, "bound": "hbm", "peak": peak, "unit": "GB/s", "peak_source": peak_kind,
            "launches": dcount, "ms_total": dms, "traffic": None,
            "bytes_rule": "algorithmic bytes of the kernel group over the profiled step (see sec8d_bytes), "
                          "per distinct vertex, divided by its launches"}
    if dominant in algo and dms > 0:
        ach = algo[dominant] / (dms / 1000.0) / 1e9
        roof.update(achieved=ach, frac=ach / peak, algo_bytes_per_launch=algo[dominant] / max(1, dcount))
    else:
        roof.update(achieved=None, frac=None)
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            tj = json.load(f)
        ent = tj.get(wname, {}).get(dominant)
        if ent and ent.get("csrc") == csrc_hash(ent.get("files")):
            roof["traffic"] = ent["bytes_per_launch"]
    except Exception:
        pass
    step_ms_prof = sum(m for m, _ in prof.values())
    step_bytes = sum(algo.values())
    roof["step"] = {"algo_bytes": step_bytes, "ms": step_ms_prof,
                    "achieved_gbs": step_bytes / (step_ms_prof / 1000.0) / 1e9,
                    "frac": step_bytes / (step_ms_prof / 1000.0) / 1e9 / peak}
    groups = {g: {"ms": round(m, 3), "launches": c} for g, (m, c) in prof.items()}
    group_roof = {g: {"algo_gb": round(algo[g] / 1e9, 4),
                      "gbs": round(algo[g] / (gms[g][0] / 1000.0) / 1e9, 2) if gms[g][0] > 0 else None}
                  for g in algo}

    # ---- end to end through the C ABI with host buffers ----
    e2e_n = 1
    hx = [(timed_inputs[0].cpu().numpy(), timed_inputs[1].cpu().numpy())]
    hout = np.empty((n, 3))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for k in range(e2e_n):
        gpu.step_host(hx[k][0], hx[k][1], out=hout)
    e2e_s = time.perf_counter() - t0
    e2e_same = bool(np.array_equal(hout, prof_out.cpu().numpy()))
    log(f"end to end: {e2e_s:.2f} s")
    e2e = {"value": job_total(float(e2e_n), dev) / slowest(e2e_s, dev), "unit": "steps/s",
           "h2d_bytes_per_step": 2 * n * 24, "d2h_bytes_per_step": n * 24}
    gpu.close()

    # ---- the metric's comparisons: mixed precision on the same inputs,
    # batched against a plain loop, served against plain ----
    compare = None
    if rank == 0 and world == 1 and not args.no_compare:
        compare = {}
        tune_it = 0 if args.no_tune else args.tune_iters
        if keep and args.precision == "fp64":
            compare["mixed"] = variant_compare(sc, dict(precision=1, colouring=args.colouring), kept_in, kept_out,
                                               dev, stream, flush, tune_it, log, "mixed")
        if keep and gs and args.colouring == 1:
            compare["greedy_colouring"] = variant_compare(sc, dict(precision=prm.precision, colouring=0), kept_in,
                                                          kept_out, dev, stream, flush, tune_it, log, "greedy")
        del kept_in, kept_out
        if args.batch_scenes:
            compare["batched"] = batch_compare(dev, stream, args.batch_scenes, 2, flush)
            log(f"batched: {compare['batched']}")
        if args.requests:
            compare["served"] = serve_compare(dev, args.requests, args.rate, args.max_active, precisions=("mixed",),
                                              group=args.serve_group)
            log(f"served: {compare['served']}")

    # ---- CPU baseline: the oracle on a bounded sample (rank 0, N = 1) ----
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cores = args.ref_cores or host_cores()
        res = oracle_samples(args.config, x0, xt0, args.cpu_budget, cores, 0 if gs else 1,
                             1 if args.step_rule == "ccd" else 0)
        mean_it = float(np.mean(iters))
        rates = [1.0 / (spi * mean_it) for spi, _, _ in res]
        spi, its = res[0][0], res[0][1]
        cpu = {"value": float(np.sum(rates)), "unit": "steps/s", "cores": cores, "kind": "oracle",
               "per_core_value": float(np.mean(rates)),
               "sample": f"{cores} single-threaded oracles side by side, one per host core, each on the first "
                         f"{its} iterations of the chain's first step ({spi * its:.1f} s); seconds per iteration "
                         f"times the {mean_it:.1f} iterations per step of the timed run, steps per second added "
                         f"over the cores (later steps hold more pairs, so this favours the oracle)"}

    if rank == 0:
        out = {"metric": METRIC, "value": steps_per_s, "unit": "steps/s", "n_gpus": world, "steps": K, "warmup": W,
               "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
               "config": {"workload": f"{wname}_{args.precision}" + ("_jacobi" if not gs else "")
                          + ("_greedy" if gs and args.colouring == 0 else "")
                          + ("_gap" if args.gap else "") + ("_ccdstep" if args.step_rule == "ccd" else ""),
                          "verts": n, "tris": T, "edges": E, "len_edges": NL, "dt": sc.dt,
                          "l2": "flushed between steps (256 MiB write)",
                          "parallelism": "replicas" if world > 1 else "single",
                          "acceptance": "exact-filtered intersection test of every x^{t+1} inside the timed step"},
               "contact_pairs_per_sec": pairs / (total_ms / 1000.0),
               "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
               "iterations_per_step": float(np.mean(iters)), "converged_steps": int(sum(s["converged"] for s in stats)),
               "final_r_inf": [round(s["final_r_inf"], 6) for s in stats],
               "frozen_vertices": [int(s["frozen_vertices"]) for s in stats],
               "searches_per_step": [int(s["searches"]) for s in stats],
               "intersections": int(sum(s["intersections"] for s in stats)),
               "uncertain": int(sum(s["uncertain"] for s in stats)),
               "sweep_depth": int(pst["gs_depth"]), "contact_colours": int(max(s["contact_colours"] for s in stats)),
               "edge_colours": int(stats[0]["edge_colours"]),
               "max_vertex_contacts": int(max(s["max_vertex_contacts"] for s in stats)),
               "ccd_hits": int(sum(s["ccd_clamps"] for s in stats)),
               "deterministic_replay": bool(deterministic and e2e_same),
               "autotune": tune, "roofline": roof, "kernel_groups": groups, "group_roofline": group_roof,
               "compare": compare, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "gpu_launches": launches}
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
