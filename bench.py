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
import math
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


def min_iterations(x_t, x_tilde, d_max, gamma):
    """Fewest iterations a step can take: every vertex moves at most
    0.5 gamma D^max per iteration (Eq. forward2 with D_i <= D^max)."""
    far = float(np.max(np.linalg.norm(x_tilde - x_t, axis=1)))
    return max(1, math.ceil(far / (0.5 * gamma * d_max)))


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


def serving_mix():
    """Resident scenes of the serving workload: the paper's scene kinds at
    2K-73K triangles."""
    from paper_2211_04045_gb300 import scenes
    return [scenes.cloth_over_sphere(n=16, side=0.5, sphere_subdiv=3, sphere_r=0.15, noise=0.5, seed=11),
            scenes.cloth_over_sphere(n=32, seed=12),
            scenes.two_cloths(n=48, side=0.4, sep=0.01, omega=6.0, noise=0.3, seed=13),
            scenes.two_cloths(n=136, side=1.0, sep=0.01, omega=6.0, noise=0.3, seed=14),
            scenes.tet_bodies(n_bodies=8, n=6, side=0.2, box=0.8, seed=15),
            scenes.tube_knot(around=32, rings=121, r=0.008, helix_r=0.0095, pitch=0.03, ring_dz=0.002)]


def run_serving(args):
    """Poisson request stream served with continuous batching, against the
    same requests run one at a time in plain FP64."""
    import torch
    from paper_2211_04045_gb300 import cch, scenes
    dev = torch.device("cuda:0")
    scs = serving_mix()
    rng = np.random.default_rng(0)
    N = args.requests
    arrivals = np.cumsum(rng.exponential(1.0 / args.rate, size=N))
    which = rng.integers(0, len(scs), size=N)
    inputs = []
    for i in range(N):
        sc = scs[which[i]]
        x, xt, v = scenes.initial(sc)
        xt = xt + rng.normal(0.0, 1e-4, size=xt.shape) * (sc.inv_mass > 0)[:, None]
        inputs.append((torch.tensor(x, device=dev), torch.tensor(xt, device=dev)))
    # plain: one request at a time, FP64, one resident scene per kind
    base = cch.params_for(scs[0], iters_per_launch=8)
    plain = [cch.Scene(sc, base) for sc in scs]
    for g, sc in zip(plain, scs):  # warm-up: builds and graph capture
        x, xt, _ = scenes.initial(sc)
        g.step(torch.tensor(x, device=dev), torch.tensor(xt, device=dev))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain_ms = []
    for i in range(N):
        a = time.perf_counter()
        plain[which[i]].step(inputs[i][0], inputs[i][1])
        plain_ms.append(1000.0 * (time.perf_counter() - a))
    plain_s = time.perf_counter() - t0
    for g in plain:
        g.close()
    # served: requests arrive on the Poisson clock while others run
    prm = cch.params_for(scs[0], precision=1 if args.precision == "mixed" else 0, iters_per_launch=8,
                         solver=1 if args.solver == "jacobi" else 0)
    sv = cch.Server(80 << 30, prm, max_active=args.max_active)
    ids = [sv.add_scene(sc) for sc in scs]
    # one warm request per scene (pool build, graph capture)
    outs = [torch.empty_like(inputs[0][0])]
    for k, sc in enumerate(scs):
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
    lat = []
    iters = []
    for tk in tickets:
        st, ms = sv.wait(tk)
        lat.append(ms)
        iters.append(st["iterations"])
    served_s = time.perf_counter() - t0
    sv.close()
    tris = [len(sc.tris) for sc in scs]
    out = {"metric": METRIC, "value": N / served_s, "unit": "steps/s", "n_gpus": 1, "steps": N, "warmup": len(scs),
           "ms_per_step": 1000.0 * served_s / N, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
           "config": {"workload": f"serving_mix_{args.precision}" + ("_jacobi" if args.solver == "jacobi" else ""),
                      "requests": N, "rate_per_s": args.rate,
                      "scene_tris": tris, "max_active": args.max_active, "budget_bytes": 80 << 30},
           "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
           "plain_fp64": {"value": N / plain_s, "unit": "steps/s", "p50_ms": float(np.percentile(plain_ms, 50)),
                          "p99_ms": float(np.percentile(plain_ms, 99))},
           "speedup_vs_plain": plain_s / served_s, "iterations_per_step": float(np.mean(iters))}
    print(json.dumps(out), flush=True)
    return 0


def run_reference(args):
    """CPU oracle as the reference arm (rank 0 only)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2211_04045_gb300 import scenes
    sc, wname = workload(args.config)
    x, xt, v = scenes.initial(sc)
    prm_d = dict(sc.params)
    d_max = prm_d.get("d_max", 4e-3)
    gamma = 0.9
    per_step = []
    pairs = 0
    it_total = 0
    budget = max(2.0, args.ref_budget / max(1, args.steps + args.warmup))
    for s in range(args.warmup + args.steps):
        spi, its, pe = oracle_sample(sc, x, xt, budget)
        need = min_iterations(x, xt, d_max, gamma)
        if s >= args.warmup:
            per_step.append(spi * need)
            pairs += pe
            it_total += its
    tot = float(np.sum(per_step))
    val = len(per_step) / tot
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "steps/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * tot / len(per_step),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"{wname}_fp64", "verts": sc.n_verts, "tris": len(sc.tris), "dt": sc.dt},
           "cpu_baseline": {"value": val, "unit": "steps/s", "cores": 1, "kind": "oracle",
                            "sample": "per step: the oracle's first iterations of the workload's first step (about "
                                      f"{budget:.0f} s), seconds per iteration times the fewest iterations that "
                                      "step needs (max target displacement / 0.45 D^max), which favours the oracle"},
           "e2e": {"value": val, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


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
    ap.add_argument("--gap", action="store_true", help="gap contact constraints instead of the volume-based ones")
    ap.add_argument("--step-rule", default="distance", choices=["distance", "ccd"],
                    help="forward step size: the distance bound (Eq. forward2) or the CCD-based scheme of Sec. 5.1")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the launch-configuration autotuner")
    ap.add_argument("--tune-iters", type=int, default=48, help="iterations of the autotuner's probe step")
    ap.add_argument("--requests", type=int, default=48, help="serving: requests in the stream")
    ap.add_argument("--rate", type=float, default=200.0, help="serving: mean arrivals per second")
    ap.add_argument("--max-active", type=int, default=16, help="serving: requests batched at once")
    ap.add_argument("--ncu-warm", type=int, default=0, help="full chain steps before the --ncu-case step")
    ap.add_argument("--ncu-case", type=int, default=0,
                    help="profiling aid: run one step of the workload capped at this many iterations and exit "
                         "(prints no bench line)")
    args = ap.parse_args()
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
    prm = cch.params_for(sc, precision=1 if args.precision == "mixed" else 0,
                         solver=1 if args.solver == "jacobi" else 0, constraint_form=1 if args.gap else 0,
                         step_rule=1 if args.step_rule == "ccd" else 0)
    if args.ncu_case:
        x0, xt0, v0 = scenes.initial(sc)
        x, xt, v = (torch.tensor(a, device=dev) for a in (x0, xt0, v0))
        if args.ncu_warm:
            dyn = scenes.TorchDynamics(sc, dev)
            gw = cch.Scene(sc, prm)
            for _ in range(args.ncu_warm):
                out, _ = gw.step(x, xt)
                v = dyn.next_velocity(out, x)
                x, xt = out, dyn.predict(out, v)
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
                         f"{st['max_vertex_contacts']} contacts at one vertex, sweep depth {st['gs_depth']}\n")
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
        xt = dyn.predict(x, v)
        log(f"warm-up step {s}: {st['iterations']} iterations, {time.perf_counter() - t0:.2f} s")
    torch.cuda.synchronize(dev)
    timed_inputs = (x.clone(), xt.clone())
    tune = None
    if not args.no_tune:
        tune = gpu.autotune(x, xt, probe_iters=args.tune_iters)
        log(f"autotune: {tune}")

    # ---- timed region: K further steps of the chain ----
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
        ev[k][0].record(stream)
        _, st = gpu.step(x, xt, out=outbuf)
        ev[k][1].record(stream)
        stats.append(st)
        v = dyn.next_velocity(outbuf, x)
        x = outbuf.clone()
        xt = dyn.predict(x, v)
    t_end.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    step_ms = np.array([a.elapsed_time(b) for a, b in ev])
    log(f"timed {K} steps in {total_ms / 1000:.2f} s: " + ", ".join(f"{m:.0f} ms" for m in step_ms))
    total_ms = slowest(total_ms, dev)
    # replaying the first timed step must give the same result (determinism)
    first_out = None

    iters = np.array([s["iterations"] for s in stats])
    pairs = job_total(float(np.sum([s["pairs_evaluated"] for s in stats])), dev)
    launches = int(job_total(float(np.sum([s["kernel_launches"] for s in stats])), dev))
    steps_per_s = job_total(float(K), dev) / (total_ms / 1000.0)

    # ---- per-kernel timing (events on the launching stream, no graphs) ----
    gpu.set_profiling(True)
    flush.zero_()
    prof_out, pst = gpu.step(timed_inputs[0], timed_inputs[1])
    pstats = [pst]
    prof = gpu.profile()
    gpu.set_profiling(False)
    deterministic = pst["iterations"] == stats[0]["iterations"] and pst["pairs_evaluated"] == stats[0]["pairs_evaluated"]
    log(f"profiled one step: {pst['iterations']} iterations")

    nvc = int(np.count_nonzero(np.isin(np.arange(n), np.concatenate([sc.tris.ravel(), sc.edges.ravel(),
                                                                        np.asarray(sc.points).ravel()]))))
    T, E, NL = len(sc.tris), len(sc.edges), len(sc.len_edges)
    searches = sum(s["searches"] for s in pstats)
    p_pairs = sum(s["pairs_evaluated"] for s in pstats)
    p_cons = sum(s["active_contacts"] for s in pstats)
    p_iters = sum(s["iterations"] for s in pstats)
    ppi = p_pairs / max(1, p_iters)      # |P| per iteration
    cpi = p_cons / max(1, p_iters)       # contacts per iteration
    fp = 8 if args.precision == "fp64" else 4
    # algorithmic bytes of each kernel group over the profiled step: what the
    # method must read and write at least (positions 24 B per vertex in FP64,
    # pair records 32 B, contact records 144 B in FP64 / 96 B mixed)
    crec = 144 if args.precision == "fp64" else 96
    algo = {
        "query_vt": searches * (16.0 * nvc + 12.0 * T + 16.0 * nvc),
        "query_ee": searches * (8.0 * E + 32.0 * nvc),
        "finalize": p_iters * ppi * (24.0 + 96.0 + 32.0) * (searches / max(1, p_iters)),
        "refresh": (p_iters - searches) * (32.0 * ppi * 2 + 24.0 * min(n, 4 * ppi)),
        "assemble": p_iters * cpi * (4.0 + 32.0 + 4 * 3 * fp + crec),
        "order": p_iters * cpi * (24.0 * 4 + 48.0 * 3 + 16.0),
        "sweep": p_iters * (cpi * (crec + 4 * 3 * (3 * fp)) + NL * (8.0 + 4 * fp + 4 * 3 * fp)),
        "forward": p_iters * 96.0 * n,
        "refit": searches * (24.0 * n + 12.0 * T + 8.0 * E),
    }
    dominant = max(prof, key=lambda g: prof[g][0])
    peak, peak_kind = peaks()
    dms, dcount = prof[dominant]
    roof = {"kernel": dominant, "bound": "hbm", "peak": peak, "unit": "GB/s", "peak_source": peak_kind,
            "launches": dcount, "ms_total": dms, "traffic": None}
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
    groups = {g: {"ms": round(m, 3), "launches": c} for g, (m, c) in prof.items()}

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

    # ---- CPU baseline: the oracle on a bounded sample (rank 0, N = 1) ----
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        spi, its, pe = oracle_sample(sc, x0, xt0, args.cpu_budget, 1 if args.solver == "jacobi" else 0,
                                     1 if args.step_rule == "ccd" else 0)
        mean_it = float(np.mean(iters))
        cpu = {"value": 1.0 / (spi * mean_it), "unit": "steps/s", "cores": 1, "kind": "oracle",
               "sample": f"first {its} iterations of the chain's first step ({spi * its:.1f} s), seconds per "
                         f"iteration times the {mean_it:.1f} iterations per step of the timed run (later steps "
                         f"hold more pairs, so this favours the oracle)"}

    if rank == 0:
        out = {"metric": METRIC, "value": steps_per_s, "unit": "steps/s", "n_gpus": world, "steps": K, "warmup": W,
               "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
               "config": {"workload": f"{wname}_{args.precision}" + ("_jacobi" if args.solver == "jacobi" else "")
                          + ("_gap" if args.gap else "") + ("_ccdstep" if args.step_rule == "ccd" else ""), "verts": n, "tris": T, "edges": E,
                          "len_edges": len(sc.len_edges), "dt": sc.dt, "l2": "flushed between steps (256 MiB write)",
                          "parallelism": "replicas" if world > 1 else "single"},
               "contact_pairs_per_sec": pairs / (total_ms / 1000.0),
               "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
               "iterations_per_step": float(np.mean(iters)), "converged_steps": int(sum(s["converged"] for s in stats)),
               "sweep_depth": int(pst["gs_depth"]),
               "max_vertex_contacts": int(max(s["max_vertex_contacts"] for s in stats)),
               "ccd_hits": int(sum(s["ccd_clamps"] for s in stats)),
               "deterministic_replay": bool(deterministic and e2e_same),
               "autotune": tune, "roofline": roof, "kernel_groups": groups, "cpu_baseline": cpu, "e2e": e2e,
               "clocks": clk,
               "gpu_launches": launches}
        print(json.dumps(out), flush=True)
    gpu.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
