"""Benchmark of the GB300 short-range tree force (the hot path of GreeM's PP part).

One step = one call of greem_short_force_ex over the whole particle set: keys, radix
sort, tree + moments, groups, interaction lists and the FP32 force (S1-S6), inputs
resident in HBM.  Workload: 256^3 particles (Zel'dovich P(k) ~ k^-2 grid, rms 0.5
spacing, plus 5000 NFW halos), L = 1, r_cut = 3/256, theta = 0.5, n_leaf = 10, n_crit
autotuned (untimed, before the warm-up).  Inputs (470 MB) are larger than the 129 MB L2.

The e2e figure runs the same steps through greem_short_force_host: each step copies its
inputs in from pinned host memory and its result out, the copies overlapping the
neighbouring steps' computation.

With N > 1 processes (torchrun) the same box is split over them as the paper does it
(recursive multisection from sampled particles, local essential trees exchanged by one
all-to-all-v per step; paper_0910_0121_gb300/domain.py): strong scaling, each step timed
on every process and the slowest taken.

Prints one JSON line.  --impl reference times the FP64 CPU oracle instead (on the host
cores, on a bounded sample of the same workload).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("short-range tree force particles/s & interactions/s at θ=0.5, % FP32 peak, FP32 vs FP64")
WORKLOAD = "zeldovich256+5000nfw_theta0.5"
# FP32 flops credited per interaction (FMA = 2): 3 subtractions, 5 for r^2, 1 for r, 1 for R,
# 12 for the inner polynomial of Eq. 2, 10 for its (R-1)^6 correction, 4 for m g / r^3, 6 to accumulate
FLOPS_PER_INTERACTION = 42
SM_COUNT_NOMINAL = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n-crit", type=int, default=0, help="skip autotuning and use this n_crit")
    ap.add_argument("--no-extras", action="store_true", help="skip the graph, theta-scan and batched lines")
    ap.add_argument("--config5", action="store_true",
                    help="time the 512^3 full TreePM step (PP + TSC PM on 512^3) in one CUDA graph instead")
    ap.add_argument("--no-config5", action="store_true",
                    help="leave the 512^3 TreePM graph out of the default line's extras")
    ap.add_argument("--dist-backend", default="nccl", choices=["nccl", "gloo"],
                    help="N > 1: the collective backend of the domain exchange (gloo stages through the host)")
    ap.add_argument("--no-direct", action="store_true",
                    help="leave out the tree-against-direct error (oracle direct sums for sampled particles)")
    ap.add_argument("--quad", action="store_true",
                    help="with --profile-case: add the second-order (quadrupole) terms, theta = 0.7")
    ap.add_argument("--profile-case", choices=["nfw128", "zel256", "zel256tree"], default=None,
                    help="run --steps short-force calls on this workload (n_crit from --n-crit, else 128; "
                         "zel256tree: tree builds only, about 2 GB on the device) and print the stats; no "
                         "timing (the small cases for profiler captures)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def across_ranks(ms_local: float, n_local: int, dist=None, device=None):
    """Whole-job numbers for N independent replicas (weak scaling): the step time is
    the slowest rank's, and the particle count is every rank's.  Returns
    (ms_per_step, particles_per_s).  With dist=None this is one rank."""
    if dist is None:
        return ms_local, n_local / (ms_local * 1e-3)
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    n = torch.tensor([float(n_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    ms = float(t.item())
    return ms, float(n.item()) / (ms * 1e-3)


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *exc):
        self.rows = []
        if self.p is None:
            return False
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                self.rows.append(f)
        return False

    def summary(self):
        rows = getattr(self, "rows", [])
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


# ----------------------------------------------------------------------------- CPU oracle
def oracle_tree(pos, mass, prm, n_crit):
    """FP64 oracle S1-S4 (wrap, keys, stable sort, tree + moments, groups) on the whole
    set, as it stands (one thread, C).  Returns (tree, seconds)."""
    import oracle
    t0 = time.perf_counter()
    T = oracle.Tree(pos, mass, prm["L"], prm["r_cut"], n_crit=n_crit, n_leaf=prm.get("n_leaf", 10))
    return T, time.perf_counter() - t0


def oracle_force_sample(T, prm, frac, seed):
    """Oracle S5-S6 (lists, FP64 list force) for a seeded sample of groups on all host
    cores.  Returns (seconds, scale to all groups by particle count, groups sampled, threads)."""
    import oracle
    nthreads = oracle.max_threads()
    G = T.n_groups
    rng = np.random.default_rng(seed)
    ns = max(8, int(G * frac))
    sel = np.sort(rng.choice(G, size=ns, replace=False))
    t1 = time.perf_counter()
    T.build_lists(prm["theta"], sel)
    T.list_force(0.0, nthreads)
    t_sample = time.perf_counter() - t1
    nodes = T.nodes()
    grp = T.groups()
    cnt = nodes[grp, 5] - nodes[grp, 4]
    return t_sample, float(cnt.sum()) / float(cnt[sel].sum()), ns, nthreads


# The paper's own rate, for context only: the whole TreePM step at theta = 0.5 ran at about
# 5e4 particles/s per core on the Cray XT4 (2.2 GHz quad-core Opteron; abstract, Sec. 5),
# for a 512^3 LCDM run with more than 1e6 particles per core.
PAPER_RATE = {"value": 5.0e4, "unit": "particles/s per core",
              "hardware": "Cray XT4, quad-core Opteron 2.2 GHz (FP64 storage, single-precision pair kernel)",
              "workload": "whole TreePM step, 512^3 LCDM, theta = 0.5, > 1e6 particles per core",
              "source": "abstract; Sec. 5", "kind": "context, not the target"}


def oracle_sample(pos, mass, prm, n_crit, frac=0.02, seed=7, frac1=0.0025):
    """One oracle step on a bounded sample: S1-S4 on everything (one thread), S5-S6 on a
    group sample on all host cores scaled to all groups, and again on a smaller sample on
    one thread.  Returns (seconds for the whole step, description, threads, seconds for the
    whole step on one thread)."""
    T, t_tree = oracle_tree(pos, mass, prm, n_crit)
    t_s, scale, ns, nth = oracle_force_sample(T, prm, frac, seed)
    import oracle
    G = T.n_groups
    rng = np.random.default_rng(seed + 1)
    sel1 = np.sort(rng.choice(G, size=max(8, int(G * frac1)), replace=False))
    t1 = time.perf_counter()
    T.build_lists(prm["theta"], sel1)
    T.list_force(0.0, 1)
    t_1 = time.perf_counter() - t1
    nodes, grp = T.nodes(), T.groups()
    cnt = nodes[grp, 5] - nodes[grp, 4]
    scale1 = float(cnt.sum()) / float(cnt[sel1].sum())
    desc = (f"S1-S4 on all {len(pos)} particles ({t_tree:.1f} s, 1 thread); lists+force on a seeded "
            f"{ns}/{G} group sample ({t_s:.2f} s, {nth} threads) scaled x{scale:.0f} by particle count; "
            f"1-thread leg: lists+force on {len(sel1)} groups ({t_1:.2f} s) scaled x{scale1:.0f}")
    return t_tree + t_s * scale, desc, nth, t_tree + t_1 * scale1


def reference_arm(args, rank, world):
    if rank != 0:
        return
    from paper_0910_0121_gb300 import synth
    pos, mass, prm = synth.config_zel256()
    N = len(pos)
    # the n_crit the GPU arm's autotuner settles on for this workload (its config line)
    n_crit = args.n_crit or 192
    times, walls, trees = [], [], []
    nth, ns, G = 1, 0, 0
    for k in range(args.warmup + args.steps):
        w0 = time.perf_counter()
        T, t_tree = oracle_tree(pos, mass, prm, n_crit)
        t_s, scale, ns, nth = oracle_force_sample(T, prm, 0.0005, 100 + k)
        G = T.n_groups
        del T
        if k >= args.warmup:
            times.append(t_tree + t_s * scale)
            walls.append(time.perf_counter() - w0)
            trees.append(t_tree)
    desc = (f"every step: S1-S4 on all {N} particles (1 thread, {statistics.mean(trees):.1f} s) and lists+force on "
            f"a fresh seeded {ns}/{G} group sample ({nth} threads), scaled to all groups by particle count; "
            f"ms_per_step is that projection, sample_wall_ms_per_step the measured time of the sampled step")
    v = N / statistics.mean(times)
    line = {"metric": METRIC, "value": v, "unit": "particles/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "N": N, "L": 1.0, "r_cut": prm["r_cut"], "theta": prm["theta"],
                       "n_crit": n_crit, "n_leaf": 10, "list_chunk": 256, "block_shape": 16,
                       "l2": "inputs (470 MB) larger than L2, no flush", "parallelism": "domains 1x1x1"},
            "cpu_baseline": {"value": v, "unit": "particles/s", "cores": nth, "kind": "oracle", "sample": desc},
            "projected": True, "sample_wall_ms_per_step": 1e3 * statistics.mean(walls),
            "e2e": {"value": v, "unit": "particles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def traffic_per_launch(list_entries):
    """DRAM bytes of one force launch, from the ncu record in profiles/ (bytes per list
    entry on a smaller case) scaled by this launch's list entries; None when the force
    kernel's source changed since the record was taken."""
    import hashlib
    rec = os.path.join(ROOT, "profiles", "force_f32_traffic.txt")
    src = os.path.join(ROOT, "paper_0910_0121_gb300", "csrc", "force.cu")
    try:
        kv = dict(l.split(":", 1) for l in open(rec) if ":" in l and not l.startswith("#"))
        if kv["force_cu_sha256_16"].strip() != hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]:
            return None
        return float(kv["bytes_per_list_entry"]) * list_entries
    except (OSError, KeyError, ValueError):
        return None


def extras(ctx, P, M, p, prm, acc, stream, rows=None, tvd_dev=None):
    """Context numbers beside the headline: CUDA-graph replay of the same step, the
    opening-angle scan, the distance-dependent opening angle of Eq. 12, the integration
    kernels, the second-order terms, and the 64-box batched workload (one call vs per-box
    calls)."""
    import torch
    from paper_0910_0121_gb300 import greem, synth
    out = {}
    N = P.shape[0]
    ev = lambda: torch.cuda.Event(enable_timing=True)
    # graph replay of the whole step
    ctx.graph_capture(P, M, greem.params(L=p.L, r_cut=p.r_cut, theta=p.theta, n_crit=p.n_crit, n_leaf=p.n_leaf,
                                         list_chunk=p.list_chunk, block_shape=p.block_shape), acc)
    for _ in range(2):
        ctx.graph_launch()
    a, b = ev(), ev()
    a.record(stream)
    reps = 5
    for _ in range(reps):
        rc = ctx.graph_launch()
        if rc != greem.OK:
            raise greem.GreemError(rc, "greem_graph_launch")
    b.record(stream)
    torch.cuda.synchronize()
    gms = a.elapsed_time(b) / reps
    out["graph_replay"] = {"ms_per_step": gms, "particles_per_s": N / (gms * 1e-3)}
    # opening-angle scan at the tuned n_crit
    scan = {}
    for th in (0.3, 0.5, 0.7):
        q = greem.params(L=p.L, r_cut=p.r_cut, theta=th, n_crit=p.n_crit, n_leaf=p.n_leaf, list_chunk=p.list_chunk,
                         block_shape=p.block_shape, flags=greem.FLAG_STAGE_TIMES)
        ctx.short_force(P, M, q, acc)
        a, b = ev(), ev()
        a.record(stream)
        ctx.short_force(P, M, q, acc)
        b.record(stream)
        torch.cuda.synchronize()
        s = ctx.stats()
        if rows is not None:
            rows[f"theta{th}"] = acc[tvd_dev].double().cpu().numpy()
        scan[str(th)] = {"ms_per_step": a.elapsed_time(b), "N_int": s["n_interactions"] / N,
                         "force_tflops": FLOPS_PER_INTERACTION * s["n_interactions"] / (s["ms_force"] * 1e-3) / 1e12}
    out["theta_scan"] = scan
    # distance-dependent opening angle of Eq. 12 (Sec. 4.1), theta0 = 0.25 capped at 0.7: on
    # a 32^3 NFW mix it matches theta = 0.5's interaction count with a lower error tail
    q = greem.params(L=p.L, r_cut=p.r_cut, theta=0.7, n_crit=p.n_crit, n_leaf=p.n_leaf, list_chunk=p.list_chunk,
                     block_shape=p.block_shape, flags=greem.FLAG_STAGE_TIMES | greem.FLAG_THETA_EQ12, theta0=0.25)
    ctx.short_force(P, M, q, acc)
    a, b = ev(), ev()
    a.record(stream)
    ctx.short_force(P, M, q, acc)
    b.record(stream)
    torch.cuda.synchronize()
    s = ctx.stats()
    if rows is not None:
        rows["eq12_theta0_0.25_max0.7"] = acc[tvd_dev].double().cpu().numpy()
    out["theta_eq12"] = {"theta0": 0.25, "theta_max": 0.7, "ms_per_step": a.elapsed_time(b),
                         "N_int": s["n_interactions"] / N, "lists_ms": s["ms_lists"], "force_ms": s["ms_force"]}
    # the integration around the force (Sec. 2.2 steps 1, 6, 7; Eq. 7): kick, drift and the
    # shared timestep on the bench particles (velocities zero, the force of the last call)
    vel = torch.zeros((N, 3), dtype=torch.float32, device=P.device)
    Pc = P.clone()
    ctx.kick(vel, acc, 1e-3)
    a, b = ev(), ev()
    a.record(stream)
    ctx.kick(vel, acc, 1e-3)
    ctx.drift(Pc, vel, p.L, 1e-3)
    dtq = ctx.timestep(vel, acc, 1e-4, 1.0)
    b.record(stream)
    torch.cuda.synchronize()
    out["kick_drift_timestep_ms"] = a.elapsed_time(b)
    del Pc, vel
    # second-order (quadrupole) terms of Sec. 4.1 at theta = 0.5 and 0.7
    quad = {}
    for th in (0.5, 0.7):
        q = greem.params(L=p.L, r_cut=p.r_cut, theta=th, n_crit=p.n_crit, n_leaf=p.n_leaf, list_chunk=p.list_chunk,
                         block_shape=p.block_shape, flags=greem.FLAG_STAGE_TIMES | greem.FLAG_QUADRUPOLE)
        ctx.short_force(P, M, q, acc)
        a, b = ev(), ev()
        a.record(stream)
        ctx.short_force(P, M, q, acc)
        b.record(stream)
        torch.cuda.synchronize()
        s = ctx.stats()
        if rows is not None:
            rows[f"quadrupole_theta{th}"] = acc[tvd_dev].double().cpu().numpy()
        quad[str(th)] = {"ms_per_step": a.elapsed_time(b), "N_int": s["n_interactions"] / N, "force_ms": s["ms_force"]}
    out["quadrupole"] = quad
    # 64 independent boxes: one batched call vs one call per box (FP32) and per-box FP64 calls
    bpos, bmass, boff, bprm = synth.config_batched()
    BP = torch.from_numpy(bpos).cuda()
    BM = torch.from_numpy(bmass).cuda()
    per = [greem.params(L=q["L"], r_cut=q["r_cut"], theta=q["theta"], n_crit=p.n_crit, n_leaf=10,
                        list_chunk=p.list_chunk, block_shape=p.block_shape) for q in bprm]
    bacc = ctx.short_force_batched(BP, BM, boff, per)
    a, b = ev(), ev()
    a.record(stream)
    ctx.short_force_batched(BP, BM, boff, per, bacc)
    b.record(stream)
    torch.cuda.synchronize()
    t_batched = a.elapsed_time(b)
    views = [(BP[boff[k]:boff[k + 1]], BM[boff[k]:boff[k + 1]]) for k in range(len(per))]
    for (vp, vm), q in zip(views, per):
        ctx.short_force(vp, vm, q)
    a.record(stream)
    for (vp, vm), q in zip(views, per):
        ctx.short_force(vp, vm, q)
    b.record(stream)
    torch.cuda.synchronize()
    t_single = a.elapsed_time(b)
    per64 = [greem.params(L=q.L, r_cut=q.r_cut, theta=q.theta, n_crit=q.n_crit, n_leaf=10, precision=greem.F64)
             for q in per]
    a.record(stream)
    for (vp, vm), q in zip(views, per64):
        ctx.short_force(vp, vm, q)
    b.record(stream)
    torch.cuda.synchronize()
    t64 = a.elapsed_time(b)
    NB = int(boff[-1])
    out["batched64"] = {"N": NB, "boxes": len(per), "batched_ms": t_batched, "per_box_fp32_ms": t_single,
                        "per_box_fp64_ms": t64, "batched_particles_per_s": NB / (t_batched * 1e-3),
                        "speedup_vs_per_box_fp32": t_single / t_batched, "speedup_vs_per_box_fp64": t64 / t_batched}
    return out


N_DIRECT, SEED_DIRECT = 512, 9100777


def guarded(fn, *a, **kw):
    """A context leg of the line: its dict, or its error, without losing the line."""
    try:
        return fn(*a, **kw)
    except Exception as e:  # noqa: BLE001 - reported in the line
        return {"error": f"{type(e).__name__}: {e}"}


def error_stats(a, ref):
    """Relative error |a - ref| / |ref| per particle; particles with |ref| below 1e-6 of the
    median are left out (reading C13)."""
    n = np.linalg.norm(ref, axis=1)
    keep = n > 1e-6 * np.median(n[n > 0])
    e = np.linalg.norm(a - ref, axis=1)[keep] / n[keep]
    return {"median": float(np.median(e)), "p90": float(np.quantile(e, 0.9)), "p99": float(np.quantile(e, 0.99)),
            "p999": float(np.quantile(e, 0.999)), "max": float(e.max()), "n": int(keep.sum())}


def tree_vs_direct(pos, mass, prm, rows):
    """The error of the GPU tree force (FP32) against the brute-force minimum-image sum of
    Eq. 1-2 over all N particles (the oracle's FP64 direct sum, O(N) per particle) at a
    seeded sample of particles: the tree approximation error of Sec. 3.1.2, reported, not
    bounded."""
    import oracle
    idx = rows["idx"]
    t0 = time.perf_counter()
    ref = oracle.direct_at(pos, mass, prm["L"], prm["r_cut"], idx)
    out = {"particles": len(idx), "seed": SEED_DIRECT, "direct_s": time.perf_counter() - t0,
           "reference": "oracle direct_at: FP64 brute-force minimum-image sum over all N",
           "denominator": "|a_direct|, particles below 1e-6 of the median left out"}
    for k, v in rows.items():
        if k != "idx":
            out[k] = error_stats(v, ref)
    return out


def config1_leg(ctx, stream, steps=50):
    """The 32^3 uniform set (r_cut = 3/32, theta = 0.5, n_crit = 64), whose whole step is
    short next to the launch cost of its kernels: the call timed as a user repeating it
    (a graph replay of the whole call from the third call on) and with replays off (every
    kernel launched on its own)."""
    import torch
    from paper_0910_0121_gb300 import greem, synth
    pos, mass, prm = synth.config_uniform32()
    N = len(pos)
    P, M = torch.from_numpy(pos).cuda(), torch.from_numpy(mass).cuda()
    acc = torch.empty((N, 3), dtype=torch.float32, device="cuda")
    q = greem.params(L=prm["L"], r_cut=prm["r_cut"], theta=prm["theta"], n_crit=prm["n_crit"] or 64,
                     n_leaf=prm.get("n_leaf", 10))
    out = {"workload": "uniform32: 32^3 uniform", "N": N, "r_cut": prm["r_cut"], "theta": prm["theta"],
           "n_crit": q.n_crit}
    try:
        for name, replay in (("replayed", 1), ("launched", 0)):
            ctx.debug_set(greem.DEBUG_REPLAY, replay)
            for _ in range(3):
                ctx.short_force(P, M, q, acc)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            for _ in range(steps):
                ctx.short_force(P, M, q, acc)
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / steps
            st = ctx.stats()
            out[name] = {"ms_per_step": ms, "particles_per_s": N / (ms * 1e-3), "replayed": st["replayed"],
                         "kernels": st["kernel_launches"]}
    finally:
        ctx.debug_set(greem.DEBUG_REPLAY, 1)
    return out


def config2_leg(ctx, stream, steps=5):
    """The 128^3 NFW mix (half uniform, half in 1000 NFW halos), r_cut = 3/128, theta = 0.5,
    n_crit = 64: the FP32 relative-coordinate force against the plain FP64 form, step and
    force times, and each form's error against the oracle's FP64 list force on a seeded
    2% group sample."""
    import torch
    import oracle
    from paper_0910_0121_gb300 import greem, synth
    pos, mass, prm = synth.config_nfw128()
    N = len(pos)
    P, M = torch.from_numpy(pos).cuda(), torch.from_numpy(mass).cuda()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    out = {"workload": "nfw128: 128^3, 50% uniform + 1000 NFW halos", "N": N, "r_cut": prm["r_cut"],
           "theta": prm["theta"], "n_crit": prm["n_crit"], "n_leaf": prm["n_leaf"]}
    accs = {}
    for name, prec, dt, reps in (("fp32", greem.F32_REL, torch.float32, steps), ("fp64", greem.F64, torch.float64, 2)):
        q = greem.params(L=prm["L"], r_cut=prm["r_cut"], theta=prm["theta"], n_crit=prm["n_crit"],
                         n_leaf=prm["n_leaf"], precision=prec, flags=greem.FLAG_STAGE_TIMES)
        acc = torch.empty((N, 3), dtype=dt, device="cuda")
        ctx.short_force(P, M, q, acc)
        a, b = ev(), ev()
        fms = []
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(reps):
            ctx.short_force(P, M, q, acc)
            fms.append(ctx.stats()["ms_force"])
        b.record(stream)
        torch.cuda.synchronize()
        s = ctx.stats()
        ms = a.elapsed_time(b) / reps
        out[name] = {"ms_per_step": ms, "particles_per_s": N / (ms * 1e-3), "force_kernel_ms": statistics.mean(fms),
                     "N_int": s["n_interactions"] / N}
        accs[name] = acc.double().cpu().numpy()
    out["fp32"]["force_tflops"] = (FLOPS_PER_INTERACTION * out["fp32"]["N_int"] * N
                                   / (out["fp32"]["force_kernel_ms"] * 1e-3) / 1e12)
    out["force_speedup_fp32_vs_fp64"] = out["fp64"]["force_kernel_ms"] / out["fp32"]["force_kernel_ms"]
    out["step_speedup_fp32_vs_fp64"] = out["fp64"]["ms_per_step"] / out["fp32"]["ms_per_step"]
    T = oracle.Tree(pos, mass, prm["L"], prm["r_cut"], n_crit=prm["n_crit"], n_leaf=prm["n_leaf"])
    G = T.n_groups
    sel = np.sort(np.random.default_rng(SEED_DIRECT + 2).choice(G, size=max(8, int(0.02 * G)), replace=False))
    T.build_lists(prm["theta"], sel)
    ref_sorted = T.list_force()
    _, perm, _, _ = T.sorted()
    nodes, grp = T.nodes(), T.groups()
    srt = np.concatenate([np.arange(nodes[grp[g], 4], nodes[grp[g], 5]) for g in sel])
    ref = ref_sorted[srt]
    for name in ("fp32", "fp64"):
        out[name]["error_vs_oracle"] = error_stats(accs[name][perm[srt]], ref)
    out["oracle_sample"] = f"FP64 list force on identical lists, {len(sel)}/{G} seeded groups, {len(srt)} particles"
    return out


def domains8_leg(P, M, p, stream, nproc=8, seed=91001):
    """The 256^3 set split into 2x2x2 boxes as the multi-process step does it, emulated on
    this one GPU: the boxes from a seeded sample (Eq. 3 at R = 4e-4, recursive multisection),
    the particles packed by box, then per box its tree and LET export for the other boxes
    and its force over its particles and the items the other boxes sent it, each call timed
    on the device.  There is no exchange here (the items are sliced on this device); the
    per-process compute of the split is what is measured.  Also the split accelerations
    against the one-process ones."""
    import torch
    from paper_0910_0121_gb300 import domain, greem
    N = P.shape[0]
    grid = domain_grid(nproc)
    ctx = greem.Context(stream)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    try:
        prm = dict(L=p.L, r_cut=p.r_cut, theta=p.theta, n_crit=p.n_crit, n_leaf=p.n_leaf, list_chunk=p.list_chunk,
                   block_shape=p.block_shape)
        one = ctx.short_force(P, M, greem.params(**prm)).clone()
        ns = greem.sample_count(N, N, 1, 4e-4, 0.0, 0.0, 0.2)
        idx = torch.from_numpy(np.sort(np.random.default_rng(seed).choice(N, size=ns, replace=False))).cuda()
        boxes = greem.domain_boxes(ctx.cell_index(P, p.L, idx).cpu().numpy(), grid)
        ids = torch.arange(N, dtype=torch.int64, device="cuda")
        po, mo, io, counts = ctx.domain_pack(P, M, ids, p.L, boxes)
        off = np.concatenate([[0], np.cumsum(counts)])
        exports, t_let, t_force, n_imp = [], [], [], []
        for d in range(nproc):
            a, b = ev(), ev()
            a.record(stream)
            ctx.build_tree(po[off[d]:off[d + 1]], mo[off[d]:off[d + 1]], greem.params(**prm))
            ip, im, _, c = ctx.let_export(boxes, d)
            b.record(stream)
            b.synchronize()
            t_let.append(a.elapsed_time(b))
            exports.append((ip.clone(), im.clone(), np.concatenate([[0], np.cumsum(c)])))
        acc = torch.empty((N, 3), dtype=torch.float32, device="cuda")
        for d in range(nproc):
            rp = [e[0][e[2][d]:e[2][d + 1]] for s_, e in enumerate(exports) if s_ != d]
            rm = [e[1][e[2][d]:e[2][d + 1]] for s_, e in enumerate(exports) if s_ != d]
            n_imp.append(int(sum(x.shape[0] for x in rp)))
            allp = torch.cat([po[off[d]:off[d + 1]]] + rp)
            allm = torch.cat([mo[off[d]:off[d + 1]]] + rm)
            a, b = ev(), ev()
            a.record(stream)
            ad = ctx.short_force(allp, allm, greem.params(**prm))
            b.record(stream)
            b.synchronize()
            t_force.append(a.elapsed_time(b))
            acc[io[off[d]:off[d + 1]]] = ad[: off[d + 1] - off[d]]
        torch.cuda.synchronize()
        split = acc.double().cpu().numpy()
        ref = one.double().cpu().numpy()
        n = np.linalg.norm(ref, axis=1)
        keep = n > 1e-6 * np.median(n)
        dif = np.linalg.norm(split - ref, axis=1)[keep] / n[keep]
        per = [a_ + b_ for a_, b_ in zip(t_let, t_force)]
        return {"grid": list(grid), "samples": ns, "n_local": [int(x) for x in counts], "n_import": n_imp,
                "let_bytes": [28 * int(e[2][-1]) for e in exports],
                "tree_and_let_ms": t_let, "force_ms": t_force, "slowest_domain_ms": max(per),
                "sum_over_domains_ms": sum(per),
                "split_vs_one_process": {"median": float(np.median(dif)), "p99": float(np.quantile(dif, 0.99)),
                                         "p999": float(np.quantile(dif, 0.999))},
                "note": "per-process compute of the 2x2x2 split, run one box after another on one GPU; no exchange"}
    finally:
        ctx.close()


def config5_leg(args):
    """512^3 Zel'dovich (rms 1 spacing) + 20000 NFW halos, theta = 0.5, r_cut = 3/512: the
    whole TreePM force (short-range tree force plus PM with TSC on 512^3) replayed as one
    CUDA graph.  Returns its line (a dict)."""
    import torch
    from paper_0910_0121_gb300 import greem, synth
    t0 = time.time()
    pos, mass, prm = synth.config_zel512()
    gen_s = time.time() - t0
    N = len(pos)
    P = torch.from_numpy(pos).cuda()
    M = torch.from_numpy(mass).cuda()
    del pos
    acc = torch.empty((N, 3), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    ctx = greem.Context(stream)
    nc = args.n_crit or 192
    p = greem.params(L=1.0, r_cut=prm["r_cut"], theta=0.5, n_crit=nc, flags=greem.FLAG_ADD_PM, n_pm=512,
                     assign=greem.ASSIGN_TSC)
    try:
        ctx.graph_capture(P, M, p, acc)
        st = ctx.stats()
        for _ in range(max(3, args.warmup)):
            ctx.graph_launch()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        with ClockSampler(torch.cuda.current_device()) as clk:
            e0.record(stream)
            for _ in range(args.steps):
                rc = ctx.graph_launch()
                if rc != greem.OK:
                    raise greem.GreemError(rc, "greem_graph_launch")
            e1.record(stream)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        s = ctx.stats()
        free, total = torch.cuda.mem_get_info()
        return {"metric": "full TreePM step particles/s (short-range tree force + PM)", "value": N / (ms * 1e-3),
                "unit": "particles/s", "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
                "workload": "zeldovich512+20000nfw_theta0.5_pm512_tsc", "N": N, "r_cut": prm["r_cut"], "theta": 0.5,
                "n_crit": nc, "n_pm": 512, "assign": "TSC", "graph": True,
                "N_int": s["n_interactions"] / N, "n_groups": s["n_groups"], "n_nodes": s["n_nodes"],
                "list_capacity_entries": s["list_capacity"], "kernel_launches_per_step": st["kernel_launches"],
                "device_mem_gb": (total - free) / 1e9, "generation_s": gen_s, "clocks": clk.summary()}
    finally:
        ctx.close()
        del P, M, acc
        torch.cuda.empty_cache()


def domain_grid(p: int):
    """px, py, pz with px*py*pz = p, as even as the factors allow (largest factor to the
    axis with the fewest cuts so far)."""
    fac, n, q = [], p, 2
    while n > 1:
        while n % q == 0:
            fac.append(q)
            n //= q
        q += 1
    g = [1, 1, 1]
    for f in sorted(fac, reverse=True):
        g[g.index(min(g))] *= f
    return tuple(sorted(g, reverse=True))


class CountingCompute:
    """domain.GpuCompute that adds up the kernel launches of every library call."""

    def __init__(self, ctx):
        from paper_0910_0121_gb300 import domain
        self.inner = domain.GpuCompute(ctx)
        self.ctx = ctx
        self.launches = 0

    def _count(self, out):
        self.launches += self.ctx.stats()["kernel_launches"]
        return out

    def cells(self, *a):
        return self._count(self.inner.cells(*a))

    def pack(self, *a):
        return self._count(self.inner.pack(*a))

    def let_export(self, pos, mass, prm, boxes, self_index):
        from paper_0910_0121_gb300 import greem
        self.ctx.build_tree(pos, mass, greem.params(**prm))
        self.launches += self.ctx.stats()["kernel_launches"]
        po, mo, _, counts = self.ctx.let_export(boxes, self_index)
        self.launches += self.ctx.stats()["kernel_launches"]
        return po, mo, counts

    def short_force(self, *a):
        return self._count(self.inner.short_force(*a))


def domain_arm(args, rank, world, local):
    """N > 1: the 256^3 box split over the processes as the paper does it (Sec. 2.2 steps
    3-5 and 7, Sec. 2.3.1): recursive multisection from sampled particles, first by
    particle count, then by the measured force times (Eq. 4); each timed step is every
    process's tree, LET export, LET all-to-all-v and force.  Strong scaling: the whole
    job is the one box, its time the slowest process's."""
    import torch
    import torch.distributed as dist
    from paper_0910_0121_gb300 import build as _build
    from paper_0910_0121_gb300 import domain, greem, synth

    _build.build()
    # NCCL takes one GPU per process; gloo exchanges through the host, so its processes
    # may share the GPUs there are
    torch.cuda.set_device(local if args.dist_backend == "nccl" else local % torch.cuda.device_count())
    local = torch.cuda.current_device()
    if args.dist_backend == "nccl":
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        comm = domain.TorchComm("cuda")
    else:
        dist.init_process_group("gloo")
        comm = domain.TorchComm("cpu")
    grid = domain_grid(world)
    pos, mass, prm = synth.config_zel256()
    N = len(pos)
    mine = np.arange(rank, N, world)
    P = torch.from_numpy(pos[mine].copy()).cuda()
    M = torch.from_numpy(mass[mine].copy()).cuda()
    I = torch.from_numpy(mine.astype(np.int64)).cuda()
    del mine
    stream = torch.cuda.current_stream()
    ctx = greem.Context(stream)
    comp = CountingCompute(ctx)
    fprm = dict(L=prm["L"], r_cut=prm["r_cut"], theta=prm["theta"], n_crit=args.n_crit or 192, n_leaf=10,
                list_chunk=256, block_shape=16)
    step = domain.DomainStep(comm, comp, fprm, grid, rate=4e-4, alpha=0.2, seed=synth.SEED0)
    P, M, I = step.decompose(P, M, I, N)       # by particle count
    step.force(P, M)
    P, M, I = step.decompose(P, M, I, N)       # by the measured force times (Eq. 4)
    for _ in range(max(3, args.warmup)):
        step.force(P, M)
    torch.cuda.synchronize()
    comp.launches = 0
    info = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            acc = step.force(P, M)
            info.append(dict(step.info))
        e1.record(stream)
        torch.cuda.synchronize()
    dist.barrier()
    launches = comp.launches
    ms_local = e0.elapsed_time(e1) / args.steps
    ms = max(comm.allgather_float(ms_local))
    # end to end: each step's particles in from pinned host memory and accelerations out
    hp, hm = P.cpu().pin_memory(), M.cpu().pin_memory()
    ha = torch.empty((P.shape[0], 3), dtype=torch.float32).pin_memory()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dist.barrier()
    torch.cuda.synchronize()
    f0.record(stream)
    for _ in range(args.steps):
        P.copy_(hp, non_blocking=True)
        M.copy_(hm, non_blocking=True)
        acc = step.force(P, M)
        ha.copy_(acc, non_blocking=True)
    f1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = max(comm.allgather_float(f0.elapsed_time(f1) / args.steps))
    per = {k: comm.allgather_float(statistics.mean(x[k] for x in info))
           for k in ("n_local", "n_import", "force_ms", "let_bytes_sent")}
    n_local_max = max(per["n_local"])
    line = {
        "metric": METRIC, "value": N / (ms * 1e-3), "unit": "particles/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N, "L": 1.0, "r_cut": fprm["r_cut"], "theta": fprm["theta"],
                   "n_crit": fprm["n_crit"], "n_leaf": 10, "list_chunk": 256, "block_shape": 16,
                   "l2": "inputs (470 MB) larger than L2, no flush",
                   "parallelism": f"domains {grid[0]}x{grid[1]}x{grid[2]}",
                   "dist_backend": args.dist_backend},
        "domains": {"grid": list(grid), "n_local": per["n_local"], "n_import": per["n_import"],
                    "force_ms": per["force_ms"], "let_bytes_sent": per["let_bytes_sent"],
                    "load_balance_max_over_mean_force": max(per["force_ms"]) / statistics.mean(per["force_ms"]),
                    "particles_max_over_mean": n_local_max / (N / world)},
        "e2e": {"value": N / (ms_e2e * 1e-3), "unit": "particles/s", "h2d_bytes_per_step": N * (24 + 4),
                "d2h_bytes_per_step": N * 12, "ms_per_step": ms_e2e,
                "call": "domain.DomainStep.force per process, local particles copied in and out"},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    dist.destroy_process_group()


# ----------------------------------------------------------------------------- GPU arm
def gpu_arm(args, rank, world, local):
    import torch
    from paper_0910_0121_gb300 import build as _build
    from paper_0910_0121_gb300 import greem, synth

    _build.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    pos, mass, prm = synth.config_zel256(seed=synth.SEED0 + 3 + rank)
    N = len(pos)
    P = torch.from_numpy(pos).cuda()
    M = torch.from_numpy(mass).cuda()
    acc = torch.empty((N, 3), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    ctx = greem.Context(stream)

    base = greem.params(L=prm["L"], r_cut=prm["r_cut"], theta=prm["theta"], n_crit=128, n_leaf=10)
    if args.n_crit:
        best = greem.params(L=prm["L"], r_cut=prm["r_cut"], theta=prm["theta"], n_crit=args.n_crit, n_leaf=10)
    else:
        best = ctx.autotune(P, M, base, acc, candidates=[48, 64, 96, 128, 192, 256])
    p = greem.params(L=best.L, r_cut=best.r_cut, theta=best.theta, n_crit=best.n_crit, n_leaf=best.n_leaf,
                     list_chunk=best.list_chunk, block_shape=best.block_shape, flags=greem.FLAG_STAGE_TIMES)

    for _ in range(max(3, args.warmup)):
        ctx.short_force(P, M, p, acc)
    torch.cuda.synchronize()
    st = ctx.stats()
    launches_per_step = st["kernel_launches"]
    inter = st["n_interactions"]

    # ---- timed region: device-resident inputs
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    force_ms, lists_ms, stage = [], [], {k: [] for k in ("keys", "sort", "tree", "groups", "lists", "force")}
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            ctx.short_force(P, M, p, acc)
            s = ctx.stats()
            force_ms.append(s["ms_force"])
            lists_ms.append(s["ms_lists"])
            for k in stage:
                stage[k].append(s["ms_" + k])
        e1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms, value = across_ranks(e0.elapsed_time(e1) / args.steps, N, dist, "cuda")
    clocks = clk.summary()
    # the particles whose tree force is compared with the direct sum (Sec. 3.1.2), and the
    # accelerations of the timed call (theta = 0.5) at them
    tvd_idx = np.sort(np.random.default_rng(SEED_DIRECT).choice(N, size=N_DIRECT, replace=False))
    tvd_dev = torch.from_numpy(tvd_idx).cuda()
    rows = {"idx": tvd_idx, "theta0.5": acc[tvd_dev].double().cpu().numpy()}

    # ---- end to end through the public API with host buffers: greem_short_force_host
    # copies every step's inputs in (pinned host -> device) and its result out (device ->
    # pinned host) on two more streams, beside the neighbouring steps' computation
    hpos = torch.from_numpy(pos).pin_memory()
    hmass = torch.from_numpy(mass).pin_memory()
    hacc = [torch.empty((N, 3), dtype=torch.float32).pin_memory() for _ in range(2)]
    ctx.short_force_host([hpos, hpos], [hmass, hmass], p, hacc)   # sizes the staging slots
    torch.cuda.synchronize()
    barrier()
    e2 = max(3, args.steps)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    ctx.short_force_host([hpos] * e2, [hmass] * e2, p, [hacc[k & 1] for k in range(e2)])
    f1.record(stream)   # the call returns once every result is in host memory
    torch.cuda.synchronize()
    ms_e2e, value_e2e = across_ranks(f0.elapsed_time(f1) / e2, N, dist, "cuda")

    # ---- FP64 form on the same lists, and the measured FP32 FMA peak
    p64 = greem.params(L=p.L, r_cut=p.r_cut, theta=p.theta, n_crit=p.n_crit, n_leaf=p.n_leaf,
                       precision=greem.F64, flags=greem.FLAG_STAGE_TIMES)
    acc64 = torch.empty((N, 3), dtype=torch.float64, device="cuda")
    ctx.short_force(P, M, p64, acc64)
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    ctx.short_force(P, M, p64, acc64)
    g1.record(stream)
    torch.cuda.synchronize()
    ms64 = g0.elapsed_time(g1)
    force64_ms = ctx.stats()["ms_force"]
    peak_meas = ctx.peak_tflops(0)
    pairloop = ctx.peak_tflops(2)      # the kernel's own pair loop with no list or group overhead
    sms = torch.cuda.get_device_properties(local).multi_processor_count

    # ---- roofline of the dominant kernel (S6 force): plain FP32 ALU arithmetic
    fms = statistics.mean(force_ms)
    achieved = FLOPS_PER_INTERACTION * inter / (fms * 1e-3) / 1e12
    peak = sms * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    traffic = traffic_per_launch(st["n_list_entries"])

    line = {
        "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N, "L": 1.0, "r_cut": p.r_cut, "theta": p.theta, "n_crit": p.n_crit,
                   "n_leaf": p.n_leaf, "list_chunk": p.list_chunk or 256, "block_shape": p.block_shape or 16,
                   "l2": "inputs (470 MB) larger than L2, no flush", "parallelism": "domains 1x1x1"},
        "interactions_per_s": world * inter / (ms * 1e-3),
        "N_int": inter / N,
        "force_kernel_ms": fms, "lists_kernel_ms": statistics.mean(lists_ms),
        "stage_ms": {k: round(statistics.mean(v), 3) for k, v in stage.items()},
        "n_groups": st["n_groups"], "n_nodes": st["n_nodes"], "n_list_entries": st["n_list_entries"],
        "list_walks_from_level_K": st["n_start_table"], "step_replays_a_graph": bool(st["replayed"]),
        "pct_fp32_peak_force": 100.0 * achieved / peak,
        "pct_fp32_measured_ffma_force": 100.0 * achieved / peak_meas,
        "fp32_ffma_microbench_tflops": peak_meas,
        "pair_loop_microbench_tflops": pairloop,
        "pct_of_pair_loop_force": 100.0 * achieved / pairloop,
        "fp64_form": {"ms_per_step": ms64, "force_kernel_ms": force64_ms,
                      "particles_per_s": world * N / (ms64 * 1e-3),
                      "force_speedup_fp32_vs_fp64": force64_ms / fms, "step_speedup": ms64 / ms},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "k_force_f32", "work_per_launch": f"{inter} interactions x 42 flops",
                     "peak_source": f"{sms} SMs x 128 FP32 lanes x 2 x {SM_MAX_MHZ:.0f} MHz"},
        "e2e": {"value": value_e2e, "unit": "particles/s", "h2d_bytes_per_step": N * (24 + 4),
                "d2h_bytes_per_step": N * 12, "ms_per_step": ms_e2e, "call": "greem_short_force_host",
                "steps": e2},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
    }
    if not args.no_extras:
        line["extras"] = extras(ctx, P, M, p, prm, acc, stream, rows, tvd_dev)
    if rank == 0 and not args.no_direct:
        line["tree_vs_direct"] = tree_vs_direct(pos, mass, prm, rows)
    if rank == 0 and not args.no_extras:
        line["extras"]["config1"] = guarded(config1_leg, ctx, stream)
        line["extras"]["config2"] = guarded(config2_leg, ctx, stream)
        line["extras"]["domains8"] = guarded(domains8_leg, P, M, p, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t_cpu, desc, nth, t_cpu1 = oracle_sample(pos, mass, prm, n_crit=p.n_crit)
        line["cpu_baseline"] = {"value": N / t_cpu, "unit": "particles/s", "cores": nth, "kind": "oracle",
                                "sample": desc, "one_thread": {"value": N / t_cpu1, "unit": "particles/s",
                                                               "cores": 1},
                                "paper_context": dict(PAPER_RATE, gpu_equivalent_cores=value / PAPER_RATE["value"])}
    ctx.close()
    if rank == 0 and world == 1 and not args.no_extras and not args.no_config5:
        # the 512^3 TreePM step holds about 135 GB: the 256^3 buffers go first
        del P, M, acc, acc64
        torch.cuda.empty_cache()
        line["extras"]["config5"] = guarded(config5_leg, args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def config5_arm(args):
    """--config5: the 512^3 TreePM graph of config5_leg as a line of its own."""
    from paper_0910_0121_gb300 import build as _build

    _build.build()
    leg = config5_leg(args)
    line = {k: leg[k] for k in ("metric", "value", "unit", "steps", "warmup", "ms_per_step")}
    line.update({"n_gpus": 1, "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
                 "data": "synthetic",
                 "config": {k: leg[k] for k in ("workload", "N", "r_cut", "theta", "n_crit", "n_pm", "assign",
                                                 "graph")}})
    line.update({k: v for k, v in leg.items() if k not in line and k not in line["config"]})
    print(json.dumps(line), flush=True)


def profile_case(args):
    """A bare call sequence for profiler captures: the workload's short-range force,
    --steps times, with nothing else on the device."""
    import torch
    from paper_0910_0121_gb300 import build as _build
    from paper_0910_0121_gb300 import greem, synth

    _build.build()
    pos, mass, prm = synth.config_nfw128() if args.profile_case == "nfw128" else synth.config_zel256()
    P = torch.from_numpy(pos).cuda()
    M = torch.from_numpy(mass).cuda()
    ctx = greem.Context()
    acc = torch.empty((len(pos), 3), dtype=torch.float32, device="cuda")
    p = greem.params(L=prm["L"], r_cut=prm["r_cut"], theta=0.7 if args.quad else prm["theta"],
                     n_crit=args.n_crit or 128, n_leaf=prm["n_leaf"],
                     flags=greem.FLAG_QUADRUPOLE if args.quad else 0)
    for _ in range(args.steps):
        if args.profile_case == "zel256tree":
            ctx.build_tree(P, M, p)
        else:
            ctx.short_force(P, M, p, acc)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": args.profile_case, "n_crit": p.n_crit, **ctx.stats()}), flush=True)
    ctx.close()


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.profile_case:
        profile_case(args)
        return
    if args.config5:
        config5_arm(args)
        return
    if args.impl == "reference":
        reference_arm(args, rank, world)
    elif world > 1:
        domain_arm(args, rank, world, local)
    else:
        gpu_arm(args, rank, world, local)


if __name__ == "__main__":
    main()
