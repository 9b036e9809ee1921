#!/usr/bin/env python3
"""Benchmark of the tree-gravity hot path on one GB300 (or N replicas).

Workload (default ``plummer_1m``): Plummer sphere, N = 2^20 equal masses,
eps = 1/1024, theta = 0.5, n_leaf = 16, n_grp = 256, monopole superparticles,
FP32 force kernel on FP64 particle data, indirect index lists reused over 4
kick-drift-kick steps (dt = 1/256). One bench step = one KDK timestep: kick +
drift, then force evaluation k (a construction step -- tree build + lists --
when k % 4 == 0, a reusing step otherwise), then kick.

Metric: force interactions per second (interactions = sum over i-groups of
n_i * (n_epj + n_spj)) over the timed steps, plus ms per step.

  value     device time (CUDA events on the library's stream), inputs
            resident in HBM, L2 flushed (256 MB write) between timed steps.
  e2e       the same steps through the host-array entry point
            (afd_calc_force_all_host): pinned host x, y, z, m copied in and
            the n x 4 float result copied out every step.
  roofline  the force kernel, ALU-bound: 23 flops per interaction (the
            paper's n_op) / its event-timed duration, against the FP32 peak
            152 SMs x 128 lanes x 2 flops x the median SM clock sampled
            during the timed region; the FMA rate measured by afd_fp32_peak
            is reported beside it.
  cpu_baseline  the FP64 CPU oracle on the host cores, bounded sample.

``--impl reference`` times the oracle itself on the same workload (whole
measured steps; a stated sample of the i-groups only when K + W whole steps
would take more than about two minutes) and prints its own line.
Multi-GPU (torchrun): every rank runs an independent replica of the
workload (the path has no exchange step at one tree per GPU); value is the
sum of all ranks' interactions over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FLOPS_PER_INTERACTION = 23  # n_op, Section 6.2 / Appendix A
SMS, FP32_LANES = 152, 128
# FP32 operations of the distance test k_density makes for every candidate
# pair (3 differences, 3 for r^2, 1 for q^2 = r^2 / h^2, in packed f32x2);
# the spline itself runs only for the pairs inside the support
DENSITY_OPS_PER_PAIR = 7
L2_FLUSH_BYTES = 256 << 20
# dram__bytes_read.sum + dram__bytes_write.sum of one force-kernel launch on
# this workload, from the capture summarised in profiles/ (None until taken
# on the current kernel).
FORCE_TRAFFIC_BYTES = 600_969_472  # 569.35 MB read + 31.62 MB written (k_force, --set full)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=4)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", default="plummer_1m")
    ap.add_argument("--far", type=int, choices=(0, 1, 2), default=None,
                    help="far-field precision of quadrupole superparticles: 0 fp32, 1 bf16, 2 fp16")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true",
                    help="run the reusing steps eagerly instead of replaying a captured "
                         "CUDA graph of them")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned-criterion form and the equal-error comparison")
    ap.add_argument("--mac-samples", type=int, default=1_000_000)
    ap.add_argument("--mac-epochs", type=int, default=12)
    ap.add_argument("--mac-lr", type=float, default=2e-3)
    ap.add_argument("--mac-band", default="0.4,1.0",
                    help="theta_lo,theta_hi of the learned criterion's band")
    ap.add_argument("--sweep", action="store_true",
                    help="instead of the benchmark line: theta x n_grp and n_reuse sweeps of "
                         "the workload, one JSON line per configuration")
    ap.add_argument("--shard", choices=("replica", "groups"), default="replica",
                    help="one system on N > 1 ranks: an independent replica per rank, or "
                         "disjoint slices of its i-groups with the forces combined by an "
                         "all-reduce (strong scaling)")
    ap.add_argument("--launch", default=None, metavar="WARPS,CHUNK",
                    help="fix the force kernel's block shape and list-chunk size instead of "
                         "timing the six candidates (for profiler runs, where the candidates' "
                         "event timings are not meaningful)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other workloads' summary (batched systems with the learned "
                         "criterion, the mixed-precision far field, the galaxy), each measured by a "
                         "child run of this script after the main timing")
    ap.add_argument("--sph", action="store_true",
                    help="instead of the benchmark line: the short-range neighbour walk and "
                         "gather density on the workload's particles, one line per n_grp")
    return ap.parse_args()


def workload(name):
    import ics

    wl = dict(ics.WORKLOADS[name])
    if wl["model"] == "batch":
        _, off, _ = ics.make_batch(wl["n_systems"], wl["seed"])
        wl["n"] = int(off[-1])
        wl["sys_off"] = off
    wl.setdefault("n_reuse", 4)
    wl.setdefault("dt", 1.0 / 256)
    wl["name"] = name
    return wl


def describe(wl):
    if wl["model"] == "batch":
        return (f"{wl['name']}: {wl['n_systems']} Plummer systems (N log-uniform in [2^12, 2^20], "
                f"virial ratio uniform in [0.3, 0.7]) N_total={wl['n']} eps={wl['eps']:.6g} "
                f"theta={wl['theta']} n_leaf=16 n_grp autotuned per system, monopole, one launch "
                f"per kernel over all systems, reusing steps replayed from a CUDA graph, lists "
                f"reused over {wl['n_reuse']} KDK steps dt={wl['dt']:.6g}")
    far = {0: "", 1: " (bf16 far field)", 2: " (fp16 far field)"}[wl.get("far", 0)]
    return (f"{wl['name']}: {wl['model']} N={wl['n']} eps={wl['eps']:.6g} theta={wl['theta']} "
            f"n_leaf=16 n_grp={wl['n_grp']} {'quadrupole' + far if wl['quad'] else 'monopole'} "
            f"lists reused over {wl['n_reuse']} KDK steps dt={wl['dt']:.6g}")


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "20"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self, window=None):
        """Summary of the samples taken inside window = (t0, t1) (time.time()
        seconds; all samples when none falls inside)."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        import datetime

        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                ts = None
            try:
                sm, smx = float(parts[2]), float(parts[3])
            except ValueError:
                continue
            act = {nm for nm, v in zip(names, parts[6:10]) if v.lower() == "active"}
            rows.append((ts, sm, smx, act))
        os.unlink(self.path)
        inside = [r for r in rows if window and r[0] is not None
                  and window[0] <= r[0] <= window[1]]
        use = inside or rows
        mhz = [r[1] for r in use]
        return {"sm_mhz": statistics.median(mhz) if mhz else None,
                "sm_max_mhz": max(r[2] for r in use) if use else None,
                "reasons": sorted(set().union(*(r[3] for r in use))) if use else [],
                "samples": len(use),
                "samples_in": "timed region" if inside else "sampler run (none inside the "
                                                             "timed region)"}


def particles(wl):
    import ics

    if wl["model"] == "batch":
        return ics.make_batch(wl["n_systems"], wl["seed"])[0]
    return ics.make(wl["model"], wl["n"], wl["seed"])


def shard_systems(sizes, world):
    """Independent systems over ranks: largest first, each to the rank with
    the fewest particles so far (ties to the lower rank). Returns one sorted
    list of system indices per rank; every system lands on exactly one."""
    load = [0] * world
    out = [[] for _ in range(world)]
    for s in sorted(range(len(sizes)), key=lambda k: (-int(sizes[k]), k)):
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(s)
        load[r] += int(sizes[s])
    return [sorted(o) for o in out]


def rank_batch(wl, rank, world):
    """This rank's share of a batched workload: its particles and system
    offsets (the systems are independent, so ranks need no exchange)."""
    import numpy as np

    import ics

    systems, sizes, _ = ics.batch(wl["n_systems"], wl["seed"])
    mine = shard_systems(sizes, world)[rank]
    cat = ics.Particles(*(np.concatenate([getattr(systems[k], a) for k in mine])
                          for a in ("x", "y", "z", "vx", "vy", "vz", "m")))
    off = np.concatenate([[0], np.cumsum([int(sizes[k]) for k in mine])]).astype(np.int64)
    return cat, off, mine


def combine_forces(dist, acc):
    """The whole system's forces from the ranks' disjoint group slices: each
    rank's rows of its own groups, zero elsewhere, summed over the ranks
    (x + 0 = x exactly, so every rank ends with the same bits)."""
    if dist is not None:
        dist.all_reduce(acc)


def aggregate(dist, device, ms, count):
    """Whole-job figures over ranks: the slowest rank's time, the sum of the
    units all ranks processed."""
    if dist is None:
        return ms, count
    import torch

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(count)], dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), float(c.item())


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), and nproc."""
    name = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() in ("Model name", "Model"):
                name = ln.split(":", 1)[1].strip()
                if not name.isdigit():
                    break
    except (OSError, subprocess.SubprocessError):
        pass
    if not name:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith(("model name", "cpu model")):
                    name = ln.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return name or "unknown", os.cpu_count()


def bench_config(wl, world, *, shard=False, groups_shared=False):
    """The ``config`` object of the bench line; both arms print this one."""
    return {"workload": describe(wl), "n": int(wl["n"]),
            "l2": "flushed (256 MB write) between timed steps, outside the timed events",
            "parallelism": ("systems sharded over ranks" if shard else
                            "group slices over ranks, forces all-reduced" if groups_shared
                            else "replicas") if world > 1 else "single GPU"}


def oracle_steps(wl, steps, warmup, budget_s):
    """The FP64 oracle on the host cores, timed on whole KDK steps of the
    workload: kick-drift (numpy), force evaluation k -- a new tree and lists
    when k % n_reuse == 0, else the reusing step on the kept lists -- and
    kick. Every step is measured; nothing is extrapolated. The force runs on
    every s-th i-group: s = 1 (whole steps) unless the run's estimated
    length exceeds budget_s, then the smallest power of two that fits, and
    the line states it. Returns the measured totals."""
    import numpy as np

    import ics
    import oracle

    p = particles(wl)
    label = wl["name"]
    if wl["model"] == "batch":  # the largest system stands for the batch
        off = wl["sys_off"]
        k = int(np.argmax(np.diff(off)))
        p = ics.Particles(*(getattr(p, a)[off[k]:off[k + 1]].copy()
                            for a in ("x", "y", "z", "vx", "vy", "vz", "m")))
        label = f"{wl['name']} (largest system, N={p.n})"
    kw = dict(n_grp=wl["n_grp"], theta=wl["theta"], eps=wl["eps"], quad=wl["quad"])
    R, dt = wl["n_reuse"], wl["dt"]
    x, y, z = p.x.copy(), p.y.copy(), p.z.copy()
    vx, vy, vz, m = p.vx.copy(), p.vy.copy(), p.vz.copy(), p.m
    ax = ay = az = np.zeros(p.n)
    t = None
    stride = None
    tot = {"s": 0.0, "tree_s": 0.0, "force_s": 0.0, "inter": 0.0, "inter_all": 0.0}
    for k in range(warmup + steps):
        t0 = time.perf_counter()
        vx += 0.5 * dt * ax
        vy += 0.5 * dt * ay
        vz += 0.5 * dt * az
        x += dt * vx
        y += dt * vy
        z += dt * vz
        if t is None or k % R == 0:
            t = oracle.Tree(x, y, z, m, **kw)
        else:
            t.update(x, y, z, m)
        t1 = time.perf_counter()
        g = t.groups()
        eo, _, so, _ = t.lists()
        per_group = g["count"] * ((eo[1:] - eo[:-1]) + (so[1:] - so[:-1]))
        if stride is None:  # a probe on every 16th group sets the sample
            probe = np.arange(0, len(per_group), 16)
            tp = time.perf_counter()
            t.force_groups(probe)
            rate = float(per_group[probe].sum()) / max(time.perf_counter() - tp, 1e-9)
            full = float(per_group.sum()) / rate
            tree = t1 - t0
            stride = 1
            while (warmup + steps) * (tree / R + full / stride) > budget_s and stride < 64:
                stride *= 2
            t1 = time.perf_counter()  # the probe is not part of the step
        sel = np.arange(k % stride, len(per_group), stride)
        t2 = time.perf_counter()
        fx, fy, fz, _ = t.force_groups(sel) if stride > 1 else t.force()
        if stride > 1:
            fx, fy, fz = (np.nan_to_num(a) for a in (fx, fy, fz))
        ax, ay, az = fx, fy, fz
        vx += 0.5 * dt * ax
        vy += 0.5 * dt * ay
        vz += 0.5 * dt * az
        t3 = time.perf_counter()
        if k >= warmup:
            tot["s"] += t3 - t0 - (t2 - t1)
            tot["tree_s"] += t1 - t0
            tot["force_s"] += t3 - t2
            tot["inter"] += float(per_group[sel].sum())
            tot["inter_all"] += float(per_group.sum())
    model, nproc = cpu_model()
    frac = "all i-groups" if stride == 1 else f"every {stride}th i-group"
    sample = (f"{label}: {steps} whole KDK steps after {warmup} warm-up (a new tree and lists "
              f"every {R}th step, reusing steps between), tree and integration on all N, force "
              f"on {frac}; measured {tot['s']:.2f} s for {tot['inter']:.4g} interactions "
              f"({tot['inter'] / max(tot['inter_all'], 1):.3f} of the steps' interactions), "
              f"nothing extrapolated")
    return {"value": tot["inter"] / tot["s"], "unit": "interactions/s",
            "cores": oracle.num_threads(), "cpu_model": model, "nproc": nproc,
            "kind": "oracle", "sample": sample, "ms_per_step": 1e3 * tot["s"] / steps,
            "measured_s": tot["s"], "tree_s": tot["tree_s"], "force_s": tot["force_s"],
            "group_stride": stride, "interactions_computed": tot["inter"],
            "interactions_of_whole_steps": tot["inter_all"]}


def cpu_baseline(wl):
    """The oracle on the host cores over one list-reuse window of whole
    steps (about 5-10 s of CPU work on the 2^20 workload)."""
    return oracle_steps(wl, wl["n_reuse"], 0, budget_s=30.0)


def run_reference(args, wl):
    """--impl reference: the oracle as it stands, K timed steps after W
    warm-up steps, whole steps while the run stays within about two
    minutes (a stated group sample beyond that)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    r = oracle_steps(wl, args.steps, args.warmup, budget_s=120.0)
    base = {k: r[k] for k in ("value", "unit", "cores", "cpu_model", "nproc", "kind", "sample",
                              "measured_s", "group_stride")}
    line = {
        "impl": "reference", "metric": "force interactions/s", "value": r["value"],
        "unit": "interactions/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(wl, world, shard=wl["model"] == "batch" and world > 1),
        "cpu_baseline": base,
        "e2e": {"value": r["value"], "unit": "interactions/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def other_configs(args):
    """The other workloads, each a child run of this script (its own CUDA
    context) after the main timing, summarised: the 32 batched systems with
    the learned criterion against the plain form at equal error, the 2^22
    mixed-precision far field in FP32 / BF16 / FP16, the 2^23 galaxy with
    quadrupoles."""
    runs = [("batch32", ["--workload", "batch32", "--steps", "20", "--warmup", "5"]),
            ("plummer_4m_mixed_fp32", ["--workload", "plummer_4m_mixed", "--far", "0", "--steps",
                                       "20", "--warmup", "5", "--no-learned"]),
            ("plummer_4m_mixed_bf16", ["--workload", "plummer_4m_mixed", "--far", "1", "--steps",
                                       "20", "--warmup", "5", "--no-learned"]),
            ("plummer_4m_mixed_fp16", ["--workload", "plummer_4m_mixed", "--far", "2", "--steps",
                                       "20", "--warmup", "5", "--no-learned"]),
            ("galaxy_8m", ["--workload", "galaxy_8m", "--steps", "12", "--warmup", "4",
                           "--no-learned"])]
    out = {}
    for name, extra in runs:
        cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--no-cpu-baseline", "--no-e2e",
               "--no-configs"] + extra
        t0 = time.perf_counter()
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
            lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
            if r.returncode != 0 or not lines:
                out[name] = {"error": f"rc {r.returncode}: {r.stderr.strip()[-300:]}"}
                continue
            d = json.loads(lines[-1])
        except (subprocess.SubprocessError, ValueError) as e:
            out[name] = {"error": str(e)[:300]}
            continue
        o = {"workload": d["config"]["workload"], "interactions_per_s": d["value"],
             "ms_per_step": d["ms_per_step"],
             "ms_per_construction_step": d["ms_per_construction_step"],
             "ms_per_reuse_step": d["ms_per_reuse_step"],
             "force_kernel_ms": d["roofline"]["launch_ms"], "clocks": d["clocks"],
             "wall_s": round(time.perf_counter() - t0, 1)}
        L = d.get("learned_mac")
        if L:
            o["learned"] = {"ms_per_step": L["ms_per_step"],
                            "speedup_ms_per_step_vs_plain": L["speedup_ms_per_step_vs_plain"],
                            "rms_rel_err_plain": L["equal_error"]["plain_rms_rel_err"],
                            "rms_rel_err_learned": L["equal_error"]["learned_rms_rel_err"],
                            "interactions_plain": L["equal_error"]["plain_interactions"],
                            "interactions_learned": L["equal_error"]["learned_interactions"]}
        out[name] = o
    return out


def run_loop(afd, torch, ctx, g, st, *, steps, warmup, graph, R, dt, flush, stream, dev,
             before_timed=None, combine=None, count=None):
    """Warm-up, then `steps` timed KDK steps (CUDA events around each, L2
    flushed in between). st: dict of the state tensors and the evaluation
    counter. combine (optional): makes this rank's forces (its groups' rows,
    the rest zero) the whole system's, e.g. an all-reduce; count (optional):
    this rank's interactions of a step. graph: the reusing steps replay the
    context's captured graph (kick-drift, reorder, moments, force, kick),
    captured again after each construction step while its force kernel
    runs. Returns per-step ms, force ms (the eager steps'), interactions,
    modes, launches."""
    x, y, z, vx, vy, vz, m, acc = (st[k] for k in ("x", "y", "z", "vx", "vy", "vz", "m", "acc"))

    def step():
        k = st["k"]
        mode = afd.AFD_MAKE_LIST_FOR_REUSE if k % R == 0 else afd.AFD_REUSE_LIST
        if graph and mode == afd.AFD_REUSE_LIST:
            afd.afd_graph_launch(ctx)  # kick-drift, reusing step, force, kick
        else:
            afd.afd_kick_drift(ctx, x, y, z, vx, vy, vz, acc, 0.5 * dt, dt)
            if combine:
                acc.zero_()
            afd.afd_calc_force_all(ctx, x, y, z, m, acc, mode)
            if combine:
                combine(acc)
            afd.afd_kick(ctx, vx, vy, vz, acc, 0.5 * dt)
            if graph:  # buffers may have moved: capture the new reusing step
                afd.afd_graph_capture_step(ctx, x, y, z, vx, vy, vz, m, acc, dt)
        st["k"] = k + 1
        return mode

    for _ in range(warmup):
        step()
    torch.cuda.synchronize(dev)
    if before_timed:
        before_timed()
    launches0 = g.stats()["launches"]
    step_ms, force_ms, inter, modes = [], [], [], []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mode = step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        if not (graph and mode == afd.AFD_REUSE_LIST):  # graph replays carry no events
            force_ms.append(afd.afd_last_force_ms(ctx))
        inter.append(count() if count else g.stats()["interactions"])
        modes.append(mode)
    torch.cuda.synchronize(dev)
    return step_ms, force_ms, inter, modes, g.stats()["launches"] - launches0


def learned_study(args, wl, afd, torch, np, dev, stream, local, p, tuned, launch, flush, plain):
    """The learned opening criterion against the plain theta form at equal
    rms force error (error against the FP64 direct sum of sampled
    particles): train the network on the GPU from a sphere like the N = 2^20
    workload, calibrate tau so the learned form's error matches the plain
    form's, then time the learned form's steps like the plain ones."""
    import ics

    t0 = time.perf_counter()
    lo, hi = (float(v) for v in args.mac_band.split(","))
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    batch = wl["model"] == "batch"
    R, dt = wl["n_reuse"], wl["dt"]
    base = dict(n_leaf=16, multipole=int(wl["quad"]), far_precision=int(wl.get("far", 0)))

    # ---- training samples from a sphere like the N = 2^20 workload ----
    tw = dict(ics.WORKLOADS["plummer_1m"])
    q = ics.plummer(tw["n"], tw["seed"] + 1000)
    qx = [T(a) for a in (q.x, q.y, q.z, q.m)]
    gt = afd.Gravity(afd.Config(eps=tw["eps"], theta=tw["theta"], n_grp=tw["n_grp"], mac=1,
                                **base), local, stream)
    acc_t = torch.empty(q.n, 4, dtype=torch.float32, device=dev)
    gt.force_all(*qx, acc_t, afd.AFD_MAKE_LIST)  # the plain form's |a| becomes the reference
    cap = int(args.mac_samples)
    feat = torch.empty(cap, 8, dtype=torch.float32, device=dev)
    lab = torch.empty(cap, dtype=torch.float32, device=dev)
    total = afd.afd_mac_samples(gt.ctx, lo, hi, 1.0, 0, feat[:0], lab[:0])
    keep = min(1.0, cap / max(total, 1))
    n_s = afd.afd_mac_samples(gt.ctx, lo, hi, keep, 7, feat, lab)
    n_s = min(n_s, cap)
    gt.close()
    t_samp = time.perf_counter() - t0
    epochs = int(args.mac_epochs)
    params, hist = afd.afd_mlp_train(feat[:n_s], lab[:n_s], epochs=epochs, batch=1024,
                                     lr=float(args.mac_lr),
                                     seed=5, stream=stream)
    t_train = time.perf_counter() - t0 - t_samp
    del feat, lab

    # ---- exact forces of sampled particles (FP64 direct sum per system) ----
    off = wl["sys_off"] if batch else np.array([0, p.n])
    n_sys = len(off) - 1
    per = max(1, 4096 // n_sys)
    xs0 = [T(a) for a in (p.x, p.y, p.z, p.m)]
    tg_all, ex = [], []
    for s_ in range(n_sys):
        a, b = int(off[s_]), int(off[s_ + 1])
        loc = np.unique(np.linspace(0, b - a - 1, min(per, b - a)).astype(np.int64))
        out = torch.empty(len(loc), 4, dtype=torch.float64, device=dev)
        afd.afd_direct_sum(*(v[a:b] for v in xs0),
                           torch.tensor(loc.astype(np.int32), device=dev), wl["eps"], out, stream)
        tg_all.append(loc + a)
        ex.append(out)
    tg = np.concatenate(tg_all)
    ex = torch.cat(ex).cpu().numpy()
    tg_t = torch.tensor(tg, device=dev)

    def rms_err(acc):
        a = acc[tg_t].double().cpu().numpy()
        num = ((a[:, :3] - ex[:, :3]) ** 2).sum(1)
        return float(np.sqrt(np.mean(num / (ex[:, :3] ** 2).sum(1))))

    def ctx_for(mac):
        cfg = afd.Config(eps=wl["eps"], theta=wl["theta"], n_grp=wl["n_grp"], mac=mac, **base)
        gg = afd.Gravity(cfg, local, stream)
        if batch:
            afd.afd_set_systems(gg.ctx, wl["sys_off"], tuned)
        afd.afd_set_launch(gg.ctx, *launch[:2])
        return gg

    # plain form at the initial positions; its |a| is the learned form's reference
    gp = ctx_for(0)
    acc_p = torch.empty(p.n, 4, dtype=torch.float32, device=dev)
    gp.force_all(*xs0, acc_p, afd.AFD_MAKE_LIST)
    e_plain = rms_err(acc_p)
    i_plain0 = gp.stats()["interactions"]
    gp.close()
    amag = torch.sqrt((acc_p[:, :3].double() ** 2).sum(1)).float().contiguous()

    gl = ctx_for(1)
    acc_l = torch.empty(p.n, 4, dtype=torch.float32, device=dev)

    def learned_err(tau):
        afd.afd_mac_set(gl.ctx, params, lo, hi, tau)
        afd.afd_tree_build(gl.ctx, *xs0)
        afd.afd_mac_set_reference(gl.ctx, amag)
        afd.afd_make_interaction_lists(gl.ctx, afd.AFD_MAKE_LIST)
        afd.afd_calc_force(gl.ctx, acc_l)
        return rms_err(acc_l), gl.stats()["interactions"]

    # tau: coarse grid, then bisection on log error toward e_plain
    grid = {}
    for tau in np.arange(-18.0, -6.0, 1.0):
        grid[float(tau)] = learned_err(float(tau))
    taus = sorted(grid)
    lo_t, hi_t = None, None
    for a_, b_ in zip(taus, taus[1:]):
        if grid[a_][0] <= e_plain <= grid[b_][0]:
            lo_t, hi_t = a_, b_
    if lo_t is None:  # no crossing: the most accurate tau below the plain error
        ok = [t_ for t_ in taus if grid[t_][0] <= e_plain]
        tau_star = max(ok) if ok else min(taus)
    else:
        for _ in range(6):
            mid = 0.5 * (lo_t + hi_t)
            grid[mid] = learned_err(mid)
            if grid[mid][0] <= e_plain:
                lo_t = mid
            else:
                hi_t = mid
        tau_star = lo_t  # error not above the plain form's
    e_learned, i_learned0 = grid[tau_star]
    # the learned lists are shorter: their own force-kernel launch shape,
    # timed on the calibrated lists (unless the shape is fixed by --launch)
    launch_l = launch
    if launch[2] is not None:
        learned_err(tau_star)
        launch_l = afd.afd_autotune_launch(gl.ctx, acc_l, reps=3)
    gl.close()
    t_cal = time.perf_counter() - t0 - t_samp - t_train

    # ---- the learned form timed like the plain one ----
    gl = ctx_for(1)
    afd.afd_set_launch(gl.ctx, *launch_l[:2])
    afd.afd_mac_set(gl.ctx, params, lo, hi, tau_star)
    st = {k: T(getattr(p, k)) for k in ("x", "y", "z", "vx", "vy", "vz", "m")}
    st["acc"] = torch.zeros(p.n, 4, dtype=torch.float32, device=dev)
    st["k"] = 1
    # evaluation 0 has no reference accelerations yet: theta lists; the
    # learned criterion decides every later construction step
    afd.afd_calc_force_all(gl.ctx, st["x"], st["y"], st["z"], st["m"], st["acc"],
                           afd.AFD_MAKE_LIST_FOR_REUSE)
    if not args.no_graph:
        afd.afd_graph_capture_step(gl.ctx, st["x"], st["y"], st["z"], st["vx"], st["vy"],
                                   st["vz"], st["m"], st["acc"], dt)
    step_ms, force_ms, inter, modes, launches = run_loop(
        afd, torch, gl.ctx, gl, st, steps=args.steps, warmup=args.warmup,
        graph=not args.no_graph, R=R, dt=dt, flush=flush, stream=stream, dev=dev)
    info = afd.afd_mac_info(gl.ctx)
    gl.close()
    cons = [v for v, md in zip(step_ms, modes) if md == afd.AFD_MAKE_LIST_FOR_REUSE]
    reus = [v for v, md in zip(step_ms, modes) if md == afd.AFD_REUSE_LIST]
    ms_l = float(np.mean(step_ms))
    return {
        "criterion": "8-32-32-1 network (FP16 weights, FP32 arithmetic) inside the walk for "
                     f"cells with theta_lo={lo} <= s/d < theta_hi={hi}; accepted below, opened "
                     "above; reference |a| from the previous force evaluation",
        "tau": tau_star,
        "equal_error": {"plain_rms_rel_err": e_plain, "learned_rms_rel_err": e_learned,
                        "targets": int(len(tg)), "reference": "FP64 direct sum (afd_direct_sum)",
                        "plain_interactions": i_plain0, "learned_interactions": i_learned0},
        "ms_per_step": ms_l,
        "ms_per_step_median": float(np.median(step_ms)),
        "ms_per_construction_step": float(np.mean(cons)) if cons else None,
        "ms_per_reuse_step": float(np.mean(reus)) if reus else None,
        "ms_per_construction_step_median": float(np.median(cons)) if cons else None,
        "ms_per_reuse_step_median": float(np.median(reus)) if reus else None,
        "interactions_per_step": float(np.mean(inter)),
        "interactions_per_s": float(sum(inter)) / (sum(step_ms) * 1e-3),
        "force_ms_mean": float(np.mean(force_ms)) if force_ms else None,
        "plain_ms_per_step": plain["ms_per_step"],
        "speedup_ms_per_step_vs_plain": plain["ms_per_step"] / ms_l,
        "interaction_ratio_plain_over_learned": plain["interactions_per_step"] / float(np.mean(inter)),
        "gpu_launches": launches,
        "force_launch": {"warps_per_block": launch_l[0], "chunk": launch_l[1],
                         "tuned_on": "the calibrated learned lists" if launch_l is not launch
                         else "the plain lists (--launch)"},
        "walk_network_evaluations_last_construction": info["evaluations"],
        "walk_network_accepts_last_construction": info["accepted"],
        "walk_steps_with_network_last_construction": info["rounds"],
        "training": {"samples": n_s, "band_pairs_total": total, "epochs": epochs,
                     "batch": 1024, "final_mse_log2": float(hist[-1]),
                     "first_epoch_mse_log2": float(hist[0]), "sample_s": t_samp,
                     "train_s": t_train, "calibrate_s": t_cal,
                     "data": f"Plummer N={tw['n']} seed {tw['seed'] + 1000}, eps={tw['eps']:.6g}, "
                             f"n_grp={tw['n_grp']}, reference |a| from theta={tw['theta']}"},
    }


def sph_study(wl, afd, torch, np, dev, stream, ev, T, p):
    """Short-range neighbour walk and gather density (Section 2 /
    Section 4.2) on the workload's particles with search radii for 64
    neighbours under the Plummer sphere's analytic density: per n_grp the
    list construction (cell and search boxes, walk, compaction) and the
    density kernel, CUDA events, median of five after a warm-up."""
    import ics

    xs = [T(a) for a in (p.x, p.y, p.z, p.m)]
    h = T(ics.plummer_search_radii(p, 64))
    rho = torch.empty(p.n, dtype=torch.float32, device=dev)
    nnb = torch.empty_like(rho)
    mhz = 2070.0
    for n_grp in (32, 64, 128, 256):
        g = afd.Gravity(afd.Config(eps=wl["eps"], theta=wl["theta"], n_grp=n_grp), 0, stream)
        t_tree, t_list, t_dens = [], [], []
        for rep in range(6):
            e0 = ev()
            afd.afd_tree_build(g.ctx, *xs)
            e1 = ev()
            afd.afd_make_neighbour_lists(g.ctx, h, 0.0)
            e2 = ev()
            afd.afd_calc_density(g.ctx, h, rho, nnb)
            e3 = ev()
            e3.synchronize()
            if rep:
                t_tree.append(e0.elapsed_time(e1))
                t_list.append(e1.elapsed_time(e2))
                t_dens.append(e2.elapsed_time(e3))
        st = afd.afd_neighbour_stats(g.ctx)
        gs = g.stats()
        td = float(np.median(t_dens))
        pairs_s = st["pairs"] / (td * 1e-3)
        peak_ops = SMS * FP32_LANES * mhz * 1e6
        # lists kept over steps (Section 4.2): made with a margin of a tenth of
        # the median radius, then reusing steps = reorder + density
        reuse = None
        if n_grp in (128, 256):
            skin = 0.1 * float(h.median().item())
            afd.afd_make_neighbour_lists(g.ctx, h, skin)
            st_s = afd.afd_neighbour_stats(g.ctx)
            t_re = []
            for rep in range(6):
                e0 = ev()
                afd.afd_reuse_lists(g.ctx, *xs)
                afd.afd_calc_density(g.ctx, h, rho, nnb)
                e1 = ev()
                e1.synchronize()
                if rep:
                    t_re.append(e0.elapsed_time(e1))
            reuse = {"skin": skin, "candidate_pairs": st_s["pairs"],
                     "reusing_step_ms": float(np.median(t_re))}
        print(json.dumps({
            "sweep": "sph_density", "workload": wl["name"], "n_nb_target": 64, "n_grp": n_grp,
            "groups": gs["n_groups"], "tree_ms": float(np.median(t_tree)),
            "neighbour_lists_ms": float(np.median(t_list)), "density_ms": td,
            "list_entries": st["entries"], "candidate_pairs": st["pairs"],
            "candidates_per_particle": st["pairs"] / p.n,
            "mean_smooth_neighbours": float(nnb.double().mean().item()),
            "pairs_per_s": pairs_s,
            "roofline": {"bound": "alu", "kernel": "k_density",
                         "ops_per_pair": DENSITY_OPS_PER_PAIR,
                         "achieved_ops_per_s": pairs_s * DENSITY_OPS_PER_PAIR,
                         "peak_ops_per_s": peak_ops,
                         "frac": pairs_s * DENSITY_OPS_PER_PAIR / peak_ops,
                         "peak_basis": f"{SMS} SMs x {FP32_LANES} FP32 lanes x {mhz:.0f} MHz"},
            "lists_kept": reuse}),
              flush=True)
        g.close()


def sweep(args, wl, sph_only=False):
    """The method's two knobs on this GPU (the paper's Section 6 measures the
    same dependences on its systems): for theta x n_grp, the construction
    time (tree + lists), the force-kernel time, interactions, mean group size
    <n_i> and list length, time per interaction and the rms force error
    against the FP64 direct sum of 4096 particles; then ms per KDK step for
    n_reuse in 1, 2, 4, 8, 16 (32 steps each)."""
    import numpy as np
    import torch

    import __graft_entry__

    __graft_entry__.build()
    import paper_1907_02290_gb300 as afd

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    p = particles(wl)
    n = p.n
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    xs = [T(a) for a in (p.x, p.y, p.z, p.m)]
    def ev():
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e

    if sph_only:
        sph_study(wl, afd, torch, np, dev, stream, ev, T, p)
        return
    tg = np.unique(np.linspace(0, n - 1, 4096).astype(np.int64))
    ex = torch.empty(len(tg), 4, dtype=torch.float64, device=dev)
    afd.afd_direct_sum(*xs, torch.tensor(tg.astype(np.int32), device=dev), wl["eps"], ex, stream)
    ex = ex.cpu().numpy()
    tg_t = torch.tensor(tg, device=dev)
    acc = torch.empty(n, 4, dtype=torch.float32, device=dev)

    for theta in (0.3, 0.4, 0.5, 0.6, 0.7):
        for n_grp in (32, 64, 128, 256, 512, 1024):
            cfg = afd.Config(eps=wl["eps"], theta=theta, n_leaf=16, n_grp=n_grp,
                             multipole=int(wl["quad"]))
            g = afd.Gravity(cfg, 0, stream)
            afd.afd_set_launch(g.ctx, 2, 32)
            t_cons, t_force = [], []
            for rep in range(4):
                e0 = ev()
                afd.afd_tree_build(g.ctx, *xs)
                afd.afd_make_interaction_lists(g.ctx, afd.AFD_MAKE_LIST_FOR_REUSE)
                e1 = ev()
                afd.afd_calc_force(g.ctx, acc)
                e2 = ev()
                e2.synchronize()
                if rep:  # the first pass warms up
                    t_cons.append(e0.elapsed_time(e1))
                    t_force.append(e1.elapsed_time(e2))
            st = g.stats()
            a = acc[tg_t].double().cpu().numpy()
            err = float(np.sqrt(np.mean(((a[:, :3] - ex[:, :3]) ** 2).sum(1)
                                        / (ex[:, :3] ** 2).sum(1))))
            tf = float(np.median(t_force))
            print(json.dumps({
                "sweep": "theta_n_grp", "workload": wl["name"], "theta": theta, "n_grp": n_grp,
                "construction_ms": float(np.median(t_cons)), "force_ms": tf,
                "interactions": st["interactions"], "groups": st["n_groups"],
                "mean_n_i": n / st["n_groups"],
                "mean_list": (st["n_epj"] + st["n_spj"]) / st["n_groups"],
                "ns_per_interaction": 1e6 * tf / st["interactions"],
                "rms_rel_force_error": err}), flush=True)
            g.close()

    # the non-indirect ablation: j-data copied into list order every
    # evaluation (the copy must follow the particles), then read without
    # indices; the indirect kernel reads the same data by index
    cfg = afd.Config(eps=wl["eps"], theta=wl["theta"], n_leaf=16, n_grp=wl["n_grp"])
    g = afd.Gravity(cfg, 0, stream)
    afd.afd_set_launch(g.ctx, 2, 32)
    afd.afd_tree_build(g.ctx, *xs)
    afd.afd_make_interaction_lists(g.ctx, afd.AFD_MAKE_LIST_FOR_REUSE)
    t_ind, t_copy, t_dir = [], [], []
    for rep in range(6):
        e0 = ev()
        afd.afd_calc_force(g.ctx, acc)
        e1 = ev()
        e1.synchronize()
        c_ms, f_ms = afd.afd_calc_force_materialized(g.ctx, acc)
        if rep:
            t_ind.append(e0.elapsed_time(e1))
            t_copy.append(c_ms)
            t_dir.append(f_ms)
    st = g.stats()
    print(json.dumps({"sweep": "indirect_ablation", "workload": wl["name"], "theta": wl["theta"],
                      "n_grp": wl["n_grp"], "list_entries": st["n_epj"] + st["n_spj"],
                      "indirect_force_ms": float(np.median(t_ind)),
                      "materialize_ms": float(np.median(t_copy)),
                      "materialized_force_ms": float(np.median(t_dir)),
                      "materialized_bytes": 32 * (st["n_epj"] + st["n_spj"])}), flush=True)
    g.close()

    # local essential tree: the domain x >= 0 exports to the domain x < 0; a
    # tree over x < 0 plus the imports gives the forces there
    A = p.x < 0.0
    B = ~A
    box = [p.x[A].min(), p.y[A].min(), p.z[A].min(), p.x[A].max(), p.y[A].max(), p.z[A].max()]
    cfg = afd.Config(eps=wl["eps"], theta=wl["theta"], n_leaf=16, n_grp=wl["n_grp"])
    gb = afd.Gravity(cfg, 0, stream)
    afd.afd_tree_build(gb.ctx, T(p.x[B]), T(p.y[B]), T(p.z[B]), T(p.m[B]))
    t_let = []
    for rep in range(4):
        e0 = ev()
        lx, ly, lz, lm, lk = afd.afd_let_export(gb.ctx, box, wl["theta"])
        e1 = ev()
        e1.synchronize()
        if rep:
            t_let.append(e0.elapsed_time(e1))
    gb.close()
    na = int(A.sum())
    ga = afd.Gravity(cfg, 0, stream)
    afd.afd_set_launch(ga.ctx, 2, 32)
    XA = [torch.cat([T(getattr(p, k)[A]), v]) for k, v in zip("xyzm", (lx, ly, lz, lm))]
    acc_a = torch.empty(len(XA[0]), 4, dtype=torch.float32, device=dev)
    ga.force_all(*XA, acc_a, afd.AFD_MAKE_LIST)
    ia = np.nonzero(A)[0]
    sel = np.isin(tg, ia)
    pos = np.searchsorted(ia, tg[sel])
    a = acc_a[torch.tensor(pos, device=dev)].double().cpu().numpy()
    exa = ex[sel]
    err_split = float(np.sqrt(np.mean(((a[:, :3] - exa[:, :3]) ** 2).sum(1)
                                      / (exa[:, :3] ** 2).sum(1))))
    ga.close()
    print(json.dumps({"sweep": "let_split", "workload": wl["name"], "theta": wl["theta"],
                      "exporting_particles": int(B.sum()), "exported_elements": int(len(lm)),
                      "exported_superparticles": int(lk.sum().item()),
                      "export_ms": float(np.median(t_let)), "receiving_particles": na,
                      "rms_rel_force_error_split": err_split}), flush=True)

    sph_study(wl, afd, torch, np, dev, stream, ev, T, p)

    R_list = (1, 2, 4, 8, 16)
    for R in R_list:
        cfg = afd.Config(eps=wl["eps"], theta=wl["theta"], n_leaf=16, n_grp=wl["n_grp"],
                         multipole=int(wl["quad"]))
        g = afd.Gravity(cfg, 0, stream)
        afd.afd_set_launch(g.ctx, 2, 32)
        st = {k: T(getattr(p, k)) for k in ("x", "y", "z", "vx", "vy", "vz", "m")}
        st["acc"] = torch.zeros(n, 4, dtype=torch.float32, device=dev)
        st["k"] = 1
        afd.afd_calc_force_all(g.ctx, st["x"], st["y"], st["z"], st["m"], st["acc"],
                               afd.AFD_MAKE_LIST_FOR_REUSE)
        flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
        step_ms, _, inter, _, _ = run_loop(afd, torch, g.ctx, g, st, steps=32, warmup=R,
                                           graph=False, R=R, dt=wl["dt"], flush=flush,
                                           stream=stream, dev=dev)
        print(json.dumps({"sweep": "n_reuse", "workload": wl["name"], "n_reuse": R,
                          "theta": wl["theta"], "n_grp": wl["n_grp"],
                          "ms_per_step": float(np.mean(step_ms)),
                          "interactions_per_step": float(np.mean(inter))}), flush=True)
        g.close()


def main():
    args = parse()
    wl = workload(args.workload)
    if args.far is not None:
        wl["far"] = args.far
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args, wl)
        return
    if args.sweep or args.sph:
        if rank == 0:
            sweep(args, wl, sph_only=args.sph)
        return

    import numpy as np
    import torch

    import __graft_entry__

    __graft_entry__.build()
    import ics
    import paper_1907_02290_gb300 as afd

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)  # a capturable (non-default) stream
    torch.cuda.set_stream(stream)
    shard = None
    config = bench_config(wl, world, shard=wl["model"] == "batch" and world > 1,
                          groups_shared=args.shard == "groups" and world > 1
                          and wl["model"] != "batch")
    if wl["model"] == "batch" and world > 1:  # independent systems: shard them
        p, wl["sys_off"], shard = rank_batch(wl, rank, world)
        wl["n_systems"] = len(shard)
        wl["n"] = p.n
    else:  # one system: every rank runs a replica
        p = particles(wl)
    n = p.n
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    x, y, z, vx, vy, vz, m = (T(a) for a in (p.x, p.y, p.z, p.vx, p.vy, p.vz, p.m))
    acc = torch.zeros(n, 4, dtype=torch.float32, device=dev)
    cfg = afd.Config(eps=wl["eps"], theta=wl["theta"], n_leaf=16, n_grp=wl["n_grp"],
                     multipole=int(wl["quad"]), far_precision=int(wl.get("far", 0)))
    g = afd.Gravity(cfg, local, stream)
    ctx = g.ctx
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    dt, R = wl["dt"], wl["n_reuse"]
    batch = wl["model"] == "batch"
    tuned = None
    if batch:
        afd.afd_set_systems(ctx, wl["sys_off"])
        tuned = afd.afd_autotune_n_grp(ctx, x, y, z, m, acc, [32, 64, 128, 256, 512], R,
                                       n_sys=wl["n_systems"])

    # one system over several ranks by group slices: each rank computes its
    # part of the groups, the forces are combined by an all-reduce
    groups_shared = args.shard == "groups" and world > 1 and not batch
    combine = count = None
    if groups_shared:
        afd.afd_set_work_share(ctx, rank, world)
        combine = lambda a: combine_forces(dist, a)
        count = lambda: afd.afd_get_work_share(ctx)["interactions"]

    afd.afd_calc_force_all(ctx, x, y, z, m, acc, afd.AFD_MAKE_LIST_FOR_REUSE)  # evaluation 0
    # force-kernel block shape and list-chunk size, timed on these lists
    if args.launch:
        w_fix, ch_fix = (int(v) for v in args.launch.split(","))
        afd.afd_set_launch(ctx, w_fix, ch_fix)
        launch = (w_fix, ch_fix, None)
    else:
        launch = afd.afd_autotune_launch(ctx, acc, reps=3)
    if groups_shared:
        acc.zero_()
    afd.afd_calc_force(ctx, acc)  # evaluation 0's forces for the first kick
    if groups_shared:
        combine(acc)
    use_graph = not args.no_graph and not groups_shared  # (the all-reduce is not captured)
    if use_graph:
        afd.afd_graph_capture_step(ctx, x, y, z, vx, vy, vz, m, acc, dt)
    state = {"x": x, "y": y, "z": z, "vx": vx, "vy": vy, "vz": vz, "m": m, "acc": acc, "k": 1}
    sampler = ClockSampler(local)
    t_wall = [0.0, 0.0]

    def before_timed():
        if dist:
            dist.barrier()
        sampler.start()
        time.sleep(0.3)
        t_wall[0] = time.perf_counter()
        t_wall[1] = time.time()

    step_ms, force_ms, inter, modes, launches = run_loop(
        afd, torch, ctx, g, state, steps=args.steps, warmup=args.warmup, graph=use_graph, R=R,
        dt=dt, flush=flush, stream=stream, dev=dev, before_timed=before_timed, combine=combine,
        count=count)
    t_epoch = (t_wall[1], time.time())
    t_wall = time.perf_counter() - t_wall[0]
    clocks = sampler.stop(t_epoch)
    total_ms = float(sum(step_ms))
    total_i = float(sum(inter))
    total_ms, total_i_all = aggregate(dist, dev, total_ms, total_i)
    value = total_i_all / (total_ms * 1e-3)

    # ---- roofline of the force kernel ----
    if not force_ms:  # no eager step in a short timed region: time the kernel on its own
        for _ in range(3):
            flush.zero_()
            afd.afd_calc_force(ctx, acc)
            force_ms.append(afd.afd_last_force_ms(ctx))
    f_ms = float(np.mean(force_ms)) if force_ms else float("nan")
    i_launch = float(np.mean(inter))
    achieved = FLOPS_PER_INTERACTION * i_launch / (f_ms * 1e-3) / 1e12
    mhz = clocks.get("sm_mhz") or 2070.0
    peak = SMS * FP32_LANES * 2 * mhz * 1e6 / 1e12
    measured = afd.afd_fp32_peak(local, stream)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": FORCE_TRAFFIC_BYTES,
                "measured_fp32_fma_tflops": measured,
                "frac_of_measured_fma": achieved / measured,
                "kernel": "k_force", "flops_per_interaction": FLOPS_PER_INTERACTION,
                "interactions_per_launch": i_launch, "launch_ms": f_ms,
                "peak_basis": f"{SMS} SMs x {FP32_LANES} FP32 lanes x 2 x {mhz:.0f} MHz "
                              "(median SM clock sampled during the timed region)"}
    cons = [s for s, md in zip(step_ms, modes) if md == afd.AFD_MAKE_LIST_FOR_REUSE]
    reus = [s for s, md in zip(step_ms, modes) if md == afd.AFD_REUSE_LIST]

    # ---- end to end through the host-array entry point ----
    e2e = None
    if not args.no_e2e and not groups_shared:
        hx, hy, hz, hm = (torch.tensor(a, dtype=torch.float64).pin_memory()
                          for a in (p.x, p.y, p.z, p.m))
        hacc = torch.zeros(n, 4, dtype=torch.float32).pin_memory()
        g2 = afd.Gravity(cfg, local, stream)
        afd.afd_set_launch(g2.ctx, *launch[:2])
        if batch:
            afd.afd_set_systems(g2.ctx, wl["sys_off"], tuned)
        afd.afd_calc_force_all_host(g2.ctx, hx, hy, hz, hm, hacc, afd.AFD_MAKE_LIST_FOR_REUSE)
        for k in range(1, args.warmup + 1):
            afd.afd_calc_force_all_host(g2.ctx, hx, hy, hz, hm, hacc,
                                        afd.AFD_MAKE_LIST_FOR_REUSE if k % R == 0
                                        else afd.AFD_REUSE_LIST)
        if dist:
            dist.barrier()
        e_i, t0 = 0.0, time.perf_counter()
        for k in range(args.warmup + 1, args.warmup + 1 + args.steps):
            afd.afd_calc_force_all_host(g2.ctx, hx, hy, hz, hm, hacc,
                                        afd.AFD_MAKE_LIST_FOR_REUSE if k % R == 0
                                        else afd.AFD_REUSE_LIST)
            e_i += g2.stats()["interactions"]
        e_s = time.perf_counter() - t0
        e_s, e_i = aggregate(dist, dev, e_s, e_i)
        e2e = {"value": e_i / e_s, "unit": "interactions/s", "h2d_bytes_per_step": 4 * 8 * n,
               "d2h_bytes_per_step": 16 * n, "ms_per_step": 1e3 * e_s / args.steps,
               "call": "afd_calc_force_all_host: per step the force evaluation with its "
                       "copies (x, y, z, m in from pinned memory; the n x 4 floats out written "
                       "into the pinned output by the force kernel over the host link); the kick "
                       "and drift that value's steps include are not in it (device kernels, about "
                       "1% of a step)"}
        g2.close()

    if rank != 0:
        g.close()
        if dist:
            dist.destroy_process_group()
        return
    line = {
        "metric": "force interactions/s", "value": value, "unit": "interactions/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "strong" if (shard is not None or groups_shared) else "weak",
        "vs_baseline": None, "dtype": "f32",
        "dtype_detail": "force kernel FP32 (hi/lo group-relative coordinates); tree, "
                        "moments and integration FP64",
        "data": "synthetic (seeded " + {"plummer": "Plummer sphere", "batch": "Plummer spheres",
                                        "uniform_sphere": "cold uniform sphere",
                                        "galaxy": "halo + disk galaxy"}.get(wl["model"],
                                                                            wl["model"]) + ")",
        "config": config,
        "ms_per_step_median": float(np.median(step_ms)),
        "ms_per_construction_step": float(np.mean(cons)) if cons else None,
        "ms_per_reuse_step": float(np.mean(reus)) if reus else None,
        "ms_per_construction_step_median": float(np.median(cons)) if cons else None,
        "ms_per_reuse_step_median": float(np.median(reus)) if reus else None,
        "interactions_per_step": total_i / args.steps,
        "roofline": roofline,
        "clocks": clocks,
        "gpu_launches": launches,
        "reusing_steps": ("replayed from a CUDA graph of the step (afd_graph_capture_step after "
                          "each construction step, afd_graph_launch); the force kernel's time "
                          "from the construction steps' events" if use_graph else "eager"),
        "n_grp_autotuned": None if tuned is None else [int(v) for v in tuned],
        "force_launch_autotuned": ({"warps_per_block": launch[0], "chunk": launch[1],
                                    "ms_chunk32_w2_4_8": [float(v) for v in launch[2][0]],
                                    "ms_chunk64_w2_4_8": [float(v) for v in launch[2][1]]}
                                   if launch[2] is not None else
                                   {"warps_per_block": launch[0], "chunk": launch[1],
                                    "fixed": "--launch"}),
        "wall_s_timed_region": t_wall,
    }
    if e2e:
        line["e2e"] = e2e
    elif groups_shared:
        line["e2e_skipped"] = ("group slices: a rank's host-array call computes its slice only; "
                               "the forces are combined on the device")
    if not args.no_learned and world == 1 and not wl["quad"]:
        line["learned_mac"] = learned_study(args, wl, afd, torch, np, dev, stream, local, p,
                                            tuned, launch, flush, line)
    if not args.no_configs and world == 1 and args.workload == "plummer_1m" and args.far is None:
        g.close()
        line["configs"] = other_configs(args)
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(wl)
    print(json.dumps(line))
    g.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
