#!/usr/bin/env python
"""Benchmark of the Hermite block-timestep force path on GB300.

Workload (the force sweep the headline metric is quoted on): Plummer model,
N = 16384, seed 2, eps = 1/256, standard N-body units.  One bench step is one
full block step of the Hermite scheme (select -> predict -> force -> correct,
steps 1-8 of Sec. 2) for each active-block size n_act in {32, 256, 2048,
16384}; before each block step the state is restored on the device so every
step does identical work.  The active block of size n_act is the first n_act
particles of a seeded permutation (their dt is 2^-10, everyone else's 2^-4).

Four precision modes run the same timed step: MIXED (the paper's scheme on
FP32 pipes), HYBRID (FP32 far pairs, double-single near pairs), DS
(double-single pair arithmetic) and FP64.  Each is checked on every particle
against the FP64 CPU oracle (evaluated by the CPU-baseline leg on rank 0
before any GPU work); the headline value is acc+jerk interactions per second
(n_act * N per block step, self pair counted) of the fastest mode whose
largest relative error in acc, jerk and pot is <= 1e-6.  Every mode's launch
shapes are autotuned on the workload first.  The force kernel's roofline, an
end-to-end figure through host buffers, the CPU oracle baseline and the
paper's own mixed-precision CPU loop are reported on the same JSON line.

Under torchrun (--gpus N > 1) every rank runs an independent replica of the
workload on its own GPU (weak scaling); the timed region is bracketed by a
barrier and the slowest rank's time is used.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1104_2700_gb300 import ics  # noqa: E402

METRIC = "acc+jerk interactions/s on 1 GB300, mixed vs FP64, at rel. force err ≤1e-6"
UNIT = "interactions/s"
FLOPS_PER_INTERACTION = 60  # the paper's convention (Sec. 5)
CROSSING_TIME = 2.0 * math.sqrt(2.0)  # one crossing time in N-body units (Sec. 4)
ENERGY_STUDY_T_END = 0.375  # the span of Sec. 4's energy test, as the paper states it
NACTS = ics.FORCE_SWEEP_NACT
WL = ics.FORCE_SWEEP_N16K
L2_FLUSH_BYTES = 512 << 20


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-extra", action="store_true",
                   help="skip the N = 65536 roofline and the ensemble measurement")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--modes", default="mixed,hybrid,ds,fp64",
                   help="comma-separated precision modes to time")
    p.add_argument("--profile", choices=["mixed", "hybrid", "ds", "fp64"], default=None,
                   help="only run --launches force launches (for ncu), no timing")
    p.add_argument("--profile-nact", type=int, default=16384)
    p.add_argument("--profile-n", type=int, choices=[16384, 65536], default=16384,
                   help="the profiled workload: the N = 16384 sweep (a random active "
                        "list) or the N = 65536 roofline workload (every particle, in the "
                        "context's spatial order, no noise history)")
    p.add_argument("--profile-steps", choices=["sweep", "ensemble"], default=None,
                   help="only run a few eager HYBRID block steps of the N = 16384 "
                        "workload or the 256-system ensemble (for ncu), no timing")
    p.add_argument("--profile-shape", default="0,0,0",
                   help="i per thread, j split, CTAs per SM of the profiled launch "
                        "(0 = the default)")
    p.add_argument("--launches", type=int, default=3)
    p.add_argument("--integrate", choices=sorted(INTEGRATIONS), default=None,
                   help="instead of the sweep: integrate one workload in --modes "
                        "(default ds,fp64) to --t-end and report steps, rate, energy drift")
    p.add_argument("--t-end", type=float, default=None,
                   help="end time for --integrate (a multiple of dt_max = 1/16)")
    p.add_argument("--energy-study", action="store_true",
                   help="instead of the sweep: energy error against step count over "
                        "eta (Sec. 4, Fig. err_itg): Plummer N = 1024, eps = 4/N, "
                        "t = 0 -> 0.375")
    p.add_argument("--jerk-energy-study", action="store_true",
                   help="instead of the sweep: the N = 262144 Plummer + Salpeter model "
                        "(eps = 1e-4) integrated to t = 1/8 with the far-field jerk summed "
                        "in runs folded into double-single sums (hybrid) and in one plain "
                        "FP32 sum (hybrid_spj): block steps and energy drift (Sec. 4)")
    p.add_argument("--jerk-study", action="store_true",
                   help="instead of the sweep: error distributions of acc, jerk, pot "
                        "with the jerk summed in FP32 or compensated (Sec. 4, "
                        "Fig. err_snp_djerk), Plummer N = 1K, 4K, 16K, 64K")
    return p.parse_args()


def kernel_source_hash():
    """sha256 (first 16 hex) of what the force kernel is built from:
    csrc/force_kernel.cuh, force.cu, force_cta.cu, nb_device.cuh and
    nb_launch.h with comments and whitespace stripped (so that a comment edit
    does not orphan the ncu summaries taken of the same code), plus the
    force translation units' compiler flags."""
    import hashlib
    import re
    from paper_1104_2700_gb300 import build as nb_build
    h = hashlib.sha256()
    for f in ("force_kernel.cuh", "force.cu", "force_cta.cu", "nb_device.cuh", "nb_launch.h"):
        with open(os.path.join(ROOT, "paper_1104_2700_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    flags = nb_build.COMMON + nb_build.PER_FILE.get("force.cu", [])
    h.update(" ".join(x for x in flags if not x.startswith("/")).encode())
    return h.hexdigest()[:16]


def profiled_metric(prec, key="traffic_bytes_per_launch", shape=None, n=16384):
    """A figure of the force launch at n_act = N from the committed ncu summary
    of the N = n workload (DRAM bytes per launch, thread instructions per
    interaction), or None when the kernel sources changed since it was
    captured or it was captured with another kernel shape (i per thread, j
    split) than `shape`; the CTAs per SM only change how far the j range
    splits over warps."""
    import re
    path = os.path.join(ROOT, "profiles", f"force_{prec}_n{n}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    h = re.search(r"source_hash:\s*([0-9a-f]+)", text)
    t = re.search(key + r":\s*([0-9.]+)", text)
    if not h or not t or h.group(1) != kernel_source_hash():
        return None
    if shape is not None:
        sh = re.search(r"launch_shape:\s*([0-9]+),([0-9]+),([0-9]+)", text)
        if not sh or tuple(int(x) for x in sh.groups())[:2] != tuple(shape)[:2]:
            return None
    return float(t.group(1))


def run_profile_steps(args):
    """Load a workload in HYBRID and run eight eager block steps (for ncu
    captures of the select, predictor and corrector kernels)."""
    from paper_1104_2700_gb300 import build as nb_build
    from paper_1104_2700_gb300 import nbody
    nb_build.build()
    with nbody.Context("hybrid") as ctx:
        if args.profile_steps == "ensemble":
            sizes, off, ms, rs, vs, eps = ics.ensemble()
            ctx.set_ensemble(off, ms, rs, vs, eps, ics.ENSEMBLE_K256["eta"])
            n = int(off[-1])
        else:
            m, r, v = WL.particles()
            ctx.set_particles(m, r, v, WL.eps, WL.eta)
            n = WL.n
        for _ in range(8):
            ctx.block_step(1.0)
        ctx.synchronize()
    print(json.dumps({"profile_steps": args.profile_steps, "n": n, "block_steps": 8}))


def run_profile(args):
    """A few force launches of one precision on the sweep workload or the
    N = 65536 roofline workload (for ncu)."""
    import torch
    from paper_1104_2700_gb300 import build as nb_build
    from paper_1104_2700_gb300 import nbody
    nb_build.build()
    wl = WL if args.profile_n == 16384 else ics.MIXED_N64K
    n, eps = wl.n, wl.eps
    m, r, v = wl.particles()
    it, split, cps = (int(x) for x in args.profile_shape.split(","))
    with nbody.Context(args.profile, i_per_thread=it, j_split=split, ctas_per_sm=cps) as ctx:
        # loading evaluates every force once (the launch ncu skips with -s 1)
        # and leaves a, j in the state for the hybrid near-pair test
        ctx.set_particles(m, r, v, eps, wl.eta)
        # the state reloaded, so that no noise history arms the hybrid guard:
        # the state the bench times (its sweep blocks and roofline launches)
        st = ctx.get_state()
        ctx.set_state(m, st["r"], st["v"], st["a"], st["j"], st["t"], st["dt"], eps, wl.eta)
        if args.profile_n == 16384:
            # a block of the sweep, listed as the bench lists it: in the
            # context's spatial order
            members = ics.permutation(n, WL.seed)[:args.profile_nact]
            rank = np.empty(n, dtype=np.int64)
            rank[ctx.spatial_order()] = np.arange(n)
            members = members[np.argsort(rank[members])]
        else:
            # as the bench's roofline: every particle in the spatial order
            members = ctx.spatial_order()
        idx = torch.from_numpy(np.asarray(members).astype(np.int32)).cuda()
        ctx.predict(0.0)
        for _ in range(args.launches):
            ctx.force(idx)
        ctx.synchronize()
    print(json.dumps({"profile": args.profile, "n": n, "n_act": len(members),
                      "launches": args.launches, "shape": [it, split, cps]}))


# --- distributed plumbing -------------------------------------------------------
def dist_setup(backend):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend=backend)
    return rank, local, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --- clocks ---------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows
                                   if r[3].replace(".", "").isdigit()) if rows else None}


# --- workload -------------------------------------------------------------------
def block_states(base, perm):
    """Per n_act: the state whose scheduler picks the first n_act of perm."""
    n = len(base["m"])
    out = []
    for k in NACTS:
        dt = np.full(n, 2.0 ** -4)
        dt[perm[:k]] = 2.0 ** -10
        st = dict(base)
        st["t"] = np.zeros(n)
        st["dt"] = dt
        out.append(st)
    return out


def to_device(st, torch, dev):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k, v in st.items()}


def to_pinned(st, torch):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in st.items()}


def run_ours(args):
    import torch
    from paper_1104_2700_gb300 import build as nb_build
    from paper_1104_2700_gb300 import nbody

    rank, local, world = dist_setup("nccl" if args.gpus > 1 else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    nb_build.build()
    # One explicit stream carries the library's kernels, the L2 flush and the
    # timing events (the legacy default stream has handle 0, which the
    # library would replace by a private stream).
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)

    n, eps, eta = WL.n, WL.eps, WL.eta
    m, r, v = WL.particles()
    perm = ics.permutation(n, WL.seed)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    inter_per_step = sum(k * n for k in NACTS)
    all_idx = np.arange(n, dtype=np.int32)

    def forces_at_t0(ctx, a0, j0):
        # the state's a, j matter only to the hybrid precision's near-pair test
        ctx.set_state(m, r, v, a0, j0, np.zeros(n), np.full(n, 1.0 / 16), eps, eta)
        ctx.predict(0.0)
        return ctx.force(all_idx)

    # Accuracy reference of every gate on the line: the FP64 oracle, run on
    # rank 0 by the CPU-baseline leg (which also times it) before any GPU work.
    leg = None
    if rank == 0:
        leg = cpu_baseline_leg(m, r, v, eps, args.cpu_seconds,
                               timed=not args.no_cpu_baseline, extra=not args.no_extra)
    ref = leg["refs"]["sweep"] if leg else None

    def accuracy(ctx):
        """Every particle of the workload against the oracle (rank 0 only)."""
        if ref is None:
            return None
        a, j, p = forces_at_t0(ctx, ref[0], ref[1])
        return error_stats((a, j, p), ref)

    def measure(precision, steps, warmup):
        ctx = nbody.Context(precision, device=local, stream=stream)
        ctx.set_particles(m, r, v, eps, eta)
        ctx.tuning = ctx.autotune()  # launch shapes measured on this workload
        base = ctx.get_state()
        base["m"] = m
        states = block_states({k: base[k] for k in ("m", "r", "v", "a", "j")}, perm)
        dstates = [to_device(s, torch, dev) for s in states]
        # one device snapshot per block: the step rolls the state back with
        # nb_restore (a single copy kernel) before each block step
        snaps = []
        for s in dstates:
            ctx.set_state(s["m"], s["r"], s["v"], s["a"], s["j"], s["t"], s["dt"], eps, eta)
            buf = torch.empty(ctx.snapshot_bytes() // 8, dtype=torch.float64, device=dev)
            ctx.snapshot(buf)
            snaps.append(buf)
        ctx.snaps = snaps

        def enqueue_step():
            for buf in snaps:
                ctx.restore(buf)
                ctx.block_step(1.0)

        # Every call above is stream-ordered and device-resident, so the whole
        # step is captured once as a CUDA graph and replayed (one launch per
        # step instead of ~100 host calls).
        enqueue_step()
        ctx.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            enqueue_step()
        torch.cuda.set_stream(stream)
        for _ in range(warmup):
            graph.replay()
        ctx.synchronize()
        barrier(world)
        torch.cuda.synchronize(dev)
        times = []
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            graph.replay()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        ctx.synchronize()
        torch.cuda.synchronize(dev)
        barrier(world)
        total = reduce_max(sum(times), world, dev)
        del graph
        return ctx, states, dstates, total

    def timed_forces(ctx, buf, idx, reps):
        """Average force-launch duration (CUDA events around each launch).
        Each launch starts from the block's snapshot, as in the timed step:
        no far-field noise estimate yet, so the hybrid integration guard is
        idle (it needs the history of an integration, which a sweep block
        does not have)."""
        total = 0.0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for r in range(reps + 3):
            ctx.restore(buf)
            e0.record(stream)
            ctx.force(idx)
            e1.record(stream)
            e1.synchronize()
            if r >= 3:
                total += e0.elapsed_time(e1) / 1e3
        return total / reps

    def spatial_list(ctx, members):
        """`members` (particle indices) as the block step lists them: in the
        context's spatial order (the order the force kernel's i-groups are
        cut in), as a device tensor."""
        order = ctx.spatial_order()
        rank = np.empty(n, dtype=np.int64)
        rank[order] = np.arange(n)
        members = np.asarray(members)
        return torch.from_numpy(members[np.argsort(rank[members])].astype(np.int32)).to(dev)

    def force_launch_time(ctx, reps=20):
        """Average duration of one force launch with n_act = N."""
        ctx.restore(ctx.snaps[-1])
        ctx.predict(0.0)
        idx_all = spatial_list(ctx, np.arange(n))
        return timed_forces(ctx, ctx.snaps[-1], idx_all, reps)

    def breakdown(ctx, dstates, reps=50):
        """Per block size, warm CUDA-event times (us) of: the state roll-back
        alone (nb_restore, bench scaffolding), roll-back + one block step,
        roll-back + the force call on that block's active list (all three as
        replayed CUDA graphs, as the timed step runs), and the force call
        issued eagerly from Python (host overhead included)."""
        out = {}
        for k, buf in zip(NACTS, ctx.snaps):
            ctx.restore(buf)
            ctx.predict(0.0)
            idx_k = spatial_list(ctx, perm[:k])

            def restore():
                ctx.restore(buf)

            def step():
                restore()
                ctx.block_step(1.0)

            def force():
                restore()
                ctx.force(idx_k)

            row = {}
            for name, fn in (("restore_us", restore), ("restore_and_block_step_us", step),
                             ("restore_and_force_us", force)):
                fn()
                ctx.synchronize()
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=stream):
                    fn()
                torch.cuda.set_stream(stream)
                for _ in range(3):
                    g.replay()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    g.replay()
                e1.record(stream)
                e1.synchronize()
                row[name] = e0.elapsed_time(e1) * 1e3 / reps
                del g
            row["force_us"] = row["restore_and_force_us"] - row["restore_us"]
            row["force_us_eager"] = timed_forces(ctx, buf, idx_k, reps) * 1e6
            row["block_step_us"] = row["restore_and_block_step_us"] - row["restore_us"]
            row["non_force_us"] = row["block_step_us"] - row["force_us"]
            out[str(k)] = row
        return out

    modes = {}
    contexts = {}
    clocks = ClockSampler(local)
    wanted = [x.strip() for x in args.modes.split(",") if x.strip()]
    if args.no_fp64 and "fp64" in wanted:
        wanted.remove("fp64")
    # the headline mode runs exactly --steps; FP64 (~60x slower) runs a tenth
    order = [(p, args.steps if p != "fp64" else max(2, args.steps // 10)) for p in wanted]
    clk = None
    for prec, k in order:
        sampler = ClockSampler(local)
        sampler.start()
        ctx, states, dstates, total = measure(prec, k, args.warmup)
        c = sampler.stop()
        t_force = force_launch_time(ctx)
        per_nact = breakdown(ctx, dstates) if prec != "fp64" else None
        acc = accuracy(ctx)
        modes[prec] = {"value": world * inter_per_step * k / total, "unit": UNIT, "steps": k,
                       "ms_per_step": 1e3 * total / k,
                       "force_launch_ms_nact_N": t_force * 1e3,
                       "autotuned_launch": ctx.tuning,
                       "force_interactions_per_s": n * n / t_force,
                       "per_block_size": per_nact,
                       "accuracy_vs_oracle": acc, "clocks": c}
        contexts[prec] = (ctx, states)
    gate = None
    if rank == 0:
        gate = {p: mo["accuracy_vs_oracle"]["max_rel"] <= 1e-6 for p, mo in modes.items()}
    if world > 1:
        import torch.distributed as dist
        box = [gate]
        dist.broadcast_object_list(box, src=0)
        gate = box[0]
    passing = [p for p in modes if gate[p]]
    # fastest mode meeting the gate; if none ran that meets it, the fastest
    # mode (its line then records meets_1e-6_gate = false)
    pool = passing or list(modes)
    head = max(pool, key=lambda p: modes[p]["value"])
    hm = modes[head]
    for p in modes:
        modes[p]["meets_1e-6_gate"] = gate[p]

    props = torch.cuda.get_device_properties(dev)
    clk = hm["clocks"]
    sm_max = clk.get("sm_max_mhz") or 2070.0
    peak32 = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
    # Measured FMA throughput (FP32 and FP64 chains on every SM), outside any
    # timed region: a cross-check of the derived peak, and the FP64 denominator.
    meas = {}
    try:
        meas["fp32"], meas["fp64"] = nbody.measure_peaks(dev.index)
    except nbody.NbError as exc:
        meas["error"] = str(exc)

    def large_shape(p):
        t = modes[p].get("autotuned_launch") or {}
        return (t.get("large_i_per_thread", 1), t.get("large_j_split", 1),
                t.get("large_ctas_per_sm", 0))

    def kernel_name(p):
        it, split, cps = large_shape(p)
        pol = {"mixed": "Mixed", "ds": "DS", "hybrid": "Hybrid", "fp64": "FP64"}[p]
        return (f"force_kernel<Policy{pol}<{it}>, IT={it}, j_split={split}, UniformPlan> "
                f"({cps} CTAs/SM)")

    def roofline_of(p, kernel):
        ach = FLOPS_PER_INTERACTION * modes[p]["force_interactions_per_s"] / 1e12
        ipi = profiled_metric(p, "thread_instructions_per_interaction", large_shape(p))
        issue = None
        if ipi:
            # one warp instruction per clock per SM sub-partition (4 per SM)
            peak_ti = props.multi_processor_count * 4 * 32 * sm_max * 1e6
            ach_ti = ipi * modes[p]["force_interactions_per_s"]
            issue = {"thread_instructions_per_interaction": ipi,
                     "achieved_per_s": ach_ti, "peak_per_s": peak_ti, "frac": ach_ti / peak_ti,
                     "basis": "ncu smsp__inst_executed.sum x 32 / interactions (same kernel "
                              "source hash); peak = SMs x 4 schedulers x 32 lanes x max clock"}
        if p == "fp64":
            pk, basis = meas.get("fp64"), "measured DFMA throughput (nb_measure_peaks, this run)"
            return {"bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                    "frac": (ach / pk) if pk else None, "kernel": kernel, "peak_basis": basis,
                    "launch_ms": modes[p]["force_launch_ms_nact_N"], "issue": issue}
        return {"bound": "alu", "achieved": ach, "peak": peak32, "unit": "TFLOP/s",
                "frac": ach / peak32, "traffic": profiled_metric(p, shape=large_shape(p)),
                "kernel": kernel,
                "peak_measured": meas.get("fp32"),
                "frac_of_measured": (ach / meas["fp32"]) if meas.get("fp32") else None,
                "issue": issue,
                "traffic_source": f"profiles/force_{p}_n16384.md (ncu, kernel source "
                                  f"hash {kernel_source_hash()}, launch shape "
                                  f"{','.join(str(x) for x in large_shape(p))}; null if the "
                                  f"kernel source or its i-tile / j split differs)",
                "algorithmic_bytes_per_launch": algorithmic_bytes(p, n, n),
                "algorithmic_bytes_basis": ALGO_BYTES_BASIS,
                "launch_ms": modes[p]["force_launch_ms_nact_N"],
                "peak_basis": f"{props.multi_processor_count} SMs x 128 FP32 lanes x 2 flop x "
                              f"{sm_max:.0f} MHz max SM clock (derived; peak_measured is this "
                              f"run's FFMA-chain throughput); "
                              f"60 flop per interaction (paper convention)"}

    roofline = roofline_of(head, kernel_name(head))
    roofline_mixed = roofline_of("mixed", kernel_name("mixed")) if "mixed" in modes else None
    if "fp64" in modes:
        modes["fp64"]["roofline"] = roofline_of("fp64", kernel_name("fp64"))

    # End to end through the public API with host buffers: every step copies
    # the state in from pinned host memory and the corrected state back out.
    e2e = None
    if not args.no_e2e:
        ctx, states = contexts[head]
        hst = [to_pinned(s, torch) for s in states]
        outs = {k: torch.empty((n, 3), dtype=torch.float64).pin_memory() for k in ("r", "v", "a", "j")}
        outs.update({k: torch.empty(n, dtype=torch.float64).pin_memory() for k in ("t", "dt")})
        lib = nbody

        def e2e_step():
            for s in hst:
                st = lib.nb_set_state(ctx.handle, n, *[ctypes_ptr(s[k]) for k in
                                                       ("m", "r", "v", "a", "j", "t", "dt")],
                                      eps, eta, 0)
                assert st == 0, lib.nb_last_error(ctx.handle)
                ctx.block_step(1.0)
                st = lib.nb_get_state(ctx.handle, *[ctypes_ptr(outs[k]) for k in
                                                    ("r", "v", "a", "j", "t", "dt")], 0)
                assert st == 0, lib.nb_last_error(ctx.handle)

        ke = max(2, min(args.steps, 200))
        for _ in range(min(args.warmup, 3)):
            e2e_step()
        barrier(world)
        torch.cuda.synchronize(dev)
        w0 = time.perf_counter()
        for _ in range(ke):
            e2e_step()
        torch.cuda.synchronize(dev)
        w = reduce_max(time.perf_counter() - w0, world, dev)
        e2e = {"value": world * inter_per_step * ke / w, "unit": UNIT, "steps": ke,
               "precision": head,
               "h2d_bytes_per_step": len(NACTS) * n * 8 * (1 + 12 + 2),
               "d2h_bytes_per_step": len(NACTS) * n * 8 * (12 + 2)}
    for ctx, _ in contexts.values():
        ctx.close()

    extra = {}
    if not args.no_extra:
        extra = extra_measurements(nbody, torch, dev, stream, world, peak32,
                                   leg["refs"] if leg else None)

    cpu = cpu_paper = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = leg["cpu"]
        cpu_paper = paper_cpu_baseline(m, r, v, eps, args.cpu_seconds / 2, ref)

    if rank == 0:
        line = {
            "metric": METRIC, "value": hm["value"], "unit": UNIT, "n_gpus": world,
            "steps": hm["steps"], "warmup": args.warmup, "ms_per_step": hm["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[head], "data": "synthetic",
            "config": {"workload": WL.name, "n": n, "n_act": list(NACTS), "eps": eps,
                       "seed": WL.seed, "precision": head, "parallelism": f"replicas{world}",
                       "step": "select+predict+force+correct per n_act, state rolled back "
                               "on the device (nb_restore) before each, whole step replayed "
                               "as one CUDA graph",
                       "l2": "flushed (512 MiB write) between timed steps",
                       "interactions_per_step": inter_per_step,
                       "gflops_60flop": hm["value"] * FLOPS_PER_INTERACTION / 1e9,
                       "gate": "max over all N particles of rel. err of acc, jerk, pot "
                               "against the FP64 oracle <= 1e-6"},
            "roofline": roofline,
            "roofline_mixed_kernel": roofline_mixed,
            "modes": modes,
            "fp64_speedup": (hm["value"] / modes["fp64"]["value"]) if "fp64" in modes else None,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "cpu_paper_kernel": cpu_paper,
            "gpu_launches": LAUNCHES_PER_BLOCK_STEP * len(NACTS) * hm["steps"],
            "clocks": clk,
            **extra,
        }
        print(json.dumps(line), flush=True)


def error_stats(got, ref):
    """Relative errors of (acc, jerk, pot) against a reference (the oracle's):
    |x - x_ref| / |x_ref| per particle (Sec. 4's error definition)."""
    a, j, p = got
    a0, j0, p0 = ref
    ea = np.linalg.norm(a - a0, axis=1) / np.linalg.norm(a0, axis=1)
    ej = np.linalg.norm(j - j0, axis=1) / np.linalg.norm(j0, axis=1)
    ep = np.abs(p - p0) / np.abs(p0)
    return {"particles": int(len(ea)),
            "acc_rel_max": float(ea.max()), "acc_rel_p50": float(np.median(ea)),
            "acc_rel_p99": float(np.quantile(ea, 0.99)),
            "jerk_rel_max": float(ej.max()), "jerk_rel_p50": float(np.median(ej)),
            "jerk_rel_p99": float(np.quantile(ej, 0.99)),
            "pot_rel_max": float(ep.max()),
            "max_rel": float(max(ea.max(), ej.max(), ep.max())),
            "n_above_1e-6": int(np.sum((ea > 1e-6) | (ej > 1e-6) | (ep > 1e-6))),
            "reference": "FP64 CPU oracle"}


# Algorithmic DRAM bytes of one force launch: the j layout once (bytes per j
# record), and per active i its layout record, its index, the state it reads
# (HYBRID: a, j, dt and the noise estimate for the near test and the guard)
# and the acc, jerk, pot it writes (HYBRID also its noise estimate).
J_RECORD_BYTES = {"mixed": 40, "mixed_spj": 40, "ds": 64, "hybrid": 64, "fp64": 64}
I_BYTES = {"mixed": 40 + 4 + 56, "mixed_spj": 40 + 4 + 56, "ds": 64 + 4 + 56,
           "fp64": 64 + 4 + 56, "hybrid": 64 + 4 + 64 + 56 + 8}
ALGO_BYTES_BASIS = ("n_j x j-record bytes (mixed 40, ds/hybrid/fp64 64) + n_act x (i record + "
                    "4 B index + 56 B acc/jerk/pot written; hybrid also 48 B state a, j + "
                    "8 B dt + 8 B noise estimate read and 8 B written)")


def algorithmic_bytes(prec, n_j, n_act):
    return n_j * J_RECORD_BYTES[prec] + n_act * I_BYTES[prec]



# Kernels of one graph-replayed block step of the sweep (N = 16384): the
# state roll-back (nb_restore), the one-CTA select (systems up to 32768
# particles), predict, the two force launch variants (each returns at once
# outside its n_act window), correct.
LAUNCHES_PER_BLOCK_STEP = 6
DTYPES = {"ds": "f32x2 (double-single on the FP32 pipes)", "mixed": "f32", "fp64": "f64",
          "mixed_spj": "f32", "hybrid_spj": "f32 (far pairs) + f32x2 double-single (near pairs)",
          "hybrid": "f32 (far pairs) + f32x2 double-single (near pairs)"}


def extra_measurements(nbody, torch, dev, stream, world, peak32, refs):
    """Context beside the headline (not part of `value`):
    * the force kernel at n_act = N for N = 65536 (Plummer, the size the
      FP32-roofline target is stated for) and N = 262144 (Plummer with
      Salpeter masses, eps = 1e-4), in MIXED, HYBRID and DS (CUDA events),
      each with its errors against the oracle on 256 random + the 64 most
      central particles (rank 0);
    * the 256-system ensemble (log-uniform N in [256, 8192], eps = 4/N)
      integrated from t = 0 to 1 in one HYBRID context: total interactions
      per second of the whole integration and per-system energy drift; DS to
      t = 1/16 beside it; and 16 sampled members integrated together to
      t = 1/16 against the oracle's integration of each alone;
    * block steps, smallest timestep and energy drift of short integrations
      in every mode (MIXED's timestep collapse)."""
    out = {}

    def force_roofline(wl, key, modes):
        m, r, v = wl.particles()
        n = wl.n
        acc = torch.empty((n, 3), dtype=torch.float64, device=dev)
        jerk = torch.empty((n, 3), dtype=torch.float64, device=dev)
        pot = torch.empty(n, dtype=torch.float64, device=dev)
        res = {"workload": wl.name, "n": n, "eps": wl.eps,
               "state": "a, j and dt from the load evaluation, no far-field noise history "
                        "(as the sweep's blocks: the hybrid integration guard idle); every "
                        "particle active, listed in the context's spatial order"}

        def time_force(ctx, idx, snap=None):
            """Mean force-launch time (CUDA events around each launch); with
            `snap`, the state is rolled back to it before every launch, so
            each evaluation starts from the same noise history."""
            reps = max(2, min(5, int(4e11 // (n * n))))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            total = 0.0
            for rep in range(reps + 1):
                if snap is not None:
                    ctx.restore(snap)
                ctx.predict(0.0)
                e0.record(stream)
                ctx.force(idx, acc, jerk, pot)
                e1.record(stream)
                e1.synchronize()
                if rep > 0:
                    total += e0.elapsed_time(e1) / 1e3
            return total / reps

        for prec in modes:
            with nbody.Context(prec, device=dev.index, stream=stream) as ctx:
                # loading evaluates every force once and leaves a, j in the
                # state, which the hybrid near-pair test reads
                ctx.set_particles(m, r, v, wl.eps, wl.eta)
                tun = ctx.autotune()
                order = ctx.spatial_order()
                idx = torch.from_numpy(order).to(dev)
                t_guard = None
                if prec == "hybrid":
                    snap = torch.empty(ctx.snapshot_bytes() // 8 + 1, dtype=torch.float64,
                                       device=dev)
                    ctx.snapshot(snap)
                    t_guard = time_force(ctx, idx, snap)
                # reloading the same state clears the noise history
                st = ctx.get_state()
                ctx.set_state(m, st["r"], st["v"], st["a"], st["j"], st["t"], st["dt"],
                              wl.eps, wl.eta)
                snap = torch.empty(ctx.snapshot_bytes() // 8 + 1, dtype=torch.float64, device=dev)
                ctx.snapshot(snap)
                t = time_force(ctx, idx, snap)
            ach = FLOPS_PER_INTERACTION * n * n / t / 1e12
            row = {"bound": "alu", "achieved": ach, "peak": peak32, "unit": "TFLOP/s",
                   "frac": ach / peak32, "launch_ms": t * 1e3,
                   "interactions_per_s": n * n / t, "autotuned_launch": tun,
                   "algorithmic_bytes_per_launch": algorithmic_bytes(prec, n, n)}
            # the committed ncu summary of this launch, when its kernel source
            # and shape are this run's (else null)
            shape = (tun["large_i_per_thread"], tun["large_j_split"])
            row["traffic"] = profiled_metric(prec, shape=shape, n=n)
            row["thread_instructions_per_interaction"] = profiled_metric(
                prec, "thread_instructions_per_interaction", shape, n=n)
            if row["traffic"] is not None:
                row["traffic_source"] = f"profiles/force_{prec}_n{n}.md"
            if t_guard is not None:
                row["launch_ms_right_after_load"] = t_guard * 1e3
                row["right_after_load_note"] = (
                    "the first evaluation after nb_set_particles, with the noise history "
                    "of the load's own evaluation: the integration guard sends particles "
                    "whose start-rule timestep is short to double-single")
            if refs is not None and key in refs:
                sidx, ref = refs[key]
                rows = np.empty(n, dtype=np.int64)
                rows[order] = np.arange(n)  # output row of each particle
                sel = rows[sidx]
                got = (acc.cpu().numpy()[sel], jerk.cpu().numpy()[sel], pot.cpu().numpy()[sel])
                row["accuracy_vs_oracle"] = error_stats(got, ref)
                row["accuracy_vs_oracle"]["sample"] = "256 random + the 64 most central particles"
                row["meets_1e-6_gate"] = row["accuracy_vs_oracle"]["max_rel"] <= 1e-6
            res[prec] = row
        return res

    out["roofline_n65536"] = force_roofline(ics.MIXED_N64K, "n65536", ("mixed", "hybrid", "ds"))
    out["salpeter_n262144"] = force_roofline(ics.SALPETER_N256K, "n262144",
                                             ("mixed", "hybrid", "ds"))

    kw = {k: ics.ENSEMBLE_K256[k] for k in ("k", "size_seed", "member_seed0")}
    sizes, off, ms, rs, vs, eps = ics.ensemble(**kw)
    eta = ics.ENSEMBLE_K256["eta"]
    ens = {"systems": int(len(sizes)), "particles": int(off[-1]),
           "precision_note": "hybrid and DS: with FP32 pair arithmetic (MIXED) the "
                             "Aarseth timesteps collapse (see precision_ablation)"}
    # t_end is a multiple of dt_max = 1/16, so every particle ends synchronised
    # and the per-system energies are those of one time
    for prec, t_end in (("hybrid", 1.0), ("ds", 1.0 / 16)):
        with nbody.Context(prec, device=dev.index, stream=stream) as ctx:
            ctx.set_ensemble(off, ms, rs, vs, eps, eta)
            tun = ctx.autotune()
            ctx.set_ensemble(off, ms, rs, vs, eps, eta)
            k0, w0 = ctx.energy_systems(fp64_potential=True)
            torch.cuda.synchronize(dev)
            w0c = time.perf_counter()
            steps, inter = ctx.step_until(t_end)
            torch.cuda.synchronize(dev)
            w = time.perf_counter() - w0c
            k1, w1 = ctx.energy_systems(fp64_potential=True)
            de = np.abs((k1 + w1) - (k0 + w0)) / np.abs(k0 + w0)
            ens[prec] = {"t_end": t_end, "value": world * inter / w, "unit": UNIT,
                         "block_steps": int(steps), "interactions": int(inter), "wall_s": w,
                         "us_per_block_step": 1e6 * w / max(steps, 1),
                         "rel_energy_drift_max": float(de.max()),
                         "rel_energy_drift_p50": float(np.median(de)),
                         "autotuned_launch": tun}
    if refs is not None and "ensemble16" in refs:
        ens["oracle_check_16"] = ensemble_oracle_check(nbody, dev, stream, refs["ensemble16"])
    out["ensemble_k256"] = ens
    # Precision ablation of the integration (Sec. 4 measures energy error
    # against step count in mixed and DP): block steps, smallest timestep and
    # energy drift from t = 0 to 1/64 in each mode.  The N = 256 system is
    # member 119 of the ensemble: a particle there with |a| = 0.1, |j| = 80
    # (nearly cancelling pair forces) drives MIXED into a timestep collapse.
    abl = {"t_end": 1.0 / 64}
    wl1 = ics.FP64_N1K
    m1, r1, v1 = wl1.particles()
    q = 119
    cases = {"plummer_n1024_eps1/64": (m1, r1, v1, wl1.eps),
             "plummer_n%d_eps4/n_ensemble_member%d" % (sizes[q], q):
                 (ms[off[q]:off[q + 1]], rs[off[q]:off[q + 1]], vs[off[q]:off[q + 1]], float(eps[q]))}
    for name, (m1, r1, v1, e1) in cases.items():
        row = {}
        for prec in ("fp64", "ds", "hybrid", "mixed", "mixed_spj"):
            # dt_max = t_end, so that every particle ends synchronised at t_end
            with nbody.Context(prec, device=dev.index, stream=stream, dt_max=1.0 / 64) as ctx:
                ctx.set_particles(m1, r1, v1, e1, 0.02)
                k0, w0 = ctx.energy(fp64_potential=True)
                s0 = ctx.get_state()
                steps, inter = ctx.step_until(1.0 / 64)
                k1, w1 = ctx.energy(fp64_potential=True)
                s1 = ctx.get_state()
                row[prec] = {"block_steps": int(steps), "interactions": int(inter),
                             "log2_min_dt_start": float(np.log2(s0["dt"].min())),
                             "log2_min_dt_end": float(np.log2(s1["dt"].min())),
                             "rel_energy_drift": abs((k1 + w1) - (k0 + w0)) / abs(k0 + w0)}
        abl[name] = row
    out["precision_ablation"] = abl
    return out


def ensemble_oracle_check(nbody, dev, stream, ref):
    """16 ensemble members integrated together (one HYBRID context) to
    t = 1/16, each against the oracle's integration of that member alone:
    energy drift ratio, final position / velocity differences, share of
    particles on the oracle's timestep, total interactions."""
    pick, off, m, r, v, eps, t_end, orc = ref
    with nbody.Context("hybrid", device=dev.index, stream=stream) as ctx:
        ctx.set_ensemble(off, m, r, v, eps, ics.ENSEMBLE_K256["eta"])
        steps, inter = ctx.step_until(t_end)
        k1, w1 = ctx.energy_systems(fp64_potential=True)
        st = ctx.get_state()
    rows = []
    for q in range(len(pick)):
        lo, hi = off[q], off[q + 1]
        o = orc[q]
        de = abs(k1[q] + w1[q] - o["e0"]) / abs(o["e0"])
        rows.append({"member": int(pick[q]), "n": int(hi - lo), "rel_energy_drift": float(de),
                     "oracle_rel_energy_drift": o["de"],
                     "drift_ratio": float(de / o["de"]) if o["de"] > 0 else None,
                     "max_abs_dr": float(np.max(np.abs(st["r"][lo:hi] - o["r"]))),
                     "max_abs_dv": float(np.max(np.abs(st["v"][lo:hi] - o["v"]))),
                     "same_dt_share": float(np.mean(st["dt"][lo:hi] == o["dt"]))})
    orc_inter = sum(o["inter"] for o in orc)
    ok = all(x["rel_energy_drift"] <= 2 * x["oracle_rel_energy_drift"] + 1e-13 and
             x["max_abs_dr"] < 1e-6 and x["max_abs_dv"] < 1e-5 and x["same_dt_share"] >= 0.95
             for x in rows) and abs(inter / orc_inter - 1) <= 0.05
    return {"t_end": t_end, "members": [int(x) for x in pick], "block_steps": int(steps),
            "interactions": int(inter), "oracle_interactions": float(orc_inter),
            "max_drift_ratio": max(x["drift_ratio"] or 0.0 for x in rows),
            "max_abs_dr": max(x["max_abs_dr"] for x in rows),
            "max_abs_dv": max(x["max_abs_dv"] for x in rows),
            "min_same_dt_share": min(x["same_dt_share"] for x in rows),
            "gate": "per member: drift <= 2x oracle's (+1e-13), |dr| < 1e-6, |dv| < 1e-5, "
                    ">= 95 % on the oracle's dt; interactions within 5 %",
            "meets_gate": bool(ok), "rows": rows}


def ctypes_ptr(t):
    import ctypes
    return ctypes.c_void_p(t.data_ptr())


# --- CPU baseline: the oracle as it stands ------------------------------------------
def cpu_baseline_leg(m, r, v, eps, seconds, timed=True, extra=True):
    """The CPU-baseline leg (rank 0, before any GPU work): the FP64 oracle,
    as it stands, on the host cores.  Its outputs are also the reference of
    every accuracy gate on the bench line:
      * "sweep": every particle of the N = 16384 workload at t = 0 (timed as
        one whole-workload sample);
      * "n65536", "n262144": 256 random + the 64 most central particles of
        the N = 65536 and N = 262144 (Salpeter) workloads at t = 0;
      * "ensemble16": 16 members of the ensemble workload, each integrated
        alone to t = 1/16.
    With `timed`, the repeated-sample timing of the oracle force follows."""
    from oracle import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    n = len(m)
    out = {"refs": {}, "samples": {}}
    t0 = time.perf_counter()
    out["refs"]["sweep"] = oracle.force(m, r, v, eps, nthreads=cores)
    dt = time.perf_counter() - t0
    out["samples"]["sweep_all_particles"] = {"value": n * n / dt, "unit": UNIT, "wall_s": dt,
                                             "cores": cores}
    if extra:
        for key, wl in (("n65536", ics.MIXED_N64K), ("n262144", ics.SALPETER_N256K)):
            mm, rr, vv = wl.particles()
            sidx = ics.gate_sample(rr, wl.seed)
            out["refs"][key] = (sidx, oracle.force(mm, rr, vv, wl.eps, idx=sidx, nthreads=cores))
        t_end = 1.0 / 16
        pick, off, ms, rs, vs, es = ics.ensemble_subset(16, 2048)
        orc = []
        t0 = time.perf_counter()
        for q in range(len(pick)):
            lo, hi = off[q], off[q + 1]
            st = oracle.State(ms[lo:hi], rs[lo:hi], vs[lo:hi], float(es[q]),
                              ics.ENSEMBLE_K256["eta"], nthreads=cores)
            e0 = st.energy()
            status = st.run(t_end)
            if status != oracle.OK:
                raise RuntimeError(f"oracle integration of member {pick[q]} failed: {status}")
            orc.append({"e0": e0, "de": abs(st.energy() - e0) / abs(e0), "r": st.r.copy(),
                        "v": st.v.copy(), "dt": st.dt.copy(), "inter": st.n_inter})
        dt = time.perf_counter() - t0
        out["refs"]["ensemble16"] = (pick, off, ms, rs, vs, es, t_end, orc)
        inter = sum(o["inter"] for o in orc)
        out["samples"]["ensemble16_integration"] = {
            "value": inter / dt, "unit": UNIT, "wall_s": dt, "cores": cores,
            "sample": "16 ensemble members (N <= 2048) each integrated alone to t = 1/16"}
    if timed:
        out["cpu"] = cpu_baseline(m, r, v, eps, seconds)
        out["cpu"]["other_samples"] = out["samples"]
    return out


def cpu_baseline(m, r, v, eps, seconds):
    from oracle import oracle
    n = len(m)
    cores = os.cpu_count() or 1
    perm = ics.permutation(n, 5)
    probe = perm[:max(cores, 32)]
    t0 = time.perf_counter()
    oracle.force(m, r, v, eps, idx=probe, nthreads=cores)
    dt = time.perf_counter() - t0
    k = int(min(n, max(len(probe), seconds / max(dt, 1e-9) * len(probe))))
    sample = perm[:k]
    reps = 0
    t0 = time.perf_counter()
    while True:  # the whole sample, repeated until the time budget is used
        oracle.force(m, r, v, eps, idx=sample, nthreads=cores)
        reps += 1
        dt = time.perf_counter() - t0
        if dt >= 0.5 * seconds:
            break
    inter = reps * k * n
    # one core: the same oracle on a sample sized for ~3 s at the measured
    # per-core rate
    per_particle_1core = dt * cores / (reps * k)
    k1 = int(max(16, min(n, 3.0 / max(per_particle_1core, 1e-12))))
    t0 = time.perf_counter()
    oracle.force(m, r, v, eps, idx=perm[:k1], nthreads=1)
    dt1 = time.perf_counter() - t0
    return {"value": inter / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle force (Eqs. acc, jrk, pot) on {k} of the {n} particles "
                      f"against all {n} j, x{reps}, OpenMP over i, {dt:.1f} s",
            "gflops_60flop": inter / dt * FLOPS_PER_INTERACTION / 1e9,
            "one_core": {"value": k1 * n / dt1, "unit": UNIT,
                         "gflops_60flop": k1 * n / dt1 * FLOPS_PER_INTERACTION / 1e9,
                         "sample": f"{k1} of the {n} particles against all j, 1 thread, "
                                   f"{dt1:.1f} s"},
            "cpu_model": cpu_model()}


# --- second CPU baseline: the paper's own mixed-precision loop ---------------------
def paper_cpu_baseline(m, r, v, eps, seconds, ref):
    """The paper's force loop (Sec. 3.2-3.3: DP relative positions, SP pair
    arithmetic, DP acc/pot sums, SP jerk sums, 2 i x 4 j per vector) on the
    host cores, on the same workload: all cores and one core, plus its
    accuracy on the sample against the FP64 reference."""
    from baseline import paper_cpu
    n = len(m)
    cores = os.cpu_count() or 1
    lay = paper_cpu.Layout(m, r, v)
    perm = ics.permutation(n, 5).astype(np.int32)
    probe = perm[:max(2 * cores, 64)]
    t0 = time.perf_counter()
    lay.force(eps, probe, nthreads=cores)
    dt = time.perf_counter() - t0
    k = int(min(n, max(len(probe), seconds / 2 / max(dt, 1e-9) * len(probe))))
    sample = perm[:k]
    reps = 0
    t0 = time.perf_counter()
    while True:
        acc, jerk, pot = lay.force(eps, sample, nthreads=cores)
        reps += 1
        dt = time.perf_counter() - t0
        if dt >= 0.5 * seconds:
            break
    per_particle_1core = dt * cores / (reps * k)
    k1 = int(max(16, min(n, 2.0 / max(per_particle_1core, 1e-12))))
    t0 = time.perf_counter()
    lay.force(eps, perm[:k1], nthreads=1)
    dt1 = time.perf_counter() - t0
    a_ref, j_ref, p_ref = (x[sample] for x in ref)
    ea = np.linalg.norm(acc - a_ref, axis=1) / np.linalg.norm(a_ref, axis=1)
    ej = np.linalg.norm(jerk - j_ref, axis=1) / np.linalg.norm(j_ref, axis=1)
    ep = np.abs(pot - p_ref) / np.abs(p_ref)
    value = reps * k * n / dt
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "paper_mixed_simd",
            "openmp": paper_cpu.has_openmp(),
            "sample": f"mixed-precision loop of Sec. 3.2-3.3 (GCC vector extensions, "
                      f"no -march) on {k} of the {n} particles against all j, x{reps}, "
                      f"OpenMP over i pairs, {dt:.1f} s",
            "gflops_60flop": value * FLOPS_PER_INTERACTION / 1e9,
            "one_core": {"value": k1 * n / dt1, "unit": UNIT,
                         "gflops_60flop": k1 * n / dt1 * FLOPS_PER_INTERACTION / 1e9,
                         "sample": f"{k1} of the {n} particles, 1 thread, {dt1:.1f} s"},
            "accuracy_vs_oracle": {"particles": k,
                                 "acc_rel_p50": float(np.median(ea)),
                                 "acc_rel_max": float(ea.max()),
                                 "jerk_rel_p50": float(np.median(ej)),
                                 "jerk_rel_max": float(ej.max()),
                                 "pot_rel_max": float(ep.max())}}


def cpu_model():
    """The host CPU's name: lscpu's model name, else /proc/cpuinfo."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def run_reference(args):
    """The FP64 oracle timed on the host cores on a bounded sample of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle
    oracle.build()
    n, eps = WL.n, WL.eps
    m, r, v = WL.particles()
    perm = ics.permutation(n, WL.seed)
    cores = os.cpu_count() or 1
    # each step: the force sweep with every block capped at 64 i particles
    blocks = [perm[:min(k, 64)] for k in NACTS]
    inter = sum(len(b) * n for b in blocks)

    def step():
        for b in blocks:
            oracle.force(m, r, v, eps, idx=b, nthreads=cores)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = inter * args.steps / dt
    sample = (f"force sweep N={n} with each active block capped at 64 i "
              f"({inter} interactions per step), FP64 oracle, OpenMP over i")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WL.name, "n": n, "n_act": list(NACTS), "eps": eps,
                   "seed": WL.seed, "precision": "fp64-oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# Integration workloads (Plummer, standard N-body units) and their end times.
INTEGRATIONS = {"c1": ("FP64_N1K", 0.5), "c3": ("MIXED_N64K", 1.0),
                "c5": ("SALPETER_N256K", 0.25)}


def run_integration(args):
    """Block-step integration of one workload from t = 0 to t_end in each
    precision mode: block steps, interactions per second of the whole run
    (wall clock around nb_step_until, CUDA-synchronised), the smallest
    timestep reached and the relative energy drift with the FP64 potential
    (Sec. 4 measures the energy error the same way).  For the N = 1024
    workload the FP64 oracle runs the same integration on the host cores as
    the CPU baseline ("cpu_baseline", kind "oracle")."""
    name, t_default = INTEGRATIONS[args.integrate]
    wl = getattr(ics, name)
    t_end = args.t_end if args.t_end is not None else t_default
    if t_end <= 0 or (t_end * 16) != int(t_end * 16):
        raise SystemExit("--t-end must be a positive multiple of 1/16")
    import torch
    from paper_1104_2700_gb300 import build as nb_build
    from paper_1104_2700_gb300 import nbody
    nb_build.build()
    modes = [x for x in args.modes.split(",") if x] if args.modes != "mixed,hybrid,ds,fp64" \
        else ["hybrid", "ds", "fp64"]
    m, r, v = wl.particles()
    out = {"metric": "block-step integration interactions/s", "unit": UNIT,
           "workload": wl.name, "n": wl.n, "eps": wl.eps, "eta": wl.eta, "t_end": t_end,
           "data": "synthetic", "modes": {}}
    for prec in modes:
        with nbody.Context(prec) as ctx:
            ctx.set_particles(m, r, v, wl.eps, wl.eta)
            k0, w0 = ctx.energy(fp64_potential=True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            steps, inter = ctx.step_until(t_end)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            k1, w1 = ctx.energy(fp64_potential=True)
            st = ctx.get_state()
            out["modes"][prec] = {
                "block_steps": int(steps), "interactions": int(inter), "wall_s": wall,
                "value": inter / wall, "log2_min_dt": float(np.log2(st["dt"].min())),
                "mean_steps_per_particle": inter / wl.n / wl.n,
                "rel_energy_drift": abs((k1 + w1) - (k0 + w0)) / abs(k0 + w0)}
            if prec != "fp64":
                # every particle's force at the evolved (synchronised) state, in
                # this mode as the integration would evaluate it next, against
                # the FP64 path on the same state
                idx = np.arange(wl.n, dtype=np.int32)
                ctx.predict(t_end)
                acc, jerk, pot = ctx.force(idx)
                with nbody.Context("fp64") as ref:
                    ref.set_state(m, st["r"], st["v"], st["a"], st["j"], st["t"], st["dt"],
                                  wl.eps, wl.eta)
                    ref.predict(t_end)
                    a64, j64, p64 = ref.force(idx)
                ea = np.linalg.norm(acc - a64, axis=1) / np.linalg.norm(a64, axis=1)
                ej = np.linalg.norm(jerk - j64, axis=1) / np.linalg.norm(j64, axis=1)
                ep = np.abs(pot - p64) / np.abs(p64)
                out["modes"][prec]["force_error_at_t_end"] = {
                    "particles": int(wl.n), "acc_rel_max": float(ea.max()),
                    "acc_rel_p50": float(np.median(ea)), "jerk_rel_max": float(ej.max()),
                    "jerk_rel_p50": float(np.median(ej)), "pot_rel_max": float(ep.max()),
                    "n_above_1e-6": int(np.sum((ea > 1e-6) | (ej > 1e-6) | (ep > 1e-6))),
                    "reference": "FP64 GPU path on the same state"}
        print(json.dumps({"partial": prec, **out["modes"][prec]}), file=sys.stderr, flush=True)
    if wl.n <= 4096:
        from oracle import oracle
        oracle.build()
        t0 = time.perf_counter()
        s = oracle.State(m, r, v, wl.eps, wl.eta, nthreads=os.cpu_count() or 1)
        e0 = s.energy()
        status = s.run(t_end)
        e1 = s.energy()
        wall = time.perf_counter() - t0
        # the CPU baseline of this workload: the oracle's own integration
        out["cpu_baseline"] = {"kind": "oracle", "status": int(status), "block_steps": s.n_steps,
                         "interactions": s.n_inter, "wall_s": wall,
                         "value": s.n_inter / wall,
                         "rel_energy_drift": abs(e1 - e0) / abs(e0),
                         "cores": os.cpu_count() or 1}
    print(json.dumps(out), flush=True)


def run_energy_study(args):
    """Sec. 4's integration test (Fig. err_itg): relative error of the total
    energy, averaged over the outputs t = k/16 up to 1/8 of a crossing time
    (t = 0.375, as Sec. 4 states it), against the number of steps per
    particle per crossing time (2 sqrt 2), for a range of eta.  The potential is the FP64 one in every
    mode, so the error is the integration's.  As the CPU baseline of each row
    ("cpu_baseline", kind "oracle"), the FP64 oracle runs the same
    integrations on the host cores."""
    import torch
    from paper_1104_2700_gb300 import build as nb_build
    from paper_1104_2700_gb300 import nbody
    from oracle import oracle
    nb_build.build()
    oracle.build()
    n, seed = 1024, 1
    eps, t_end, crossing = 4.0 / n, ENERGY_STUDY_T_END, CROSSING_TIME
    m, r, v = ics.plummer(n, seed)
    # eta enters Eq. timestep outside the square root (dt = eta (...)^(1/2));
    # the start rule scales with it (eta_start = eta / 4), since a fixed
    # eta_start lets the first steps set an eta-independent error floor
    etas = [0.01, 0.02, 0.04, 0.08, 0.16, 0.32]
    # MIXED is left out by default: its timestep collapse (precision_ablation)
    # makes its step count say nothing about the integrator's order
    modes = [x for x in args.modes.split(",") if x] if args.modes != "mixed,hybrid,ds,fp64" \
        else ["fp64", "ds", "hybrid"]
    outs = [k / 16 for k in range(1, int(round(t_end * 16)) + 1)]
    rows = []
    for eta in etas:
        row = {"eta": eta}
        for prec in modes:
            with nbody.Context(prec, eta_start=eta / 4) as ctx:
                ctx.set_particles(m, r, v, eps, eta)
                k0, w0 = ctx.energy(fp64_potential=True)
                errs, inter = [], 0
                for t in outs:
                    _, i = ctx.step_until(t)
                    inter += i
                    k1, w1 = ctx.energy(fp64_potential=True)
                    errs.append(abs((k1 + w1) - (k0 + w0)) / abs(k0 + w0))
            row[prec] = {"n_step": inter / n / n * crossing / t_end,
                         "mean_rel_energy_error": float(np.mean(errs)),
                         "final_rel_energy_error": errs[-1]}
        s = oracle.State(m, r, v, eps, eta, eta_start=eta / 4, nthreads=os.cpu_count() or 1)
        e0 = s.energy()
        errs = []
        for t in outs:
            s.run(t)
            errs.append(abs(s.energy() - e0) / abs(e0))
        # the CPU baseline of each row: the oracle's own integration
        row["cpu_baseline"] = {"kind": "oracle",
                               "n_step": s.n_inter / n / n * crossing / t_end,
                               "mean_rel_energy_error": float(np.mean(errs)),
                               "final_rel_energy_error": errs[-1]}
        rows.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    print(json.dumps({"study": "energy error vs steps per crossing time (Sec. 4)",
                      "eta_start": "eta / 4",
                      "workload": f"plummer_n{n}_seed{seed}_eps4/n", "t_end": t_end,
                      "outputs": outs, "data": "synthetic", "rows": rows}), flush=True)


def run_jerk_study(args):
    """Sec. 4's accumulation study (Figs. err_snp and err_snp_djerk): the
    distribution over particles of the relative errors of acc, jerk and pot
    against the FP64 path, for Plummer models of N = 1K, 4K, 16K and 64K
    (eps = 4/N, all particles active), with the jerk summed in plain FP32
    (mixed_spj, the paper's production kernel) and compensated (mixed), plus
    hybrid and DS for scale.  Also the force-launch time of each mode (CUDA
    events, n_act = N): the paper found DP jerk sums 20-25 % slower."""
    import torch
    from paper_1104_2700_gb300 import build as nb_build
    from paper_1104_2700_gb300 import nbody
    nb_build.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    modes = [x for x in args.modes.split(",") if x] if args.modes != "mixed,hybrid,ds,fp64" \
        else ["mixed_spj", "mixed", "hybrid", "ds"]
    qs = [0.5, 0.9, 0.99, 0.999, 1.0]
    rows = []
    for n in (1024, 4096, 16384, 65536):
        m, r, v = ics.plummer(n, 11)
        eps = 4.0 / n
        idx = np.arange(n, dtype=np.int32)
        idx_dev = torch.arange(n, dtype=torch.int32, device=dev)
        z3, t0, dt0 = np.zeros((n, 3)), np.zeros(n), np.full(n, 1.0 / 16)

        def forces(ctx, a, j):
            ctx.set_state(m, r, v, a, j, t0, dt0, eps, 0.02)
            ctx.predict(0.0)
            return ctx.force(idx)

        with nbody.Context("fp64", device=0, stream=stream) as ctx:
            a_ref, j_ref, p_ref = forces(ctx, z3, z3)
        row = {"n": n, "eps": eps}
        for prec in modes:
            with nbody.Context(prec, device=0, stream=stream) as ctx:
                a, j, p = forces(ctx, a_ref, j_ref)
                errs = {"acc": np.linalg.norm(a - a_ref, axis=1) / np.linalg.norm(a_ref, axis=1),
                        "jerk": np.linalg.norm(j - j_ref, axis=1) / np.linalg.norm(j_ref, axis=1),
                        "pot": np.abs(p - p_ref) / np.abs(p_ref)}
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                for _ in range(3):
                    ctx.force(idx_dev)
                e0.record(stream)
                reps = max(3, int(2e9 // (n * n)))
                for _ in range(reps):
                    ctx.force(idx_dev)
                e1.record(stream)
                e1.synchronize()
                ms = e0.elapsed_time(e1) / reps
            row[prec] = {k: {f"p{100 * q:g}": float(np.quantile(e, q)) for q in qs}
                         for k, e in errs.items()}
            row[prec]["force_ms"] = ms
            row[prec]["interactions_per_s"] = n * n / (ms * 1e-3)
        rows.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    print(json.dumps({"study": "force error distributions, jerk summed in FP32 vs "
                               "compensated (Sec. 4, Figs. err_snp, err_snp_djerk)",
                      "workload": "plummer seed 11, eps = 4/N, all particles active, t = 0",
                      "reference": "FP64 path (every operation in double)",
                      "data": "synthetic", "rows": rows}), flush=True)


def run_jerk_energy_study(args):
    """Sec. 4 reports that summing the jerk in SP or DP makes no significant
    difference to the energy error up to N = 256K at t = 0.125.  The same
    comparison on the precision that integrates: the N = 262144 Plummer model
    with Salpeter masses (eps = 1e-4, eta = 0.02) from t = 0 to 1/8, with the
    far pairs' jerk folded into double-single sums every run (hybrid) or kept
    in one plain FP32 sum across each warp's j (hybrid_spj): block steps,
    interactions per second and the relative energy drift (FP64 potential)."""
    import torch
    from paper_1104_2700_gb300 import build as nb_build
    from paper_1104_2700_gb300 import nbody
    nb_build.build()
    wl = ics.SALPETER_N256K
    t_end = args.t_end if args.t_end is not None else 1.0 / 8
    m, r, v = wl.particles()
    modes = [x for x in args.modes.split(",") if x] if args.modes != "mixed,hybrid,ds,fp64" \
        else ["hybrid", "hybrid_spj"]
    out = {"study": "jerk accumulation and energy drift (Sec. 4, Fig. err_snp_djerk text)",
           "workload": wl.name, "n": wl.n, "eps": wl.eps, "eta": wl.eta, "t_end": t_end,
           "data": "synthetic", "modes": {}}
    for prec in modes:
        with nbody.Context(prec) as ctx:
            ctx.set_particles(m, r, v, wl.eps, wl.eta)
            ctx.autotune()
            ctx.set_particles(m, r, v, wl.eps, wl.eta)
            k0, w0 = ctx.energy(fp64_potential=True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            steps, inter = ctx.step_until(t_end)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            k1, w1 = ctx.energy(fp64_potential=True)
            st = ctx.get_state()
        out["modes"][prec] = {
            "block_steps": int(steps), "interactions": int(inter), "wall_s": wall,
            "value": inter / wall, "unit": UNIT, "log2_min_dt": float(np.log2(st["dt"].min())),
            "rel_energy_drift": abs((k1 + w1) - (k0 + w0)) / abs(k0 + w0)}
        print(json.dumps({"partial": prec, **out["modes"][prec]}), file=sys.stderr, flush=True)
    print(json.dumps(out), flush=True)


def main():
    args = parse_args()
    if args.jerk_energy_study:
        run_jerk_energy_study(args)
    elif args.jerk_study:
        run_jerk_study(args)
    elif args.energy_study:
        run_energy_study(args)
    elif args.integrate:
        run_integration(args)
    elif args.profile:
        run_profile(args)
    elif args.profile_steps:
        run_profile_steps(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
