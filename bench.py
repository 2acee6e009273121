#!/usr/bin/env python3
"""Benchmark: pair-interactions/s of the direct-summation Hermite-4 step on GB300.

Workload (N = 2^20 by default): a Plummer sphere with Kroupa-IMF masses
(0.1-100, renormalised to M = 1), eps = 1e-4, Henon units, seeded synthetic
initial conditions.  One step = one block time step of the whole hot path
(next block time, active compaction, prediction of all N sources, force on the
active set, i-split reduction, Hermite correction) with every particle on the
same level, i.e. active fraction 1 (m = N): m * N pair interactions per step.

Reported (one JSON line from rank 0):
  value      interactions/s over the timed steps, device time (CUDA events on
             the library's stream), L2 flushed between steps, max over ranks;
  e2e        the same through the C ABI with pinned HOST buffers: state copied
             in, one block step, state copied out, every step;
  roofline   the mixed force kernel at 38 flops per interaction against the
             FP32 peak (SM count read at run time) x 128 lanes x 2 flops x 2.070
             GHz, and the measured f32x2 FMA rate (nb_measure_rate);
  sweep      nb_force alone at active fractions 2^-10 .. 1 (mixed) and
             2^-10 .. 2^-6 (FP64), with the mixed path's error vs the FP64
             path (the oracle checks both paths in tests/);
  cpu_baseline  the FP64 CPU oracle on the host cores, on a sample of targets.
Multi-GPU (torchrun): every rank integrates its own independent cluster
(seed = rank), no data-path collective; value sums the ranks' interactions.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FLOPS_PER_INTERACTION = 38          # acceleration + jerk convention
FLOPS_PER_INTERACTION_ACC = 20      # acceleration-only convention
FP32_LANES, SM_MAX_MHZ = 128, 2070.0
_SMS = []


def sm_count():
    """SMs of the GPU in use (read once at run time; GB300: 152)."""
    if not _SMS:
        import torch
        _SMS.append(torch.cuda.get_device_properties(torch.cuda.current_device())
                    .multi_processor_count)
    return _SMS[0]


def fp32_peak_flops(mhz=SM_MAX_MHZ):
    """Nominal FP32 FMA peak: SMs x 128 lanes x 2 flops x clock."""
    return sm_count() * FP32_LANES * 2 * mhz * 1e6
METRIC = "pair-interactions/s (and % FP32 peak) at N=2^20, mixed vs FP64, at stated error"
KERNEL_FILES = [os.path.join(ROOT, "paper_1411_5234_gb300", "csrc", f)
                for f in ("nb_force_mixed.cuh", "nb_force_mixed.cu", "nb_internal.cuh")]
UNIT = "pair-interactions/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--n", type=int, default=1 << 20)
    p.add_argument("--level", type=int, default=10, help="shared step 2^-level")
    p.add_argument("--no-sweep", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-tune", action="store_true", help="skip nb_autotune before timing")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--kernel-case", choices=["mixed", "fp64", "mixed-acc"], default=None,
                   help="run only nb_force on m random targets of N (profiling case)")
    p.add_argument("--m", type=int, default=16384)
    p.add_argument("--variant", type=int, default=None, help="mixed force kernel shape")
    p.add_argument("--bfactor", type=int, default=0,
                   help="i-split factor B of the headline step (0: the plan's or the table's)")
    p.add_argument("--workload", default="step",
                   choices=["step", "batch", "drift", "binaries", "leapfrog", "hermite6"],
                   help="step: the headline line; batch / drift / binaries: the other "
                        "configurations (their own JSON lines)")
    p.add_argument("--clusters", type=int, default=512)
    p.add_argument("--rerun-worst", type=int, default=0,
                   help="batch: re-run the K clusters of largest drift alone (mixed, FP64, "
                        "FP64 with eta/4, FP64 with level_min 6)")
    p.add_argument("--t-end", type=float, default=None)
    p.add_argument("--max-seconds", type=float, default=600.0,
                   help="drift / binaries: wall-time bound of each integration")
    p.add_argument("--fp64-n", type=int, default=None,
                   help="binaries: N of the FP64 comparison run (default: the same N)")
    return p.parse_args()


def integrate(sim, t_end, chunk=512, max_seconds=None, near=None, resort_factor=None):
    """Block steps until every cluster reaches t_end, or until max_seconds of
    wall time have passed; returns (device seconds, steps, time reached).

    With a list ``near``, the share of near (target warp, cell) pairs of the
    mixed kernel over every chunk of steps is appended to it; with
    ``resort_factor`` the sources are re-sorted (inside the timed run) when a
    chunk's share exceeds that factor times the share of the first chunk
    after the last sort (and 2 %); ``near`` then ends with the re-sort count."""
    import torch
    sim.set_end_time(sim.ticks(t_end))
    target = sim.ticks(t_end)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(sim.stream)
    steps = 0
    t_wall = time.perf_counter()
    wt0, nt0 = sim.tile_stats() if near is not None else (0, 0)
    base, resorts = None, 0
    while True:
        sim.step(chunk)
        steps += chunk
        st = sim.stats()
        if near is not None:
            wt, nt = sim.tile_stats()
            share = (nt - nt0) / max(wt - wt0, 1)
            near.append(share)
            wt0, nt0 = wt, nt
            if base is None:
                base = share
            elif resort_factor is not None and share > max(resort_factor * base, 0.02):
                sim.resort_sources()
                resorts += 1
                base = None
        if st.t_min >= target:
            break
        if max_seconds is not None and time.perf_counter() - t_wall > max_seconds:
            break
    if near is not None and resort_factor is not None:
        near.append(resorts)
    ev1.record(sim.stream)
    ev1.synchronize()
    return ev0.elapsed_time(ev1) * 1e-3, steps, sim.time(st.t_min)


def per_kernel_shares(kinds, seconds, steps):
    """Per kind of launch: device microseconds per block step and share of
    the run's device time (direct launches with events); "gaps" is the rest:
    time between the launches."""
    out = {k: {"us_per_step": ms * 1e3 / max(steps, 1), "share": ms * 1e-3 / seconds,
               "launches": n} for k, (ms, n) in kinds.items()}
    out["gaps"] = {"share": 1.0 - sum(v["share"] for v in out.values())}
    return out


def workload_batch(args):
    """Independent Plummer clusters of log-uniform size in one context: every
    block step advances every cluster; CUDA-graph-captured step sequences."""
    import torch
    from paper_1411_5234_gb300 import inputs, nbody
    torch.cuda.set_device(0)
    t_end = 0.25 if args.t_end is None else args.t_end
    cl = inputs.plummer_batch(args.clusters, 256, 16384, seed0=0)
    sizes = np.diff(cl.offsets)
    kw = {} if args.variant is None else {"variant": args.variant}
    out = {"workload": f"batch: {args.clusters} Plummer clusters, N_k log-uniform in [256, 16384] "
                       f"(sum N = {cl.n}, sum N^2 = {float((sizes.astype(float) ** 2).sum()):.4g}), "
                       f"seeds 0..{args.clusters - 1}, eps=1e-4, mixed, t = 0 -> {t_end}",
           "metric": "pair-interactions/s over the run", "unit": UNIT}
    # 1) the production run: graphs of 16 block steps
    sim = nbody.Sim(cl.pos, cl.vel, cl.mass, offsets=cl.offsets, eps=1e-4,
                    precision=nbody.NB_MIXED, level_min=3, graph_steps=16, **kw)
    import tempfile
    cache = os.path.join(tempfile.mkdtemp(prefix="nbody_tune_"), "tune.txt")
    if args.variant is None and not args.no_tune:
        # the table per ceil(log2 m), cached for the second run below
        out["autotuned_variant"] = sim.autotune(cache)[0]
        v, b = sim.tune_table()
        out["tune_table"] = {f"2^{k}": [int(v[k]), int(b[k])] for k in range(6, 16)}
    e0 = np.add(*sim.energies())
    secs, steps, _ = integrate(sim, t_end)
    st = sim.stats()
    e1 = np.add(*sim.energies())
    drift_signed = (e1 - e0) / np.abs(e0)
    drift = np.abs(drift_signed)
    assert sim.status() == nbody.NB_OK
    out.update({"value": st.interactions / secs, "seconds": secs, "interactions": st.interactions,
                "block_steps": st.block_steps,
                "energy_drift": {"median": float(np.median(drift)), "max": float(drift.max())}})
    sim.close()
    # 2) the same run with force-kernel events (direct launches): its share
    sim = nbody.Sim(cl.pos, cl.vel, cl.mass, offsets=cl.offsets, eps=1e-4,
                    precision=nbody.NB_MIXED, level_min=3, graph_steps=0, **kw)
    if args.variant is None and not args.no_tune:
        sim.autotune(cache)   # the same table, from the cache
    sim.profile(True)
    sim.profile_kernels()
    secs2, _, _ = integrate(sim, t_end)
    fms, nlaunch = sim.profile_read()
    out["per_kernel"] = per_kernel_shares(sim.profile_kernels(), secs2, sim.stats().block_steps)
    out["force_kernel_share"] = fms * 1e-3 / secs2
    out["nongraph_seconds"] = secs2
    out["force_launches"] = nlaunch
    sim.close()
    # 3) the clusters of largest drift, each integrated alone: the mixed path
    # against FP64 (whose drift is the integrator's), and FP64 with shorter
    # steps (eta and eta_start / 4; the largest step 2^-6 instead of 2^-3)
    if args.rerun_worst > 0:
        worst = []
        for k in np.argsort(-drift)[:args.rerun_worst]:
            o0, o1 = int(cl.offsets[k]), int(cl.offsets[k + 1])
            row = {"cluster": int(k), "N": o1 - o0, "batch_drift": float(drift_signed[k])}
            for name, prec, extra in (
                    ("alone_mixed", nbody.NB_MIXED, {}), ("alone_fp64", nbody.NB_FP64, {}),
                    ("fp64_eta_and_start_div4", nbody.NB_FP64, {"eta": 0.0025,
                                                                "eta_start": 0.0025}),
                    ("fp64_level_min_6", nbody.NB_FP64, {"level_min": 6})):
                cfg = dict(eps=1e-4, precision=prec, level_min=3, graph_steps=16)
                cfg.update(extra)
                s1 = nbody.Sim(cl.pos[o0:o1], cl.vel[o0:o1], cl.mass[o0:o1], **cfg)
                a0 = sum(s1.energy())
                integrate(s1, t_end)
                row[name] = (sum(s1.energy()) - a0) / abs(a0)
                assert s1.status() == nbody.NB_OK
                s1.close()
            worst.append(row)
        out["worst_clusters_alone"] = worst
    print(json.dumps(out), flush=True)
    return 0


def workload_drift(args):
    """Energy drift over block steps, FP64 path vs mixed path, same initial conditions."""
    import torch
    from paper_1411_5234_gb300 import inputs, nbody
    torch.cuda.set_device(0)
    n = args.n if args.n != (1 << 20) else (262144 if args.workload == "binaries" else 65536)
    t_end = (0.125 if args.workload == "binaries" else 1.0) if args.t_end is None else args.t_end
    if args.workload == "binaries":
        cl = inputs.plummer_binaries(n, seed=0)
        eps, lmax, label = 1e-5, 30, "Plummer with 10% binaries (a log-uniform 1e-4..1e-2, f(e)=2e)"
    else:
        cl = inputs.plummer(n, seed=0)
        eps, lmax, label = 1e-4, 20, "Plummer equal mass"
    out = {"workload": f"{label}, N={n}, eps={eps}, block steps 2^-3..2^-{lmax}, eta=0.01, "
                       f"t = 0 -> {t_end}", "unit": UNIT}
    runs = [("mixed", nbody.NB_MIXED, cl)]
    if args.workload == "binaries" and args.fp64_n and args.fp64_n != n:
        runs.append(("fp64", nbody.NB_FP64, inputs.plummer_binaries(args.fp64_n, seed=0)))
        runs.append(("mixed_at_fp64_n", nbody.NB_MIXED, runs[-1][2]))
    else:
        runs.append(("fp64", nbody.NB_FP64, cl))
    for name, prec, c in runs:
        sim = nbody.Sim(c.pos, c.vel, c.mass, eps=eps, precision=prec, level_min=3,
                        level_max=lmax, graph_steps=16)
        if prec == nbody.NB_MIXED and not args.no_tune:
            sim.autotune()
        mixed = prec == nbody.NB_MIXED
        near = [] if mixed else None
        e0 = sum(sim.energy())
        secs, _, t_reached = integrate(sim, t_end, max_seconds=args.max_seconds, near=near,
                                       resort_factor=1.5 if mixed else None)
        e1 = sum(sim.energy())
        st = sim.stats()
        assert sim.status() == nbody.NB_OK
        out[name] = {"N": c.n, "energy_drift": (e1 - e0) / abs(e0), "E0": e0,
                     "t_reached": t_reached, "interactions": st.interactions,
                     "block_steps": st.block_steps, "seconds": secs,
                     "interactions_per_s": st.interactions / secs}
        if mixed:
            shares = near[:-1]
            out[name]["near_share"] = {"first_chunk": shares[0], "last_chunk": shares[-1],
                                       "max": max(shares), "chunks": len(shares),
                                       "resorts": near[-1],
                                       "rule": "re-sort when a chunk of 512 steps exceeds "
                                               "1.5x the first chunk after the last sort"}
        sim.close()
        if mixed and name == "mixed":
            # the force kernel's share of the device time: direct launches
            # with events over the first 1/8 time unit
            sim = nbody.Sim(c.pos, c.vel, c.mass, eps=eps, precision=prec, level_min=3,
                            level_max=lmax, graph_steps=0)
            if not args.no_tune:
                sim.autotune()
            sim.profile(True)
            sim.profile_kernels()
            secs2, _, _ = integrate(sim, min(t_end, 0.125), max_seconds=args.max_seconds)
            fms, nlaunch = sim.profile_read()
            kinds = sim.profile_kernels()
            assert sim.status() == nbody.NB_OK
            nsteps = sim.stats().block_steps
            out[name]["force_kernel_share"] = {
                "share": fms * 1e-3 / secs2, "t_end": min(t_end, 0.125),
                "block_steps": nsteps, "force_launches": nlaunch,
                "us_per_step": secs2 / max(nsteps, 1) * 1e6}
            out[name]["per_kernel"] = per_kernel_shares(kinds, secs2, nsteps)
            sim.close()
    base = out.get("fp64", {}).get("energy_drift")
    comp = out.get("mixed_at_fp64_n", out["mixed"])["energy_drift"]
    if base:
        out["mixed_over_fp64_drift"] = abs(comp) / abs(base)
    print(json.dumps(out), flush=True)
    return 0


def workload_leapfrog(args):
    """Acceleration-only workload: kick-drift-kick leapfrog with a shared step
    (nb_step_leapfrog) on the N = 2^20 Kroupa Plummer sphere, mixed precision;
    interactions/s over K timed steps, the force kernel at 20 flops per
    interaction against the FP32 peak, and the relative energy change."""
    import torch
    from paper_1411_5234_gb300 import nbody
    torch.cuda.set_device(0)
    n, L = args.n, args.level
    cl = make_cluster(n, 0)
    sim = nbody.Sim(cl.pos, cl.vel, cl.mass, eps=1e-4, precision=nbody.NB_MIXED, graph_steps=0)
    dt_ticks = 1 << (sim.cfg.tick_exp - L)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    sim.leapfrog(args.warmup, dt_ticks)
    e0 = sum(sim.energy())
    sim.profile(True)
    sim.profile_read()
    evs = []
    with torch.cuda.stream(sim.stream):
        for _ in range(args.steps):
            flush.zero_()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(sim.stream)
            sim.leapfrog(1, dt_ticks)
            ev1.record(sim.stream)
            evs.append((ev0, ev1))
    sim.synchronize()
    total_ms = sum(a.elapsed_time(b) for a, b in evs)
    force_ms, launches = sim.profile_read()
    e1 = sum(sim.energy())
    assert sim.status() == nbody.NB_OK
    rate = args.steps * n * n / (total_ms * 1e-3)
    per = force_ms * 1e-3 / max(launches, 1)
    achieved = FLOPS_PER_INTERACTION_ACC * n * n / per / 1e12
    peak = fp32_peak_flops() / 1e12
    print(json.dumps({
        "workload": f"leapfrog (kick-drift-kick, shared step 2^-{L}): Plummer N={n} Kroupa, "
                    "eps=1e-4, mixed, acceleration-only force",
        "metric": "pair-interactions/s", "unit": UNIT, "value": rate, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "roofline": {"bound": "alu", "kernel": "k_force_mixed (acceleration only)",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "flops_per_interaction": FLOPS_PER_INTERACTION_ACC,
                     "force_ms_per_launch": per * 1e3},
        "energy_rel_change": (e1 - e0) / abs(e0),
        "l2": "flushed between timed steps (256 MiB write)"}), flush=True)
    sim.close()
    return 0


# 6th-order convention: the acceleration + jerk convention (38) plus the snap
# terms counted the same way (FMA = 2 flops): u = a_j - a_i 3, w.w + d.u 11,
# alpha, beta and the two coefficients 6, u - 6 alpha J' - 3 beta d 12, the
# accumulation of m/s^3 times it 6
FLOPS_PER_INTERACTION_SNAP = 76
LANE_OPS_SNAP = 48          # FP32 lane-operations per interaction in the snap kernel


def workload_hermite6(args):
    """6th-order Hermite block steps (force with snap, Sec. 2 item 1) on the
    N = 2^20 Kroupa Plummer sphere, every particle on one level (m = N),
    mixed precision: interactions/s, the snap kernel against the FP32 peak at
    76 flops and against the FMA pipe at its 48 lane-ops per interaction;
    FP64 nb_force_snap at m = 2^10; mixed against FP64 on 1024 targets."""
    import torch
    from paper_1411_5234_gb300 import inputs, nbody
    torch.cuda.set_device(0)
    n, L = args.n, args.level
    cl = make_cluster(n, 0)
    sim = nbody.Sim(cl.pos, cl.vel, cl.mass, eps=1e-4, precision=nbody.NB_MIXED, order=6,
                    level_min=L, level_max=L, graph_steps=0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    sim.step(args.warmup)
    sim.profile(True)
    sim.synchronize()
    sim.profile_read()
    evs = []
    with torch.cuda.stream(sim.stream):
        for _ in range(args.steps):
            flush.zero_()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(sim.stream)
            sim.step(1)
            ev1.record(sim.stream)
            evs.append((ev0, ev1))
    sim.synchronize()
    total_ms = sum(a.elapsed_time(b) for a, b in evs)
    force_ms, launches = sim.profile_read()
    assert sim.status() == nbody.NB_OK
    rate = args.steps * n * n / (total_ms * 1e-3)
    per = force_ms * 1e-3 / max(launches, 1)
    achieved = FLOPS_PER_INTERACTION_SNAP * n * n / per / 1e12
    peak = fp32_peak_flops() / 1e12
    pipe = LANE_OPS_SNAP * n * n / per / (sm_count() * FP32_LANES * SM_MAX_MHZ * 1e6)
    idx = inputs.random_active(n, 1024, seed=9)
    act = torch.as_tensor(idx, device="cuda")
    sim.predict(sim.stats().t_min)
    am, jm, sm, _ = (x.cpu().numpy() for x in sim.force_snap(act))
    st = sim.get_state()
    sn, cr = sim.get_derivs()
    sim.close()
    # FP64 from the same state: its force with snap on 1024 targets, timed
    s64 = nbody.Sim(cl.pos, cl.vel, cl.mass, eps=1e-4, precision=nbody.NB_FP64, order=6,
                    level_min=L, level_max=L, graph_steps=0)
    s64.set_state(st["pos"], st["vel"], st["acc"], st["jerk"], st["t"], st["level"])
    s64.set_derivs(sn, cr)
    s64.predict(int(st["t"][0]))
    s64.profile(True)
    s64.force_snap(act)
    s64.synchronize()
    s64.profile_read()
    a6, j6, s6, _ = s64.force_snap(act)
    ms64, cnt64 = s64.profile_read()
    a6, j6, s6 = a6.cpu().numpy(), j6.cpu().numpy(), s6.cpu().numpy()
    s64.close()
    rel = lambda x, r: np.linalg.norm(x - r, axis=1) / np.linalg.norm(r, axis=1)
    es, ea = rel(sm, s6), rel(am, a6)
    print(json.dumps({
        "workload": f"hermite6 (6th-order block steps, shared level 2^-{L}): Plummer N={n} "
                    "Kroupa, eps=1e-4, mixed, force with snap",
        "metric": "pair-interactions/s", "unit": UNIT, "value": rate, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "roofline": {"bound": "alu", "kernel": "k_force_mixed (snap shape)",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "flops_per_interaction": FLOPS_PER_INTERACTION_SNAP,
                     "fma_pipe_frac": pipe, "lane_ops_per_interaction": LANE_OPS_SNAP,
                     "force_ms_per_launch": per * 1e3,
                     "force_share_of_step": force_ms / max(total_ms, 1e-9)},
        "fp64_force_snap": {"m": 1024, "interactions_per_s": 1024 * n / (ms64 / max(cnt64, 1)
                                                                           * 1e-3)},
        "mixed_vs_fp64_1024_targets": {
            "acc_rel_max": float(ea.max()), "acc_rel_median": float(np.median(ea)),
            "snap_rel_median": float(np.median(es)),
            "snap_rel_p99": float(np.quantile(es, 0.99))},
        "l2": "flushed between timed steps (256 MiB write)"}), flush=True)
    return 0


def kernel_case(args):
    """nb_force alone (W + K launches) on m random targets of the N-body workload."""
    import torch
    from paper_1411_5234_gb300 import inputs, nbody
    torch.cuda.set_device(0)
    cl = make_cluster(args.n, 0)
    prec = nbody.NB_FP64 if args.kernel_case == "fp64" else nbody.NB_MIXED
    want_jerk = args.kernel_case != "mixed-acc"
    flops = FLOPS_PER_INTERACTION if want_jerk else FLOPS_PER_INTERACTION_ACC
    kw = {} if args.variant is None else {"variant": args.variant}
    sim = nbody.Sim(cl.pos, cl.vel, cl.mass, eps=1e-4, precision=prec, graph_steps=0, **kw)
    sim.predict(0)
    act = torch.as_tensor(inputs.random_active(cl.n, args.m, seed=1), device="cuda")
    acc = torch.empty((args.m, 3), dtype=torch.float64, device="cuda")
    jerk = torch.empty_like(acc) if want_jerk else None
    for _ in range(args.warmup):
        sim.force(act, acc, jerk, None, want_pot=False, want_jerk=want_jerk)
    sim.synchronize()
    wt0, nt0 = sim.tile_stats()
    sim.profile(True)
    for _ in range(args.steps):
        sim.force(act, acc, jerk, None, want_pot=False, want_jerk=want_jerk)
    ms, cnt = sim.profile_read()
    assert sim.status() == nbody.NB_OK
    per = ms / max(cnt, 1)
    rate = args.m * cl.n / (per * 1e-3)
    wt, nt = sim.tile_stats()
    print(json.dumps({"kernel_case": args.kernel_case, "variant": sim.cfg.variant,
                      "near_tile_share": (nt - nt0) / max(wt - wt0, 1),
                      "N": cl.n, "m": args.m,
                      "ms_per_launch": per, "interactions_per_s": rate,
                      "flops_per_interaction": flops,
                      "frac_fp32_peak": flops * rate
                      / fp32_peak_flops()}), flush=True)
    sim.close()
    return 0


def reduce_max(value, dist=None, device="cuda"):
    """The maximum of a per-rank number over all ranks (the job's timed
    region ends when its slowest rank ends); `value` itself on one rank."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, seconds_max):
    """Whole-job throughput: every rank processed units_per_rank in at most
    seconds_max (weak scaling: the per-rank work is fixed)."""
    return world * units_per_rank / seconds_max


def workload_config(n):
    return {"workload": f"Plummer N={n} Kroupa IMF 0.1-100 (M=1), eps=1e-4, Henon units; "
                        "one Hermite-4 block step per step with all particles active "
                        "(active fraction 1, shared level)",
            "N": n, "eps": 1e-4, "imf": "kroupa", "active_fraction": 1.0,
            "precision": "mixed: FP32 pair arithmetic on double-single separations, "
                         "compensated FP32 per-tile sums combined in FP64, FP64 state",
            "l2": "flushed between timed steps (256 MiB write)"}


def make_cluster(n, seed):
    from paper_1411_5234_gb300 import inputs
    return inputs.plummer(n, seed=seed, imf="kroupa")


# ------------------------------------------------------------------ oracle --

def oracle_sample(cl, seconds, seed=0):
    """Time the FP64 CPU oracle on a random sample of targets vs all N sources."""
    import oracle
    from paper_1411_5234_gb300 import inputs
    n = cl.n
    probe = inputs.random_active(n, 128, seed=seed + 1).astype(np.int64)
    t0 = time.perf_counter()
    oracle.force(cl.pos, cl.vel, cl.mass, 1e-4, idx=probe)
    dt = max(time.perf_counter() - t0, 1e-6)
    rate = 128 * n / dt
    nt = int(min(max(rate * seconds / n, 128), n))
    idx = inputs.random_active(n, nt, seed=seed + 2).astype(np.int64)
    t0 = time.perf_counter()
    oracle.force(cl.pos, cl.vel, cl.mass, 1e-4, idx=idx)
    dt = time.perf_counter() - t0
    return {"value": nt * n / dt, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{nt} random targets x all {n} sources (acc+jerk+pot, FP64, "
                      f"Neumaier sums), {dt:.1f} s"}


def run_reference(args):
    """The oracle as the reference arm (bounded samples of the same workload)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_1411_5234_gb300 import inputs
    cl = make_cluster(args.n, 0)
    # size each step to ~10 s of CPU work
    probe = inputs.random_active(cl.n, 16, seed=99).astype(np.int64)
    t0 = time.perf_counter()
    oracle.force(cl.pos, cl.vel, cl.mass, 1e-4, idx=probe)
    rate = 16 * cl.n / max(time.perf_counter() - t0, 1e-6)
    nt = int(min(max(rate * 10.0 / cl.n, 16), cl.n))
    times = []
    for s in range(args.warmup + args.steps):
        idx = inputs.random_active(cl.n, nt, seed=s).astype(np.int64)
        t0 = time.perf_counter()
        oracle.force(cl.pos, cl.vel, cl.mass, 1e-4, idx=idx)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = args.steps * nt * cl.n / tot
    cfg = workload_config(args.n)
    cfg["reference_sample"] = f"{nt} random targets x all {cl.n} sources per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": f"{nt} random targets x {cl.n} sources per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id):
        self.rows = []
        self.proc = None
        self.device_id = device_id

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device_id), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 8:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        pw = [float(r[2]) for r in self.rows if re.match(r"^[0-9.]+$", r[2])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4)
                          if r[4 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None,
                "samples": len(self.rows), "reasons": reasons}


def kernel_source_sha(files):
    h = hashlib.sha256()
    for f in files:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def traffic_from_profile(kernel_files):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source (same sha256 of the kernel files), else None."""
    path = os.path.join(ROOT, "profiles", "force_mixed_n1048576.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    sha = kernel_source_sha(kernel_files)
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)\s+source_sha256:\s*([0-9a-f]+)", text)
    if m and m.group(2) == sha:
        return float(m.group(1))
    return None


# ------------------------------------------------------------------- main ---

def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.kernel_case:
        return kernel_case(args)
    if args.workload == "batch":
        return workload_batch(args)
    if args.workload in ("drift", "binaries"):
        return workload_drift(args)
    if args.workload == "leapfrog":
        return workload_leapfrog(args)
    if args.workload == "hermite6":
        return workload_hermite6(args)

    import torch
    from paper_1411_5234_gb300 import inputs, nbody

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    n = args.n
    cl = make_cluster(n, seed=rank)
    L = args.level
    kw = {} if args.variant is None else {"variant": args.variant}
    if args.bfactor > 0:
        kw["bfactor"] = args.bfactor
    sim = nbody.Sim(cl.pos, cl.vel, cl.mass, eps=1e-4, precision=nbody.NB_MIXED,
                    level_min=L, level_max=L, graph_steps=0, **kw)
    stream = sim.stream
    tune = None
    import tempfile
    cache = os.path.join(tempfile.mkdtemp(prefix="nbody_tune_"), "tune.txt")
    if not args.no_tune and args.variant is None:
        variant, tms = sim.autotune(cache)
        tv, tb = sim.tune_table()
        tune = {"table_ceil_log2_m": {f"2^{k}": [int(tv[k]), int(tb[k])]
                                      for k in range(6, 21) if (1 << k) <= 2 * n},
                "step_bucket": [int(tv[(n - 1).bit_length()]), int(tb[(n - 1).bit_length()])],
                "ms_per_variant_at_m_every_4^k_th_slot": tms,
                "cache": "written to a temporary file; the sweep below loads it"}
    else:
        cache = None
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    sim.profile(True)

    def one_step():
        with torch.cuda.stream(stream):
            flush.zero_()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            sim.step(1)
            ev1.record(stream)
        return ev0, ev1

    for _ in range(args.warmup):
        one_step()
    stream.synchronize()
    sim.profile_read()                      # drop warm-up launches
    wt0, nt0 = sim.tile_stats()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    dev_id = local
    try:
        dev_id = str(torch.cuda.get_device_properties(local).uuid)
        dev_id = dev_id if dev_id.startswith("GPU-") else f"GPU-{dev_id}"
    except Exception:
        pass
    with ClockSampler(dev_id) as clk:
        evs = [one_step() for _ in range(args.steps)]
        stream.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    force_ms, force_launches = sim.profile_read()
    total_ms = reduce_max(sum(step_ms), dist)
    assert sim.status() == nbody.NB_OK, nbody.strerror(sim.status())
    inter_step = n * n
    value = job_rate(args.steps * inter_step, world, total_ms * 1e-3)
    launches_per_step = 7   # tmin, predict, scan+plan, scatter, force, reduce, correct

    clocks = clk.summary()
    force_avg_s = force_ms * 1e-3 / max(force_launches, 1)
    achieved = FLOPS_PER_INTERACTION * inter_step / force_avg_s / 1e12
    peak = fp32_peak_flops() / 1e12
    traffic = traffic_from_profile(KERNEL_FILES)
    roofline = {"bound": "alu", "kernel": "k_force_mixed", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                "flops_per_interaction": FLOPS_PER_INTERACTION,
                "peak_basis": f"FP32 FMA: {sm_count()} SMs (read at run time) x 128 lanes x 2 "
                              f"flops x 2070 MHz (max clock)",
                "force_ms_per_launch": force_avg_s * 1e3,
                "force_share_of_step": force_ms / max(total_ms, 1e-9) if world == 1 else None}
    if clocks.get("sm_mhz"):
        pk = fp32_peak_flops(clocks["sm_mhz"]) / 1e12
        roofline["peak_at_sampled_clock"] = pk
        roofline["frac_at_sampled_clock"] = achieved / pk

    # measured FMA rates of this GPU (nb_measure_rate: SM-clock cycles, so
    # independent of the clock it ran at) beside the nominal 128 lanes/SM/clk
    r2 = sim.measure_rate(0)
    r64 = sim.measure_rate(2)
    mhz = clocks.get("sm_mhz") or SM_MAX_MHZ
    pk_meas = sm_count() * r2 * 2 * mhz * 1e6 / 1e12
    roofline["measured_rates"] = {
        "ffma2_lanes_per_sm_clk": r2, "dfma_lanes_per_sm_clk": r64,
        "peak_measured_ffma2": pk_meas, "frac_of_measured_ffma2": achieved / pk_meas,
        "basis": f"measured f32x2 FMA lanes/SM/clk x {sm_count()} SMs x 2 flops x {mhz:.0f} MHz "
                 "(sampled clock)"}
    roofline["kernel_shape_variant"] = sim.cfg.variant
    if tune:
        roofline["autotune"] = tune
    wt, nt = sim.tile_stats()
    roofline["near_tile_share"] = (nt - nt0) / max(wt - wt0, 1)   # timed steps only
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": workload_config(n), "roofline": roofline,
            "clocks": clocks, "gpu_launches": launches_per_step * args.steps}

    # ---- end to end through the C ABI with pinned host buffers ----
    if not args.no_e2e:
        pin = lambda shape, dt: torch.empty(shape, dtype=dt).pin_memory().numpy()
        hp, hv, ha, hj = (pin((n, 3), torch.float64) for _ in range(4))
        ht, hl = pin((n,), torch.int64), pin((n,), torch.int32)
        sim.profile(False)
        sim.get_state_into(hp, hv, ha, hj, ht, hl)
        e2e_t = []
        for k in range(args.warmup + args.steps):
            if dist:
                dist.barrier()
            t0 = time.perf_counter()
            sim.set_state(hp, hv, ha, hj, ht, hl)
            sim.step(1)
            sim.get_state_into(hp, hv, ha, hj, ht, hl)
            if k >= args.warmup:
                e2e_t.append(time.perf_counter() - t0)
        tot = reduce_max(sum(e2e_t), dist)
        h2d = 4 * 24 * n + 8 * n + 4 * n
        line["e2e"] = {"value": job_rate(args.steps * inter_step, world, tot), "unit": UNIT,
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d,
                       "api": "nb_set_state + nb_step_block + nb_get_state (pinned host)"}
    sim.close()

    # ---- nb_force sweep over the active fraction, mixed and FP64 ----
    if not args.no_sweep and rank == 0:
        line["sweep"] = sweep(nbody, inputs, torch, cl, cache)
    if not args.no_cpu and rank == 0 and world == 1:
        line["cpu_baseline"] = oracle_sample(cl, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def sweep(nbody, inputs, torch, cl, cache=None):
    n = cl.n
    out = {"unit": UNIT, "timing": "force kernel via CUDA events (nb_profile), best of 3",
           "mixed": [], "fp64": []}
    sims = {}
    for name, prec in (("mixed", nbody.NB_MIXED), ("fp64", nbody.NB_FP64)):
        s = nbody.Sim(cl.pos, cl.vel, cl.mass, eps=1e-4, precision=prec, graph_steps=0)
        if name == "mixed" and cache is not None:
            s.autotune(cache)          # the headline's table, from its cache file
            out["mixed_table"] = "autotune table per ceil(log2 m) (shape, B) in each entry"
        s.predict(0)
        s.profile(True)
        sims[name] = s
    tv, tb = sims["mixed"].tune_table()
    for name, kmin, kmax in (("mixed", 10, 0), ("fp64", 10, 6)):
        s = sims[name]
        for k in range(kmin, kmax - 1, -1):
            m = n >> k
            act = torch.as_tensor(inputs.random_active(n, m, seed=k), device="cuda")
            acc = torch.empty((m, 3), dtype=torch.float64, device="cuda")
            jerk = torch.empty_like(acc)
            s.force(act, acc, jerk, None, want_pot=False)
            s.synchronize()
            s.profile_read()
            best = math.inf
            for _ in range(3):
                s.force(act, acc, jerk, None, want_pot=False)
                ms, cnt = s.profile_read()
                best = min(best, ms / max(cnt, 1))
            rate = m * n / (best * 1e-3)
            entry = {"active_fraction": f"2^-{k}", "m": m, "interactions_per_s": rate,
                     "ms": best}
            if name == "mixed":
                entry["frac_fp32_peak"] = (FLOPS_PER_INTERACTION * rate
                                           / fp32_peak_flops())
                b = (m - 1).bit_length()
                entry["shape_B"] = [int(tv[b]), int(tb[b])]
            out[name].append(entry)
    # acceleration only (nb_force with jerk == NULL), 20 flops per interaction
    out["mixed_acc_only"] = []
    s = sims["mixed"]
    for k in (10, 6, 0):
        m = n >> k
        act = torch.as_tensor(inputs.random_active(n, m, seed=k), device="cuda")
        acc = torch.empty((m, 3), dtype=torch.float64, device="cuda")
        s.force(act, acc, None, None, want_pot=False, want_jerk=False)
        s.synchronize()
        s.profile_read()
        best = math.inf
        for _ in range(3):
            s.force(act, acc, None, None, want_pot=False, want_jerk=False)
            ms, cnt = s.profile_read()
            best = min(best, ms / max(cnt, 1))
        rate = m * n / (best * 1e-3)
        out["mixed_acc_only"].append({
            "active_fraction": f"2^-{k}", "m": m, "interactions_per_s": rate, "ms": best,
            "flops_per_interaction": FLOPS_PER_INTERACTION_ACC,
            "frac_fp32_peak": (FLOPS_PER_INTERACTION_ACC * rate
                               / fp32_peak_flops())})
    # the mixed path's separation-mode bounds (NB_DS, NB_FP32) at m = 2^14
    idx = inputs.random_active(n, 4096, seed=123)
    act = torch.as_tensor(idx, device="cuda")
    ref = sims["fp64"].force(act)
    sims["fp64"].synchronize()
    ra, rj = ref[0].cpu().numpy(), ref[1].cpu().numpy()
    rel = lambda x, r: np.linalg.norm(x - r, axis=1) / np.linalg.norm(r, axis=1)
    out["separation_modes"] = {}
    for name, prec in (("ds", nbody.NB_DS), ("fp32", nbody.NB_FP32)):
        s = nbody.Sim(cl.pos, cl.vel, cl.mass, eps=1e-4, precision=prec, graph_steps=0)
        s.predict(0)
        s.profile(True)
        m = n >> 6
        a14 = torch.as_tensor(inputs.random_active(n, m, seed=6), device="cuda")
        acc = torch.empty((m, 3), dtype=torch.float64, device="cuda")
        jerk = torch.empty_like(acc)
        s.force(a14, acc, jerk, None, want_pot=False)
        s.synchronize()
        s.profile_read()
        best = math.inf
        for _ in range(3):
            s.force(a14, acc, jerk, None, want_pot=False)
            ms, cnt = s.profile_read()
            best = min(best, ms / max(cnt, 1))
        a, j, _ = s.force(act)
        s.synchronize()
        ea = rel(a.cpu().numpy(), ra)
        ej = rel(j.cpu().numpy(), rj)
        out["separation_modes"][name] = {
            "m": m, "interactions_per_s": m * n / (best * 1e-3), "ms": best,
            "acc_rel_max": float(ea.max()), "acc_rel_median": float(np.median(ea)),
            "jerk_rel_median": float(np.median(ej))}
        s.close()
    # accuracy: mixed vs FP64 on 4096 targets (GPU against GPU; the oracle
    # checks both paths at this size in tests/test_gpu_full_size.py)
    act = torch.as_tensor(idx, device="cuda")
    res = {}
    for name in ("mixed", "fp64"):
        a, j, p = sims[name].force(act)
        sims[name].synchronize()
        res[name] = (a.cpu().numpy(), j.cpu().numpy(), p.cpu().numpy())
    a_acc, _, _ = sims["mixed"].force(act, want_jerk=False)
    sims["mixed"].synchronize()
    rel = lambda x, r: np.linalg.norm(x - r, axis=1) / np.linalg.norm(r, axis=1)
    ea, ej = rel(res["mixed"][0], res["fp64"][0]), rel(res["mixed"][1], res["fp64"][1])
    ep = np.abs(res["mixed"][2] / res["fp64"][2] - 1)
    eaa = rel(a_acc.cpu().numpy(), res["fp64"][0])
    out["accuracy"] = {
        "mixed_vs_fp64_4096_targets": {
            "acc_rel_max": float(ea.max()), "acc_rel_median": float(np.median(ea)),
            "acc_rel_p999": float(np.quantile(ea, 0.999)),
            "jerk_rel_max": float(ej.max()), "jerk_rel_median": float(np.median(ej)),
            "pot_rel_max": float(ep.max())},
        "mixed_acc_only_vs_fp64_4096_targets": {
            "acc_rel_max": float(eaa.max()), "acc_rel_median": float(np.median(eaa))}}
    mx = {e["m"]: e["interactions_per_s"] for e in out["mixed"]}
    out["mixed_over_fp64_speedup"] = {e["active_fraction"]: mx[e["m"]] / e["interactions_per_s"]
                                      for e in out["fp64"]}
    for s in sims.values():
        s.close()
    return out


if __name__ == "__main__":
    sys.exit(main())
