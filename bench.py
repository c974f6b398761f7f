"""Throughput of the multi-detection GLMB update on one GB300.

A step is one frame of the whole update (predict, compatibility table,
death probabilities, child expansion and scoring, normalisation and top-H,
track update, estimates) on a seeded synthetic scene: 2-D constant velocity,
100 objects appearing over the first 50 frames, 100 frames, clutter
Poisson(20), 1 + Poisson(1.5) detections per detected object, H_max = 1000,
H_up = 100.  Steps walk through the scene's frames in order; the filter is
reset when the scene restarts.  Before the warm-up steps, one untimed set-up
pass over the scene captures the frame graphs its plans need (reported as
config.graph_precapture_frames; --no-precapture skips it).

value  frames/s with each frame's detections already in device memory.
e2e    frames/s through the same C ABI with host buffers: detections copied
       host->device and the estimates read back inside every step.
Between steps a 256 MiB buffer is written to flush L2 (outside the timed
events).  Under torchrun every rank runs its own independent scene (no
collective on the data path); value is the frames of all ranks over the
slowest rank's time.

--impl reference times the FP64 CPU oracle (the reference implementation of
this method in this repository) on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import scenes  # noqa: E402

METRIC = "GLMB update frames/sec & hypothesis-track updates/s vs N objects, H cap (1 GB300)"
UNIT = "frames/s"
INT_PEAK_NOTE = "152 SMs x 128 lanes x 2070 MHz"


def expansion_traffic():
    """DRAM bytes per frame of the expansion kernels from the committed ncu
    summary, or None when the kernels changed since it was captured."""
    import hashlib
    here = os.path.dirname(os.path.abspath(__file__))
    try:
        txt = open(os.path.join(here, "profiles", "expansion_traffic_mid.md")).read()
        src = open(os.path.join(here, "paper_2512_06230_gb300", "csrc", "kernels_expand.cu"), "rb").read()
    except OSError:
        return None
    vals = dict(l.split(":", 1) for l in txt.splitlines() if ":" in l and not l.startswith(("#", " ", "`")))
    want = vals.get("kernels_expand.cu sha256 (first 16 hex)", "").strip()
    if want != hashlib.sha256(src).hexdigest()[:16]:
        return None
    try:
        return float(vals["traffic_bytes_per_frame"])
    except (KeyError, ValueError):
        return None


def max_over_ranks(value: float, device, world: int) -> float:
    """The largest of the ranks' values (every rank gets it): the job's time
    is its slowest rank's.  One rank: the value itself."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(steps_per_rank: int, world: int, max_ms: float) -> float:
    """Whole-job throughput: the frames of all ranks over the slowest rank's
    time (ms)."""
    return steps_per_rank * world / (max_ms / 1000.0)


def scene_for_rank(args, rank):
    p = scenes.preset(args.scene)
    return scenes.make_scene(p, 1000 * 2 + rank if args.seed is None else args.seed + rank)


def filter_cfg(sc):
    n_max_births = max(len(f.births) for f in sc.frames)
    cfg = sc.filter_config(max_meas=max(64, max(len(f.Z) for f in sc.frames) + 16),
                           max_births=max(8, n_max_births),
                           max_tracks=sc.params.n_objects * 2 + n_max_births + 64)
    return cfg


def sample_clocks(stop, out):
    cmd = ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
           "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
           "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
           "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"]
    try:
        p = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except OSError:
        return
    def reader():
        for line in p.stdout:
            out.append(line.strip())
    t = threading.Thread(target=reader, daemon=True)
    t.start()
    stop.wait()
    p.terminate()
    try:
        p.wait(timeout=5)
    except Exception:
        p.kill()
    t.join(timeout=2)


def summarize_clocks(lines, dev):
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 9 or f[0] != str(dev):
            continue
        try:
            sm.append(float(f[1]))
            mx.append(float(f[2]))
        except ValueError:
            continue
        for n, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(n)
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
            "samples": len(sm)}


def run_oracle(args, sc, cfg, budget_s):
    """FP64 oracle over the scene's frames from the initial GLMB, all host
    threads, until the scene ends or the time budget is spent."""
    import oracle
    threads = args.cpu_threads if args.cpu_threads > 0 else (os.cpu_count() or 1)
    o = oracle.Oracle(cfg, n_threads=threads)
    t0 = time.perf_counter()
    n = 0
    for fr in sc.frames:
        o.step(fr.births, fr.Z)
        o.estimates()
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return n / dt, threads, f"{args.scene} scene frames 0..{n - 1} of {len(sc.frames)} " \
        f"from the initial GLMB ({dt:.1f} s, {threads} threads)"


def workload_config(args, sc, cfg) -> dict:
    """The workload of the default run, named the same in both arms."""
    F = len(sc.frames)
    return {"workload": f"{args.scene} scene: 2-D CV, {sc.params.n_objects} objects, "
                        f"{F} frames, H_max={cfg['h_max']}, H_up={cfg['h_up']}",
            "scene": args.scene, "h_max": cfg["h_max"], "h_up": cfg["h_up"], "frames_per_scene": F}


def batch_cfg(p, sc):
    return sc.filter_config(max_meas=int(p.n_objects * 0.9 * 6 + 4 * p.clutter_rate + 64),
                            max_births=64, max_tracks=p.n_objects + 48,
                            max_components=400 * (p.n_objects + 48), max_pairs=1 << 20)


def run_batch(args, glmb, torch, dev):
    """The batched form: --scenes independent scenes per frame (N ~ U{5..300},
    H ~ U{100..5000}, clutter ~ U(5, 40)), --steps frames each, stepped together
    by glmb_step_batch (each filter on its own stream), against the plain
    path stepping the same scenes one after another.  One untimed pass fills
    the graph caches; the filters are then reset and the second pass timed
    (host wall clock, every scene's results synchronised each frame)."""
    F = args.steps
    specs = scenes.batch_scenes(args.scenes, 4000 if args.seed is None else args.seed, frames=F)
    scs = [scenes.make_scene(p, s) for p, s in specs]
    cfgs = [batch_cfg(p, sc) for (p, _), sc in zip(specs, scs)]
    on_dev = args.batch_detections == "device"
    if on_dev:
        Z = [[torch.from_numpy(fr.Z).to(dev) if len(fr.Z) else torch.zeros((0, 2), device=dev)
              for fr in sc.frames] for sc in scs]
    else:
        Z = [[fr.Z for fr in sc.frames] for sc in scs]
    B = [[glmb.births_array(fr.births, sc.dim_x) for fr in sc.frames] for sc in scs]
    torch.cuda.synchronize()

    def run_pass(filters, batched):
        t = 0.0
        for k in range(F):
            t0 = time.perf_counter()
            if batched:
                glmb.step_batch(filters, [(B[i][k], Z[i][k]) for i in range(len(filters))], device=on_dev)
            else:
                for i, f in enumerate(filters):
                    f.step(B[i][k], Z[i][k], device=on_dev)
            for f in filters:
                f.estimates(cap=f.cfg["max_tracks"], pmf_cap=64)
            t += time.perf_counter() - t0
        return t

    out = {}
    for name, batched in (("sequential", False), ("batched", True)):
        filters = [glmb.Filter(c) for c in cfgs]
        run_pass(filters, batched)               # warm-up pass (graph captures)
        for f in filters:
            f.reset()
        t = run_pass(filters, batched)
        work = sum(f.info()["n_children"] for f in filters)   # the last frame's
        out[name] = dict(seconds=t, scene_frames_per_s=len(filters) * F / t,
                         children_per_frame=work)
        for f in filters:
            f.close()
        torch.cuda.synchronize()
    line = {"metric": "scene-frames/s, batched multi-scene GLMB (1 GB300)",
            "value": out["batched"]["scene_frames_per_s"], "unit": "scene-frames/s", "n_gpus": 1,
            "steps": F, "warmup": F, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.scenes} scenes x {F} frames, N~U{{5..300}}, H~U{{100..5000}}, "
                                   "clutter~U(5,40), 2-D CV",
                       "detections": args.batch_detections,
                       "h_max": [p.h_max for p, _ in specs], "n_objects": [p.n_objects for p, _ in specs]},
            "sequential": out["sequential"], "batched": out["batched"],
            "speedup_vs_sequential": out["batched"]["scene_frames_per_s"] / out["sequential"]["scene_frames_per_s"]}
    print(json.dumps(line))


def _ints(text):
    return [int(v) for v in str(text).split(",") if v]


def run_convoy(args, glmb, torch):
    """Section 4.1's scalability grid on the convoy workload: N copies of one
    closed track (offset delta = 2 steps), five detections per object, no
    clutter, 548 steps of 0.1 s; N x H_max over --convoy-n x --convoy-h,
    for each score mode in --convoy-modes (0 the joint multi-detection
    likelihood, 1 the product of C entries), --runs seeds each.  One update
    is glmb_step with the frame's detections in host memory plus the
    estimates read back (host wall clock, as the paper times an update);
    one untimed pass per filter first fills its graph cache.  Accuracy is
    the paper's: relative cardinality error and the Hungarian-matched mean
    distance, averaged over the steps of a run.  --convoy-oracle-steps
    steps of the FP64 oracle (single thread) are timed per (N, H_max) of
    mode 0 beside it."""
    from scenes.metrics import RunAccuracy
    import oracle
    steps = args.convoy_steps
    grid = []
    for N in _ints(args.convoy_n):
        for H in _ints(args.convoy_h):
            for mode in _ints(args.convoy_modes):
                upd, acc_runs = [], []
                for r in range(args.runs):
                    seed = (0 if args.seed is None else args.seed) + 1000 * r + N
                    sc = scenes.convoy_scene(N, seed, steps=steps, h_max=H)
                    cfg = sc.filter_config(score_mode=mode)
                    f = glmb.Filter(cfg)
                    B = [glmb.births_array(fr.births, sc.dim_x) for fr in sc.frames]
                    for k, fr in enumerate(sc.frames):            # untimed: graph captures
                        f.step(B[k], fr.Z)
                    f.reset()
                    acc = RunAccuracy()
                    t_run = []
                    for k, fr in enumerate(sc.frames):
                        t0 = time.perf_counter()
                        f.step(B[k], fr.Z)
                        e = f.estimates(cap=256, pmf_cap=64)
                        t_run.append(time.perf_counter() - t0)
                        acc.add(e["mean"][:, :2], fr.truth[:, :2])
                    f.close()
                    upd.append(1000.0 * statistics.fmean(t_run))
                    acc_runs.append(acc.summary())
                row = dict(N=N, H_max=H, mode=mode, runs=args.runs, steps=steps,
                           update_ms=statistics.fmean(upd),
                           update_ms_sem=(statistics.stdev(upd) / math.sqrt(len(upd)) if len(upd) > 1 else 0.0),
                           rel_card_error=statistics.fmean(a["rel_card_error"] for a in acc_runs),
                           tracking_error_m=statistics.fmean(a["tracking_error_m"] for a in acc_runs))
                if mode == 0 and args.convoy_oracle_steps > 0:
                    sc = scenes.convoy_scene(N, 0 if args.seed is None else args.seed, steps=args.convoy_oracle_steps,
                                             h_max=H)
                    o = oracle.Oracle(sc.filter_config())
                    t0 = time.perf_counter()
                    for fr in sc.frames:
                        o.step(fr.births, fr.Z)
                        o.estimates()
                    row["oracle_ms"] = 1000.0 * (time.perf_counter() - t0) / len(sc.frames)
                    row["oracle_steps"] = len(sc.frames)
                grid.append(row)
                print(json.dumps(row), file=sys.stderr, flush=True)
    print(json.dumps({"metric": "convoy update time and accuracy (Section 4.1 grid, 1 GB300)",
                      "unit": "ms/update", "higher_is_better": False, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": f"convoy, D=5, lambda=0, sigma=0.25, delta=2, H_up=100, "
                                             f"tau=1e-5, {steps} steps of 0.1 s",
                                 "update": "glmb_step, host detections + estimates read back"},
                      "grid": grid}))


def run_sweep(args, glmb, torch, dev):
    """The 3-D scalability grid: N objects alive from frame 0 (held near N by
    Poisson(0.01 N) births per frame), clutter Poisson(50), P_D 0.85,
    1 + Poisson(2) detections, 50 frames, for N in --sweep-n and H_max in
    --sweep-h.  Per cell: one untimed pass fills the graph cache, then every
    frame is timed with CUDA events (detections resident, L2 flushed between
    frames, estimates read back inside the frame).  Reports frames/s over
    all frames and over frames 10-49 (after the birth transient) and
    hypothesis-track updates/s.  The FP64 oracle (all host threads) is timed
    on the first --sweep-oracle-frames frames of the cells with N * H_max up
    to --sweep-oracle-max, the rest are "not run"."""
    import oracle
    grid = []
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for N in _ints(args.sweep_n):
        for H in _ints(args.sweep_h):
            sc = scenes.make_scene(scenes.preset(f"sweep_N{N}", h_max=H),
                                   3000 + N if args.seed is None else args.seed)
            cfg = filter_cfg(sc)
            try:
                row = _sweep_cell(args, glmb, torch, dev, flush, sc, cfg)
            except glmb.GlmbError as e:
                row = dict(error=str(e))
            row = dict(N=N, H_max=H, **row)
            if N * H <= args.sweep_oracle_max and args.sweep_oracle_frames > 0:
                threads = os.cpu_count() or 1
                o = oracle.Oracle(cfg, n_threads=threads)
                per = []
                for fr in sc.frames[:args.sweep_oracle_frames]:
                    t0 = time.perf_counter()
                    o.step(fr.births, fr.Z)
                    o.estimates()
                    per.append(time.perf_counter() - t0)
                row["oracle_ms_last_frame"] = 1e3 * per[-1]
                row["oracle"] = f"frames 0..{len(per) - 1}, {threads} threads"
                if "frame_ms" in row:
                    row["gpu_ms_same_frame"] = row["frame_ms"][len(per) - 1]
            else:
                row["oracle"] = "not run"
            row.pop("frame_ms", None)
            grid.append(row)
            print(json.dumps(row), file=sys.stderr, flush=True)
    print(json.dumps({"metric": "3-D sweep: GLMB update frames/s and hypothesis-track updates/s vs N, H_max (1 GB300)",
                      "unit": "frames/s", "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": "3-D CV in [0,5000]^3, N alive from frame 0, clutter Poisson(50), "
                                             "P_D 0.85, 1+Poisson(2) detections, 50 frames, H_up=100",
                                 "l2": "flushed between frames (256 MiB write, outside the timed events)"},
                      "grid": grid}))


def _sweep_cell(args, glmb, torch, dev, flush, sc, cfg):
    """One (N, H_max) cell of the sweep: per-frame CUDA-event times."""
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    f = glmb.Filter(cfg, stream=stream.cuda_stream)
    try:
        Zdev = [torch.from_numpy(fr.Z).to(dev) for fr in sc.frames]
        B = [glmb.births_array(fr.births, sc.dim_x) for fr in sc.frames]
        for k in range(len(sc.frames)):                    # untimed: graph captures
            f.step(B[k], Zdev[k], device=True)
        f.estimates(cap=cfg["max_tracks"], pmf_cap=64)
        f.reset()
        torch.cuda.synchronize()
        times, entries, hyps = [], [], []
        for k in range(len(sc.frames)):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            f.step(B[k], Zdev[k], device=True)
            f.estimates(cap=cfg["max_tracks"], pmf_cap=64)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            info = f.info()
            entries.append(info["n_entries"])
            hyps.append(info["n_hyp"])
    finally:
        f.close()
        torch.cuda.synchronize()
    steady = slice(10, len(times))
    return dict(frames=len(times),
                frames_per_s=len(times) / (sum(times) / 1e3),
                frames_per_s_steady=len(times[steady]) / (sum(times[steady]) / 1e3),
                ms_per_frame_steady=statistics.fmean(times[steady]),
                hypothesis_track_updates_per_s=sum(entries) / (sum(times) / 1e3),
                hypothesis_track_updates_per_s_steady=sum(entries[steady]) / (sum(times[steady]) / 1e3),
                mean_M=statistics.fmean(len(fr.Z) for fr in sc.frames),
                mean_hypotheses_steady=statistics.fmean(hyps[steady]), frame_ms=times)


def _timed_run(f, frames, B, Zdev, torch, stream, flush, truth_dim, lost=False):
    """One pass of the scene through glmb_step with per-frame CUDA-event
    times (after an untimed pass that fills the graph cache); returns
    times, OSPA per frame, pairs after / before the gate, lost mass."""
    from scenes.metrics import ospa
    f.set_profiling(["table", "expand", "select", "materialize"])
    for k in range(len(frames)):
        f.step(B[k], Zdev[k], device=True)
    f.reset()
    torch.cuda.synchronize()
    f.set_profiling(["table", "expand", "select", "materialize"])   # clears the totals
    times, osp, pairs, pre, lm = [], [], [], [], []
    for k, fr in enumerate(frames):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        f.step(B[k], Zdev[k], device=True)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        est = f.estimates(cap=f.cfg["max_tracks"], pmf_cap=64)
        osp.append(ospa(est["mean"][:, :truth_dim], fr.truth[:, :truth_dim], c=100.0))
        info = f.info()
        pairs.append(info["n_pairs"])
        pre.append(info["n_pairs_pregate"])
        if lost:
            _, flag = f.gate_usage()
            w = np.exp(f.hypotheses()["logw"])
            lm.append(float(np.sum(w * flag) / np.sum(w)))
    stages = {k: v[0] / max(v[1], 1) for k, v in f.timing().items() if v[1]}
    return times, osp, pairs, pre, lm, stages


def run_gate(args, glmb, torch, dev):
    """The learned pair gate on the 3-D workload (N objects alive from frame
    0, clutter Poisson(50), P_D 0.85, 1 + Poisson(2) detections, H_max):
    training data (features and usage labels) from the ungated filter on
    --gate-train scenes, training by the library's kernels, a threshold that
    keeps --gate-keep of the used training pairs, then --gate-eval held-out
    scenes run three ways: without the gate (frame time, OSPA), with the gate
    scoring only (lost mass: the weight of retained hypotheses that use a
    pair the gate would prune) and with the gate pruning (frame time, OSPA,
    pairs).  Repeated for each base Mahalanobis gate tail in --gate-tails."""
    from paper_2512_06230_gb300 import gate as G
    N, H, F = args.gate_n, args.gate_h, args.gate_frames
    base = scenes.preset("sweep_N200", n_objects=N, births_per_frame=0.01 * N, h_max=H, frames=F)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    rows = []
    for tail in [float(t) for t in args.gate_tails.split(",")]:
        def cfg_for(sc):
            c = filter_cfg(sc)
            c["gate"] = scenes.chi2_gate(3, tail)
            c["max_pairs"] = 1 << 22
            return c
        t0 = time.perf_counter()
        Xs, ys = [], []
        for s in range(args.gate_train):
            sc = scenes.make_scene(base, 50000 + s)
            X, y = G.collect(cfg_for(sc), [(glmb.births_array(fr.births, sc.dim_x), fr.Z) for fr in sc.frames],
                             skip=2)
            Xs.append(X)
            ys.append(y)
        X, y = np.concatenate(Xs), np.concatenate(ys)
        t_collect = time.perf_counter() - t0
        t0 = time.perf_counter()
        params, hist = G.train(X, y, steps=args.gate_steps, batch=32768, lr=2e-3, seed=1, log_every=500)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        thr = G.threshold(params, X, y, keep_used=args.gate_keep)
        z = G.logits(params, X)
        keep = z >= thr
        ev = dict(plain_ms=[], gated_ms=[], plain_ospa=[], gated_ospa=[], plain_pairs=[], gated_pairs=[],
                  lost=[], plain_stages=[], gated_stages=[])
        for s in range(args.gate_eval):
            sc = scenes.make_scene(base, 60000 + s)
            cfg = cfg_for(sc)
            Zdev = [torch.from_numpy(fr.Z).to(dev) for fr in sc.frames]
            B = [glmb.births_array(fr.births, sc.dim_x) for fr in sc.frames]
            for mode in ("plain", "score", "gated"):
                f = glmb.Filter(cfg, stream=stream.cuda_stream)
                if mode == "score":
                    f.set_gate(params, thr, glmb.Filter.GATE_SCORE)
                elif mode == "gated":
                    f.set_gate(params, thr, glmb.Filter.GATE_PRUNE)
                try:
                    tm, osp, pairs, pre, lm, stg = _timed_run(f, sc.frames, B, Zdev, torch, stream, flush, 3,
                                                              lost=(mode == "score"))
                finally:
                    f.close()
                if mode != "score":
                    ev[mode + "_stages"].append(stg)
                if mode == "plain":
                    ev["plain_ms"] += tm[2:]
                    ev["plain_ospa"] += osp
                    ev["plain_pairs"] += pairs[2:]
                elif mode == "score":
                    ev["lost"] += lm[2:]
                else:
                    ev["gated_ms"] += tm[2:]
                    ev["gated_ospa"] += osp
                    ev["gated_pairs"] += pairs[2:]
            del Zdev
        row = {"gate_tail": tail, "gate_G": scenes.chi2_gate(3, tail), "threshold": thr,
               "train": {"scenes": args.gate_train, "frames_per_scene": F - 2, "pairs": int(len(y)),
                         "used_fraction": float(y.mean()), "collect_s": round(t_collect, 2),
                         "train_s": round(t_train, 2), "steps": args.gate_steps,
                         "loss_history": hist, "used_kept": float(keep[y > 0].mean()),
                         "pairs_kept": float(keep.mean())},
               "held_out": {"scenes": args.gate_eval,
                            "plain_ms_per_frame": statistics.fmean(ev["plain_ms"]),
                            "gated_ms_per_frame": statistics.fmean(ev["gated_ms"]),
                            "speedup": statistics.fmean(ev["plain_ms"]) / statistics.fmean(ev["gated_ms"]),
                            "plain_pairs_per_frame": statistics.fmean(ev["plain_pairs"]),
                            "gated_pairs_per_frame": statistics.fmean(ev["gated_pairs"]),
                            "lost_mass_mean": statistics.fmean(ev["lost"]),
                            "lost_mass_max": max(ev["lost"]),
                            "ospa_plain": statistics.fmean(ev["plain_ospa"]),
                            "ospa_gated": statistics.fmean(ev["gated_ospa"]),
                            "stage_ms_plain": {k: statistics.fmean(d[k] for d in ev["plain_stages"])
                                               for k in ev["plain_stages"][0]},
                            "stage_ms_gated": {k: statistics.fmean(d[k] for d in ev["gated_stages"])
                                               for k in ev["gated_stages"][0]}}}
        rows.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    print(json.dumps({"metric": "learned pair gate: frame time, lost mass and OSPA, gated vs plain (1 GB300)",
                      "unit": "ms/frame", "higher_is_better": False, "dtype": "bf16 (gate MLP) / f32",
                      "data": "synthetic",
                      "config": {"workload": f"3-D CV in [0,5000]^3, N={N}, H_max={H}, H_up=100, clutter Poisson(50), "
                                             f"P_D 0.85, 1+Poisson(2) detections, {F} frames per scene (first 2 "
                                             "not scored)", "ospa": "c = 100 m, p = 1, MAP estimates",
                                 "l2": "flushed between frames"},
                      "rows": rows}))


def run_mlp(args, glmb, torch, dev):
    """The learned gate's MLP kernels alone on --mlp-rows synthetic feature
    rows (features resident in device memory): forward (glmb_mlp_forward)
    and forward + backward (glmb_mlp_backward), --steps timed launches each
    after --warmup, CUDA events on the launching stream.  Dense work per row:
    forward 2 (5*64 + 64*64 + 64*64 + 64) flops, the backward's two
    activation-gradient products and three weight-gradient products add
    2 (2*64*64 + 5*64 + 2*64*64 + 64) more after its own forward."""
    rng = np.random.default_rng(0 if args.seed is None else args.seed)
    n = args.mlp_rows
    X = np.stack([rng.chisquare(2, n) * 3, rng.gamma(2.0, 4.0, n), rng.uniform(0, 1, n),
                  rng.integers(0, 40, n).astype(float), rng.normal(5.0, 1.5, n)], 1).astype(np.float32)
    mu, sd = X.mean(0), X.std(0)
    from paper_2512_06230_gb300 import gate as G
    P = torch.from_numpy(G.init_params(1, mu, sd)).to(dev)
    Xd = torch.from_numpy(X).to(dev)
    y = torch.from_numpy((rng.uniform(size=n) < 0.3).astype(np.float32)).to(dev)
    wt = torch.full((n,), 1.0 / n, device=dev)
    grad = torch.zeros(glmb.GATE_NPARAM, device=dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    out = {}
    f_fwd = 2.0 * (5 * 64 + 64 * 64 + 64 * 64 + 64)
    f_bwd = f_fwd + 2.0 * (2 * 64 * 64 + 5 * 64 + 2 * 64 * 64 + 64)
    for name, call, flops in (("forward", lambda: glmb.mlp_forward(P, Xd, err), f_fwd),
                              ("forward+backward", lambda: glmb.mlp_backward(P, Xd, y, wt, grad, loss, err), f_bwd)):
        for _ in range(args.warmup):
            call()
        torch.cuda.synchronize()
        st = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(args.steps):
            call()
        e1.record(st)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        out[name] = dict(ms=ms, rows_per_s=n / (ms / 1e3), tflops=n * flops / (ms * 1e-3) / 1e12)
    assert int(err.item()) == 0
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = peaks.get("bf16_tflops", 1900.0)
    fw = out["forward"]
    print(json.dumps({"metric": "learned-gate MLP rows/s (5-64-64-64-1 GELU, bf16 tcgen05)", "value": fw["rows_per_s"],
                      "unit": "rows/s", "higher_is_better": True, "dtype": "bf16 x bf16 -> f32", "data": "synthetic",
                      "config": {"workload": f"{n} feature rows resident in device memory", "rows": n},
                      "kernels": out,
                      "roofline": {"bound": "tensor", "achieved": fw["tflops"], "peak": peak, "unit": "TFLOP/s",
                                   "frac": fw["tflops"] / peak,
                                   "peak_source": "MEASURED_PEAKS.json bf16_tflops" if "bf16_tflops" in peaks
                                   else "fallback 1900"}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10,
                    help="untimed warm-up steps (after the set-up pass that captures the frame graphs)")
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--scene", default="mid")
    ap.add_argument("--seed", type=int, default=None)
    ap.add_argument("--no-flush", action="store_true")
    ap.add_argument("--no-precapture", action="store_true",
                    help="skip the untimed set-up pass that captures the scene's frame graphs")
    ap.add_argument("--cpu-budget", type=float, default=25.0)
    ap.add_argument("--cpu-threads", type=int, default=0,
                    help="host threads of the oracle leg (0: all cores)")
    ap.add_argument("--stages", action="store_true", help="also report per-stage times")
    ap.add_argument("--batch-detections", default="device", choices=["device", "host"],
                    help="--scene batch: detections resident in device memory or copied from the host")
    ap.add_argument("--scenes", type=int, default=64,
                    help="--scene batch: independent scenes per frame")
    ap.add_argument("--convoy-n", default="1,2,5,10,20", help="--scene convoy: object counts")
    ap.add_argument("--convoy-h", default="5,10,25,50,100", help="--scene convoy: H_max values")
    ap.add_argument("--convoy-modes", default="0,1", help="--scene convoy: score modes")
    ap.add_argument("--convoy-steps", type=int, default=548)
    ap.add_argument("--convoy-oracle-steps", type=int, default=20)
    ap.add_argument("--runs", type=int, default=3, help="--scene convoy: seeds per configuration")
    ap.add_argument("--sweep-n", default="50,200,500,1000", help="--scene sweep: object counts")
    ap.add_argument("--sweep-h", default="1000,5000,20000", help="--scene sweep: H_max values")
    ap.add_argument("--sweep-oracle-frames", type=int, default=4)
    ap.add_argument("--sweep-oracle-max", type=int, default=200 * 1000,
                    help="--scene sweep: largest N * H_max the oracle is timed on")
    ap.add_argument("--gate-n", type=int, default=300, help="--scene gate: objects")
    ap.add_argument("--gate-h", type=int, default=5000, help="--scene gate: H_max")
    ap.add_argument("--gate-frames", type=int, default=30)
    ap.add_argument("--gate-train", type=int, default=40, help="--scene gate: training scenes")
    ap.add_argument("--gate-eval", type=int, default=8, help="--scene gate: held-out scenes")
    ap.add_argument("--gate-steps", type=int, default=3000)
    ap.add_argument("--gate-keep", type=float, default=0.99999, help="fraction of used training pairs kept")
    ap.add_argument("--gate-tails", default="1e-4,1e-12,1e-30", help="chi-square tails of the base gate")
    ap.add_argument("--mlp-rows", type=int, default=1 << 22, help="--scene mlp: feature rows")
    ap.add_argument("--profile-frames", type=int, default=0,
                    help="only run this many frames of the scene through glmb_step (for ncu captures) and exit")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        sc = scene_for_rank(args, 0)
        cfg = filter_cfg(sc)
        v, threads, sample = run_oracle(args, sc, cfg, min(args.cpu_budget, 20.0 + 2 * args.steps))
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / v,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": workload_config(args, sc, cfg),
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                                 "sample": sample},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2512_06230_gb300 as glmb
    if rank == 0:
        glmb.build()
    if world > 1:
        torch.distributed.barrier()
    glmb.load()

    if args.scene == "batch":
        return run_batch(args, glmb, torch, dev)
    if args.scene == "convoy":
        return run_convoy(args, glmb, torch)
    if args.scene == "sweep":
        return run_sweep(args, glmb, torch, dev)
    if args.scene == "gate":
        return run_gate(args, glmb, torch, dev)
    if args.scene == "mlp":
        return run_mlp(args, glmb, torch, dev)

    sc = scene_for_rank(args, rank)
    cfg = filter_cfg(sc)
    F = len(sc.frames)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    f = glmb.Filter(cfg, stream=stream.cuda_stream)
    Zdev = [torch.from_numpy(fr.Z).to(dev) if len(fr.Z) else torch.zeros((0, sc.dim_z), device=dev)
            for fr in sc.frames]
    Bhost = [glmb.births_array(fr.births, sc.dim_x) for fr in sc.frames]
    if args.profile_frames:
        for k in range(args.profile_frames):
            fr = sc.frames[k % F]
            if k % F == 0:
                f.reset()
            f.step(Bhost[k % F], Zdev[k % F], device=True)
        torch.cuda.synchronize()
        print(json.dumps({"profile_frames": args.profile_frames, "info": {
            k: v for k, v in f.info().items() if isinstance(v, (int, float))}}))
        return
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    h_up = cfg["h_up"]

    host_times = []

    def run(n_steps, start, host):
        """Runs n_steps frames starting at global step index `start`; returns
        per-step event times (ms) and per-step work counters."""
        times, work = [], []
        host_times.clear()
        for s in range(start, start + n_steps):
            fi = s % F
            fr = sc.frames[fi]
            if not args.no_flush:
                flush.zero_()
            info0 = f.info() if fi != 0 else None
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if fi == 0:
                f.reset()
            t0 = time.perf_counter()
            if host:
                f.step(Bhost[fi], fr.Z)
            else:
                f.step(Bhost[fi], Zdev[fi], device=True)
            t1 = time.perf_counter()
            est = f.estimates(cap=cfg["max_tracks"], pmf_cap=64)
            t2 = time.perf_counter()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            host_times.append((t1 - t0, t2 - t1))
            info = f.info()
            H_par = 1 if info0 is None else info0["n_hyp"]
            E_par = 0 if info0 is None else info0["n_entries"]
            M = len(fr.Z)
            work.append(dict(entries=info["n_entries"], n_est=est["n"], M=M,
                             draws=h_up * (E_par + H_par * (len(fr.births) + M)),
                             h2d=fr.Z.nbytes + len(fr.births) * 43 * 8,
                             d2h=est["n"] * 352 + 64 * 8))
        return times, work

    # set-up: one untimed pass over the scene captures the frame graphs of
    # every plan the scene needs (a reset restarts the planning state, so a
    # later pass replays the same plans); then the warm-up, then the timed
    # steps.  The expansion is timed with events in every run (the same mask
    # throughout, so the set-up pass's graphs are reused).
    f.set_profiling(["expand"])
    precapture = 0 if args.no_precapture else F
    if precapture:
        run(precapture, 0, host=False)
    run(args.warmup, 0, host=False)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk_lines, stop = [], threading.Event()
    th = threading.Thread(target=sample_clocks, args=(stop, clk_lines), daemon=True)
    th.start()
    time.sleep(0.3)
    info_t0 = f.info()
    launches0 = info_t0["n_launches"]
    torch.cuda.synchronize()
    f.set_profiling(["expand"])   # clears the totals
    times, work = run(args.steps, args.warmup, host=False)
    torch.cuda.synchronize()
    host_step_ms = 1e3 * sum(t[0] for t in host_times) / max(1, len(host_times))
    host_est_ms = 1e3 * sum(t[1] for t in host_times) / max(1, len(host_times))
    info1 = f.info()
    launches = info1["n_launches"] - launches0
    tim = f.timing()
    stop.set()
    th.join(timeout=10)
    total_ms = max_over_ranks(float(sum(times)), dev, world)
    if world > 1:
        torch.distributed.barrier()
    # end to end through the host-buffer path
    times_h, work_h = run(args.steps, args.warmup, host=True)
    total_h = max_over_ranks(float(sum(times_h)), dev, world)
    stage = None
    if args.stages:
        f.set_profiling(list(glmb.Filter.STAGES))
        run(args.steps, args.warmup, host=False)
        stage = {k: {"ms_per_step": v[0] / max(v[1], 1), "calls": v[1]} for k, v in f.timing().items()}
        f.set_profiling([])

    if rank != 0:
        return
    frames = args.steps * world
    value = job_rate(args.steps, world, total_ms)
    entries = sum(w["entries"] for w in work)
    # roofline of the dominant kernel (child expansion): integer ALU work of
    # the counter-based sampler, 100 32-bit operations per Philox4x32-10
    # call and one call per four uniforms, one uniform per slot and per
    # detection row of every child drawn
    exp_ms, exp_calls = tim["expand"]
    draws = sum(w["draws"] for w in work)
    ops = 25.0 * draws
    clocks = summarize_clocks(clk_lines, local)
    peak_ops = 152 * 128 * 2070e6
    achieved = ops / (exp_ms / 1000.0) if exp_ms > 0 else None
    cpu_v, cpu_threads, cpu_sample = run_oracle(args, sc, cfg, args.cpu_budget)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {**workload_config(args, sc, cfg),
                   "l2": "flushed between steps (256 MiB write, outside "
                   "the timed events)" if not args.no_flush else "not flushed",
                   "inputs": "detections resident in device memory; births (<1 KB) copied in predict",
                   "graph_precapture_frames": precapture},
        "hypothesis_track_updates_per_s": entries * world / (total_ms / 1000.0),
        "e2e": {"value": frames / (total_h / 1000.0), "unit": UNIT,
                "h2d_bytes_per_step": sum(w["h2d"] for w in work_h) / len(work_h),
                "d2h_bytes_per_step": sum(w["d2h"] for w in work_h) / len(work_h)},
        "gpu_launches": int(launches),
        "host_ms_per_step": {"step_call": round(host_step_ms, 4), "estimates_call": round(host_est_ms, 4)},
        "graphs": {"captured": info1["n_graph_captures"], "replayed": info1["n_graph_launches"],
                   "captured_in_timed_steps": info1["n_graph_captures"] - info_t0["n_graph_captures"],
                   "redone_frames": info1["n_redo"],
                   "capture_ms_total": round(info1["graph_capture_ms"], 3)},
        "expand_plan": {"smem_bytes": info1["expand_smem_bytes"],
                        "ctas_per_sm": info1["expand_ctas_per_sm"],
                        "threads": info1["expand_threads"],
                        "T": info1["expand_plan_T"], "K": info1["expand_plan_K"],
                        "M": info1["expand_plan_M"]},
        "roofline": {"bound": "alu", "kernel": "child expansion and scoring (stage_kernel, draw_kernel, warp_kernel, dedup_kernel of one frame)",
                     "achieved": achieved / 1e12 if achieved else None,
                     "peak": peak_ops / 1e12, "unit": "Tops/s (int32 lane ops)",
                     "frac": achieved / peak_ops if achieved else None, "traffic": expansion_traffic(),
                     "peak_source": INT_PEAK_NOTE,
                     "kernel_ms_per_step": exp_ms / max(exp_calls, 1),
                     "kernel_share_of_step": exp_ms / total_ms if total_ms else None},
        "cpu_baseline": {"value": cpu_v, "unit": UNIT, "cores": cpu_threads, "kind": "oracle",
                         "sample": cpu_sample},
        "clocks": clocks,
    }
    if stage:
        line["stages"] = stage
    print(json.dumps(line))


if __name__ == "__main__":
    main()
