"""Throughput of the multi-detection GLMB update on one GB300.

A step is one frame of the whole update (predict, compatibility table,
death probabilities, child expansion and scoring, normalisation and top-H,
track update, estimates).  The default workload is the largest cell of the
3-D scalability sweep whose hypothesis cap binds: N = 200 objects held near
N (deaths at P_S 0.99, Poisson(0.01 N) births per frame) in [0, 5000]^3,
clutter Poisson(50), P_D 0.85, 1 + Poisson(2) detections per detected
object, H_max = 20000, H_up = 100, 50 frames.  Steps walk the steady frames
10-49 in order and wrap; the filter reaches a window frame by a reset and an
untimed replay of the frames before it, so the timed frames do not depend
on --steps.  Before the warm-up steps, one untimed set-up pass over the
scene captures the frame graphs its plans need.  Further cells (N = 1000 and
N = 50 of the sweep, and the 2-D mid scene) are measured the same way and
reported under "cells".

value  frames/s with each frame's detections already in device memory.
e2e    frames/s of the same frames through the same C ABI with host
       buffers: detections copied host->device and the estimates read back
       inside every step.
Every step is timed alone with CUDA events on the filter's stream; a 256 MiB
buffer is written before it to flush L2 (outside the events).  Under
torchrun every rank runs its own independent scene (no collective on the
data path); value is the frames of all ranks over the slowest rank's time.

cpu_baseline times the FP64 CPU oracle on the host cores on a bounded sample
of the workload (the last frame it reaches from the initial GLMB within
--cpu-budget seconds); oracle_error re-runs one frame of the workload from
the oracle's own state and reports the library's largest error against the
oracle for every output.  --impl reference prints the oracle's line alone.
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

# The default workload: the largest cell of the 3-D scalability sweep whose
# hypothesis cap binds (N = 200 objects, H_max = 20000: about 10^4 retained
# hypotheses of about 200 tracks each, 580 detections per frame), timed on
# its steady-state frames 10-49 (frames 0-9 are the transient in which the
# hypothesis count grows to the cap).  Extra cells of the same sweep are
# measured with the same protocol and reported in the same line.
DEFAULT_SCENE = "sweep_N200"
DEFAULT_H_MAX = 20000
PARTICLES = 256           # particles per track of the ctrv_N<n> (particle model) cells
DEFAULT_EXTRA = "sweep_N1000:20000,sweep_N50:1000,mid,ctrv_N200:1000"


def expansion_traffic(workload=DEFAULT_SCENE):
    """DRAM bytes per frame of the expansion kernels on a workload, from the
    committed ncu summary profiles/expansion_traffic_<workload>.md, or None
    when there is none or the kernels changed since it was captured."""
    import hashlib
    try:
        txt = open(os.path.join(ROOT, "profiles", f"expansion_traffic_{workload}.md")).read()
        src = open(os.path.join(ROOT, "paper_2512_06230_gb300", "csrc", "kernels_expand.cu"), "rb").read()
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


def scene_params(name: str, h_max=None):
    """Scene parameters and the seed base of a named workload: "sweep_N<n>"
    (3-D sweep, seed 3000 + n), "mid" (2-D, seed 2000), "tiny" (seed 1000)."""
    if name.startswith("sweep_N"):
        p = scenes.preset(name, h_max=DEFAULT_H_MAX if h_max is None else h_max)
        return p, 3000 + p.n_objects
    if name.startswith("ctrv_N"):   # particle track model (CTRV vehicles)
        n = int(name[len("ctrv_N"):])
        p = scenes.CtrvParams(name=name, n_objects=n, frames=40, h_max=1000 if h_max is None else h_max,
                              clutter_rate=0.2 * n, n_particles=PARTICLES)
        return p, 5000 + n
    p = scenes.preset(name) if h_max is None else scenes.preset(name, h_max=h_max)
    return p, {"tiny": 1000, "mid": 2000}.get(name, 2000)


def window_start(name: str) -> int:
    """First frame of the steady window: after the birth transient."""
    if name.startswith("sweep_N"):
        return 10
    if name.startswith("ctrv_N"):
        return 20
    return {"tiny": 25, "mid": 50}.get(name, 0)


def scene_for_rank(args, rank, name=None, h_max=None):
    """The scene a rank runs: every rank its own seed (independent scenes)."""
    name = args.scene if name is None else name
    p, base = scene_params(name, getattr(args, "h_max", None) if h_max is None else h_max)
    seed = base + 7919 * rank if args.seed is None else args.seed + rank
    if isinstance(p, scenes.CtrvParams):
        return scenes.ctrv_scene(p, seed)
    return scenes.make_scene(p, seed)


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


def run_oracle(args, sc, cfg, budget_s, state_frame=None):
    """The FP64 oracle on the host cores over a bounded sample of the
    workload: from the initial GLMB it steps the scene's frames in order
    until budget_s is spent (the frame in progress is finished); the rate is
    that of the last frame it completed, the largest of the sample (the
    hypothesis count grows over the first frames), whose predecessors only
    build its state.  With state_frame set, the oracle's own state before
    that frame is also returned (for an error report against the GPU).
    Returns (frames/s, threads, sample text, details, state)."""
    import oracle
    threads = args.cpu_threads if args.cpu_threads > 0 else (os.cpu_count() or 1)
    o = oracle.Oracle(cfg, n_threads=threads)
    t_start = time.perf_counter()
    per, state = [], None
    for k, fr in enumerate(sc.frames):
        if state_frame is not None and k == state_frame:
            state = o.export_state()
        t0 = time.perf_counter()
        o.step(fr.births, fr.Z)
        o.estimates()
        per.append((k, time.perf_counter() - t0, o.num_parents()))
        if time.perf_counter() - t_start > budget_s:
            break
    if state_frame is not None and state is None and len(per) > state_frame:
        state = o.export_state()
    k, dt, parents = per[-1]
    total = time.perf_counter() - t_start
    sample = (f"frame {k} of the {sc.params.name} scene (seed {sc.seed}; {parents} parent hypotheses, "
              f"{len(sc.frames[k].Z)} detections), reached by the oracle itself from the initial GLMB through "
              f"frames 0..{k - 1} untimed; {dt:.2f} s for the frame, {total:.1f} s in all, {threads} threads")
    details = {"frames": [{"frame": a, "s": round(b, 4), "parents": c} for a, b, c in per]}
    return 1.0 / dt, threads, sample, details, state


def workload_config(args, sc, cfg, w0=None) -> dict:
    """The workload of the default run, named the same in both arms."""
    F = len(sc.frames)
    w0 = window_start(sc.params.name) if w0 is None else w0
    p = sc.params
    if isinstance(p, scenes.CtrvParams):
        shape = (f"{p.name} cell: {p.n_objects} CTRV vehicles, {p.n_particles} FP64 particles per track, "
                 f"H_max={cfg['h_max']}, clutter Poisson({p.clutter_rate:g}), P_D {p.p_d:g}, "
                 f"1+Poisson({p.lambda_d:g}) detections")
    elif p.dim == 3:
        shape = (f"3-D sweep cell N={p.n_objects}, H_max={cfg['h_max']}: CV in [0,{p.extent:g}]^3, "
                 f"clutter Poisson({p.clutter_rate:g}), P_D {p.p_d:g}, 1+Poisson({p.lambda_d:g}) detections")
    else:
        shape = (f"{p.name} scene: 2-D CV, {p.n_objects} objects, clutter Poisson({p.clutter_rate:g}), "
                 f"H_max={cfg['h_max']}")
    return {"workload": f"{shape}, H_up={cfg['h_up']}; steady frames {w0}-{F - 1} of a {F}-frame scene, cycled",
            "scene": p.name, "n_objects": p.n_objects, "h_max": cfg["h_max"], "h_up": cfg["h_up"],
            "frames_per_scene": F, "timed_frames": [w0, F - 1], "seed": sc.seed}


class Cell:
    """One workload stepped by the library: steps walk the steady window
    [w0, F) in order and wrap; the filter is brought to a window frame by a
    reset and an untimed replay of the frames before it (the filter is
    deterministic, so a replay reproduces the state exactly).  Every step
    is timed alone with CUDA events on the filter's stream; L2 is flushed
    before it, outside the events."""

    def __init__(self, glmb, torch, dev, sc, cfg, w0, stages=("expand", "select"), flush=None):
        self.glmb, self.torch, self.sc, self.cfg, self.w0 = glmb, torch, sc, cfg, w0
        self.F = len(sc.frames)
        self.stream = torch.cuda.Stream(dev)
        torch.cuda.set_stream(self.stream)
        self.f = glmb.Filter(cfg, stream=self.stream.cuda_stream)
        self.Zdev = [torch.from_numpy(fr.Z).to(dev) if len(fr.Z) else torch.zeros((0, sc.dim_z), device=dev)
                     for fr in sc.frames]
        self.B = [glmb.births_array(fr.births, sc.dim_x) for fr in sc.frames]
        self.flush = flush
        self.stages = list(stages)
        self.f.set_profiling(self.stages)
        self.pos = 0
        torch.cuda.synchronize()

    def close(self):
        self.f.close()
        self.torch.cuda.synchronize()

    def goto(self, k):
        """Reset, then step frames 0..k-1 untimed."""
        self.f.reset()
        for j in range(k):
            self.f.step(self.B[j], self.Zdev[j], device=True)
        self.pos = k

    def precapture(self):
        """One untimed pass over the whole scene: captures the frame graph of
        every plan the scene needs (a later pass replays them)."""
        self.goto(self.F)
        self.f.estimates(cap=self.cfg["max_tracks"], pmf_cap=64)
        self.torch.cuda.synchronize()

    def run(self, n_steps, start, host=False):
        """Steps start .. start + n_steps - 1 of the window cycle; returns per
        step: event time (ms), stage times, launches and work counters."""
        torch, f, cfg = self.torch, self.f, self.cfg
        W = self.F - self.w0
        out = []
        for s in range(start, start + n_steps):
            fi = self.w0 + s % W
            if self.pos != fi:
                self.goto(fi)
            fr = self.sc.frames[fi]
            info0 = f.info()
            tim0 = f.timing()
            if self.flush is not None:
                self.flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            if host:
                f.step(self.B[fi], fr.Z)
            else:
                f.step(self.B[fi], self.Zdev[fi], device=True)
            est = f.estimates(cap=cfg["max_tracks"], pmf_cap=64)
            e1.record(self.stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            info = f.info()
            tim = f.timing()
            self.pos = fi + 1
            M = len(fr.Z)
            out.append(dict(
                ms=ms, frame=fi, M=M, parents=info0["n_hyp"], retained=info["n_hyp"],
                entries=info["n_entries"], children=info["n_children"], unique=info["n_unique"],
                n_est=est["n"], launches=info["n_launches"] - info0["n_launches"],
                captures=info["n_graph_captures"] - info0["n_graph_captures"],
                redo=info["n_redo"] - info0["n_redo"],
                draws=cfg["h_up"] * (info0["n_entries"] + info0["n_hyp"] * (len(fr.births) + M)),
                stage_ms={k: tim[k][0] - tim0.get(k, (0.0, 0))[0] for k in tim},
                h2d=(fr.Z.nbytes + len(fr.births) * 43 * 8) if host else 0,
                d2h=est["n"] * 352 + 64 * 8))
        return out


def summarize(steps, world=1):
    """Rates of a list of step records (one rank)."""
    ms = sum(s["ms"] for s in steps)
    n = len(steps)
    return dict(frames_per_s=n / (ms / 1e3), ms_per_step=ms / n,
                hypothesis_track_updates_per_s=sum(s["entries"] for s in steps) / (ms / 1e3),
                mean_parents=statistics.fmean(s["parents"] for s in steps),
                mean_retained=statistics.fmean(s["retained"] for s in steps),
                mean_M=statistics.fmean(s["M"] for s in steps),
                children_per_step=statistics.fmean(s["children"] for s in steps),
                launches=sum(s["launches"] for s in steps),
                captures_in_timed_steps=sum(s["captures"] for s in steps),
                redone_frames=sum(s["redo"] for s in steps),
                stage_ms_per_step={k: sum(s["stage_ms"].get(k, 0.0) for s in steps) / n
                                   for k in steps[0]["stage_ms"]})


def rooflines(steps, peaks, workload=DEFAULT_SCENE):
    """Roofline objects of the expansion (int32 issue, the dominant kernel
    group) and of the selection (HBM), from the timed steps' stage events.

    Expansion: 25 int32 lane operations per uniform (one Philox4x32-10 call
    of about 100 operations gives four uniforms), one uniform per slot and
    per detection row of every child drawn, against 152 SMs x 128 lanes x
    2070 MHz.  Selection: the algorithmic bytes of normalisation and top-H,
    8 B per child key per pass over two passes plus 16 B per retained
    hypothesis written, against the measured HBM copy bandwidth."""
    peak_ops = 152 * 128 * 2070e6
    exp_ms = sum(s["stage_ms"].get("expand", 0.0) for s in steps)
    sel_ms = sum(s["stage_ms"].get("select", 0.0) for s in steps)
    total_ms = sum(s["ms"] for s in steps)
    ops = 25.0 * sum(s["draws"] for s in steps)
    n = len(steps)
    exp = None
    if exp_ms > 0:
        a = ops / (exp_ms / 1e3)
        exp = {"bound": "alu", "kernel": "child expansion and scoring (stage_kernel, draw_kernel, warp_kernel, "
                                         "dedup_kernel of one frame)",
               "achieved": a / 1e12, "peak": peak_ops / 1e12, "unit": "Tops/s (int32 lane ops)",
               "frac": a / peak_ops, "traffic": expansion_traffic(workload), "peak_source": INT_PEAK_NOTE,
               "algorithmic_per_step": ops / n, "kernel_ms_per_step": exp_ms / n,
               "kernel_share_of_step": exp_ms / total_ms}
    sel = None
    hbm = peaks.get("hbm_gbs")
    if sel_ms > 0:
        byts = sum(16.0 * s["children"] + 16.0 * s["retained"] for s in steps)
        a = byts / (sel_ms / 1e3) / 1e9
        p = hbm if hbm else 6800.0
        sel = {"bound": "hbm", "kernel": "normalisation and top-H selection (select_cluster_kernel, or the "
                                         "lse/radix/compact chain)",
               "achieved": a, "peak": p, "unit": "GB/s", "frac": a / p, "traffic": None,
               "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if hbm else "fallback 6800 GB/s",
               "algorithmic_per_step": byts / n, "kernel_ms_per_step": sel_ms / n,
               "kernel_share_of_step": sel_ms / total_ms}
    return exp, sel


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


def run_target(args, glmb, torch, dev):
    """The target comparison: the batched form with the learned gate
    against the plain single-scene form, on the same scenes and GPU.
    Scenes: --scenes held-out scenes of the batched workload's distribution
    (2-D, N ~ U{5..--target-nmax}, H ~ U{100..5000}, clutter ~ U(5, 40)),
    --steps frames each.  The gate is trained on --gate-train other scenes
    of the same distribution (features and usage labels from the ungated
    filter, the library's training kernels), its threshold keeping
    --gate-keep of the used training pairs.  Plain: each scene alone, frame
    after frame (glmb_step, gate off).  Batched + gate: every scene's frame
    at once (glmb_step_batch), gate pruning.  Both with device-resident
    detections and the estimates read every frame, timed on the host wall
    clock over a second pass (the first fills the graph caches).  Accuracy:
    OSPA (order 1, cut-off 50 m) of the MAP estimates against the scene's
    truth, per frame; the FP64 oracle runs the plain method on the scenes
    it finishes within --cpu-budget seconds in all, and each GPU form's
    mean OSPA over those scenes is compared with the oracle's."""
    from paper_2512_06230_gb300 import gate as G
    from scenes.metrics import ospa
    import oracle
    F = args.steps
    seed0 = 7000 if args.seed is None else args.seed
    specs = scenes.batch_scenes(args.scenes, seed0, frames=F, n_range=(5, args.target_nmax))
    train_specs = scenes.batch_scenes(args.gate_train, seed0 + 1, frames=F, n_range=(5, args.target_nmax))
    scs = [scenes.make_scene(p, s) for p, s in specs]
    cfgs = [batch_cfg(p, sc) for (p, _), sc in zip(specs, scs)]
    t0 = time.perf_counter()
    Xs, ys = [], []
    for p, s in train_specs:
        sc = scenes.make_scene(p, s)
        X, y = G.collect(batch_cfg(p, sc), [(glmb.births_array(fr.births, sc.dim_x), fr.Z) for fr in sc.frames],
                         skip=2)
        Xs.append(X)
        ys.append(y)
    X, y = np.concatenate(Xs), np.concatenate(ys)
    params, hist = G.train(X, y, steps=args.gate_steps, batch=32768, lr=2e-3, seed=1)
    thr = G.threshold(params, X, y, keep_used=args.gate_keep)
    t_train = time.perf_counter() - t0
    Z = [[torch.from_numpy(fr.Z).to(dev) if len(fr.Z) else torch.zeros((0, 2), device=dev) for fr in sc.frames]
         for sc in scs]
    B = [[glmb.births_array(fr.births, sc.dim_x) for fr in sc.frames] for sc in scs]
    torch.cuda.synchronize()

    def arm(batched):
        filters = [glmb.Filter(c) for c in cfgs]
        if batched:
            for f in filters:
                f.set_gate(params, thr, glmb.Filter.GATE_PRUNE)
        res = {}
        for pass_ in range(2):
            if pass_:
                for f in filters:
                    f.reset()
            est = [[None] * F for _ in filters]
            t_s = time.perf_counter()
            if batched:
                for k in range(F):
                    glmb.step_batch(filters, [(B[i][k], Z[i][k]) for i in range(len(filters))], device=True)
                    for i, f in enumerate(filters):
                        est[i][k] = f.estimates(cap=f.cfg["max_tracks"], pmf_cap=64)["mean"][:, :2].copy()
            else:
                for i, f in enumerate(filters):
                    for k in range(F):
                        f.step(B[i][k], Z[i][k], device=True)
                        est[i][k] = f.estimates(cap=f.cfg["max_tracks"], pmf_cap=64)["mean"][:, :2].copy()
            torch.cuda.synchronize()
            seconds = time.perf_counter() - t_s
            osp = [[ospa(est[i][k], scs[i].frames[k].truth[:, :2], c=50.0) for k in range(F)]
                   for i in range(len(filters))]
            res = dict(seconds=seconds, ospa=osp, pairs=sum(f.info()["n_pairs"] for f in filters) / len(filters))
        for f in filters:
            f.close()
        return res

    plain = arm(False)
    bat = arm(True)
    # the oracle (plain method, FP64) on the smallest scenes within the budget
    order = sorted(range(len(scs)), key=lambda i: (specs[i][0].n_objects, specs[i][0].h_max))
    threads = args.cpu_threads if args.cpu_threads > 0 else (os.cpu_count() or 1)
    o_osp, o_idx, t_o = {}, [], time.perf_counter()
    for i in order:
        if time.perf_counter() - t_o > args.cpu_budget:
            break
        o = oracle.Oracle(cfgs[i], n_threads=threads)
        vals = []
        for k, fr in enumerate(scs[i].frames):
            o.step(fr.births, fr.Z)
            vals.append(ospa(o.estimates()["mean"][:, :2], fr.truth[:, :2], c=50.0))
        o_osp[i] = vals
        o_idx.append(i)

    def mean_over(osp, idx):
        v = [x for i in idx for x in osp[i]]
        return float(np.mean(v)) if v else None

    all_idx = list(range(len(scs)))
    n_sf = len(scs) * F
    line = {"metric": "batched + learned-gate GLMB vs plain single-scene GLMB: scene-frames/s at equal OSPA (1 GB300)",
            "value": n_sf / bat["seconds"], "unit": "scene-frames/s", "higher_is_better": True,
            "dtype": "f32 (bf16 gate MLP)", "data": "synthetic", "n_gpus": 1, "steps": F,
            "config": {"workload": f"{len(scs)} scenes x {F} frames, 2-D CV, N~U{{5..{args.target_nmax}}}, "
                                   "H~U{100..5000}, clutter~U(5,40), device detections, estimates read every frame",
                       "gate": {"train_scenes": args.gate_train, "pairs": int(len(y)), "used_fraction": float(y.mean()),
                                "steps": args.gate_steps, "keep_used": args.gate_keep, "threshold": thr,
                                "train_s": round(t_train, 1)},
                       "ospa": "order 1, cut-off 50 m, MAP estimates vs truth"},
            "plain": {"scene_frames_per_s": n_sf / plain["seconds"], "ospa_mean": mean_over(plain["ospa"], all_idx),
                      "pairs_last_frame_per_scene": plain["pairs"]},
            "batched_gate": {"scene_frames_per_s": n_sf / bat["seconds"], "ospa_mean": mean_over(bat["ospa"], all_idx),
                             "pairs_last_frame_per_scene": bat["pairs"]},
            "speedup": plain["seconds"] / bat["seconds"],
            "oracle": {"scenes": len(o_idx), "n_objects": [specs[i][0].n_objects for i in o_idx],
                       "ospa_mean": mean_over(o_osp, o_idx), "threads": threads,
                       "plain_ospa_mean_same_scenes": mean_over(plain["ospa"], o_idx),
                       "batched_gate_ospa_mean_same_scenes": mean_over(bat["ospa"], o_idx)}}
    om = line["oracle"]["ospa_mean"]
    if om:
        line["oracle"]["plain_rel_diff"] = line["oracle"]["plain_ospa_mean_same_scenes"] / om - 1.0
        line["oracle"]["batched_gate_rel_diff"] = line["oracle"]["batched_gate_ospa_mean_same_scenes"] / om - 1.0
    print(json.dumps(line))


def _ints(text):
    return [int(v) for v in str(text).split(",") if v]


def run_convoy(args, glmb, torch):
    """Section 4.1's scalability grid on the convoy workload: N copies of one
    closed track (offset delta = 2 steps), five detections per object, no
    clutter, 548 steps of 0.1 s; N x H_max over --convoy-n x --convoy-h,
    for each mode in --convoy-modes (0 the joint multi-detection
    likelihood, 1 the product of C entries, 2 the paper's particle (CTRV)
    track model with --particles particles per track), --runs seeds each.  One update
    is glmb_step with the frame's detections in host memory plus the
    estimates read back (host wall clock, as the paper times an update);
    one untimed pass per filter first fills its graph cache.  Accuracy is
    the paper's: relative cardinality error and the Hungarian-matched mean
    distance, averaged over the steps of a run.  --convoy-oracle-steps
    steps of the FP64 oracle (single thread) are timed per (N, H_max) of
    modes 0 and 2 beside it."""
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
                    sc = scenes.convoy_scene(N, seed, steps=steps, h_max=H,
                                             particles=args.particles if mode == 2 else 0)
                    cfg = sc.filter_config() if mode == 2 else sc.filter_config(score_mode=mode)
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
                if mode in (0, 2) and args.convoy_oracle_steps > 0:
                    sc = scenes.convoy_scene(N, 0 if args.seed is None else args.seed, steps=args.convoy_oracle_steps,
                                             h_max=H, particles=args.particles if mode == 2 else 0)
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
                                             f"tau=1e-5, {steps} steps of 0.1 s; mode 2: {args.particles} "
                                             f"FP64 particles per track",
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


def peaks_file():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def oracle_error(oracle_state, glmb, sc, cfg, k):
    """Error of the library against the FP64 oracle for every output of one
    frame of the timed workload (the per-output error report): both
    import the oracle's own state before frame k and run frame k; the
    step-by-step comparison of the parity tests gives the largest error of
    each output and the decisions it excused."""
    import oracle
    from tests import parity
    oracle.build()
    fr = sc.frames[k]
    o, g, d = parity.run_frame(oracle, glmb, cfg, oracle_state, fr.births, fr.Z,
                               n_threads=os.cpu_count() or 1)
    rep = parity.compare(o, g, d, cfg, fr.Z)
    g.close()
    return {"frame": k, "max_err": {a: float(f"{b:.3g}") for a, b in sorted(rep.max_err.items())},
            "checks": rep.checks, "excused": rep.excused, "failures": len(rep.failures),
            "tolerances": {"logw_abs": parity.LOGW_TOL, "mean_cov_rel": parity.REL_TOL}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5,
                    help="untimed warm-up steps (after the set-up pass that captures the frame graphs)")
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--scene", default=DEFAULT_SCENE,
                    help="sweep_N<n> (3-D sweep cell, H_max from --h-max), mid, tiny, or one of the "
                         "workload modes batch, convoy, sweep, gate, mlp")
    ap.add_argument("--h-max", type=int, default=None, help="H_max of the scene (sweep cells: 20000)")
    ap.add_argument("--extra-cells", default=DEFAULT_EXTRA,
                    help="further workloads measured the same way in the same line: name[:H_max],...")
    ap.add_argument("--seed", type=int, default=None)
    ap.add_argument("--no-flush", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0,
                    help="seconds of oracle work after which its sample ends (the frame in progress finishes)")
    ap.add_argument("--cpu-threads", type=int, default=0,
                    help="host threads of the oracle leg (0: all cores)")
    ap.add_argument("--error-frame", type=int, default=4,
                    help="frame of the default workload re-run against the oracle for the error report "
                         "(-1: none)")
    ap.add_argument("--stages", action="store_true", help="time every stage of the frame, not only two")
    ap.add_argument("--batch-detections", default="device", choices=["device", "host"],
                    help="--scene batch: detections resident in device memory or copied from the host")
    ap.add_argument("--scenes", type=int, default=64,
                    help="--scene batch: independent scenes per frame")
    ap.add_argument("--convoy-n", default="1,2,5,10,20", help="--scene convoy: object counts")
    ap.add_argument("--convoy-h", default="5,10,25,50,100", help="--scene convoy: H_max values")
    ap.add_argument("--convoy-modes", default="0,1",
                    help="--scene convoy: 0 Gaussian tracks, joint likelihood; 1 Gaussian tracks, product of "
                         "C entries; 2 the particle (CTRV) track model, product of C entries")
    ap.add_argument("--particles", type=int, default=PARTICLES,
                    help="particles per track of the particle track model (--scene convoy mode 2)")
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
    ap.add_argument("--target-nmax", type=int, default=300, help="--scene target: largest object count")
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
        v, threads, sample, details, _ = run_oracle(args, sc, cfg, args.cpu_budget)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / v,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": workload_config(args, sc, cfg),
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                                 "sample": sample},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                "oracle_frames": details["frames"]}
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
    if args.scene == "target":
        return run_target(args, glmb, torch, dev)

    sc = scene_for_rank(args, rank)
    cfg = filter_cfg(sc)
    w0 = window_start(sc.params.name)
    if args.profile_frames:
        stream = torch.cuda.Stream(dev)
        torch.cuda.set_stream(stream)
        f = glmb.Filter(cfg, stream=stream.cuda_stream)
        F = len(sc.frames)
        Zdev = [torch.from_numpy(fr.Z).to(dev) for fr in sc.frames]
        B = [glmb.births_array(fr.births, sc.dim_x) for fr in sc.frames]
        for k in range(args.profile_frames):
            if k % F == 0:
                f.reset()
            f.step(B[k % F], Zdev[k % F], device=True)
        torch.cuda.synchronize()
        print(json.dumps({"profile_frames": args.profile_frames, "info": {
            k: v for k, v in f.info().items() if isinstance(v, (int, float))}}))
        return
    flush = None if args.no_flush else torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stages = list(glmb.Filter.STAGES) if args.stages else ["expand", "select"]
    cell = Cell(glmb, torch, dev, sc, cfg, w0, stages=stages, flush=flush)
    # set-up: one untimed pass over the scene captures the frame graphs of
    # every plan it needs; then the warm-up steps, then the timed steps (the
    # same window frames, replayed from a reset)
    cell.precapture()
    cell.run(args.warmup, 0)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk_lines, stop = [], threading.Event()
    th = threading.Thread(target=sample_clocks, args=(stop, clk_lines), daemon=True)
    th.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    steps = cell.run(args.steps, args.warmup)
    torch.cuda.synchronize()
    stop.set()
    th.join(timeout=10)
    total_ms = max_over_ranks(float(sum(s["ms"] for s in steps)), dev, world)
    if world > 1:
        torch.distributed.barrier()
    # end to end through the host-buffer path: the same frames, from the same state
    steps_h = cell.run(args.steps, args.warmup, host=True)
    total_h = max_over_ranks(float(sum(s["ms"] for s in steps_h)), dev, world)
    cell.close()
    # further cells of the sweep, the same protocol
    extra = {}
    for spec in [s for s in args.extra_cells.split(",") if s]:
        name, _, hm = spec.partition(":")
        sc2 = scene_for_rank(args, rank, name=name, h_max=int(hm) if hm else None)
        cfg2 = filter_cfg(sc2)
        c2 = Cell(glmb, torch, dev, sc2, cfg2, window_start(name), stages=stages, flush=flush)
        try:
            c2.precapture()
            c2.run(args.warmup, 0)
            st2 = c2.run(args.steps, args.warmup)
            sh2 = c2.run(args.steps, args.warmup, host=True)
        finally:
            c2.close()
        s2 = summarize(st2)
        ex2, sel2 = rooflines(st2, peaks_file(), name)
        extra[f"{name}:{cfg2['h_max']}"] = {
            "workload": workload_config(args, sc2, cfg2)["workload"], "value": s2["frames_per_s"],
            "ms_per_step": s2["ms_per_step"],
            "hypothesis_track_updates_per_s": s2["hypothesis_track_updates_per_s"],
            "e2e": summarize(sh2)["frames_per_s"], "mean_parents": s2["mean_parents"],
            "mean_M": s2["mean_M"], "stage_ms_per_step": s2["stage_ms_per_step"],
            "roofline_frac": {"expansion_alu": ex2["frac"] if ex2 else None,
                              "selection_hbm": sel2["frac"] if sel2 else None}}
    if rank != 0:
        return
    summ = summarize(steps)
    summ_h = summarize(steps_h)
    value = job_rate(args.steps, world, total_ms)
    clocks = summarize_clocks(clk_lines, local)
    peaks = peaks_file()
    exp, sel = rooflines(steps, peaks, sc.params.name)
    ef = args.error_frame if 0 <= args.error_frame < w0 else None
    cpu_v, cpu_threads, cpu_sample, cpu_det, ostate = run_oracle(args, sc, cfg, args.cpu_budget, state_frame=ef)
    err = oracle_error(ostate, glmb, sc, cfg, ef) if ostate is not None else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {**workload_config(args, sc, cfg),
                   "l2": "flushed between steps (256 MiB write, outside the timed events)" if flush is not None
                   else "not flushed",
                   "inputs": "detections resident in device memory; births (<4 KB) copied in the frame graph",
                   "graph_precapture": "one untimed pass over the scene before the warm-up"},
        "hypothesis_track_updates_per_s": summ["hypothesis_track_updates_per_s"] * world,
        "e2e": {"value": job_rate(args.steps, world, total_h), "unit": UNIT,
                "h2d_bytes_per_step": statistics.fmean(s["h2d"] for s in steps_h),
                "d2h_bytes_per_step": statistics.fmean(s["d2h"] for s in steps_h),
                "ms_per_step": total_h / args.steps},
        "gpu_launches": int(summ["launches"]),
        "work": {k: summ[k] for k in ("mean_parents", "mean_retained", "mean_M", "children_per_step",
                                      "captures_in_timed_steps", "redone_frames")},
        "stage_ms_per_step": summ["stage_ms_per_step"],
        "roofline": exp,
        "roofline_selection": sel,
        "cpu_baseline": {"value": cpu_v, "unit": UNIT, "cores": cpu_threads, "kind": "oracle",
                         "sample": cpu_sample},
        "oracle_error": err,
        "cells": extra,
        "clocks": clocks,
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
