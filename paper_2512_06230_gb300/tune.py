"""Autotuner of the launch shapes (glmb_set_tuning) for a workload.

The shapes do not change results; they move time between the thread-per-
child and warp-per-child draws and change CTA sizes.  autotune() runs the
given frames once per candidate on a fresh filter (one untimed pass to
capture graphs, then a timed pass from a reset) and returns the fastest
candidate with every timing."""
from __future__ import annotations

import itertools
import time

DEFAULT_SPACE = {
    "thread_warps_per_sm": (1, 2, 4, 8),
    "draw_threads": (0, 128, 256),
    "warp_cta_warps": (8, 16),
    "stage_threads": (0, 64, 128, 256),
}


def candidates(space=None, limit=None):
    space = dict(DEFAULT_SPACE if space is None else space)
    keys = list(space)
    out = [dict(zip(keys, v)) for v in itertools.product(*(space[k] for k in keys))]
    return out if limit is None else out[:limit]


def time_frames(filt, frames, device=False):
    """Wall time of one pass over frames, estimates read each frame."""
    t0 = time.perf_counter()
    for births, Z in frames:
        filt.step(births, Z, device=device)
        filt.estimates(cap=int(filt.cfg.get("max_tracks", 256)), pmf_cap=16)
    return time.perf_counter() - t0


def autotune(cfg, frames, space=None, device=False, make_filter=None):
    """Fastest launch shapes for (cfg, frames); frames is a list of
    (births, Z).  Returns (best tuning, [(tuning, seconds), ...])."""
    import paper_2512_06230_gb300 as glmb
    make_filter = make_filter or (lambda c: glmb.Filter(c))
    results = []
    for cand in candidates(space):
        f = make_filter(cfg)
        try:
            f.set_tuning(**cand)
            time_frames(f, frames, device)      # graphs for this shape
            f.reset()
            results.append((cand, time_frames(f, frames, device)))
        finally:
            f.close()
    best = min(results, key=lambda r: r[1])[0]
    return best, results
