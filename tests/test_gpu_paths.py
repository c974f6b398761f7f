"""The expansion's launch paths compute the same arithmetic: shared-memory or
global-memory staging of the per-parent tables, and one thread or one warp
per child, give bit-identical children (keys, statuses, surviving track
counts) and the same retained set on every frame.  Section 3's sampling and
weighting do not depend on how the work is mapped to the GPU."""
from __future__ import annotations

import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def glmb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_06230_gb300 as g
    g.build()
    return g


def _run_lockstep(glmb, preset, seed, n_frames, opts_list, **cfg_over):
    sc = scenes.make_scene(scenes.preset(preset), seed)
    cfg = sc.filter_config(**cfg_over)
    fs = []
    for o in opts_list:
        f = glmb.Filter(cfg)
        f.set_launch_options(o)
        fs.append(f)
    paths_seen = set()
    for k, fr in enumerate(sc.frames[:n_frames]):
        ch = []
        for f in fs:
            f.predict(fr.births)
            f.update(fr.Z)
            ch.append(f.children())
            paths_seen.add(f.info()["expand_threads"])
        for o, c in zip(opts_list[1:], ch[1:]):
            for key in ("logw", "status", "n_alive"):
                a, b = ch[0][key], c[key]
                assert a.shape == b.shape, (k, o, key)
                same = (a == b) | (np.isneginf(a) & np.isneginf(b)) if a.dtype.kind == "f" else a == b
                assert same.all(), f"frame {k}, options {o}: {key} differs at {np.flatnonzero(~same)[:5]}"
        ret = []
        for f in fs:
            f.prune()
            ret.append(f.retained()[0])
        for o, r in zip(opts_list[1:], ret[1:]):
            assert np.array_equal(ret[0], r), (k, o)
    # the whole state (hypotheses, components, theta) after the last frame
    s0 = fs[0].export_state()
    for o, f in zip(opts_list[1:], fs[1:]):
        assert f.export_state() == s0, o
    return paths_seen


def test_paths_agree_tiny(glmb):
    F = glmb.Filter
    _run_lockstep(glmb, "tiny", 11, 20, [0, F.OPT_STAGE_GLOBAL, F.OPT_DRAW_THREAD,
                                         F.OPT_DRAW_THREAD | F.OPT_STAGE_GLOBAL, F.OPT_DRAW_WARP,
                                         F.OPT_DRAW_WARP | F.OPT_WARP_GROUPS, F.OPT_WARP_GROUPS])


def test_paths_agree_mid(glmb):
    F = glmb.Filter
    seen = _run_lockstep(glmb, "mid", 12, 16, [0, F.OPT_DRAW_WARP, F.OPT_DRAW_THREAD | F.OPT_STAGE_GLOBAL,
                                               F.OPT_DRAW_WARP | F.OPT_WARP_GROUPS],
                         max_meas=400, max_births=16, max_tracks=300)
    assert len(seen) >= 2   # both draw mappings ran


def test_paths_agree_3d(glmb):
    F = glmb.Filter
    _run_lockstep(glmb, "sweep_N50", 13, 6, [0, F.OPT_DRAW_WARP | F.OPT_STAGE_GLOBAL, F.OPT_DRAW_THREAD,
                                             F.OPT_STAGE_SHARED, F.OPT_STAGE_SHARED | F.OPT_DRAW_WARP,
                                             F.OPT_STAGE_GLOBAL | F.OPT_STAGE_SCRATCH_ROWS,
                                             F.OPT_STAGE_GLOBAL | F.OPT_STAGE_SCRATCH_NONE])


def _burst_frames(seed, k_burst, n_extra):
    """The tiny scene with a burst of extra detections at frame k_burst,
    all near existing detections: a parent's gated pairs jump past the
    estimate from earlier frames, so the frame's expansion is redone with
    the exact maxima."""
    sc = scenes.make_scene(scenes.preset("tiny"), seed)
    rng = np.random.default_rng(seed)
    frames = []
    for k, fr in enumerate(sc.frames[:k_burst + 3]):
        Z = fr.Z
        if k == k_burst and len(fr.truth):
            # around one object's true position: every extra detection gates
            # with its track, so the pair count of every parent holding the
            # track jumps by n_extra
            extra = fr.truth[0, :2] + rng.normal(scale=2.0, size=(n_extra, 2))
            Z = np.concatenate([Z, extra.astype(np.float32)])
        frames.append((fr.births, Z))
    return sc, frames


def test_redone_frame_in_the_graph_path_matches_separate_calls(glmb):
    """A frame whose expansion plan is exceeded is redone.  Through
    glmb_step (frame graph, estimates inside the graph) it must give the same
    hypotheses and estimates as predict / update / prune, and every later
    frame must run."""
    sc, frames = _burst_frames(1011, 8, 400)
    cfg = sc.filter_config()
    a, b = glmb.Filter(cfg), glmb.Filter(cfg)
    redo = 0
    for k, (births, Z) in enumerate(frames):
        a.step(births, Z)
        b.predict(births)
        b.update(Z)
        b.prune()
        ha, hb = a.hypotheses(), b.hypotheses()
        np.testing.assert_array_equal(ha["uid"], hb["uid"])
        np.testing.assert_array_equal(ha["logw"], hb["logw"])
        ea, eb = a.estimates(), b.estimates()
        np.testing.assert_array_equal(ea["labels"], eb["labels"])
        np.testing.assert_array_equal(ea["pmf"], eb["pmf"])
        redo = a.info()["n_redo"]
    assert redo >= 1, "the burst did not exceed the plan"


def test_torch_allocator_hook_gives_the_same_results(glmb):
    """glmb_config's allocation hook: every device buffer from PyTorch's
    caching allocator (the images grown mid-run included), identical results,
    and the memory back in torch's cache after destroy."""
    import torch
    sc = scenes.make_scene(scenes.preset("tiny"), 1012)
    cfg = sc.filter_config()
    base = torch.cuda.memory_allocated()
    a = glmb.Filter(cfg)
    b = glmb.Filter(cfg, allocator="torch")
    held = torch.cuda.memory_allocated() - base
    assert held > 0
    for fr in sc.frames[:15]:
        a.step(fr.births, fr.Z)
        b.step(fr.births, fr.Z)
        ha, hb = a.hypotheses(), b.hypotheses()
        np.testing.assert_array_equal(ha["uid"], hb["uid"])
        np.testing.assert_array_equal(ha["logw"], hb["logw"])
    assert torch.cuda.memory_allocated() - base >= held
    a.close()
    b.close()
    assert torch.cuda.memory_allocated() == base


def test_step_graphs_with_device_detections_match_separate_calls(glmb):
    """The configuration the benchmark times: the mid scene stepped through
    replayed frame graphs with detections resident in device memory.  Every
    frame must equal predict / update / prune with host detections (the path
    the oracle parity tests check) bit for bit: retained hypotheses, their
    weights, and the estimates."""
    import torch
    sc = scenes.make_scene(scenes.preset("mid"), 1015)
    import bench
    cfg = bench.filter_cfg(sc)
    a, b = glmb.Filter(cfg), glmb.Filter(cfg)
    dev = torch.device("cuda", torch.cuda.current_device())
    for k, fr in enumerate(sc.frames[:40]):
        Zd = torch.from_numpy(fr.Z).to(dev) if len(fr.Z) else torch.zeros((0, sc.dim_z), device=dev)
        a.step(fr.births, Zd, device=True)
        b.predict(fr.births)
        b.update(fr.Z)
        b.prune()
        ha, hb = a.hypotheses(), b.hypotheses()
        np.testing.assert_array_equal(ha["uid"], hb["uid"], err_msg=f"frame {k}")
        np.testing.assert_array_equal(ha["logw"], hb["logw"], err_msg=f"frame {k}")
        ea = a.estimates(cap=cfg["max_tracks"], pmf_cap=64)
        eb = b.estimates(cap=cfg["max_tracks"], pmf_cap=64)
        assert ea["n"] == eb["n"], k
        for key in ("labels", "r", "mean", "cov", "pmf"):
            np.testing.assert_array_equal(ea[key], eb[key], err_msg=f"frame {k}: {key}")
    info = a.info()
    assert info["n_graph_launches"] >= 30 and info["n_graph_captures"] < info["n_graph_launches"]
