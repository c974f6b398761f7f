"""CUDA library against the FP64 oracle, step by step, through the C ABI.

Every test imports the same state into both implementations (a state the
oracle produced on a seeded synthetic scene), runs one frame and compares
each step of the update (tests/parity.py lists the tolerances)."""
from __future__ import annotations

import numpy as np
import pytest

import scenes
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def glmb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_06230_gb300 as g
    g.build()
    g.load()
    return g


def _frame(oracle_mod, glmb, cfg, scene, k):
    state = parity.oracle_state(oracle_mod, cfg, scene, k)
    fr = scene.frames[k]
    o, g, d = parity.run_frame(oracle_mod, glmb, cfg, state, fr.births, fr.Z)
    rep = parity.compare(o, g, d, cfg, fr.Z)
    print(f"\nchecks {rep.checks} excused {rep.excused} max_err "
          + " ".join(f"{k}={v:.2e}" for k, v in sorted(rep.max_err.items())))
    assert rep.ok(), rep.failures[:10]
    return rep


@pytest.mark.parametrize("k", [0, 1, 6, 20, 35])
def test_tiny_scene_frame(oracle_mod, glmb, k):
    sc = scenes.make_scene(scenes.preset("tiny"), 1001)
    _frame(oracle_mod, glmb, sc.filter_config(), sc, k)


@pytest.mark.parametrize("k", [12, 40])
def test_mid_scene_frame(oracle_mod, glmb, k):
    """The 2-D scene with 100 objects and H_max = 1000 at full size."""
    sc = scenes.make_scene(scenes.preset("mid"), 2001)
    rep = _frame(oracle_mod, glmb, sc.filter_config(), sc, k)
    assert rep.checks["children"] >= 1000
    assert rep.excused["children"] <= parity.excused_children_bound(rep, sc.filter_config(), len(sc.frames[k].Z))
    assert rep.excused["boundary"] <= 2 + 0.001 * rep.checks["retained"]


def test_3d_scene_frame(oracle_mod, glmb):
    sc = scenes.make_scene(scenes.preset("sweep_N50", frames=12), 3050)
    _frame(oracle_mod, glmb, sc.filter_config(h_max=200), sc, 8)


def test_no_detections(oracle_mod, glmb):
    sc = scenes.make_scene(scenes.preset("tiny"), 1003)
    cfg = sc.filter_config()
    state = parity.oracle_state(oracle_mod, cfg, sc, 10)
    fr = sc.frames[10]
    Z = np.zeros((0, 2), np.float32)
    o, g, d = parity.run_frame(oracle_mod, glmb, cfg, state, fr.births, Z)
    rep = parity.compare(o, g, d, cfg, Z)
    assert rep.ok(), rep.failures[:10]


def test_no_births_and_no_clutter(oracle_mod, glmb):
    """kappa = 0: every detection must go to a track.  The frame keeps only
    the detections that gate some track of the first hypothesis (found with
    the oracle), so children without a zero-weight row exist."""
    sc = scenes.make_scene(scenes.preset("tiny"), 1004)
    cfg = sc.filter_config(clutter_rate=0.0)
    state = parity.oracle_state(oracle_mod, sc.filter_config(), sc, 15)
    fr = sc.frames[15]
    o = oracle_mod.Oracle(cfg)
    o.import_state(*state)
    o.predict([])
    o.update(fr.Z)
    keep = [i for i in range(len(fr.Z))
            if any(o.pair(0, t, i)["gated"] for t in range(o.parent_slots(0)))]
    Z = fr.Z[keep]
    assert 0 < len(Z) < len(fr.Z)
    o2, g, d = parity.run_frame(oracle_mod, glmb, cfg, state, [], Z)
    rep = parity.compare(o2, g, d, cfg, Z)
    assert rep.ok(), rep.failures[:10]


def test_zero_weight_frame_is_an_error_and_keeps_state(oracle_mod, glmb):
    """kappa = 0 and a detection far from every track: no child has a
    finite weight.  Both implementations report it; the library keeps the
    previous state and accepts the frame again."""
    sc = scenes.make_scene(scenes.preset("tiny"), 1004)
    cfg = sc.filter_config(clutter_rate=0.0)
    state = parity.oracle_state(oracle_mod, sc.filter_config(), sc, 10)
    Z = np.array([[-5.0e4, -5.0e4]], np.float32)
    o = oracle_mod.Oracle(cfg)
    o.import_state(*state)
    o.predict([])
    o.update(Z)
    with pytest.raises(oracle_mod.OracleError):
        o.prune()
    g = glmb.Filter(cfg)
    g.import_state(glmb.pack_state(*state, g.dx))
    before = g.export_state()
    g.predict([])
    g.update(Z)
    with pytest.raises(glmb.GlmbError) as ei:
        g.prune()
    assert ei.value.status == 5
    assert g.export_state() == before
    g.predict([])
    g.update(sc.frames[10].Z[:0])
    g.prune()


def test_invalid_inputs_are_rejected(glmb):
    sc = scenes.make_scene(scenes.preset("tiny"), 1006)
    g = glmb.Filter(sc.filter_config())
    with pytest.raises(glmb.GlmbError) as ei:
        g.update(sc.frames[0].Z)
    assert ei.value.status == 6
    g.predict(sc.frames[0].births)
    Z = sc.frames[0].Z.copy()
    Z[0, 0] = np.nan
    with pytest.raises(glmb.GlmbError) as ei:
        g.update(Z)
    assert ei.value.status == 1
    import torch
    g.predict(sc.frames[0].births)
    g.update(torch.from_numpy(Z).cuda(), device=True)   # checked on the device
    with pytest.raises(glmb.GlmbError) as ei:
        g.prune()
    assert ei.value.status == 1
    g.predict(sc.frames[0].births)
    g.update(torch.from_numpy(sc.frames[0].Z).cuda(), device=True)
    g.prune()
    assert g.info()["n_hyp"] >= 1
    with pytest.raises(glmb.GlmbError) as ei:
        g.predict([(1.5, np.zeros(4), np.eye(4))])
    assert ei.value.status == 1


def test_certain_detection(oracle_mod, glmb):
    sc = scenes.make_scene(scenes.preset("tiny"), 1005)
    cfg = sc.filter_config(p_d=1.0)
    state = parity.oracle_state(oracle_mod, cfg, sc, 8)
    fr = sc.frames[8]
    o, g, d = parity.run_frame(oracle_mod, glmb, cfg, state, fr.births, fr.Z)
    rep = parity.compare(o, g, d, cfg, fr.Z)
    assert rep.ok(), rep.failures[:10]


def test_multi_frame_run_tracks_the_oracle(oracle_mod, glmb):
    """Both filters from the initial GLMB over a whole scene.  Random draws
    are keyed by hypothesis uid, so the two stay identical as long as their
    retained sets agree; frames are counted until an excused decision makes
    them part."""
    sc = scenes.make_scene(scenes.preset("tiny"), 1001)
    cfg = sc.filter_config()
    o = oracle_mod.Oracle(cfg, n_threads=8)
    g = glmb.Filter(cfg)
    same = 0
    card = 0
    for f, fr in enumerate(sc.frames):
        o.step(fr.births, fr.Z)
        g.step(fr.births, fr.Z)
        ou = set(o.export_state()[2].tolist())
        gu = set(g.hypotheses()["uid"].tolist())
        if ou == gu:
            same += 1
        card += o.estimates()["n"] == g.estimates()["n"]
    print(f"\nframes with identical hypothesis sets: {same}/{len(sc.frames)}, "
          f"equal MAP cardinality: {card}/{len(sc.frames)}")
    assert same >= len(sc.frames) // 2
    assert card >= 0.9 * len(sc.frames)


@pytest.mark.parametrize("k", [1, 6, 20])
def test_factorised_mode_tiny_frame(oracle_mod, glmb, k):
    """Section 4: the factorised score (product of C entries of Eq. 2)."""
    sc = scenes.make_scene(scenes.preset("tiny"), 1004)
    _frame(oracle_mod, glmb, sc.filter_config(score_mode=1), sc, k)


def test_factorised_mode_mid_frame(oracle_mod, glmb):
    sc = scenes.make_scene(scenes.preset("mid"), 2001)
    rep = _frame(oracle_mod, glmb, sc.filter_config(score_mode=1), sc, 12)
    assert rep.checks["children"] >= 1000


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("k", [0, 3, 15])
def test_convoy_frame(oracle_mod, glmb, mode, k):
    """Section 4.1's workload shape: five detections per object, no clutter."""
    sc = scenes.convoy_scene(5, 77, steps=16, h_max=50)
    _frame(oracle_mod, glmb, sc.filter_config(score_mode=mode), sc, k)


@pytest.mark.parametrize("N,k", [(200, 4), (1000, 3)])
def test_sweep_full_size_frame(oracle_mod, glmb, N, k):
    """The 3-D sweep at full size, H_max = 20000: N = 200 (the cap binds as
    hypotheses grow) and N = 1000 (the largest configuration, about 2600
    detections and 1000 tracks per hypothesis)."""
    sc = scenes.make_scene(scenes.preset(f"sweep_N{N}", h_max=20000, frames=k + 1), 3000 + N)
    nb = max(len(f.births) for f in sc.frames)
    cfg = sc.filter_config(max_meas=max(len(f.Z) for f in sc.frames) + 16, max_births=max(8, nb),
                           max_tracks=2 * N + nb + 64)
    rep = _frame(oracle_mod, glmb, cfg, sc, k)
    assert rep.checks["slots"] > 10000
    # what the excuses admitted: few decisions near a boundary of a row or of
    # the death probability, and few retained hypotheses near the cut
    assert rep.excused["children"] <= parity.excused_children_bound(rep, cfg, len(sc.frames[k].Z))
    assert rep.excused["boundary"] <= 2 + 0.001 * rep.checks["retained"]


@pytest.mark.parametrize("h_up,h_max,k", [(1, 50, 12), (300, 200, 8), (1000, 400, 10)])
def test_draw_counts_and_caps(oracle_mod, glmb, h_up, h_max, k):
    """H_up = 1 (one child per parent: every frame keeps the reference-most
    draw or nothing), and H_up of 300 and 1000, whose draws span several
    ragged 256-child slices of a parent in the thread-per-child kernel."""
    sc = scenes.make_scene(scenes.preset("tiny"), 1021)
    rep = _frame(oracle_mod, glmb, sc.filter_config(h_up=h_up, h_max=h_max), sc, k)
    assert rep.checks["children"] % h_up == 0


@pytest.mark.parametrize("h_max,tau,k,kept", [(1, 1e-5, 9, "one"), (100000, 1e-300, 4, "all"),
                                               (5000, 1e-300, 5, "cap")])
def test_truncation_extremes(oracle_mod, glmb, h_max, tau, k, kept):
    """H_max = 1 keeps only the heaviest child (ties to the lower child
    index).  With tau ~ 0: a frame of 573 parents whose ~3200 unique
    children all fit under H_max = 100 000 keeps every one (no radix round
    decides anything), and a frame of 3231 parents with ~17 000 unique
    children fills H_max = 5000 exactly."""
    sc = scenes.make_scene(scenes.preset("tiny"), 1022)
    rep = _frame(oracle_mod, glmb, sc.filter_config(h_max=h_max, tau=tau), sc, k)
    if kept == "one":
        assert rep.checks["retained"] == 1
    elif kept == "all":
        # nothing is cut by the cap (the unique count leaves out children
        # whose uniqueness decision is excused as a near tie)
        assert 3000 < rep.checks["unique_children"] <= rep.checks["retained"] < h_max
    else:
        assert rep.checks["retained"] == h_max


def test_detections_at_capacity(oracle_mod, glmb):
    """A frame whose detection count equals max_meas exactly (the detection
    buffers and per-hypothesis association rows full to the last entry)."""
    sc = scenes.make_scene(scenes.preset("tiny"), 1023)
    k = 8
    cfg = sc.filter_config(max_meas=len(sc.frames[k].Z))
    assert cfg["max_meas"] > 0
    _frame(oracle_mod, glmb, cfg, sc, k)


@pytest.mark.parametrize("shape", ["diagonal", "correlated"])
def test_ill_conditioned_innovation_takes_the_fp64_factorisation(oracle_mod, glmb, shape):
    """Precision management: the Cholesky factor of an ill-conditioned
    innovation covariance is computed in FP64 on the GPU (counted in
    glmb_info.n_fp64_chol); the frame then matches the FP64 oracle at the
    usual tolerances."""
    cfg, state, Z, _ = parity.ill_conditioned_case(shape)
    o, g, d = parity.run_frame(oracle_mod, glmb, cfg, state, [], Z)
    rep = parity.compare(o, g, d, cfg, Z)
    n64 = g.info()["n_fp64_chol"]
    print(f"\n{shape}: n_fp64_chol {n64} checks {rep.checks} max_err "
          + " ".join(f"{k}={v:.2e}" for k, v in sorted(rep.max_err.items())))
    assert rep.ok(), rep.failures[:10]
    assert n64 >= 4
    assert rep.checks["unique_children"] >= 10 and rep.checks["retained"] >= 10


def _ospa_run(filt_step, filt_est, scene, dim):
    from scenes.metrics import ospa
    out = []
    for fr in scene.frames:
        filt_step(fr)
        out.append(ospa(filt_est()[:, :dim], fr.truth[:, :dim], c=50.0, p=1.0))
    return np.array(out)


@pytest.mark.parametrize("preset,seed", [("tiny", 1001), ("tiny", 1002), ("mid", 2001)])
def test_multi_frame_ospa_within_one_percent_of_the_oracle(oracle_mod, glmb, preset, seed):
    """Multi-frame runs are compared by OSPA (order 1, cut-off 50 m, MAP
    estimates against the scene's truth): the GPU filter and the oracle,
    each from the initial GLMB over the whole scene, give mean OSPA within
    1 % of each other."""
    sc = scenes.make_scene(scenes.preset(preset), seed)
    cfg = sc.filter_config()
    o = oracle_mod.Oracle(cfg, n_threads=8)
    g = glmb.Filter(cfg)
    d = sc.dim_z
    oo = _ospa_run(lambda fr: o.step(fr.births, fr.Z), lambda: o.estimates()["mean"], sc, d)
    og = _ospa_run(lambda fr: g.step(fr.births, fr.Z), lambda: g.estimates()["mean"], sc, d)
    g.close()
    print(f"\n{preset}/{seed}: mean OSPA oracle {oo.mean():.4f} m, GPU {og.mean():.4f} m, "
          f"frames equal {np.sum(np.abs(oo - og) < 1e-6)}/{len(oo)}")
    assert abs(og.mean() - oo.mean()) <= 0.01 * oo.mean()
