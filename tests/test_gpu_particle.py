"""The particle track model (model 1: weighted particles with constant
turn rate and velocity, Section 3) on the GPU against the FP64 oracle,
through the C ABI: one frame from a shared state, step by step
(tests/parity.py lists the tolerances; particles are compared state by
state), and the state round trip."""
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


def _cfg(p, seed, **kw):
    cfg = scenes.ctrv_filter_config(p, seed, max_tracks=64, max_meas=512, max_births=32,
                                    max_components=20000, **kw)
    return cfg


def _frame(oracle_mod, glmb, cfg, scene, k):
    state = parity.oracle_state(oracle_mod, cfg, scene, k)
    fr = scene.frames[k]
    o, g, d = parity.run_frame(oracle_mod, glmb, cfg, state, fr.births, fr.Z)
    rep = parity.compare(o, g, d, cfg, fr.Z)
    print(f"\nchecks {rep.checks} excused {rep.excused} max_err "
          + " ".join(f"{k}={v:.2e}" for k, v in sorted(rep.max_err.items())))
    assert rep.ok(), rep.failures[:10]
    return rep


@pytest.mark.parametrize("k", [0, 3, 9, 15])
def test_ctrv_scene_frame(oracle_mod, glmb, k):
    p = scenes.CtrvParams(n_objects=8, frames=20, h_max=200, n_particles=128)
    sc = scenes.ctrv_scene(p, 501)
    rep = _frame(oracle_mod, glmb, _cfg(p, 501), sc, k)
    if k:
        assert rep.checks["matched_hypotheses"] >= 1
        assert "particle_x_rel" in rep.max_err or rep.excused.get("resample_near_tie")


@pytest.mark.parametrize("np_,ess", [(1, 0.5), (32, 1.0), (300, 0.0), (1024, 0.5), (4096, 0.5)])
def test_particle_counts_and_resampling_rules(oracle_mod, glmb, np_, ess):
    """A single particle (a point mass), particle counts that are not a
    multiple of the block, one particle per thread and several, the largest
    count (4096), resampling always (ess_frac 1) and never (0)."""
    p = scenes.CtrvParams(n_objects=5, frames=12, h_max=100, n_particles=np_, ess_frac=ess)
    sc = scenes.ctrv_scene(p, 502)
    _frame(oracle_mod, glmb, _cfg(p, 502), sc, 8)


def test_ctrv_frame_without_detections(oracle_mod, glmb):
    p = scenes.CtrvParams(n_objects=6, frames=12, h_max=100, n_particles=64)
    sc = scenes.ctrv_scene(p, 503)
    cfg = _cfg(p, 503)
    state = parity.oracle_state(oracle_mod, cfg, sc, 6)
    Z = np.zeros((0, 2), np.float32)
    o, g, d = parity.run_frame(oracle_mod, glmb, cfg, state, sc.frames[6].births, Z)
    rep = parity.compare(o, g, d, cfg, Z)
    assert rep.ok(), rep.failures[:10]


def test_particle_state_round_trip(oracle_mod, glmb):
    p = scenes.CtrvParams(n_objects=6, frames=10, h_max=100, n_particles=64)
    sc = scenes.ctrv_scene(p, 504)
    cfg = _cfg(p, 504)
    frame, logw, uid, tracks = parity.oracle_state(oracle_mod, cfg, sc, 8)
    g = glmb.Filter(cfg)
    g.import_state(glmb.pack_state(frame, logw, uid, tracks, 5, 64))
    fr2, lw2, uid2, tr2 = glmb.unpack_state(g.export_state(), 64)
    assert fr2 == frame and np.array_equal(uid2, uid)
    for a, b in zip(tracks, tr2):
        for r1, r2 in zip(a, b):
            assert r1[:2] == r2[:2]
            np.testing.assert_array_equal(r1[4], r2[4])
            np.testing.assert_array_equal(r1[5], r2[5])
            # moments: the particles' weighted moments, mean rounded to FP32
            np.testing.assert_allclose(r2[2], r1[2], rtol=1e-6)


def test_particle_model_rejects_bad_configurations(glmb):
    p = scenes.CtrvParams(n_objects=2, frames=2)
    for bad in (dict(dim_x=4), dict(score_mode=0), dict(n_particles=0), dict(n_particles=5000),
                dict(ess_frac=2.0)):
        with pytest.raises(glmb.GlmbError):
            glmb.Filter(_cfg(p, 1, **bad))
    g = glmb.Filter(_cfg(p, 1))
    with pytest.raises(glmb.GlmbError):
        g.set_gate(np.zeros(8779, np.float32), 0.0, glmb.Filter.GATE_PRUNE)
    # a birth covariance that is not positive definite is refused
    bad_birth = [(0.5, np.array([300.0, 300.0, 10.0, 0.0, 0.0]), np.diag([1.0, 1.0, 1.0, 0.0, 1.0]))]
    with pytest.raises(glmb.GlmbError):
        g.predict(bad_birth)


def test_ctrv_bench_cell_frame(oracle_mod, glmb):
    """The benchmark's particle cell (50 CTRV vehicles, 256 particles per
    track, H_max = 1000, seed 5050) at a steady-window frame, every step
    compared with the oracle."""
    p = scenes.CtrvParams(name="ctrv_N50", n_objects=50, frames=40, h_max=1000, clutter_rate=10.0,
                          n_particles=256)
    sc = scenes.ctrv_scene(p, 5050)
    cfg = scenes.ctrv_filter_config(p, 5050, max_tracks=171, max_meas=256, max_births=64)
    rep = _frame(oracle_mod, glmb, cfg, sc, 21)
    assert rep.checks["retained"] >= 500 and rep.checks["matched_hypotheses"] >= 400
    assert rep.excused["children"] <= parity.excused_children_bound(rep, cfg, len(sc.frames[21].Z))
    assert rep.excused["boundary"] <= 2 + 0.001 * rep.checks["retained"]


def test_ctrv_multi_frame_run_tracks_the_oracle(oracle_mod, glmb):
    """Both filters from the initial GLMB over a whole CTRV scene: identical
    hypothesis sets in most frames (random draws are keyed by hypothesis uid
    and track label, so the two stay identical while their retained sets
    agree), and mean OSPA (order 1, cut-off 50 m, MAP estimates against the
    truth) within 1 % of the oracle's."""
    from scenes.metrics import ospa
    p = scenes.CtrvParams(n_objects=8, frames=25, h_max=100, n_particles=128)
    sc = scenes.ctrv_scene(p, 505)
    cfg = _cfg(p, 505)
    o = oracle_mod.Oracle(cfg, n_threads=8)
    g = glmb.Filter(cfg)
    same, oo, og = 0, [], []
    for fr in sc.frames:
        o.step(fr.births, fr.Z)
        g.step(fr.births, fr.Z)
        same += set(o.export_state()[2].tolist()) == set(g.hypotheses()["uid"].tolist())
        oo.append(ospa(o.estimates()["mean"][:, :2], fr.truth[:, :2], c=50.0, p=1.0))
        og.append(ospa(g.estimates()["mean"][:, :2], fr.truth[:, :2], c=50.0, p=1.0))
    g.close()
    oo, og = np.array(oo), np.array(og)
    print(f"\nframes with identical hypothesis sets {same}/{len(sc.frames)}; mean OSPA oracle "
          f"{oo.mean():.4f} m, GPU {og.mean():.4f} m")
    assert same >= len(sc.frames) // 2
    assert abs(og.mean() - oo.mean()) <= 0.01 * oo.mean()
