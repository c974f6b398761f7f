"""Synthetic workloads and the accuracy metrics (CPU)."""
from __future__ import annotations

import numpy as np
import pytest

import scenes
from scenes.metrics import RunAccuracy, matched_distance


def test_convoy_shape_follows_section_4_1():
    N, D, delta = 4, 5, 2
    sc = scenes.convoy_scene(N, 3, steps=40, detections=D, delta=delta)
    track = scenes.convoy_path(548, 3 ^ 0xC0)
    for k, fr in enumerate(sc.frames):
        assert fr.Z.shape == (N * D, 2)
        # copy n is the base track offset by n * delta steps
        for n in range(N):
            np.testing.assert_allclose(fr.truth[n], track[(k + n * delta) % 548])
        # detections in sorted order (object by object), spread sigma
        for n in range(N):
            err = fr.Z[n * D:(n + 1) * D] - fr.truth[n, :2]
            assert np.all(np.abs(err) < 6 * sc.params.sigma)
    assert len([b for b in sc.frames[0].births if b[0] == sc.params.r_birth]) == N
    cfg = sc.filter_config()
    assert sc.params.clutter_rate == 0.0 and cfg["lambda_d"] == D - 1
    assert cfg["h_up"] == 100 and cfg["tau"] == 1e-5


def test_convoy_path_is_smooth_closed_and_inside_the_area():
    tr = scenes.convoy_path(548, 9)
    assert tr[:, :2].min() >= 0 and tr[:, :2].max() <= 80
    # constant speed, and the wrap from the last sample to the first is an
    # ordinary step: copies offset modulo the track length never jump
    step = np.linalg.norm(np.roll(tr[:, :2], -1, axis=0) - tr[:, :2], axis=1)
    assert step.max() / step.min() < 1.01
    assert 5.0 < step.mean() / 0.1 < 15.0
    acc = np.linalg.norm(np.roll(tr[:, 2:], -1, axis=0) - tr[:, 2:], axis=1) / 0.1
    assert acc.max() < 15.0


def test_detection_noise_has_the_stated_spread():
    sc = scenes.convoy_scene(5, 4, steps=200)
    err = np.concatenate([fr.Z - np.repeat(fr.truth[:, :2], 5, axis=0) for fr in sc.frames])
    assert abs(err.std() - 0.25) < 0.01
    assert np.all(np.abs(err.mean(0)) < 0.01)


def test_matched_distance_brute_force():
    rng = np.random.default_rng(0)
    from itertools import permutations
    for _ in range(5):
        a, b = rng.normal(size=(3, 2)), rng.normal(size=(4, 2))
        best = min(np.mean([np.linalg.norm(a[i] - b[p[i]]) for i in range(3)])
                   for p in permutations(range(4), 3))
        assert abs(matched_distance(a, b) - best) < 1e-12


def test_run_accuracy_cardinality():
    acc = RunAccuracy()
    acc.add(np.zeros((3, 2)), np.zeros((4, 2)))
    acc.add(np.zeros((4, 2)), np.zeros((4, 2)))
    s = acc.summary()
    assert s["rel_card_error"] == pytest.approx(0.125) and s["tracking_error_m"] == 0.0


def test_oracle_tracks_a_short_convoy(oracle_mod):
    """The FP64 filter on the convoy workload: after a short settling time the
    cardinality is right and the estimates sit within the detection spread."""
    sc = scenes.convoy_scene(3, 5, steps=25, h_max=25)
    o = oracle_mod.Oracle(sc.filter_config())
    acc = RunAccuracy()
    for k, fr in enumerate(sc.frames):
        o.step(fr.births, fr.Z)
        e = o.estimates()
        if k >= 5:
            acc.add(e["mean"][:, :2], fr.truth[:, :2])
    s = acc.summary()
    assert s["rel_card_error"] < 0.05, s
    assert s["tracking_error_m"] < 0.25, s


def test_ospa_closed_forms():
    from scenes.metrics import ospa
    a = np.array([[0.0, 0.0], [10.0, 0.0]])
    assert ospa(a, a) == 0.0
    assert ospa(np.zeros((0, 2)), a, c=50) == 50.0
    # one missed object out of two: (0 + c) / 2
    assert ospa(a[:1], a, c=40.0) == pytest.approx(20.0)
    # shifted by 3 and the cut-off not reached: mean distance
    assert ospa(a + [0.0, 3.0], a, c=100.0) == pytest.approx(3.0)
    # order 2 with one far pair: sqrt((d1^2 + c^2) / 2)
    b = np.array([[0.0, 4.0], [500.0, 0.0]])
    assert ospa(b, a, c=30.0, p=2) == pytest.approx(np.sqrt((16 + 900) / 2))


def test_batch_workload_draws_the_stated_ranges():
    """The batched workload: N ~ U{5..300}, H_max ~ U{100..5000}, clutter
    ~ U(5, 40), every scene with its own seed, the same list for the same
    seed."""
    specs = scenes.batch_scenes(256, 4000, frames=100)
    n = np.array([p.n_objects for p, _ in specs])
    h = np.array([p.h_max for p, _ in specs])
    lam = np.array([p.clutter_rate for p, _ in specs])
    assert n.min() >= 5 and n.max() <= 300 and h.min() >= 100 and h.max() <= 5000
    assert lam.min() >= 5.0 and lam.max() <= 40.0
    # roughly uniform: each half of each range holds a fair share of 256
    for v, lo, hi in ((n, 5, 300), (h, 100, 5000), (lam, 5.0, 40.0)):
        assert 0.35 < np.mean(v < (lo + hi) / 2) < 0.65
    assert len({s for _, s in specs}) == 256
    assert [(p.n_objects, p.h_max, s) for p, s in scenes.batch_scenes(256, 4000)] == \
        [(p.n_objects, p.h_max, s) for p, s in specs]
    p0, s0 = specs[0]
    sc = scenes.make_scene(p0, s0)
    assert len(sc.frames) == 100 and sc.dim_z == 2


def test_presets_follow_the_stated_recipes():
    """Tiny, mid and the 3-D sweep scenes carry the parameters of the input
    recipes, and a generated mid scene's detection counts match them:
    alive objects x P_D x (1 + lambda_d) + clutter per frame."""
    t, m = scenes.preset("tiny"), scenes.preset("mid")
    assert (t.dim, t.n_objects, t.frames, t.extent, t.birth_window, t.lambda_d, t.clutter_rate, t.h_max) == \
        (2, 10, 50, 1000.0, (0, 24), 1.0, 5.0, 100)
    assert (m.dim, m.n_objects, m.frames, m.extent, m.birth_window, m.lambda_d, m.clutter_rate, m.h_max) == \
        (2, 100, 100, 1000.0, (0, 49), 1.5, 20.0, 1000)
    for p in (t, m):
        assert (p.p_s, p.p_d, p.sigma, p.speed_max, p.h_up, p.tau) == (0.99, 0.9, 5.0, 10.0, 100, 1e-5)
    for n in (50, 200, 500, 1000):
        s = scenes.preset(f"sweep_N{n}")
        assert (s.dim, s.n_objects, s.frames, s.extent, s.p_d, s.lambda_d, s.clutter_rate, s.sigma) == \
            (3, n, 50, 5000.0, 0.85, 2.0, 50.0, 5.0)
        assert s.births_per_frame == pytest.approx(0.01 * n) and s.birth_window is None
    sc = scenes.make_scene(m, 2024)
    alive = np.array([len(fr.truth) for fr in sc.frames[50:]])
    M = np.array([len(fr.Z) for fr in sc.frames[50:]])
    want = alive * m.p_d * (1 + m.lambda_d) + m.clutter_rate
    assert abs(M.mean() / want.mean() - 1) < 0.05


@pytest.mark.parametrize("p", [1.0, 2.0])
def test_ospa_equals_brute_force_over_assignments(p):
    """OSPA from its definition, every injection of the smaller set into the
    larger enumerated, on small random sets (both orders, cut-off binding
    for some pairs)."""
    import itertools

    from scenes.metrics import ospa
    rng = np.random.default_rng(5 + int(p))
    c = 30.0
    for _ in range(25):
        m, n = rng.integers(1, 5, size=2)
        X = rng.uniform(0, 60, size=(m, 2))
        Y = rng.uniform(0, 60, size=(n, 2))
        A, B = (X, Y) if m <= n else (Y, X)
        best = min(sum(min(np.linalg.norm(A[i] - B[j]), c) ** p for i, j in enumerate(perm))
                   for perm in itertools.permutations(range(len(B)), len(A)))
        want = ((best + c ** p * (len(B) - len(A))) / len(B)) ** (1 / p)
        assert ospa(X, Y, c=c, p=p) == pytest.approx(want, rel=1e-12)
        assert ospa(Y, X, c=c, p=p) == pytest.approx(want, rel=1e-12)
