"""Pins of the oracle's particle track model (model 1: weighted particles with
constant-turn-rate-and-velocity motion, Section 3 of the paper, reading R15)
against closed forms, the textbook Kalman filter in the linear-Gaussian
limit, brute force on tiny inputs and sampling statistics.  CPU only."""
from __future__ import annotations

import math

import numpy as np
import pytest
from scipy.stats import kstest, multivariate_normal

R2 = 4.0 * np.eye(2)


def pcfg(**kw):
    cfg = dict(dim_x=5, dim_z=2, dt=1.0, q=0.0, R=R2.tolist(), p_s=0.95, p_d=0.8, lambda_d=0.7,
               clutter_rate=2.0, volume=1.0e4, gate=float("inf"), h_max=50, h_up=200, tau=1e-9,
               seed=12345, score_mode=1, model=1, n_particles=4, sigma_a=0.0, sigma_w=0.0,
               ess_frac=0.0)
    cfg.update(kw)
    return cfg


def cloud_track(lk, lb, x, lw):
    """A state track record carrying particles (the moments are recomputed
    by the oracle on import)."""
    x = np.asarray(x, float)
    lw = np.asarray(lw, float)
    return (lk, lb, np.zeros(5), np.eye(5), x, lw)


def run_update(oracle_mod, cfg, tracks, Z, births=(), logw=0.0, frame=3):
    o = oracle_mod.Oracle(cfg)
    o.import_state(frame, np.array([logw]), np.array([99], np.uint64), [tracks])
    o.predict(list(births))
    o.update(np.asarray(Z, np.float32).reshape(-1, 2))
    return o


def mixture_loglik(z, pts, w):
    return math.log(sum(wk * multivariate_normal(p, R2).pdf(z) for p, wk in zip(pts, w)))


# --------------------------------------------------------------------------
# CTRV kinematics (R15a)
# --------------------------------------------------------------------------
def test_ctrv_straight_line_without_turn(oracle_mod):
    x = np.array([10.0, -3.0, 7.0, 0.4, 0.0])
    out = oracle_mod.ctrv(x, 2.0)
    ref = [10.0 + 14.0 * math.cos(0.4), -3.0 + 14.0 * math.sin(0.4), 7.0, 0.4, 0.0]
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("om,dt", [(0.3, 1.0), (-0.7, 0.5), (1e-3, 2.0)])
def test_ctrv_arc_matches_the_textbook_form(oracle_mod, om, dt):
    px, py, v, psi = 5.0, 8.0, 12.0, -1.1
    out = oracle_mod.ctrv([px, py, v, psi, om], dt)
    ref = [px + v / om * (math.sin(psi + om * dt) - math.sin(psi)),
           py + v / om * (math.cos(psi) - math.cos(psi + om * dt)), v, psi + om * dt, om]
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-9)


def test_ctrv_quarter_and_full_circles(oracle_mod):
    v, dt = 6.0, 1.0
    om = (math.pi / 2) / dt
    out = oracle_mod.ctrv([0.0, 0.0, v, 0.0, om], dt)       # quarter turn, radius v / om
    np.testing.assert_allclose(out[:2], [v / om, v / om], atol=1e-12)
    out = oracle_mod.ctrv([3.0, 4.0, v, 0.2, 2 * math.pi / dt], dt)   # full turn: back to the start
    np.testing.assert_allclose(out[:2], [3.0, 4.0], atol=1e-12)
    assert out[3] == pytest.approx(0.2 + 2 * math.pi)


def test_ctrv_is_continuous_at_zero_turn_rate(oracle_mod):
    a = oracle_mod.ctrv([1.0, 2.0, 9.0, 0.7, 0.0], 1.5)
    b = oracle_mod.ctrv([1.0, 2.0, 9.0, 0.7, 1e-9], 1.5)
    np.testing.assert_allclose(a[:2], b[:2], atol=1e-7)


def test_ctrv_acceleration_terms(oracle_mod):
    dt, a, al, psi = 0.5, 1.3, -0.4, 0.9
    out = oracle_mod.ctrv([0.0, 0.0, 0.0, psi, 0.0], dt, a, al)
    ref = [0.5 * dt * dt * math.cos(psi) * a, 0.5 * dt * dt * math.sin(psi) * a, dt * a,
           psi + 0.5 * dt * dt * al, dt * al]
    np.testing.assert_allclose(out, ref, atol=1e-15)
    # while turning, the accelerations act along the heading before the step
    x = [5.0, 6.0, 9.0, psi, 0.8]
    d = oracle_mod.ctrv(x, dt, a, al) - oracle_mod.ctrv(x, dt)
    np.testing.assert_allclose(d, [ref[0], ref[1], dt * a, 0.5 * dt * dt * al, dt * al], atol=1e-12)


# --------------------------------------------------------------------------
# random draws (R15b): standard normal, independent pairs and streams
# --------------------------------------------------------------------------
def test_particle_normals_are_standard_and_independent(oracle_mod):
    o = oracle_mod.Oracle(pcfg())
    n = 20000
    a = np.array([o.particle_normals(7, 3, p, 1, 0) for p in range(n)])
    b = np.array([o.particle_normals(7, 3, p, 2, 0) for p in range(n)])
    for col in (a[:, 0], a[:, 1], b[:, 0]):
        assert abs(col.mean()) < 5 / math.sqrt(n)
        assert abs(col.var() - 1.0) < 5 * math.sqrt(2.0 / n)
        assert kstest(col, "norm").pvalue > 1e-4
    for u, v in ((a[:, 0], a[:, 1]), (a[:, 0], b[:, 0]), (a[:, 1], b[:, 1])):
        assert abs(np.corrcoef(u, v)[0, 1]) < 5 / math.sqrt(n)


# --------------------------------------------------------------------------
# prediction and births (R15a, b, f)
# --------------------------------------------------------------------------
def test_prediction_spread_is_the_linear_noise_covariance(oracle_mod):
    """Identical particles take the same deterministic step; the
    accelerations then enter linearly, so the predicted cloud's covariance
    is G diag(sigma_a^2, sigma_w^2) G^T."""
    Np, dt, sa, sw = 20000, 0.8, 0.7, 0.03
    x0 = np.array([100.0, 50.0, 8.0, 0.3, 0.05])
    cfg = pcfg(n_particles=Np, dt=dt, sigma_a=sa, sigma_w=sw)
    o = run_update(oracle_mod, cfg, [cloud_track(2, 0, np.tile(x0, (Np, 1)), np.full(Np, -math.log(Np)))],
                   np.zeros((0, 2)))
    x, lw = o.slot_particles(0, 0)
    np.testing.assert_allclose(lw, -math.log(Np))
    G = np.array([[0.5 * dt * dt * math.cos(x0[3]), 0], [0.5 * dt * dt * math.sin(x0[3]), 0], [dt, 0],
                  [0, 0.5 * dt * dt], [0, dt]])
    C = G @ np.diag([sa * sa, sw * sw]) @ G.T
    mu = oracle_mod.ctrv(x0, dt)
    se = np.sqrt(np.diag(C) / Np)
    assert np.all(np.abs(x.mean(0) - mu) < 6 * se + 1e-12)
    emp = np.cov(x.T, bias=True)
    for i in range(5):
        assert emp[i, i] == pytest.approx(C[i, i], rel=6 * math.sqrt(2.0 / Np))
    # the slot's moments are the weighted moments of its particles
    s = o.slot(0, 0)
    np.testing.assert_allclose(s["mean"], x.mean(0), rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(s["cov"], emp, rtol=1e-9, atol=1e-12)


def test_birth_particles_follow_the_birth_density(oracle_mod):
    Np = 20000
    m = np.array([300.0, 400.0, 10.0, 0.5, 0.01])
    L = np.array([[3, 0, 0, 0, 0], [1, 2, 0, 0, 0], [0, 0, 4, 0, 0], [0, 0, 0.5, 0.3, 0],
                  [0, 0, 0, 0.01, 0.02]], float)
    P = L @ L.T
    o = run_update(oracle_mod, pcfg(n_particles=Np), [], np.zeros((0, 2)), births=[(0.4, m, P)])
    x, lw = o.slot_particles(0, 0)
    np.testing.assert_allclose(lw, -math.log(Np))
    se = np.sqrt(np.diag(P) / Np)
    assert np.all(np.abs(x.mean(0) - m) < 6 * se)
    emp = np.cov(x.T, bias=True)
    for i in range(5):
        for j in range(5):
            tol = 6 * math.sqrt((P[i, i] * P[j, j] + P[i, j] ** 2) / Np)
            assert abs(emp[i, j] - P[i, j]) < tol, (i, j)
    assert o.slot(0, 0)["label"] == (4, 0)   # label (frame, birth index)


# --------------------------------------------------------------------------
# compatibility entries, weights and death probability (R15c, d; R2)
# --------------------------------------------------------------------------
def test_compatibility_entry_is_pd_times_the_particle_mixture(oracle_mod):
    pts = [np.array([10.0, 20.0]), np.array([13.0, 18.0])]
    x = np.array([[*pts[0], 0, 0.1, 0.0], [*pts[1], 0, 0.2, 0.0], [*pts[1], 0, 0.3, 0.0],
                  [*pts[1], 0, 0.4, 0.0]])
    w = np.array([0.4, 0.2, 0.2, 0.2])
    Z = [[11.0, 19.0], [14.0, 17.5], [30.0, 40.0]]
    o = run_update(oracle_mod, pcfg(), [cloud_track(2, 0, x, np.log(w))], Z)
    for i, z in enumerate(Z):
        ref = math.log(0.8) + mixture_loglik(z, pts, [0.4, 0.6])
        assert o.pair(0, 0, i)["logC"] == pytest.approx(ref, rel=1e-12, abs=1e-12)


def _two_track_state():
    x1 = np.array([[10.0, 20.0, 0, 0, 0], [12.0, 21.0, 0, 0, 0], [9.0, 19.0, 0, 0, 0], [11.0, 18.0, 0, 0, 0]])
    x2 = np.array([[40.0, 20.0, 0, 0, 0], [41.0, 22.0, 0, 0, 0], [39.0, 21.0, 0, 0, 0], [40.0, 18.0, 0, 0, 0]])
    w1 = np.log([0.1, 0.2, 0.3, 0.4])
    w2 = np.log([0.25, 0.25, 0.25, 0.25])
    return [cloud_track(2, 0, x1, w1), cloud_track(2, 1, x2, w2)], [(x1, w1), (x2, w2)]


def test_child_weights_are_products_of_particle_entries(oracle_mod):
    """Every enumerated child's weight against an independent restatement:
    parent weight, (1 - p) per dead track, p (1 - P_D) per missed track,
    p prod C[i, t] over a detected track's detections, kappa per clutter
    detection, with C from the particle mixture."""
    tracks, clouds = _two_track_state()
    Z = [[11.0, 19.5], [40.5, 20.0], [25.0, 25.0]]
    cfg = pcfg()
    o = run_update(oracle_mod, cfg, tracks, Z, logw=-0.37)
    dead, theta, lw = o.bruteforce(0)
    kappa = cfg["clutter_rate"] / cfg["volume"]
    logC = [[math.log(0.8) + mixture_loglik(z, [p[:2] for p in cx], np.exp(cw)) for z in Z]
            for cx, cw in clouds]
    assert len(lw) == 3 ** 3 + 2 * 2 ** 3 + 1   # associations to the alive tracks only
    for j in range(len(lw)):
        ref = -0.37
        for t in range(2):
            if dead[j, t]:
                ref += math.log(1 - 0.95)
                continue
            ref += math.log(0.95)
            rows = [i for i in range(3) if theta[j, i] == t + 1]
            ref += sum(logC[t][i] for i in rows) if rows else math.log(1 - 0.8)
        ref += sum(1 for i in range(3) if theta[j, i] == 0) * math.log(kappa)
        assert abs(lw[j] - ref) < 1e-9, (j, lw[j], ref)


def test_death_probability_is_the_exact_marginal_with_particles(oracle_mod):
    """Reading R2 with a particle C entry, where it is exact under the
    product-of-entries weights: one track, one detection.  The marginal
    probability of death over every enumerated child (dead; alive and
    missed; alive with the detection) is what R2 computes."""
    tracks, _ = _two_track_state()
    o = run_update(oracle_mod, pcfg(p_s=0.9), tracks[:1], [[11.0, 19.5]])
    dead, theta, lw = o.bruteforce(0)
    assert len(lw) == 3
    w = np.exp(lw - lw.max())
    p_dead = w[dead[:, 0] == 1].sum() / w.sum()
    assert o.slot(0, 0)["dprob"] == pytest.approx(p_dead, rel=1e-10, abs=1e-14)


def test_death_probability_follows_reading_with_particle_entries(oracle_mod):
    tracks, clouds = _two_track_state()
    Z = [[11.0, 19.5], [13.0, 22.0], [60.0, 60.0]]
    cfg = pcfg(p_s=0.9)
    o = run_update(oracle_mod, cfg, tracks, Z)
    kappa = cfg["clutter_rate"] / cfg["volume"]
    for t, (cx, cw) in enumerate(clouds):
        psi = (1 - 0.8) + sum(0.8 * math.exp(mixture_loglik(z, [p[:2] for p in cx], np.exp(cw)))
                              for z in Z) / kappa
        assert o.slot(0, t)["dprob"] == pytest.approx(0.1 / (0.1 + 0.9 * psi), rel=1e-12)


# --------------------------------------------------------------------------
# particle update and resampling (R15e)
# --------------------------------------------------------------------------
def test_particle_update_weights_are_prior_times_likelihoods(oracle_mod):
    tracks, clouds = _two_track_state()
    Z = [[11.0, 19.5], [10.0, 20.5], [40.5, 20.0]]
    cfg = pcfg(p_d=0.95, clutter_rate=0.01, h_max=200)
    o = run_update(oracle_mod, cfg, tracks, Z)
    o.prune()
    _, _, _, hyps = o.export_state()
    th = o.kept_theta()
    checked = 0
    for h, tr in enumerate(hyps):
        for a, rec in enumerate(tr):
            src = 0 if rec[1] == 0 else 1
            cx, cw = clouds[src]
            rows = [i for i in range(3) if th[h, i] == a + 1]
            ref = cw.copy()
            for i in rows:
                ref += np.array([multivariate_normal(p[:2], R2).logpdf(Z[i]) for p in cx])
            ref -= np.log(np.exp(ref).sum())
            np.testing.assert_allclose(rec[5], ref, rtol=0, atol=1e-12)
            np.testing.assert_array_equal(rec[4], cx)       # no resampling at ess_frac 0
            # the track's moments are its particles' weighted moments
            wv = np.exp(ref)
            np.testing.assert_allclose(rec[2], wv @ cx, rtol=1e-12, atol=1e-12)
            checked += bool(rows)
    assert checked >= 2


def test_systematic_resampling_counts(oracle_mod):
    """With resampling on every update, particle k is copied floor(P w_k) or
    ceil(P w_k) times (a property of systematic resampling), P in all, with
    weights 1/P."""
    rng = np.random.default_rng(5)
    Np = 64
    x = np.zeros((Np, 5))
    x[:, :2] = [50.0, 50.0] + rng.normal(scale=3.0, size=(Np, 2))
    x[:, 3] = np.arange(Np) * 0.01           # distinct headings identify the particles
    lw0 = np.full(Np, -math.log(Np))
    z = [51.0, 49.0]
    cfg = pcfg(n_particles=Np, ess_frac=1.0, p_d=0.99, clutter_rate=0.001, h_max=5)
    o = run_update(oracle_mod, cfg, [cloud_track(2, 0, x, lw0)], [z])
    o.prune()
    _, _, _, hyps = o.export_state()
    th = o.kept_theta()
    h = next(j for j in range(len(hyps)) if len(hyps[j]) == 1 and th[j, 0] == 1)
    xr, lwr = hyps[h][0][4], hyps[h][0][5]
    np.testing.assert_allclose(lwr, -math.log(Np))
    lik = np.array([multivariate_normal(p[:2], R2).pdf(z) for p in x])
    w = lik / lik.sum()
    ids = np.rint(xr[:, 3] / 0.01).astype(int)
    counts = np.bincount(ids, minlength=Np)
    assert counts.sum() == Np
    assert np.all(counts >= np.floor(Np * w) - 1e-9) and np.all(counts <= np.ceil(Np * w) + 1e-9)
    assert o.resample_margin() < math.inf


def test_particle_update_approaches_the_kalman_filter(oracle_mod):
    """Linear-Gaussian limit: a birth's particles drawn from N(m, P) and
    updated with one detection have the Kalman posterior mean (within the
    importance-sampling error)."""
    Np = 20000
    m = np.array([300.0, 400.0, 0.0, 0.0, 0.0])
    P = np.diag([9.0, 16.0, 1e-6, 0.01, 1e-4])
    z = np.array([302.0, 397.0])
    cfg = pcfg(n_particles=Np, p_d=0.99, clutter_rate=0.001, h_max=5)
    o = oracle_mod.Oracle(cfg)
    o.predict([(0.99, m, P)])
    o.update(np.array([z], np.float32))
    o.prune()
    _, _, _, hyps = o.export_state()
    th = o.kept_theta()
    h = next(j for j in range(len(hyps)) if len(hyps[j]) == 1 and th[j, 0] == 1)
    mean, w = hyps[h][0][2], np.exp(hyps[h][0][5])
    H = np.zeros((2, 5))
    H[:, :2] = np.eye(2)
    S = H @ P @ H.T + R2
    K = P @ H.T @ np.linalg.inv(S)
    m_post = m + K @ (z - H @ m)
    P_post = P - K @ H @ P
    ess = 1.0 / np.sum(w * w)
    se = np.sqrt(np.diag(P_post)[:2] / ess)
    assert np.all(np.abs(mean[:2] - m_post[:2]) < 6 * se)


def test_particle_state_round_trip(oracle_mod):
    tracks, clouds = _two_track_state()
    o = oracle_mod.Oracle(pcfg())
    o.import_state(3, np.array([0.0]), np.array([9], np.uint64), [tracks])
    fr, lw, uid, hyps = o.export_state()
    assert fr == 3 and len(hyps[0]) == 2
    for rec, (cx, cw) in zip(hyps[0], clouds):
        np.testing.assert_array_equal(rec[4], cx)
        np.testing.assert_array_equal(rec[5], cw)
        np.testing.assert_allclose(rec[2], np.exp(cw) @ cx, rtol=1e-14)


def test_particle_model_rejects_other_shapes(oracle_mod):
    for bad in (dict(dim_x=4), dict(score_mode=0), dict(n_particles=0), dict(ess_frac=1.5)):
        with pytest.raises(oracle_mod.OracleError):
            oracle_mod.Oracle(pcfg(**bad))
