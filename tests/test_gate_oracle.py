"""Pins of the learned gate's FP64 reference (oracle/gate_mlp.py and the C
oracle's gate) against facts that do not come from the oracle itself:
central finite differences, closed forms of degenerate networks, values of
the normal distribution function, exact bf16 roundings, an independent
restatement of the features, and the gate's invariants.  CPU only."""
from __future__ import annotations

import math

import numpy as np
import pytest

import scenes
from oracle import gate_mlp as gm
from tests._helpers import base_cfg, state_tracks

PHI1 = 0.8413447460685429          # standard normal distribution function at 1


def _feat(rng, n):
    return np.stack([rng.chisquare(2, n), rng.gamma(2.0, 3.0, n), rng.uniform(0, 1, n),
                     rng.integers(0, 40, n).astype(float), rng.normal(4.0, 1.0, n)], 1)


def test_bf16_rounding_exact_values():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -8 + 2 ** -20, 1.0 + 3 * 2 ** -8, -2.0 ** -130,
                  3.0e38, np.inf, -np.inf])
    r = gm.bf16(x)
    assert r[0] == 1.0
    assert r[1] == 1.0                       # halfway, ties to the even neighbour
    assert r[2] == 1.0 + 2 ** -7             # above halfway
    assert r[3] == 1.0 + 2 ** -6             # halfway between 1+2^-7 and 1+2^-6: even is 2^-6
    assert r[4] == -2.0 ** -130              # subnormal with short mantissa is exact
    assert np.isposinf(r[6]) and np.isneginf(r[7])


def test_gelu_values_of_the_normal_distribution():
    assert gm.gelu(np.array([1.0]))[0] == pytest.approx(PHI1, abs=1e-15)
    assert gm.gelu(np.array([-1.0]))[0] == pytest.approx(-(1 - PHI1), abs=1e-15)
    assert gm.gelu(np.array([0.0]))[0] == 0.0
    # derivative against a central difference
    x = np.linspace(-4, 4, 33)
    h = 1e-6
    fd = (gm.gelu(x + h) - gm.gelu(x - h)) / (2 * h)
    np.testing.assert_allclose(gm.gelu_grad(x), fd, atol=1e-8)


def test_zero_weight_network_is_a_closed_form():
    """With W1 = W2 = W3 = 0 every hidden layer is GELU of its bias, so the
    logit is b4 + sum_o bf16(w4_o) GELU(b3_o) whatever the input."""
    p = scenes.gate_params(3)
    w = gm.unpack(p)
    for k in ("W1", "W2", "W3"):
        p[gm.OFF[k]:gm.OFF[k] + w[k].size] = 0.0
    w = gm.unpack(p)
    ref = float(p[gm.OFF["b4"]]) + sum(float(w["w4"][o]) * 0.5 * float(w["b3"][o])
                                       * (1 + math.erf(float(w["b3"][o]) / math.sqrt(2)))
                                       for o in range(64))
    X = _feat(np.random.default_rng(0), 7)
    z, _ = gm.forward(p, X)
    np.testing.assert_allclose(z, ref, rtol=1e-13)
    # the loss gradient of the output bias is sum wt (sigmoid(z) - y)
    y = np.array([1, 0, 1, 1, 0, 0, 1], float)
    wt = np.linspace(0.5, 2.0, 7)
    _, g = gm.loss_and_grad(p, X, y, wt)
    assert g[gm.OFF["b4"]] == pytest.approx(np.sum(wt * (1 / (1 + np.exp(-ref)) - y)), rel=1e-12)


@pytest.mark.parametrize("seed", [1, 2])
def test_gradient_matches_central_differences(seed):
    rng = np.random.default_rng(seed)
    mu = np.array([2.0, 6.0, 0.5, 20.0, 4.0])
    sd = np.array([2.0, 4.0, 0.3, 12.0, 1.0])
    p = scenes.gate_params(seed, mu, sd, scale=1.5, bias=-0.5).astype(np.float64)
    X = _feat(rng, 40)
    y = (rng.uniform(size=40) < 0.4).astype(float)
    wt = rng.uniform(0.2, 2.0, 40)
    _, g = gm.loss_and_grad(p, X, y, wt)
    # perturb the bf16-rounded weights directly: the gradient is taken with
    # respect to the weights the network uses
    w = gm.unpack(p)
    idx = np.concatenate([rng.choice(np.arange(gm.OFF[k], gm.OFF[k] + w[k].size), 6, replace=False)
                          for k in ("W1", "b1", "W2", "b2", "W3", "b3", "w4")] + [[gm.OFF["b4"]]])
    for j in idx:
        def f(delta):
            q = {k: v.copy() for k, v in w.items()}
            name = max((k for k in gm.OFF if gm.OFF[k] <= j), key=lambda k: gm.OFF[k])
            flat = q[name].reshape(-1)
            flat[j - gm.OFF[name]] += delta
            return _loss_from(q, X, y, wt)
        h = 1e-5
        fd = (f(h) - f(-h)) / (2 * h)
        assert g[j] == pytest.approx(fd, rel=1e-6, abs=1e-9), j
    assert np.all(g[gm.NTRAIN:] == 0.0)


def _loss_from(w, X, y, wt):
    """The loss written once more from the unpacked weights (float64, no
    rounding): the network restated layer by layer."""
    x = (X - w["mu"]) / w["sd"]
    a = x
    for Wk, bk in (("W1", "b1"), ("W2", "b2"), ("W3", "b3")):
        zz = a @ w[Wk].T + w[bk]
        a = zz * 0.5 * (1 + np.vectorize(math.erf)(zz / math.sqrt(2)))
    z = a @ w["w4"] + w["b4"][0]
    return float(np.sum(wt * (np.logaddexp(0.0, z) - y * z)))


def test_c_and_numpy_forward_agree(oracle_mod):
    rng = np.random.default_rng(4)
    mu = np.array([2.0, 6.0, 0.5, 20.0, 4.0])
    sd = np.array([2.0, 4.0, 0.3, 12.0, 1.0])
    p = scenes.gate_params(9, mu, sd, scale=1.3, bias=0.2)
    X = _feat(rng, 50)
    for ra in (False, True):
        z, _ = gm.forward(p, X, round_act=ra)
        zc = np.array([oracle_mod.mlp_logit(p, X[j], round_act=ra) for j in range(len(X))])
        np.testing.assert_allclose(zc, z, rtol=1e-12, atol=1e-12)


def test_adam_first_step_moves_by_lr_times_sign():
    """At t = 1 the bias-corrected moments are g and g^2, so each trained
    parameter moves by lr * g / (|g| + eps)."""
    rng = np.random.default_rng(5)
    p = rng.normal(size=gm.NPARAM)
    g = rng.normal(size=gm.NPARAM)
    q, m, v = gm.adam_step(p, g, np.zeros(gm.NPARAM), np.zeros(gm.NPARAM), 1, lr=0.01, eps=1e-8)
    s = slice(0, gm.NTRAIN)
    np.testing.assert_allclose(q[s], p[s] - 0.01 * g[s] / (np.abs(g[s]) + 1e-8), rtol=1e-12)
    assert np.all(q[gm.NTRAIN:] == p[gm.NTRAIN:])


# --------------------------------------------------------------------------
# the gate inside the oracle filter
# --------------------------------------------------------------------------
def _gated(oracle_mod, seed, params, thr, dim=2, M=6):
    rng = np.random.default_rng(seed)
    tracks = state_tracks(rng, dim, 3, spread=10.0)
    cfg = base_cfg(dim, gate=30.0)
    o = oracle_mod.Oracle(cfg)
    o.import_state(3, [-0.2], [7], [tracks])
    o.set_gate(params, thr)
    bl = [(0.4, np.concatenate([rng.uniform(0, 10, dim), np.zeros(dim)]),
           np.diag([30.0] * dim + [4.0] * dim))]
    Z = rng.uniform(-2, 12, size=(M, dim)).astype(np.float32)
    o.predict(bl)
    o.update(Z)
    return o, Z


def test_features_restated_from_the_slot(oracle_mod):
    p = scenes.gate_params(1)
    o, Z = _gated(oracle_mod, 11, p, -np.inf)
    dz = Z.shape[1]
    for t in range(o.parent_slots(0)):
        s = o.slot(0, t)
        S = s["cov"][:dz, :dz] + 4.0 * np.eye(dz)
        for i in range(len(Z)):
            e = Z[i].astype(float) - s["mean"][:dz]
            feat, lg = o.gate_eval(0, t, i)
            np.testing.assert_allclose(feat, [e @ np.linalg.solve(S, e), np.linalg.norm(e), s["p"],
                                              4 - s["label"][0], np.log(np.linalg.det(S))],
                                       rtol=1e-10, atol=1e-12)
            assert lg == pytest.approx(gm.forward(p, feat[None], round_act=True)[0][0], rel=1e-12)


def test_threshold_minus_infinity_keeps_the_plain_table(oracle_mod):
    p = scenes.gate_params(2)
    o, Z = _gated(oracle_mod, 12, p, -np.inf)
    ref, _ = _gated(oracle_mod, 12, None, 0.0)
    a, b = o.children(), ref.children()
    np.testing.assert_array_equal(a["status"], b["status"])
    np.testing.assert_allclose(a["logw"], b["logw"], rtol=0, atol=0)


def test_threshold_plus_infinity_leaves_only_clutter(oracle_mod):
    """With every pair pruned no detection can be assigned to a track, so
    every child assigns every detection to clutter."""
    p = scenes.gate_params(3)
    o, Z = _gated(oracle_mod, 13, p, np.inf)
    st = o.children()["status"]
    for n in np.nonzero(st == 1)[0]:
        dead, theta = o.child(0, int(n))
        assert not theta.any()


def test_gate_prunes_exactly_the_pairs_below_threshold(oracle_mod):
    p = scenes.gate_params(4, scale=2.0)
    plain, Z = _gated(oracle_mod, 14, None, 0.0)
    logits = []
    for t in range(plain.parent_slots(0)):
        for i in range(len(Z)):
            if plain.pair(0, t, i)["gated"]:
                logits.append(gm.forward(p, plain.gate_eval(0, t, i)[0][None], round_act=True)[0][0])
    thr = float(np.median(logits))
    o, _ = _gated(oracle_mod, 14, p, thr)
    for t in range(o.parent_slots(0)):
        for i in range(len(Z)):
            g0 = plain.pair(0, t, i)["gated"]
            lg = gm.forward(p, plain.gate_eval(0, t, i)[0][None], round_act=True)[0][0]
            assert o.pair(0, t, i)["gated"] == (g0 and lg >= thr)
    assert 0 < o.mlp_margin(0) < np.inf
