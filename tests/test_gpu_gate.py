"""The learned pair gate on the GPU against its FP64 reference: forward pass
(tensor cores) and backward pass against oracle/gate_mlp.py, Adam, a frame
of the filter with the gate pruning against the oracle filter with the same
gate, and the training labels against a host restatement."""
from __future__ import annotations

import numpy as np
import pytest

import scenes
from oracle import gate_mlp as gm
from tests import parity

pytestmark = pytest.mark.gpu

MU = np.array([6.0, 8.0, 0.6, 10.0, 5.0])
SD = np.array([5.0, 6.0, 0.35, 10.0, 1.5])


@pytest.fixture(scope="module")
def glmb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_06230_gb300 as g
    g.build()
    g.load()
    return g


def _feat(rng, n):
    return np.stack([rng.chisquare(2, n) * 3, rng.gamma(2.0, 4.0, n), rng.uniform(0, 1, n),
                     rng.integers(0, 40, n).astype(float), rng.normal(5.0, 1.5, n)], 1).astype(np.float32)


def _dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t.to(dtype) if dtype is not None else t).cuda()


@pytest.mark.parametrize("n", [1, 5, 128, 129, 1000, 20000])
def test_forward_matches_oracle(glmb, n):
    import torch
    rng = np.random.default_rng(n)
    p = scenes.gate_params(n, MU, SD, scale=1.5, bias=0.3)
    X = _feat(rng, n)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    z = glmb.mlp_forward(_dev(p), _dev(X), err).cpu().numpy().astype(np.float64)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    # the same precision the kernel decides in: bf16 inputs and activations
    ref, _ = gm.forward(p, X.astype(np.float64), round_act=True)
    d = np.abs(z - ref)
    print(f"\nmax |dz| {d.max():.3g}  median {np.median(d):.3g}  |z| max {np.abs(ref).max():.3g}")
    assert np.all(d <= 0.02 + 0.01 * np.abs(ref))
    assert np.median(d) < 1e-3
    # and the plain FP64 network: agreement to bf16 precision
    ref64, _ = gm.forward(p, X.astype(np.float64), round_act=False)
    assert np.max(np.abs(z - ref64)) <= 0.05 * (1.0 + np.max(np.abs(ref64)))


def test_forward_empty_launches_nothing(glmb):
    import torch
    p = _dev(scenes.gate_params(1))
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    z = glmb.mlp_forward(p, torch.zeros((0, 5), dtype=torch.float32, device="cuda"), err)
    assert z.numel() == 0


@pytest.mark.parametrize("n", [100, 777, 5000])
def test_backward_matches_oracle(glmb, n):
    import torch
    rng = np.random.default_rng(100 + n)
    p = scenes.gate_params(n, MU, SD, scale=1.3, bias=-0.4)
    X = _feat(rng, n)
    y = (rng.uniform(size=n) < 0.3).astype(np.float32)
    wt = rng.uniform(0.5, 2.0, n).astype(np.float32) / n
    grad = torch.zeros(gm.NPARAM, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    glmb.mlp_backward(_dev(p), _dev(X), _dev(y), _dev(wt), grad, loss, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    L, g_ref = gm.loss_and_grad(p, X.astype(np.float64), y, wt)
    g = grad.cpu().numpy().astype(np.float64)
    assert float(loss.item()) == pytest.approx(L, rel=1e-2)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4"):
        s = slice(gm.OFF[k], gm.OFF[k] + int(np.prod(gm.SHAPES[k])))
        rel = np.linalg.norm(g[s] - g_ref[s]) / max(np.linalg.norm(g_ref[s]), 1e-12)
        print(f"{k}: rel L2 {rel:.3g}")
        assert rel < 3e-2, k
    assert np.all(g[gm.NTRAIN:] == 0.0)


def test_adam_matches_oracle(glmb):
    import torch
    rng = np.random.default_rng(7)
    p = rng.normal(size=gm.NPARAM).astype(np.float32)
    g = rng.normal(size=gm.NPARAM).astype(np.float32)
    m = rng.normal(scale=0.1, size=gm.NPARAM).astype(np.float32)
    v = rng.uniform(0.0, 0.1, size=gm.NPARAM).astype(np.float32)
    pt, mt, vt = _dev(p), _dev(m[:gm.NTRAIN]), _dev(v[:gm.NTRAIN])
    glmb.mlp_adam(pt, _dev(g), mt, vt, 3, 1e-3)
    torch.cuda.synchronize()
    q_ref, m_ref, v_ref = gm.adam_step(p, g, m, v, 3, lr=1e-3)
    np.testing.assert_allclose(pt.cpu().numpy(), q_ref, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(mt.cpu().numpy(), m_ref[:gm.NTRAIN], rtol=1e-5, atol=1e-7)
    # 1 - beta2 in float32 (0.999f is not 0.999) carries a relative error of
    # about 1.7e-5 into the second moment's new term
    np.testing.assert_allclose(vt.cpu().numpy(), v_ref[:gm.NTRAIN], rtol=5e-5, atol=1e-9)


def test_training_separates_a_learnable_rule(glmb):
    """Labels from a fixed rule of the features (small d^2 and high
    existence): Adam on the GPU gradients drives the loss well down."""
    import torch
    rng = np.random.default_rng(11)
    n = 8192
    X = _feat(rng, n)
    y = ((X[:, 0] < 6.0) & (X[:, 2] > 0.3)).astype(np.float32)
    wt = np.full(n, 1.0 / n, np.float32)
    P = _dev(scenes.gate_params(5, MU, SD, scale=1.0))
    m = torch.zeros(gm.NTRAIN, device="cuda")
    v = torch.zeros(gm.NTRAIN, device="cuda")
    grad = torch.zeros(gm.NPARAM, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    Xd, yd, wd = _dev(X), _dev(y), _dev(wt)
    first = None
    for t in range(1, 301):
        glmb.mlp_backward(P, Xd, yd, wd, grad, loss, err)
        glmb.mlp_adam(P, grad, m, v, t, 3e-3)
        if first is None:
            first = float(loss.item())
    last = float(loss.item())
    assert int(err.item()) == 0
    z = glmb.mlp_forward(P, Xd, err).cpu().numpy()
    acc = np.mean((z >= 0) == (y > 0.5))
    print(f"\nloss {first:.4f} -> {last:.4f}, accuracy {acc:.4f}")
    assert last < 0.3 * first and acc > 0.97


def _oracle_logits(oracle_mod, cfg, state, births, Z, params):
    """FP64 logits (bf16-activation forward) of every pair of the frame that
    passes the Mahalanobis test, from the oracle without the gate."""
    frame, logw, uid, tracks = state
    o = oracle_mod.Oracle(cfg, n_threads=8)
    o.import_state(frame, logw, uid, tracks)
    o.predict(births)
    o.update(Z)
    out = []
    for h in range(o.num_parents()):
        for t in range(o.parent_slots(h)):
            for i in range(len(Z)):
                if o.pair(h, t, i)["gated"]:
                    out.append(o.gate_eval(h, t, i)[0])
    X = np.array(out)
    return gm.forward(params, X, round_act=True)[0]


def _threshold_in_gap(z, q):
    """A threshold near quantile q of z with no logit within 4 MLP_MARGIN."""
    zs = np.sort(np.unique(z))
    gaps = np.diff(zs)
    target = np.quantile(zs, q)
    ok = np.nonzero(gaps > 8 * parity.MLP_MARGIN)[0]
    assert len(ok), "no gap wide enough"
    j = ok[np.argmin(np.abs(zs[ok] - target))]
    return float(0.5 * (zs[j] + zs[j + 1]))


@pytest.mark.parametrize("k,q", [(6, 0.3), (20, 0.5)])
def test_gated_frame_matches_oracle(oracle_mod, glmb, k, q):
    sc = scenes.make_scene(scenes.preset("tiny"), 1001)
    cfg = sc.filter_config()
    state = parity.oracle_state(oracle_mod, cfg, sc, k)
    fr = sc.frames[k]
    params = scenes.gate_params(21, MU, SD, scale=1.5, bias=0.5)
    z = _oracle_logits(oracle_mod, cfg, state, fr.births, fr.Z, params)
    thr = _threshold_in_gap(z, q)
    o, g, d = parity.run_frame(oracle_mod, glmb, cfg, state, fr.births, fr.Z, gate=(params, thr))
    assert all(o.mlp_margin(h) >= parity.MLP_MARGIN for h in range(o.num_parents()))
    info = g.info()
    assert info["n_pairs"] < info["n_pairs_pregate"]
    rep = parity.compare(o, g, d, cfg, fr.Z)
    print(f"\nthr {thr:.3f}: pairs {info['n_pairs']} of {info['n_pairs_pregate']}; checks {rep.checks} "
          f"excused {rep.excused}")
    assert rep.ok(), rep.failures[:10]


def test_score_mode_changes_nothing_and_logits_match_features(glmb):
    """SCORE mode leaves every result of the frame as it is, and its in-table
    logits equal the forward pass on the features the library exports."""
    import torch
    sc = scenes.make_scene(scenes.preset("tiny"), 1002)
    cfg = sc.filter_config()
    params = scenes.gate_params(22, MU, SD, scale=1.2)
    a, b = glmb.Filter(cfg), glmb.Filter(cfg)
    b.set_gate(params, 0.0, glmb.Filter.GATE_SCORE)
    for fr in sc.frames[:12]:
        a.step(fr.births, fr.Z)
        b.step(fr.births, fr.Z)
        ha, hb = a.hypotheses(), b.hypotheses()
        np.testing.assert_array_equal(ha["logw"], hb["logw"])
        np.testing.assert_array_equal(ha["uid"], hb["uid"])
    X = b.gate_features()
    zl = b.gate_logits()
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    zr = glmb.mlp_forward(_dev(params), _dev(X), err).cpu().numpy()
    np.testing.assert_array_equal(zl, zr)


def test_usage_labels_match_host_restatement(glmb):
    """The usage kernel against the same labels built on the host from the
    retained hypotheses, their parents and the pair table."""
    sc = scenes.make_scene(scenes.preset("tiny"), 1005)
    cfg = sc.filter_config()
    f = glmb.Filter(cfg)
    for fr in sc.frames[:8]:
        f.step(fr.births, fr.Z)
    fr = sc.frames[8]
    f.predict(fr.births)
    f.update(fr.Z)
    pptr, pcomp = f.parents()
    comps = f.components()
    pairs = f.pairs()
    n_comp = len(comps["p"]) - len(fr.births)
    f.prune()
    idx, _ = f.retained()
    hyp = f.hypotheses()
    used, flag = f.gate_usage()
    ref = np.zeros(len(pairs["meas"]), np.uint8)
    lab = list(zip(comps["label_k"].tolist(), comps["label_b"].tolist()))
    for j, ch in enumerate(idx.tolist()):
        p = ch // cfg["h_up"]
        slots = [int(c) for c in pcomp[pptr[p]:pptr[p + 1]]] + [n_comp + b for b in range(len(fr.births))]
        by_label = {lab[c]: c for c in slots}
        new = list(zip(hyp["label_k"][hyp["ptr"][j]:hyp["ptr"][j + 1]].tolist(),
                       hyp["label_b"][hyp["ptr"][j]:hyp["ptr"][j + 1]].tolist()))
        for i, t in enumerate(hyp["theta"][j].tolist()):
            if t:
                c = by_label[new[t - 1]]
                lo, hi = pairs["ptr"][c], pairs["ptr"][c + 1]
                k = lo + int(np.searchsorted(pairs["meas"][lo:hi], i))
                assert pairs["meas"][k] == i
                ref[k] = 1
    assert ref.sum() > 0
    np.testing.assert_array_equal(used, ref)
    assert not flag.any()
