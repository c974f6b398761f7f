"""Step-by-step comparison of the CUDA library with the FP64 oracle on one
frame from a shared state.  Used by the GPU tests and by the smoke check.

Tolerances (FP32 kernels against the FP64 oracle):
  * association indices, labels, gate sets, duplicate structure: exact,
    except decisions whose oracle margin is below DECISION_MARGIN (the
    24-bit uniform lies that close to a boundary of the normalised row, or
    to the death probability) and children within the boundary window of
    the tau / H_max boundary; those are excused and counted;
  * the boundary window is max(TIE_TOL, 2 x the largest normalised
    log-weight error measured on the children both sides hold in the same
    frame): a child can land on the other side of the cut only if its own
    error and the boundary child's together exceed its distance to it;
  * normalised log-weights: LOGW_TOL absolute;
  * means and covariances: REL_TOL relative (covariances relative to their
    largest entry).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

LOGW_TOL = 1e-4
REL_TOL = 1e-5
DECISION_MARGIN = 1e-5
TIE_TOL = 1e-6
GATE_MARGIN = 1e-5
# learned gate: a pair whose oracle logit is within MLP_MARGIN of the
# threshold may be decided either way (the kernel standardises fp32 features,
# so an input can round to the neighbouring bf16 value; a one-ulp change of
# an input moves the logit by about 1e-2 for unit-scale weights)
MLP_MARGIN = 0.05
# particle model: the moments that gate the pairs hold the mean rounded to
# FP32 (half an ulp, 3e-5 m below 2048 m), which moves d^2 by at most
# 2 sqrt(G) |de| / sqrt(lambda_min(S)), about 7e-6 G for R = 9 m^2
GATE_MARGIN_PARTICLE = 5e-5
# particles are FP64 on both sides (rounding of sin, cos, log, exp and of
# sums in another order): states and log-weights agree to PARTICLE_TOL,
# unless a resampling target lies within RESAMPLE_MARGIN of a cumulative
# weight (the oracle records the smallest distance of the frame)
PARTICLE_TOL = 1e-9
RESAMPLE_MARGIN = 1e-9


@dataclass
class Report:
    checks: dict = field(default_factory=dict)
    excused: dict = field(default_factory=dict)
    max_err: dict = field(default_factory=dict)
    failures: list = field(default_factory=list)

    def fail(self, msg):
        self.failures.append(msg)

    def err(self, key, v):
        self.max_err[key] = max(self.max_err.get(key, 0.0), float(v))

    def ok(self):
        return not self.failures


def excused_children_bound(rep: Report, cfg, M: int) -> float:
    """Upper bound on the children a frame may excuse for close random
    decisions: a child takes one death draw per slot and one categorical
    draw per detection row, and a uniform falls within DECISION_MARGIN of
    one of the (at most two) boundaries next to it with probability at
    most 2 DECISION_MARGIN, so a child is excused with probability at most
    1 - (1 - 2 DECISION_MARGIN)^(T + M); three times that, plus five."""
    children = rep.checks["children"]
    parents = max(1, children // cfg["h_up"])
    decisions = rep.checks["slots"] / parents + M
    frac = 1.0 - (1.0 - 2.0 * DECISION_MARGIN) ** decisions
    return 5.0 + 3.0 * frac * children


def oracle_state(oracle_mod, cfg, scene, n_frames, n_threads=8):
    o = oracle_mod.Oracle(cfg, n_threads=n_threads)
    for fr in scene.frames[:n_frames]:
        o.step(fr.births, fr.Z)
    return o.export_state()


def run_frame(oracle_mod, glmb, cfg, state, births, Z, n_threads=8, gate=None):
    """Both implementations from the same state through one frame; returns
    (oracle, filter, data) with every intermediate needed by compare().
    gate: (params, threshold) of a learned gate that prunes pairs on both sides."""
    frame, logw, uid, tracks = state
    o = oracle_mod.Oracle(cfg, n_threads=n_threads)
    o.import_state(frame, logw, uid, tracks)
    if gate is not None:
        o.set_gate(gate[0], gate[1])
    o.predict(births)
    o.update(Z)
    g = glmb.Filter(cfg)
    if gate is not None:
        g.set_gate(gate[0], gate[1], glmb.Filter.GATE_PRUNE)
    n_part = cfg.get("n_particles", 0) if cfg.get("model", 0) == 1 else 0
    g.import_state(glmb.pack_state(frame, logw, uid, tracks, g.dx, n_part))
    g.predict(births)
    g.update(Z)
    d = dict(g_parents=g.parents(), g_comp=g.components(), g_pairs=g.pairs(),
             g_children=g.children(), o_children=o.children())
    o.prune()
    g.prune()
    d.update(o_state=o.export_state(), o_kept=o.kept(), o_theta=o.kept_theta(),
             g_hyp=g.hypotheses(), g_state=glmb.unpack_state(g.export_state(), n_part),
             o_resample_margin=o.resample_margin(),
             g_retained=g.retained(),
             o_est=o.estimates(), g_est=g.estimates(), o_ru=o.meas_assoc(), g_ru=g.meas_assoc())
    return o, g, d


def _rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.max(np.abs(b)))))


def compare(o, g, d, cfg, Z, report: Report | None = None) -> Report:
    r = report or Report()
    HU = cfg["h_up"]
    H = o.num_parents()
    gptr, gcomp = d["g_parents"]
    gc = d["g_comp"]
    gp = d["g_pairs"]
    dz = cfg["dim_z"]
    G = cfg["gate"]
    particle = cfg.get("model", 0) == 1
    # particles: FP64 on both sides; a resampling decision closer than this
    # to a cumulative weight may go either way
    part_ok = not particle or d.get("o_resample_margin", math.inf) > RESAMPLE_MARGIN
    if particle and not part_ok:
        r.excused["resample_near_tie"] = 1
    # ---- a1 prediction, a2 table, a3 death probability, per (parent, slot)
    n_slots = 0
    # parents with a pair close to either gate's decision: their tables may
    # legitimately differ by that pair (the oracle records both margins
    # while it builds each parent's table)
    gate_margin = GATE_MARGIN_PARTICLE if particle else GATE_MARGIN
    near_gate_parents = {h for h in range(H)
                         if o.mlp_margin(h) < MLP_MARGIN or o.gate_margin(h) < gate_margin}
    for h in range(H):
        T = o.parent_slots(h)
        if gptr[h + 1] - gptr[h] != T:
            r.fail(f"parent {h}: {gptr[h + 1] - gptr[h]} slots on GPU, {T} in oracle")
            continue
        op = o.parent_pairs(h)
        for t in range(T):
            n_slots += 1
            s = o.slot(h, t)
            c = int(gcomp[gptr[h] + t])
            if (int(gc["label_k"][c]), int(gc["label_b"][c])) != s["label"]:
                r.fail(f"label ({h},{t})")
            r.err("mean_rel", _rel(gc["mean"][c], s["mean"]))
            r.err("cov_rel", _rel(gc["cov"][c], s["cov"]))
            r.err("p_abs", abs(gc["p"][c] - s["p"]))
            r.err("dprob_abs", abs(gc["dprob"][c] - s["dprob"]))
            lo, hi = gp["ptr"][c], gp["ptr"][c + 1]
            gm = gp["meas"][lo:hi]
            a, b = op["ptr"][t], op["ptr"][t + 1]
            om = op["meas"][a:b]
            # values of the pairs both sides hold
            both, gi, oi = np.intersect1d(gm, om, assume_unique=True, return_indices=True)
            if len(both):
                j = lo + gi
                k = a + oi
                r.err("logC_abs", np.max(np.abs(gp["logC"][j] - op["logC"][k])))
                if not particle:   # (the particle model's C does not use them)
                    r.err("q_rel", np.max(np.abs(gp["q"][j] - op["q"][k]) / np.maximum(1.0, np.abs(op["q"][k]))))
                    r.err("e_rel", float(np.max(np.max(np.abs(gp["e"][j] - op["e"][k]), axis=1)
                                                / np.maximum(1.0, np.max(np.abs(op["e"][k]), axis=1)))))
            if h not in near_gate_parents and not np.array_equal(gm, om):
                r.fail(f"gate set ({h},{t}): gpu {list(gm)} oracle {list(om)}")
    r.checks["slots"] = n_slots
    for key, tol in (("mean_rel", REL_TOL), ("cov_rel", REL_TOL), ("p_abs", 1e-6),
                     ("dprob_abs", 2e-6), ("logC_abs", 5e-5), ("q_rel", 2e-5), ("e_rel", 2e-5)):
        if r.max_err.get(key, 0.0) > tol:
            r.fail(f"{key} {r.max_err[key]:.3g} > {tol}")
    # ---- a4/a5 children: status and weights, excusing close decisions
    oc, gch = d["o_children"], d["g_children"]
    margin = oc["margin"].copy()
    for h in near_gate_parents:
        margin[h * HU:(h + 1) * HU] = 0.0
    exc = margin <= DECISION_MARGIN
    r.excused["children"] = int(exc.sum())
    r.checks["children"] = len(margin)
    par_exc = exc.reshape(H, HU).any(axis=1)
    for j in np.nonzero((oc["status"] != gch["status"]) & ~exc)[0]:
        h = j // HU
        if par_exc[h] and {int(oc["status"][j]), int(gch["status"][j])} == {1, 2}:
            r.excused["dup_status"] = r.excused.get("dup_status", 0) + 1
            continue
        r.fail(f"child {j}: status gpu {gch['status'][j]} oracle {oc['status'][j]}")
        if len(r.failures) > 20:
            break
    both = (oc["status"] == 1) & (gch["status"] == 1) & ~exc
    if both.any():
        lo_ = oc["logw"][both]
        lg = gch["logw"][both]
        no = lo_ - np.logaddexp.reduce(lo_)
        ng = lg - np.logaddexp.reduce(lg)
        r.err("child_logw", np.max(np.abs(no - ng)))
        if r.max_err["child_logw"] > LOGW_TOL:
            r.fail(f"child log-weight {r.max_err['child_logw']:.3g} > {LOGW_TOL}")
    r.checks["unique_children"] = int(both.sum())
    # ---- a6/a7 retained set, by uid
    kidx, klw, lse = d["o_kept"]
    o_uid = d["o_state"][2]
    g_hyp = d["g_hyp"]
    g_uid = g_hyp["uid"]
    ol = oc["logw"] - lse                       # oracle normalised, all children
    kept_o = dict(zip(o_uid.tolist(), range(len(o_uid))))
    kept_g = dict(zip(g_uid.tolist(), range(len(g_uid))))
    all_uid = oc["uid"]
    uid_to_child = {int(u): j for j, u in enumerate(all_uid.tolist()) if oc["status"][j] == 1}
    boundary = np.min(ol[kidx]) if len(kidx) else 0.0
    log_tau = math.log(cfg["tau"])
    bwin = max(TIE_TOL, 2.0 * r.max_err.get("child_logw", LOGW_TOL))
    r.checks["boundary_window"] = bwin
    n_boundary = 0
    for u in set(kept_o) ^ set(kept_g):
        j = uid_to_child.get(u)
        if j is None:
            # a child unique only on the GPU: allowed only where decisions were excused
            jj = np.nonzero(all_uid == np.uint64(u))[0]
            if len(jj) and (exc[jj[0]] or par_exc[jj[0] // HU]):
                continue
            r.fail(f"retained uid {u:x} has no oracle counterpart")
            continue
        if exc[j]:
            continue
        if abs(ol[j] - boundary) <= bwin or abs(ol[j] - log_tau) <= bwin:
            n_boundary += 1
            continue
        r.fail(f"retained sets differ at child {j} (oracle normalised {ol[j]:.6f}, "
               f"boundary {boundary:.6f})")
    r.excused["boundary"] = n_boundary
    r.checks["retained"] = len(kept_g)
    # retained child indices: the same children in the same (parent, draw) order
    gidx, glw_ret = d["g_retained"]
    if not np.array_equal(glw_ret, g_hyp["logw"]):
        r.fail("retained log-weights differ from the hypothesis table")
    if len(gidx) != len(g_uid) or np.any(np.diff(gidx) <= 0):
        r.fail("retained child indices not strictly ascending")
    elif not np.array_equal(oc["uid"][gidx], g_uid):
        r.fail("retained child indices do not match the hypothesis uids")
    # ---- a8 theta, labels, tracks, weights of hypotheses kept on both sides
    o_tr = d["o_state"][3]
    g_tr = d["g_state"][3]
    o_lw = d["o_state"][1]
    g_lw = g_hyp["logw"]
    o_th = d["o_theta"]
    g_th = g_hyp["theta"]
    matched = 0
    common = [u for u in kept_o if u in kept_g and not exc[uid_to_child.get(u, 0)]]
    if common:
        # renormalisation over different sets shifts all weights by a constant
        off = np.median([o_lw[kept_o[u]] - g_lw[kept_g[u]] for u in common])
        exact_set = set(kept_o) == set(kept_g)
        for u in common:
            a, b = kept_o[u], kept_g[u]
            if not np.array_equal(o_th[a], g_th[b]):
                r.fail(f"theta differs for uid {u:x}")
                continue
            la = [tuple(rec[:2]) for rec in o_tr[a]]
            lb = [tuple(rec[:2]) for rec in g_tr[b]]
            if la != lb:
                r.fail(f"labels differ for uid {u:x}")
                continue
            for r1, r2 in zip(o_tr[a], g_tr[b]):
                r.err("track_mean_rel", _rel(r2[2], r1[2]))
                r.err("track_cov_rel", _rel(r2[3], r1[3]))
                if particle and part_ok:
                    r.err("particle_x_rel", _rel(r2[4], r1[4]))
                    r.err("particle_logw_abs", float(np.max(np.abs(r2[5] - r1[5]))))
            r.err("hyp_logw", abs(o_lw[a] - g_lw[b] - (0.0 if exact_set else off)))
            matched += 1
    r.checks["matched_hypotheses"] = matched
    for key, tol in (("track_mean_rel", REL_TOL), ("track_cov_rel", REL_TOL), ("hyp_logw", LOGW_TOL),
                     ("particle_x_rel", PARTICLE_TOL), ("particle_logw_abs", PARTICLE_TOL)):
        if r.max_err.get(key, 0.0) > tol:
            r.fail(f"{key} {r.max_err[key]:.3g} > {tol}")
    # ---- a9 estimates
    oe, ge = d["o_est"], d["g_est"]
    pm = np.sort(oe["pmf"])[::-1]
    if oe["n"] != ge["n"] and not (len(pm) > 1 and pm[0] - pm[1] < 1e-3):
        r.fail(f"MAP cardinality gpu {ge['n']} oracle {oe['n']}")
    if set(kept_o) == set(kept_g):
        r.err("pmf_abs", np.max(np.abs(oe["pmf"][:50] - ge["pmf"][:50])))
        r.err("ru_abs", np.max(np.abs(d["o_ru"] - d["g_ru"])) if len(d["o_ru"]) else 0.0)
        if oe["n"] == ge["n"] and list(map(tuple, oe["labels"])) == list(map(tuple, np.asarray(ge["labels"]).tolist())):
            r.err("r_abs", np.max(np.abs(oe["r"] - ge["r"])) if oe["n"] else 0.0)
            for m1, m2 in zip(oe["mean"], ge["mean"]):
                r.err("est_mean_rel", _rel(m2, m1))
        # weights carry the log-weight tolerance: |dw| <= w * LOGW_TOL
        for key, tol in (("pmf_abs", 2 * LOGW_TOL), ("ru_abs", 2 * LOGW_TOL),
                         ("r_abs", 2 * LOGW_TOL), ("est_mean_rel", REL_TOL)):
            if r.max_err.get(key, 0.0) > tol:
                r.fail(f"{key} {r.max_err[key]:.3g} > {tol}")
    return r


def ill_conditioned_case(shape):
    """Four tracks whose innovation covariance S = H P H^T + R has a pivot
    below 16 eps32 trace(S).  Every entry of P, R and S lies on the 2^-23
    grid, so S is the same in FP32 and FP64 (q = 0, zero mean velocities, a
    velocity variance of 2^-40 that FP32 rounds away next to the position
    block).  "diagonal": a sensor precise along y and tracks already precise
    there, S = diag(1 + 2r, 2r); "correlated": S with entries of full
    mantissa and det S ~ 2e-6, so that an FP32 factorisation rounds its
    pivot by a few per cent.  Detections are offset from the tracks along
    the small eigen-direction of S, by up to two of its standard
    deviations."""
    r = 2.0 ** -22
    g = lambda x: np.round(x * 2.0 ** 23) / 2.0 ** 23      # onto the 2^-23 grid
    if shape == "diagonal":
        R = np.diag([1.0, r])
        S = np.diag([1.0 + 2 * r, 2 * r])
    else:
        R = r * np.eye(2)
        s00, s11 = g(1.3), g(0.9)
        s01 = g(np.sqrt(s00 * s11 - 2e-6))
        S = np.array([[s00, s01], [s01, s11]])
    P = np.zeros((4, 4))
    P[:2, :2] = S - R
    P[2:, 2:] = 2.0 ** -40 * np.eye(2)
    lam, V = np.linalg.eigh(S)
    vs, ls = V[:, 0], lam[0]
    # clutter intensity of the order of the tracks' likelihoods (N(0; S) ~ 10^2
    # with det S ~ 10^-6), so that rows go to clutter or to their track and
    # children differ; the fourth track has no detection (it may die)
    cfg = dict(dim_x=4, dim_z=2, dt=1.0, q=0.0, R=R.tolist(), p_s=0.99, p_d=0.9, lambda_d=0.5,
               clutter_rate=50.0, volume=1.0, gate=18.420680743952367, h_max=100, h_up=200,
               tau=1e-9, seed=777, score_mode=0, max_tracks=16, max_meas=32, max_births=4)
    means = [np.array([10.0, 20.0, 0.0, 0.0]), np.array([40.0, 25.0, 0.0, 0.0]),
             np.array([70.0, 60.0, 0.0, 0.0]), np.array([20.0, 80.0, 0.0, 0.0])]
    tracks = [[(3, j, m, P.copy()) for j, m in enumerate(means)]]
    offs = [[0.7], [-1.3, 0.4], [1.8], []]
    Z = np.array([m[:2] + a * np.sqrt(ls) * vs for m, o in zip(means, offs) for a in o] + [[55.0, 5.0]],
                 np.float32)
    return cfg, (4, np.array([0.0]), np.array([12345], np.uint64), tracks), Z, S
