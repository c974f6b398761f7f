"""Tracking accuracy against the scene's ground truth (Section 4.2).

* relative cardinality error: |N_true - N_est| / N_true at one time step,
  averaged over the steps of a run;
* tracking error: the minimum-total-distance matching (Hungarian
  algorithm) between estimated and true positions at one time step, the
  mean distance of the matched pairs, averaged over the steps of a run.

Evaluation only: neither the filter nor the oracle uses this module."""
from __future__ import annotations

import numpy as np


def matched_distance(est_pos: np.ndarray, true_pos: np.ndarray) -> float:
    """Mean distance of the optimal matching of the two point sets (NaN when
    either set is empty)."""
    from scipy.optimize import linear_sum_assignment
    if len(est_pos) == 0 or len(true_pos) == 0:
        return float("nan")
    est_pos = np.asarray(est_pos, float).reshape(len(est_pos), -1)
    true_pos = np.asarray(true_pos, float).reshape(len(true_pos), -1)
    d = np.linalg.norm(est_pos[:, None, :] - true_pos[None, :, :], axis=2)
    i, j = linear_sum_assignment(d)
    return float(d[i, j].mean())


class RunAccuracy:
    """Accumulates the two per-step errors over one run."""

    def __init__(self):
        self.card = []
        self.dist = []

    def add(self, est_pos: np.ndarray, true_pos: np.ndarray):
        n_true, n_est = len(true_pos), len(est_pos)
        if n_true > 0:
            self.card.append(abs(n_true - n_est) / n_true)
        d = matched_distance(est_pos, true_pos)
        if not np.isnan(d):
            self.dist.append(d)

    def summary(self) -> dict:
        return dict(rel_card_error=float(np.mean(self.card)) if self.card else float("nan"),
                    tracking_error_m=float(np.mean(self.dist)) if self.dist else float("nan"),
                    steps=len(self.card))


def ospa(est_pos: np.ndarray, true_pos: np.ndarray, c: float = 100.0, p: float = 1.0) -> float:
    """OSPA distance of order p with cut-off c (Schuhmacher, Vo and Vo,
    "A consistent metric for performance evaluation of multi-object
    filters", IEEE TSP 2008): the minimum over assignments of the smaller
    set into the larger of the mean p-th power of min(c, distance), with c^p
    for each unassigned element of the larger set, all to the power 1/p."""
    from scipy.optimize import linear_sum_assignment
    m, n = len(est_pos), len(true_pos)
    if m == 0 and n == 0:
        return 0.0
    if m == 0 or n == 0:
        return float(c)
    X = np.asarray(est_pos, float).reshape(m, -1)
    Y = np.asarray(true_pos, float).reshape(n, -1)
    if m > n:
        X, Y, m, n = Y, X, n, m
    D = np.minimum(np.linalg.norm(X[:, None, :] - Y[None, :, :], axis=2), c) ** p
    i, j = linear_sum_assignment(D)
    return float(((D[i, j].sum() + (c ** p) * (n - m)) / n) ** (1.0 / p))
