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
    est_pos = np.asarray(est_pos, float).reshape(len(est_pos), -1)
    true_pos = np.asarray(true_pos, float).reshape(len(true_pos), -1)
    if len(est_pos) == 0 or len(true_pos) == 0:
        return float("nan")
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
