"""Shared test helpers: tiny hand-made scenarios and independent textbook
formulas used to pin the oracle.  Nothing here calls the CUDA library."""
from __future__ import annotations

import numpy as np
from scipy.integrate import quad_vec
from scipy.linalg import expm


def base_cfg(dim=2, **kw):
    cfg = dict(dim_x=2 * dim, dim_z=dim, dt=1.0, q=1.0, R=(4.0 * np.eye(dim)).tolist(),
               p_s=0.95, p_d=0.8, lambda_d=0.7, clutter_rate=2.0, volume=1.0e4,
               gate=float("inf"), h_max=50, h_up=200, tau=1e-9, seed=12345, score_mode=0)
    cfg.update(kw)
    return cfg


def cv_continuous(dim, dt, q):
    """F = expm(A dt) and Q = int_0^dt e^{As} G q G^T e^{A^T s} ds for the
    white-acceleration model x' = A x + G w, computed numerically."""
    A = np.zeros((2 * dim, 2 * dim))
    A[:dim, dim:] = np.eye(dim)
    G = np.zeros((2 * dim, dim))
    G[dim:, :] = np.eye(dim)
    F = expm(A * dt)
    Q, _ = quad_vec(lambda s: expm(A * s) @ G @ G.T @ expm(A * s).T * q, 0.0, dt,
                    epsabs=1e-13, epsrel=1e-13)
    return F, Q


def spd(rng, n, scale=1.0, floor=0.5):
    A = rng.normal(size=(n, n))
    return scale * (A @ A.T / n + floor * np.eye(n))


def kf_update_info(m, P, z, R):
    """Posterior of N(m, P) after one detection z ~ N(Hx, R), information form."""
    dz = len(z)
    H = np.zeros((dz, len(m)))
    H[:, :dz] = np.eye(dz)
    Pi = np.linalg.inv(P)
    Ri = np.linalg.inv(R)
    Pn = np.linalg.inv(Pi + H.T @ Ri @ H)
    mn = Pn @ (Pi @ m + H.T @ Ri @ z)
    return mn, Pn


def kf_sequential(m, P, Zs, R):
    for z in Zs:
        m, P = kf_update_info(m, P, np.asarray(z, float), R)
    return m, P


def state_tracks(rng, dim, n, spread=20.0, frame=3):
    dx = 2 * dim
    out = []
    for j in range(n):
        mean = np.concatenate([rng.uniform(0, spread, dim), rng.normal(size=dim)])
        P = spd(rng, dx, scale=3.0)
        out.append((frame - 1, j, mean, P))
    return out
