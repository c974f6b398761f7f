"""Training of the learned pair gate, an extension beyond the paper's fixed
gate g_ijk (Section 3): a 5-64-64-64-1 GELU MLP scoring each pair of the
compatibility table (Eq. 2) that passes the Mahalanobis test.

collect          features and usage labels of every pair of every frame of
                 a scene, from the filter run without the gate (the library
                 computes both: glmb_gate_features, glmb_gate_usage)
standardisation  mu and sd of the training features
train            weighted binary cross-entropy, Adam; the forward and
                 backward passes and the update are the library's kernels
                 (glmb_mlp_backward, glmb_mlp_adam); mini-batches are drawn
                 on the device
threshold        the largest threshold that keeps a given fraction of the
                 used pairs of a data set

Classes are balanced in the loss (used pairs are a minority): each batch
weighs its used and its unused pairs 1/2 in total each.
"""
from __future__ import annotations

from typing import Iterable, List, Tuple

import numpy as np

from . import GATE_NPARAM, GATE_NTRAIN, Filter, mlp_adam, mlp_backward, mlp_forward

OFF_MU, OFF_SD = 8769, 8774


def init_params(seed: int, mu, sd) -> np.ndarray:
    """He-normal matrices, zero biases, the given standardisation."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, n_out in ((5, 64), (64, 64), (64, 64)):
        parts += [rng.normal(scale=np.sqrt(2.0 / fan_in), size=n_out * fan_in), np.zeros(n_out)]
    parts += [rng.normal(scale=np.sqrt(1.0 / 64), size=64), np.zeros(1), np.asarray(mu, float),
              np.asarray(sd, float)]
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == GATE_NPARAM
    return p


def collect(cfg: dict, frames: Iterable[Tuple[list, np.ndarray]], skip: int = 0) -> Tuple[np.ndarray, np.ndarray]:
    """Runs the ungated filter over (births, Z) frames and returns the
    features (n x 5 float32) and usage labels (n uint8) of the pairs of every
    frame after the first `skip`."""
    f = Filter(cfg)
    Xs: List[np.ndarray] = []
    ys: List[np.ndarray] = []
    try:
        for k, (births, Z) in enumerate(frames):
            f.step(births, Z)
            if k < skip:
                continue
            X = f.gate_features()
            used, _ = f.gate_usage()
            Xs.append(X)
            ys.append(used)
    finally:
        f.close()
    if not Xs:
        return np.zeros((0, 5), np.float32), np.zeros(0, np.uint8)
    return np.concatenate(Xs), np.concatenate(ys)


def standardisation(X: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    mu = X.mean(axis=0).astype(np.float64)
    sd = X.std(axis=0).astype(np.float64)
    return mu, np.where(sd > 1e-6, sd, 1.0)


def train(X: np.ndarray, y: np.ndarray, steps: int = 2000, batch: int = 32768, lr: float = 2e-3,
          seed: int = 0, device: str = "cuda", log_every: int = 0):
    """Trains on (X, y); returns (params float32, loss history)."""
    import torch
    mu, sd = standardisation(X)
    P = torch.from_numpy(init_params(seed, mu, sd)).to(device)
    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).to(device)
    yd = torch.from_numpy(np.ascontiguousarray(y, np.float32)).to(device)
    m = torch.zeros(GATE_NTRAIN, device=device)
    v = torch.zeros(GATE_NTRAIN, device=device)
    grad = torch.zeros(GATE_NPARAM, device=device)
    loss = torch.zeros(1, dtype=torch.float64, device=device)
    err = torch.zeros(1, dtype=torch.int32, device=device)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    n = Xd.shape[0]
    hist = []
    for t in range(1, steps + 1):
        idx = torch.randint(0, n, (min(batch, n),), device=device, generator=gen)
        xb, yb = Xd[idx].contiguous(), yd[idx].contiguous()
        npos = yb.sum().clamp(min=1.0)
        nneg = (yb.numel() - yb.sum()).clamp(min=1.0)
        wb = torch.where(yb > 0.5, 0.5 / npos, 0.5 / nneg).contiguous()
        mlp_backward(P, xb, yb, wb, grad, loss, err)
        mlp_adam(P, grad, m, v, t, lr)
        if log_every and (t % log_every == 0 or t == 1):
            hist.append((t, float(loss.item())))
    if int(err.item()) != 0:
        raise RuntimeError("learned gate: a tensor-core wait ran out of time during training")
    return P.cpu().numpy(), hist


def logits(params: np.ndarray, X: np.ndarray, device: str = "cuda") -> np.ndarray:
    import torch
    err = torch.zeros(1, dtype=torch.int32, device=device)
    z = mlp_forward(torch.from_numpy(params).to(device),
                    torch.from_numpy(np.ascontiguousarray(X, np.float32)).to(device), err)
    out = z.cpu().numpy()
    if int(err.item()) != 0:
        raise RuntimeError("learned gate: a tensor-core wait ran out of time")
    return out


def threshold(params: np.ndarray, X: np.ndarray, y: np.ndarray, keep_used: float = 0.999,
              device: str = "cuda") -> float:
    """The largest threshold that keeps at least keep_used of the used pairs."""
    z = logits(params, X, device)
    zp = np.sort(z[y > 0])
    if len(zp) == 0:
        return float(np.min(z)) if len(z) else 0.0
    k = int(np.floor((1.0 - keep_used) * len(zp)))
    return float(np.nextafter(np.float32(zp[k]), np.float32(-np.inf)))
