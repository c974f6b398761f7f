"""FP64 reference of the learned gate's MLP: forward pass, weighted
binary cross-entropy, backward pass and one Adam step.

TEST INFRASTRUCTURE ONLY: the tests and the smoke check call it; the
library never does.  It shares no code with the CUDA path.

The gate is an extension beyond the paper (whose gate g_ijk of Section 3 is
a plain threshold on the compatibility entry): a 5-64-64-64-1 multilayer
perceptron with GELU activations scores every pair that passes the
Mahalanobis test, and the pair enters the compatibility table only when its
logit reaches a threshold.

Parameter vector (float32, NPARAM values):
    W1[64][5] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] w4[64] b4 mu[5] sd[5]
The first NTRAIN values are trained; mu and sd standardise the raw
features, x = (f - mu) / sd.  The matrices W1, W2, W3 and w4 are used
rounded to bf16 (round to nearest, ties to even); biases are used as given.

Features of a pair (slot with predicted existence p, label (k, b); detection
with innovation e):
    d^2 (Mahalanobis), |e| (Euclidean), p, age = frame - k, log det S.

Loss over a batch: L = sum_m wt_m * (softplus(z_m) - y_m * z_m), z the
logit, y in {0, 1} (pair used by a retained hypothesis or not).  Gradients
are taken with respect to the bf16-rounded weights and reported for the
float32 master values (rounding passed straight through).

Adam (Kingma and Ba, "Adam: A Method for Stochastic Optimization", 2015,
Algorithm 1) with bias-corrected moments.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

NPARAM = 8779
NTRAIN = 8769
H = 64
NF = 5
OFF = dict(W1=0, b1=320, W2=384, b2=4480, W3=4544, b3=8640, w4=8704, b4=8768, mu=8769, sd=8774)
SHAPES = dict(W1=(H, NF), b1=(H,), W2=(H, H), b2=(H,), W3=(H, H), b3=(H,), w4=(H,), b4=(1,),
              mu=(NF,), sd=(NF,))
MATRICES = ("W1", "W2", "W3", "w4")


def bf16(x) -> np.ndarray:
    """Round to the nearest bf16 value (ties to even) through float32."""
    f = np.ascontiguousarray(np.asarray(x, np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    finite = (u & 0x7F800000) != 0x7F800000
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    u = np.where(finite, r, u).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


def unpack(p) -> dict:
    """Named float64 views of a parameter vector, matrices rounded to bf16."""
    p = np.asarray(p, np.float32).reshape(-1)
    assert p.size == NPARAM
    out = {}
    for k, off in OFF.items():
        n = int(np.prod(SHAPES[k]))
        v = p[off:off + n].astype(np.float64).reshape(SHAPES[k])
        out[k] = bf16(v) if k in MATRICES else v
    return out


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    """d/dx x Phi(x) = Phi(x) + x phi(x)."""
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def forward(p, X, round_act: bool = False):
    """Logits of the raw feature rows X (n x 5) and the intermediate values.
    round_act rounds the standardised features and the hidden activations
    to bf16, as the library's kernels feed them to the tensor cores."""
    w = unpack(p)
    r = bf16 if round_act else (lambda a: a)
    x = r((np.asarray(X, np.float64) - w["mu"]) / w["sd"])
    z1 = x @ w["W1"].T + w["b1"]
    h1 = r(gelu(z1))
    z2 = h1 @ w["W2"].T + w["b2"]
    h2 = r(gelu(z2))
    z3 = h2 @ w["W3"].T + w["b3"]
    h3 = r(gelu(z3))
    z = h3 @ w["w4"] + w["b4"][0]
    return z, dict(w=w, x=x, z1=z1, h1=h1, z2=z2, h2=h2, z3=z3, h3=h3)


def softplus(z):
    return np.maximum(z, 0.0) + np.log1p(np.exp(-np.abs(z)))


def sigmoid(z):
    return 0.5 * (1.0 + np.tanh(0.5 * z))


def loss(p, X, y, wt) -> float:
    z, _ = forward(p, X)
    return float(np.sum(np.asarray(wt, np.float64) * (softplus(z) - np.asarray(y, np.float64) * z)))


def loss_and_grad(p, X, y, wt):
    """Loss and its gradient (NPARAM values, zero for mu and sd)."""
    z, c = forward(p, X)
    w = c["w"]
    y = np.asarray(y, np.float64)
    wt = np.asarray(wt, np.float64)
    L = float(np.sum(wt * (softplus(z) - y * z)))
    dz = wt * (sigmoid(z) - y)
    g = {"w4": c["h3"].T @ dz, "b4": np.array([dz.sum()])}
    dz3 = np.outer(dz, w["w4"]) * gelu_grad(c["z3"])
    g["W3"] = dz3.T @ c["h2"]
    g["b3"] = dz3.sum(0)
    dz2 = (dz3 @ w["W3"]) * gelu_grad(c["z2"])
    g["W2"] = dz2.T @ c["h1"]
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ w["W2"]) * gelu_grad(c["z1"])
    g["W1"] = dz1.T @ c["x"]
    g["b1"] = dz1.sum(0)
    grad = np.zeros(NPARAM)
    for k, v in g.items():
        grad[OFF[k]:OFF[k] + v.size] = np.ravel(v)
    return L, grad


def adam_step(p, g, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update of the trained entries (t counts from 1); returns new
    (p, m, v) in float64."""
    p = np.asarray(p, np.float64).copy()
    m = np.asarray(m, np.float64).copy()
    v = np.asarray(v, np.float64).copy()
    g = np.asarray(g, np.float64)
    s = slice(0, NTRAIN)
    m[s] = b1 * m[s] + (1.0 - b1) * g[s]
    v[s] = b2 * v[s] + (1.0 - b2) * g[s] * g[s]
    mh = m[s] / (1.0 - b1 ** t)
    vh = v[s] / (1.0 - b2 ** t)
    p[s] -= lr * mh / (np.sqrt(vh) + eps)
    return p, m, v
