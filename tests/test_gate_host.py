"""Host logic of the learned gate's training pipeline (CPU only): the
parameter vector's layout and initialisation, and the feature
standardisation that the vector carries."""
from __future__ import annotations

import numpy as np

from oracle import gate_mlp as gm
from paper_2512_06230_gb300 import gate


def test_init_params_layout_and_scale():
    mu = np.array([1.0, 2.0, 0.5, 10.0, 3.0])
    sd = np.array([0.5, 1.5, 0.2, 4.0, 1.0])
    p = gate.init_params(7, mu, sd)
    assert p.dtype == np.float32 and p.size == gm.NPARAM
    w = {k: p[gm.OFF[k]:gm.OFF[k] + int(np.prod(gm.SHAPES[k]))] for k in gm.OFF}
    for b in ("b1", "b2", "b3", "b4"):
        assert not w[b].any()
    np.testing.assert_allclose(w["mu"], mu, rtol=1e-7)
    np.testing.assert_allclose(w["sd"], sd, rtol=1e-7)
    # He-normal: the sample deviation of each matrix near sqrt(2 / fan_in)
    for k, fan_in in (("W2", 64), ("W3", 64)):
        assert abs(w[k].std() / np.sqrt(2.0 / fan_in) - 1) < 0.05
    assert abs(w["w4"].std() / np.sqrt(1.0 / 64) - 1) < 0.3
    # the same seed gives the same vector
    np.testing.assert_array_equal(p, gate.init_params(7, mu, sd))


def test_standardisation_floors_constant_features():
    rng = np.random.default_rng(3)
    X = np.stack([rng.normal(5, 2, 1000), np.full(1000, 4.0), rng.uniform(0, 1, 1000),
                  rng.integers(0, 3, 1000).astype(float), rng.normal(0, 1e-9, 1000)], 1)
    mu, sd = gate.standardisation(X)
    np.testing.assert_allclose(mu, X.mean(0))
    assert sd[1] == 1.0 and sd[4] == 1.0          # constant or near-constant: no division blow-up
    np.testing.assert_allclose(sd[[0, 2, 3]], X.std(0)[[0, 2, 3]])
