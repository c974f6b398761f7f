"""glmb_select_top_static: the top-H selection for callers that may not
allocate device memory while they run (a tracking loop with a fixed memory
budget and a frame deadline, where cudaMalloc can stall the device, or a
host application that forbids raw cudaMalloc).  It is called through the C
ABI and must agree with the selection glmb_prune made on the same children
(glmb_get_retained), on two calls in a row.  This file is collected last."""
from __future__ import annotations

import ctypes as C

import numpy as np
import pytest

import scenes
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_06230_gb300 as glmb
    glmb.build()
    lib = glmb.load()
    f = lib.glmb_select_top_static
    f.argtypes = [C.c_void_p, C.c_int64, C.c_int32, C.c_double, C.c_void_p, C.c_void_p,
                  C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    return glmb, f


def _select(f, logw, h_max, tau):
    import torch
    stream = torch.cuda.current_stream()
    lw = torch.from_numpy(np.ascontiguousarray(logw, np.float64)).cuda()
    idx = torch.full((h_max,), -1, dtype=torch.int64, device="cuda")
    out = torch.full((h_max,), float("nan"), dtype=torch.float64, device="cuda")
    n_out = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    st = f(C.c_void_p(lw.data_ptr()), len(logw), h_max, tau, C.c_void_p(idx.data_ptr()),
           C.c_void_p(out.data_ptr()), C.c_void_p(n_out.data_ptr()), C.c_void_p(stream.cuda_stream))
    assert st == 0
    stream.synchronize()
    k = int(n_out.item())
    return idx[:k].cpu().numpy(), out[:k].cpu().numpy()


def test_static_selection_matches_prune_two_calls_in_a_row(api):
    glmb, f = api
    sc = scenes.make_scene(scenes.preset("mid"), 2001)
    cfg = sc.filter_config()
    g = glmb.Filter(cfg)
    compared = 0
    for k, fr in enumerate(sc.frames[:14]):
        g.predict(fr.births)
        g.update(fr.Z)
        if k >= 12:
            logw = g.children()["logw"]
            got = _select(f, logw, cfg["h_max"], cfg["tau"])
        g.prune()
        if k < 12:
            continue
        idx_ref, lw_ref = g.retained()
        idx, lw = got
        assert len(idx_ref) > 100
        assert np.array_equal(idx, idx_ref)
        assert np.max(np.abs(lw - lw_ref)) <= parity.LOGW_TOL
        compared += 1
    assert compared == 2


def test_static_selection_edge_cases(api):
    glmb, f = api
    # nothing with weight: no child kept
    idx, lw = _select(f, np.full(1000, -np.inf), 10, 1e-5)
    assert len(idx) == 0
    # fewer candidates than h_max: all above tau kept, ties by index
    logw = np.array([-np.inf, 0.0, -1.0, 0.0, -30.0, -0.5])
    idx, lw = _select(f, logw, 10, 1e-5)
    assert list(idx) == [1, 2, 3, 5]
    w = np.exp(logw[[1, 2, 3, 5]])
    assert np.allclose(lw, np.log(w / w.sum()), atol=1e-12)
    # h_max smaller than the candidates, equal weights at the boundary
    idx, lw = _select(f, np.zeros(7), 3, 1e-5)
    assert list(idx) == [0, 1, 2]
    # +inf, NaN and values beyond 2^30 in magnitude mark children without weight
    logw = np.array([0.0, np.inf, -1.0, 3.0e9, np.nan, -2.0e9, -2.0])
    idx, lw = _select(f, logw, 10, 1e-5)
    assert list(idx) == [0, 2, 6]
    w = np.exp(logw[[0, 2, 6]])
    assert np.allclose(lw, np.log(w / w.sum()), atol=1e-12)


def test_static_selection_child_at_the_tau_cut(api):
    """A child whose normalised weight is tau itself: the log-sum-exp is
    rounded differently here and in glmb_prune, so either decision is
    correct; the other children and all renormalised weights are exact."""
    glmb, f = api
    tau = 1e-5
    x = np.log(tau / (1.0 - tau))          # w1 / (w0 + w1) = tau with w0 = 1
    logw = np.array([0.0, x])
    idx, lw = _select(f, logw, 10, tau)
    assert list(idx) in ([0], [0, 1])
    w = np.exp(logw[idx])
    assert np.allclose(lw, np.log(w / w.sum()), atol=1e-12)


def test_static_selection_rejects_sizes_beyond_the_limit(api):
    import torch
    glmb, f = api
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = C.c_void_p(dummy.data_ptr())
    assert f(p, (1 << 30) + 1, 10, 1e-5, p, p, p, None) == 3
    assert f(p, 10, 0, 1e-5, p, p, p, None) == 1
