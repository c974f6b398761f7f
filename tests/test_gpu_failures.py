"""Failure detection without a GPU fault: a device allocation that fails
during glmb_create (the allocation hook of glmb_config returns NULL on its
Nth call) must give GLMB_E_OOM and return every block the handle had
taken; the filter created afterwards with a working allocator runs."""
from __future__ import annotations

import pytest

import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def glmb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_06230_gb300 as g
    g.build()
    g.load()
    return g


class CountingAllocator:
    """Device memory from torch's caching allocator; the fail_at-th call
    (1-based) returns None, as a failed cudaMalloc would."""

    def __init__(self, fail_at=None):
        self.fail_at = fail_at
        self.calls = 0
        self.live = {}

    def alloc(self, nbytes):
        import torch
        self.calls += 1
        if self.fail_at is not None and self.calls == self.fail_at:
            return None
        p = torch.cuda.caching_allocator_alloc(nbytes)
        self.live[p] = nbytes
        return p

    def free(self, p):
        import torch
        assert p in self.live, "freed a block the allocator never gave"
        del self.live[p]
        torch.cuda.caching_allocator_delete(p)


def test_allocation_failure_in_create_is_reported_and_cleaned_up(glmb):
    sc = scenes.make_scene(scenes.preset("tiny"), 1001)
    cfg = sc.filter_config()
    ok = CountingAllocator()
    f = glmb.Filter(cfg, allocator=(ok.alloc, ok.free))
    n_allocs = ok.calls
    assert n_allocs > 20 and len(ok.live) == n_allocs
    for fr in sc.frames[:3]:
        f.step(fr.births, fr.Z)
    f.close()
    assert not ok.live                       # destroy returned every block
    for k in sorted({1, 2, n_allocs // 2, n_allocs - 1, n_allocs}):
        bad = CountingAllocator(fail_at=k)
        with pytest.raises(glmb.GlmbError) as ei:
            glmb.Filter(cfg, allocator=(bad.alloc, bad.free))
        assert ei.value.status == 2          # GLMB_E_OOM
        assert bad.calls == k                # nothing allocated after the failure
        assert not bad.live                  # every block taken before it was freed
    g2 = glmb.Filter(cfg)
    g2.step(sc.frames[0].births, sc.frames[0].Z)
    assert g2.info()["n_hyp"] >= 1
    g2.close()


def _wide_state(n_hyp=2000, per_hyp=9, extent=1000.0, seed=5):
    """A GLMB of n_hyp equally weighted hypotheses holding per_hyp tracks
    each, every track its own label: n_hyp * per_hyp distinct components
    (more than 16384), so the frame's pair-count scan runs in several tiles
    with look-back waits while every hypothesis stays small."""
    import numpy as np
    rng = np.random.default_rng(seed)
    logw = np.full(n_hyp, -np.log(n_hyp))
    uid = np.arange(1, n_hyp + 1, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15)
    tracks = []
    for h in range(n_hyp):
        tr = []
        for j in range(per_hyp):
            m = np.concatenate([rng.uniform(0, extent, 2), rng.normal(size=2)])
            tr.append((2, h * per_hyp + j, m, np.diag([25.0, 25.0, 4.0, 4.0])))
        tracks.append(tr)
    return 3, logw, uid, tracks


def _run_to(f, sc, k):
    for fr in sc.frames[:k]:
        f.predict(fr.births)
        f.update(fr.Z)
        f.prune()


def test_scan_wait_that_runs_out_fails_the_frame_and_keeps_the_state(glmb):
    """A scan tile whose predecessor never publishes its prefix gives up
    after its limit: the frame fails with GLMB_E_TIMEOUT, the state is the
    previous frame's, and with the normal limits the same frame then gives
    the result of a filter that never failed."""
    sc = scenes.make_scene(scenes.preset("tiny"), 1001)
    cfg = sc.filter_config(h_max=2000, h_up=10, max_tracks=64, max_components=60000)
    state = glmb.pack_state(*_wide_state(), 4)
    f, ref = glmb.Filter(cfg), glmb.Filter(cfg)
    f.import_state(state)
    ref.import_state(state)
    before = f.export_state()
    fr = sc.frames[3]
    try:
        glmb.set_wait_test(glmb.WAIT_TEST_SCAN, 1 << 12)
        with pytest.raises(glmb.GlmbError) as ei:
            f.predict(fr.births)
            f.update(fr.Z)
            f.prune()
        assert ei.value.status == 7          # GLMB_E_TIMEOUT
    finally:
        glmb.set_wait_test(glmb.WAIT_TEST_OFF)
    assert f.export_state() == before
    for g in (f, ref):
        g.predict(fr.births)
        g.update(fr.Z)
        g.prune()
        assert g.info()["n_components"] > 0
    assert f.export_state() == ref.export_state()
    f.close()
    ref.close()


def test_gate_wait_that_runs_out_fails_the_frame_and_keeps_the_state(glmb):
    """The learned gate's tensor-core completion wait gives up after its
    limit (CTA 0 issued no work): the frame fails with GLMB_E_TIMEOUT, the
    CTA returns its tensor memory, the state is the previous frame's, and
    the next attempt with the normal limits succeeds."""
    from paper_2512_06230_gb300 import gate as G
    import numpy as np
    sc = scenes.make_scene(scenes.preset("tiny"), 1001)
    cfg = sc.filter_config()
    params = G.init_params(3, np.zeros(5, np.float32), np.ones(5, np.float32))
    f = glmb.Filter(cfg)
    f.set_gate(params, -1e30, glmb.Filter.GATE_PRUNE)
    _run_to(f, sc, 5)
    before = f.export_state()
    fr = sc.frames[5]
    try:
        glmb.set_wait_test(glmb.WAIT_TEST_GATE, 20000)
        with pytest.raises(glmb.GlmbError) as ei:
            f.predict(fr.births)
            f.update(fr.Z)
            f.prune()
        assert ei.value.status == 7          # GLMB_E_TIMEOUT
    finally:
        glmb.set_wait_test(glmb.WAIT_TEST_OFF)
    assert f.export_state() == before
    f.predict(fr.births)
    f.update(fr.Z)
    f.prune()
    assert f.info()["n_hyp"] >= 1
    f.close()


def test_wait_test_arguments_are_checked(glmb):
    with pytest.raises(glmb.GlmbError):
        glmb.set_wait_test(9, 10)
    with pytest.raises(glmb.GlmbError):
        glmb.set_wait_test(glmb.WAIT_TEST_SCAN, 0)
    glmb.set_wait_test(glmb.WAIT_TEST_OFF)


def test_device_detections_must_be_device_memory(glmb):
    """Detections passed as device memory are read by the kernels with
    global-memory loads: a host address (pageable or pinned) or a misaligned
    one is refused by the call before any kernel runs, through the C ABI
    itself (a caller other than the Python binding gets the same check)."""
    import ctypes as C
    import numpy as np
    import torch
    sc = scenes.make_scene(scenes.preset("tiny"), 1001)
    f = glmb.Filter(sc.filter_config())
    fr = sc.frames[0]
    host = np.ascontiguousarray(fr.Z, np.float32)
    pinned = torch.from_numpy(host).pin_memory()
    dev = torch.from_numpy(host).cuda()
    M = len(host)
    for ptr in (host.ctypes.data, pinned.data_ptr(), dev.data_ptr() + 2):
        f.predict(fr.births)
        st = f.lib.glmb_update(f.h, C.c_void_p(ptr), M, 1)
        assert st == 1                       # GLMB_E_INVALID, nothing launched
        assert f.lib.glmb_prune(f.h) == 6    # GLMB_E_STATE: the update did not happen
    f.predict(fr.births)
    assert f.lib.glmb_update(f.h, C.c_void_p(dev.data_ptr()), M, 1) == 0
    assert f.lib.glmb_prune(f.h) == 0
    f.close()


def test_update_table_overflow_fails_the_frame_and_the_next_frames_are_exact(glmb):
    """A frame whose distinct track updates exceed the component capacity
    fails with GLMB_E_CAPACITY and leaves the state as it was.  The update
    hash table is cleared frame to frame only where the last frame filled
    it; after an overflow (updates that found no room are not on that list)
    the whole table is cleared, so the frames that follow equal those of a
    filter that never saw the failing frame."""
    import numpy as np
    sc = scenes.make_scene(scenes.preset("tiny"), 1001)
    big = sc.filter_config(max_components=20000, max_meas=1024)
    k_spike, k_end = 12, 18
    fr = sc.frames[k_spike]
    rng = np.random.default_rng(3)
    # seven more detections about every detection of the frame, ~28 m out
    # (near the gate's edge, where a track and clutter are about equally
    # likely), so the hypotheses take many distinct detection sets and the
    # frame's updates spike (the FP64 oracle on this frame: 109 distinct
    # tracks after it against at most 55 after any earlier frame)
    extra = []
    for _ in range(7):
        ang = rng.uniform(0.0, 2.0 * np.pi, len(fr.Z))
        extra.append(fr.Z + 28.0 * np.stack([np.cos(ang), np.sin(ang)], axis=1) + rng.normal(0.0, 1.0, fr.Z.shape))
    Zs = np.concatenate([fr.Z] + extra).astype(np.float32)
    ref = glmb.Filter(big)
    need = 0
    for k in range(k_spike):
        ref.step(sc.frames[k].births, sc.frames[k].Z)
        need = max(need, ref.info()["n_components"] + len(sc.frames[k + 1].births))
    probe = glmb.Filter(big)
    probe.import_state(ref.export_state())
    probe.step(fr.births, Zs)
    spike_updates = probe.info()["n_updates"]
    probe.close()
    for k in range(k_spike + 1, k_end):
        ref.step(sc.frames[k].births, sc.frames[k].Z)
        need = max(need, ref.info()["n_components"] + len(sc.frames[k + 1].births))
    ref.close()
    cap = need
    assert spike_updates > cap, (spike_updates, cap)
    a = glmb.Filter(sc.filter_config(max_components=cap, max_meas=1024))
    b = glmb.Filter(big)
    for k in range(k_spike):
        a.step(sc.frames[k].births, sc.frames[k].Z)
        b.step(sc.frames[k].births, sc.frames[k].Z)
    before = a.export_state()
    with pytest.raises(glmb.GlmbError) as ei:
        a.step(fr.births, Zs)
    assert ei.value.status == 3              # GLMB_E_CAPACITY
    assert "distinct track updates exceed capacity" in str(ei.value), str(ei.value)
    assert a.export_state() == before
    for k in range(k_spike + 1, k_end):
        a.step(sc.frames[k].births, sc.frames[k].Z)
        b.step(sc.frames[k].births, sc.frames[k].Z)
        ia, la = a.retained()
        ib, lb = b.retained()
        assert np.array_equal(ia, ib) and np.array_equal(la, lb), k
        ea, eb = a.estimates(), b.estimates()
        assert ea["n"] == eb["n"] and np.array_equal(ea["mean"], eb["mean"]), k
    a.close()
    b.close()
