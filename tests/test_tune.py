"""Host logic of the launch-shape autotuner, with a stand-in filter and a
fake clock (CPU only): every candidate of the space is applied to a fresh
filter, timed on a second pass after a reset that follows an untimed pass,
the filter is closed, and the fastest candidate is returned."""
from __future__ import annotations

from paper_2512_06230_gb300 import tune


class _Clock:
    t = 0.0


class _FakeFilter:
    log = []

    def __init__(self, cfg):
        self.cfg = cfg
        self.tuning = None
        self.passes = 0
        self.steps = 0
        self.closed = False
        _FakeFilter.log.append(self)

    def set_tuning(self, **kw):
        self.tuning = kw

    def step(self, births, Z, device=False):
        # cost per frame: lowest at thread_warps_per_sm = 4, stage_threads = 256
        t = self.tuning
        _Clock.t += 1.0 + abs(t["thread_warps_per_sm"] - 4) + (t["stage_threads"] != 256) * 0.5
        self.steps += 1

    def estimates(self, cap, pmf_cap):
        return {}

    def reset(self):
        self.passes += 1

    def close(self):
        self.closed = True


def test_autotune_picks_the_fastest_candidate(monkeypatch):
    monkeypatch.setattr(tune.time, "perf_counter", lambda: _Clock.t)
    _FakeFilter.log.clear()
    space = {"thread_warps_per_sm": (1, 4, 8), "draw_threads": (0,), "warp_cta_warps": (16,),
             "stage_threads": (128, 256)}
    frames = [(None, None)] * 5
    best, res = tune.autotune({"max_tracks": 8}, frames, space=space, make_filter=_FakeFilter)
    assert best == {"thread_warps_per_sm": 4, "draw_threads": 0, "warp_cta_warps": 16, "stage_threads": 256}
    assert len(res) == len(tune.candidates(space)) == 6
    assert [r[0] for r in res] == tune.candidates(space)
    for f in _FakeFilter.log:
        assert f.closed and f.passes == 1 and f.steps == 2 * len(frames)
    # the timed pass alone: 5 frames at the candidate's cost
    assert dict((tuple(sorted(c.items())), s) for c, s in res)[tuple(sorted(best.items()))] == 5.0


def test_candidates_enumerate_the_product_in_order():
    c = tune.candidates({"a": (1, 2), "b": (3,), "c": (4, 5)})
    assert c == [{"a": 1, "b": 3, "c": 4}, {"a": 1, "b": 3, "c": 5},
                 {"a": 2, "b": 3, "c": 4}, {"a": 2, "b": 3, "c": 5}]
    assert len(tune.candidates()) == 4 * 3 * 2 * 4
    assert tune.candidates(limit=3) == tune.candidates()[:3]
