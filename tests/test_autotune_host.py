"""Host logic of the autotuner (candidate handling, one launch or two, the
cache) with the timing of a candidate replaced by a fake: no GPU needed."""
import json

import pytest

from paper_2501_18630_gb300 import autotune, scenes


class _Planes:
    device = "cuda:0"


@pytest.fixture
def fake(monkeypatch, tmp_path):
    monkeypatch.setenv("BETA_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    monkeypatch.setattr(autotune.torch.cuda, "get_device_name", lambda dev=None: "fake GB300")
    timed = []

    def time_candidate(planes, n, n_lobes, cameras, target, cand, reps=5, hit_masks=True):
        timed.append(tuple(cand))
        # two launches faster at 16x8 / 64, otherwise by tile area
        return 1.0 if tuple(cand) == (16, 8, 64, False, False) else 2.0 + cand[0] * cand[1] / 1000.0

    monkeypatch.setattr(autotune, "time_candidate", time_candidate)
    return timed, tmp_path / "tune.json"


def test_fused_flag_defaults_to_one_launch():
    assert autotune.fused_of((16, 8, 64, False)) is True
    assert autotune.fused_of((16, 8, 64, False, False)) is False
    assert any(len(c) > 4 and not c[4] for c in autotune.CANDIDATES)


def test_tune_picks_the_fastest_and_caches_it(fake):
    timed, path = fake
    cams = [scenes.ring_camera(4.0, 15.0, 0.0, 320, 240)]
    best, times = autotune.tune(_Planes(), 1000, 3, cams, None)
    assert best == (16, 8, 64, False, False)
    assert set(times) == {tuple(c) for c in autotune.CANDIDATES}
    assert timed == [tuple(c) for c in autotune.CANDIDATES]
    d = json.load(open(path))
    assert len(d) == 1 and list(d.values())[0]["best"] == list(best)
    timed.clear()
    assert autotune.tune(_Planes(), 1000, 3, cams, None)[0] == best      # from the cache
    assert timed == []


def test_tune_two_launches_only(fake):
    timed, path = fake
    cams = [scenes.ring_camera(4.0, 15.0, 0.0, 320, 240)]
    cands = [(16, 16, 256, True), (16, 8, 64, False), (16, 8, 64, False, False)]
    best, times = autotune.tune(_Planes(), 1000, 3, cams, None, candidates=cands, fused=False)
    # duplicates after the conversion to two launches are timed once
    assert timed == [(16, 16, 256, True, False), (16, 8, 64, False, False)]
    assert best == (16, 8, 64, False, False) and set(times) == set(timed)
    # another candidate list is another cache entry
    autotune.tune(_Planes(), 1000, 3, cams, None, candidates=cands)
    assert len(json.load(open(path))) == 2
