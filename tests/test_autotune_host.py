"""The tile-shape autotuner's search and cache on CPU: the batch timing is replaced by a synthetic
cost of the tile shapes, so the search, the per-size refinement and the JSON cache are checked
without a GPU."""
import json

import pytest

torch = pytest.importorskip("torch")

from paper_2103_06644_gb300 import autotune  # noqa: E402

FRAMES = [dict(W=640, H=480, window=7), dict(W=640, H=480, window=7), dict(W=1920, H=1080, window=21),
          dict(W=320, H=240, window=5)]

# the best shape per (W, H, k) class of the synthetic cost
BEST = {(640, 480, 7): (64, 128), (1920, 1080, 21): (64, 32), (320, 240, 5): (64, 256)}


def fake_time(calls):
    def t(frames, shapes, method, reps=5, **kw):
        calls.append(dict(shapes))
        cost = 0.0
        for c, (hs, vb) in shapes.items():
            bh, bv = BEST[c]
            cost += abs(autotune.HSEGS.index(hs) - autotune.HSEGS.index(bh)) * 3.0
            cost += abs(autotune.VBANDS.index(vb) - autotune.VBANDS.index(bv))
        return cost
    return t


@pytest.fixture
def tuner(tmp_path, monkeypatch):
    calls = []
    monkeypatch.setenv("SF_TILE_CACHE", str(tmp_path / "tiles.json"))
    monkeypatch.setattr(autotune, "_time", fake_time(calls))
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "test GPU")
    return calls, tmp_path / "tiles.json"


def test_search_finds_the_best_shapes_and_caches_them(tuner):
    calls, path = tuner
    out = autotune.tune(FRAMES)
    assert len(out) == len(FRAMES)
    for f, o in zip(FRAMES, out):
        assert (o["hseg"], o["vband"]) == BEST[(f["W"], f["H"], f["window"])]
        assert {k: o[k] for k in f} == f  # the frames themselves are unchanged
    # a shared grid over every (hseg, vband), then one band sweep per class
    n_grid = len(autotune.HSEGS) * len(autotune.VBANDS)
    assert all(len(set(c.values())) == 1 for c in calls[:n_grid])
    assert n_grid < len(calls) <= n_grid + 3 * len(autotune.VBANDS)
    db = json.load(open(path))
    (key, entry), = db.items()
    assert key.startswith("test GPU|disparity|")
    assert entry == {"%d,%d,%d" % c: list(v) for c, v in BEST.items()}
    # the second call of the same batch reads the cache and times nothing
    calls.clear()
    assert autotune.tune(FRAMES) == out
    assert calls == []


def test_cache_is_per_batch_signature_and_method(tuner):
    calls, path = tuner
    autotune.tune(FRAMES)
    n = len(calls)
    autotune.tune(FRAMES[:3])          # a different batch (one frame less): tuned anew
    assert len(calls) > n
    n = len(calls)
    autotune.tune(FRAMES, method="standard")
    assert len(calls) > n
    assert len(json.load(open(path))) == 3


def test_unwritable_cache_only_costs_the_cache(tuner, monkeypatch, tmp_path):
    calls, _ = tuner
    blocker = tmp_path / "file"
    blocker.write_text("not a directory")
    monkeypatch.setenv("SF_TILE_CACHE", str(blocker / "tiles.json"))
    out = autotune.tune(FRAMES)
    assert [(o["hseg"], o["vband"]) for o in out] == [BEST[(f["W"], f["H"], f["window"])] for f in FRAMES]
    n = len(calls)
    autotune.tune(FRAMES)              # nothing was stored: tuned again
    assert len(calls) > n
