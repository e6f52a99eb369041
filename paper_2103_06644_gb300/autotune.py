"""Tile-shape autotuner for mixed-resolution batches.

For a batch, every frame's tile shape (hseg columns per horizontal tile,
vband rows per vertical band) is chosen by timing the real batch pass with
CUDA events: first one shape shared by all frames (the best of a small
candidate grid), then a round of per-size refinement where each (W, H, k)
class tries the other band heights while the rest stay fixed.  The choice is cached
in a JSON file keyed by the GPU name, the method and the batch signature.
Results never depend on the tile shape (the window sums are exact); only the
speed does.
"""
from __future__ import annotations

import json
import os
from typing import Dict, List, Sequence, Tuple

HSEGS = (32, 64, 128)
VBANDS = (32, 64, 128, 256)


def cache_path() -> str:
    p = os.environ.get("SF_TILE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "surffit_gb300", "tiles.json")


def _load() -> Dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(db: Dict) -> None:
    p = cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        tmp = p + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(db, f, indent=1, sort_keys=True)
        os.replace(tmp, p)
    except OSError:
        pass  # a read-only home only costs the cache


def _classes(frames) -> List[Tuple[int, int, int]]:
    return sorted({(int(f["W"]), int(f["H"]), int(f["window"])) for f in frames})


def _time(frames, shapes, method, reps=5, **kw) -> float:
    import torch

    from . import SurfaceFitBatch

    fr = [dict(f, hseg=shapes[(f["W"], f["H"], f["window"])][0], vband=shapes[(f["W"], f["H"], f["window"])][1])
          for f in frames]
    b = SurfaceFitBatch(fr, method=method, use_graph=True, **kw)
    b.run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        b.run()
    e1.record()
    torch.cuda.synchronize()
    b.close()
    return e0.elapsed_time(e1) / reps


def tune(frames: Sequence[dict], method: str = "disparity", use_cache: bool = True, **kw) -> List[dict]:
    """Return copies of ``frames`` with tuned 'hseg' and 'vband' entries."""
    import torch

    classes = _classes(frames)
    key = "%s|%s|%s" % (torch.cuda.get_device_name(), method,
                        ";".join("%dx%dk%d*%d" % (W, H, k, sum(1 for f in frames if (f["W"], f["H"], f["window"]) ==
                                                               (W, H, k))) for (W, H, k) in classes))
    db = _load() if use_cache else {}
    if key in db:
        shapes = {tuple(map(int, c.split(","))): tuple(v) for c, v in db[key].items()}
    else:
        best, shapes = None, None
        for hs in HSEGS:
            for vb in VBANDS:
                cand = {c: (hs, vb) for c in classes}
                t = _time(frames, cand, method, **kw)
                if best is None or t < best:
                    best, shapes = t, cand
        for c in classes:  # per-size refinement of the band height
            for vb in VBANDS:
                if vb == shapes[c][1]:
                    continue
                cand = dict(shapes)
                cand[c] = (shapes[c][0], vb)
                t = _time(frames, cand, method, **kw)
                if t < best:
                    best, shapes = t, cand
        db[key] = {"%d,%d,%d" % c: list(v) for c, v in shapes.items()}
        if use_cache:
            _store(db)
    return [dict(f, hseg=shapes[(f["W"], f["H"], f["window"])][0], vband=shapes[(f["W"], f["H"], f["window"])][1])
            for f in frames]
