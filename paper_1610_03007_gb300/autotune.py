"""Autotuner for the build's tile parameters.

Two knobs of the build trade occupancy against per-tile work and are picked
by measurement rather than fixed:

- ``sort_items`` -- keys per thread of the one-sweep radix pass (tile =
  256 x 8, 12 or 16 keys): larger tiles amortise the per-tile look-back and
  barriers, smaller ones fit more blocks per SM.
- ``refine_shape`` -- threads x items of the small-group refine (128 x 1024,
  256 x 2048, 256 x 4096, 256 x 1024). It also sets the segment threshold:
  groups of up to half a tile are refined inside one block, larger ones take
  the global radix sort.

``tune`` times the candidates through the C-ABI on the caller's own input
(coordinate search: the radix tile first, then the refine shape, each
candidate the median of ``reps`` builds, timed with CUDA events) and
``Table`` keeps the winners per workload class and power-of-two size bucket
in a JSON file. The radix digit width is fixed at 8 bits: the look-back gives
one thread per digit bin, so the bin count is the block size.
"""
from __future__ import annotations

import json
import math
import os

SORT_ITEMS = (16, 12, 8)
REFINE_SHAPES = (1, 2, 3, 4)
DEFAULTS = {"sort_items": 16, "refine_shape": 1}


def _time_build(gbsa, text, workspace, params, reps):
    import torch
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        gbsa.sa_build_ex(text, workspace=workspace, **params)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    times.sort()
    return times[len(times) // 2]


def tune(text, workspace=None, reps: int = 3) -> dict:
    """Best {sort_items, refine_shape} for this input (a uint8 CUDA tensor)
    with the milliseconds measured for every candidate tried."""
    import torch

    import paper_1610_03007_gb300 as gbsa
    if workspace is None:
        workspace = torch.empty(gbsa.workspace_bytes(text.numel()), dtype=torch.uint8,
                                device=text.device)
    best = dict(DEFAULTS)
    tried = {}
    gbsa.sa_build_ex(text, workspace=workspace, **best)  # warm-up
    for items in SORT_ITEMS:
        p = dict(best, sort_items=items)
        tried[f"items={items},shape={p['refine_shape']}"] = ms = _time_build(
            gbsa, text, workspace, p, reps)
        if ms < tried.get("_best", math.inf):
            tried["_best"], best = ms, p
    for shape in REFINE_SHAPES:
        p = dict(best, refine_shape=shape)
        key = f"items={p['sort_items']},shape={shape}"
        if key not in tried:
            tried[key] = ms = _time_build(gbsa, text, workspace, p, reps)
            if ms < tried["_best"]:
                tried["_best"], best = ms, p
    best_ms = tried.pop("_best")
    return {"params": best, "ms": best_ms, "tried": tried}


def bucket(n: int) -> int:
    return max(0, int(n).bit_length() - 1)


class Table:
    """Tuned parameters per (workload class, log2 size bucket), as JSON."""

    def __init__(self, path: str | None = None):
        self.path = path or os.environ.get(
            "GBSA_TUNING", os.path.join(os.path.expanduser("~"), ".cache", "gbsa", "tuning.json"))
        self.entries = {}
        if os.path.exists(self.path):
            with open(self.path) as f:
                self.entries = json.load(f)

    def put(self, workload: str, n: int, params: dict, ms: float | None = None):
        self.entries[f"{workload}/{bucket(n)}"] = {"params": params, "ms": ms}

    def get(self, workload: str, n: int) -> dict:
        """Parameters of the nearest tuned bucket of this workload class,
        else the defaults."""
        b = bucket(n)
        best, dist = None, None
        for key, val in self.entries.items():
            w, _, kb = key.rpartition("/")
            if w != workload:
                continue
            d = abs(int(kb) - b)
            if dist is None or d < dist:
                best, dist = val["params"], d
        return dict(best) if best else dict(DEFAULTS)

    def save(self):
        os.makedirs(os.path.dirname(self.path) or ".", exist_ok=True)
        tmp = self.path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(self.entries, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)
