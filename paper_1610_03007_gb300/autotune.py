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
- ``h0_chars`` -- characters per initial key (0: as many as fit in 64
  bits). Fewer characters mean fewer key bits, so fewer radix passes in
  round 0 (the digit positions the keys never use are skipped), at the cost
  of more doubling rounds for the suffixes they leave tied. Candidates are
  the widest keys that fit 7, 6, 5, 4 and 3 digit passes.

``tune`` times the candidates through the C-ABI on the caller's own input
(coordinate search: the radix tile, then the refine shape, then the key
width, each candidate the median of ``reps`` builds, timed with CUDA
events; ``tune_batched`` does the same for one batched build) and
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
DEFAULTS = {"sort_items": 16, "refine_shape": 1, "h0_chars": 0}


def key_width_candidates(c0max: int, bits_per_char: int):
    """h0_chars values below the alphabet's maximum c0max worth timing: for
    P = 7 .. 3 radix passes, the most characters whose key (c * bits per
    character, plus the text-id bits 64 - c0max * bits the batched key
    carries) fits in P 8-bit digits."""
    b = max(1, bits_per_char)
    seg = max(0, 64 - c0max * b)
    out = []
    for passes in (7, 6, 5, 4, 3):
        c = (8 * passes - seg) // b
        if 2 <= c < c0max and c not in out:
            out.append(c)
    return out


def _median_ms(fn, reps):
    import torch
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    times.sort()
    return times[len(times) // 2]


def _time_build(gbsa, text, workspace, params, reps):
    return _median_ms(lambda: gbsa.sa_build_ex(text, workspace=workspace, **params), reps)


def _search(time_fn, coords, start):
    """Coordinate search: for each (name, values) in turn keep the fastest."""
    best, tried, best_ms = dict(start), {}, math.inf
    for name, values in coords:
        for v in values:
            p = dict(best, **{name: v})
            key = ",".join(f"{k}={p[k]}" for k in sorted(p))
            if key in tried:
                continue
            tried[key] = ms = time_fn(p)
            if ms < best_ms:
                best_ms, best = ms, p
    return best, best_ms, tried


def tune(text, workspace=None, reps: int = 3) -> dict:
    """Best {sort_items, refine_shape, h0_chars} for this input (a uint8
    CUDA tensor) with the milliseconds measured for every candidate tried."""
    import torch

    import paper_1610_03007_gb300 as gbsa
    if workspace is None:
        workspace = torch.empty(gbsa.workspace_bytes(text.numel()), dtype=torch.uint8,
                                device=text.device)
    _, _, st, _ = gbsa.sa_build_ex(text, workspace=workspace, **DEFAULTS)  # warm-up
    coords = [("sort_items", SORT_ITEMS), ("refine_shape", REFINE_SHAPES),
              ("h0_chars", [0] + key_width_candidates(st["chars_per_key"],
                                                      st["bits_per_char"]))]
    best, ms, tried = _search(lambda p: _time_build(gbsa, text, workspace, p, reps),
                              coords, DEFAULTS)
    return {"params": best, "ms": ms, "tried": tried}


def tune_batched(texts, offsets, sa_out, workspace, reps: int = 1) -> dict:
    """The same search for one sa_build_batched call over these texts."""
    import paper_1610_03007_gb300 as gbsa

    def run(p):
        return gbsa.sa_build_batched(texts, offsets, sa_out=sa_out, workspace=workspace,
                                     stats=True, **p)

    _, st = run(DEFAULTS)  # warm-up
    coords = [("sort_items", SORT_ITEMS),
              ("h0_chars", [0] + key_width_candidates(st["chars_per_key"],
                                                      st["bits_per_char"]))]
    best, ms, tried = _search(lambda p: _median_ms(lambda: run(p), reps), coords, DEFAULTS)
    return {"params": best, "ms": ms, "tried": tried}


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
