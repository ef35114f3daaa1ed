"""Autotuner for the build's parameters, and the table the library reads.

Four knobs of a build are picked by measurement rather than fixed:

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
- ``bucket_min`` -- the discard threshold: how many pending ISA writes (the
  names of suffixes discarded as unique or renamed in a round) make the
  build bucket them by position before writing; below it they are written
  directly (0xFFFFFFFF: never bucket).

The radix digit width is not a knob: it is fixed at 8 bits, because the
look-back gives one thread per digit bin, so the bin count is the block
size (256).

``tune`` times the candidates through the C-ABI on one input (coordinate
search: the radix tile, the refine shape, the key width, then the discard
threshold; each candidate the median of ``reps`` builds timed with CUDA
events); ``tune_batched`` does the same for one batched build. ``Table``
holds the winners per class -- (batched, bits per character, floor(log2)
of the total length) -- in the library's own text format, which
libgbsa.so reads at its first build (tuning.txt beside the library, or the
file named by GBSA_TUNING_TABLE) so that sa_build and sa_build_batched take
tuned values for every knob their options leave at 0.

    python -m paper_1610_03007_gb300.autotune [--out PATH] [--quick]

tunes the representative inputs below on the current GPU (seeds distinct
from the benchmark's) and writes the table (default: tuning.txt beside the
library).
"""
from __future__ import annotations

import argparse
import math
import os

SORT_ITEMS = (16, 12, 8)
REFINE_SHAPES = (1, 2, 3, 4)
BUCKET_MINS = (1 << 20, 1 << 22, 1 << 24, 0xFFFFFFFF)
DEFAULTS = {"sort_items": 16, "refine_shape": 1, "h0_chars": 0, "bucket_min": 1 << 22}
FIELDS = ("sort_items", "refine_shape", "h0_chars", "bucket_min")
HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_TABLE = os.path.join(HERE, "tuning.txt")


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


def widest_key(bits_per_char: int, texts: int = 1) -> int:
    """Characters of the widest initial key: as many as fit in 64 bits
    beside the text-id bits of a batch of `texts` texts."""
    seg = (texts - 1).bit_length() if texts > 1 else 0
    return (64 - seg) // max(1, bits_per_char)


def tune(text, workspace=None, reps: int = 3) -> dict:
    """Best {sort_items, refine_shape, h0_chars, bucket_min} for this input
    (a uint8 CUDA tensor), the alphabet's bits per character, and the
    milliseconds measured for every candidate tried. Every candidate is
    passed explicitly (a 0 would mean "the library's table" and make the
    search depend on the table it is writing)."""
    import torch

    import paper_1610_03007_gb300 as gbsa
    if workspace is None:
        workspace = torch.empty(gbsa.workspace_bytes(text.numel()), dtype=torch.uint8,
                                device=text.device)

    def run(p):
        return gbsa.sa_build_ex(text, workspace=workspace, **p)

    _, _, st, _ = run(DEFAULTS)  # warm-up; gives the alphabet's bits per character
    c0max = widest_key(st["bits_per_char"])
    start = dict(DEFAULTS, h0_chars=c0max)
    coords = [("sort_items", SORT_ITEMS), ("refine_shape", REFINE_SHAPES),
              ("h0_chars", [c0max] + key_width_candidates(c0max, st["bits_per_char"])),
              ("bucket_min", BUCKET_MINS)]
    best, ms, tried = _search(lambda p: _median_ms(lambda: run(p), reps), coords, start)
    return {"params": best, "ms": ms, "tried": tried, "bits_per_char": st["bits_per_char"]}


def tune_batched(texts, offsets, sa_out, workspace, reps: int = 1) -> dict:
    """The same search for one sa_build_batched call over these texts (the
    refine shape is left at its default: batched texts of uniform DNA are
    resolved in round 0)."""
    import paper_1610_03007_gb300 as gbsa

    def run(p):
        return gbsa.sa_build_batched(texts, offsets, sa_out=sa_out, workspace=workspace,
                                     stats=True, **p)

    _, st = run(DEFAULTS)  # warm-up; gives the alphabet's bits per character
    c0max = widest_key(st["bits_per_char"], len(offsets) - 1)
    start = dict(DEFAULTS, h0_chars=c0max)
    coords = [("sort_items", SORT_ITEMS),
              ("h0_chars", [c0max] + key_width_candidates(c0max, st["bits_per_char"])),
              ("bucket_min", BUCKET_MINS)]
    best, ms, tried = _search(lambda p: _median_ms(lambda: run(p), reps), coords, start)
    return {"params": best, "ms": ms, "tried": tried, "bits_per_char": st["bits_per_char"]}


def bucket(n: int) -> int:
    """floor(log2 n), the table's size bucket (0 for n <= 1)."""
    return max(0, int(n).bit_length() - 1)


class Table:
    """Tuned parameters per (batched, bits per character, log2 size bucket)
    in the library's text format: one entry a line,
    "batched bits log2n sort_items refine_shape h0_chars bucket_min"."""

    def __init__(self, path: str | None = None):
        self.path = path or DEFAULT_TABLE
        self.entries = {}
        self.notes = {}
        if os.path.exists(self.path):
            with open(self.path) as f:
                for line in f:
                    body, _, note = line.partition("#")
                    parts = body.split()
                    if not parts:
                        continue
                    if len(parts) != 7:
                        raise ValueError(f"{self.path}: malformed line {line!r}")
                    b, bits, lg = (int(x) for x in parts[:3])
                    self.entries[(b, bits, lg)] = dict(zip(FIELDS, (int(x) for x in parts[3:])))
                    self.notes[(b, bits, lg)] = note.strip()

    def put(self, batched: bool, bits: int, n: int, params: dict, note: str = ""):
        key = (1 if batched else 0, int(bits), bucket(n))
        self.entries[key] = {f: int(params.get(f, 0)) for f in FIELDS}
        self.notes[key] = note

    def get(self, batched: bool, bits: int, n: int) -> dict:
        """The entry of this (batched, bits) class with the nearest size
        bucket -- the library's own rule -- else the defaults."""
        b = bucket(n)
        best, dist = None, None
        for (tb, tbits, lg), params in sorted(self.entries.items()):
            if tb != (1 if batched else 0) or tbits != bits:
                continue
            d = abs(lg - b)
            if dist is None or d < dist:
                best, dist = params, d
        return dict(best) if best else dict(DEFAULTS)

    def save(self):
        os.makedirs(os.path.dirname(self.path) or ".", exist_ok=True)
        tmp = self.path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            f.write("# gbsa tuning table: batched bits log2n sort_items refine_shape "
                    "h0_chars bucket_min\n")
            for key in sorted(self.entries):
                p = self.entries[key]
                note = self.notes.get(key, "")
                f.write(" ".join(str(x) for x in key + tuple(p[k] for k in FIELDS)) +
                        (f"  # {note}" if note else "") + "\n")
        os.replace(tmp, self.path)


# Representative inputs of each class (seeds distinct from the benchmark's).
SINGLE_INPUTS = (
    ("markov", 3101, 1 << 31),        # DNA, order-3 Markov with copies (2 bits)
    ("dna", 1101, 1 << 20),           # uniform DNA
    ("dna", 5101, 1 << 16),
    ("dna", 5102, 1 << 24),
    ("zipf_repeats", 2101, 1 << 28),  # Zipf(1.1) bytes, 256 repeats (8 bits)
    ("zipf", 5103, 1 << 16),          # i.i.d. Zipf bytes
    ("zipf", 5104, 1 << 20),
    ("zipf", 5105, 1 << 24),
)
BATCH_INPUT = (4101, 4096, 1 << 10, 4 << 20)  # seed, texts, shortest, longest


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--out", default=DEFAULT_TABLE)
    ap.add_argument("--quick", action="store_true", help="inputs up to 2^20 only")
    ap.add_argument("--reps", type=int, default=2)
    args = ap.parse_args(argv)
    import sys

    import torch
    sys.path.insert(0, os.path.dirname(HERE))
    import gen
    import paper_1610_03007_gb300 as gbsa
    from paper_1610_03007_gb300 import _build
    _build.build()
    gbsa.load()
    table = Table(args.out)
    gpu = torch.cuda.get_device_name()
    for recipe, seed, n in SINGLE_INPUTS:
        if args.quick and n > 1 << 20:
            continue
        text = torch.from_numpy(gen.text(recipe, seed, n)).cuda()
        r = tune(text, reps=args.reps)
        table.put(False, r["bits_per_char"], n, r["params"],
                  f"{recipe} n=2^{bucket(n)} seed {seed}: {r['ms']:.3f} ms on {gpu}")
        print(recipe, n, r["params"], round(r["ms"], 3), flush=True)
        del text
        torch.cuda.empty_cache()
    if not args.quick:
        seed, count, lo, hi = BATCH_INPUT
        flat, off = gen.batch(seed, count, lo, hi)
        texts = torch.from_numpy(flat).cuda()
        N = int(off[-1])
        sa = torch.empty(N, dtype=torch.int32, device="cuda")
        ws = torch.empty(int(gbsa.load().sa_batched_workspace_bytes(off.ctypes.data, count)),
                         dtype=torch.uint8, device="cuda")
        r = tune_batched(texts, off, sa, ws, reps=args.reps)
        table.put(True, r["bits_per_char"], N, r["params"],
                  f"{count} DNA texts, {N} bytes, seed {seed}: {r['ms']:.3f} ms on {gpu}")
        print("batched", N, r["params"], round(r["ms"], 3), flush=True)
    table.save()
    print("wrote", table.path)


if __name__ == "__main__":
    main()
