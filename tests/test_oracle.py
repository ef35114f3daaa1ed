"""Pins for the CPU oracle, independent of the oracle itself.

Each pin checks the oracle against something the paper or the mathematics
fixes: the worked examples of Section 2.1/2.2 (tests/golden/), closed forms,
brute force against Python's own bytes ordering, invariants (permutation,
ISA[SA[j]] = j, BWT inversion) and a textbook BWT. A planted-mutant build of
the oracle for each plausible mistake must fail at least one pin.
"""
import itertools

import numpy as np
import pytest

import gen
import oracle
from conftest import ints, read_golden


def py_sa(t: bytes):
    """Suffix order by Python's bytes comparison (lexicographic, unsigned,
    a proper prefix first): an implementation independent of oracle.c."""
    return sorted(range(len(t)), key=lambda i: t[i:])


# ---- pin functions: each returns a list of failure messages -------------

def pin_examples(o):
    bad = []
    g = read_golden("ex1_ex2_bdacbdacb.txt")
    t, sa = g["text"].encode(), ints(g["sa"])
    if list(o.naive_sa(t)) != sa:
        bad.append("Ex1 naive")
    for h0 in (1, 2, 3):
        if list(o.pd_sa(t, h0=h0)[0]) != sa:
            bad.append(f"Ex1 pd h0={h0}")
    _, isa, rounds, trace = o.pd_sa(t, h0=int(g["h0"]), trace_cap=8)
    want = [ints(g[f"names_{k}"]) for k in range(3)]
    if rounds != int(g["rounds"]) or [list(r) for r in trace] != want:
        bad.append(f"Ex2 names {trace.tolist()} rounds {rounds}")
    if list(isa) != want[-1]:
        bad.append("Ex2 final ISA")
    g3 = read_golden("ex3_dbacbacbd.txt")
    t3 = g3["text"].encode()
    if list(o.naive_sa(t3)) != ints(g3["sa"]) or list(o.pd_sa(t3)[0]) != ints(g3["sa"]):
        bad.append("Ex3")
    sub = bytes(ints(g3["sub_text_bytes"]))
    if list(o.naive_sa(sub)) != ints(g3["sub_sa"]) or list(o.pd_sa(sub)[0]) != ints(g3["sub_sa"]):
        bad.append("Ex3 sub-problem")
    return bad


def pin_closed_forms(o):
    bad = []
    for n in list(range(0, 40)) + [257, 1000]:
        t = b"a" * n
        want = list(range(n - 1, -1, -1))  # a^n: shorter suffixes first
        for name, sa in (("naive", o.naive_sa(t)), ("pd", o.pd_sa(t)[0]),
                         ("pd2", o.pd_sa(t, h0=2)[0])):
            if list(sa) != want:
                bad.append(f"a^{n} {name}")
                break
    for m in (1, 2, 3, 10, 50):
        t = b"ab" * m
        want = list(range(2 * m - 2, -1, -2)) + list(range(2 * m - 1, 0, -2))
        if list(o.naive_sa(t)) != want or list(o.pd_sa(t)[0]) != want:
            bad.append(f"(ab)^{m}")
    rng = np.random.default_rng(7)
    for n in (1, 2, 17, 256):
        t = rng.permutation(256)[:n].astype(np.uint8)
        want = list(np.argsort(t, kind="stable"))  # all distinct: by first char
        if list(o.naive_sa(t)) != want or list(o.pd_sa(t)[0]) != want:
            bad.append(f"distinct n={n}")
    return bad


def pin_bruteforce(o, max_ab=12, max_4=6):
    bad = []
    for alpha, top in ((b"ab", max_ab), (bytes([0, 1, 2, 255]), max_4)):
        for L in range(1, top + 1):
            for tup in itertools.product(alpha, repeat=L):
                t = bytes(tup)
                want = py_sa(t)
                if list(o.naive_sa(t)) != want:
                    bad.append(f"naive {t!r}")
                for h0 in (1, 2):
                    if list(o.pd_sa(t, h0=h0)[0]) != want:
                        bad.append(f"pd h0={h0} {t!r}")
                for a in (3, 4):
                    if list(o.pd_sa(t, h0=1, a=a)[0]) != want:
                        bad.append(f"pq a={a} {t!r}")
                if bad:
                    return bad
    return bad


def pin_random(o):
    bad = []
    for seed in range(6):
        for recipe, n in (("dna", 3000), ("zipf_repeats", 4096), ("markov", 5000),
                          ("bytes", 2000), ("zipf", 3000)):
            t = gen.text(recipe, 100 + seed, n)
            tb = t.tobytes()
            want = py_sa(tb) if n <= 3000 else list(o.naive_sa(t))
            sa, isa, _, _ = o.pd_sa(t)
            if list(sa) != want:
                bad.append(f"pd {recipe} seed {seed}")
            if not np.array_equal(isa[sa], np.arange(n, dtype=np.uint32)):
                bad.append(f"ISA[SA] {recipe}")
    return bad


def pin_checker(o):
    bad = []
    for seed in range(4):
        t = gen.text("dna", 500 + seed, 600).tobytes()
        good = np.array(py_sa(t), dtype=np.uint32)
        if o.check_sa(t, good)[0] != 0:
            bad.append("rejects a correct SA")
        for j in (0, 1, 299, 598):
            s = good.copy()
            s[j], s[j + 1] = s[j + 1], s[j]
            if o.check_sa(t, s)[0] == 0:
                bad.append(f"accepts adjacent swap at {j}")
        s = good.copy()
        s[10] = s[20]
        if o.check_sa(t, s)[0] != 1:
            bad.append("accepts a duplicate")
        s = good.copy()
        s[5] = 600
        if o.check_sa(t, s)[0] != 1:
            bad.append("accepts out of range")
        s = good.copy()
        s[100], s[400] = s[400], s[100]
        if o.check_sa(t, s)[0] == 0:
            bad.append("accepts a far swap")
    if o.check_permutation(np.array(py_sa(b"banana"), dtype=np.uint32)) != 0:
        bad.append("permutation check rejects a permutation")
    for wrong in ([0, 1, 1], [0, 3, 1], [2, 0]):
        if o.check_permutation(np.array(wrong, dtype=np.uint32)) == 0:
            bad.append(f"permutation check accepts {wrong}")
    t = b"aaaa"
    if o.check_sa(t, np.array([0, 1, 2, 3], dtype=np.uint32))[0] == 0:
        bad.append("accepts a^4 in text order")
    if o.check_sa(t, np.array([3, 2, 1, 0], dtype=np.uint32))[0] != 0:
        bad.append("rejects a^4")
    return bad


def py_adjacent_violations(t: bytes, sa, idx):
    """Violations of SA order at the sampled j, by Python's bytes order (no
    oracle code): j with a pair (j, j+1) whose entries are not both < n or
    whose suffixes are not strictly increasing."""
    n = len(t)
    bad = 0
    for j in idx:
        j = int(j)
        if j < 0 or j + 1 >= n:
            continue
        a, b = int(sa[j]), int(sa[j + 1])
        if a >= n or b >= n or not t[a:] < t[b:]:
            bad += 1
    return bad


def pin_adjacent(o):
    """The sampled adjacent-suffix check, on SAs that are right and on SAs
    with one planted error, against counts fixed by construction or by
    Python's bytes order."""
    bad = []
    for recipe, seed, n in (("dna", 41, 700), ("zipf_repeats", 42, 900), ("bytes", 43, 257)):
        t = gen.text(recipe, seed, n).tobytes()
        good = np.array(py_sa(t), dtype=np.uint32)
        every = np.arange(-2, n + 2)
        if o.check_adjacent(t, good, every) != 0:
            bad.append(f"{recipe}: counts violations in a correct SA")
        for j in (0, 1, n // 2, n - 2):  # an adjacent swap breaks exactly pair j
            s = good.copy()
            s[j], s[j + 1] = s[j + 1], s[j]
            if o.check_adjacent(t, s, [j]) != 1:
                bad.append(f"{recipe}: swap at {j} not counted once")
            if o.check_adjacent(t, s, [j, j]) != 2:
                bad.append(f"{recipe}: a repeated sample not counted twice")
            # Pairs away from the swap stay in order: a sample that misses
            # j - 1, j, j + 1 counts nothing.
            others = [k for k in range(n - 1) if abs(k - j) > 1]
            if o.check_adjacent(t, s, others) != 0:
                bad.append(f"{recipe}: swap at {j} counted outside the sample")
        s = good.copy()
        s[n // 3] = n  # out of range: breaks the pairs on both sides
        if o.check_adjacent(t, s, [n // 3 - 1, n // 3, n // 3 + 1]) != 2:
            bad.append(f"{recipe}: out-of-range entry")
        s = good.copy()
        s[5] = s[4]  # a repeated entry: equal suffixes are not increasing
        if o.check_adjacent(t, s, [4]) != 1:
            bad.append(f"{recipe}: repeated entry accepted")
        rng = np.random.default_rng(seed)
        for _ in range(3):  # random wrong orders against Python's count
            s = good.copy()
            k = rng.integers(0, n, 40)
            s[k] = s[rng.permutation(k)]
            idx = rng.integers(-1, n + 1, 300)
            if o.check_adjacent(t, s, idx) != py_adjacent_violations(t, s, idx):
                bad.append(f"{recipe}: shuffled SA count")
    for n in (2, 3, 17, 64):  # a^n in text order: every pair is decreasing
        t = b"a" * n
        inc = np.arange(n, dtype=np.uint32)
        if o.check_adjacent(t, inc, np.arange(n - 1)) != n - 1:
            bad.append(f"a^{n} in text order")
        if o.check_adjacent(t, inc[::-1].copy(), np.arange(n - 1)) != 0:
            bad.append(f"a^{n} in SA order")
    if o.check_adjacent(b"ab", np.array([0, 1], dtype=np.uint32), [-1, 1, 2, 9]) != 0:
        bad.append("indices without a pair are not skipped")
    return bad


def pin_bwt(o):
    bad = []
    t = b"banana"  # textbook: BWT(banana$) = annb$aa
    b, p = o.bwt(t, np.array(py_sa(t), dtype=np.uint32))
    if bytes(b) != b"annb\x00aa" or p != 4:
        bad.append(f"banana {bytes(b)!r} {p}")
    for recipe in ("dna", "zipf_repeats", "markov", "bytes"):
        t = gen.text(recipe, 9, 4096)
        sa = o.pd_sa(t)[0]
        b, p = o.bwt(t, sa)
        try:
            if not np.array_equal(o.bwt_invert(b, p), t):
                bad.append(f"roundtrip {recipe}")
        except ValueError:
            bad.append(f"roundtrip {recipe} failed")
    return bad


def pin_rank(o):
    bad = []
    t = gen.text("zipf_repeats", 3, 2048)
    isa = np.empty(2048, dtype=np.int64)
    isa[np.array(py_sa(t.tobytes()))] = np.arange(2048)
    for i in (0, 1, 77, 1024, 2047):
        if o.suffix_rank(t, i) != isa[i]:
            bad.append(f"rank {i}")
    return bad


def py_lcp(t: bytes):
    """LCP of adjacent suffixes in Python's bytes order: independent of
    oracle.c (os.path.commonprefix on the two suffixes)."""
    import os
    order = py_sa(t)
    return [0] + [len(os.path.commonprefix([t[order[j - 1]:], t[order[j]:]]))
                  for j in range(1, len(t))]


def pin_lcp(o):
    bad = []
    if list(o.lcp(b"banana", o.naive_sa(b"banana"))) != [0, 1, 3, 0, 0, 2]:  # textbook
        bad.append("banana")
    for n in (1, 2, 5, 64):  # a^n: adjacent suffixes a^j, a^(j+1)
        if list(o.lcp(b"a" * n, o.naive_sa(b"a" * n))) != list(range(n)):
            bad.append(f"a^{n}")
    for m in (1, 4, 9):  # (ab)^m: 0, 2, .., 2m-2 | 0, 1, 3, .., 2m-3
        t = b"ab" * m
        want = [2 * k for k in range(m)] + [0] + [2 * k + 1 for k in range(m - 1)]
        if list(o.lcp(t, o.naive_sa(t))) != want:
            bad.append(f"(ab)^{m}")
    t = bytes(range(200))  # all distinct: no shared prefix
    if any(o.lcp(t, o.naive_sa(t))):
        bad.append("distinct")
    for L in range(1, 11):
        for tup in itertools.product(b"ab", repeat=L):
            t = bytes(tup)
            if list(o.lcp(t, o.naive_sa(t))) != py_lcp(t):
                bad.append(f"brute {t!r}")
                return bad
    t = gen.text("zipf_repeats", 21, 3000).tobytes()
    if list(o.lcp(t, o.naive_sa(t))) != py_lcp(t):
        bad.append("zipf_repeats")
    if o.lcp_pair(b"abcabd", 0, 3) != 2 or o.lcp_pair(b"aaaa", 1, 2) != 2:
        bad.append("pair")
    return bad


def head_ranks(t: bytes, H: int):
    """Name of every suffix after resolving H characters, by definition:
    the number of suffixes whose first H characters compare smaller (the
    head rank of its group, Section 2's lexicographic names; a unique
    suffix's head rank is its rank). Python's bytes order, no oracle code."""
    import bisect
    keys = [t[i:i + H] for i in range(len(t))]
    order = sorted(keys)
    return [bisect.bisect_left(order, k) for k in keys]


def pin_multiplier(o):
    """Prefix doubling and its a-fold form (Prefix Quadrupling): after round
    k the names are the head ranks of the (h0 * a^k)-character prefixes, and
    the rounds stop at the first k where those prefixes are all distinct."""
    bad = []
    g = read_golden("ex1_ex2_bdacbdacb.txt")
    texts = [g["text"].encode(), b"a" * 37, b"ab" * 19, b"abaababaabaab", b"mississippi"]
    rng = np.random.default_rng(11)
    for n, sigma in ((60, 2), (90, 3), (150, 4), (120, 26)):
        texts.append(bytes(rng.integers(97, 97 + sigma, n, dtype=np.uint8)))
    texts.append(gen.text("zipf_repeats", 5, 200).tobytes())
    texts.append(gen.text("dna", 6, 256).tobytes())
    for t in texts:
        n = len(t)
        for a in (2, 3, 4):
            for h0 in (1, 2, 3):
                _, isa, rounds, trace = o.pd_sa(t, h0=h0, trace_cap=64, a=a)
                want_rounds = 0
                while len(set(t[i:i + h0 * a ** want_rounds] for i in range(n))) < n:
                    want_rounds += 1
                if rounds != want_rounds:
                    bad.append(f"a={a} h0={h0} rounds {rounds} != {want_rounds} ({t[:12]!r})")
                    continue
                for k in range(rounds + 1):
                    if list(trace[k]) != head_ranks(t, h0 * a ** k):
                        bad.append(f"a={a} h0={h0} names after round {k} ({t[:12]!r})")
                        break
                if sorted(isa.tolist()) != list(range(n)):
                    bad.append(f"a={a} h0={h0} final names not a permutation")
    for n in (1, 2, 5, 16, 17, 64, 65, 1000):  # a^n: smallest k with h0 * a^k >= n
        for a in (3, 4):
            k = 0
            while a ** k < n:
                k += 1
            if o.pd_sa(b"z" * n, h0=1, a=a)[2] != k:
                bad.append(f"z^{n} a={a} rounds")
    return bad


def py_dc7_names(t: bytes):
    """DC7's first recursion text by definition, in Python: the samples
    i = 0, 1, 3 (mod 7) with i <= n, class by class; each named 1 + the
    number of distinct smaller 7-character windows (the end of text below
    every byte, encoded -1)."""
    n = len(t)
    wins = []
    for a in (0, 1, 3):
        for i in range(a, n + 1, 7):
            wins.append(tuple(t[i + k] if i + k < n else -1 for k in range(7)))
    order = {w: r + 1 for r, w in enumerate(sorted(set(wins)))}
    return [order[w] for w in wins]


def pin_dc7_names(o):
    bad = []
    texts = [b"", b"x", b"ab", b"abcdefg", b"abcdefgh", b"a" * 50, b"ab" * 40,
             b"mississippi" * 3, bytes(range(256))]
    rng = np.random.default_rng(3)
    for n, sigma in ((100, 2), (301, 3), (700, 256)):
        texts.append(bytes(rng.integers(0, sigma, n, dtype=np.uint8)))
    texts.append(gen.text("zipf_repeats", 8, 1500).tobytes())
    for t in texts:
        if list(o.dc7_names(t)) != py_dc7_names(t):
            bad.append(f"dc7 names {t[:10]!r} (n={len(t)})")
    for n in range(0, 30):  # sizes: every class runs to i <= n
        if len(o.dc7_names(b"q" * n)) != sum(len(range(a, n + 1, 7)) for a in (0, 1, 3)):
            bad.append(f"dc7 size n={n}")
    return bad


PINS = [pin_examples, pin_closed_forms, pin_bruteforce, pin_random, pin_checker,
        pin_adjacent, pin_bwt, pin_rank, pin_lcp, pin_multiplier, pin_dc7_names]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_oracle_pins(orc, pin):
    assert pin(orc) == []


@pytest.mark.parametrize("mutant", oracle.MUTANTS)
def test_every_planted_mistake_fails_a_pin(mutant):
    m = oracle.Oracle(mutant)
    failed = []
    for pin in PINS:
        if pin is pin_bruteforce:
            res = pin(m, max_ab=8, max_4=4)
        else:
            res = pin(m)
        if res:
            failed.append(pin.__name__)
            break
    assert failed, f"mutant {mutant} passes every pin"


def test_empty_and_tiny(orc):
    assert orc.naive_sa(b"").size == 0
    assert orc.pd_sa(b"")[0].size == 0
    assert list(orc.pd_sa(b"x")[0]) == [0]
    assert list(orc.pd_sa(b"ba")[0]) == [1, 0]
    assert list(orc.pd_sa(b"\x00\x00")[0]) == [1, 0]
    assert orc.check_sa(b"", np.zeros(0, dtype=np.uint32))[0] == 0
    for a in (3, 4):
        assert orc.pd_sa(b"", a=a)[0].size == 0
        assert list(orc.pd_sa(b"x", a=a)[0]) == [0]
        assert list(orc.pd_sa(b"ba", a=a)[0]) == [1, 0]
    with pytest.raises(ValueError):
        orc.pd_sa(b"abc", a=5)
