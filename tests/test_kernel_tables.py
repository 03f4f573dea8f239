"""Host checks of constant tables and arithmetic identities the chunk sort's
kernels rely on, read from the kernel source as text (no GPU, no library).

* The per-thread sorting network of the chunk sort (Batcher's odd-even merge
  network for 16 inputs with every comparator on slots 13..15 dropped) sorts
  every 0/1 input of 13 slots, which by the 0-1 principle (Knuth, TAOCP
  vol. 3, 5.3.4) means it sorts every input.
* The pair comparison of (key, index) as the borrow out of one 96-bit
  subtraction (index in the low word, then the key's low and high words)
  equals the lexicographic comparison, including ties on the key and the
  extremes of every word."""
import os
import random
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LEARNED = os.path.join(ROOT, "paper_1109_2348_gb300", "csrc", "learned.cu")


def _network():
    src = open(LEARNED).read()
    m = re.search(r"void sort13\(.*?constexpr int NET\[(\d+)\]\[2\] = \{(.*?)\};", src, re.S)
    assert m, "sort13's comparator table not found"
    pairs = [(int(a), int(b)) for a, b in re.findall(r"\{\s*(\d+)\s*,\s*(\d+)\s*\}", m.group(2))]
    assert len(pairs) == int(m.group(1))
    width = int(re.search(r"constexpr int MS_IT = (\d+);", src).group(1))
    return pairs, width


def _unsorted_inputs(pairs, n):
    """How many of the 2^n 0/1 inputs the network leaves unsorted (all
    inputs at once, one row per slot)."""
    x = np.arange(1 << n, dtype=np.uint32)
    a = np.stack([(x >> i) & 1 for i in range(n)]).astype(np.uint8)
    for i, j in pairs:
        lo, hi = np.minimum(a[i], a[j]), np.maximum(a[i], a[j])
        a[i], a[j] = lo, hi
    return int((a[:-1] > a[1:]).any(axis=0).sum())


def test_chunk_sort_network_sorts_every_zero_one_input():
    pairs, n = _network()
    assert n == 13 and len(pairs) == 48
    assert all(0 <= i < j < n for i, j in pairs)
    assert _unsorted_inputs(pairs, n) == 0


def test_chunk_sort_network_fails_without_any_one_comparator():
    # every comparator is needed: dropping any one leaves some 0/1 input unsorted
    pairs, n = _network()
    for drop in range(len(pairs)):
        assert _unsorted_inputs(pairs[:drop] + pairs[drop + 1:], n) > 0, f"comparator {pairs[drop]} is redundant"


def _borrow_mask(ak, ai, bk, bi):
    """The carry chain as the kernel writes it: sub.cc on the indices, then
    subc.cc on the key's low and high words, then subc of zeros."""
    M = 1 << 32
    words_a = [ai, ak & (M - 1), ak >> 32]
    words_b = [bi, bk & (M - 1), bk >> 32]
    borrow = 0
    for wa, wb in zip(words_a, words_b):
        d = wa - wb - borrow
        borrow = 1 if d < 0 else 0
    return (0 - borrow) & (M - 1)


def test_pair_compare_as_one_borrow_chain():
    rng = random.Random(20261203)
    edge_k = [0, 1, (1 << 32) - 1, 1 << 32, (1 << 63), (1 << 64) - 2, (1 << 64) - 1]
    edge_i = [0, 1, (1 << 24) - 1, 0xFFFF0000, (1 << 32) - 2, (1 << 32) - 1]
    cases = [(ak, ai, bk, bi) for ak in edge_k for ai in edge_i for bk in edge_k for bi in edge_i]
    for _ in range(20000):
        ak = rng.getrandbits(64)
        bk = ak if rng.random() < 0.3 else rng.getrandbits(64)
        if rng.random() < 0.2:
            bk = ak ^ (1 << rng.randrange(64))
        cases.append((ak, rng.getrandbits(32), bk, rng.getrandbits(32)))
    for ak, ai, bk, bi in cases:
        want = 0xFFFFFFFF if (ak, ai) < (bk, bi) else 0
        assert _borrow_mask(ak, ai, bk, bi) == want, (hex(ak), ai, hex(bk), bi)
