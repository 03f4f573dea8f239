"""Pins of the stage oracles (run-length, move-to-front and variable-length
encoding, Sections 3.2-3.4): the paper's worked examples (Fig. 1, Fig. 2,
Fig. 3 in tests/golden/), hand-worked move-to-front words, closed forms and
properties of the definitions, and round trips."""
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _fields(name):
    out = {}
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, v = line.split(":", 1)
        out[k.strip()] = v.split()
    return out


def _bytes(vals):
    return np.array([ord(v) for v in vals], dtype=np.uint8)


def _ints(vals):
    return np.array([int(v) for v in vals], dtype=np.int64)


def test_rle_encode_matches_fig1():
    f = _fields("rle_fig1_fig2.txt")
    S = _bytes(f["input"])
    chars, lens = oracle.rle_encode(S)
    assert np.array_equal(chars, _bytes(f["data_values"]))
    assert np.array_equal(lens, _ints(f["run_lengths"]))
    # the figure's intermediate arrays follow from the runs
    ends = np.cumsum(lens)
    assert np.array_equal(ends, _ints(f["data_index"]))
    flags = np.zeros(S.size, dtype=np.int64)
    flags[ends - 1] = 1
    assert np.array_equal(flags, _ints(f["run_boundaries"]))
    assert np.array_equal(np.cumsum(flags) - flags, _ints(f["output_positions"]))


def test_rle_decode_matches_fig2():
    f = _fields("rle_fig1_fig2.txt")
    out = oracle.rle_decode(_bytes(f["data_values"]), _ints(f["run_lengths"]))
    assert np.array_equal(out, _bytes(f["decode_output"]))
    bpos = np.cumsum(_ints(f["run_lengths"]))
    assert np.array_equal(bpos, _ints(f["decode_boundary_positions"]))
    flags = np.zeros(out.size, dtype=np.int64)
    flags[bpos - 1] = 1
    assert np.array_equal(flags, _ints(f["decode_run_boundaries"]))
    assert np.array_equal(np.cumsum(flags) - flags, _ints(f["decode_scatter_positions"]))


def test_rle_closed_forms_and_properties():
    c, ln = oracle.rle_encode(b"a" * 1000)
    assert list(c) == [97] and list(ln) == [1000]
    c, ln = oracle.rle_encode(b"ab" * 50)
    assert c.size == 100 and np.all(ln == 1)
    rng = np.random.default_rng(3)
    for n in [1, 2, 3, 17, 1000, 20_000]:
        S = rng.integers(0, 3, n).astype(np.uint8)
        c, ln = oracle.rle_encode(S)
        assert ln.min() >= 1 and int(ln.sum()) == n
        assert np.all(c[1:] != c[:-1])  # runs are maximal
        assert np.array_equal(oracle.rle_decode(c, ln), S)


def test_vle_positions_match_fig3():
    f = _fields("vle_fig3.txt")
    lens = _ints(f["lengths"])
    printed = _ints(f["positions_printed"])
    fixed = _ints(f["positions"])
    assert np.array_equal(np.delete(printed, 4), np.delete(fixed, 4))  # only the typo differs
    # eight distinct characters with the figure's codeword lengths (all-ones codes)
    code = np.zeros(256, dtype=np.uint32)
    length = np.ones(256, dtype=np.uint8)
    for i, L in enumerate(lens):
        code[i] = (1 << int(L)) - 1
        length[i] = L
    out, bits, pos = oracle.vle_encode(np.arange(8, dtype=np.uint8), code, length, with_pos=True)
    assert np.array_equal(pos, fixed) and bits == int(lens.sum()) == 63
    assert out.size == 8 and np.all(out[:7] == 0xFF) and out[7] == 0xFE  # 63 one bits, MSB first


def _canonical_code(lengths):
    """A prefix code with the given lengths (Kraft sum <= 1), assigned in
    (length, symbol) order -- an independent way to build decodable tables."""
    code = np.zeros(256, dtype=np.uint32)
    nxt, prev = 0, 0
    for sym in sorted(range(256), key=lambda s: (lengths[s], s)):
        L = int(lengths[sym])
        nxt <<= L - prev
        code[sym] = nxt
        nxt += 1
        prev = L
    return code


def test_vle_round_trip_with_a_prefix_code():
    rng = np.random.default_rng(4)
    lengths = np.full(256, 8, dtype=np.uint8)  # all 8-bit: the canonical code of byte c is c
    code = _canonical_code(lengths)
    S = rng.integers(0, 256, 5000).astype(np.uint8)
    out, bits = oracle.vle_encode(S, code, lengths)
    assert bits == 8 * S.size and np.array_equal(out, S)  # 8-bit canonical code of all bytes = identity
    # a skewed code: decode bit by bit and compare
    lengths = np.concatenate([[2, 2, 3], np.full(253, 11)]).astype(np.uint8)
    # Kraft: 2/4 + 1/8 + 253/2048 <= 1
    code = _canonical_code(lengths)
    S = rng.choice(256, 3000, p=np.r_[[0.3, 0.3, 0.2], np.full(253, 0.2 / 253)]).astype(np.uint8)
    out, bits = oracle.vle_encode(S, code, lengths)
    assert bits == int(lengths[S].astype(np.int64).sum())
    table = {(int(lengths[s]), int(code[s])): s for s in range(256)}
    got, acc, al = [], 0, 0
    for p in range(bits):
        acc = (acc << 1) | ((int(out[p >> 3]) >> (7 - (p & 7))) & 1)
        al += 1
        if (al, acc) in table:
            got.append(table[(al, acc)])
            acc, al = 0, 0
    assert np.array_equal(np.array(got, dtype=np.uint8), S)


@pytest.mark.parametrize("word,outs", [(w, v) for w, v in _fields("mtf_words.txt").items()])
def test_mtf_hand_worked_words(word, outs):
    assert np.array_equal(oracle.mtf_encode(word.encode()), _ints(outs))


def test_mtf_closed_forms_and_round_trip():
    assert np.array_equal(oracle.mtf_encode(np.arange(256, dtype=np.uint8)), np.arange(256))
    out = oracle.mtf_encode(b"x" * 500)
    assert out[0] == ord("x") and np.all(out[1:] == 0)
    rng = np.random.default_rng(5)
    for n in [1, 2, 255, 256, 257, 10_000]:
        S = rng.integers(0, 256, n).astype(np.uint8)
        out = oracle.mtf_encode(S)
        assert np.array_equal(oracle.mtf_decode(out), S)
        # the first occurrence of a byte sits behind the distinct bytes seen before it
        seen = []
        for i in range(min(n, 300)):
            c = int(S[i])
            if c not in seen:
                assert out[i] == len(seen) + sum(1 for v in range(c) if v not in seen)
                seen.append(c)


def test_stage_oracles_against_plain_python():
    """The three definitions written out in plain Python, independent of the
    oracle's C code, on random short inputs over small and full alphabets:
    maximal runs in order; the position of each byte in a list that starts
    0..255 and moves every byte to the front; codewords concatenated most
    significant bit first, the last byte padded with zeros."""
    import itertools
    rng = np.random.default_rng(23)
    code = rng.integers(0, 1 << 12, 256).astype(np.uint32)
    length = rng.integers(1, 13, 256).astype(np.uint8)
    code &= (np.uint32(1) << length.astype(np.uint32)) - np.uint32(1)
    for trial in range(200):
        alpha = int(rng.choice([1, 2, 3, 256]))
        s = rng.integers(0, alpha, int(rng.integers(1, 400))).astype(np.uint8)
        runs = [(k, len(list(g))) for k, g in itertools.groupby(s.tolist())]
        chars, lens = oracle.rle_encode(s)
        assert chars.tolist() == [k for k, _ in runs] and lens.tolist() == [n for _, n in runs]
        lst, mtf = list(range(256)), []
        for c in s.tolist():
            i = lst.index(c)
            mtf.append(i)
            lst.insert(0, lst.pop(i))
        assert oracle.mtf_encode(s).tolist() == mtf
        bits = "".join(format(int(code[c]), "0%db" % int(length[c])) for c in s.tolist())
        want = bytes(int((bits + "0" * 7)[i:i + 8], 2) for i in range(0, len(bits), 8))
        out, nbits = oracle.vle_encode(s, code, length)
        assert nbits == len(bits) and bytes(out) == want
