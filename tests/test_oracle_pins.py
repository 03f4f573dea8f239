"""Pins of the CPU oracle against what the transform's definition fixes.

The oracle (oracle/bwt_oracle.c) is checked here against values that do not
come from itself: hand-worked words (tests/golden/bwt_words.txt), the
inverse transform's round trip, permutation invariants, closed forms for
constant blocks and exact powers, exhaustive brute force on tiny inputs, and
central finite differences for the MLP gradient. A plausible slip in the
oracle -- an off-by-one in the last-column index, a reversed tie-break, a
dropped rename step, a transposed weight -- fails at least one test.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_1109_2348_gb300 import datagen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "bwt_words.txt")


def golden_words():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        w, L, p = line.split()
        rows.append((w, L, int(p)))
    return rows


@pytest.mark.parametrize("word,L,primary", golden_words())
def test_hand_checked_words(word, L, primary):
    for fn in (oracle.bwt_bruteforce, oracle.bwt_block):
        got_L, got_p = fn(word)
        assert bytes(got_L).decode() == L and got_p == primary, fn.__name__


def _rotation_leq(S, a, b):
    n = len(S)
    for j in range(n):
        ca, cb = S[(a + j) % n], S[(b + j) % n]
        if ca != cb:
            return ca < cb
    return a < b


def test_bruteforce_rows_are_sorted_and_valid():
    rng = np.random.default_rng(7)
    for n in list(range(1, 40)) + [101, 257]:
        for alpha in (1, 2, 3, 256):
            S = rng.integers(0, alpha, n, dtype=np.uint8)
            L, p, SA = oracle.bwt_bruteforce(S, with_sa=True)
            assert sorted(SA.tolist()) == list(range(n))
            assert SA[p] == 0
            for k in range(n - 1):
                assert _rotation_leq(S, SA[k], SA[k + 1])
            for k in range(n):
                assert L[k] == S[(SA[k] - 1) % n]


def test_doubling_equals_bruteforce_all_ab_strings_up_to_12():
    for n in range(1, 13):
        for bits in itertools.product(b"ab", repeat=n):
            S = np.frombuffer(bytes(bits), dtype=np.uint8)
            L1, p1, SA1 = oracle.bwt_bruteforce(S, with_sa=True)
            L2, p2, SA2 = oracle.bwt_block(S, with_sa=True)
            assert p1 == p2 and np.array_equal(SA1, SA2), bytes(bits)


def test_every_abc_string_up_to_7_against_python_sort():
    """The definition in plain Python, independent of the oracle's C code: SA
    sorts the rotations as byte strings, ties by lower index."""
    for n in range(1, 8):
        for chars in itertools.product(b"abc", repeat=n):
            s = bytes(chars)
            sa = sorted(range(n), key=lambda i: (s[i:] + s[:i], i))
            want_L = bytes(s[(i - 1) % n] for i in sa)
            L, p = oracle.bwt_block(np.frombuffer(s, dtype=np.uint8))
            assert bytes(L) == want_L and p == sa.index(0), s


def test_doubling_equals_bruteforce_random():
    rng = np.random.default_rng(11)
    for trial in range(120):
        n = int(rng.integers(1, 2000))
        alpha = int(rng.choice([1, 2, 4, 16, 256]))
        S = rng.integers(0, alpha, n, dtype=np.uint8)
        if trial % 5 == 0:  # periodic structure: deep ties
            unit = rng.integers(0, alpha, int(rng.integers(1, 9)), dtype=np.uint8)
            S = np.resize(unit, n)
        L1, p1, SA1 = oracle.bwt_bruteforce(S, with_sa=True)
        L2, p2, SA2 = oracle.bwt_block(S, with_sa=True)
        assert p1 == p2 and np.array_equal(SA1, SA2)


def test_inverse_round_trip_and_permutation():
    rng = np.random.default_rng(3)
    for src in range(9):
        S = datagen.block(src, 17 + src, 5000)
        L, p = oracle.bwt_block(S)
        assert np.array_equal(np.bincount(L, minlength=256), np.bincount(S, minlength=256))
        assert np.array_equal(oracle.inverse_bwt(L, p), S)
    for _ in range(50):
        S = rng.integers(0, 3, int(rng.integers(1, 300)), dtype=np.uint8)
        L, p = oracle.bwt_block(S)
        assert np.array_equal(oracle.inverse_bwt(L, p), S)


def test_inverse_detects_wrong_primary():
    S = np.frombuffer(b"abracadabra", dtype=np.uint8)
    L, p = oracle.bwt_block(S)
    for q in range(len(S)):
        if q != p:
            assert not np.array_equal(oracle.inverse_bwt(L, q), S)


def test_constant_block_closed_form():
    for n in (1, 2, 7, 8, 9, 1000):
        S = np.full(n, 0x61, dtype=np.uint8)
        L, p, SA = oracle.bwt_block(S, with_sa=True)
        assert p == 0 and np.array_equal(SA, np.arange(n)) and np.array_equal(L, S)


def test_exact_power_closed_form():
    """S = u^k: rows come in runs of k identical rotations, so L is L(u) with
    every symbol repeated k times and primary = k * primary(u)."""
    rng = np.random.default_rng(5)
    for _ in range(40):
        m = int(rng.integers(1, 30))
        k = int(rng.integers(1, 12))
        u = rng.integers(0, 4, m, dtype=np.uint8)
        # make u primitive: a word equal to a proper rotation of itself is a power
        if any(np.array_equal(u, np.roll(u, -d)) for d in range(1, m) if m % d == 0):
            continue
        Lu, pu = oracle.bwt_block(u)
        L, p = oracle.bwt_block(np.tile(u, k))
        assert np.array_equal(L, np.repeat(Lu, k)) and p == k * pu


def test_batch_matches_per_block():
    w = datagen.mixed_64x900k(num_blocks=6, n=3000)
    buf, off = w.generate()
    L, prim = oracle.bwt_batch(buf, off, threads=3)
    for b in range(6):
        Lb, pb = oracle.bwt_block(buf[off[b]:off[b + 1]])
        assert np.array_equal(L[off[b]:off[b + 1]], Lb) and prim[b] == pb


def test_degenerate_sources_small():
    w = datagen.degenerate_5x900k(n=4000)
    buf, off = w.generate()
    L, prim = oracle.bwt_batch(buf, off)
    assert prim[0] == 0  # constant block: rotation 0 is first of identical rows
    # period-1000 exact power (4000 = 4 x 1000): closed form
    u = buf[off[2]:off[2] + 1000]
    Lu, pu = oracle.bwt_block(u)
    assert np.array_equal(L[off[2]:off[3]], np.repeat(Lu, 4)) and prim[2] == 4 * pu
    for b in range(5):
        assert np.array_equal(oracle.inverse_bwt(L[off[b]:off[b + 1]], prim[b]), buf[off[b]:off[b + 1]])


# ----------------------------------------------------------------- MLP ---

def _rand_params(seed, scale=0.4):
    return np.random.default_rng(seed).normal(0, scale, oracle.MLP_NPARAMS)


def test_mlp_layout_closed_forms():
    p = np.zeros(oracle.MLP_NPARAMS)
    p[-1] = 0.25  # b3 only: the network is the constant 0.25
    x = np.random.default_rng(0).random((10, 8))
    assert np.allclose(oracle.mlp_forward(p, x), 0.25)
    t = np.linspace(0, 1, 10)
    loss, g = oracle.mlp_loss_grad(p, x, t)
    assert np.isclose(loss, np.mean((0.25 - t) ** 2))
    assert np.isclose(g[-1], 2 * np.mean(0.25 - t))
    assert np.allclose(g[:-1], 0)  # all hidden units are dead (ReLU(0) = 0)
    # one active path: W1[0][3] = 1, W2[0][0] = 1, W3[0] = 1 -> y = x[3]
    p = np.zeros(oracle.MLP_NPARAMS)
    p[0 * 8 + 3] = 1.0
    p[256 + 32 + 0] = 1.0
    p[256 + 32 + 1024 + 32 + 0] = 1.0
    assert np.allclose(oracle.mlp_forward(p, x), x[:, 3])


def test_mlp_gradient_finite_differences():
    rng = np.random.default_rng(1)
    p = _rand_params(2)
    x = rng.random((64, 8))
    t = rng.random(64)
    _, g = oracle.mlp_loss_grad(p, x, t)
    eps = 1e-6
    idx = list(range(0, oracle.MLP_NPARAMS, 7)) + [oracle.MLP_NPARAMS - 1]
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += eps
        pm[i] -= eps
        fd = (oracle.mlp_loss_grad(pp, x, t)[0] - oracle.mlp_loss_grad(pm, x, t)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-8, i


def test_adam_first_step_closed_form():
    """From m = v = 0 the bias-corrected first step is lr * g / (|g| + eps)."""
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    p = np.zeros(4)
    m = np.zeros(4)
    v = np.zeros(4)
    oracle.adam_step(p, g, m, v, 1, lr=1e-3)
    assert np.allclose(p, -1e-3 * g / (np.abs(g) + 1e-8))
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


# A hand-built network for the closed forms below (every number worked out on
# paper from the definitions: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2),
# y = W3 h2 + b3, loss = mean (y - t)^2, W row-major [out][in]):
#   h1[1] = relu(2 x[2] - 1)        clamps for x[2] = 0.25 (pre-activation -0.5)
#   h1[4] = relu(0.3 - x[5])        clamps for x[5] = 0.6  (pre-activation -0.3)
#   h2[3] = relu(h1[1] + 2 h1[4])   W2[3][1] and W2[3][4]: off-diagonal entries
#   h2[6] = relu(0.2 - h1[1])       clamps when h1[1] = 0.5 (pre-activation -0.3)
#   y     = 0.1 + h2[3] + 3 h2[6]
# x[0] = 0.4 in every sample (it feeds no unit, but its gradient pins W1's
# orientation: W1[1][0] sees d1[1] * x[0]).
_W1, _B1, _W2, _B2, _W3, _B3 = 0, 256, 288, 1312, 1344, 1376


def _relu_net():
    p = np.zeros(oracle.MLP_NPARAMS)
    p[_W1 + 1 * 8 + 2] = 2.0
    p[_B1 + 1] = -1.0
    p[_W1 + 4 * 8 + 5] = -1.0
    p[_B1 + 4] = 0.3
    p[_W2 + 3 * 32 + 1] = 1.0
    p[_W2 + 3 * 32 + 4] = 2.0
    p[_W2 + 6 * 32 + 1] = -1.0
    p[_B2 + 6] = 0.2
    p[_W3 + 3] = 1.0
    p[_W3 + 6] = 3.0
    p[_B3] = 0.1
    x = np.zeros((4, 8))
    x[:, 0] = 0.4
    x[:, 2] = [0.25, 0.75, 0.75, 0.25]
    x[:, 5] = [0.1, 0.6, 0.1, 0.6]
    return p, x


def test_mlp_forward_relu_clamps_and_w2_orientation():
    """Per sample (h1[1], h1[4]) = (0, .2), (.5, 0), (.5, .2), (0, 0) and
    (h2[3], h2[6]) = (.4, .2), (.5, 0), (.9, 0), (0, .2), so y = 1.1, 0.6,
    1.0, 0.7. A dropped first-layer ReLU gives 2.2 for sample 0, a dropped
    second-layer ReLU -0.3 for sample 1, and W2 read transposed loses h2[3]."""
    p, x = _relu_net()
    assert np.allclose(oracle.mlp_forward(p, x), [1.1, 0.6, 1.0, 0.7], rtol=0, atol=1e-12)


def test_mlp_gradient_closed_form_through_clamped_units():
    """t = (1.0, 0.6, 0.5, 0.9): errors e = (0.1, 0, 0.5, -0.2), loss = 0.075,
    dL/dy = 2e/4 = (.05, 0, .25, -.1). Back through the layers:
      d2[3] = dy * W3[3] where h2[3] > 0 = (.05, 0, .25, 0)   (sample 3 clamped)
      d2[6] = dy * W3[6] where h2[6] > 0 = (.15, 0, 0, -.3)   (samples 1, 2 clamped)
      d1[1] = (W2[3][1] d2[3] + W2[6][1] d2[6]) where h1[1] > 0 = (0, 0, .25, 0)
      d1[4] = W2[3][4] d2[3] where h1[4] > 0 = (.1, 0, .5, 0)
    so gb3 = .2, gW3[3] = .05*.4 + .25*.9 = .245, gW3[6] = .05*.2 - .1*.2 = -.01,
    gb2[3] = .3, gb2[6] = -.15, gW2[3][1] = .25*.5 = .125,
    gW2[3][4] = .05*.2 + .25*.2 = .06, gW2[6][4] = .15*.2 = .03 (a weight that
    is zero still gets a gradient), gb1[1] = .25, gb1[4] = .6,
    gW1[1][2] = .25*.75 = .1875, gW1[1][0] = .25*.4 = .1,
    gW1[4][5] = .1*.1 + .5*.1 = .06, gW1[4][0] = .6*.4 = .24, and the
    transposed slots W2[1][3], W2[4][3], W2[1][6] get 0."""
    p, x = _relu_net()
    t = np.array([1.0, 0.6, 0.5, 0.9])
    loss, g = oracle.mlp_loss_grad(p, x, t)
    assert abs(loss - 0.075) < 1e-12
    want = {
        _B3: 0.2, _W3 + 3: 0.245, _W3 + 6: -0.01,
        _B2 + 3: 0.3, _B2 + 6: -0.15,
        _W2 + 3 * 32 + 1: 0.125, _W2 + 3 * 32 + 4: 0.06, _W2 + 6 * 32 + 1: 0.0, _W2 + 6 * 32 + 4: 0.03,
        _W2 + 1 * 32 + 3: 0.0, _W2 + 4 * 32 + 3: 0.0, _W2 + 1 * 32 + 6: 0.0,
        _B1 + 1: 0.25, _B1 + 4: 0.6,
        _W1 + 1 * 8 + 2: 0.1875, _W1 + 1 * 8 + 0: 0.1, _W1 + 4 * 8 + 5: 0.06, _W1 + 4 * 8 + 0: 0.24,
        _W1 + 2 * 8 + 1: 0.0,
    }
    for i, v in want.items():
        assert abs(g[i] - v) < 1e-12, (i, g[i], v)
    # every parameter not listed has zero gradient here except the first-layer
    # weights of units 1 and 4 on the inputs that are not zero (x[0], x[2], x[5])
    nonzero = set(np.flatnonzero(np.abs(g) > 1e-15))
    allowed = {i for i, v in want.items() if v != 0.0} | {_W1 + 1 * 8 + 5, _W1 + 4 * 8 + 2}
    assert nonzero <= allowed, sorted(nonzero - allowed)
    assert abs(g[_W1 + 1 * 8 + 5] - 0.25 * 0.1) < 1e-12   # d1[1] x[5] in sample 2
    assert abs(g[_W1 + 4 * 8 + 2] - (0.1 * 0.25 + 0.5 * 0.75)) < 1e-12   # d1[4] x[2]


def test_adam_second_step_bias_correction():
    """Two steps at lr = 0.01 (beta1 0.9, beta2 0.999, eps 1e-8), worked out
    by hand. Element 0, g = 1 then -1: m2 = .9 * .1 - .1 = -.01, v2 = .999 *
    .001 + .001 = .001999; the corrections at t = 2 are 1 - .81 = .19 and
    1 - .998001 = .001999, so m^ = -.01 / .19 and v^ = 1 and the second step
    is +.01 * (.01 / .19) / (1 + eps). Element 1, g = 2 then 2: m2 = .38,
    v2 = .007996, m^ = 2, v^ = 4, both steps are -.01 * 2 / (2 + eps). A
    correction that ignored t (1 - beta instead of 1 - beta^t) would give m^ =
    -.1, v^ = 1.999 for element 0."""
    p = np.array([0.5, -0.25])
    m = np.zeros(2)
    v = np.zeros(2)
    oracle.adam_step(p, np.array([1.0, 2.0]), m, v, 1, lr=0.01)
    oracle.adam_step(p, np.array([-1.0, 2.0]), m, v, 2, lr=0.01)
    eps = 1e-8
    p0 = 0.5 - 0.01 * 1.0 / (1.0 + eps) + 0.01 * (0.01 / 0.19) / (1.0 + eps)
    p1 = -0.25 - 2 * 0.01 * 2.0 / (2.0 + eps)
    assert abs(p[0] - p0) < 1e-13 and abs(p[1] - p1) < 1e-13, (p, p0, p1)
    assert np.allclose(m, [-0.01, 0.38], rtol=0, atol=1e-15)
    assert np.allclose(v, [0.001999, 0.007996], rtol=0, atol=1e-15)
