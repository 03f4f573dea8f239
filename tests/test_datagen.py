"""The seeded generators: pinned to the published SplitMix64 sequence, and
the sources have the statistics their names promise."""
import numpy as np

from paper_1109_2348_gb300 import datagen


def test_splitmix64_published_sequence():
    # SplitMix64 (Steele, Lea, Flood 2014) from state 0: its first three outputs
    assert datagen.splitmix_probe(0, 3) == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_sources_are_deterministic_and_shaped():
    for src in range(9):
        a = datagen.block(src, 42, 10_000)
        b = datagen.block(src, 42, 10_000)
        assert np.array_equal(a, b)
    m3 = datagen.block(datagen.MARKOV3_Z96, 1, 200_000)
    assert m3.min() >= 0x20 and m3.max() <= 0x7F
    m2 = datagen.block(datagen.MARKOV2_Z64, 1, 200_000)
    assert m2.min() >= 0x20 and m2.max() <= 0x5F
    runs = datagen.block(datagen.RUNS16, 1, 500_000)
    assert runs.max() <= 15
    nruns = 1 + np.count_nonzero(runs[1:] != runs[:-1])
    assert 40 < runs.size / nruns < 60  # geometric runs of mean 50
    assert np.all(datagen.block(datagen.CONST, 1, 100) == 0x61)
    p7 = datagen.block(datagen.PERIOD7, 1, 100)
    assert np.array_equal(p7[:93], p7[7:])
    fib = bytes(datagen.block(datagen.FIBONACCI, 1, 13))
    assert fib == b"abaababaabaab"


def test_permutation_and_sizes():
    p = datagen.permutation(3, 1000)
    assert np.array_equal(np.sort(p), np.arange(1000))
    w = datagen.uneven_markov3()
    assert w.num_blocks == 256 and min(w.sizes) >= 10_000 and max(w.sizes) <= 900_000
    w5 = datagen.learned_eval()
    assert w5.num_blocks == 1200 and w5.sources.count(datagen.UNIFORM) == 120
