"""Pins of the oracle's counter-based noise source (Philox4x32-10, Salmon et
al., SC'11) and of the uniform / Gaussian mapping that feeds Sec. 3.5's r_k."""
import os

import numpy as np

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    with open(os.path.join(GOLD, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(x, 16) for x in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_known_answers(ora):
    for ctr, key, want in _kat():
        assert ora.philox(ctr, key) == want


def test_uniform_exact(ora):
    assert ora.uniform(0) == 2.0 ** -24
    assert ora.uniform(0xffffffff) == (2.0 ** 24 - 1) * 2.0 ** -24
    assert ora.uniform(1 << 31) == (2.0 * (1 << 22) + 1) * 2.0 ** -24
    # strictly inside (0, 1), hence log() finite
    assert 0.0 < ora.uniform(511) < 1.0


def test_counter_layout(ora):
    """raw_words uses counter (node, step, domain<<8 | block, replica), key (seed lo, hi)."""
    seed = 0x1234567890abcdef
    w = ora.raw_words(seed, 17, 5, domain=1, replica=3, nblocks=2)
    key = [seed & 0xffffffff, seed >> 32]
    assert w[:4].tolist() == ora.philox([17, 5, (1 << 8) | 0, 3], key)
    assert w[4:8].tolist() == ora.philox([17, 5, (1 << 8) | 1, 3], key)


def test_gaussian_statistics(ora):
    """Box-Muller output: mean 0, variance 1, kurtosis 3, independent pairs."""
    g = np.concatenate([ora.gaussians(0, n, 0) for n in range(6000)])
    assert g.size == 96000
    assert abs(g.mean()) < 0.015
    assert abs(g.var() - 1.0) < 0.02
    assert abs((g ** 4).mean() / g.var() ** 2 - 3.0) < 0.1
    pairs = g.reshape(-1, 2)
    assert abs(np.corrcoef(pairs[:, 0], pairs[:, 1])[0, 1]) < 0.02


def test_gaussian_matches_box_muller(ora):
    """The Gaussians are the Box-Muller map of consecutive uniforms."""
    raw = ora.raw_words(9, 4, 2, domain=0)
    g = ora.gaussians(9, 4, 2, domain=0)
    for p in range(8):
        v1 = (2.0 * (int(raw[2 * p]) >> 9) + 1) * 2.0 ** -24
        v2 = (2.0 * (int(raw[2 * p + 1]) >> 9) + 1) * 2.0 ** -24
        r = np.sqrt(-2 * np.log(v1))
        assert np.isclose(g[2 * p], r * np.cos(2 * np.pi * v2), rtol=1e-14, atol=1e-15)
        assert np.isclose(g[2 * p + 1], r * np.sin(2 * np.pi * v2), rtol=1e-14, atol=1e-15)


def test_box_muller_of_words_matches_gaussians(ora):
    """The word-pair map is the one the noise streams use, pair by pair."""
    for node in (0, 7, 123456):
        w = ora.raw_words(99, node, 5, domain=0, replica=2, nblocks=4)
        assert np.array_equal(ora.box_muller(w), ora.gaussians(99, node, 5, domain=0, replica=2, nblocks=4))
