"""Pins of the oracle's Huffman coding (Sec. IV-A: variable-length coding of
the quantization codes over any number of symbols): Kraft equality,
prefix-freeness, optimality against brute force and against a textbook
heap-based Huffman code."""
import heapq
import itertools

import numpy as np
import pytest


def _kraft(lens):
    return sum(2.0 ** -int(l) for l in lens if l > 0)


def _heap_huffman_cost(freq):
    """Textbook Huffman (priority queue); its total cost is the unique optimum
    even though the length vector is not unique."""
    h = [int(f) for f in freq if f > 0]
    if len(h) == 1:
        return h[0]
    heapq.heapify(h)
    cost = 0
    while len(h) > 1:
        a, b = heapq.heappop(h), heapq.heappop(h)
        cost += a + b
        heapq.heappush(h, a + b)
    return cost


def _brute_force_cost(freq):
    """Minimum of sum f*len over all length vectors with sum 2^-len <= 1."""
    f = [int(v) for v in freq if v > 0]
    best = None
    for ls in itertools.product(range(1, len(f)), repeat=len(f)):
        if sum(2.0 ** -l for l in ls) <= 1.0:
            c = sum(a * b for a, b in zip(f, ls))
            best = c if best is None else min(best, c)
    return best


@pytest.mark.parametrize("seed", range(40))
def test_optimal_on_tiny_histograms(szo, seed):
    rng = np.random.default_rng(seed)
    k = int(rng.integers(2, 7))
    freq = np.zeros(16, np.uint64)
    idx = rng.choice(16, k, replace=False)
    freq[idx] = rng.integers(1, 50, k)
    lens = szo.huffman_lengths(freq)
    assert abs(_kraft(lens) - 1.0) < 1e-12
    cost = int((freq * lens).sum())
    assert cost == _brute_force_cost(freq)
    assert cost == _heap_huffman_cost(freq)


@pytest.mark.parametrize("seed", range(10))
def test_kraft_prefix_free_and_optimal_large(szo, seed):
    rng = np.random.default_rng(100 + seed)
    nsym = 1 << int(rng.integers(4, 17))
    freq = np.zeros(nsym, np.uint64)
    used = rng.choice(nsym, int(rng.integers(2, min(nsym, 3000))), replace=False)
    # peaked distribution like the quantization codes (Fig. 3)
    freq[used] = (rng.pareto(1.2, used.size) * 10 + 1).astype(np.uint64)
    lens = szo.huffman_lengths(freq)
    assert np.all((lens > 0) == (freq > 0))
    assert abs(_kraft(lens) - 1.0) < 1e-9
    assert int((freq * lens).sum()) == _heap_huffman_cost(freq)
    codes = szo.canonical_codes(lens)
    words = sorted(format(int(codes[s]), "0%db" % lens[s]) for s in np.nonzero(lens)[0])
    for a, b in zip(words, words[1:]):
        assert not b.startswith(a)


def test_single_symbol_length_one(szo):
    freq = np.zeros(256, np.uint64)
    freq[128] = 1000
    lens = szo.huffman_lengths(freq)
    assert lens[128] == 1 and lens.sum() == 1


def test_canonical_assignment(szo):
    """Canonical codes: ordered by (length, symbol), consecutive within a
    length, first code 0."""
    lens = np.array([3, 0, 2, 3, 2, 2], np.uint8)
    codes = szo.canonical_codes(lens)
    assert [int(codes[s]) for s in [2, 4, 5, 0, 3]] == [0b00, 0b01, 0b10, 0b110, 0b111]


def test_tie_break_is_deterministic(szo):
    """Equal weights: leaves ordered by symbol, leaf queue first; the result
    depends only on the histogram."""
    freq = np.array([5, 5, 5, 5, 5, 5], np.uint64)
    a = szo.huffman_lengths(freq)
    assert list(a) == list(szo.huffman_lengths(freq.copy()))
    assert abs(_kraft(a) - 1.0) < 1e-12 and sorted(a) == [2, 2, 3, 3, 3, 3]
