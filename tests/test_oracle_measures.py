"""Pins Run(A), Mono(A) and Inv(A) (Section 2) to brute force, the worked
example and the closed forms the paper states for its input classes."""
import itertools
from functools import lru_cache

import numpy as np
import pytest

import oracle
import sortrace_inputs as si


def _mono_brute(seq):
    """Fewest monotone pieces by dynamic programming over all cut points."""
    n = len(seq)

    def monotone(i, j):
        s = seq[i:j]
        return all(s[k] <= s[k + 1] for k in range(len(s) - 1)) or \
            all(s[k] >= s[k + 1] for k in range(len(s) - 1))

    @lru_cache(None)
    def best(i):
        if i == n:
            return 0
        return min(1 + best(j) for j in range(i + 1, n + 1) if monotone(i, j))

    return best(0)


def test_mono_runs_inv_brute_force():
    for n in range(0, 8):
        for seq in itertools.product(range(3), repeat=n):
            a = np.array(seq, dtype=np.int32)
            assert oracle.mono(a) == _mono_brute(seq), seq
            desc = sum(1 for i in range(n - 1) if seq[i] > seq[i + 1])
            assert oracle.runs(a) == (desc + 1 if n else 0)
            inv = sum(1 for i in range(n) for j in range(i + 1, n) if seq[i] > seq[j])
            assert oracle.inversions(a) == inv


def test_worked_example():
    a = np.array([1, 15, 18, 19, 20, 16, 11, 10, 9, 8, 7, 6, 5, 4, 3, 2], dtype=np.int32)
    assert oracle.runs(a) == 12
    assert oracle.mono(a) == 2


@pytest.mark.parametrize("n", [1, 2, 17, 1000])
def test_reversed_and_sorted(n):
    r = si.reversed_i32(n, 1)
    assert oracle.runs(r) == n
    assert oracle.mono(r) == 1
    assert oracle.inversions(r) == n * (n - 1) // 2
    s = np.sort(r)
    assert oracle.runs(s) == 1 and oracle.mono(s) == 1 and oracle.inversions(s) == 0


@pytest.mark.parametrize("k", [1, 2, 4, 8, 64])
def test_teeth_closed_forms(k):
    n = 4096
    eq = si.k_equal_teeth(n, k)
    assert oracle.runs(eq) == k and oracle.mono(eq) == k
    ev = si.k_even_teeth(n, k)
    assert oracle.mono(ev) == k          # k <= n/3
    sh = si.k_sharp_teeth(n, k)
    assert oracle.mono(sh) == k
    if k == 1:
        assert np.array_equal(sh, np.arange(n, 0, -1, dtype=np.int32))


def test_even_teeth_half_n():
    """k = n/2: (2,1,1,2,2,1,1,2,...) with Mono = n/4 + 1 (Section 2)."""
    n = 4096
    a = si.k_even_teeth(n, n // 2)
    assert a[:8].tolist() == [2, 1, 1, 2, 2, 1, 1, 2]
    assert oracle.mono(a) == n // 4 + 1


@pytest.mark.parametrize("k", [1, 5, 40])
def test_k_exchange_bounds(k):
    n = 5000
    a = si.k_exchange(n, k, seed=k)
    rank = np.argsort(np.argsort(a, kind="stable"), kind="stable")
    assert np.count_nonzero(rank != np.arange(n)) <= 2 * k
    assert oracle.mono(a) <= 2 * k + 1


@pytest.mark.parametrize("k", [1, 7, 256])
def test_k_distance_bound(k):
    n = 5000
    a = si.k_distance(n, k, seed=k)
    rank = np.argsort(np.argsort(a, kind="stable"), kind="stable")
    assert np.max(np.abs(rank - np.arange(n))) <= k


def test_nearly_sorted_is_k_exchange():
    n = 1 << 16
    a = si.nearly_sorted_i32(n, 2)
    m = n // 100
    s = np.sort(a)
    assert np.count_nonzero(a != s) <= 2 * m
    assert oracle.mono(a) <= 2 * m + 1


@pytest.mark.parametrize("k", [0, 1, 4, 12])
def test_k_limited(k):
    """At most 2^k distinct values, all in [0, 2^k) (Section 2); k = 0 gives
    one value."""
    a = si.k_limited(20_000, k, seed=3)
    u = np.unique(a)
    assert u.size <= (1 << k) and u.min() >= 0 and u.max() < (1 << k)
    if k == 12:
        assert u.size > 3000            # 20,000 draws cover most of 4,096 values


@pytest.mark.parametrize("k", [1, 2, 8])
def test_k_shuffled_teeth(k):
    """A permutation of 1..n in which the values of each k-sharp-teeth section
    appear in that section's order (Section 2); one section is the reversed
    list, and the interleaving is not the unshuffled teeth for k > 1."""
    n = 4096
    a = si.k_shuffled_teeth(n, k, seed=5)
    assert np.array_equal(np.sort(a), np.arange(1, n + 1, dtype=np.int32))
    sharp = si.k_sharp_teeth(n, k)
    L = n // k
    pos = np.empty(n + 1, np.int64)
    pos[a] = np.arange(n)
    for j in range(k):
        sec = sharp[j * L:(j + 1) * L]
        assert np.all(np.diff(pos[sec]) > 0)
    if k == 1:
        assert np.array_equal(a, sharp)
    else:
        assert not np.array_equal(a, sharp)


def _rem_brute(a):
    """The fewest removals that leave a sorted list, over every subset kept."""
    n = len(a)
    best = n
    for mask in range(1 << n):
        kept = [a[i] for i in range(n) if mask >> i & 1]
        if all(kept[i] <= kept[i + 1] for i in range(len(kept) - 1)):
            best = min(best, n - len(kept))
    return best


def test_rem_brute_force():
    """Rem(A) against its definition on every small input drawn (ties included)."""
    rng = np.random.default_rng(80)
    for _ in range(300):
        n = int(rng.integers(0, 10))
        a = rng.integers(-3, 4, n).astype(np.int32)
        assert oracle.rem(a) == _rem_brute(a.tolist())


def test_rem_closed_forms():
    n = 1000
    assert oracle.rem(np.arange(n, dtype=np.int32)) == 0
    assert oracle.rem(np.zeros(n, np.int32)) == 0
    assert oracle.rem(np.arange(n, 0, -1).astype(np.int32)) == n - 1
    # one exchange: two items out of place, one if they were neighbours
    assert oracle.rem(np.array([1, 4, 3, 2, 5], np.int32)) == 2
    assert oracle.rem(np.array([1, 3, 2, 4, 5], np.int32)) == 1
    # float32 totalOrder: -0.0 before +0.0
    f = np.array([0x00000000, 0x80000000], np.uint32).view(np.float32)
    assert oracle.rem(f) == 1


@pytest.mark.parametrize("k", [1, 5, 40])
def test_rem_of_k_exchange_lists(k):
    """A k-exchange list leaves a sorted list once the at most 2k items out of
    place are removed (Section 2)."""
    a = si.k_exchange(5000, k, seed=k)
    r = oracle.rem(a)
    assert 0 < r <= 2 * k
