"""The order keys of bbe_order_histogram (include/bbe.h): host-only encode and decode in the C
library, checked without a GPU against the definition.  A key is the mixed-radix number whose
digit j (radix n - j) counts the not-yet-placed competitors of lower index than the place-j
finisher, i.e. the rank of the ordered tuple in the lexicographic list of all K-tuples of
distinct competitors; itertools.permutations lists those tuples in exactly that order."""
import itertools
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def bbe():
    from paper_2108_02419_gb300 import bbe as B
    from paper_2108_02419_gb300 import build

    build.build()
    B.lib()
    return B


@pytest.mark.parametrize("n,places", [(1, 1), (2, 2), (3, 1), (3, 3), (4, 2), (5, 3), (5, 5), (6, 4)])
def test_keys_are_lexicographic_ranks(bbe, n, places):
    kk = min(places, n)
    for rank, tup in enumerate(itertools.permutations(range(n), kk)):
        assert bbe.bbe_order_key_encode(n, places, tup) == rank
        assert tuple(bbe.bbe_order_key_decode(n, places, rank)) == tup
    assert rank == math.perm(n, kk) - 1


def test_full_orders_of_twenty_and_the_largest_keys(bbe):
    rng = np.random.default_rng(5)
    for _ in range(200):
        p = rng.permutation(20)
        key = bbe.bbe_order_key_encode(20, 20, p)
        # the same rank from the factorial number system
        want, left = 0, list(range(20))
        for j, c in enumerate(p):
            want = want * (20 - j) + left.index(int(c))
            left.remove(int(c))
        assert key == want and np.array_equal(bbe.bbe_order_key_decode(20, 20, key), p)
    top = math.factorial(20) - 1  # the last order, 19 18 .. 0
    assert list(bbe.bbe_order_key_decode(20, 20, top)) == list(range(19, -1, -1))
    assert bbe.bbe_order_key_encode(32, 13, list(range(31, 18, -1))) == math.perm(32, 13) - 1


def test_rejects_bad_orders_keys_and_ranges(bbe):
    for n, places, order in [(4, 3, [0, 0, 1]), (4, 2, [4, 1]), (4, 2, [-1, 1])]:
        with pytest.raises(bbe.BbeError) as ei:
            bbe.bbe_order_key_encode(n, places, order)
        assert ei.value.status == -1
    with pytest.raises(bbe.BbeError):
        bbe.bbe_order_key_decode(5, 3, math.perm(5, 3))  # one past the last key
    with pytest.raises(bbe.BbeError):
        bbe.bbe_order_key_encode(21, 21, list(range(21)))  # 21! keys exceed 64 bits
    with pytest.raises(bbe.BbeError):
        bbe.bbe_order_key_decode(32, 14, 0)
    assert bbe.bbe_order_key_encode(21, 18, list(range(18))) == 0
