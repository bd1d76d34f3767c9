"""Pins for the oracle's Philox4x64-10 against numpy's independent implementation.

numpy.random.Philox implements the same generator (Salmon et al., SC'11);
it advances its 256-bit counter by one before producing each block of four
words, so the block for counter c is read with numpy's counter set to c - 1.
"""
import numpy as np
import pytest

import oracle


def _numpy_block(ctr, key):
    c = [int(x) for x in ctr]
    # subtract one from the 256-bit little-endian counter
    for i in range(4):
        if c[i] > 0:
            c[i] -= 1
            break
        c[i] = (1 << 64) - 1
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(c, dtype=np.uint64))
    return [int(x) for x in bg.random_raw(4)]


@pytest.mark.parametrize("ctr,key", [
    ([0, 0, 0, 0], [0, 0]),
    ([1, 0, 0, 0], [42, 0]),
    ([1843199, 7, 6, 0], [42, 1]),
    ([0, 3, 1, 0], [42, 5]),                                     # borrow across words
    ([2**64 - 1, 2**64 - 1, 2**63, 12345], [2**64 - 1, 2**63 + 5]),
    ([123456789, 0, 0, 0], [0xDEADBEEF, 0xCAFEBABE]),
])
def test_philox_matches_numpy(ctr, key):
    assert oracle.philox4x64_10(ctr, key) == _numpy_block(ctr, key)


def test_philox_random_counters():
    rng = np.random.default_rng(3)
    for _ in range(50):
        ctr = [int(x) for x in rng.integers(0, 2**63, size=4, dtype=np.int64)]
        ctr[0] += 1
        key = [int(x) for x in rng.integers(0, 2**63, size=2, dtype=np.int64)]
        assert oracle.philox4x64_10(ctr, key) == _numpy_block(ctr, key)


def test_u24_mapping():
    assert oracle.u24(0) == 0.0
    assert oracle.u24(2**64 - 1) == 1.0 - 2.0**-24
    assert oracle.u24(1 << 63) == 0.5
    assert oracle.u24((1 << 40) - 1) == 0.0          # low 40 bits are discarded
