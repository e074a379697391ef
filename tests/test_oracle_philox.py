"""Pins of the oracle's counter-based generator.

Philox4x64-10 is fixed by its published definition (Salmon et al., SC'11);
numpy ships an independent implementation (``numpy.random.Philox``, which
increments its 256-bit counter before each block), so the oracle must agree
with it word for word.
"""
import numpy as np


def _numpy_block(ctr, key):
    c = 0
    for k, w in enumerate(ctr):
        c |= int(w) << (64 * k)
    c = (c - 1) % (1 << 256)  # numpy increments before producing a block
    words = np.array([(c >> (64 * k)) & (2**64 - 1) for k in range(4)], dtype=np.uint64)
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=words)
    return [int(x) for x in bg.random_raw(4)]


def test_philox_matches_numpy(orc):
    rng = np.random.default_rng(7)
    cases = [([0, 0, 0, 0], [0, 0]), ([1, 0, 0, 0], [0, 0]),
             ([2**64 - 1] * 4, [2**64 - 1] * 2), ([123456, 5000, 3, 0], [0, orc.TAG_SEE])]
    for _ in range(40):
        cases.append(([int(x) for x in rng.integers(0, 2**63, 4)],
                      [int(x) for x in rng.integers(0, 2**63, 2)]))
    for ctr, key in cases:
        assert orc.philox4x64_10(ctr, key) == _numpy_block(ctr, key), (ctr, key)


def test_philox_known_block(orc):
    # Zero counter and key: the first block of the published generator.
    assert orc.philox4x64_10([0, 0, 0, 0], [0, 0]) == [
        0x16554D9ECA36314C, 0xDB20FE9D672D0FDC, 0xD7E772CEE186176B, 0x7E68B68AEC7BA23B]


def test_u01_open_interval(orc):
    lo = orc.u01(0)
    hi = orc.u01(2**64 - 1)
    assert lo == 0.5 * 2.0**-52
    assert hi == 1.0 - 0.5 * 2.0**-52
    assert 0.0 < lo < hi < 1.0
    # only the top 52 bits matter, and every value is exact
    assert orc.u01(0xFFF) == lo
    assert orc.u01(1 << 12) == 1.5 * 2.0**-52
    rng = np.random.default_rng(3)
    for w in rng.integers(0, 2**63, 1000, dtype=np.uint64):
        k = int(w) >> 12
        assert orc.u01(int(w)) == (2 * k + 1) / 2.0**53
