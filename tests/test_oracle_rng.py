"""Pins of the oracle's counter-based Philox4x32-10 and Box-Muller normals.

The paper draws its Wiener increments from Philox4_32_10 (Sec. IV.A) and uses
dW = sqrt(ds) N(0,1) (Sec. III).  On the CPU the generator is pinned by the
statistical properties any correct Philox stream has (uniform words, balanced
bits, full avalanche over counter and key); the bit-exact pin against
NVIDIA's own Philox4_32_10 runs in the GPU suite.
"""
import math

import numpy as np
import pytest
from scipy import stats


def _ctr(n, step=0, tag=0, pid0=0):
    c = np.zeros((n, 4), np.uint32)
    c[:, 0] = step
    pid = np.arange(pid0, pid0 + n, dtype=np.uint64)
    c[:, 1] = (pid & 0xFFFFFFFF).astype(np.uint32)
    c[:, 2] = (pid >> np.uint64(32)).astype(np.uint32)
    c[:, 3] = tag
    return c


def test_philox_deterministic_and_distinct(orc):
    c = _ctr(100_000)
    a = orc.philox(c, (1, 0))
    b = orc.philox(c, (1, 0))
    assert np.array_equal(a, b)
    # a bijection of the counter for a fixed key: no repeated 128-bit blocks
    blocks = a.view(np.dtype((np.void, 16))).ravel()
    assert len(np.unique(blocks)) == len(blocks)
    # the key matters
    assert not np.array_equal(a, orc.philox(c, (2, 0)))
    assert not np.array_equal(a, orc.philox(c, (1, 1)))


def test_philox_words_uniform(orc):
    w = orc.philox(_ctr(250_000, step=3), (0xDEADBEEF, 0x12345678)).ravel()
    # chi^2 on the top 10 bits
    h = np.bincount(w >> np.uint32(22), minlength=1024)
    chi2, p = stats.chisquare(h)
    assert p > 1e-4, p
    # every bit position balanced (4 sigma)
    n = w.size
    for bit in range(32):
        ones = int(((w >> np.uint32(bit)) & np.uint32(1)).sum())
        assert abs(ones - n / 2) < 4 * math.sqrt(n / 4), (bit, ones)


@pytest.mark.parametrize("which", ["counter", "key"])
def test_philox_avalanche(orc, which):
    rng = np.random.default_rng(5)
    n = 4000
    c = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, size=2, dtype=np.uint64).astype(np.uint32)
    base = orc.philox(c, key)
    flips = []
    nbits = 128 if which == "counter" else 64
    for bit in range(0, nbits, 7):
        if which == "counter":
            c2 = c.copy()
            c2[:, bit // 32] ^= np.uint32(1 << (bit % 32))
            other = orc.philox(c2, key)
        else:
            k2 = key.copy()
            k2[bit // 32] ^= np.uint32(1 << (bit % 32))
            other = orc.philox(c, k2)
        x = base ^ other
        nb = np.unpackbits(x.view(np.uint8), axis=None).reshape(n, 128).sum(axis=1)
        flips.append(nb.mean())
    flips = np.asarray(flips)
    # each flipped input bit changes half of the 128 output bits on average
    assert np.all(np.abs(flips - 64.0) < 0.5), flips


def test_normals_moments_and_law(orc):
    n = 400_000
    z = orc.normals(1, 0, n, 17)
    for j in range(3):
        x = z[:, j]
        assert abs(x.mean()) < 5 / math.sqrt(n)
        assert abs(x.var() - 1.0) < 5 * math.sqrt(2.0 / n)
        assert abs(stats.skew(x)) < 5 * math.sqrt(6.0 / n)
        assert abs(stats.kurtosis(x)) < 5 * math.sqrt(24.0 / n)
        assert stats.kstest(x, "norm").pvalue > 1e-4
    c = np.corrcoef(z.T)
    assert np.all(np.abs(c - np.eye(3)) < 5 / math.sqrt(n))
    # consecutive steps of one particle are independent
    z2 = orc.normals(1, 0, n, 18)
    assert abs(np.corrcoef(z[:, 0], z2[:, 0])[0, 1]) < 5 / math.sqrt(n)


def test_normals_tail_bound(orc):
    # u = (x + 1/2) 2^-32 is never 0 or 1, so every normal is finite and
    # bounded by sqrt(-2 ln(2^-33)) ~ 6.76
    z = orc.normals(99, 0, 200_000, 0)
    assert np.all(np.isfinite(z))
    assert np.abs(z).max() < math.sqrt(-2.0 * math.log(2.0**-33)) + 1e-12


def test_normals_keyed_by_particle_not_slot(orc):
    # the stream of particle pid does not depend on which other particles are drawn
    a = orc.normals(3, 1000, 10, 5)
    b = orc.normals(3, 1005, 3, 5)
    assert np.array_equal(a[5:8], b)
