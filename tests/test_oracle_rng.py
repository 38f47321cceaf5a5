"""Pins of the oracle's random-number path (Algorithm 4 and the Box-Muller
transform of Sec. 3.5) against values fixed outside the oracle: published and
hand-traced TEA vectors, bit-reversal identities, the Gaussian distribution
and the symmetry the pair hash must have."""
import math
import os

import numpy as np
import pytest

import oracle




def _tea_rows(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "tea_vectors.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            t = line.split()
            rows.append((int(t[0]), [int(x, 16) for x in t[1:5]], int(t[5], 16), int(t[6], 16),
                         int(t[7], 16), int(t[8], 16)))
    return rows


def test_tea_known_answers(golden_dir):
    rows = _tea_rows(golden_dir)
    assert len(rows) == 3
    for rounds, key, v0, v1, e0, e1 in rows:
        assert oracle.tea(rounds, key, v0, v1) == (e0, e1)


def test_key_reading():
    # k0/k1 = low/high words of the seed, k2/k3 = the fixed hex digits of pi
    assert oracle.key(42) == [42, 0, 0x243F6A88, 0x85A308D3]
    assert oracle.key((7 << 32) | 9) == [9, 7, 0x243F6A88, 0x85A308D3]


def test_tea_rounds_compose():
    # n rounds then m more is not n+m rounds (sum restarts) -- but 0 rounds
    # is the identity and the map is a bijection on small samples
    k = oracle.key(42)
    assert oracle.tea(0, k, 123, 456) == (123, 456)
    outs = {oracle.tea(4, k, a, b) for a in range(40) for b in range(40)}
    assert len(outs) == 1600


def test_bitrev():
    assert oracle.bitrev32(1) == 0x80000000
    assert oracle.bitrev32(0x80000000) == 1
    assert oracle.bitrev32(0x12345678) == 0x1E6A2C48
    assert oracle.bitrev32(0xFFFFFFFF) == 0xFFFFFFFF
    assert oracle.bitrev32(0x0000FFFF) == 0xFFFF0000
    for x in (0, 3, 0xDEADBEEF, 0x9E3779B9):
        assert oracle.bitrev32(oracle.bitrev32(x)) == x


def test_signature_definition():
    # signature = v0 ^ v1 after 16 TEA rounds on (bitrev(tag), step)
    k = oracle.key(42)
    v0, v1 = oracle.tea(16, k, oracle.bitrev32(5), 7)
    assert oracle.signature(42, 5, 7) == v0 ^ v1
    # only the low 32 bits of the step enter
    assert oracle.signature(42, 5, 7 + (1 << 32)) == oracle.signature(42, 5, 7)
    sigs = {oracle.signature(42, t, 3) for t in range(5000)}
    assert len(sigs) == 5000


def test_pair_hash_symmetric_and_keyed():
    for (i, j) in [(0, 1), (17, 4), (123456, 7)]:
        assert oracle.pair_hash(42, 9, i, j) == oracle.pair_hash(42, 9, j, i)
        assert oracle.xi(42, 9, i, j) == oracle.xi(42, 9, j, i)
    assert oracle.pair_hash(42, 9, 0, 1) != oracle.pair_hash(42, 10, 0, 1)
    assert oracle.pair_hash(42, 9, 0, 1) != oracle.pair_hash(43, 9, 0, 1)
    si, sj = oracle.signature(42, 3, 5), oracle.signature(42, 8, 5)
    assert oracle.pair_hash(42, 5, 3, 8) == oracle.tea(4, oracle.key(42), min(si, sj), max(si, sj))


def test_pair_hash_batch_is_the_per_pair_hash():
    # the batched call (used for the all-pairs GPU comparison) marshals the
    # same per-pair routine: composition from the signatures, symmetric
    rng = np.random.default_rng(3)
    ti = rng.integers(0, 2**32, 64, dtype=np.uint64).astype(np.uint32)
    tj = rng.integers(0, 2**32, 64, dtype=np.uint64).astype(np.uint32)
    hb = oracle.pair_hash_batch(42, 11, ti, tj)
    for k in range(64):
        si, sj = oracle.signature(42, int(ti[k]), 11), oracle.signature(42, int(tj[k]), 11)
        assert tuple(int(w) for w in hb[k]) == oracle.tea(4, oracle.key(42), min(si, sj), max(si, sj))
    assert np.array_equal(hb, oracle.pair_hash_batch(42, 11, tj, ti))


def test_box_muller_special_values():
    # u1 = 1 (a = 2^32 - 1): radius sqrt(-2 ln 1) = 0
    assert oracle.gauss(0xFFFFFFFF, 12345) == 0.0
    # b = 0: phase 0, cos = 1, sign +; b = 2^31: same phase, sign -
    g = oracle.gauss(1000, 0)
    assert g > 0 and oracle.gauss(1000, 0x80000000) == -g
    # u2 = 1/2: cos(pi/2) = 0
    assert abs(oracle.gauss(1000, 0x40000000)) < 1e-15
    # radius at u1 = 2^-32 * (a + 1) with a = 2^32 e^{-1/2} - 1 is close to 1
    a = int(round(2**32 * math.exp(-0.5))) - 1
    assert abs(oracle.gauss(a, 0) - 1.0) < 1e-9


def test_gaussian_moments_and_ks():
    """E7 of the paper: the pair random numbers are standard normal up to the
    4th moment; here also a Kolmogorov-Smirnov distance against Phi."""
    m = 2_000_000
    ti = np.arange(m, dtype=np.uint32) * 2
    tj = ti + 1
    z = oracle.xi_batch(42, 1, ti, tj)
    mean = z.mean()
    var = z.var()
    skew = ((z - mean) ** 3).mean() / var ** 1.5
    kurt = ((z - mean) ** 4).mean() / var ** 2
    se = 1.0 / math.sqrt(m)
    assert abs(mean) < 5 * se
    assert abs(var - 1.0) < 5 * math.sqrt(2.0) * se
    assert abs(skew) < 5 * math.sqrt(6.0) * se
    assert abs(kurt - 3.0) < 5 * math.sqrt(24.0) * se
    zs = np.sort(z[:200_000])
    cdf = 0.5 * (1.0 + np.vectorize(math.erf)(zs / math.sqrt(2.0)))
    n = zs.size
    d = max(np.max(np.arange(1, n + 1) / n - cdf), np.max(cdf - np.arange(n) / n))
    assert d < 1.63 / math.sqrt(n)  # KS 1% critical value


def test_xi_uncorrelated_across_steps_and_pairs():
    m = 400_000
    ti = np.arange(m, dtype=np.uint32)
    tj = ti + 1
    z1 = oracle.xi_batch(42, 100, ti, tj)
    z2 = oracle.xi_batch(42, 101, ti, tj)
    assert abs(np.corrcoef(z1, z2)[0, 1]) < 5 / math.sqrt(m)
    # neighbouring pairs sharing a particle are uncorrelated too
    assert abs(np.corrcoef(z1[:-1], z1[1:])[0, 1]) < 5 / math.sqrt(m)
