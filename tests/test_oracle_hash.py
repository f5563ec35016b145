"""Pins for the oracle's hash and random draws against published values and
algebraic facts (not against a retyped formula)."""
import numpy as np

import oracle
from paper_1605_05236_gb300 import inputs


def test_fmix32_smhasher_vectors():
    # MurmurHash3_x86_32 of the empty input reduces to fmix32(seed); SMHasher's
    # published results for seeds 0, 1 and 0xFFFFFFFF are 0, 0x514E28B7 and
    # 0x81F16F39.
    assert oracle.fmix32(0) == 0
    assert oracle.fmix32(1) == 0x514E28B7
    assert oracle.fmix32(0xFFFFFFFF) == 0x81F16F39


def _inv_xorshift(y, s, bits=32):
    x = y
    for _ in range(bits // s + 1):
        x = y ^ (x >> s)
    return x & ((1 << bits) - 1)


def test_fmix32_is_a_bijection():
    # Undo each step with the modular inverse of the multipliers: a dropped or
    # altered step in the oracle makes the round trip fail.
    m = 1 << 32
    i1, i2 = pow(0x85EBCA6B, -1, m), pow(0xC2B2AE35, -1, m)
    rng = np.random.default_rng(5)
    for x in rng.integers(0, m, 200, dtype=np.uint64):
        h = oracle.fmix32(int(x))
        y = _inv_xorshift(h, 16)
        y = (y * i2) % m
        y = _inv_xorshift(y, 13)
        y = (y * i1) % m
        y = _inv_xorshift(y, 16)
        assert y == int(x)


def test_splitmix64_published_vector():
    # SplitMix64 seeded with 0 (Vigna's reference generator): first outputs.
    assert oracle.splitmix64_at(0) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64_at(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4
    assert oracle.splitmix64_at(2 * 0x9E3779B97F4A7C15 % (1 << 64)) == 0x06C45D188009454F
    s = inputs.splitmix64_stream(0, 0, 3)
    assert [int(x) for x in s] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_bins_distinct_in_range_and_uniform():
    for d, n in ((2, 64), (3, 61), (4, 5), (2, 2), (4, 4)):
        t = oracle.OracleTable(n, 1 if d > 2 else 4, d, oracle.RANDOM)
        keys, _ = inputs.distinct_keys(4000, 9)
        counts = np.zeros(n)
        for k in keys[:4000]:
            b = t.bins_of(int(k))
            assert len(set(b)) == d and all(0 <= x < n for x in b)
            counts[b[0]] += 1
        if n >= 61:
            # first choice: chi-square over n cells, loose bound
            e = len(keys) / n
            chi = ((counts - e) ** 2 / e).sum()
            assert chi < 2 * n + 60


def test_first_bin_is_fmix_of_key_xor_seed_mod_n():
    # h_0(k) = fmix32(k ^ seed_0) mod n (the hash the library also uses):
    # the SMHasher vector above pins fmix32, so a key equal to seed_0 ^ 1
    # lands in bin 0x514E28B7 mod n.
    n = 1000
    t = oracle.OracleTable(n, 4, 2, oracle.RANDOM)
    assert t.bins_of(0x9E3779B9 ^ 1)[0] == 0x514E28B7 % n
    assert t.bins_of(0x9E3779B9)[0] == 0


def test_xor_seeded_family_swaps_bins_decorrelated_does_not():
    """Hash family 0, fmix32(k ^ seed_i), maps k' = k ^ seed_0 ^ seed_1 to
    k's first two bins swapped (an algebraic fact: k' ^ seed_0 = k ^ seed_1);
    family 1 breaks that structure."""
    n = 1 << 20
    t0 = oracle.OracleTable(n, 1, 3, oracle.RANDOM)
    t1 = oracle.OracleTable(n, 1, 3, oracle.RANDOM)
    t1.set_hash_family(1)
    keys, _ = inputs.distinct_keys(300, 77)
    swapped = 0
    for k in keys:
        k2 = int(k) ^ 0x9E3779B9 ^ 0x85EBCA6B
        a, b = t0.bins_of(int(k)), t0.bins_of(k2)
        if a[0] != a[1] and b[0] != b[1]:
            assert (b[0], b[1]) == (a[1], a[0])
        a1, b1 = t1.bins_of(int(k)), t1.bins_of(k2)
        swapped += (b1[0], b1[1]) == (a1[1], a1[0])
    assert swapped == 0
