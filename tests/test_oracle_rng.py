"""Pins of the oracle's counter-based RNG, its exp and its rank selection."""
import math
import os
import struct
from fractions import Fraction

import numpy as np

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers(oracle_mod):
    rows = [l.split() for l in open(os.path.join(GOLD, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle_mod.philox(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_stream_layout(oracle_mod):
    """word t of (seed, individual, generation, purpose) = lane t%4 of Philox(ctr=(t/4, i, g, p),
    key=(seed lo, seed hi))."""
    seed = 0x1234_5678_9ABC_DEF0
    for (i, g, p, t) in [(0, 0, 1, 0), (5, 7, 3, 6), (127, 499, 2, 13)]:
        blk = oracle_mod.philox([t // 4, i, g, p], [seed & 0xFFFFFFFF, seed >> 32])
        assert oracle_mod.rng_word(seed, i, g, p, t) == int(blk[t % 4])


def test_u01_exact(oracle_mod):
    for w in [0, 255, 256, 0xFFFFFFFF, 0x80000000, 12345678]:
        assert oracle_mod.lib().or_u01(w) == (w >> 8) / 2.0 ** 24


def _f32_bits(x):
    return struct.unpack("<i", struct.pack("<f", x))[0]


def test_exp_ct_error_bound(oracle_mod):
    """Cody-Waite + degree-7 Taylor exp within 2 ulp of the correctly rounded value on [-80, 0]."""
    xs = np.concatenate([np.linspace(-80.0, 0.0, 20001, dtype=np.float32),
                         -np.float32(2.0) ** -np.arange(1, 30, dtype=np.float32),
                         np.float32([0.0, -0.5, -0.34657359, -0.34657360, -1e-8])])
    worst = 0
    for x in xs:
        got = oracle_mod.exp_ct(float(x))
        ref = float(np.float32(math.exp(float(x))))
        worst = max(worst, abs(_f32_bits(got) - _f32_bits(ref)))
    assert worst <= 2
    assert oracle_mod.exp_ct(-81.0) == 0.0 and oracle_mod.exp_ct(0.0) == 1.0


def test_beta_pick_exact_boundaries(oracle_mod):
    """k is chosen iff w / 2^32 lies in [F(k-1), F(k)), F(k) = 1 - ((P-1-k)/P)^3 (Beta(1,3)
    shaped rank distribution); checked with exact rationals."""
    for P in (2, 3, 20, 128, 1024):
        for k in list(range(min(P, 6))) + [P // 2, P - 1]:
            Fk = 1 - Fraction(P - 1 - k, P) ** 3
            # smallest w with w/2^32 >= F(k) must map to k+1 (or clamp), the one below to <= k
            wb = math.ceil(Fk * 2 ** 32)
            if wb < 2 ** 32:
                assert oracle_mod.beta_pick(wb, P) == k + 1
            if 0 <= wb - 1 < 2 ** 32:
                assert oracle_mod.beta_pick(wb - 1, P) <= k
    # frequencies follow the pmf
    P = 20
    rng = np.random.default_rng(1)
    ws = rng.integers(0, 2 ** 32, 200000, dtype=np.uint64)
    picks = np.array([oracle_mod.beta_pick(int(w), P) for w in ws[:20000]])
    pmf = np.array([float((Fraction(P - k, P) ** 3) - Fraction(P - k - 1, P) ** 3) for k in range(P)])
    freq = np.bincount(picks, minlength=P) / len(picks)
    assert np.max(np.abs(freq - pmf)) < 0.01
    assert pmf[0] > pmf[-1] and abs(pmf.sum() - 1) < 1e-12
