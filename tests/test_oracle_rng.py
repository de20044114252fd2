"""Pins of the oracle's counter-based generator and samplers.

Known answers for the generator come from test_oracle_philox_kat.py (an
independent open-source Philox4x32-10); here it is also checked for the
properties any correct Philox4x32-10 has: uniform 32-bit output, strong
avalanche on single counter/key bit flips, and no correlation between
neighbouring counters. The samplers are pinned by their distributions."""
import math

import numpy as np
import pytest
from scipy import stats


def _block(orc, n, key=(7, 0), lane=0):
    out = np.empty((n, 4), np.uint64)
    for i in range(n):
        out[i] = orc.philox([i, lane, 0, 0], key)
    return out


def test_philox_uniform_bytes(orc):
    v = _block(orc, 4000).reshape(-1)
    # every byte lane uniform (chi-square over 256 cells)
    for shift in (0, 8, 16, 24):
        b = ((v >> np.uint64(shift)) & np.uint64(255)).astype(np.int64)
        chi2, p = stats.chisquare(np.bincount(b, minlength=256))
        assert p > 1e-4, (shift, p)


def test_philox_avalanche(orc):
    rng = np.random.default_rng(3)
    flips = []
    for _ in range(200):
        ctr = [int(x) for x in rng.integers(0, 2 ** 32, 4)]
        key = [int(x) for x in rng.integers(0, 2 ** 32, 2)]
        a = orc.philox(ctr, key)
        word, bit = int(rng.integers(0, 6)), int(rng.integers(0, 32))
        c2, k2 = list(ctr), list(key)
        if word < 4:
            c2[word] ^= 1 << bit
        else:
            k2[word - 4] ^= 1 << bit
        b = orc.philox(c2, k2)
        flips.append(sum(bin(x ^ y).count("1") for x, y in zip(a, b)))
    m = np.mean(flips)
    # 128 output bits: a random function flips 64 +- 5.7 bits
    assert abs(m - 64.0) < 2.0, m
    assert min(flips) > 30


def test_philox_counter_neighbours_uncorrelated(orc):
    v = _block(orc, 3000).astype(np.float64) / 2 ** 32
    for lane in range(4):
        r = np.corrcoef(v[:-1, lane], v[1:, lane])[0, 1]
        assert abs(r) < 0.06
    r01 = np.corrcoef(v[:, 0], v[:, 1])[0, 1]
    assert abs(r01) < 0.06


def test_uniform_map_exact_and_open(orc):
    u = np.concatenate([orc.uniforms(1, p, 0, 0, 0) for p in range(2000)])
    assert np.all(u > 0) and np.all(u < 1)
    k = u * 2 ** 23 - 0.5  # (x >> 9) recovered exactly
    assert np.all(k == np.round(k))
    assert stats.kstest(u, "uniform").pvalue > 1e-3


def test_beta_partition_moments(orc):
    """1-B for B ~ Beta(a, 2) via U1^(1/a) U2^(1/(a+1)): mean 2/(a+2), variance
    2a/((a+2)^2 (a+3))."""
    rng = np.random.default_rng(11)
    for a in (1.0, 3.0, 300.0, 6000.0):
        u = rng.random((40000, 2)) * (1 - 2 ** -24) + 2 ** -25
        omb = np.array([orc.one_minus_beta(a, x, y) for x, y in u])
        mean, var = 2.0 / (a + 2.0), 2.0 * a / ((a + 2.0) ** 2 * (a + 3.0))
        assert abs(omb.mean() - mean) < 4 * math.sqrt(var / len(omb))
        assert abs(omb.var() / var - 1) < 0.05
        # distribution: KS against scipy's Beta(2, a) for 1-B
        assert stats.kstest(omb, stats.beta(2.0, a).cdf).pvalue > 1e-3


def test_heat_capacity_profile(orc):
    from paper_2609_31258_b300 import workloads as W
    for ion in (W.ION_1KDA, W.ION_15KDA):
        for T in (1.0, 150.0, 300.0, 999.0, 1000.0, 1001.0, 2500.0):
            e = orc.eint_of_T(ion, T)
            assert abs(orc.T_of_eint(ion, e) - T) < 1e-9 * max(T, 1)
            h = 1e-3
            dEdT = (orc.eint_of_T(ion, T + h) - orc.eint_of_T(ion, T - h)) / (2 * h)
            if abs(T - 1000.0) > 1e-2:
                assert abs(dEdT - orc.cv_of_T(ion, T)) < 1e-6 * dEdT
    # classical: E = 3 N T exactly, linear fit capped at 3N above 1000 K
    assert orc.eint_of_T(W.ION_1KDA, 300.0) == 3 * 100 * 300.0
    assert orc.cv_of_T(W.ION_15KDA, 2000.0) == 3 * 2000
    assert abs(orc.cv_of_T(W.ION_15KDA, 500.0) - 3 * 2000 * (0.3 + 0.35)) < 1e-9


def test_rf_scalar_phase(orc):
    from paper_2609_31258_b300 import workloads as W
    run = W.Run(dt=0.5e-9, v_rf=100.0, f_rf=1e6, phi_rf=-math.pi / 2)
    # period is exactly 2000 steps; phase -90 deg gives sin(2 pi f t)
    for n in (0, 1, 250, 500, 1999, 2000, 123456):
        s = orc.rf_scalar(run, n)
        assert abs(s - 100.0 * math.sin(2 * math.pi * (n % 2000) / 2000)) < 1e-9
        assert abs(s - orc.rf_scalar(run, n + 2000 * 37)) < 1e-9
    assert orc.rf_scalar(W.Run(dt=1e-9), 5) == 0.0
