"""Pins of the oracle's photon synthesis against published values and statistics."""
import os

import numpy as np
import pytest
from scipy import stats

import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers(orc):
    for ctr, key, want in _kat():
        assert list(orc.philox(ctr, key)) == want


def test_poisson_fixed_point_matches_inverse_cdf(orc):
    """The fixed-point inversion returns the Poisson quantile of u / 2^32 except
    within 1e-9 of a CDF step (fixed-point truncation)."""
    rng = np.random.default_rng(0)
    for mu in (0.05, 0.7, 3.0, 9.5, 16.0):
        parts, p0, mfx = scenes.generator._poisson_fixed(np.array([mu]))
        assert parts[0] == 1
        us = np.concatenate([rng.integers(0, 2 ** 32, 4000, dtype=np.uint64),
                             np.array([0, 1, 2 ** 32 - 1], dtype=np.uint64)])
        for u in us:
            k = orc.poisson_fixed(int(u), int(p0[0]), int(mfx[0]))
            q = (int(u) + 0.5) / 2.0 ** 32
            want = int(stats.poisson.ppf(q, mu))
            if k != want:
                edge = stats.poisson.cdf(min(k, want), mu)
                assert abs(edge - q) < 1e-9, (mu, u, k, want)


def test_irf_thresholds_cover_pmf():
    irf = scenes.gamma_irf(3, 5, 80)
    pmf = scenes.generator.quantised_irf_pmf(irf)
    assert abs(pmf.sum() - 1.0) < 1e-12
    np.testing.assert_allclose(pmf, irf.normalised(), atol=2e-9)


def test_histogram_moments_match_model(orc):
    """Per-bin mean and variance of many synthesised histograms agree with the
    expected counts (Poisson: variance = mean) within 4 sigma."""
    base = scenes.Scene(
        h=1, w=3, t=48,
        depth=np.array([[[10.25, 20.0, np.nan]], [[30.6, np.nan, 5.5]]]),
        signal=np.array([[[4.0, 2.5, 0.0]], [[3.0, 0.0, 40.0]]]),
        bkg=np.full((1, 3), 0.05), irf=scenes.gaussian_irf(2.0, 6), seed=0)
    lam = scenes.expected_histogram(base)
    n = 4000
    acc = np.zeros(lam.shape)
    acc2 = np.zeros(lam.shape)
    for s in range(n):
        sc = scenes.Scene(**{**base.__dict__, "seed": 1000 + s})
        z = orc.synthesize(scenes.sampling_tables(sc)).astype(np.float64)
        acc += z
        acc2 += z * z
    mean = acc / n
    var = acc2 / n - mean ** 2
    se = np.sqrt(np.maximum(lam, 1e-3) / n)
    assert np.all(np.abs(mean - lam) < 4.5 * se + 1e-3)
    big = lam > 0.5
    np.testing.assert_allclose(var[big], lam[big], rtol=0.2)
    # total photons of the 40-photon surface (split into 3 Poisson parts)
    tot = acc[0, 2].sum() / n
    assert abs(tot - (40.0 + 0.05 * 48)) < 4.5 * np.sqrt(42.4 / n)


def test_synthesis_deterministic_and_seeded(orc):
    sc = scenes.small_random(5, 7, 96, seed=3)
    tab = scenes.sampling_tables(sc)
    a = orc.synthesize(tab)
    b = orc.synthesize(tab)
    c = orc.synthesize(tab, seed=tab["seed"] + 1)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)
