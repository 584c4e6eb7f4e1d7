"""Pins of the oracle's sensor noise: Philox4x32-10 against the published
known-answer vectors, the Poisson sampler (inversion below 10, PTRS above)
against the exact pmf by chi-square and against the moments, the normal
deviates against N(0, 1), and the noise model's definition."""
import math

import numpy as np
import pytest

import oracle

stats = pytest.importorskip("scipy.stats")

# Random123's known-answer vectors for philox4x32-10: counter, key, output
KAT = [
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


@pytest.mark.parametrize("ctr,key,want", KAT)
def test_philox_known_answers(ctr, key, want):
    assert oracle.philox4x32(ctr, key) == want


def counts(lam, n=200_000, seed=7):
    img = np.full(n, lam, dtype=np.float32)
    k = oracle.sensor_noise(img, 1.0, 0.0, seed)
    assert np.array_equal(k, np.round(k)) and k.min() >= 0
    return k.astype(np.int64)


@pytest.mark.parametrize("lam", [0.3, 4.0, 9.75, 10.25, 37.0, 1000.0, 123456.0])
def test_poisson_matches_the_pmf(lam):
    lam = float(np.float32(lam))
    k = counts(lam)
    n = len(k)
    assert abs(k.mean() - lam) <= 5 * math.sqrt(lam / n)
    assert abs(k.var() / lam - 1) <= 5 * math.sqrt(2.0 / n) + 1e-3
    # chi-square over the central bins (expected count >= 20), tails merged
    lo, hi = int(stats.poisson.ppf(1e-4, lam)), int(stats.poisson.isf(1e-4, lam))
    edges = np.arange(lo, hi + 2)
    obs = np.histogram(k, bins=edges)[0].astype(float)
    exp = n * stats.poisson.pmf(edges[:-1], lam)
    keep = exp >= 20
    obs_t = np.array([obs[keep].sum(), n - obs[keep].sum()])
    exp_t = np.array([exp[keep].sum(), n - exp[keep].sum()])
    chi2 = ((obs[keep] - exp[keep]) ** 2 / exp[keep]).sum() + \
        (obs_t[1] - exp_t[1]) ** 2 / max(exp_t[1], 1e-9)
    dof = keep.sum()
    assert stats.chi2.sf(chi2, dof) > 1e-4, (lam, chi2, dof)


def test_normal_deviates():
    z = np.array([oracle.normal(3, i) for i in range(50_000)])
    assert abs(z.mean()) < 5 / math.sqrt(len(z))
    assert abs(z.var() - 1) < 5 * math.sqrt(2 / len(z))
    assert stats.kstest(z, "norm").pvalue > 1e-4


def test_noise_model_definition():
    rng = np.random.default_rng(1)
    img = rng.uniform(-0.2, 2.0, 4096).astype(np.float32)
    g, sigma, seed = 300.0, 2.5, 99
    out = oracle.sensor_noise(img, g, sigma, seed)
    for i in (0, 17, 4095):
        lam = g * max(float(img[i]), 0.0)
        want = (oracle.poisson(lam, seed, i) + sigma * oracle.normal(seed, i)) / g
        assert out[i] == want
    # same seed, same draw; another seed, another draw
    assert np.array_equal(out, oracle.sensor_noise(img, g, sigma, seed))
    assert not np.array_equal(out, oracle.sensor_noise(img, g, sigma, seed + 1))
    # negative intensities carry read noise only
    neg = img <= 0
    shot = oracle.sensor_noise(img, g, 0.0, seed)
    assert np.all(shot[neg] == 0.0)
