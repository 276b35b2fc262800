"""Host-side Monte Carlo diagnostics of sampler output (no sampler arithmetic).

* effective sample size by Geyer's initial monotone sequence estimator
  (Geyer 1992, "Practical Markov chain Monte Carlo", Stat. Sci. 7);
* batch-means standard errors;
* pairwise merge of (count, mean, M2) moment accumulators across independent
  chains (Chan, Golub & LeVeque 1979), used to combine replica chains run on
  separate GPUs.
"""
from __future__ import annotations

import numpy as np


def autocovariance(x: np.ndarray) -> np.ndarray:
    """Biased sample autocovariances gamma_0..gamma_{n-1} of a 1-D series (FFT)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    d = x - x.mean()
    nfft = 1 << int(np.ceil(np.log2(2 * n)))
    f = np.fft.rfft(d, nfft)
    ac = np.fft.irfft(f * np.conj(f), nfft)[:n]
    return ac / n


def ess_geyer(x: np.ndarray) -> float:
    """ESS = N / tau with tau = -1 + 2 sum_m Gamma_m / gamma_0, where
    Gamma_m = gamma_{2m} + gamma_{2m+1} is summed while positive and forced
    to be non-increasing (initial monotone sequence)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    if n < 4:
        return float(n)
    g = autocovariance(x)
    if g[0] <= 0.0:
        return float(n)
    m_max = (n - 1) // 2
    pairs = g[0:2 * m_max:2] + g[1:2 * m_max + 1:2]
    total = 0.0
    prev = np.inf
    for G in pairs:
        if G <= 0.0:
            break
        G = min(G, prev)
        total += G
        prev = G
    tau = -1.0 + 2.0 * total / g[0]
    tau = max(tau, 1.0 / n)
    return float(n / tau)


def batch_means_se(x: np.ndarray, n_batches: int = 50) -> np.ndarray:
    """Standard error of the mean from n_batches contiguous batch means (per column)."""
    x = np.asarray(x, dtype=np.float64)
    b = x.shape[0] // n_batches
    bm = x[: b * n_batches].reshape(n_batches, b, *x.shape[1:]).mean(axis=1)
    return bm.std(axis=0, ddof=1) / np.sqrt(n_batches)


def merge_moments(n_a, mean_a, m2_a, n_b, mean_b, m2_b):
    """Combine two (count, mean, sum of squared deviations) accumulators."""
    n = n_a + n_b
    delta = mean_b - mean_a
    mean = mean_a + delta * (n_b / n)
    m2 = m2_a + m2_b + delta * delta * (n_a * n_b / n)
    return n, mean, m2
