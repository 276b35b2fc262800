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


def _initial_monotone_tau(rho: np.ndarray) -> float:
    """tau = -1 + 2 sum_m P_m, P_m = rho_{2m} + rho_{2m+1} summed while positive
    and forced non-increasing (Geyer's initial monotone sequence)."""
    n = rho.size
    m_max = (n - 1) // 2
    pairs = rho[0:2 * m_max:2] + rho[1:2 * m_max + 1:2]
    total, prev = 0.0, np.inf
    for P in pairs:
        if P <= 0.0:
            break
        P = min(P, prev)
        total += P
        prev = P
    return -1.0 + 2.0 * total


def ess_multichain(chains: np.ndarray, acov=None) -> float:
    """Effective sample size of K chains of length n (array [K, n]) together:
    the autocorrelation at lag t is 1 - (W - mean_k gamma_{k,t}) / var+,
    with W the mean within-chain variance and var+ = (n-1)/n W + B/n the
    pooled variance estimate (B = n times the variance of the chain means),
    then Geyer's initial monotone sequence; ESS = K n / tau (the multi-chain
    estimator of Gelman et al., Bayesian Data Analysis, 3rd ed., Sec. 11.5,
    without rank normalisation).  acov: the chains' autocovariances if already
    computed."""
    x = np.asarray(chains, dtype=np.float64)
    K, n = x.shape
    if n < 4:
        return float(K * n)
    g = np.array([autocovariance(c) for c in x]) if acov is None else acov
    g = g * (n / (n - 1.0))  # unbiased lag-0 variance: s_k^2 = g_k0 n / (n - 1)
    W = g[:, 0].mean()
    B = n * x.mean(axis=1).var(ddof=1) if K > 1 else 0.0
    var_plus = (n - 1.0) / n * W + B / n
    if var_plus <= 0.0:
        return float(K * n)
    rho = 1.0 - (W - g.mean(axis=0)) / var_plus
    tau = max(_initial_monotone_tau(rho), 1.0 / (K * n))
    return float(K * n / tau)


def split_rhat(chains: np.ndarray) -> float:
    """Split potential scale reduction: each chain cut into halves, then
    sqrt(var+ / W) over the 2K half chains (Gelman et al., Bayesian Data
    Analysis, 3rd ed., Sec. 11.4)."""
    x = np.asarray(chains, dtype=np.float64)
    K, n = x.shape
    h = n // 2
    halves = np.concatenate([x[:, :h], x[:, n - h:]], axis=0)
    W = halves.var(axis=1, ddof=1).mean()
    B = h * halves.mean(axis=1).var(ddof=1)
    var_plus = (h - 1.0) / h * W + B / h
    return float(np.sqrt(var_plus / W)) if W > 0 else float("nan")


def ess_chain_means(chains: np.ndarray) -> float:
    """ESS from the spread of independent chains' means: K var / var(chain
    means), var the pooled variance.  Valid when the chains start from
    independent draws of the target; a cross-check of ess_multichain."""
    x = np.asarray(chains, dtype=np.float64)
    K = x.shape[0]
    v = x.var()
    vm = x.mean(axis=1).var(ddof=1)
    return float(K * v / vm) if vm > 0 else float("inf")


def ess_with_se(chains: np.ndarray, n_boot: int = 200, seed: int = 0):
    """ess_multichain and its standard error by a bootstrap over chains
    (chains resampled with replacement; autocovariances computed once)."""
    x = np.asarray(chains, dtype=np.float64)
    K = x.shape[0]
    g = np.array([autocovariance(c) for c in x])
    est = ess_multichain(x, g)
    rng = np.random.default_rng(seed)
    boots = [ess_multichain(x[idx], g[idx]) for idx in (rng.integers(0, K, K) for _ in range(n_boot))]
    return est, float(np.std(boots, ddof=1))
