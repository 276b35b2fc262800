"""Pins of the host diagnostics: Geyer ESS against the closed form of an AR(1)
chain, batch-means SE against the iid formula, and the pairwise moment merge
against pooled numpy statistics (also across gloo ranks, the replica path)."""
import os

import numpy as np
import pytest

from paper_1103_4887_gb300 import diagnostics as dg


@pytest.mark.parametrize("rho", [0.0, 0.5, 0.9])
def test_ess_of_ar1_matches_closed_form(rho):
    # AR(1): tau = (1 + rho) / (1 - rho)
    rng = np.random.default_rng(3)
    n = 400_000
    e = rng.standard_normal(n)
    x = np.empty(n)
    x[0] = e[0] / np.sqrt(1 - rho ** 2)
    for i in range(1, n):
        x[i] = rho * x[i - 1] + e[i]
    expect = n * (1 - rho) / (1 + rho)
    assert abs(dg.ess_geyer(x) / expect - 1.0) < 0.06


def test_batch_means_se_iid():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((100_000, 3))
    se = dg.batch_means_se(x, 100)
    np.testing.assert_allclose(se, 1 / np.sqrt(100_000), rtol=0.25)


def test_merge_moments_equals_pooled():
    rng = np.random.default_rng(2)
    a = rng.standard_normal((500, 4)) + 3.0
    b = 2.0 * rng.standard_normal((800, 4)) - 1.0
    n, m, m2 = dg.merge_moments(len(a), a.mean(0), ((a - a.mean(0)) ** 2).sum(0),
                                len(b), b.mean(0), ((b - b.mean(0)) ** 2).sum(0))
    ab = np.vstack([a, b])
    assert n == 1300
    np.testing.assert_allclose(m, ab.mean(0), rtol=1e-12)
    np.testing.assert_allclose(m2 / (n - 1), ab.var(0, ddof=1), rtol=1e-12)


def _rank_merge(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(10 + rank)
    x = rng.standard_normal((300 + 50 * rank, 3)) + rank
    local = torch.tensor(np.concatenate([[len(x)], x.mean(0), ((x - x.mean(0)) ** 2).sum(0)]))
    parts = [torch.zeros_like(local) for _ in range(world)]
    dist.all_gather(parts, local)
    n, m, m2 = parts[0][0].item(), parts[0][1:4].numpy(), parts[0][4:7].numpy()
    for p in parts[1:]:
        n, m, m2 = dg.merge_moments(n, m, m2, p[0].item(), p[1:4].numpy(), p[4:7].numpy())
    if rank == 0:
        allx = np.vstack([np.random.default_rng(10 + r).standard_normal((300 + 50 * r, 3)) + r
                          for r in range(world)])
        out.put((np.abs(m - allx.mean(0)).max(), np.abs(m2 / (n - 1) - allx.var(0, ddof=1)).max()))
    dist.destroy_process_group()


def test_replica_moment_merge_over_gloo_ranks():
    """Replica chains on separate GPUs merge their moments on the host: two
    gloo ranks all-gather (count, mean, M2) and merge pairwise."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29511 + os.getpid() % 1000
    ps = [ctx.Process(target=_rank_merge, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
    assert all(p.exitcode == 0 for p in ps)
    dm, dv = q.get(timeout=10)
    assert dm < 1e-12 and dv < 1e-12


def _ar1_chains(K, n, phi, seed):
    rng = np.random.default_rng(seed)
    x = np.empty((K, n))
    x[:, 0] = rng.standard_normal(K) / np.sqrt(1 - phi * phi)  # stationary start
    e = rng.standard_normal((K, n))
    for t in range(1, n):
        x[:, t] = phi * x[:, t - 1] + e[:, t]
    return x


def test_multichain_ess_matches_ar1_closed_form():
    # AR(1): integrated autocorrelation time (1 + phi) / (1 - phi)
    for phi in (0.0, 0.5, 0.9):
        x = _ar1_chains(32, 4000, phi, seed=int(phi * 10))
        tau = (1 + phi) / (1 - phi)
        ess, se = dg.ess_with_se(x, n_boot=50)
        assert abs(ess - x.size / tau) < 4 * se + 0.05 * x.size / tau, (phi, ess, x.size / tau, se)
        assert dg.split_rhat(x) < 1.02
        # the chain-means estimate agrees within its own spread (relative SE ~ sqrt(2/(K-1)))
        cm = dg.ess_chain_means(x)
        assert abs(np.log(cm / (x.size / tau))) < 3 * np.sqrt(2 / 31), (phi, cm)


def test_multichain_ess_single_chain_equals_geyer():
    x = _ar1_chains(1, 5000, 0.7, seed=3)
    # one chain: B = 0 and var+ = (n-1)/n W, the pooled estimator is Geyer's up to that factor
    a = dg.ess_multichain(x)
    b = dg.ess_geyer(x[0])
    assert abs(a - b) / b < 0.01


def test_split_rhat_flags_chains_that_disagree():
    x = _ar1_chains(8, 2000, 0.5, seed=4)
    x[:4] += 3.0  # half the chains in another place
    assert dg.split_rhat(x) > 1.5
    y = _ar1_chains(8, 2000, 0.5, seed=5)
    y += np.linspace(0, 5, 2000)  # a drift within every chain
    assert dg.split_rhat(y) > 1.1
