"""Host-side statistics of many chains and their merge across ranks (no GPU).

Pins: the binned error of one chain equals the oracle's ``binned_error``
(an independent implementation); sums of interleaved chains equal the sums
of per-chain estimators merged; two gloo ranks that all-reduce their
estimators get the single-process result.
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import chain as ochain
from paper_1910_09142_gb300.estimators import Estimator


def _ar1(n, n_obs, seed, rho=0.8):
    """Correlated synthetic series (AR(1)), shape (n, n_obs)."""
    rng = np.random.default_rng(seed)
    x = np.zeros((n, n_obs))
    for t in range(1, n):
        x[t] = rho * x[t - 1] + rng.standard_normal(n_obs)
    return x - 3.0


def test_single_chain_matches_oracle_binning():
    x = _ar1(200, 3, 0)
    est = Estimator(3, bin_size=20)
    est.add(0, x)
    for q in range(3):
        m, e = ochain.binned_error(x[:, q], n_bins=10)
        assert abs(est.mean()[q] - m) < 1e-13
        assert abs(est.stderr()[q] - e) < 1e-13
    assert est.count == 200
    # correlated samples: the naive error underestimates the binned one
    assert np.all(est.naive_stderr() < est.stderr())


def test_warmup_and_open_bins():
    x = _ar1(27, 2, 1)
    est = Estimator(2, bin_size=10, n_warmup=5)
    for row in x:
        est.add("a", row)
    kept = x[5:]
    assert est.count == 22
    assert np.allclose(est.mean(), kept.mean(axis=0), rtol=0, atol=1e-13)
    assert est.sums[5][0] == 2                                  # bins 5..14, 15..24; 25, 26 open
    b = kept[:20].reshape(2, 10, 2).mean(axis=1)
    assert np.allclose(est.sums[3], b.sum(axis=0), atol=1e-13)


def test_interleaved_chains_equal_merged_estimators():
    xs = [_ar1(40 + 7 * c, 4, 10 + c) for c in range(4)]
    together = Estimator(4, bin_size=8, n_warmup=3)
    step = 0
    while any(step < len(x) for x in xs):
        for c, x in enumerate(xs):
            if step < len(x):
                together.add(c, x[step])
        step += 1
    merged = Estimator(4, bin_size=8, n_warmup=3)
    for c, x in enumerate(xs):
        e = Estimator(4, bin_size=8, n_warmup=3)
        e.add(c, x)
        merged.merge(e)
    assert np.allclose(together.sums, merged.sums, rtol=1e-14, atol=1e-12)
    allx = np.concatenate([x[3:] for x in xs])
    assert np.allclose(merged.mean(), allx.mean(axis=0), atol=1e-13)


def test_errors():
    with pytest.raises(ValueError):
        Estimator(0)
    e = Estimator(2, bin_size=4)
    with pytest.raises(ValueError):
        e.mean()
    e.add(0, np.ones((5, 2)))
    with pytest.raises(ValueError):
        e.stderr()                                              # one completed bin
    with pytest.raises(ValueError):
        e.merge(Estimator(2, bin_size=5))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        est = Estimator(3, bin_size=5, n_warmup=2)
        for c in range(rank * 3, rank * 3 + 3):                # this rank's chains
            est.add(c, _ar1(30, 3, 100 + c))
        est.all_reduce(dist)
        out[rank] = est.to_vector()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_all_reduce_to_the_single_process_sums():
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    ref = Estimator(3, bin_size=5, n_warmup=2)
    for c in range(6):
        ref.add(c, _ar1(30, 3, 100 + c))
    assert np.allclose(out[0], out[1], rtol=0, atol=0)
    assert np.allclose(out[0], ref.to_vector(), rtol=1e-14, atol=1e-12)


def test_all_reduce_without_process_group_is_identity():
    e = Estimator(1)
    e.add(0, np.arange(20.0))
    v = e.to_vector()
    e.all_reduce(dist)
    assert np.array_equal(e.to_vector(), v)
