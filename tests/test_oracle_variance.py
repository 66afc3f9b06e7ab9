"""The cluster lowers the sample-to-sample variance of bonds inside it (Sec. II.B, Fig. Var),
and raises the work per sample (the other side of the trade-off).

Per-sample <S_x,0 . S_x,1> on every rung of an Lx=4 ladder (beta=1), from
seeded oracle chains: with the central column paired with ancillas (2W=2)
the rung inside the cluster fluctuates far less than the environment rungs
and than the same rung in plain METTS (2W=0); with every site paired
(pure ancilla) nothing fluctuates.  Deterministic (fixed seeds).
"""
import numpy as np
import pytest

from oracle.chain import HybridChain


def _rung_samples(two_W, n=25):
    Lx = 4
    ch = HybridChain(Lx, two_W, 1.0, 1.0, beta=1.0, tau=0.1, chi_max=32, cutoff=1e-10, seed=1,
                     meas_cols=(0, Lx))
    rungs = []
    for x in range(Lx):
        key = (ch.ladder.phys[(x, 0)], ch.ladder.phys[(x, 1)])
        rungs.append(next(b for b, (i, j, _) in enumerate(ch.meas_bonds) if (i, j) == key))
    for _ in range(3):
        ch.sample()
    vals = np.array([[ch.sample()["obs"][1 + 2 * b] for b in rungs] for _ in range(n)])
    return ch, vals


@pytest.mark.slow
def test_cluster_rung_variance_is_lowest():
    hyb, v = _rung_samples(2)
    assert hyb.ladder.cluster_cols == [1]
    var = v.var(axis=0)
    env = [var[x] for x in (0, 2, 3)]
    assert var[1] < 0.2 * min(env)
    _, m = _rung_samples(0)
    assert var[1] < 0.2 * m.var(axis=0)[1]


def test_pure_ancilla_has_no_variance():
    _, v = _rung_samples(8, n=3)
    assert np.abs(v - v[0]).max() < 1e-12


def _flops(log):
    """Algorithmic count of one evolution: theta GEMM, gate, dense-SVD count."""
    tot = 0.0
    for kind, _, cl, cm, cr, _, _ in log:
        if kind != 0:
            continue
        m, n = 3 * cl, 3 * cr
        M, N = max(m, n), min(m, n)
        tot += 2 * cl * 3 * cm * 3 * cr + 162 * cl * cr + 4 * M * M * N + 8 * M * N * N + 9 * N ** 3
    return tot


def test_cost_per_sample_grows_with_the_cluster():
    """The other side of the trade-off (Sec. II.B): pairing more sites with
    ancillas entangles the state more, so bonds and the work per sample
    grow from METTS (2W = 0) to the ancilla method (2W = 2 Lx)."""
    Lx, cost, chi = 5, [], []
    for two_W in (0, 4, 10):
        ch = HybridChain(Lx, two_W, 1.0, 1.0, beta=1.0, tau=0.1, chi_max=128, cutoff=1e-8, seed=2)
        log = []
        ch.sample(log)
        cost.append(_flops(log))
        chi.append(max(r[5] for r in log if r[0] == 0))
    assert cost[0] < cost[1] < cost[2]
    assert chi[0] < chi[1] <= chi[2]
