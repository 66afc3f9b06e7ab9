"""The cluster lowers the sample-to-sample variance of bonds inside it (Sec. II.B, Fig. Var).

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
