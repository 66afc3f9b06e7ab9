"""Pins of oracle/u1.py: total-S^z block-sparse evolution (Sec. II.C, Fig. qn).

* Without truncation the block evolution gives the dense oracle's state,
  and that state is the dense Trotterised evolver's (1e-12).
* With truncation the block-sparse chain gives the dense chain's
  (S^z-basis) samples: same observables (1e-10 relative), same collapse
  outcomes.  The kept set is the same because the singular values of a
  block-diagonal matrix are the union of its blocks' values.
* Every tensor obeys the charge rule, and the right edge carries Q, the sum
  of the environment's m values.
* METTS (2W = 0) keeps Q from sample to sample.  The hybrid chain's Q
  fluctuates.  The pure-ancilla state has Q = 0.
* The blocks are smaller than theta, so the blocked SVD work is a fraction
  of the dense one.
"""
import math

import numpy as np
import pytest

from oracle import chain, collapse, ed, model, mps, u1


def _evolve_both(Lx, two_W, seed, chi_max, cutoff, beta=0.6, tau=0.1, sched=model.SCHEDULE_PLAIN):
    lad = model.Ladder(Lx, two_W, 1.0, 0.7)
    n, teff = model.trotter_steps(beta, tau)
    ops, gates = model.schedule(lad, n, teff, sched)
    env = collapse.initial_env(len(lad.env), seed, 0)
    dense = mps.evolve(mps.MPS(collapse.product_state(lad, env, collapse.BASIS_Z)), ops, gates, chi_max, cutoff)
    st = u1.product_state(lad, env)
    assert st.violation() == 0.0
    sizes = []
    u1.evolve(st, ops, gates, chi_max, cutoff, sizes)
    return lad, env, n, teff, dense, st, sizes


@pytest.mark.parametrize("Lx,two_W,sched", [(3, 2, "plain"), (2, 4, "plain"), (3, 0, "plain"),
                                             (3, 2, "fused"), (2, 2, "fused")])
def test_block_evolution_equals_dense_without_truncation(Lx, two_W, sched):
    lad, env, n, teff, dense, st, _ = _evolve_both(Lx, two_W, 3, 3 ** 12, 0.0, sched=sched)
    v, w = st.to_dense(), dense.to_dense()
    assert st.centre == 0
    assert np.abs(v - np.sign(v @ w) * w).max() < 1e-12
    phi, nrm = ed.dense_evolve(lad, env, np.eye(3), n, teff)
    psi = phi.reshape(-1) / math.sqrt(nrm)
    assert np.abs(v - np.sign(v @ psi) * psi).max() < 1e-12
    assert st.violation() < 1e-14
    assert st.total_charge == sum(int(u1.M_OF[s]) for s in env)


def test_charge_labels_follow_every_op():
    _, env, _, _, _, st, sizes = _evolve_both(4, 4, 1, 64, 1e-12, beta=1.0)
    assert st.violation() < 1e-14
    assert all(len(q) == t.shape[2] for q, t in zip(st.q[1:], st.tensors))
    assert len(st.q[0]) == 1 and st.q[0][0] == 0
    assert st.total_charge == sum(int(u1.M_OF[s]) for s in env)
    # every split decomposed at least two blocks once the state spreads
    assert max(len(b) for b in sizes) >= 3


@pytest.mark.parametrize("cfg", [
    dict(Lx=4, two_W=4, J_leg=1.0, J_rung=1.0, beta=2.0, tau=0.1, chi_max=64, cutoff=1e-12),
    dict(Lx=5, two_W=2, J_leg=1.0, J_rung=1.0, beta=0.8, tau=0.1, chi_max=12, cutoff=1e-8),
    dict(Lx=4, two_W=0, J_leg=1.0, J_rung=0.5, beta=1.0, tau=0.1, chi_max=27, cutoff=1e-10),
])
def test_block_chain_reproduces_dense_z_chain(cfg):
    dense = chain.HybridChain(seed=2, chain_id=4, basis_zx=False, **cfg)
    block = u1.U1Chain(seed=2, chain_id=4, **cfg)
    for _ in range(3):
        r0, r1 = dense.sample(), block.sample()
        assert np.allclose(r1["obs"], r0["obs"], rtol=1e-10, atol=1e-12)
        assert r1["env_out"] == r0["env_out"]
        assert abs(r1["logp"] - r0["logp"]) < 1e-9
        assert r1["Q"] == sum(int(u1.M_OF[s]) for s in r0["env_in"])
        assert block.last_mps.violation() < 1e-12


def test_metts_stays_in_one_sector_and_hybrid_does_not():
    """Fig. qn: collapsing every site keeps Q; collapsing the environment only
    lets Q move from sample to sample (both in the S^z basis)."""
    base = dict(J_leg=1.0, J_rung=1.0, beta=1.0, tau=0.1, chi_max=27, cutoff=1e-10, seed=7)
    metts = u1.U1Chain(3, 0, **base)
    qs_m = [metts.sample()["Q"] for _ in range(12)]
    assert len(set(qs_m)) == 1
    hyb = u1.U1Chain(3, 2, **base)
    qs_h = [hyb.sample()["Q"] for _ in range(40)]
    assert len(set(qs_h)) >= 3
    assert abs(np.mean(qs_h)) < 1.5                      # centred near S^z = 0
    anc = u1.U1Chain(2, 4, **base)
    assert {anc.sample()["Q"] for _ in range(3)} == {0}


def test_blocked_svd_work_is_a_fraction_of_dense():
    _, _, _, _, _, _, sizes = _evolve_both(4, 4, 0, 64, 1e-12, beta=1.0)
    dense = blocked = 0.0
    for blocks in sizes:
        m = sum(r for r, _ in blocks)
        n = sum(c for _, c in blocks)
        dense += u1.svd_cost(m, n)
        blocked += sum(u1.svd_cost(r, c) for r, c in blocks if r and c)
    assert blocked < 0.35 * dense


def test_x_basis_rejected():
    with pytest.raises(ValueError):
        u1.U1Chain(3, 2, basis_zx=True)
