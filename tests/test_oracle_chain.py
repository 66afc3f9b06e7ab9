"""Pins of oracle/chain.py: limits and thermal averages of the hybrid chain.

* beta = 0: the state is the initial state, so cluster-internal bonds are
  maximally mixed (<S.S> = 0 exactly) and environment bonds give m_i m_j;
* unbiasedness (Sec. I.C, "does not bias the outcome"): chain averages agree
  with the exact Trotterised thermal average within 3 sigma (binning error);
* Markov step bookkeeping: alternating Sz / Sx collapse bases.
"""
import numpy as np
import pytest

from oracle import chain, collapse, ed, model


def test_beta_zero_sample_values():
    ch = chain.HybridChain(4, 4, 1.0, 1.0, beta=0.0, tau=0.1, chi_max=16, cutoff=1e-12,
                           seed=3, meas_cols=(0, 4))
    sz = np.diag([1.0, 0.0, -1.0])
    m_of = {k: 1.0 - o for k, o in zip(ch.ladder.env, ch.env)}
    rec = ch.sample()
    for b, (i, j, J) in enumerate(ch.meas_bonds):
        ss, zz = rec["obs"][1 + 2 * b], rec["obs"][2 + 2 * b]
        if i in m_of and j in m_of:
            assert abs(zz - m_of[i] * m_of[j]) < 1e-14
            assert abs(ss - m_of[i] * m_of[j]) < 1e-14   # product z states: <S+S-> = 0
        else:
            assert abs(ss) < 1e-14 and abs(zz) < 1e-14
    assert sz is not None
    # the next sample is collapsed in the x basis (n = 0 -> z, n = 1 -> x)
    assert rec["basis"] == collapse.BASIS_Z
    assert ch.sample()["basis"] == collapse.BASIS_X


def _thermal_target(ch, Lx):
    lad = ch.ladder
    inv = {k: (x, y) for (x, y), k in lad.phys.items()}
    bonds_xy = [(inv[i], inv[j], J) for i, j, J in lad.bonds]
    hm = sum(J * ed.dense_bond_operator(Lx, inv[i], inv[j], "ss") for i, j, J in ch.meas_bonds)
    (val,) = ed.trotter_thermal(Lx, bonds_xy, ch.n_steps, ch.tau_eff, [hm])
    return val


@pytest.mark.slow
@pytest.mark.parametrize("two_W,basis_zx", [(2, True), (0, True), (2, False)])
def test_thermal_average_within_3_sigma(two_W, basis_zx):
    Lx = 3
    ch = chain.HybridChain(Lx, two_W, 1.0, 0.5, beta=1.0, tau=0.1, chi_max=64, cutoff=1e-12,
                           seed=1, basis_zx=basis_zx, meas_cols=(0, Lx))
    for _ in range(5):
        ch.sample()
    e = [ch.sample()["obs"][0] for _ in range(120)]
    mean, err = chain.binned_error(e, 12)
    target = _thermal_target(ch, Lx)
    assert abs(mean - target) < 3 * err + 1e-12, (mean, err, target)
    assert err > 0.0


def test_binned_error():
    x = np.arange(100.0)
    m, e = chain.binned_error(x, 10)
    assert m == 49.5 and e > 0
    with pytest.raises(ValueError):
        chain.binned_error([1.0], 2)
    assert model is not None


@pytest.mark.parametrize("basis_zx,cut", [(True, 2), (True, 3), (False, 2)])
def test_resume_from_checkpoint_is_exact(basis_zx, cut):
    """Between samples a chain is only its environment outcomes and the sample
    index: step 4 resets the cluster to Bell pairs.  A chain rebuilt from the
    outcomes of sample cut-1 (read in that sample's basis) and index cut
    draws exactly what the uninterrupted chain draws."""
    cfg = dict(Lx=3, two_W=2, J_leg=1.0, J_rung=0.7, beta=0.6, tau=0.1, chi_max=16, cutoff=1e-10,
               seed=9, chain_id=2, basis_zx=basis_zx)
    full = chain.HybridChain(**cfg)
    recs = [full.sample() for _ in range(cut + 2)]
    res = chain.HybridChain(**cfg)
    res.env = list(recs[cut - 1]["env_out"])
    res.env_basis = collapse.sample_basis(cut - 1, basis_zx)     # derived from the index alone
    assert res.env_basis == recs[cut - 1]["basis"]
    res.n = cut
    for r in recs[cut:]:
        q = res.sample()
        assert np.array_equal(q["obs"], r["obs"]) and q["env_out"] == r["env_out"] and q["logp"] == r["logp"]
