"""Pins of oracle/mps.py and oracle/measure.py.

* the truncation rule against its definition on hand-made spectra;
* the MPS evolution (swaps, splits, centre moves) against the dense
  Trotterised evolver, which applies the same gates directly to the physical
  legs with no SVD at all;
* cluster observables against dense expectation values;
* the pure-ancilla limit against the dense Trotter operator and ED.
"""
import math

import numpy as np
import pytest

from oracle import chain, collapse, ed, measure, model, mps


def test_truncation_rank_cutoff():
    s = np.array([1.0, 0.5, 1e-3, 1e-7])
    w = s ** 2
    # discarded weight after k=2 is (1e-6 + 1e-14)/sum ~ 8e-7
    assert mps.truncation_rank(s, 10, 1e-6) == 2
    assert mps.truncation_rank(s, 10, 7e-7) == 3
    assert mps.truncation_rank(s, 10, 0.0) == 4
    assert mps.truncation_rank(s, 1, 0.0) == 1
    assert mps.truncation_rank(s, 10, 1.0) == 1
    assert abs(w[2:].sum() / w.sum() - 8e-7) < 1e-9


def test_truncation_rank_keeps_multiplets_whole():
    s = np.array([1.0, 0.6, 0.6 * (1 - 1e-10), 0.6 * (1 - 2e-10), 0.1])
    assert mps.truncation_rank(s, 3, 0.0) == 1      # chi_max would cut the triplet
    assert mps.truncation_rank(s, 4, 0.0) == 4
    s2 = np.array([1.0, 1.0 - 1e-12, 0.5])
    assert mps.truncation_rank(s2, 1, 0.0) == 1      # never below 1


def test_truncation_rank_zero_matrix():
    with pytest.raises(FloatingPointError):
        mps.truncation_rank(np.zeros(3), 4, 0.0)


def _dense_vs_mps(Lx, two_W, beta, tau, seed, basis=collapse.BASIS_Z, Jr=0.7):
    lad = model.Ladder(Lx, two_W, 1.0, Jr)
    n, teff = model.trotter_steps(beta, tau)
    env = collapse.initial_env(len(lad.env), seed, 0)
    rows = collapse.basis_matrix(basis)
    st = mps.MPS(collapse.product_state(lad, env, basis))
    ops = model.plan_ops(lad, n)
    mps.evolve(st, ops, model.gate_table(lad, teff), chi_max=3 ** lad.n_sites, cutoff=0.0)
    phi, nrm = ed.dense_evolve(lad, env, rows, n, teff)
    return lad, st, phi / math.sqrt(nrm)


@pytest.mark.parametrize("Lx,two_W,basis", [(3, 2, collapse.BASIS_Z), (2, 4, collapse.BASIS_Z),
                                             (3, 0, collapse.BASIS_X), (2, 2, collapse.BASIS_X)])
def test_mps_evolution_matches_dense(Lx, two_W, basis):
    lad, st, psi = _dense_vs_mps(Lx, two_W, 0.6, 0.1, seed=3, basis=basis)
    v = st.to_dense()
    assert st.centre == 0
    assert abs(np.linalg.norm(v) - 1) < 1e-12
    # compare up to the global sign of the state
    sgn = np.sign(v @ psi.reshape(-1))
    assert np.abs(v - sgn * psi.reshape(-1)).max() < 1e-12


def test_right_canonical_after_evolution():
    lad, st, _ = _dense_vs_mps(3, 2, 0.6, 0.1, seed=1)
    for t in st.tensors[1:]:
        m = t.reshape(t.shape[0], -1)
        assert np.allclose(m @ m.T, np.eye(t.shape[0]), atol=1e-12)


@pytest.mark.parametrize("Lx,two_W", [(3, 2), (2, 4), (3, 0)])
def test_measure_matches_dense(Lx, two_W):
    lad, st, psi = _dense_vs_mps(Lx, two_W, 0.8, 0.1, seed=5)
    sz, sp, sm = model.spin1_operators()
    bonds = lad.measured_bonds(0, Lx)
    out = measure.measure(st, bonds)
    e = 0.0
    for b, (i, j, J) in enumerate(bonds):
        zz = ed.dense_expect(psi, i, j, sz, sz)
        ss = zz + 0.5 * (ed.dense_expect(psi, i, j, sp, sm) + ed.dense_expect(psi, i, j, sm, sp))
        assert abs(out[1 + 2 * b] - ss) < 1e-12
        assert abs(out[2 + 2 * b] - zz) < 1e-12
        e += J * ss
    assert abs(out[0] - e) < 1e-12


def test_truncated_evolution_is_close_to_dense():
    # a tight chi cap must still give a normalised state close to the exact one
    lad = model.Ladder(3, 2, 1.0, 1.0)
    n, teff = model.trotter_steps(1.0, 0.1)
    env = collapse.initial_env(len(lad.env), 0, 0)
    phi, nrm = ed.dense_evolve(lad, env, np.eye(3), n, teff)
    fid = []
    for chi in (6, 12, 18):
        st = mps.MPS(collapse.product_state(lad, env, collapse.BASIS_Z))
        mps.evolve(st, model.plan_ops(lad, n), model.gate_table(lad, teff), chi_max=chi, cutoff=1e-10)
        assert max(st.bond_dims()) <= chi
        v = st.to_dense()
        assert abs(np.linalg.norm(v) - 1) < 1e-12
        fid.append(abs(v @ phi.reshape(-1)) / math.sqrt(nrm))
    assert fid[0] < fid[1] < fid[2] and fid[2] > 0.99


def _pure_ancilla_energy(Lx, beta, tau, Jr):
    ch = chain.HybridChain(Lx, 2 * Lx, 1.0, Jr, beta=beta, tau=tau, chi_max=3 ** Lx * 9,
                           cutoff=0.0, meas_cols=(0, Lx))
    return ch, ch.sample()


def test_pure_ancilla_matches_trotter_operator():
    Lx, beta, tau, Jr = 2, 1.2, 0.1, 0.6
    ch, rec = _pure_ancilla_energy(Lx, beta, tau, Jr)
    lad = ch.ladder
    inv = {k: (x, y) for (x, y), k in lad.phys.items()}
    bonds_xy = [(inv[i], inv[j], J) for i, j, J in lad.bonds]
    mats = []
    for i, j, J in ch.meas_bonds:
        mats.append(ed.dense_bond_operator(Lx, inv[i], inv[j], "ss"))
        mats.append(ed.dense_bond_operator(Lx, inv[i], inv[j], "zz"))
    ref = ed.trotter_thermal(Lx, bonds_xy, ch.n_steps, ch.tau_eff, mats)
    assert np.abs(rec["obs"][1:] - np.array(ref)).max() < 1e-10
    # SU(2) symmetry of e^{-beta H}: <S.S> = 3 <Sz Sz> bond by bond
    assert np.abs(rec["obs"][1::2] - 3 * rec["obs"][2::2]).max() < 1e-10


def test_pure_ancilla_zero_variance_and_ed_limit():
    Lx, beta, Jr = 2, 1.0, 1.0
    ch, r0 = _pure_ancilla_energy(Lx, beta, 0.05, Jr)
    r1 = ch.sample()
    assert abs(r0["obs"][0] - r1["obs"][0]) < 1e-13     # one sample suffices
    e = ed.LadderED(Lx, 1.0, Jr)
    _, H = e.bond_thermal(beta, [])
    assert abs(r0["obs"][0] - H) < 2e-3                  # O(tau^2) Trotter error


def test_fully_polarised_environment_evolves():
    """Environment all m = +1 around the Lx=4, 2W=4 cluster (beta=2, chi=64):
    its two-site tensors are strongly rank deficient (one is 192 x 192 of
    rank 121), where LAPACK's gesdd does not converge.  The split falls back
    to gesvd.  The dense-SVD chain and the block-sparse one (other
    decompositions, same kept values) agree, and Q = 4."""
    from oracle import u1
    cfg = dict(Lx=4, two_W=4, J_leg=1.0, J_rung=1.0, beta=2.0, tau=0.1, chi_max=64, cutoff=1e-12,
               basis_zx=False)
    dense = chain.HybridChain(**cfg)
    block = u1.U1Chain(**cfg)
    dense.env = [0, 0, 0, 0]
    block.env = [0, 0, 0, 0]
    r0, r1 = dense.sample(), block.sample()
    assert np.allclose(r0["obs"], r1["obs"], rtol=1e-10, atol=1e-12)
    assert r1["Q"] == 4 and abs(np.linalg.norm(dense.last_mps.tensors[0]) - 1.0) < 1e-12
