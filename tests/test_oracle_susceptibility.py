"""Pins of oracle.measure.susceptibility (Eq. sus, Sec. II.A).

* pure-ancilla limit, region = every site: the raw sum is <S_tot^2>, which
  SU(2) symmetry turns into 3 <(S^z_tot)^2> = 3 sum_q q^2 Z_q / Z, read off the
  S^z-sector spectra of exact diagonalisation (no S.S operator involved);
  against the dense Trotter operator it holds to 1e-10;
* a hybrid sample against dense expectation values of S_j . S_i;
* beta = 0: product environment and maximally mixed cluster.
"""
import math

import numpy as np

from oracle import chain, collapse, ed, measure, model, mps


def _phys(lad):
    return [k for k, (kind, _, _) in enumerate(lad.sites) if kind == "P"]


def test_pure_ancilla_total_spin_against_sector_sums():
    Lx, beta = 2, 1.0
    for tau, tol in ((0.1, None), (0.025, 2e-3)):
        ch = chain.HybridChain(Lx, 2 * Lx, 1.0, 0.7, beta=beta, tau=tau, chi_max=81, cutoff=0.0)
        st = ch.evolve()
        chi_val, raw = measure.susceptibility(st, ch.ladder, _phys(ch.ladder), beta)
        assert abs(chi_val - beta / 3.0 * raw / (2 * Lx)) < 1e-15
        # dense Trotter operator: S_tot^2 = 2N + sum_{a != b} S_a . S_b
        inv = {k: (x, y) for (x, y), k in ch.ladder.phys.items()}
        bonds_xy = [(inv[i], inv[j], J) for i, j, J in ch.ladder.bonds]
        sites = [(x, y) for x in range(Lx) for y in (0, 1)]
        s2 = 2.0 * len(sites) * np.eye(3 ** (2 * Lx))
        for a in sites:
            for b in sites:
                if a != b:
                    s2 = s2 + ed.dense_bond_operator(Lx, a, b, "ss")
        (ref,) = ed.trotter_thermal(Lx, bonds_xy, ch.n_steps, ch.tau_eff, [s2])
        assert abs(raw - ref) < 1e-10
        exact = 3.0 * ed.total_sz_squared(ed.LadderED(Lx, 1.0, 0.7), beta)
        if tol is not None:
            assert abs(raw - exact) < tol * exact          # O(tau^2) Trotter error


def test_hybrid_sample_against_dense_expectations():
    lad = model.Ladder(3, 2, 1.0, 0.6)
    n, teff = model.trotter_steps(0.8, 0.1)
    env = collapse.initial_env(len(lad.env), 4, 0)
    st = mps.MPS(collapse.product_state(lad, env, collapse.BASIS_Z))
    mps.evolve(st, model.plan_ops(lad, n), model.gate_table(lad, teff), 3 ** lad.n_sites, 0.0)
    phi, nrm = ed.dense_evolve(lad, env, np.eye(3), n, teff)
    psi = phi / math.sqrt(nrm)
    sz, sp, sm = model.spin1_operators()
    region = [lad.phys[(1, 0)], lad.phys[(1, 1)]]
    want = 0.0
    for j in region:
        for i in _phys(lad):
            if i == j:
                want += 2.0
                continue
            want += ed.dense_expect(psi, i, j, sz, sz) + 0.5 * (
                ed.dense_expect(psi, i, j, sp, sm) + ed.dense_expect(psi, i, j, sm, sp))
    _, raw = measure.susceptibility(st, lad, region, 0.8)
    assert abs(raw - want) < 1e-11


def test_beta_zero_product_environment():
    ch = chain.HybridChain(3, 2, beta=0.0, tau=0.1, chi_max=8, seed=2)
    st = ch.initial_mps()
    m = {k: 1.0 - o for k, o in zip(ch.ladder.env, ch.env)}
    j = ch.ladder.env[0]
    want = 2.0 + sum(m[j] * m[i] for i in ch.ladder.env if i != j)   # cluster sites give 0
    _, raw = measure.susceptibility(st, ch.ladder, [j], 0.0)
    assert abs(raw - want) < 1e-14
