"""Pins of oracle/collapse.py and oracle/brute.py.

* Philox4x32-10 against the published known-answer vectors of Salmon et al.
  (SC'11; the Random123 distribution's kat_vectors for philox4x32, 10 rounds);
* collapse: the product of the sequential conditional probabilities equals the
  brute-force joint probability ||Pi_j psi||^2 of every outcome (Sec. I.C.2);
* detailed balance P_i p(i->j) = P_j p(j->i) and stationarity across a change
  of measurement basis, by brute force on a tiny ladder (Sec. I.C.2).
"""
import itertools
import math

import numpy as np
import pytest

from oracle import brute, collapse, ed, model, mps

KAT = [  # (counter, key, output), Philox4x32-10
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


@pytest.mark.parametrize("ctr,key,out", KAT)
def test_philox_known_answers(ctr, key, out):
    assert collapse.philox4x32_10(ctr, key) == out


def test_uniform_range_and_moments():
    u = np.array([collapse.uniform(7, 3, n, e) for n in range(40) for e in range(50)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.02 and abs(u.var() - 1 / 12) < 0.01


def test_choose_rule():
    p = [0.2, 0.0, 0.8]
    assert collapse.choose(p, 0.0) == 0
    assert collapse.choose(p, 0.1999) == 0
    assert collapse.choose(p, 0.2) == 2
    assert collapse.choose([0.5, 0.5, 0.0], 1.0) == 1   # rounding overflow -> last p>0


def test_x_basis_is_sx_eigenbasis():
    sz, sp, sm = model.spin1_operators()
    sx = 0.5 * (sp + sm)
    rows = collapse.basis_matrix(collapse.BASIS_X)
    assert np.allclose(rows @ rows.T, np.eye(3), atol=1e-15)
    for r, m in zip(rows, (1.0, 0.0, -1.0)):
        assert np.allclose(sx @ r, m * r, atol=1e-15)


def _evolved(Lx, two_W, beta, basis_in, seed=2):
    lad = model.Ladder(Lx, two_W, 1.0, 0.8)
    n, teff = model.trotter_steps(beta, 0.1)
    env = collapse.initial_env(len(lad.env), seed, 0)
    st = mps.MPS(collapse.product_state(lad, env, basis_in))
    mps.evolve(st, model.plan_ops(lad, n), model.gate_table(lad, teff), 3 ** lad.n_sites, 0.0)
    return lad, st


@pytest.mark.parametrize("Lx,two_W,basis", [(3, 2, collapse.BASIS_Z), (3, 2, collapse.BASIS_X),
                                             (2, 0, collapse.BASIS_X), (3, 4, collapse.BASIS_Z)])
def test_collapse_conditionals_match_brute_force(Lx, two_W, basis):
    lad, st = _evolved(Lx, two_W, 0.8, collapse.BASIS_Z)
    rows = collapse.basis_matrix(basis)
    joint = brute.joint_probabilities(st.to_dense().reshape((3,) * lad.n_sites), lad, rows)
    assert abs(sum(joint.values()) - 1.0) < 1e-12
    for js in itertools.product(range(3), repeat=len(lad.env)):
        _, logp, conds = collapse.collapse(st, lad, basis, 0, 0, 0, forced=list(js))
        prod = math.prod(c[j] for c, j in zip(conds, js))
        assert abs(prod - joint[js]) < 1e-12


def test_collapse_sampling_uses_the_rng_stream():
    lad, st = _evolved(3, 2, 0.8, collapse.BASIS_Z)
    out, logp, conds = collapse.collapse(st, lad, collapse.BASIS_Z, 11, 4, 9)
    for e, (b, p) in enumerate(zip(out, conds)):
        assert b == collapse.choose(p, collapse.uniform(11, 4, 9, e))
    assert abs(logp - sum(math.log(c[b]) for c, b in zip(conds, out))) < 1e-14


def test_detailed_balance_same_basis():
    lad = model.Ladder(2, 2, 1.0, 0.6)
    n, teff = model.trotter_steps(1.0, 0.1)
    z = collapse.basis_matrix(collapse.BASIS_Z)
    P, T = brute.transition_matrix(lad, n, teff, z, z)
    assert np.allclose(T.sum(axis=1), 1.0, atol=1e-12)
    flux = P[:, None] * T
    assert np.abs(flux - flux.T).max() < 1e-12 * flux.max()


def test_stationarity_across_basis_change():
    # collapsing in x maps the z-basis weights P^z onto the x-basis weights P^x
    lad = model.Ladder(2, 2, 1.0, 0.6)
    n, teff = model.trotter_steps(1.0, 0.1)
    z = collapse.basis_matrix(collapse.BASIS_Z)
    x = collapse.basis_matrix(collapse.BASIS_X)
    Pz, Tzx = brute.transition_matrix(lad, n, teff, z, x)
    Px, _ = brute.transition_matrix(lad, n, teff, x, x)
    assert np.allclose(Pz @ Tzx, Px, rtol=1e-11, atol=0)


def test_initial_env_draws():
    out = collapse.initial_env(6, 5, 2)
    third = 1.0 / 3.0
    assert out == [collapse.choose([third] * 3, collapse.uniform(5, 2, -1, e)) for e in range(6)]
    assert set(out) <= {0, 1, 2}


def test_product_state_norm_and_canonical_form():
    lad = model.Ladder(4, 4)
    ts = collapse.product_state(lad, [0, 1, 2, 0], collapse.BASIS_X)
    st = mps.MPS(ts)
    assert abs(np.linalg.norm(st.to_dense()) - 1.0) < 1e-14
    for t in ts:
        m = t.reshape(t.shape[0], -1)
        assert np.allclose(m @ m.T, np.eye(t.shape[0]), atol=1e-15)
    _ = ed  # dense helpers are pinned in test_oracle_ed
