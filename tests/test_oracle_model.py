"""Pins of oracle/model.py: spin algebra, gates, site map and op schedule."""
import numpy as np
import pytest
import scipy.linalg

from oracle import model


def test_spin1_algebra():
    sz, sp, sm = model.spin1_operators()
    # [Sz, S+] = S+, [S+, S-] = 2 Sz, S^2 = s(s+1) = 2 for S = 1
    assert np.allclose(sz @ sp - sp @ sz, sp, atol=0)
    assert np.allclose(sp @ sm - sm @ sp, 2 * sz, atol=1e-15)
    s2 = sz @ sz + 0.5 * (sp @ sm + sm @ sp)
    assert np.allclose(s2, 2 * np.eye(3), atol=1e-15)


def test_bond_operator_spectrum():
    # two spin-1: total S = 0, 1, 2 -> S.S = -2 (x1), -1 (x3), +1 (x5)
    w = np.linalg.eigvalsh(model.bond_operator())
    assert np.allclose(w, [-2, -1, -1, -1, 1, 1, 1, 1, 1], atol=1e-14)


@pytest.mark.parametrize("coef", [0.0, 0.025, 0.05, -0.3, 1.7])
def test_bond_gate_matches_library_expm(coef):
    g = model.bond_gate(coef)
    ref = scipy.linalg.expm(-coef * model.bond_operator())
    # scipy's Pade expm carries ~1e-13 relative error itself
    assert np.abs(g - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.allclose(g, g.T, atol=1e-15)


def test_swap_gate():
    p = model.swap_gate()
    assert np.allclose(p @ p, np.eye(9))
    a, b = np.random.default_rng(0).standard_normal((2, 3))
    assert np.allclose(p @ np.kron(a, b), np.kron(b, a))


def test_site_map_lx4_w2():
    lad = model.Ladder(4, 4)
    assert lad.cluster_cols == [1, 2]
    kinds = "".join(k for k, _, _ in lad.sites)
    assert kinds == "PP" + "PAPA" * 2 + "PP"
    assert lad.n_sites == 12 and len(lad.env) == 4
    assert len(lad.bonds) == 4 + 6


@pytest.mark.parametrize("Lx,two_W,x0", [(16, 8, 6), (5, 2, 2), (4, 0, None), (3, 6, 0), (6, 2, 2)])
def test_cluster_centring(Lx, two_W, x0):
    lad = model.Ladder(Lx, two_W)
    if x0 is None:
        assert lad.cluster_cols == []
    else:
        assert lad.cluster_cols[0] == x0 and len(lad.cluster_cols) == two_W // 2
    assert lad.n_sites == 2 * Lx + two_W


def test_invalid_ladders():
    for args in [(0, 0), (3, 3), (2, 6), (3, -2)]:
        with pytest.raises(ValueError):
            model.Ladder(*args)


def _replay(ops, n_sites):
    """Track the centre through an op list; check every op touches it."""
    c = 0
    for kind, k, g, absorb in ops:
        assert 0 <= k < n_sites
        if kind == model.SPLIT:
            assert k + 1 < n_sites and c in (k, k + 1)
            c = k if absorb == model.ABSORB_L else k + 1
        elif kind == model.MOVE_R:
            assert c == k
            c = k + 1
        else:
            assert c == k and k > 0
            c = k - 1
    return c


@pytest.mark.parametrize("Lx,two_W", [(16, 8), (4, 4), (1, 2), (3, 0), (2, 4), (5, 2)])
def test_plan_ops_structure(Lx, two_W):
    lad = model.Ladder(Lx, two_W)
    ops = model.plan_ops(lad, 2)
    assert _replay(ops, lad.n_sites) == 0
    n_gate = sum(1 for o in ops if o[0] == model.SPLIT and o[2] != model.GATE_SWAP)
    assert n_gate == 2 * 2 * len(lad.bonds)
    # a gate at distance j-i needs 2 (j-i-1) swaps
    swaps = sum(1 for o in ops if o[0] == model.SPLIT and o[2] == model.GATE_SWAP)
    assert swaps == 2 * 2 * sum(2 * (j - i - 1) for i, j, _ in lad.bonds)


def test_plan_ops_count_lx16():
    # 12 env rungs (1 op), 20 env legs (3), 4 cluster rungs (3), 6 cluster legs
    # (7), boundary legs 3+5 and 7+5: 146 splits per half step
    lad = model.Ladder(16, 8)
    ops = model.plan_ops(lad, 1)
    assert sum(1 for o in ops if o[0] == model.SPLIT) == 2 * 146


def test_gate_application_order():
    # each bond's gate appears exactly once per half step, forward then reverse
    lad = model.Ladder(3, 2)
    ops = model.plan_ops(lad, 1)
    seq = [o[2] - 1 for o in ops if o[0] == model.SPLIT and o[2] != model.GATE_SWAP]
    nb = len(lad.bonds)
    assert seq == list(range(nb)) + list(reversed(range(nb)))


def test_trotter_steps():
    assert model.trotter_steps(2.0, 0.1) == (10, 0.1)
    assert model.trotter_steps(0.0, 0.1)[0] == 0
    m, t = model.trotter_steps(1.0, 0.3)
    assert m == 2 and abs(t - 0.25) < 1e-15
    assert model.trotter_steps(1.0, 0.2)[0] == 3      # 2.5 rounds up
