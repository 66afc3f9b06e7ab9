"""Pins of the fused op schedule (oracle/model.py ``fuse_ops``).

The fused schedule applies the same product of two-site gates as the plain
one (Sec. I.A; second-order steps of Sec. II), with runs of splits on one
site pair folded into one.  Pins:
* hand-made op lists with random, non-commuting 9x9 matrices fix the
  product order, the absorb side and the SWAP SWAP cancellation (with and
  without a centre change);
* on real ladders, every fused op still touches the centre and every bond
  gate letter survives (two per bond per step);
* without truncation the fused MPS evolution equals the dense Trotterised
  state-vector evolver (no swaps, no SVD) to 1e-12;
* with truncation it stays as close to the exact state as the plain one.
"""
import math

import numpy as np
import pytest

from oracle import collapse, ed, model, mps

S, L, R = model.SPLIT, model.ABSORB_L, model.ABSORB_R


def _rand_gates(n, seed=0):
    rng = np.random.default_rng(seed)
    return [model.swap_gate()] + [rng.standard_normal((9, 9)) for _ in range(n)]


def test_product_order_and_absorb_side():
    g = _rand_gates(2)
    ops, tab = model.fuse_ops([(S, 0, 1, R), (S, 0, 2, L)], g)
    assert ops == [(S, 0, 3, L)]
    assert np.array_equal(tab[3], g[2] @ g[1])          # later gate on the left
    assert not np.allclose(g[2] @ g[1], g[1] @ g[2])
    assert len(tab) == 4


def test_three_letter_word_and_reuse_of_entries():
    g = _rand_gates(2, seed=1)
    plan = [(model.MOVE_R, 0, -1, -1), (S, 1, 1, L), (S, 1, 0, R), (S, 1, 2, L),
            (model.MOVE_L, 1, -1, -1), (S, 0, 1, R), (S, 1, 1, L), (S, 1, 0, R), (S, 1, 2, R)]
    ops, tab = model.fuse_ops(plan, g)
    assert ops == [(model.MOVE_R, 0, -1, -1), (S, 1, 3, L), (model.MOVE_L, 1, -1, -1), (S, 0, 1, R),
                   (S, 1, 3, R)]
    assert np.allclose(tab[3], g[2] @ g[0] @ g[1], atol=0)
    assert len(tab) == 4                                   # one entry for the repeated word


def test_swap_pairs_cancel():
    g = _rand_gates(2)
    # a SWAP SWAP pair inside a word drops out; the gate then meets itself
    ops, tab = model.fuse_ops([(S, 0, 1, L), (S, 0, 0, L), (S, 0, 0, R), (S, 0, 1, L)], g)
    assert ops == [(S, 0, 3, L)] and np.allclose(tab[3], g[1] @ g[1], atol=0)
    # a word of two SWAPs that moved the centre (0 -> 1) becomes an exact move
    ops, _ = model.fuse_ops([(S, 0, 0, R), (S, 0, 0, R)], g)
    assert ops == [(model.MOVE_R, 0, -1, -1)]
    # a word of two SWAPs that left the centre in place (1 -> 1) vanishes and
    # exposes the split below it, which then folds with the next one
    ops, tab = model.fuse_ops([(S, 0, 1, R), (S, 1, 0, L), (S, 1, 0, L), (S, 0, 2, L)], g)
    assert ops == [(S, 0, 3, L)] and np.allclose(tab[3], g[2] @ g[1], atol=0)


def _replay(ops, n_sites):
    c = 0
    for kind, k, _, absorb in ops:
        if kind == S:
            assert c in (k, k + 1)
            c = k if absorb == L else k + 1
        elif kind == model.MOVE_R:
            assert c == k
            c += 1
        else:
            assert c == k
            c -= 1
    assert 0 <= c < n_sites
    return c


@pytest.mark.parametrize("Lx,two_W", [(16, 8), (4, 4), (1, 2), (3, 0), (2, 4), (5, 2)])
def test_fused_schedule_is_valid_and_keeps_every_gate(Lx, two_W):
    lad = model.Ladder(Lx, two_W)
    n, t = model.trotter_steps(0.6, 0.1)
    plain, base = model.schedule(lad, n, t)
    ops, tab = model.schedule(lad, n, t, model.SCHEDULE_FUSED)
    assert _replay(ops, lad.n_sites) == 0
    assert len(ops) < len(plain) or Lx == 1
    ref = _rewrite(plain)
    letters = sum(1 for kind, _, w, _ in ref if kind == S for x in w if x != model.GATE_SWAP)
    assert letters == 2 * n * len(lad.bonds)                  # every bond gate, twice per step
    assert [(o[0], o[1], o[3]) for o in ops] == [(r[0], r[1], r[3]) for r in ref]
    for o, (kind, _, w, _) in zip(ops, ref):
        if kind == S:
            m = base[w[0]]
            for x in w[1:]:
                m = base[x] @ m
            assert np.abs(tab[o[2]] - m).max() < 1e-15


def _rewrite(plain):
    """The fused op list by rewriting to a fixed point, an algorithm unlike
    the oracle's single stack pass: repeat (1) join neighbouring splits on
    one pair into one word, (2) delete every SWAP SWAP pair inside a word,
    (3) turn an empty word into an exact move, or drop it when the centre
    did not move, until nothing changes.  Entries: (kind, k, word, absorb)."""
    items, c = [], 0
    for kind, k, g, absorb in plain:
        c1 = (k if absorb == L else k + 1) if kind == S else (k + 1 if kind == model.MOVE_R else k - 1)
        items.append([kind, k, [g] if kind == S else None, absorb, c, c1])
        c = c1
    changed = True
    while changed:
        changed = False
        joined = []
        for it in items:
            if it[0] == S and joined and joined[-1][0] == S and joined[-1][1] == it[1]:
                prev = joined[-1]
                joined[-1] = [S, it[1], prev[2] + it[2], it[3], prev[4], it[5]]
                changed = True
            else:
                joined.append(list(it))
        items = []
        for it in joined:
            if it[0] == S:
                w = it[2]
                i = 0
                while i + 1 < len(w):
                    if w[i] == model.GATE_SWAP and w[i + 1] == model.GATE_SWAP:
                        w = w[:i] + w[i + 2:]
                        i = max(i - 1, 0)
                        changed = True
                    else:
                        i += 1
                if not w:
                    changed = True
                    if it[4] != it[5]:
                        move = model.MOVE_R if it[5] > it[4] else model.MOVE_L
                        items.append([move, it[4], None, -1, it[4], it[5]])
                    continue
                it[2] = w
            items.append(it)
    return [(it[0], it[1], it[2], it[3]) for it in items]


@pytest.mark.parametrize("Lx,two_W,basis", [(3, 2, collapse.BASIS_Z), (2, 4, collapse.BASIS_X),
                                             (3, 0, collapse.BASIS_Z), (2, 2, collapse.BASIS_X)])
def test_fused_evolution_matches_dense(Lx, two_W, basis):
    lad = model.Ladder(Lx, two_W, 1.0, 0.7)
    n, teff = model.trotter_steps(0.6, 0.1)
    env = collapse.initial_env(len(lad.env), 3, 0)
    st = mps.MPS(collapse.product_state(lad, env, basis))
    ops, gates = model.schedule(lad, n, teff, model.SCHEDULE_FUSED)
    mps.evolve(st, ops, gates, chi_max=3 ** lad.n_sites, cutoff=0.0)
    phi, nrm = ed.dense_evolve(lad, env, collapse.basis_matrix(basis), n, teff)
    v, psi = st.to_dense(), phi.reshape(-1) / math.sqrt(nrm)
    assert st.centre == 0
    sgn = np.sign(v @ psi)
    assert np.abs(v - sgn * psi).max() < 1e-12


def test_fused_truncated_evolution_is_as_close_as_plain():
    # fewer truncating splits: at every chi cap the fused state is at least as
    # close to the exact Trotterised state as the plain one
    lad = model.Ladder(3, 2, 1.0, 1.0)
    n, teff = model.trotter_steps(1.0, 0.1)
    env = collapse.initial_env(len(lad.env), 0, 0)
    phi, nrm = ed.dense_evolve(lad, env, np.eye(3), n, teff)
    fused = []
    for chi in (6, 12, 18):
        fid = {}
        for kind in (model.SCHEDULE_PLAIN, model.SCHEDULE_FUSED):
            st = mps.MPS(collapse.product_state(lad, env, collapse.BASIS_Z))
            ops, gates = model.schedule(lad, n, teff, kind)
            mps.evolve(st, ops, gates, chi_max=chi, cutoff=1e-10)
            assert max(st.bond_dims()) <= chi
            fid[kind] = abs(st.to_dense() @ phi.reshape(-1)) / math.sqrt(nrm)
        assert fid[model.SCHEDULE_FUSED] >= fid[model.SCHEDULE_PLAIN] - 1e-3
        fused.append(fid[model.SCHEDULE_FUSED])
    assert fused[0] < fused[1] < fused[2] and fused[2] > 0.99


def test_fused_op_count_lx16():
    # one step of the Lx = 16, two_W = 8 ladder: 292 splits plain, 16 % fewer fused
    lad = model.Ladder(16, 8)
    n, t = model.trotter_steps(1.0, 0.05)
    plain, _ = model.schedule(lad, n, t)
    ops, tab = model.schedule(lad, n, t, model.SCHEDULE_FUSED)
    assert len(plain) == 3080 and len(ops) == 2601
    assert len(tab) == 1 + len(lad.bonds) + 17


def test_unknown_schedule_rejected():
    with pytest.raises(ValueError):
        model.schedule(model.Ladder(2, 2), 1, 0.1, "merged")


def test_observables_stable_under_gate_rounding_at_the_chi_cap():
    """Lx=4, 2W=4, beta=2, chi=64: about 300 fused splits cut at the chi cap.
    A 1e-16 relative change of every gate leaves the observables within
    1e-12 relative (the 1e-10 parity bar holds), although the dense state
    itself may move far more (the cut falls between close singular values)."""
    from oracle import chain, measure
    cfg = dict(Lx=4, two_W=4, J_leg=1.0, J_rung=1.0, beta=2.0, tau=0.1, chi_max=64, cutoff=1e-12)
    ch = chain.HybridChain(seed=5, chain_id=1, schedule=model.SCHEDULE_FUSED, **cfg)
    log = []
    ref = measure.measure(mps.evolve(ch.initial_mps(), ch.ops, ch.gates, 64, 1e-12, log), ch.meas_bonds)
    assert sum(1 for r in log if r[5] == 64) > 200
    rng = np.random.default_rng(0)
    g2 = [g * (1 + 1e-16 * rng.standard_normal(g.shape)) for g in ch.gates]
    obs = measure.measure(mps.evolve(ch.initial_mps(), ch.ops, g2, 64, 1e-12), ch.meas_bonds)
    assert np.max(np.abs(obs - ref) / np.maximum(np.abs(ref), 1e-2)) < 1e-12



@pytest.mark.parametrize("schedule, seed, chain_id, trials", [
    (model.SCHEDULE_FUSED, 5, 1, (11, 14)),
    (model.SCHEDULE_PLAIN, 0, 0, (1, 3)),
])
def test_logp_moves_under_gate_rounding_at_the_chi_cap(schedule, seed, chain_id, trials):
    """Lx=4, 2W=4, beta=2, chi=64 (the small workload), sample 1: a 1e-16
    relative change of every gate moves the oracle's own collapse
    log-probability by more than 1e-10 relative (the cut falls between
    close singular values; the fused chain moves by more than 1e-9).  So a
    1e-10 relative bar on log p is below the method's rounding noise on
    these chains.  The GPU tests compare their log p at 2e-8 absolute,
    above every deviation seen here, and every other chain's at 1e-10
    relative."""
    from oracle import chain
    cfg = dict(Lx=4, two_W=4, J_leg=1.0, J_rung=1.0, beta=2.0, tau=0.1, chi_max=64, cutoff=1e-12)
    ch = chain.HybridChain(seed=seed, chain_id=chain_id, schedule=schedule, **cfg)
    ch.sample()
    env, basis_in, n = list(ch.env), ch.env_basis, ch.n
    ref = ch.sample()
    dev = []
    for trial in trials:
        rng = np.random.default_rng(trial)
        g2 = [g * (1 + 1e-16 * rng.standard_normal(g.shape)) for g in ch.gates]
        st = mps.evolve(mps.MPS(collapse.product_state(ch.ladder, env, basis_in), 0), ch.ops, g2, 64, 1e-12)
        out, logp, _ = collapse.collapse(st, ch.ladder, collapse.sample_basis(n, True), seed, chain_id, n)
        assert list(out) == ref["env_out"]
        dev.append(abs(logp - ref["logp"]))
    assert max(dev) > 1e-10 * abs(ref["logp"])
    if schedule == model.SCHEDULE_FUSED:
        assert max(dev) > 1e-9
    assert max(dev) < 5e-9
