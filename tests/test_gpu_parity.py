"""CUDA path vs the FP64 oracle, through the C ABI (GPU tests).

Tolerances (FP64 path): per-sample observables within 1e-10 relative (1e-12
absolute floor); collapse outcomes bit-exact; log-probabilities within 1e-10 relative;
states compared as dense vectors up to the global sign at 1e-10.
"""
import math

import numpy as np
import pytest

from oracle import chain as ochain
from oracle import ed, model
from oracle import mps as omps

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-10, 1e-12
LOGP_CHI_CAP = 2e-8   # pinned by test_logp_moves_under_gate_rounding_at_the_chi_cap


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_1910_09142_gb300 import binding
    assert torch.cuda.is_available()
    c = binding.Context(1 << 30)
    yield c
    c.close()


def _b():
    from paper_1910_09142_gb300 import binding
    return binding


def _dense(tensors):
    return omps.MPS(tensors).to_dense()


def _same_state(a, b, tol=1e-10):
    va, vb = _dense(a), _dense(b)
    s = np.sign(va @ vb)
    return np.abs(va - s * vb).max() < tol


CFGS = [
    dict(Lx=3, two_W=2, J_leg=1.0, J_rung=0.5, beta=0.6, tau=0.1, chi_max=64, cutoff=1e-12),
    dict(Lx=2, two_W=4, J_leg=1.0, J_rung=1.0, beta=1.0, tau=0.1, chi_max=81, cutoff=1e-12),
    dict(Lx=3, two_W=0, J_leg=1.0, J_rung=0.7, beta=1.2, tau=0.1, chi_max=64, cutoff=1e-12),
    dict(Lx=5, two_W=2, J_leg=1.0, J_rung=1.0, beta=0.8, tau=0.1, chi_max=12, cutoff=1e-8),
]


def test_evolved_state_matches_oracle(ctx):
    """All CFGS evolved in one batched call; each state equals the oracle's."""
    b = _b()
    ps = [b.params(**cfg, seed=7, chain_id=3) for cfg in CFGS]
    ids = [ctx.init_chain(p) for p in ps]
    try:
        refs = [ochain.HybridChain(seed=7, chain_id=3, **cfg) for cfg in CFGS]
        for cid, ref in zip(ids, refs):
            assert _same_state(ctx.get_mps(cid), ref.initial_mps().tensors, 1e-15)
        ctx.evolve(ids)
        for cid, ref in zip(ids, refs):
            got = ctx.get_mps(cid)
            want = ref.evolve()
            assert [t.shape for t in got] == [t.shape for t in want.tensors]
            assert _same_state(got, want.tensors)
            for t in got[1:]:                               # right-canonical from site 1
                m = t.reshape(t.shape[0], -1)
                assert np.abs(m @ m.T - np.eye(t.shape[0])).max() < 1e-12
    finally:
        for cid in ids:
            ctx.free_chain(cid)


def test_samples_match_oracle(ctx):
    """Four Markov steps of every CFGS chain, batched; per-sample parity."""
    b = _b()
    ps = [b.params(**cfg, seed=11, chain_id=2) for cfg in CFGS]
    ids = [ctx.init_chain(p) for p in ps]
    try:
        refs = [ochain.HybridChain(seed=11, chain_id=2, **cfg) for cfg in CFGS]
        for _ in range(4):
            ctx.evolve(ids)
            for cid, p, ref in zip(ids, ps, refs):
                obs = ctx.measure([cid], b.num_obs(p))[0]
                env, logp = ctx.collapse([cid], b.num_env(p))
                r = ref.sample()
                assert np.allclose(obs, r["obs"], rtol=RTOL, atol=ATOL), (obs, r["obs"])
                assert list(env[0]) == r["env_out"]
                assert abs(logp[0] - r["logp"]) <= 1e-10 * max(1.0, abs(r["logp"]))
    finally:
        for cid in ids:
            ctx.free_chain(cid)


def test_small_config_samples(ctx):
    """Lx=4 ladder, 2W=4, beta=2, tau=0.1, chi=64, cutoff 1e-12 (2 samples)."""
    b = _b()
    cfg = dict(Lx=4, two_W=4, J_leg=1.0, J_rung=1.0, beta=2.0, tau=0.1, chi_max=64, cutoff=1e-12)
    p = b.params(**cfg, seed=0, chain_id=0)
    cid = ctx.init_chain(p)
    try:
        ref = ochain.HybridChain(seed=0, chain_id=0, **cfg)
        n_obs, n_env = b.num_obs(p), b.num_env(p)
        worst = 0.0
        for _ in range(2):
            ctx.evolve([cid])
            obs = ctx.measure([cid], n_obs)[0]
            env, logp = ctx.collapse([cid], n_env)
            r = ref.sample()
            worst = max(worst, abs(obs[0] - r["obs"][0]) / abs(r["obs"][0]))
            assert np.allclose(obs, r["obs"], rtol=RTOL, atol=ATOL)
            assert list(env[0]) == r["env_out"]
            # chi-capped chain: its log p moves by ~5e-10 under rounding alone
            # (test_logp_moves_under_gate_rounding_at_the_chi_cap)
            assert abs(logp[0] - r["logp"]) <= LOGP_CHI_CAP
        assert worst < RTOL
    finally:
        ctx.free_chain(cid)


def test_single_rung_closed_form(ctx):
    b = _b()
    for beta in (0.5, 2.0):
        p = b.params(1, 2, beta=beta, tau=0.1, chi_max=16, cutoff=0.0)
        cid = ctx.init_chain(p)
        ctx.evolve([cid])
        obs = ctx.measure([cid], b.num_obs(p))[0]
        J = 1.0
        e = J * (-2 * math.exp(2 * beta) - 3 * math.exp(beta) + 5 * math.exp(-beta)) / (
            math.exp(2 * beta) + 3 * math.exp(beta) + 5 * math.exp(-beta))
        assert abs(obs[0] - e) < 1e-12
        assert abs(obs[1] - 3 * obs[2]) < 1e-12
        env, logp = ctx.collapse([cid], 0)                  # no environment sites
        assert env.shape[1] == 0 and logp[0] == 0.0
        ctx.free_chain(cid)


def test_pure_ancilla_is_exact_and_repeatable(ctx):
    b = _b()
    Lx, beta = 2, 1.2
    p = b.params(Lx, 2 * Lx, J_rung=0.6, beta=beta, tau=0.1, chi_max=81, cutoff=0.0, meas_cols=(0, Lx))
    cid = ctx.init_chain(p)
    lad = model.Ladder(Lx, 2 * Lx, 1.0, 0.6)
    inv = {k: (x, y) for (x, y), k in lad.phys.items()}
    bonds_xy = [(inv[i], inv[j], J) for i, j, J in lad.bonds]
    n_steps, teff = model.trotter_steps(beta, 0.1)
    mats = []
    for i, j, J in lad.measured_bonds(0, Lx):
        mats += [ed.dense_bond_operator(Lx, inv[i], inv[j], "ss"), ed.dense_bond_operator(Lx, inv[i], inv[j], "zz")]
    ref = np.array(ed.trotter_thermal(Lx, bonds_xy, n_steps, teff, mats))
    vals = []
    for _ in range(2):
        ctx.evolve([cid])
        obs = ctx.measure([cid], b.num_obs(p))[0]
        ctx.collapse([cid], 0)
        assert np.abs(obs[1:] - ref).max() < 1e-10
        vals.append(obs[0])
    assert abs(vals[0] - vals[1]) < 1e-14                   # zero variance
    ctx.free_chain(cid)


def test_beta_zero_leaves_state(ctx):
    b = _b()
    p = b.params(4, 4, beta=0.0, tau=0.1, chi_max=8, seed=3, meas_cols=(0, 4))
    cid = ctx.init_chain(p)
    ref = ochain.HybridChain(4, 4, beta=0.0, tau=0.1, chi_max=8, seed=3, meas_cols=(0, 4))
    ctx.evolve([cid])
    obs = ctx.measure([cid], b.num_obs(p))[0]
    assert np.allclose(obs, ref.sample()["obs"], atol=1e-14, rtol=0)
    ctx.collapse([cid], b.num_env(p))
    ctx.free_chain(cid)


def test_batched_chains_equal_alone(ctx):
    """Chains of different shapes in one call give bit-identical results to solo runs."""
    b = _b()
    cfgs = [dict(Lx=3, two_W=2, beta=0.6, tau=0.1, chi_max=32, cutoff=1e-10, seed=1, chain_id=i) for i in range(3)]
    cfgs.append(dict(Lx=4, two_W=4, beta=0.4, tau=0.1, chi_max=16, cutoff=1e-10, seed=1, chain_id=9))
    cfgs.append(dict(Lx=2, two_W=0, beta=0.6, tau=0.1, chi_max=16, cutoff=1e-10, seed=2, chain_id=0))
    ps = [b.params(**c) for c in cfgs]
    mixed = [ctx.init_chain(p) for p in ps]
    solo = [ctx.init_chain(p) for p in ps]
    ctx.evolve(mixed)
    out_m = [ctx.measure([c], b.num_obs(p))[0] for c, p in zip(mixed, ps)]
    for c, p, om in zip(solo, ps, out_m):
        ctx.evolve([c])
        assert np.array_equal(ctx.measure([c], b.num_obs(p))[0], om)
    for c in mixed + solo:
        ctx.free_chain(c)


def test_explicit_env_init_and_x_basis(ctx):
    b = _b()
    cfg = dict(Lx=4, two_W=2, J_leg=1.0, J_rung=0.5, beta=0.5, tau=0.1, chi_max=32, cutoff=1e-12)
    p = b.params(**cfg, seed=4, chain_id=6)
    env0 = [2, 0, 1, 1, 0, 2]
    cid = ctx.init_chain(p, env_init=env0)
    ref = ochain.HybridChain(seed=4, chain_id=6, **cfg)
    ref.env = list(env0)
    n_obs, n_env = b.num_obs(p), b.num_env(p)
    for _ in range(3):                                      # z, x, z collapse bases
        ctx.evolve([cid])
        obs = ctx.measure([cid], n_obs)[0]
        env, logp = ctx.collapse([cid], n_env)
        r = ref.sample()
        assert np.allclose(obs, r["obs"], rtol=RTOL, atol=ATOL)
        assert list(env[0]) == r["env_out"]
    ctx.free_chain(cid)


def test_apply_ops_single_split_parity(ctx):
    """One truncating split and one exact move, op by op, on an evolved state."""
    b = _b()
    cfg = dict(Lx=3, two_W=2, J_leg=1.0, J_rung=0.5, beta=0.4, tau=0.1, chi_max=64, cutoff=1e-12)
    p = b.params(**cfg, seed=2)
    cid = ctx.init_chain(p)
    ref = ochain.HybridChain(seed=2, **cfg)
    st = ref.evolve()
    ctx.set_mps(cid, st.tensors)
    gates = model.gate_table(ref.ladder, ref.tau_eff)
    # truncating split with bond gate 0 on (0, 1), absorb right, then move back left
    ctx.apply_ops(cid, [[0, 2, 1, 0], [0, 0, 0, 1]])
    omps.split(st, 0, gates[1], model.ABSORB_R, cfg["chi_max"], cfg["cutoff"])
    omps.move_left(st, 1)
    assert _same_state(ctx.get_mps(cid), st.tensors)
    ctx.free_chain(cid)


def test_state_errors(ctx):
    b = _b()
    p = b.params(3, 2, beta=0.2, tau=0.1, chi_max=8)
    cid = ctx.init_chain(p)
    with pytest.raises(b.HmError) as e:
        ctx.measure([cid], b.num_obs(p))
    assert e.value.code == b.HM_ERR_STATE
    ctx.evolve([cid])
    with pytest.raises(b.HmError) as e:
        ctx.evolve([cid])
    assert e.value.code == b.HM_ERR_STATE
    with pytest.raises(b.HmError) as e:
        ctx.measure([cid], b.num_obs(p) + 1)
    assert e.value.code == b.HM_ERR_ARG
    with pytest.raises(b.HmError) as e:
        ctx.evolve([987654])
    assert e.value.code == b.HM_ERR_ARG
    ctx.free_chain(cid)


def test_admission_refused_without_side_effects():
    b = _b()
    small = b.Context(8 << 20)
    big = b.params(16, 8, chi_max=256)
    with pytest.raises(b.HmError) as e:
        small.init_chain(big)
    assert e.value.code == b.HM_ERR_NOMEM
    ok = small.init_chain(b.params(2, 2, chi_max=4))         # the arena is still usable
    small.free_chain(ok)
    small.close()


def _oracle_sample_conds(ref):
    """One oracle Markov step that also returns the collapse's conditional
    probabilities (Eq. detailbalance1, one vector per environment site)."""
    from oracle import collapse as ocol
    from oracle import measure as omeas
    st = ref.evolve()
    obs = omeas.measure(st, ref.meas_bonds)
    basis = ocol.sample_basis(ref.n, ref.basis_zx)
    out, logp, conds = ocol.collapse(st, ref.ladder, basis, ref.seed, ref.chain_id, ref.n)
    ref.env, ref.env_basis = out, basis
    ref.n += 1
    return obs, list(out), logp, np.array(conds, dtype=np.float64).reshape(-1, 3)


def test_collapse_conditionals_match_oracle(ctx):
    """Per-site conditional probabilities of the collapse (hm_collapse_conditionals)
    at 1e-10 relative (1e-14 absolute floor), three samples (S^z, S^x, S^z
    bases) of the chains whose state is stable under rounding."""
    b = _b()
    cfgs = [CFGS[0], CFGS[2], CFGS[3]]
    ps = [b.params(**cfg, seed=13, chain_id=4) for cfg in cfgs]
    ids = [ctx.init_chain(p) for p in ps]
    try:
        refs = [ochain.HybridChain(seed=13, chain_id=4, **cfg) for cfg in cfgs]
        for _ in range(3):
            ctx.evolve(ids)
            for cid, p, ref in zip(ids, ps, refs):
                n_env = b.num_env(p)
                obs = ctx.measure([cid], b.num_obs(p))[0]
                env, logp, cond = ctx.collapse_conditionals([cid], n_env)
                r_obs, r_env, r_logp, r_cond = _oracle_sample_conds(ref)
                assert np.allclose(obs, r_obs, rtol=RTOL, atol=ATOL)
                assert list(env[0]) == r_env
                assert cond[0].shape == r_cond.shape
                assert np.all(np.abs(cond[0] - r_cond) <= 1e-10 * r_cond + 1e-14), np.abs(cond[0] - r_cond).max()
                assert abs(logp[0] - r_logp) <= 1e-10 * max(1.0, abs(r_logp))
    finally:
        for cid in ids:
            ctx.free_chain(cid)


@pytest.mark.parametrize("prec", ["HM_FP64", "HM_MIXED", "HM_MIXED32"])
def test_dense_mode_after_set_mps_matches_oracle(ctx, prec):
    """hm_set_mps drops the charge labels: the chain evolves with one block
    per split (the unblocked SVD).  At chi = 96 those blocks reach 192 columns,
    more than the binary32 kernel keeps in shared memory, so the mixed paths
    take their staged global-memory Jacobi.  Sample 0 must match the oracle
    (1e-10 FP64, 1e-5 mixed); the collapse then resets the chain to labelled
    blocks, and sample 1 must match too."""
    b = _b()
    cfg = dict(Lx=3, two_W=2, J_leg=1.0, J_rung=0.5, beta=0.6, tau=0.1, chi_max=96, cutoff=1e-12)
    p = b.params(**cfg, seed=9, chain_id=2, precision=getattr(b, prec))
    cid = ctx.init_chain(p)
    rtol = RTOL if prec == "HM_FP64" else 1e-5
    atol = ATOL if prec == "HM_FP64" else 2e-5
    try:
        ctx.set_mps(cid, ctx.get_mps(cid))
        ref = ochain.HybridChain(seed=9, chain_id=2, **cfg)
        for _ in range(2):
            ctx.evolve([cid])
            obs = ctx.measure([cid], b.num_obs(p))[0]
            env, _ = ctx.collapse([cid], b.num_env(p))
            r = ref.sample()
            assert np.abs(obs - r["obs"]).max() <= rtol * np.abs(r["obs"]).max() + atol, (obs, r["obs"])
            assert list(env[0]) == r["env_out"]
        st = np.zeros(b.HM_NUM_STATS)
        st[:] = ctx.stats(cid)
        assert st[5] > 64                      # the bond grew past the shared-memory block size
    finally:
        ctx.free_chain(cid)
