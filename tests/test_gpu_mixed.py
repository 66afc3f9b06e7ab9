"""Mixed-precision paths (HM_MIXED, HM_MIXED32) vs the FP64 oracle (GPU tests).

Bars, from the method's mixed form (energy within 1e-5 of FP64 per sample):
per-sample energy estimator within 1e-5 relative of the oracle, every
per-bond correlator within 2e-5 absolute, collapse outcomes identical while
the oracle's uniform draw stays more than 1e-6 away from every
cumulative-probability edge, log p within 1e-4 absolute.  Measured on
GB300: energies ~1e-6 relative, for HM_MIXED (binary32 Jacobi finished by
binary64 sweeps) and HM_MIXED32 (binary32 Jacobi only) alike.  The chains
include the small workload (Lx=4, 2W=4, beta=2, chi=64), whose splits cut
at the chi cap: there the oracle's own energy moves by only ~1e-14 under a
1e-16 relative change of the gates, so the 1e-5 bar measures precision, not
chaos at the cut.
"""
import numpy as np
import pytest

from oracle import chain as ochain
from oracle import collapse as ocol

pytestmark = pytest.mark.gpu

E_RTOL, BOND_ATOL, LOGP_ATOL, EDGE = 1e-5, 2e-5, 1e-4, 1e-6
MIXED = ["HM_MIXED", "HM_MIXED32"]


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_1910_09142_gb300 import binding
    assert torch.cuda.is_available()
    c = binding.Context(32 << 30)
    yield c
    c.close()


def _b():
    from paper_1910_09142_gb300 import binding
    return binding


def _sample_with_margin(ref):
    """Oracle sample plus the draw margin of its collapse."""
    st = ref.evolve()
    from oracle import measure as omeas
    obs = omeas.measure(st, ref.meas_bonds)
    basis = ocol.sample_basis(ref.n, ref.basis_zx)
    out, logp, conds = ocol.collapse(st, ref.ladder, basis, ref.seed, ref.chain_id, ref.n)
    margin = 1.0
    for e, p in enumerate(conds):
        u = ocol.uniform(ref.seed, ref.chain_id, ref.n, e)
        acc = np.cumsum(p)
        margin = min(margin, float(np.min(np.abs(acc[:-1] - u))) if len(acc) > 1 else 1.0)
    ref.env, ref.env_basis = out, basis
    ref.n += 1
    return dict(obs=obs, env_out=out, logp=logp), margin


def _compare_chain(ctx, cfg, n_samples, prec, seed=0, chain_id=0):
    b = _b()
    p = b.params(**cfg, precision=getattr(b, prec), seed=seed, chain_id=chain_id)
    cid = ctx.init_chain(p)
    ref = ochain.HybridChain(seed=seed, chain_id=chain_id, **cfg)
    worst_e = worst_b = 0.0
    try:
        for _ in range(n_samples):
            ctx.evolve([cid])
            obs = ctx.measure([cid], b.num_obs(p))[0]
            env, logp = ctx.collapse([cid], b.num_env(p))
            r, margin = _sample_with_margin(ref)
            worst_e = max(worst_e, abs(obs[0] - r["obs"][0]) / abs(r["obs"][0]))
            worst_b = max(worst_b, float(np.abs(obs[1:] - r["obs"][1:]).max()))
            if margin < EDGE:
                break
            assert list(env[0]) == list(r["env_out"])
            assert abs(logp[0] - r["logp"]) < LOGP_ATOL
    finally:
        ctx.free_chain(cid)
    return worst_e, worst_b


@pytest.mark.parametrize("prec", MIXED)
@pytest.mark.parametrize("cfg", [
    dict(Lx=4, two_W=4, J_leg=1.0, J_rung=1.0, beta=2.0, tau=0.1, chi_max=64, cutoff=1e-12),
    dict(Lx=3, two_W=0, J_leg=1.0, J_rung=0.5, beta=1.0, tau=0.1, chi_max=64, cutoff=1e-10),
    dict(Lx=6, two_W=4, J_leg=1.0, J_rung=1.0, beta=1.0, tau=0.05, chi_max=96, cutoff=1e-7),
])
def test_mixed_samples_within_stated_tolerance(ctx, cfg, prec):
    worst_e, worst_b = _compare_chain(ctx, cfg, 3, prec)
    print("%s vs oracle: energy rel %.2e, bond abs %.2e" % (prec, worst_e, worst_b))
    assert worst_e < E_RTOL and worst_b < BOND_ATOL


@pytest.mark.parametrize("prec", MIXED)
def test_mixed_single_rung_closed_form(ctx, prec):
    import math
    b = _b()
    beta = 1.0
    p = b.params(1, 2, beta=beta, tau=0.1, chi_max=16, cutoff=0.0, precision=getattr(b, prec))
    cid = ctx.init_chain(p)
    ctx.evolve([cid])
    obs = ctx.measure([cid], b.num_obs(p))[0]
    e = (-2 * math.exp(2 * beta) - 3 * math.exp(beta) + 5 * math.exp(-beta)) / (
        math.exp(2 * beta) + 3 * math.exp(beta) + 5 * math.exp(-beta))
    assert abs(obs[0] - e) < 1e-6
    ctx.collapse([cid], 0)
    ctx.free_chain(cid)


def test_mixed_and_fp64_chains_in_one_call(ctx):
    """A batch mixing both precisions runs each chain on its own path."""
    b = _b()
    cfg = dict(Lx=3, two_W=2, J_leg=1.0, J_rung=0.5, beta=0.6, tau=0.1, chi_max=32, cutoff=1e-12)
    p64 = b.params(**cfg, seed=1)
    p32 = b.params(**cfg, seed=1, precision=b.HM_MIXED)
    p32b = b.params(**cfg, seed=1, precision=b.HM_MIXED32)
    ids = [ctx.init_chain(p64), ctx.init_chain(p32), ctx.init_chain(p32b)]
    ctx.evolve(ids)
    o = ctx.measure(ids, b.num_obs(p64))
    ref = ochain.HybridChain(seed=1, **cfg).sample()["obs"]
    assert np.allclose(o[0], ref, rtol=1e-10, atol=1e-12)
    for i in (1, 2):
        assert abs(o[i][0] - ref[0]) < E_RTOL * abs(ref[0])
        assert not np.array_equal(o[0], o[i])    # the binary32 path really ran
    for c in ids:
        ctx.free_chain(c)


def test_batch_wider_than_the_gpu_runs_two_chains_per_sm(ctx):
    """A batch of more binary32 chains than SMs goes to the two-chains-per-SM
    kernel (256 threads, 108 KB each): 200 small chains (Lx = 3 and 4, mixed
    cluster sizes) in one call; three of them against the oracle."""
    import torch
    b = _b()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n = max(200, sms + 8)
    cfgs = [dict(Lx=3 + i % 2, two_W=2 * (i % 3), J_leg=1.0, J_rung=0.7, beta=0.8, tau=0.1, chi_max=48,
                 cutoff=1e-10) for i in range(n)]
    ps = [b.params(**c, precision=b.HM_MIXED, seed=2, chain_id=i) for i, c in enumerate(cfgs)]
    ids = [ctx.init_chain(p) for p in ps]
    try:
        ctx.evolve(ids)
        for i in (0, n // 2 + 1, n - 1):
            obs = ctx.measure([ids[i]], b.num_obs(ps[i]))[0]
            r = ochain.HybridChain(seed=2, chain_id=i, **cfgs[i]).sample()
            assert abs(obs[0] - r["obs"][0]) < E_RTOL * abs(r["obs"][0])
            assert np.abs(obs[1:] - r["obs"][1:]).max() < BOND_ATOL
    finally:
        for c in ids:
            ctx.free_chain(c)


@pytest.mark.slow
@pytest.mark.parametrize("prec", MIXED)
def test_ladder16_launch_config_sampled_parity(ctx, prec):
    """Lx=16, 2W=8, chi=256, cutoff 1e-7, beta=1, tau=0.05: 256 chains in the
    benchmark's launch shape (more chains than SMs: two chains per SM); two
    of them checked against the oracle (about 20 s of CPU each)."""
    import synth
    b = _b()
    cfg = synth.ladder("ladder16")
    ps = [b.params(**cfg, precision=getattr(b, prec), seed=0, chain_id=i) for i in range(256)]
    ids = [ctx.init_chain(p) for p in ps]
    try:
        ctx.evolve(ids)
        obs = ctx.measure(ids, b.num_obs(ps[0]))
        env, logp = ctx.collapse(ids, b.num_env(ps[0]))
        assert np.all(np.isfinite(obs)) and np.all(np.isfinite(logp))
        for i in (0, 255):
            ref = ochain.HybridChain(seed=0, chain_id=i, **cfg)
            r, margin = _sample_with_margin(ref)
            assert abs(obs[i][0] - r["obs"][0]) < E_RTOL * abs(r["obs"][0])
            assert np.abs(obs[i][1:] - r["obs"][1:]).max() < BOND_ATOL
            if margin >= EDGE:
                assert list(env[i]) == list(r["env_out"])
    finally:
        for c in ids:
            ctx.free_chain(c)
