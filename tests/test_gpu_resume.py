"""Checkpoint / resume of a chain through hm_resume_chain (GPU tests).

Between samples a chain is only its environment outcomes and its sample
index, because step 4 of Sec. I.C.1 resets the cluster to Bell pairs.  A
chain resumed from the outcomes of sample n-1 at index n must repeat the
uninterrupted chain exactly: same kernels, same inputs, same Philox
counters, so the FP64 observables, outcomes and log-probabilities are
bit-identical.  Resuming after an odd sample checks the S^x-basis reading of
the stored outcomes, and after an even one the S^z reading.
"""
import ctypes

import numpy as np
import pytest

from oracle import chain as ochain

pytestmark = pytest.mark.gpu

CFG = dict(Lx=4, two_W=4, J_leg=1.0, J_rung=0.7, beta=0.8, tau=0.1, chi_max=32, cutoff=1e-10)


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_1910_09142_gb300 import binding
    assert torch.cuda.is_available()
    c = binding.Context(1 << 30)
    yield c
    c.close()


def _run(ctx, cid, p, n):
    from paper_1910_09142_gb300 import binding as b
    out = []
    for _ in range(n):
        ctx.evolve([cid])
        obs = ctx.measure([cid], b.num_obs(p))[0]
        env, logp = ctx.collapse([cid], b.num_env(p))
        out.append((obs, np.array(env[0]), float(logp[0])))
    return out


@pytest.mark.parametrize("cut", [2, 3])
def test_resumed_chain_repeats_the_uninterrupted_one(ctx, cut):
    from paper_1910_09142_gb300 import binding as b
    p = b.params(**CFG, seed=4, chain_id=6)
    full = ctx.init_chain(p)
    try:
        recs = _run(ctx, full, p, cut + 2)
    finally:
        ctx.free_chain(full)
    res = ctx.init_chain(p, env_init=recs[cut - 1][1], next_sample=cut)
    try:
        again = _run(ctx, res, p, 2)
    finally:
        ctx.free_chain(res)
    for (o1, e1, l1), (o2, e2, l2) in zip(recs[cut:], again):
        assert np.array_equal(o1, o2) and np.array_equal(e1, e2) and l1 == l2
    ref = ochain.HybridChain(seed=4, chain_id=6, **CFG)
    for r, (o, e, _) in zip([ref.sample() for _ in range(cut + 2)][cut:], again):
        assert np.allclose(o, r["obs"], rtol=1e-10, atol=1e-12) and list(e) == r["env_out"]


def test_resume_argument_errors(ctx):
    from paper_1910_09142_gb300 import binding as b
    p = b.params(**CFG)
    n_env = b.num_env(p)
    with pytest.raises(b.HmError) as e:                     # no outcomes to resume from
        ctx.init_chain(p, env_init=None, next_sample=2)
    assert e.value.code == b.HM_ERR_ARG
    with pytest.raises(b.HmError) as e:                     # outcome out of range
        ctx.init_chain(p, env_init=np.full(n_env, 3, np.int8), next_sample=2)
    assert e.value.code == b.HM_ERR_ARG
    out = ctypes.c_int64()                                  # index 0 belongs to hm_init_chain
    env = np.zeros(n_env, np.int8)
    rc = ctx.lib.hm_resume_chain(ctx.h, ctypes.byref(p), env.ctypes.data_as(ctypes.c_void_p), 0,
                                 ctypes.byref(out))
    assert rc == b.HM_ERR_ARG
