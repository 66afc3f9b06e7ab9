"""hm_measure_susceptibility (Eq. sus) against the oracle (GPU tests).

FP64 path: chi_M and the double sum within 1e-10 relative of
oracle.measure.susceptibility on the same evolved states; pure-ancilla limit
against 3 sum_q q^2 Z_q / Z of exact diagonalisation (O(tau^2)).
"""
import numpy as np
import pytest

from oracle import chain as ochain
from oracle import ed
from oracle import measure as omeas

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_1910_09142_gb300 import binding
    assert torch.cuda.is_available()
    c = binding.Context(1 << 30)
    yield c
    c.close()


def _region(lad, cols):
    if cols is None:
        cols = (lad.cluster_cols[0], lad.cluster_cols[-1] + 1) if lad.cluster_cols else (0, lad.Lx)
    return sorted(lad.phys[(x, y)] for x in range(*cols) for y in (0, 1))


CFGS = [
    (dict(Lx=3, two_W=2, J_leg=1.0, J_rung=0.5, beta=0.6, tau=0.1, chi_max=64, cutoff=1e-12), None),
    (dict(Lx=4, two_W=4, J_leg=1.0, J_rung=1.0, beta=1.0, tau=0.1, chi_max=64, cutoff=1e-12), None),
    (dict(Lx=3, two_W=0, J_leg=1.0, J_rung=0.7, beta=0.8, tau=0.1, chi_max=64, cutoff=1e-12), (1, 2)),
    (dict(Lx=5, two_W=2, J_leg=1.0, J_rung=1.0, beta=0.8, tau=0.1, chi_max=16, cutoff=1e-8), (1, 4)),
]


def test_susceptibility_matches_oracle(ctx):
    from paper_1910_09142_gb300 import binding as b
    ps = [b.params(**cfg, seed=3, chain_id=i, meas_cols=cols) for i, (cfg, cols) in enumerate(CFGS)]
    ids = [ctx.init_chain(p) for p in ps]
    try:
        ctx.evolve(ids)
        got = ctx.susceptibility(ids)
        for i, (cfg, cols) in enumerate(CFGS):
            ref = ochain.HybridChain(seed=3, chain_id=i, meas_cols=cols, **cfg)
            st = ref.evolve()
            chi_ref, raw_ref = omeas.susceptibility(st, ref.ladder, _region(ref.ladder, cols), cfg["beta"])
            assert abs(got[i][1] - raw_ref) <= 1e-10 * abs(raw_ref) + 1e-12, (i, got[i], raw_ref)
            assert abs(got[i][0] - chi_ref) <= 1e-10 * abs(chi_ref) + 1e-12
    finally:
        for c in ids:
            ctx.free_chain(c)


def test_pure_ancilla_total_spin(ctx):
    from paper_1910_09142_gb300 import binding as b
    Lx, beta = 2, 1.0
    p = b.params(Lx, 2 * Lx, J_rung=0.7, beta=beta, tau=0.025, chi_max=81, cutoff=0.0, meas_cols=(0, Lx))
    cid = ctx.init_chain(p)
    ctx.evolve([cid])
    chi_v, raw = ctx.susceptibility([cid])[0]
    exact = 3.0 * ed.total_sz_squared(ed.LadderED(Lx, 1.0, 0.7), beta)
    assert abs(raw - exact) < 2e-3 * exact
    assert abs(chi_v - beta / 3.0 * raw / (2 * Lx)) < 1e-14
    ctx.collapse([cid], 0)
    ctx.free_chain(cid)


def test_susceptibility_on_mixed_chain_and_state_rules(ctx):
    from paper_1910_09142_gb300 import binding as b
    cfg, cols = CFGS[0]
    p = b.params(**cfg, seed=5, precision=b.HM_MIXED)
    cid = ctx.init_chain(p)
    with pytest.raises(b.HmError) as e:
        ctx.susceptibility([cid])                       # not evolved yet
    assert e.value.code == b.HM_ERR_STATE
    ctx.evolve([cid])
    got = ctx.susceptibility([cid])[0]
    ref = ochain.HybridChain(seed=5, **cfg)
    _, raw_ref = omeas.susceptibility(ref.evolve(), ref.ladder, _region(ref.ladder, None), cfg["beta"])
    assert abs(got[1] - raw_ref) < 1e-3 * abs(raw_ref)   # binary32 evolve tolerance
    ctx.free_chain(cid)
    assert np.isfinite(got).all()
