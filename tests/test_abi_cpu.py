"""The C-ABI library: build, exported symbols and its host-side logic (no GPU).

The host planner and gate table of the CUDA library are independent
implementations of the same schedule the oracle follows; here they are
compared op by op and entry by entry, through the C ABI.
"""
import os
import re

import numpy as np
import pytest

from oracle import model
from paper_1910_09142_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(build.LIB):
        build.build()
    return binding.load()


def _header_symbols():
    text = open(os.path.join(ROOT, "include", "hmetts.h")).read()
    return sorted(set(re.findall(r"^(?:int|const char\*)\s+(hm_\w+)\s*\(", text, flags=re.M)))


def test_exports_every_declared_symbol(lib):
    syms = _header_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(lib, s), s
    assert sorted(binding.EXPORTS) == syms


CASES = [(16, 8), (4, 4), (1, 2), (3, 0), (2, 4), (5, 2), (6, 12)]


def _oracle_ops_as_abi(lad, n_steps):
    """Oracle op list in the CUDA op encoding (k, gate, absorb, exact)."""
    out = []
    for kind, k, g, absorb in model.plan_ops(lad, n_steps):
        if kind == model.SPLIT:
            gate = 1 if g == model.GATE_SWAP else 2 + (g - 1)
            out.append((k, gate, absorb, 0))
        elif kind == model.MOVE_R:
            out.append((k, 0, 1, 1))
        else:
            out.append((k - 1, 0, 0, 1))
    return np.array(out, dtype=np.int32).reshape(-1, 4)


@pytest.mark.parametrize("Lx,two_W", CASES)
def test_planner_matches_oracle(lib, Lx, two_W):
    beta, tau = 0.6, 0.1
    p = binding.params(Lx, two_W, beta=beta, tau=tau)
    lad = model.Ladder(Lx, two_W)
    n_steps, _ = model.trotter_steps(beta, tau)
    assert np.array_equal(binding.plan(p), _oracle_ops_as_abi(lad, n_steps))


def test_planner_matches_oracle_on_every_small_ladder(lib):
    """Every ladder shape up to Lx = 10 (all even cluster sizes), two steps."""
    for Lx in range(1, 11):
        for two_W in range(0, 2 * Lx + 1, 2):
            p = binding.params(Lx, two_W, beta=0.2, tau=0.05)
            lad = model.Ladder(Lx, two_W)
            assert np.array_equal(binding.plan(p), _oracle_ops_as_abi(lad, 2)), (Lx, two_W)
            assert binding.num_env(p) == len(lad.env)


def _oracle_fused(lad, n_steps, tau_eff):
    ops, gates = model.schedule(lad, n_steps, tau_eff, model.SCHEDULE_FUSED)
    out = []
    for kind, k, g, absorb in ops:
        if kind == model.SPLIT:
            out.append((k, g + 1, absorb, 0))          # oracle 0 = SWAP; library 0 = identity
        elif kind == model.MOVE_R:
            out.append((k, 0, 1, 1))
        else:
            out.append((k - 1, 0, 0, 1))
    return np.array(out, dtype=np.int32).reshape(-1, 4), gates


@pytest.mark.parametrize("Lx,two_W", CASES)
def test_fused_planner_matches_oracle(lib, Lx, two_W):
    """HM_SCHED_FUSED: same ops, same product gates (built independently)."""
    lad = model.Ladder(Lx, two_W, 1.0, 0.7)
    n_steps, teff = model.trotter_steps(0.6, 0.1)
    p = binding.params(Lx, two_W, J_rung=0.7, beta=0.6, tau=0.1, schedule="fused")
    ref_ops, ref_gates = _oracle_fused(lad, n_steps, teff)
    assert np.array_equal(binding.plan(p), ref_ops)
    cg = binding.gates(p)
    assert len(cg) == len(ref_gates) + 1
    for i, g in enumerate(ref_gates):
        assert np.abs(cg[1 + i] - g).max() < 1e-14, i
    plain = binding.plan(binding.params(Lx, two_W, J_rung=0.7, beta=0.6, tau=0.1))
    assert len(ref_ops) < len(plain) or Lx == 1


def test_fused_planner_on_every_small_ladder(lib):
    for Lx in range(1, 9):
        for two_W in range(0, 2 * Lx + 1, 2):
            lad = model.Ladder(Lx, two_W)
            p = binding.params(Lx, two_W, beta=0.2, tau=0.05, schedule=binding.HM_SCHED_FUSED)
            assert np.array_equal(binding.plan(p), _oracle_fused(lad, 2, 0.05)[0]), (Lx, two_W)


def test_fused_schedule_memory(lib):
    # 479 fewer 16-byte ops, 17 more 648-byte product gates: same size to 64 KB
    base = dict(Lx=16, two_W=8, chi_max=256, beta=1.0, tau=0.05)
    plain = binding.query_memory(binding.params(**base))
    fused = binding.query_memory(binding.params(**base, schedule="fused"))
    assert abs(plain - fused) < 64 << 10


def test_planner_beta_zero_is_empty(lib):
    assert len(binding.plan(binding.params(4, 4, beta=0.0))) == 0


@pytest.mark.parametrize("Jl,Jr,tau", [(1.0, 1.0, 0.1), (0.7, 0.5, 0.05), (1.0, 0.0, 0.2)])
def test_gate_table_matches_oracle(lib, Jl, Jr, tau):
    p = binding.params(3, 2, J_leg=Jl, J_rung=Jr, beta=1.0, tau=tau)
    lad = model.Ladder(3, 2, Jl, Jr)
    _, teff = model.trotter_steps(1.0, tau)
    og = model.gate_table(lad, teff)
    cg = binding.gates(p)
    assert len(cg) == len(og) + 1
    assert np.array_equal(cg[0], np.eye(9))
    assert np.array_equal(cg[1], og[0])                       # SWAP
    for b in range(len(lad.bonds)):
        assert np.abs(cg[2 + b] - og[1 + b]).max() < 2e-15


@pytest.mark.parametrize("Lx,two_W,cols", [(16, 8, None), (4, 4, None), (4, 0, None), (5, 2, (0, 5)), (3, 6, (1, 2))])
def test_observable_and_env_counts(lib, Lx, two_W, cols):
    p = binding.params(Lx, two_W, meas_cols=cols)
    lad = model.Ladder(Lx, two_W)
    mb = lad.measured_bonds() if cols is None else lad.measured_bonds(*cols)
    assert binding.num_obs(p) == 1 + 2 * len(mb)
    assert binding.num_env(p) == len(lad.env)


def test_memory_query_scales_with_chi(lib):
    small = binding.query_memory(binding.params(16, 8, chi_max=64))
    big = binding.query_memory(binding.params(16, 8, chi_max=256))
    assert 0 < small < big
    # site tensors alone at the full bond caps: 40 sites x 3 x 256^2 doubles
    assert big > 40 * 3 * 256 * 256 * 8 * 0.5


@pytest.mark.parametrize("kw", [dict(Lx=0, two_W=0), dict(Lx=4, two_W=3), dict(Lx=4, two_W=10),
                                dict(Lx=4, two_W=4, tau=0.0), dict(Lx=4, two_W=4, chi_max=0),
                                dict(Lx=4, two_W=4, cutoff=1.5), dict(Lx=4, two_W=4, beta=-1.0),
                                dict(Lx=4, two_W=4, meas_cols=(3, 2)), dict(Lx=4, two_W=4, schedule=2)])
def test_invalid_parameters_rejected(lib, kw):
    with pytest.raises(binding.HmError) as e:
        binding.num_obs(binding.params(**kw))
    assert e.value.code == binding.HM_ERR_ARG


def test_resume_without_context_is_an_argument_error(lib):
    import ctypes
    out = ctypes.c_int64()
    p = binding.params(3, 2)
    assert lib.hm_resume_chain(None, ctypes.byref(p), None, 2, ctypes.byref(out)) == binding.HM_ERR_ARG


def test_device_output_buffers_are_checked_before_any_launch():
    import torch
    for t in (torch.zeros(6, dtype=torch.float64), np.zeros(6)):        # host memory
        with pytest.raises(ValueError):
            binding._device_buffer(t, torch.float64, 6, 0, "out")


def test_mixed_precision_bond_cap_limit(lib):
    """The binary32 evolve stages column blocks in shared memory: its largest
    bond cap must fit 227 KB; FP64 has no such limit."""
    assert binding.query_memory(binding.params(32, 8, chi_max=2048, precision=binding.HM_MIXED)) > 0
    with pytest.raises(binding.HmError) as e:
        binding.query_memory(binding.params(32, 8, chi_max=4096, precision=binding.HM_MIXED))
    assert e.value.code == binding.HM_ERR_ARG
    assert binding.query_memory(binding.params(32, 8, chi_max=4096)) > 0


def test_susceptibility_workspace_is_optional(lib):
    full = binding.query_memory(binding.params(16, 8, chi_max=256, cutoff=1e-7))
    lean = binding.query_memory(binding.params(16, 8, chi_max=256, cutoff=1e-7, susceptibility=False))
    # the workspace holds (20 + 4 |M|) chi^2 doubles, |M| = 8 cluster sites, instead of the
    # measurement's 10 + (measured end sites): about a fifth of this chain
    assert 0.15 * full < full - lean < 0.25 * full
    p = binding.params(4, 4)
    p.no_susceptibility = 2
    with pytest.raises(binding.HmError):
        binding.num_obs(p)


def test_large_and_uneven_workloads_fit_their_memory_budgets(lib):
    """The Lx = 32, chi = 512 ladder (128 chains) and the uneven batch of 1024
    chains (Lx in {8, 16, 24, 32}, 2W in {4, 8}, beta log-uniform on
    [0.5, 16], chi_max in {64, 128, 256, 512}) are accepted by the planner and
    fit the 180 GB the workloads allow, by the library's own memory query; the
    uneven batch's op lists span two orders of magnitude, which is why launches
    go costliest chain first and serving slices evolutions per tick."""
    import synth
    p32 = binding.params(**synth.ladder("ladder32"), precision=binding.HM_MIXED)
    assert 128 * binding.query_memory(p32) < 180e9
    assert len(binding.plan(p32)) > 0
    batch = [binding.params(**cfg, precision=binding.HM_MIXED, chain_id=i)
             for i, cfg in enumerate(synth.uneven_batch(1024, seed=0))]
    total = sum(binding.query_memory(p) for p in batch)
    ops = [len(binding.plan(p)) for p in batch]
    assert total < 180e9
    assert min(ops) > 0 and max(ops) > 50 * min(ops)
