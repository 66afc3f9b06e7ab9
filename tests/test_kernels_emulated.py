"""The library's CUDA kernels, run on the CPU, against the oracle (no GPU).

``tests/simt/`` compiles ``hm_fp64.cu`` and ``hm_mixed.cu`` as host C++.
Each block's threads are cooperative fibers, __syncthreads and warp
shuffles keep their meaning, and the launches run through the unchanged host
code of ``hm_api.cu``. What runs is the kernel source itself, so these tests
check its logic (indexing, truncation, Philox draws, collapse, reset,
counters) at the GPU parity bars. They do not check GB300 behaviour (timing,
memory model, rounding of the FMA contraction); the ``-m gpu`` tests do.

Tiny chains keep each sample to seconds: Lx = 2, one cluster column,
beta = 0.2 (one Trotter step).
"""
import ctypes
import os
import sys

import numpy as np
import pytest

from oracle import chain as ochain
from oracle import measure as omeasure
from oracle import mps as omps
from paper_1910_09142_gb300 import binding

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "simt"))
import build_emulated  # noqa: E402

pytestmark = pytest.mark.slow

CFG = dict(Lx=2, two_W=2, J_leg=1.0, J_rung=0.7, beta=0.2, tau=0.1, chi_max=16, cutoff=1e-12)
RTOL, ATOL = 1e-10, 1e-12


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    try:
        path = build_emulated.build(str(tmp_path_factory.mktemp("simt")))
    except FileNotFoundError as e:
        pytest.skip(str(e))
    lib = ctypes.CDLL(path)
    P, vp, i32, i64 = ctypes.POINTER, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sig = {"hm_create": [P(vp), ctypes.c_int, vp, ctypes.c_size_t, vp], "hm_destroy": [vp],
           "hm_init_chain": [vp, P(binding.Params), vp, P(i64)],
           "hm_resume_chain": [vp, P(binding.Params), vp, i64, P(i64)],
           "hm_free_chain": [vp, i64], "hm_evolve": [vp, P(i64), i32],
           "hm_measure_cluster": [vp, P(i64), i32, vp, i32], "hm_collapse": [vp, P(i64), i32, vp, vp],
           "hm_measure_susceptibility": [vp, P(i64), i32, vp],
           "hm_evolve_partial": [vp, P(i64), i32, i32, vp],
           "hm_get_mps": [vp, i64, P(i32), i32, vp, ctypes.c_size_t, P(i32), P(ctypes.c_size_t)],
           "hm_last_error": [vp]}
    for name, args in sig.items():
        getattr(lib, name).argtypes = args
    lib.hm_last_error.restype = ctypes.c_char_p
    return lib


class Emu:
    """A context over host memory; chains advance one Markov step at a time."""

    def __init__(self, lib, nbytes=64 << 20):
        self.lib = lib
        self.mem = np.zeros(nbytes + 256, dtype=np.uint8)
        base = self.mem.ctypes.data + (-self.mem.ctypes.data) % 256
        self.h = ctypes.c_void_p()
        assert lib.hm_create(ctypes.byref(self.h), 0, ctypes.c_void_p(base), nbytes, None) == 0

    def _ok(self, rc):
        assert rc == 0, (rc, self.lib.hm_last_error(self.h))

    def init(self, p, env=None, n=0):
        out = ctypes.c_int64()
        e = None if env is None else np.ascontiguousarray(np.asarray(env, dtype=np.int8))
        ptr = None if e is None else e.ctypes.data_as(ctypes.c_void_p)
        self._ok(self.lib.hm_resume_chain(self.h, ctypes.byref(p), ptr, n, ctypes.byref(out)) if n
                 else self.lib.hm_init_chain(self.h, ctypes.byref(p), ptr, ctypes.byref(out)))
        return out.value

    def _ids(self, cid):
        self._a = np.array([cid], dtype=np.int64)
        return self._a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))

    def evolve(self, cid):
        self._ok(self.lib.hm_evolve(self.h, self._ids(cid), 1))

    def measure(self, cid, p):
        out = np.zeros(binding.num_obs(p))
        self._ok(self.lib.hm_measure_cluster(self.h, self._ids(cid), 1, out.ctypes.data_as(ctypes.c_void_p),
                                             len(out)))
        return out

    def collapse(self, cid, p):
        n_env = binding.num_env(p)
        env, lp = np.zeros(max(n_env, 1), dtype=np.int8), np.zeros(1)
        self._ok(self.lib.hm_collapse(self.h, self._ids(cid), 1, env.ctypes.data_as(ctypes.c_void_p),
                                      lp.ctypes.data_as(ctypes.c_void_p)))
        return list(env[:n_env]), float(lp[0])

    def sample(self, cid, p):
        self.evolve(cid)
        obs = self.measure(cid, p)
        env, lp = self.collapse(cid, p)
        return obs, env, lp

    def mps(self, cid):
        dims = np.zeros(64, dtype=np.int32)
        n, nd = ctypes.c_int32(), ctypes.c_size_t()
        P32 = ctypes.POINTER(ctypes.c_int32)
        self._ok(self.lib.hm_get_mps(self.h, cid, dims.ctypes.data_as(P32), 64, None, 0, ctypes.byref(n),
                                     ctypes.byref(nd)))
        buf = np.zeros(nd.value)
        self._ok(self.lib.hm_get_mps(self.h, cid, dims.ctypes.data_as(P32), 64, buf.ctypes.data_as(ctypes.c_void_p),
                                     len(buf), ctypes.byref(n), ctypes.byref(nd)))
        out, o = [], 0
        for s in range(n.value):
            size = dims[s] * 3 * dims[s + 1]
            out.append(buf[o:o + size].reshape(dims[s], 3, dims[s + 1]))
            o += size
        return out

    def close(self):
        self.lib.hm_destroy(self.h)


def _same_state(a, b, tol=1e-10):
    va, vb = omps.MPS(a).to_dense(), omps.MPS(b).to_dense()
    return np.abs(va - np.sign(va @ vb) * vb).max() < tol


@pytest.mark.parametrize("schedule", ["plain", "fused"])
def test_fp64_kernels_match_the_oracle(emu, schedule):
    """Evolved state, observables, outcomes and log p of two samples."""
    e = Emu(emu)
    p = binding.params(**CFG, seed=3, chain_id=1, schedule=schedule)
    cid = e.init(p)
    ref = ochain.HybridChain(seed=3, chain_id=1, schedule=schedule, **CFG)
    for step in range(2):
        e.evolve(cid)
        if step == 0:
            assert _same_state(e.mps(cid), ref.evolve().tensors)
        obs = e.measure(cid, p)
        env, lp = e.collapse(cid, p)
        r = ref.sample()
        assert np.allclose(obs, r["obs"], rtol=RTOL, atol=ATOL)
        assert env == r["env_out"] and abs(lp - r["logp"]) < 1e-9
    e.close()


def test_resume_through_the_kernels_repeats_the_chain(emu):
    """Resume after sample 1 (read in the S^x basis): the reset kernel builds
    the initial state from the preset counters, and sample 2 is bit-identical."""
    e = Emu(emu)
    p = binding.params(**CFG, seed=8, chain_id=2, precision=binding.HM_MIXED)
    cid = e.init(p)
    recs = [e.sample(cid, p) for _ in range(3)]
    again = e.init(p, recs[1][1], 2)
    obs, env, lp = e.sample(again, p)
    assert np.array_equal(obs, recs[2][0]) and env == recs[2][1] and lp == recs[2][2]
    # the binary32 path within its stated tolerance of the oracle
    ref = ochain.HybridChain(seed=8, chain_id=2, **CFG)
    r = ref.sample()
    assert abs(recs[0][0][0] - r["obs"][0]) < 1e-5 * abs(r["obs"][0])
    assert np.abs(recs[0][0][1:] - r["obs"][1:]).max() < 2e-5
    e.close()


def test_susceptibility_kernel_matches_the_oracle(emu):
    e = Emu(emu)
    p = binding.params(**CFG, seed=5)
    cid = e.init(p)
    e.evolve(cid)
    out = np.zeros(2)
    e._ok(emu.hm_measure_susceptibility(e.h, e._ids(cid), 1, out.ctypes.data_as(ctypes.c_void_p)))
    ref = ochain.HybridChain(seed=5, **CFG)
    lad = ref.ladder
    region = sorted({k for i, j, _ in ref.meas_bonds for k in (i, j)})
    chi, raw = omeasure.susceptibility(ref.evolve(), lad, region, CFG["beta"])
    assert abs(out[1] - raw) < 1e-10 * max(1.0, abs(raw)) and abs(out[0] - chi) < 1e-10 * max(1.0, abs(chi))
    e.close()


@pytest.mark.parametrize("cfg,precision", [
    (dict(Lx=1, two_W=2, beta=0.3), binding.HM_FP64),       # single rung, pure ancilla
    (dict(Lx=1, two_W=0, beta=0.3), binding.HM_FP64),       # single rung, METTS
    (dict(Lx=2, two_W=2, beta=0.0), binding.HM_FP64),       # no evolution at all
    (dict(Lx=1, two_W=2, beta=0.3), binding.HM_MIXED),
    (dict(Lx=2, two_W=2, beta=0.0), binding.HM_MIXED),
])
def test_edge_cases_match_the_oracle(emu, cfg, precision):
    full = dict(J_leg=1.0, J_rung=0.7, tau=0.1, chi_max=16, cutoff=1e-12, **cfg)
    e = Emu(emu)
    p = binding.params(**full, seed=4, chain_id=2, precision=precision)
    cid = e.init(p)
    ref = ochain.HybridChain(seed=4, chain_id=2, **full)
    tol = 1e-10 if precision == binding.HM_FP64 else 1e-6
    for _ in range(2):
        obs, env, _ = e.sample(cid, p)
        r = ref.sample()
        assert np.abs(obs - r["obs"]).max() <= tol * max(1.0, np.abs(r["obs"]).max())
        assert env == r["env_out"]
    e.close()


@pytest.mark.parametrize("precision,order", [(binding.HM_FP64, "reverse"), (binding.HM_MIXED, "random:7")])
def test_results_do_not_depend_on_thread_order(emu, precision, order):
    """A race check: nothing orders two threads of a block between barriers,
    so a kernel without data races gives bit-identical results whatever
    order its threads run in.  One Markov step in the default order, then
    the same step with the threads of every phase reversed or shuffled:
    states, observables, outcomes and log p must match exactly."""
    def run():
        e = Emu(emu)
        p = binding.params(**CFG, seed=6, chain_id=3, precision=precision)
        cid = e.init(p)
        e.evolve(cid)
        state = e.mps(cid)
        obs = e.measure(cid, p)
        env, lp = e.collapse(cid, p)
        e.close()
        return state, obs, env, lp
    old = os.environ.get("SIMT_ORDER")
    try:
        os.environ["SIMT_ORDER"] = "forward"
        a = run()
        os.environ["SIMT_ORDER"] = order
        b = run()
    finally:
        if old is None:
            os.environ.pop("SIMT_ORDER", None)
        else:
            os.environ["SIMT_ORDER"] = old
    assert all(np.array_equal(x, y) for x, y in zip(a[0], b[0]))
    assert np.array_equal(a[1], b[1]) and a[2] == b[2] and a[3] == b[3]


def test_allocation_free_update_matches_the_oracle_split(emu):
    """hm_two_site_update_static (its scratch is a file-scope device array,
    here host memory): the truncated two-site product equals the oracle's
    split of the same tensors, and the kept side is an isometry."""
    from oracle import model
    emu.hm_two_site_update_static.argtypes = [ctypes.c_void_p] * 2 + [ctypes.c_int32] * 3 + [
        ctypes.c_void_p, ctypes.c_int32, ctypes.c_double, ctypes.c_int32] + [ctypes.c_void_p] * 4
    rng = np.random.default_rng(11)
    chi_l, chi_m, chi_r, chi_max, cutoff = 4, 6, 5, 7, 1e-12
    A = rng.standard_normal((chi_l, 3, chi_m))
    B = rng.standard_normal((chi_m, 3, chi_r))
    gate = model.bond_gate(0.05)
    for absorb in (model.ABSORB_L, model.ABSORB_R):
        kmax = min(3 * chi_l, 3 * chi_r, chi_max)
        oA, oB = np.full(chi_l * 3 * kmax, np.nan), np.full(kmax * 3 * chi_r, np.nan)
        kk = np.zeros(1, dtype=np.int32)
        g = np.ascontiguousarray(gate.reshape(-1))
        rc = emu.hm_two_site_update_static(A.ctypes.data, B.ctypes.data, chi_l, chi_m, chi_r, g.ctypes.data,
                                           chi_max, cutoff, absorb, oA.ctypes.data, oB.ctypes.data,
                                           kk.ctypes.data, None)
        assert rc == 0
        k = int(kk[0])
        st = omps.MPS([A.copy(), B.copy()], 0 if absorb == model.ABSORB_L else 1)
        st.centre = 0
        omps.split(st, 0, gate, absorb, chi_max, cutoff)
        assert k == st.tensors[0].shape[2]
        got = oA[: chi_l * 3 * k].reshape(-1, k) @ oB[: k * 3 * chi_r].reshape(k, -1)
        want = st.tensors[0].reshape(-1, k) @ st.tensors[1].reshape(k, -1)
        assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()
        iso = oB[: k * 3 * chi_r].reshape(k, -1) if absorb == model.ABSORB_L else oA[: chi_l * 3 * k].reshape(-1, k).T
        assert np.abs(iso @ iso.T - np.eye(k)).max() < 1e-12


def test_partial_evolution_equals_one_evolve(emu):
    """hm_evolve_partial in slices of 7 ops reaches the state of one hm_evolve
    bit for bit (binary64 and binary32 paths), reports completion only on the
    last slice, and leaves the chain ready for measure and collapse."""
    for precision in (binding.HM_FP64, binding.HM_MIXED):
        e = Emu(emu)
        p = binding.params(**CFG, seed=12, chain_id=5, precision=precision)
        whole, sliced = e.init(p), e.init(p)
        e.evolve(whole)
        n_ops = len(binding.plan(p))
        done = np.zeros(1, dtype=np.int32)
        ids = np.array([sliced], dtype=np.int64)
        calls = 0
        while True:
            e._ok(emu.hm_evolve_partial(e.h, ids.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), 1, 7,
                                        done.ctypes.data_as(ctypes.c_void_p)))
            calls += 1
            if done[0]:
                break
            assert calls < n_ops
        assert calls == (n_ops + 6) // 7
        a, b = e.mps(whole), e.mps(sliced)
        assert all(np.array_equal(x, y) for x, y in zip(a, b))
        assert np.array_equal(e.measure(whole, p), e.measure(sliced, p))
        assert e.collapse(whole, p) == e.collapse(sliced, p)
        e.close()


def test_two_chains_per_sm_kernel_matches_the_oracle(emu):
    """A batch of more binary32 chains than SMs (the emulation reports one SM)
    runs two chains per SM, 256 threads each (hm_mixed_pair.cu): both chains
    follow the oracle within the binary32 bars, draw its outcomes, and the
    kernel is race-free (bit-identical under a shuffled thread order)."""
    def run(order):
        old = os.environ.get("SIMT_ORDER")
        os.environ["SIMT_ORDER"] = order
        try:
            e = Emu(emu)
            ps = [binding.params(**CFG, seed=9, chain_id=k, precision=binding.HM_MIXED) for k in (4, 5)]
            ids = np.array([e.init(p) for p in ps], dtype=np.int64)
            P64 = ctypes.POINTER(ctypes.c_int64)
            e._ok(emu.hm_evolve(e.h, ids.ctypes.data_as(P64), 2))
            n_obs = binding.num_obs(ps[0])
            obs = np.zeros((2, n_obs))
            e._ok(emu.hm_measure_cluster(e.h, ids.ctypes.data_as(P64), 2, obs.ctypes.data_as(ctypes.c_void_p), n_obs))
            n_env = binding.num_env(ps[0])
            env, lp = np.zeros((2, max(n_env, 1)), dtype=np.int8), np.zeros(2)
            e._ok(emu.hm_collapse(e.h, ids.ctypes.data_as(P64), 2, env.ctypes.data_as(ctypes.c_void_p),
                                  lp.ctypes.data_as(ctypes.c_void_p)))
            e.close()
            return obs, env[:, :n_env], lp
        finally:
            if old is None:
                os.environ.pop("SIMT_ORDER", None)
            else:
                os.environ["SIMT_ORDER"] = old
    obs, env, lp = run("forward")
    for k, cid in enumerate((4, 5)):
        r = ochain.HybridChain(seed=9, chain_id=cid, **CFG).sample()
        assert abs(obs[k][0] - r["obs"][0]) < 1e-5 * abs(r["obs"][0])
        assert np.abs(obs[k][1:] - r["obs"][1:]).max() < 2e-5
        assert list(env[k]) == r["env_out"]
    obs2, env2, lp2 = run("random:3")
    assert np.array_equal(obs, obs2) and np.array_equal(env, env2) and np.array_equal(lp, lp2)


def test_block_ordered_jacobi_matches_the_oracle(emu):
    """A ladder whose splits have charge blocks of 16 to 19 columns, where the
    binary32 sweeps take the block ordering (super-columns of four, one group
    barrier per super-round): one HM_MIXED sample within the binary32 bars of
    the oracle, the oracle's outcomes, and bit-identical under a shuffled
    thread order (a race check of the warp-local sub-rounds)."""
    cfg = dict(Lx=3, two_W=2, J_leg=1.0, J_rung=0.7, beta=0.6, tau=0.1, chi_max=48, cutoff=1e-10)

    def run(order):
        old = os.environ.get("SIMT_ORDER")
        os.environ["SIMT_ORDER"] = order
        try:
            e = Emu(emu)
            p = binding.params(**cfg, seed=1, chain_id=2, precision=binding.HM_MIXED)
            cid = e.init(p)
            out = e.sample(cid, p)
            e.close()
            return out
        finally:
            if old is None:
                os.environ.pop("SIMT_ORDER", None)
            else:
                os.environ["SIMT_ORDER"] = old
    obs, env, lp = run("forward")
    r = ochain.HybridChain(seed=1, chain_id=2, **cfg).sample()
    assert abs(obs[0] - r["obs"][0]) < 1e-5 * abs(r["obs"][0])
    assert np.abs(obs[1:] - r["obs"][1:]).max() < 2e-5
    assert env == r["env_out"]
    obs2, env2, lp2 = run("random:5")
    assert np.array_equal(obs, obs2) and env == env2 and lp == lp2


def _graded(q, p, lo, seed):
    r = np.random.default_rng(seed)
    U = np.linalg.qr(r.standard_normal((q, p)))[0]
    Vt = np.linalg.qr(r.standard_normal((p, p)))[0]
    return U @ np.diag(np.logspace(0, lo, p)) @ Vt


def _jacobi_cases():
    rng = np.random.default_rng(0)
    noisy = _graded(40, 40, -4, 2)
    # twenty columns at 1e-19 of the rest, partly along them: the case whose
    # overlaps a pair-relative size floor once kept from converging
    noisy[:, 20:] = rng.standard_normal((40, 20)) * 1e-19 + noisy[:, :20] @ rng.standard_normal((20, 20)) * 1e-16
    q1 = np.linalg.qr(rng.standard_normal((36, 36)))[0]
    q2 = np.linalg.qr(rng.standard_normal((36, 36)))[0]
    degenerate = q1 @ np.diag([1.0] * 12 + [0.5] * 12 + [0.25] * 12) @ q2.T   # exact multiplets
    # three scales: columns of order 1, 1e-4 to 1e-2, and 1e-19 to 1e-17 with
    # components along the first; a size floor relative to each pair's
    # larger column (an earlier form of the binary64 tests) never converges
    # on this one, the per-operand scaling does in ~11 sweeps
    r = np.random.default_rng(8)
    big = r.standard_normal((40, 8))
    mid = r.standard_normal((40, 16)) * 10 ** r.uniform(-4, -2, 16)
    tiny = (r.standard_normal((40, 16)) + big @ r.standard_normal((8, 16)) * 10 ** r.uniform(0, 3)) * \
        10 ** r.uniform(-19, -17, 16)
    three = np.hstack([big, mid, tiny])[:, r.permutation(40)]
    return {"graded": _graded(40, 24, -12, 1), "noise_columns": noisy, "degenerate": degenerate,
            "graded_wide": _graded(48, 32, -6, 3), "small": _graded(20, 12, -6, 4), "three_scales": three}


@pytest.mark.parametrize("binary64", [True, False])
@pytest.mark.parametrize("case", ["graded", "noise_columns", "degenerate", "graded_wide", "small", "three_scales"])
def test_block_jacobi_against_numpy(emu, case, binary64):
    """jacobi_group on one block (tests/simt/block_harness.cu), the library's
    Jacobi itself: binary64 with the binary64 kernels' stopping ratio (1e-9),
    binary32 with the mixed kernel's (2e-4; blocks of 16 columns or more take
    the block ordering).  Converged within the sweep limit; singular values
    (the column norms of W) against numpy's SVD; V orthogonal; W = A V; the
    columns of W orthogonal (relative to their norms, above 1e-12 of the
    largest).  Bars: binary64 1e-13, binary32 3e-5 (a few ulp of the
    accumulated rotations)."""
    emu.hm_probe_jacobi.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_double]
    A = _jacobi_cases()[case]
    q, p = A.shape
    dt = np.float64 if binary64 else np.float32
    W = np.asfortranarray(A.astype(dt))
    V = np.asfortranarray(np.eye(p, dtype=dt))
    sweeps = emu.hm_probe_jacobi(W.ctypes.data, q, p, V.ctypes.data, int(binary64), 256, 1e-9 if binary64 else 2e-4)
    assert 1 <= sweeps <= (20 if case == "three_scales" else 60)
    W, V = W.astype(np.float64), V.astype(np.float64)
    bar = 1e-13 if binary64 else 3e-5
    sv = np.sort(np.linalg.norm(W, axis=0))[::-1]
    ref = np.linalg.svd(A, compute_uv=False)
    assert np.abs(sv - ref).max() <= bar * ref[0]
    assert np.abs(V.T @ V - np.eye(p)).max() <= bar
    assert np.abs(W - A @ V).max() <= bar * np.abs(A).max()
    G = W.T @ W
    d = np.sqrt(np.diag(G))
    big = d > 1e-12 * d.max()
    off = np.abs(G - np.diag(np.diag(G)))[np.ix_(big, big)] / np.outer(d[big], d[big])
    assert off.max() <= bar


def test_block_jacobi_is_race_free(emu):
    """Both orderings and both precisions give bit-identical results whatever
    order the threads of the block run in."""
    emu.hm_probe_jacobi.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_double]
    cases = _jacobi_cases()

    def run(A, binary64):
        dt = np.float64 if binary64 else np.float32
        W = np.asfortranarray(A.astype(dt))
        V = np.asfortranarray(np.eye(A.shape[1], dtype=dt))
        emu.hm_probe_jacobi(W.ctypes.data, A.shape[0], A.shape[1], V.ctypes.data, int(binary64), 128,
                            1e-9 if binary64 else 2e-4)
        return W, V
    old = os.environ.get("SIMT_ORDER")
    try:
        for case, binary64 in [("graded_wide", False), ("small", False), ("degenerate", True)]:
            os.environ["SIMT_ORDER"] = "forward"
            a = run(cases[case], binary64)
            os.environ["SIMT_ORDER"] = "random:11"
            b = run(cases[case], binary64)
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), case
    finally:
        if old is None:
            os.environ.pop("SIMT_ORDER", None)
        else:
            os.environ["SIMT_ORDER"] = old


def test_truncation_rule_matches_the_oracle(emu):
    """trunc_rank (the kernels' kept count) against the oracle's rule on the
    same descending values, bit for bit: random spectra over the cutoff and
    chi-cap boundaries, exact multiplets that the tie rule must not split,
    near-ties either side of the 1e-8 relative gap, a single value, and the
    discarded weight landing exactly on the cutoff."""
    from oracle import mps as omps
    emu.hm_probe_trunc.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                                   ctypes.c_void_p]
    rng = np.random.default_rng(21)
    cases = []
    for _ in range(200):
        n = int(rng.integers(1, 120))
        s = np.sort(np.exp(rng.uniform(-12, 0, n)))[::-1]
        cases.append((s, int(rng.integers(1, 130)), float(10 ** rng.uniform(-14, -2))))
    mult = np.repeat([1.0, 0.3, 0.3 * (1 - 5e-9), 0.1, 1e-3], [1, 3, 2, 5, 3])     # a multiplet split by < 1e-8
    for chi in range(1, len(mult) + 1):
        cases.append((np.sort(mult)[::-1], chi, 1e-12))
    near = np.array([1.0, 0.5, 0.5 * (1 - 2e-8), 0.25])                        # a gap just above 1e-8
    cases += [(near, 2, 1e-14), (near, 3, 1e-14), (np.array([0.7]), 4, 1e-7)]
    w = np.array([0.8, 0.6]) ** 2
    cases.append((np.array([0.8, 0.6]), 2, float(w[1] / w.sum())))               # weight exactly at the cutoff
    for s, chi, cut in cases:
        s = np.ascontiguousarray(s, dtype=np.float64)
        tail, total = np.zeros(len(s) + 1), np.zeros(1)
        k = emu.hm_probe_trunc(s.ctypes.data, len(s), chi, cut, tail.ctypes.data, total.ctypes.data)
        assert k == omps.truncation_rank(s, chi, cut), (len(s), chi, cut)
