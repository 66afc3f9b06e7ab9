"""The host side of the C ABI, run on the CPU (no GPU).

``hm_api.cu`` is compiled as plain C++ with test-only stand-ins for the
CUDA runtime and the kernel launchers (``tests/host_abi/``).
Device memory is host memory, and each launcher records the batch it was
handed. The tests read back what the kernels would receive: the chain image
(op list, gate table, counters, environment), the launch order and batch
sizes, and the arena's admission decisions and state errors. Every value
checked here is produced by the product's own host code.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1910_09142_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
K_EVOLVE64, K_EVOLVE_MIXED, K_MEASURE, K_COLLAPSE, K_RESET, K_SUSCEPT = range(6)


@pytest.fixture(scope="module")
def host(tmp_path_factory):
    cxx = shutil.which("g++")
    inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    if not cxx or not os.path.exists(os.path.join(inc, "cuda_runtime_api.h")):
        pytest.skip("needs g++ and the CUDA headers")
    out = str(tmp_path_factory.mktemp("host_abi") / "libhm_host.so")
    src = [os.path.join(ROOT, "paper_1910_09142_gb300", "csrc", "hm_api.cu"),
           os.path.join(ROOT, "tests", "host_abi", "cuda_runtime_stub.cpp"),
           os.path.join(ROOT, "tests", "host_abi", "launch_recorder.cpp")]
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-shared", "-fPIC", "-x", "c++", *src,
                        "-I" + inc, "-o", out, "-ldl", "-Wl,-Bsymbolic"],   # the stub, not a loaded cudart
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lib = ctypes.CDLL(out)
    P, vp, i32, i64 = ctypes.POINTER, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sig = {"hm_create": [P(vp), ctypes.c_int, vp, ctypes.c_size_t, vp], "hm_destroy": [vp],
           "hm_init_chain": [vp, P(binding.Params), vp, P(i64)],
           "hm_resume_chain": [vp, P(binding.Params), vp, i64, P(i64)],
           "hm_free_chain": [vp, i64], "hm_evolve": [vp, P(i64), i32],
           "hm_measure_cluster": [vp, P(i64), i32, vp, i32], "hm_collapse": [vp, P(i64), i32, vp, vp],
           "hm_apply_ops": [vp, i64, vp, i32], "hm_query_memory": [P(binding.Params), P(ctypes.c_size_t)],
           "hmtest_launch": [ctypes.c_int] + [P(ctypes.c_int)] * 5,
           "hmtest_launch_chain": [ctypes.c_int, ctypes.c_int], "hmtest_chain_ints": [vp, P(i32)],
           "hmtest_chain_ops": [vp], "hmtest_chain_gates": [vp], "hmtest_chain_env": [vp],
           "hmtest_chain_chi": [vp],
           "hm_get_mps": [vp, i64, P(i32), i32, vp, ctypes.c_size_t, P(i32), P(ctypes.c_size_t)],
           "hm_set_mps": [vp, i64, P(i32), i32, vp, ctypes.c_size_t, i32, i32]}
    for name, args in sig.items():
        getattr(lib, name).argtypes = args
    lib.hmtest_launch_chain.restype = vp
    lib.hmtest_chain_ops.restype = P(i32)
    lib.hmtest_chain_gates.restype = P(ctypes.c_double)
    lib.hmtest_chain_env.restype = P(i32)
    lib.hmtest_chain_chi.restype = P(i32)
    return lib


class Ctx:
    """A context over a host buffer standing in for device memory."""

    def __init__(self, lib, nbytes):
        self.lib = lib
        self.mem = np.zeros(nbytes + 256, dtype=np.uint8)
        base = self.mem.ctypes.data
        self.base = base + (-base) % 256
        self.h = ctypes.c_void_p()
        assert lib.hm_create(ctypes.byref(self.h), 0, ctypes.c_void_p(self.base), nbytes, None) == 0

    def init(self, p, env=None, n=0):
        out = ctypes.c_int64()
        e = None if env is None else np.ascontiguousarray(np.asarray(env, dtype=np.int8))
        ptr = None if e is None else e.ctypes.data_as(ctypes.c_void_p)
        rc = (self.lib.hm_resume_chain(self.h, ctypes.byref(p), ptr, n, ctypes.byref(out)) if n
              else self.lib.hm_init_chain(self.h, ctypes.byref(p), ptr, ctypes.byref(out)))
        return rc, out.value

    def ids(self, ids):
        a = np.ascontiguousarray(np.asarray(ids, dtype=np.int64))
        return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))

    def close(self):
        self.lib.hm_destroy(self.h)


def _launches(lib):
    out = []
    k, n, t0, t1, x = (ctypes.c_int() for _ in range(5))
    for i in range(lib.hmtest_n_launches()):
        lib.hmtest_launch(i, *(ctypes.byref(v) for v in (k, n, t0, t1, x)))
        out.append(dict(kind=k.value, n=n.value, t0=t0.value, t1=t1.value, extra=x.value,
                        chains=[lib.hmtest_launch_chain(i, j) for j in range(n.value)]))
    return out


def _ints(lib, c):
    v = (ctypes.c_int32 * 8)()
    lib.hmtest_chain_ints(c, v)
    keys = ("n_sites", "n_ops", "n_gates", "n_env", "n", "basis", "basis_zx", "chi_max")
    return dict(zip(keys, list(v)))


@pytest.mark.parametrize("schedule", ["plain", "fused"])
def test_chain_image_holds_the_planned_ops_and_gates(host, schedule):
    ctx = Ctx(host, 64 << 20)
    p = binding.params(4, 4, beta=0.6, tau=0.1, chi_max=32, schedule=schedule)
    host.hmtest_clear()
    rc, cid = ctx.init(p)
    assert rc == 0
    (reset,) = _launches(host)
    assert reset["kind"] == K_RESET and reset["extra"] == 1 and reset["n"] == 1     # draws the first env
    c = reset["chains"][0]
    info = _ints(host, c)
    ops = binding.plan(p)
    gates = binding.gates(p)
    assert info["n_ops"] == len(ops) and info["n_gates"] == len(gates)
    assert (info["n"], info["basis"], info["basis_zx"]) == (0, 0, 1)
    got_ops = np.ctypeslib.as_array(host.hmtest_chain_ops(c), shape=(len(ops) * 4,)).reshape(-1, 4)
    assert np.array_equal(got_ops, ops)
    got_g = np.ctypeslib.as_array(host.hmtest_chain_gates(c), shape=(len(gates) * 81,)).reshape(-1, 9, 9)
    assert np.array_equal(got_g, gates)
    ctx.close()


@pytest.mark.parametrize("basis_zx,n,basis", [(True, 1, 0), (True, 2, 1), (True, 3, 0), (True, 8, 1),
                                              (False, 2, 0), (False, 7, 0)])
def test_resume_presets_sample_index_and_basis(host, basis_zx, n, basis):
    ctx = Ctx(host, 64 << 20)
    p = binding.params(5, 2, beta=0.4, tau=0.1, chi_max=16, basis_zx=basis_zx)
    n_env = binding.num_env(p)
    env = np.arange(n_env) % 3
    host.hmtest_clear()
    rc, _ = ctx.init(p, env, n)
    assert rc == 0
    (reset,) = _launches(host)
    assert reset["kind"] == K_RESET and reset["extra"] == 0                       # uses the given env
    c = reset["chains"][0]
    info = _ints(host, c)
    assert (info["n"], info["basis"]) == (n, basis)
    assert list(np.ctypeslib.as_array(host.hmtest_chain_env(c), shape=(n_env,))) == list(env)
    assert ctx.init(p, None, 2)[0] == binding.HM_ERR_ARG                          # no outcomes
    assert ctx.init(p, env, -1)[0] == binding.HM_ERR_ARG
    bad = env.copy()
    bad[0] = 3
    assert ctx.init(p, bad, 2)[0] == binding.HM_ERR_ARG
    ctx.close()


def test_admission_and_reuse_of_freed_memory(host):
    p = binding.params(6, 4, beta=0.4, tau=0.1, chi_max=32)
    need = binding.query_memory(p)
    ctx = Ctx(host, 3 * need + 4096)
    ids = []
    for _ in range(3):
        rc, cid = ctx.init(p)
        assert rc == 0
        ids.append(cid)
    rc, _ = ctx.init(p)
    assert rc == binding.HM_ERR_NOMEM                                             # refused, nothing allocated
    assert host.hm_free_chain(ctx.h, ids[1]) == 0
    rc, again = ctx.init(p)
    assert rc == 0 and again not in ids                                           # the freed block is reused
    for cid in (ids[0], ids[2], again):
        assert host.hm_free_chain(ctx.h, cid) == 0
    wide = binding.params(6, 4, beta=0.4, tau=0.1, chi_max=48)
    assert 2 * need < binding.query_memory(wide) < 3 * need
    assert ctx.init(wide)[0] == 0                         # the three freed blocks coalesced into one
    ctx.close()


def _init_tracked(host, ctx, p, where):
    """Create a chain and remember its descriptor address (from its reset launch)."""
    host.hmtest_clear()
    rc, cid = ctx.init(p)
    assert rc == 0
    where[_launches(host)[0]["chains"][0]] = cid
    return cid


def test_evolve_launches_costliest_chains_first(host):
    ctx = Ctx(host, 256 << 20)
    small = binding.params(3, 2, beta=0.4, tau=0.1, chi_max=16)
    big = binding.params(8, 4, beta=0.4, tau=0.1, chi_max=64)
    mid = binding.params(5, 4, beta=0.4, tau=0.1, chi_max=32)
    where = {}
    ids = [_init_tracked(host, ctx, p, where) for p in (small, big, small, mid, big)]
    host.hmtest_clear()
    a, ptr = ctx.ids(ids)
    assert host.hm_evolve(ctx.h, ptr, len(a)) == 0
    (ev,) = _launches(host)
    assert ev["kind"] == K_EVOLVE64 and ev["n"] == 5
    assert [where[c] for c in ev["chains"]] == [ids[1], ids[4], ids[3], ids[0], ids[2]]   # stable
    assert host.hm_evolve(ctx.h, ptr, len(a)) == binding.HM_ERR_STATE              # already evolved
    ctx.close()


def test_batches_of_448_and_op_chunks_of_4096(host):
    p = binding.params(2, 0, beta=0.2, tau=0.1, chi_max=4)
    long = binding.params(2, 2, beta=40.0, tau=0.005, chi_max=4)                  # 4000 steps
    ctx = Ctx(host, 900 * binding.query_memory(p) + binding.query_memory(long) + (1 << 20))
    ids = [ctx.init(p)[1] for _ in range(900)]
    lid = ctx.init(long)[1]
    n_long, n_short = len(binding.plan(long)), len(binding.plan(p))
    assert n_long > 4096 and n_short <= 4096
    host.hmtest_clear()
    a, ptr = ctx.ids(ids + [lid])
    assert host.hm_evolve(ctx.h, ptr, len(a)) == 0
    ev = _launches(host)
    chunks = (n_long + 4095) // 4096
    # the long chain sorts first; only its batch of 448 runs every op chunk
    assert [(l["n"], l["t0"], l["t1"]) for l in ev] == \
        [(448, 4096 * i, 4096 * (i + 1)) for i in range(chunks)] + [(448, 0, 4096), (5, 0, 4096)]
    ctx.close()


def test_precisions_run_in_separate_launches_and_state_errors(host):
    ctx = Ctx(host, 256 << 20)
    p64 = binding.params(3, 2, beta=0.4, tau=0.1, chi_max=16)
    p32 = binding.params(3, 2, beta=0.4, tau=0.1, chi_max=16, precision=binding.HM_MIXED)
    ids = [ctx.init(p64)[1], ctx.init(p32)[1]]
    a, ptr = ctx.ids(ids)
    out = np.zeros((2, binding.num_obs(p64)))
    assert host.hm_measure_cluster(ctx.h, ptr, 2, out.ctypes.data_as(ctypes.c_void_p), out.shape[1]) \
        == binding.HM_ERR_STATE                                                    # not evolved yet
    host.hmtest_clear()
    assert host.hm_evolve(ctx.h, ptr, 2) == 0
    kinds = [l["kind"] for l in _launches(host)]
    assert kinds == [K_EVOLVE64, K_EVOLVE_MIXED]
    assert host.hm_measure_cluster(ctx.h, ptr, 2, out.ctypes.data_as(ctypes.c_void_p), out.shape[1] + 1) \
        == binding.HM_ERR_ARG                                                      # wrong n_obs
    assert host.hm_collapse(ctx.h, ptr, 2, None, None) == 0
    assert host.hm_collapse(ctx.h, ptr, 2, None, None) == binding.HM_ERR_STATE      # evolve first
    ctx.close()


def test_apply_ops_accepts_the_fused_product_gates_only_inside_the_table(host):
    ctx = Ctx(host, 64 << 20)
    p = binding.params(4, 4, beta=0.6, tau=0.1, chi_max=32, schedule="fused")
    _, cid = ctx.init(p)
    n_gates = len(binding.gates(p))
    for gate, want in ((n_gates - 1, 0), (n_gates, binding.HM_ERR_ARG)):
        ops = np.array([[0, gate, 1, 0]], dtype=np.int32)
        assert host.hm_apply_ops(ctx.h, cid, ops.ctypes.data_as(ctypes.c_void_p), 1) == want
    ctx.close()


def test_host_outputs_need_a_staging_block_device_outputs_do_not(host):
    p = binding.params(3, 2, beta=0.4, tau=0.1, chi_max=16)
    need = binding.query_memory(p)
    n_obs = binding.num_obs(p)
    ctx = Ctx(host, need + 256)                          # the chain plus the error word, nothing more
    host.hm_measure_cluster_device.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32,
                                               ctypes.c_void_p, ctypes.c_int32]
    rc, cid = ctx.init(p)
    assert rc == 0
    a, ptr = ctx.ids([cid])
    assert host.hm_evolve(ctx.h, ptr, 1) == 0
    out = np.zeros(n_obs)
    assert host.hm_measure_cluster(ctx.h, ptr, 1, out.ctypes.data_as(ctypes.c_void_p), n_obs) \
        == binding.HM_ERR_NOMEM
    dev = np.zeros(n_obs)                                # stands in for a caller's device buffer
    assert host.hm_measure_cluster_device(ctx.h, ptr, 1, dev.ctypes.data_as(ctypes.c_void_p), n_obs) == 0
    assert host.hm_collapse(ctx.h, ptr, 1, None, None) == 0
    ctx.close()


def _set(host, ctx, cid, dims, buf, centre=0, evolved=0, n_sites=None):
    d = np.ascontiguousarray(np.asarray(dims, dtype=np.int32))
    b = np.ascontiguousarray(np.asarray(buf, dtype=np.float64))
    return host.hm_set_mps(ctx.h, cid, d.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                           len(d) - 1 if n_sites is None else n_sites, b.ctypes.data_as(ctypes.c_void_p),
                           len(b), centre, evolved)


def _get(host, ctx, cid, dims_cap=64, cap=None):
    dims = np.zeros(dims_cap, dtype=np.int32)
    n, nd = ctypes.c_int32(), ctypes.c_size_t()
    P32 = ctypes.POINTER(ctypes.c_int32)
    rc = host.hm_get_mps(ctx.h, cid, dims.ctypes.data_as(P32), dims_cap, None, 0, ctypes.byref(n), ctypes.byref(nd))
    if rc:
        return rc, None, None
    buf = np.zeros(max(nd.value if cap is None else cap, 1))
    rc = host.hm_get_mps(ctx.h, cid, dims.ctypes.data_as(P32), dims_cap, buf.ctypes.data_as(ctypes.c_void_p),
                         len(buf) if cap is None else cap, ctypes.byref(n), ctypes.byref(nd))
    return rc, dims[: n.value + 1], buf[: nd.value]


def test_mps_round_trip_and_its_argument_checks(host):
    ctx = Ctx(host, 64 << 20)
    p = binding.params(3, 2, beta=0.4, tau=0.1, chi_max=16)
    where = {}
    cid = _init_tracked(host, ctx, p, where)
    desc = next(iter(where))
    n = 8                                                   # Lx = 3, 2W = 2: 6 physical + 2 ancilla sites
    dims = [1, 3, 9, 16, 16, 16, 9, 3, 1]
    rng = np.random.default_rng(0)
    buf = rng.standard_normal(sum(dims[s] * 3 * dims[s + 1] for s in range(n)))
    assert _set(host, ctx, cid, dims, buf) == 0
    rc, got_dims, got = _get(host, ctx, cid)
    assert rc == 0 and list(got_dims) == dims and np.array_equal(got, buf)
    too_big = list(dims)
    too_big[3] = 17                                         # above chi_max
    bad_cases = [
        _set(host, ctx, cid, too_big, np.zeros(sum(too_big[s] * 3 * too_big[s + 1] for s in range(n)))),
        _set(host, ctx, cid, dims, buf[:-1]),                # wrong length
        _set(host, ctx, cid, dims, buf, centre=2),           # centre must be on site 0
        _set(host, ctx, cid, [2] + dims[1:], np.zeros(10)),  # open boundary needs dim 1
        _set(host, ctx, cid, dims, buf, n_sites=7),          # wrong site count
    ]
    assert bad_cases == [binding.HM_ERR_ARG] * 5
    assert _get(host, ctx, cid, dims_cap=n)[0] == binding.HM_ERR_ARG       # dims buffer needs n + 1
    assert _get(host, ctx, cid, cap=10)[0] == binding.HM_ERR_ARG           # tensor buffer too small
    chi = np.ctypeslib.as_array(host.hmtest_chain_chi(desc), shape=(n + 1,))
    chi[4] = 1000                                           # a corrupted bond dim on the "device"
    assert _get(host, ctx, cid)[0] == binding.HM_ERR_NUMERIC
    ctx.close()


def test_admission_refuses_a_mixed_chain_beyond_the_shared_memory_plan(host):
    ctx = Ctx(host, 1 << 20)
    p = binding.params(32, 8, chi_max=4096, precision=binding.HM_MIXED)
    assert ctx.init(p)[0] == binding.HM_ERR_ARG          # refused before any allocation
    ctx.close()


def test_susceptibility_is_refused_on_a_chain_without_its_workspace(host):
    host.hm_measure_susceptibility.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32,
                                               ctypes.c_void_p]
    ctx = Ctx(host, 256 << 20)
    out = np.zeros(2)
    for sus, want in ((True, 0), (False, binding.HM_ERR_ARG)):
        _, cid = ctx.init(binding.params(3, 2, beta=0.4, tau=0.1, chi_max=16, susceptibility=sus))
        a, ptr = ctx.ids([cid])
        assert host.hm_evolve(ctx.h, ptr, 1) == 0
        host.hmtest_clear()
        assert host.hm_measure_susceptibility(ctx.h, ptr, 1, out.ctypes.data_as(ctypes.c_void_p)) == want
        kinds = [l["kind"] for l in _launches(host)]
        assert kinds == ([K_SUSCEPT] if sus else [])          # never launched without the workspace
        assert host.hm_free_chain(ctx.h, cid) == 0
    ctx.close()
