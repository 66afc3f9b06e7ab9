"""ctypes binding of the C ABI in ``include/hmetts.h`` (argument marshalling only).

Every step of the sample path runs inside ``libhmetts.so``; this module only
converts Python arguments to C ones.  PyTorch supplies the device arena and
the CUDA stream.  Loading fails loudly when the library has not been built:
there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

from . import build as _build

HM_OK = 0
HM_ERR_ARG = -1
HM_ERR_NOMEM = -2
HM_ERR_CUDA = -3
HM_ERR_NUMERIC = -4
HM_ERR_TIMEOUT = -5
HM_ERR_STATE = -6
HM_FP64 = 0
HM_MIXED = 1
HM_MIXED32 = 2
HM_ZX_ALTERNATE = 0
HM_Z_ONLY = 1
HM_SCHED_PLAIN = 0
HM_SCHED_FUSED = 1
HM_NUM_STATS = 12
SCHEDULES = {"plain": HM_SCHED_PLAIN, "fused": HM_SCHED_FUSED}

_ERRNAMES = {HM_ERR_ARG: "HM_ERR_ARG", HM_ERR_NOMEM: "HM_ERR_NOMEM", HM_ERR_CUDA: "HM_ERR_CUDA",
             HM_ERR_NUMERIC: "HM_ERR_NUMERIC", HM_ERR_TIMEOUT: "HM_ERR_TIMEOUT",
             HM_ERR_STATE: "HM_ERR_STATE"}

EXPORTS = ["hm_create", "hm_destroy", "hm_query_memory", "hm_num_obs", "hm_num_env", "hm_init_chain",
           "hm_free_chain", "hm_evolve", "hm_measure_cluster", "hm_measure_cluster_device",
           "hm_collapse", "hm_collapse_device", "hm_chain_stats", "hm_get_mps", "hm_set_mps",
           "hm_apply_ops", "hm_plan", "hm_gates", "hm_last_error", "hm_two_site_update_static",
           "hm_measure_susceptibility", "hm_resume_chain", "hm_collapse_conditionals",
           "hm_evolve_partial"]


class HmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (_ERRNAMES.get(code, str(code)), msg))
        self.code = code


class Params(ctypes.Structure):
    """Mirror of ``hm_params``."""
    _fields_ = [("Lx", ctypes.c_int32), ("two_W", ctypes.c_int32),
                ("J_leg", ctypes.c_double), ("J_rung", ctypes.c_double),
                ("beta", ctypes.c_double), ("tau", ctypes.c_double),
                ("chi_max", ctypes.c_int32), ("cutoff", ctypes.c_double),
                ("precision", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("chain_id", ctypes.c_uint32), ("basis_schedule", ctypes.c_int32),
                ("meas_col_lo", ctypes.c_int32), ("meas_col_hi", ctypes.c_int32),
                ("schedule", ctypes.c_int32), ("no_susceptibility", ctypes.c_int32)]


def params(Lx, two_W, J_leg=1.0, J_rung=1.0, beta=1.0, tau=0.05, chi_max=64, cutoff=1e-12,
           precision=HM_FP64, seed=0, chain_id=0, basis_zx=True, meas_cols=None, schedule="plain",
           susceptibility=True):
    """``schedule``: "plain" / "fused" or HM_SCHED_PLAIN / HM_SCHED_FUSED;
    ``susceptibility=False`` skips the workspace of hm_measure_susceptibility."""
    lo, hi = (-1, -1) if meas_cols is None else meas_cols
    sched = SCHEDULES[schedule] if isinstance(schedule, str) else int(schedule)
    return Params(Lx, two_W, J_leg, J_rung, beta, tau, chi_max, cutoff, precision, seed, chain_id,
                  HM_ZX_ALTERNATE if basis_zx else HM_Z_ONLY, lo, hi, sched, 0 if susceptibility else 1)


_lib = None


def load(path=None):
    """Load ``libhmetts.so`` (built by ``build.py``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError("libhmetts.so not built (%s); run paper_1910_09142_gb300/build.py" % path)
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp, i32, i64, dbl, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
    sig = {
        "hm_create": [P(vp), ctypes.c_int, vp, sz, vp],
        "hm_destroy": [vp],
        "hm_query_memory": [P(Params), P(sz)],
        "hm_num_obs": [P(Params), P(i32)],
        "hm_num_env": [P(Params), P(i32)],
        "hm_init_chain": [vp, P(Params), vp, P(i64)],
        "hm_resume_chain": [vp, P(Params), vp, i64, P(i64)],
        "hm_free_chain": [vp, i64],
        "hm_evolve": [vp, P(i64), i32],
        "hm_measure_cluster": [vp, P(i64), i32, vp, i32],
        "hm_measure_cluster_device": [vp, P(i64), i32, vp, i32],
        "hm_collapse": [vp, P(i64), i32, vp, vp],
        "hm_collapse_device": [vp, P(i64), i32, vp, vp],
        "hm_collapse_conditionals": [vp, P(i64), i32, vp, vp, vp],
        "hm_evolve_partial": [vp, P(i64), i32, i32, vp],
        "hm_chain_stats": [vp, i64, vp],
        "hm_get_mps": [vp, i64, vp, i32, vp, sz, P(i32), P(sz)],
        "hm_set_mps": [vp, i64, vp, i32, vp, sz, i32, i32],
        "hm_apply_ops": [vp, i64, vp, i32],
        "hm_plan": [P(Params), vp, i32, P(i32)],
        "hm_gates": [P(Params), vp, i32, P(i32)],
        "hm_measure_susceptibility": [vp, P(i64), i32, vp],
        "hm_two_site_update_static": [vp, vp, i32, i32, i32, vp, i32, dbl, i32, vp, vp, vp, vp],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.hm_last_error.argtypes = [vp]
    lib.hm_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(rc, ctx=None):
    if rc != HM_OK:
        msg = load().hm_last_error(ctx)
        raise HmError(rc, msg.decode() if msg else "")


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _device_buffer(t, dtype, numel, device, name):
    """Device pointer of a caller tensor the kernels write ``numel`` elements
    into; refuses anything they could write past or misread."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.device.index != device:
        raise ValueError("%s must be a CUDA tensor on cuda:%d" % (name, device))
    if t.dtype != dtype or not t.is_contiguous():
        raise ValueError("%s must be a contiguous %s tensor" % (name, dtype))
    if t.numel() < numel:
        raise ValueError("%s holds %d elements, %d needed" % (name, t.numel(), numel))
    return ctypes.c_void_p(t.data_ptr())


def _ids(ids):
    arr = np.ascontiguousarray(np.asarray(ids, dtype=np.int64))
    return arr, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


# ---- context-free calls (host planner; no GPU) -------------------------------------------

def query_memory(p):
    out = ctypes.c_size_t()
    _check(load().hm_query_memory(ctypes.byref(p), ctypes.byref(out)))
    return out.value


def num_obs(p):
    out = ctypes.c_int32()
    _check(load().hm_num_obs(ctypes.byref(p), ctypes.byref(out)))
    return out.value


def num_env(p):
    out = ctypes.c_int32()
    _check(load().hm_num_env(ctypes.byref(p), ctypes.byref(out)))
    return out.value


def plan(p):
    n = ctypes.c_int32()
    _check(load().hm_plan(ctypes.byref(p), None, 0, ctypes.byref(n)))
    buf = np.zeros(4 * n.value, dtype=np.int32)
    _check(load().hm_plan(ctypes.byref(p), _ptr(buf), n.value, ctypes.byref(n)))
    return buf.reshape(-1, 4)


def gates(p):
    n = ctypes.c_int32()
    _check(load().hm_gates(ctypes.byref(p), None, 0, ctypes.byref(n)))
    buf = np.zeros(81 * n.value)
    _check(load().hm_gates(ctypes.byref(p), _ptr(buf), n.value, ctypes.byref(n)))
    return buf.reshape(-1, 9, 9)


def two_site_update_static(A, B, gate, chi_max, cutoff, absorb, A_out, B_out, k_out, stream=None):
    """hm_two_site_update_static on torch CUDA tensors (caller-owned buffers).

    A (chi_l, 3, chi_m), B (chi_m, 3, chi_r), gate (81,), outputs sized for
    k = min(3 chi_l, 3 chi_r, chi_max); k_out an int32 tensor of one element.
    """
    import torch
    for name, t in (("A", A), ("B", B), ("gate", gate), ("A_out", A_out), ("B_out", B_out)):
        if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
            raise ValueError("%s must be a contiguous float64 CUDA tensor" % name)
    if k_out.dtype != torch.int32 or not k_out.is_cuda:
        raise ValueError("k_out must be an int32 CUDA tensor")
    s = stream if stream is not None else torch.cuda.current_stream()
    chi_l, _, chi_m = A.shape
    chi_r = B.shape[2]
    _check(load().hm_two_site_update_static(
        ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()), chi_l, chi_m, chi_r,
        ctypes.c_void_p(gate.data_ptr()), chi_max, cutoff, absorb, ctypes.c_void_p(A_out.data_ptr()),
        ctypes.c_void_p(B_out.data_ptr()), ctypes.c_void_p(k_out.data_ptr()), ctypes.c_void_p(s.cuda_stream)))


# ---- context ---------------------------------------------------------------------------

class Context:
    """An ``hm_ctx`` over a torch-allocated device arena on ``device``."""

    def __init__(self, arena_bytes, device=0, stream=None):
        import torch
        self.lib = load()
        self.device = device
        self._arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device="cuda:%d" % device)
        s = stream if stream is not None else torch.cuda.current_stream(device)
        self.stream = s
        h = ctypes.c_void_p()
        _check(self.lib.hm_create(ctypes.byref(h), device, ctypes.c_void_p(self._arena.data_ptr()),
                                  int(arena_bytes), ctypes.c_void_p(s.cuda_stream)))
        self.h = h
        self._n_env = {}                 # chain -> environment sites (collapse output width)

    def close(self):
        if getattr(self, "h", None):
            self.lib.hm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:       # interpreter shutdown: the library may already be gone
            pass

    def _c(self, rc):
        _check(rc, self.h)

    def init_chain(self, p, env_init=None, next_sample=0):
        """New chain (hm_init_chain), or with ``next_sample`` >= 1 a chain
        resumed from its checkpoint (hm_resume_chain): ``env_init`` are then
        the outcomes the collapse of sample next_sample - 1 returned."""
        out = ctypes.c_int64()
        env = None if env_init is None else np.ascontiguousarray(np.asarray(env_init, dtype=np.int8))
        if next_sample:
            self._c(self.lib.hm_resume_chain(self.h, ctypes.byref(p), _ptr(env), int(next_sample),
                                             ctypes.byref(out)))
        else:
            self._c(self.lib.hm_init_chain(self.h, ctypes.byref(p), _ptr(env), ctypes.byref(out)))
        self._n_env[out.value] = num_env(p)
        return out.value

    def free_chain(self, cid):
        self._c(self.lib.hm_free_chain(self.h, cid))
        self._n_env.pop(cid, None)

    def evolve(self, ids):
        arr, ptr = _ids(ids)
        self._c(self.lib.hm_evolve(self.h, ptr, len(arr)))

    def synchronize(self):
        """Wait for every call issued on the context's stream."""
        self.stream.synchronize()

    def evolve_partial(self, ids, max_ops):
        """Advance each chain's evolution by <= max_ops ops; returns a bool
        array: True where the chain is now evolved."""
        arr, ptr = _ids(ids)
        done = np.zeros(len(arr), dtype=np.int32)
        self._c(self.lib.hm_evolve_partial(self.h, ptr, len(arr), int(max_ops), _ptr(done)))
        return done.astype(bool)

    def measure(self, ids, n_obs):
        arr, ptr = _ids(ids)
        out = np.zeros((len(arr), n_obs))
        self._c(self.lib.hm_measure_cluster(self.h, ptr, len(arr), _ptr(out), n_obs))
        return out

    def measure_device(self, ids, out_tensor):
        """Observables into a (len(ids), n_obs) float64 CUDA tensor, asynchronously."""
        import torch
        arr, ptr = _ids(ids)
        n_obs = out_tensor.shape[-1]
        buf = _device_buffer(out_tensor, torch.float64, len(arr) * n_obs, self.device, "out_tensor")
        self._c(self.lib.hm_measure_cluster_device(self.h, ptr, len(arr), buf, n_obs))

    def susceptibility(self, ids):
        """(chi_M, double sum) per chain, Eq. sus."""
        arr, ptr = _ids(ids)
        out = np.zeros((len(arr), 2))
        self._c(self.lib.hm_measure_susceptibility(self.h, ptr, len(arr), _ptr(out)))
        return out

    def collapse(self, ids, n_env):
        arr, ptr = _ids(ids)
        env = np.zeros((len(arr), max(n_env, 1)), dtype=np.int8)
        logp = np.zeros(len(arr))
        self._c(self.lib.hm_collapse(self.h, ptr, len(arr), _ptr(env), _ptr(logp)))
        return env[:, :n_env], logp

    def collapse_conditionals(self, ids, n_env):
        """Collapse and reset; returns (outcomes, log p, conditional
        probabilities of shape (len(ids), n_env, 3))."""
        arr, ptr = _ids(ids)
        env = np.zeros((len(arr), max(n_env, 1)), dtype=np.int8)
        logp = np.zeros(len(arr))
        cond = np.zeros((len(arr), max(n_env, 1), 3))
        self._c(self.lib.hm_collapse_conditionals(self.h, ptr, len(arr), _ptr(env), _ptr(logp), _ptr(cond)))
        return env[:, :n_env], logp, cond[:, :n_env]

    def collapse_device(self, ids, env_tensor=None, logp_tensor=None):
        """Collapse and reset, asynchronously; outcomes into an int8 CUDA tensor
        of (len(ids), n_env) and log-probabilities into a float64 one of
        len(ids), either may be None.  Every chain must have the same n_env
        when env_tensor is given."""
        import torch
        arr, ptr = _ids(ids)
        e = lp = None
        if env_tensor is not None:
            widths = {self._n_env.get(int(c), 0) for c in arr}
            if len(widths) > 1:
                raise ValueError("chains of one collapse call must share n_env when env_tensor is given")
            n_env = widths.pop() if widths else 0
            e = _device_buffer(env_tensor, torch.int8, len(arr) * n_env, self.device, "env_tensor")
        if logp_tensor is not None:
            lp = _device_buffer(logp_tensor, torch.float64, len(arr), self.device, "logp_tensor")
        self._c(self.lib.hm_collapse_device(self.h, ptr, len(arr), e, lp))

    def stats(self, cid):
        out = np.zeros(HM_NUM_STATS)
        self._c(self.lib.hm_chain_stats(self.h, cid, _ptr(out)))
        return out

    def get_mps(self, cid):
        n = ctypes.c_int32()
        nd = ctypes.c_size_t()
        dims = np.zeros(4096, dtype=np.int32)
        self._c(self.lib.hm_get_mps(self.h, cid, _ptr(dims), len(dims), None, 0, ctypes.byref(n), ctypes.byref(nd)))
        buf = np.zeros(max(nd.value, 1))
        self._c(self.lib.hm_get_mps(self.h, cid, _ptr(dims), len(dims), _ptr(buf), len(buf), ctypes.byref(n),
                                    ctypes.byref(nd)))
        dims = dims[: n.value + 1].copy()
        out, o = [], 0
        for s in range(n.value):
            sz = dims[s] * 3 * dims[s + 1]
            out.append(buf[o:o + sz].reshape(dims[s], 3, dims[s + 1]).copy())
            o += sz
        return out

    def set_mps(self, cid, tensors, evolved=False):
        dims = np.array([t.shape[0] for t in tensors] + [tensors[-1].shape[2]], dtype=np.int32)
        buf = np.ascontiguousarray(np.concatenate([np.asarray(t, dtype=np.float64).reshape(-1) for t in tensors]))
        self._c(self.lib.hm_set_mps(self.h, cid, _ptr(dims), len(tensors), _ptr(buf), len(buf), 0,
                                    1 if evolved else 0))

    def apply_ops(self, cid, ops):
        arr = np.ascontiguousarray(np.asarray(ops, dtype=np.int32).reshape(-1, 4))
        self._c(self.lib.hm_apply_ops(self.h, cid, _ptr(arr), len(arr)))
