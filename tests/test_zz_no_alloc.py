"""The allocation-free two-site update, against the regular path (GPU test).

hm_two_site_update_static is for callers that cannot allocate device memory
(for example code inside another framework's memory pool, or a process whose
allocator belongs to someone else): its scratch is a fixed array inside the library.
This test drives it through the C ABI twice in a row on the same inputs and
compares each result with the same update done by the regular entry point
(hm_apply_ops on a chain whose workspace lives in the caller's arena), at the
FP64 tolerance of the other parity tests (1e-10 relative).  What is compared
is what the update fixes uniquely: the kept bond dimension, the truncated
two-site tensor A_out B_out and the orthonormality of the factor that must
be orthonormal; singular vectors inside a degenerate subspace may differ by a
rotation between the two compiled kernels.  The file sorts last so that a
run stopping at the first failure has run everything else.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_static_update_matches_regular_path_twice():
    import torch
    from oracle.chain import HybridChain
    from paper_1910_09142_gb300 import binding as b

    cfg = dict(Lx=3, two_W=2, J_leg=1.0, J_rung=0.5, beta=0.4, tau=0.1, chi_max=40, cutoff=1e-12)
    p = b.params(**cfg, seed=2)
    ctx = b.Context(256 << 20)
    try:
        st = HybridChain(seed=2, **cfg).evolve()
        k = 3                                           # a pair with nontrivial bond dims
        A, B = np.ascontiguousarray(st.tensors[k]), np.ascontiguousarray(st.tensors[k + 1])
        gate_index = 2                                  # bond 0 at tau/2
        gate = b.gates(p)[gate_index].reshape(-1)
        for absorb in (0, 1):
            cid = ctx.init_chain(p)
            ctx.set_mps(cid, st.tensors)
            ctx.apply_ops(cid, [[k, gate_index, absorb, 0]])
            ref = ctx.get_mps(cid)
            ctx.free_chain(cid)
            RA, RB = ref[k], ref[k + 1]

            dev = torch.device("cuda:0")
            tA = torch.tensor(A, dtype=torch.float64, device=dev)
            tB = torch.tensor(B, dtype=torch.float64, device=dev)
            tG = torch.tensor(gate, dtype=torch.float64, device=dev)
            kmax = min(3 * A.shape[0], 3 * B.shape[2], cfg["chi_max"])
            for _ in range(2):                          # two calls in a row share the scratch
                oA = torch.full((A.shape[0] * 3 * kmax,), np.nan, dtype=torch.float64, device=dev)
                oB = torch.full((kmax * 3 * B.shape[2],), np.nan, dtype=torch.float64, device=dev)
                kk = torch.zeros(1, dtype=torch.int32, device=dev)
                b.two_site_update_static(tA, tB, tG, cfg["chi_max"], cfg["cutoff"], absorb, oA, oB, kk)
                torch.cuda.synchronize()
                kv = int(kk.item())
                assert kv == RA.shape[2] == RB.shape[0]
                gA = oA[: A.shape[0] * 3 * kv].cpu().numpy().reshape(RA.shape)
                gB = oB[: kv * 3 * B.shape[2]].cpu().numpy().reshape(RB.shape)
                got = gA.reshape(-1, kv) @ gB.reshape(kv, -1)
                want = RA.reshape(-1, kv) @ RB.reshape(kv, -1)
                assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()
                iso = gB.reshape(kv, -1) if absorb == 0 else gA.reshape(-1, kv).T
                assert np.abs(iso @ iso.T - np.eye(kv)).max() < 1e-12
    finally:
        ctx.close()


def test_static_update_rejects_oversized_bonds():
    import torch
    from paper_1910_09142_gb300 import binding as b

    dev = torch.device("cuda:0")
    A = torch.zeros((1, 3, 129), dtype=torch.float64, device=dev)
    B = torch.zeros((129, 3, 1), dtype=torch.float64, device=dev)
    g = torch.eye(9, dtype=torch.float64, device=dev).reshape(-1)
    out = torch.zeros(3 * 128, dtype=torch.float64, device=dev)
    k = torch.zeros(1, dtype=torch.int32, device=dev)
    with pytest.raises(b.HmError) as e:
        b.two_site_update_static(A, B, g, 64, 0.0, 0, out, out, k)
    assert e.value.code == b.HM_ERR_ARG and "128" in str(e.value)
