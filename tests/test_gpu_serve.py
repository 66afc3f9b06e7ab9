"""The continuous-batching server on the GPU (real library).

Jobs of different ladder sizes arrive while others run; each job's samples
must equal the samples of the same job served alone: bit-identical on the
binary64 path (every chain runs in its own CTA).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_served_jobs_equal_jobs_served_alone():
    from paper_1910_09142_gb300 import binding as b
    from paper_1910_09142_gb300 import serve

    def p(Lx, two_W, cid, chi):
        return b.params(Lx, two_W, J_rung=0.7, beta=0.2, tau=0.1, chi_max=chi, cutoff=1e-10, seed=9,
                        chain_id=cid)

    arrivals = [(0, p(3, 2, 1, 16), 3, 1), (1, p(3, 4, 2, 16), 2, 0), (1, p(2, 0, 3, 16), 4, 1),
                (3, p(3, 2, 4, 16), 1, 0)]
    arena = 1 << 30
    ctx = b.Context(arena)
    try:
        mixed = serve.Server(ctx, arena - (64 << 20))
        st = mixed.run(arrivals)
        assert st["jobs_finished"] == 4 and st["samples"] == 3 + 2 + 4 + 1
        assert st["latency_p99_s"] is not None
        for job in mixed.finished:
            alone = serve.Server(ctx, arena - (64 << 20))
            alone.submit(job.params, job.n_samples, job.n_warmup)
            alone.run()
            (a,) = alone.finished
            assert len(a.results) == len(job.results) == job.n_samples
            for x, y in zip(a.results, job.results):
                assert np.array_equal(x, y)
            for x, y in zip(a.env, job.env):
                assert np.array_equal(x, y)
    finally:
        ctx.close()
