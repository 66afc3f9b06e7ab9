"""The continuous-batching server's scheduling logic, on CPU with a fake context.

The fake stands in for binding.Context (same methods); its observables depend
only on (chain parameters, step index) -- the property the CUDA library has
(one CTA per chain) -- so a job's results must not depend on what else ran.
Memory sizes and observable counts come from the real host-side C ABI.
"""
import numpy as np
import pytest

from paper_1910_09142_gb300 import binding, build, serve


@pytest.fixture(scope="module", autouse=True)
def lib():
    import os
    if not os.path.exists(build.LIB):
        build.build()
    return binding.load()


class FakeCtx:
    def __init__(self):
        self.chains, self.next, self.calls = {}, 1, []

    def init_chain(self, p):
        cid = self.next
        self.next += 1
        self.chains[cid] = [p, 0]
        return cid

    def evolve(self, ids):
        self.calls.append(("evolve", tuple(ids)))

    def measure(self, ids, n_obs):
        self.calls.append(("measure", tuple(ids)))
        out = []
        for c in ids:
            p, step = self.chains[c]
            out.append(np.full(n_obs, 1000.0 * p.Lx + 10.0 * p.chain_id + step))
        return np.array(out)

    def collapse(self, ids, n_env):
        self.calls.append(("collapse", tuple(ids)))
        env = []
        for c in ids:
            self.chains[c][1] += 1
            env.append(np.zeros(n_env, dtype=np.int8))
        return np.array(env).reshape(len(ids), n_env), np.zeros(len(ids))

    def free_chain(self, cid):
        del self.chains[cid]


def _p(Lx, cid, chi=16):
    return binding.params(Lx, 2, beta=0.4, tau=0.1, chi_max=chi, chain_id=cid)


def test_job_results_do_not_depend_on_the_mix():
    mixed = serve.Server(FakeCtx(), 1 << 40)
    st = mixed.run([(0, _p(3, 1), 4, 1), (1, _p(5, 2), 2, 0), (2, _p(4, 3), 3, 2)])
    assert st["jobs_finished"] == 3 and st["samples"] == 9
    for job in mixed.finished:
        alone = serve.Server(FakeCtx(), 1 << 40)
        alone.submit(job.params, job.n_samples, job.n_warmup)
        alone.run()
        (a,) = alone.finished
        assert len(a.results) == job.n_samples
        assert all(np.array_equal(x, y) for x, y in zip(a.results, job.results))
        # warm-up steps are run but not reported
        assert a.results[0][0] == 1000.0 * job.params.Lx + 10.0 * job.params.chain_id + job.n_warmup


def test_one_batched_call_per_stage_and_tick():
    ctx = FakeCtx()
    srv = serve.Server(ctx, 1 << 40)
    srv.submit(_p(3, 1), 2)
    srv.submit(_p(3, 2), 2)
    srv.step()
    evolves = [c for c in ctx.calls if c[0] == "evolve"]
    assert evolves == [("evolve", (1, 2))]               # both chains in one launch
    srv.submit(_p(4, 3), 1)                              # arrives mid-run
    srv.step()
    last_evolve = [c for c in ctx.calls if c[0] == "evolve"][-1]
    assert len(last_evolve[1]) == 3                      # joined the running batch
    # chains with different environment sizes are collapsed in separate calls
    assert sum(1 for c in ctx.calls[ctx.calls.index(last_evolve):] if c[0] == "collapse") == 2
    assert srv.step() == 0 and len(srv.finished) == 3


def test_admission_by_memory_and_fifo():
    big = binding.query_memory(_p(6, 0, chi=64))
    small = binding.query_memory(_p(3, 0))
    srv = serve.Server(FakeCtx(), big + small)
    j1 = srv.submit(_p(6, 1, chi=64), 3)
    j2 = srv.submit(_p(6, 2, chi=64), 1)                 # does not fit next to j1
    j3 = srv.submit(_p(3, 3), 1)                         # fits, but waits behind j2 (FIFO)
    srv.step()
    assert srv.active == [j1] and list(srv.queue) == [j2, j3]
    while srv.step():
        assert srv.used <= srv.capacity
    assert [j.id for j in srv.finished] == [j1.id, j2.id, j3.id] or len(srv.finished) == 3
    assert srv.used == 0


def test_oversized_job_rejected_and_batch_slots_respected():
    srv = serve.Server(FakeCtx(), 1000)
    with pytest.raises(ValueError):
        srv.submit(_p(3, 1), 1)
    srv = serve.Server(FakeCtx(), 1 << 40, max_chains=2)
    for i in range(5):
        srv.submit(_p(3, i), 1)
    srv.step()
    assert len(srv.finished) == 2 and len(srv.queue) == 3


def test_latency_statistics():
    t = [0.0]

    def clock():
        t[0] += 0.5
        return t[0]
    srv = serve.Server(FakeCtx(), 1 << 40, clock=clock)
    st = srv.run([(0, _p(3, 1), 3, 0)])
    assert st["samples"] == 3 and st["latency_p50_s"] == pytest.approx(0.5)
    assert st["samples_per_s"] == pytest.approx(2.0)


def test_job_estimate_over_kept_samples():
    srv = serve.Server(FakeCtx(), 1 << 40)
    job = srv.submit(_p(3, 4), 25, 3)
    job.bin_size = 5
    assert job.estimate() == (None, None)
    srv.run()
    mean, err = job.estimate()
    x = np.array(job.results)
    assert np.allclose(mean, x.mean(axis=0), atol=1e-12)
    bins = x.reshape(5, 5, -1).mean(axis=1)
    assert np.allclose(err, bins.std(axis=0, ddof=1) / np.sqrt(5), atol=1e-12)
