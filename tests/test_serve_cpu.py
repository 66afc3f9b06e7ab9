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

    def init_chain(self, p, env_init=None, next_sample=0):
        cid = self.next
        self.next += 1
        self.chains[cid] = [p, next_sample]
        return cid

    def evolve(self, ids):
        self.calls.append(("evolve", tuple(ids)))

    def evolve_partial(self, ids, max_ops):
        """Each chain needs Lx * 10 ops per sample (a stand-in schedule length)."""
        self.calls.append(("evolve_partial", tuple(ids)))
        done = []
        for c in ids:
            p = self.chains[c][0]
            cur = self.chains[c][2] if len(self.chains[c]) > 2 else 0
            cur = min(cur + max_ops, 10 * p.Lx)
            fin = cur >= 10 * p.Lx
            self.chains[c][2:] = [0 if fin else cur]
            done.append(fin)
        return np.array(done)

    def measure(self, ids, n_obs):
        self.calls.append(("measure", tuple(ids)))
        out = []
        for c in ids:
            p, step = self.chains[c][:2]
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


class _Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 0.0)


class _TimedCtx(FakeCtx):
    """Each batched evolve takes one second of the fake clock."""

    def __init__(self, clock):
        super().__init__()
        self.clock = clock

    def evolve(self, ids):
        super().evolve(ids)
        self.clock.t += 1.0


def test_stream_admits_at_tick_boundaries_and_sleeps_when_idle():
    clk = _Clock()
    srv = serve.Server(_TimedCtx(clk), 1 << 40, clock=clk, sleep=clk.sleep)
    reqs = [(2.0, _p(3, 1), 3, 0), (2.3, _p(4, 2), 1, 0), (9.5, _p(3, 3), 1, 1)]
    st = srv.run_stream(reqs)
    assert st["jobs_finished"] == 3 and st["samples"] == 5
    a, b, c = sorted(srv.finished, key=lambda j: j.id)
    assert a.admitted == pytest.approx(2.0)            # slept until the first arrival
    assert b.admitted == pytest.approx(3.0)            # arrived mid-tick, joined at the next one
    assert b.admitted - b.arrival == pytest.approx(0.7)
    assert c.admitted == pytest.approx(9.5) and c.finished == pytest.approx(11.5)
    assert st["queue_wait_p99_s"] == pytest.approx(0.7, abs=0.02)


def test_stream_horizon_leaves_the_rest_resident_or_queued():
    clk = _Clock()
    srv = serve.Server(_TimedCtx(clk), 1 << 40, clock=clk, sleep=clk.sleep, max_chains=2)
    reqs = [(0.0, _p(3, i), 10, 0) for i in range(5)]
    st = srv.run_stream(reqs, horizon_s=3.5)
    assert st["ticks"] == 4 and st["jobs_finished"] == 0
    assert st["jobs_resident"] == 2 and st["jobs_queued"] == 3


def test_poisson_request_stream():
    import synth
    r1 = synth.poisson_requests(50.0, 20.0, seed=3)
    r2 = synth.poisson_requests(50.0, 20.0, seed=3)
    assert [x[0] for x in r1] == [x[0] for x in r2]
    assert abs(len(r1) - 1000) < 4 * np.sqrt(1000)                       # Poisson count
    t = np.array([x[0] for x in r1])
    assert np.all(np.diff(t) > 0) and t[-1] < 20.0
    for _, cfg, n in r1:
        assert cfg["Lx"] in (8, 16, 32) and cfg["two_W"] in (4, 8) and cfg["chi_max"] in (128, 256, 512)
        assert 0.5 <= cfg["beta"] <= 16.0 and 100 <= n <= 2000
        binding.params(**cfg)                                              # a valid chain
    betas = np.array([c["beta"] for _, c, _ in r1])
    assert abs(np.median(np.log(betas)) - 0.5 * (np.log(0.5) + np.log(16.0))) < 0.3   # log-uniform


def test_poisson_stream_served_end_to_end():
    import synth
    mix = dict(synth.SERVE_MIX, Lx=(3, 4), two_W=(2, 4), chi_max=(16, 32), samples=(2, 6))
    reqs = [(t, binding.params(**cfg, chain_id=i), n, 1)
            for i, (t, cfg, n) in enumerate(synth.poisson_requests(2.0, 10.0, seed=1, mix=mix))]
    clk = _Clock()
    srv = serve.Server(_TimedCtx(clk), 1 << 40, clock=clk, sleep=clk.sleep)
    st = srv.run_stream(reqs)
    assert st["jobs_finished"] == len(reqs) and st["samples"] == sum(r[2] for r in reqs)
    assert st["latency_p50_s"] == pytest.approx(1.0)
    for job in srv.finished:
        assert len(job.results) == job.n_samples and job.admitted >= job.arrival


def test_checkpoint_and_resume_continue_the_job_exactly():
    import json
    whole = serve.Server(FakeCtx(), 1 << 40)
    ref = whole.submit(_p(4, 5), 7, 2)
    whole.run()
    first = serve.Server(FakeCtx(), 1 << 40)
    job = first.submit(_p(4, 5), 7, 2)
    job.bin_size = 3
    for _ in range(4):
        first.step()
    ckpt = json.loads(json.dumps(job.checkpoint()))        # plain data, survives a round trip
    c0 = ckpt["chains"][0]
    assert c0["next_sample"] == 4 and len(c0["results"]) == 2 and len(c0["env"]) == ckpt_env_len(job)
    second = serve.Server(FakeCtx(), 1 << 40)
    again = second.resume(ckpt)
    second.run()
    assert again.complete and len(again.results) == 7
    assert all(np.array_equal(x, y) for x, y in zip(again.results, ref.results))
    assert np.allclose(again.estimate()[0], np.array(ref.results).mean(axis=0), atol=1e-12)


def ckpt_env_len(job):
    return binding.num_env(job.params)


def _crashing_worker(path, crash_after, out):
    """A serving worker that checkpoints after every tick and dies (exit 3,
    no cleanup) after ``crash_after`` ticks, or resumes from ``path``."""
    import json
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_1910_09142_gb300 import serve as srv_mod
    if os.path.exists(path):
        with open(path) as f:
            srv = srv_mod.Server.restore(json.load(f), FakeCtx(), 1 << 40)
    else:
        srv = srv_mod.Server(FakeCtx(), 1 << 40)
        for i, (lx, n, w) in enumerate([(3, 5, 1), (4, 3, 0), (5, 6, 2)]):
            srv.submit(_p(lx, i), n, w)
    ticks = 0
    while srv.step():
        ticks += 1
        with open(path + ".tmp", "w") as f:
            json.dump(srv.checkpoint(), f)
        os.replace(path + ".tmp", path)
        if crash_after and ticks == crash_after:
            os._exit(3)
    out["results"] = {j.id: [list(r) for r in j.results] for j in srv.finished}


def test_serving_worker_crash_restarts_from_checkpoint(tmp_path):
    """A failure made on the host, with no GPU involved: the worker process
    exits mid-run, and a new one restores the last checkpoint and finishes
    with the results of an uninterrupted run."""
    import multiprocessing as mpl
    ctx = mpl.get_context("spawn")
    path = str(tmp_path / "serve.json")
    out = ctx.Manager().dict()
    p = ctx.Process(target=_crashing_worker, args=(path, 3, out))
    p.start()
    p.join(60)
    assert p.exitcode == 3 and "results" not in out
    p = ctx.Process(target=_crashing_worker, args=(path, 0, out))
    p.start()
    p.join(60)
    assert p.exitcode == 0
    whole = serve.Server(FakeCtx(), 1 << 40)
    jobs = [whole.submit(_p(lx, i), n, w) for i, (lx, n, w) in enumerate([(3, 5, 1), (4, 3, 0), (5, 6, 2)])]
    whole.run()
    got = out["results"]
    for j in jobs:
        assert np.array_equal(np.array(got[j.id]), np.array(j.results)), j.id


def test_checkpoint_of_a_resumed_job_before_its_next_step():
    srv = serve.Server(FakeCtx(), 1 << 40)
    job = srv.submit(_p(3, 7), 5, 0)
    srv.step()
    srv.step()
    ckpt = job.checkpoint()
    other = serve.Server(FakeCtx(), 1 << 40)
    other._next_id = 10
    again = other.resume(ckpt)
    assert again.id == job.id and other._next_id == 10
    ckpt2 = again.checkpoint()                          # no step since the resume
    assert ckpt2["chains"][0]["env"] == ckpt["chains"][0]["env"] and ckpt2["chains"][0]["next_sample"] == 2
    third = serve.Server(FakeCtx(), 1 << 40)
    last = third.resume(ckpt2)
    third.run()
    srv.run()
    assert all(np.array_equal(x, y) for x, y in zip(last.results, job.results)) and len(last.results) == 5


def test_tick_op_budget_keeps_short_jobs_moving():
    """With tick_ops, a long chain (Lx=16: 160 stand-in ops) takes several
    ticks per sample while a short one (Lx=2: 20 ops) finishes a sample every
    tick; each job's results equal those of whole-evolution serving."""
    whole = serve.Server(FakeCtx(), 1 << 40)
    sliced = serve.Server(FakeCtx(), 1 << 40, tick_ops=40)
    for srv in (whole, sliced):
        srv.submit(_p(16, 1), 3)
        srv.submit(_p(2, 2), 3)
        srv.run()
    for a, b in zip(sorted(whole.finished, key=lambda j: j.id), sorted(sliced.finished, key=lambda j: j.id)):
        assert [list(r) for r in a.results] == [list(r) for r in b.results]
    long_job, short_job = sorted(sliced.finished, key=lambda j: j.id)
    assert short_job.finished is not None and long_job.finished is not None
    assert sliced.ticks == 12                  # 3 samples x 4 ticks of 40 ops for the long chain
    assert len(short_job.results) == 3


def test_fanned_out_job_splits_its_samples_over_independent_chains():
    """A job of 7 samples on 3 walkers: 3 + 2 + 2 kept samples after 1 warm-up
    each, every walker on its own stream (chain_id + k * 2^24), memory and
    batch slots for all three, and the same results alone and in a mix."""
    alone = serve.Server(FakeCtx(), 1 << 40)
    job = alone.submit(_p(4, 9), 7, 1, n_chains=3)
    assert [w.n_steps for w in job.walkers] == [4, 3, 3]
    assert [w.params.chain_id for w in job.walkers] == [9 + k * serve.FANOUT_STRIDE for k in range(3)]
    assert job.bytes == 3 * binding.query_memory(_p(4, 9))
    alone.run()
    assert job.complete and len(job.results) == 7 and job.estimator.count == 7
    # the fake's observable: 1000 Lx + 10 chain_id + step; warm-up step 0 dropped
    assert [r[0] for r in job.results] == [1000.0 * 4 + 10.0 * (9 + k * serve.FANOUT_STRIDE) + s
                                           for k, n in enumerate((3, 2, 2)) for s in range(1, n + 1)]
    mixed = serve.Server(FakeCtx(), 1 << 40, max_chains=4, chains_per_job=2)
    other = mixed.submit(_p(3, 1), 5)                       # 2 walkers by the server's default
    again = mixed.submit(_p(4, 9), 7, 1, n_chains=3)        # waits for slots: 2 + 3 > 4
    mixed.step()
    assert len(mixed.resident) == 2 and len(mixed.queue) == 1
    mixed.run()
    assert other.n_chains == 2 and len(other.results) == 5
    assert all(np.array_equal(x, y) for x, y in zip(again.results, job.results)) and len(again.results) == 7


def test_fanned_out_job_resumes_every_walker():
    import json
    whole = serve.Server(FakeCtx(), 1 << 40)
    ref = whole.submit(_p(5, 3), 5, 1, n_chains=2)          # walkers of 4 and 3 steps
    whole.run()
    first = serve.Server(FakeCtx(), 1 << 40)
    job = first.submit(_p(5, 3), 5, 1, n_chains=2)
    for _ in range(3):
        first.step()
    ckpt = json.loads(json.dumps(first.checkpoint()))
    assert [c["next_sample"] for c in ckpt["jobs"][0]["chains"]] == [3, 3]
    second = serve.Server.restore(ckpt, FakeCtx(), 1 << 40)
    second.step()                                           # walker 1 is done after this step
    assert not second.active and not second.resident and second.finished[0].complete
    again = second.finished[0]
    assert [list(r) for r in again.results] == [list(r) for r in ref.results]
    assert np.allclose(again.estimate()[0], np.array(ref.results).mean(axis=0), atol=1e-12)
