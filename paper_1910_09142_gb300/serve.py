"""Continuous-batching sampling server over the C ABI.

A job asks for ``n_samples`` kept samples of the hybrid-METTS chain
(Sec. I.C.1) with its own parameters (ladder length, cluster size, beta,
chi_max, ...), drawn by one or several independent chains (walkers, each
with its own random stream and warm-up), so that a few large requests still
fill the GPU's SMs (one CTA per chain).  The server keeps every admitted
chain's MPS resident on the device and, on every tick, advances *all*
resident chains by one Markov step
in one batched call per stage (``hm_evolve``, ``hm_measure_cluster``,
``hm_collapse``), whatever their sizes.  Jobs that arrive while others run
wait in a FIFO queue and are admitted at the next tick boundary as soon as
the arena bytes ``hm_query_memory`` reports for them are free and a batch
slot is open; a finished job's chain is freed at once.  Each chain's result
depends only on its own data (one CTA per chain), so a job's samples are the
same alone and in the mix: bit-identical in binary64, and within the stated
tolerance in the mixed-precision mode, whose column-block size follows the
largest bond cap in the batch.

With ``tick_ops`` set, a tick advances every resident chain's evolution by
at most that many two-site ops (``hm_evolve_partial``) and measures and
collapses only the chains whose evolution completed in it, so a long chain
(large Lx, beta or chi) takes several ticks and no longer holds every other
job's latency; the slices give the same samples as whole evolutions.

All arithmetic of a step runs in ``libhmetts.so``; this module only
schedules.  Latency of a sample = wall time from the tick its evolution
started to the end of the tick that produced it (one tick without
``tick_ops``); a job's queueing delay is reported separately.
"""
import collections
import time

import numpy as np

from . import binding
from .estimators import Estimator


# A job's k-th chain draws from Philox stream chain_id + k * FANOUT_STRIDE, so
# jobs whose chain ids stay below FANOUT_STRIDE never share a stream.
FANOUT_STRIDE = 1 << 24


class Walker:
    """One Markov chain of a job: its own random stream, warm-up and share of
    the job's samples."""

    def __init__(self, job, k, n_keep):
        self.job = job
        self.k = k
        self.params = binding.Params(*[getattr(job.params, f) for f, _ in binding.Params._fields_])
        self.params.chain_id = (int(job.params.chain_id) + k * FANOUT_STRIDE) & 0xFFFFFFFF
        self.n_steps = job.n_warmup + int(n_keep)
        self.chain = None
        self.done_steps = 0
        self.results = []                    # observable vectors of kept samples
        self.env = []                        # collapse outcomes of every step
        self.latencies = []                  # seconds per kept sample
        self.sample_t0 = None                # start of the sample now being evolved
        self.resume_from = None              # (outcomes, sample index) of a checkpoint
        self.bytes = 0

    @property
    def complete(self):
        return self.done_steps >= self.n_steps

    def checkpoint(self):
        if self.env:
            env = [int(x) for x in self.env[-1]]
        elif self.resume_from is not None:            # resumed, no step since
            env = [int(x) for x in self.resume_from[0]]
        else:
            env = None
        return dict(env=env, next_sample=self.done_steps, results=[[float(x) for x in r] for r in self.results])


class Job:
    """One sampling request: ``n_samples`` kept samples of the chain of
    Sec. I.C.1, drawn by ``n_chains`` independent chains (walkers), each
    with ``n_warmup`` discarded warm-up samples and an equal share of the
    kept ones (the first n_samples % n_chains walkers keep one more)."""

    def __init__(self, job_id, params, n_samples, n_warmup=0, arrival=None, bin_size=10, n_chains=1):
        self.id = job_id
        self.params = params                 # binding.Params
        self.n_samples = int(n_samples)
        self.n_warmup = int(n_warmup)
        self.n_chains = max(1, min(int(n_chains), max(1, self.n_samples)))
        if int(params.chain_id) >= FANOUT_STRIDE and self.n_chains > 1:
            raise ValueError("a job with several chains needs chain_id < %d" % FANOUT_STRIDE)
        self.arrival = arrival
        self.admitted = None
        self.finished = None
        self.bytes = 0
        self.bin_size = int(bin_size)
        self.estimator = None                # Estimator over the kept samples of every walker
        q, r = divmod(self.n_samples, self.n_chains)
        self.walkers = [Walker(self, k, q + (1 if k < r else 0)) for k in range(self.n_chains)]

    @property
    def results(self):
        """Kept observable vectors, walker by walker."""
        return [x for w in self.walkers for x in w.results]

    @property
    def env(self):
        """Collapse outcomes of every step, walker by walker."""
        return [x for w in self.walkers for x in w.env]

    @property
    def latencies(self):
        return [x for w in self.walkers for x in w.latencies]

    def estimate(self):
        """Mean of every observable over the kept samples, and its binned
        standard error (None until two bins are complete)."""
        if self.estimator is None or self.estimator.count == 0:
            return None, None
        err = self.estimator.stderr() if self.estimator.sums[5][0] >= 2 else None
        return self.estimator.mean(), err

    @property
    def complete(self):
        return all(w.complete for w in self.walkers)

    def checkpoint(self):
        """Everything needed to continue this job elsewhere, as plain data:
        its parameters and, per walker, the outcomes of its last collapse,
        its sample index and the samples kept so far.  Step 4 resets the
        cluster to Bell pairs, so no MPS is saved."""
        return dict(id=self.id, params={f: getattr(self.params, f) for f, _ in binding.Params._fields_},
                    n_samples=self.n_samples, n_warmup=self.n_warmup, n_chains=self.n_chains,
                    bin_size=self.bin_size, chains=[w.checkpoint() for w in self.walkers])


class Server:
    """FIFO admission by arena bytes and batch slots; one batched step per tick."""

    def __init__(self, ctx, arena_bytes, max_chains=448, clock=time.perf_counter,
                 query_memory=None, num_obs=None, num_env=None, sleep=time.sleep, tick_ops=None,
                 chains_per_job=1):
        self.ctx = ctx
        self.tick_ops = int(tick_ops) if tick_ops else None
        self.capacity = int(arena_bytes)
        self.max_chains = int(max_chains)
        self.chains_per_job = max(1, int(chains_per_job))
        self.clock = clock
        self.sleep = sleep
        self.query_memory = query_memory or binding.query_memory
        self.num_obs = num_obs or binding.num_obs
        self.num_env = num_env or binding.num_env
        self.queue = collections.deque()
        self.active = []                     # admitted, unfinished jobs
        self.resident = []                   # their walkers still drawing
        self.finished = []
        self.used = 0
        self.ticks = 0
        self.samples = 0
        self.busy_s = 0.0
        self._next_id = 0

    # -- requests ---------------------------------------------------------------------
    def submit(self, params, n_samples, n_warmup=0, arrival=None, job_id=None, n_chains=None):
        """Queue a job; returns it.  ``params`` is a binding.Params; ``arrival``
        (clock time the request came in) defaults to now; ``job_id`` keeps a
        restored job's identity (default: the next free id); ``n_chains``
        walkers share its samples (default: the server's chains_per_job)."""
        jid = self._next_id if job_id is None else int(job_id)
        job = Job(jid, params, n_samples, n_warmup, self.clock() if arrival is None else arrival,
                  n_chains=self.chains_per_job if n_chains is None else n_chains)
        for w in job.walkers:
            w.bytes = self.query_memory(w.params)
        job.bytes = sum(w.bytes for w in job.walkers)
        if job.bytes > self.capacity or job.n_chains > self.max_chains:
            raise ValueError("job %d needs %d bytes and %d chains, more than the whole arena"
                             % (job.id, job.bytes, job.n_chains))
        self._next_id = max(self._next_id, jid + 1)
        self.queue.append(job)
        return job

    def resume(self, ckpt):
        """Queue a job from ``Job.checkpoint()`` data; every walker continues
        with the draws the interrupted one would have made (hm_resume_chain)."""
        job = self.submit(binding.Params(**ckpt["params"]), ckpt["n_samples"], ckpt["n_warmup"],
                          job_id=ckpt.get("id"), n_chains=ckpt["n_chains"])
        job.bin_size = int(ckpt["bin_size"])
        for w, wc in zip(job.walkers, ckpt["chains"]):
            w.done_steps = int(wc["next_sample"])
            for r in wc["results"]:
                w.results.append(np.array(r))
                if job.estimator is None:
                    job.estimator = Estimator(len(r), job.bin_size)
                job.estimator.add((job.id, w.k), r)
            if w.done_steps > 0:
                w.resume_from = (np.array(wc["env"], dtype=np.int8), w.done_steps)
        return job

    def _admit(self):
        while self.queue:
            job = self.queue[0]
            live = [w for w in job.walkers if not w.complete]
            need = sum(w.bytes for w in live)
            if self.used + need > self.capacity or len(self.resident) + len(live) > self.max_chains:
                break                                  # FIFO: later jobs wait behind it
            self.queue.popleft()
            for w in live:
                if w.resume_from is not None:
                    env, n = w.resume_from
                    w.chain = self.ctx.init_chain(w.params, env_init=env, next_sample=n)
                else:
                    w.chain = self.ctx.init_chain(w.params)
                self.used += w.bytes
                self.resident.append(w)
            job.admitted = self.clock()
            if live:
                self.active.append(job)
            else:                                      # nothing left to draw
                job.finished = job.admitted
                self.finished.append(job)

    def checkpoint(self):
        """Checkpoint of every job, finished, resident or queued, as plain
        data (see ``Job.checkpoint``).  Taken between ticks, no kernel of
        this server is in flight; a restarted server continues from it."""
        jobs = self.finished + self.active + list(self.queue)
        return {"jobs": [j.checkpoint() for j in sorted(jobs, key=lambda j: j.id)]}

    @classmethod
    def restore(cls, ckpt, ctx, arena_bytes, **kw):
        """A new server holding the jobs of ``checkpoint()``: finished ones
        keep their results, the others are queued to resume."""
        srv = cls(ctx, arena_bytes, **kw)
        for jc in ckpt["jobs"]:
            job = srv.resume(jc)
            if job.complete:
                srv.queue.remove(job)
                srv.finished.append(job)
        return srv

    # -- one tick -----------------------------------------------------------------------
    def step(self):
        """Admit what fits, then one Markov step of every resident chain.

        Returns the number of chains stepped (0 when idle).
        """
        self._admit()
        if not self.resident:
            return 0
        t0 = self.clock()
        ids = [w.chain for w in self.resident]
        for w in self.resident:
            if w.sample_t0 is None:
                w.sample_t0 = t0
        if self.tick_ops:
            done = self.ctx.evolve_partial(ids, self.tick_ops)
            ready = [w for w, d in zip(self.resident, done) if d]
            # the slices are asynchronous: wait for them, so that a tick lasts
            # its device time and the next tick's admission sees the clock
            sync = getattr(self.ctx, "synchronize", None)
            if sync is not None:
                sync()
        else:
            self.ctx.evolve(ids)
            ready = list(self.resident)
        obs = {}
        for n_obs, group in self._groups(self.num_obs, ready).items():
            vals = self.ctx.measure([w.chain for w in group], n_obs)
            for w, v in zip(group, vals):
                obs[id(w)] = v
        for n_env, group in self._groups(self.num_env, ready).items():
            env, _ = self.ctx.collapse([w.chain for w in group], n_env)
            for w, e in zip(group, env):
                w.env.append(np.array(e))
        t1 = self.clock()
        self.busy_s += t1 - t0
        self.ticks += 1
        still = []
        for w in self.resident:
            if id(w) not in obs:
                still.append(w)                        # evolution continues next tick
                continue
            job = w.job
            if w.done_steps >= job.n_warmup:
                v = obs[id(w)]
                w.results.append(v)
                if job.estimator is None:
                    job.estimator = Estimator(len(v), job.bin_size)
                job.estimator.add((job.id, w.k), v)
                w.latencies.append(t1 - w.sample_t0)
                self.samples += 1
            w.sample_t0 = None
            w.done_steps += 1
            if w.complete:
                self.ctx.free_chain(w.chain)
                self.used -= w.bytes
            else:
                still.append(w)
        self.resident = still
        for job in [j for j in self.active if j.complete]:
            job.finished = t1
            self.active.remove(job)
            self.finished.append(job)
        return len(ids)

    def _groups(self, count, walkers=None):
        groups = collections.OrderedDict()
        for w in self.resident if walkers is None else walkers:
            groups.setdefault(count(w.params), []).append(w)
        return groups

    def run(self, arrivals=()):
        """Serve until idle.  ``arrivals``: iterable of (tick, params, n_samples,
        n_warmup); a job listed for tick t is submitted before the t-th tick of
        this call runs (immediately when the server would otherwise idle)."""
        pending = collections.deque(sorted(arrivals, key=lambda a: a[0]))
        tick = 0
        while True:
            while pending and (pending[0][0] <= tick or (not self.active and not self.queue)):
                _, p, n, w = pending.popleft()[:4]
                self.submit(p, n, w)
            if self.step() == 0 and not self.queue and not pending:
                return self.stats()
            tick += 1

    def run_stream(self, requests, horizon_s=None):
        """Serve a timed request stream.

        ``requests``: iterable of (t_s, params, n_samples, n_warmup), t_s in
        seconds after this call starts.  Each tick first submits every request
        whose time has come (stamped with its arrival time, so the queueing
        delay includes the wait for the tick boundary), then runs one step.
        When nothing is resident or queued, the loop sleeps until the next
        arrival.  It returns when everything has been served, or at the first
        tick boundary after ``horizon_s``, leaving the rest queued or resident."""
        pending = collections.deque(sorted(requests, key=lambda r: r[0]))
        t0 = self.clock()
        while True:
            now = self.clock() - t0
            if horizon_s is not None and now >= horizon_s:
                return self.stats()
            while pending and pending[0][0] <= now:
                t, p, n, w = pending.popleft()
                self.submit(p, n, w, arrival=t0 + t)
            if not self.active and not self.queue:
                if not pending:
                    return self.stats()
                self.sleep(pending[0][0] - now)
                continue
            self.step()

    # -- statistics ---------------------------------------------------------------------
    def stats(self):
        jobs = self.finished + self.active
        lat = [x for j in jobs for x in j.latencies]
        waits = [j.admitted - j.arrival for j in jobs if j.admitted is not None]
        return {"samples": self.samples, "ticks": self.ticks, "busy_s": self.busy_s,
                "samples_per_s": self.samples / self.busy_s if self.busy_s > 0 else None,
                "latency_p50_s": float(np.percentile(lat, 50)) if lat else None,
                "latency_p99_s": float(np.percentile(lat, 99)) if lat else None,
                "queue_wait_p50_s": float(np.percentile(waits, 50)) if waits else None,
                "queue_wait_p99_s": float(np.percentile(waits, 99)) if waits else None,
                "jobs_finished": len(self.finished), "jobs_resident": len(self.active),
                "chains_resident": len(self.resident),
                "jobs_queued": len(self.queue)}
