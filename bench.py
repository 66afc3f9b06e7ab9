"""Benchmark: hybrid-METTS samples/s on GB300 (Lx=16 ladder, chi=256).

One step = one Markov step (evolve by beta/2, measure the cluster, collapse
the environment and reset) of every chain of the batch.  Workload: S=1
Heisenberg ladder Lx=16 (32 spins), J_leg = J_rung = 1, 2W = 8 cluster
sites, beta = 1, tau = 0.05 (M = 10), chi_max = 256, truncation cutoff 1e-7,
256 independent chains per GPU in one batched launch; synthetic (the model
is Hamiltonian-defined), seeds (0, chain id).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
    python bench.py --impl reference ...   # the FP64 CPU oracle on host cores

Prints one JSON line on rank 0.  For N > 1 run under torchrun: each rank
owns its own chains (weak scaling, no data exchange); only the timing
barrier and the max-over-ranks reduction cross ranks.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

FP32_ALU_PEAK = 152 * 128 * 2 * 2.070e9      # 152 SMs x 128 FP32 lanes x FMA x max SM clock
FP64_ALU_PEAK = 1.25e12                      # nominal GB300 binary64 rate
METRIC = "hybrid-METTS samples/s (Lx=16 ladder, chi=256)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)    # one step is 256 samples
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "mixed32", "fp64"])
    ap.add_argument("--chains", type=int, default=256)
    ap.add_argument("--schedule", default="plain", choices=["plain", "fused"],
                    help="op schedule: plain, or fused (runs of splits on one site pair folded into one)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    # workload overrides (smaller cases for profiling; not the headline line)
    ap.add_argument("--Lx", type=int, default=None)
    ap.add_argument("--two-W", type=int, default=None)
    ap.add_argument("--beta", type=float, default=None)
    ap.add_argument("--chi-max", type=int, default=None)
    ap.add_argument("--mode", default="step", choices=["step", "serve"],
                    help="step: the headline batched Markov steps; serve: a timed Poisson request stream "
                         "through the continuous-batching server (its own JSON line)")
    ap.add_argument("--serve-rate", type=float, default=2.0, help="requests per second (serve mode)")
    ap.add_argument("--serve-duration", type=float, default=30.0, help="arrival window, s (serve mode)")
    ap.add_argument("--serve-horizon", type=float, default=120.0, help="stop serving after, s (serve mode)")
    ap.add_argument("--serve-samples", type=float, default=0.01,
                    help="scale of each request's 100-2000 samples (serve mode)")
    ap.add_argument("--tick-ops", type=int, default=512, help="two-site ops per chain per tick (serve mode)")
    ap.add_argument("--serve-chains", type=int, default=4,
                    help="independent chains a request's samples are spread over (serve mode)")
    ap.add_argument("--susceptibility", action="store_true",
                    help="after the run, time hm_measure_susceptibility on freshly evolved chains")
    return ap.parse_args()


def workload(args):
    """The benchmark ladder, with any command-line overrides applied."""
    cfg = synth.ladder("ladder16")
    for key, val in (("Lx", args.Lx), ("two_W", args.two_W), ("beta", args.beta), ("chi_max", args.chi_max)):
        if val is not None:
            cfg[key] = val
    cfg["schedule"] = getattr(args, "schedule", "plain")
    return cfg


def workload_config(args, chains, bytes_per_chain=None):
    cfg = workload(args)
    return {"workload": "S=1 Heisenberg ladder Lx=%d x 2, 2W=%d cluster sites, beta=%g, tau=%g, "
                        "chi_max=%d, cutoff=%g, %d chains/GPU" % (cfg["Lx"], cfg["two_W"], cfg["beta"], cfg["tau"],
                                                                   cfg["chi_max"], cfg["cutoff"], chains),
            "Lx": cfg["Lx"], "two_W": cfg["two_W"], "beta": cfg["beta"], "tau": cfg["tau"],
            "chi_max": cfg["chi_max"], "cutoff": cfg["cutoff"], "J_leg": cfg["J_leg"],
            "J_rung": cfg["J_rung"], "chains_per_gpu": chains, "precision": args.precision,
            "schedule": cfg["schedule"],
            "l2": "inputs larger than L2 (%s of chain state resident)" % (
                "%.1f GB" % (chains * bytes_per_chain / 1e9) if bytes_per_chain else "GBs"),
            "parallelism": "independent chains per GPU" if args.gpus > 1 else "1 GPU"}


def rank_chain_ids(rank, chains_per_rank):
    """Chain ids (Philox stream ids) owned by one rank: disjoint across ranks."""
    return [rank * chains_per_rank + i for i in range(chains_per_rank)]


def max_over_ranks(value, dist, device=None):
    """The largest value over all ranks (the job's time); identity at world size 1."""
    import torch
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _oracle_worker(args):
    """One process: `steps` Markov steps of one oracle chain; returns the seconds per step."""
    chain_id, steps, cfg = args
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    from oracle.chain import HybridChain
    ch = HybridChain(seed=0, chain_id=chain_id, **cfg)
    out = []
    for _ in range(steps):
        t0 = time.perf_counter()
        ch.sample()
        out.append(time.perf_counter() - t0)
    return out


def oracle_parallel(steps, procs=None, cfg=None):
    """The FP64 oracle as it stands, one chain per process (1 BLAS thread each)
    on `procs` host cores (default: all).  Processes are started with spawn so
    that no CUDA state is forked.  Returns (samples/s, per-step wall times, procs)."""
    import multiprocessing as mp
    if not procs:
        try:
            procs = len(os.sched_getaffinity(0))      # the cores this process may run on
        except (AttributeError, OSError):
            procs = os.cpu_count() or 1
    cfg = cfg or synth.ladder("ladder16")
    ctx = mp.get_context("spawn")
    # children read the BLAS thread count when they first import numpy, which
    # happens before any worker code runs: set it in the inherited environment
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    os.environ.update({k: "1" for k in keys})
    try:
        t0 = time.perf_counter()
        with ctx.Pool(procs) as pool:
            times = pool.map(_oracle_worker, [(i, steps, cfg) for i in range(procs)])
        wall = time.perf_counter() - t0
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    per_step = [max(t[k] for t in times) for k in range(steps)]
    return procs * steps / sum(per_step), per_step, procs, wall


def oracle_sample_rate(n_samples=1):
    """Bounded CPU baseline: one Markov step of one chain per host core."""
    rate, per_step, procs, _ = oracle_parallel(n_samples)
    return rate, sum(per_step), procs


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.rows, self.proc = index, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
        sm = [float(r[1]) for r in self.rows if len(r) >= 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 8 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 8 for i in range(4) if r[4 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # warm-up and timed steps in one pool (process start-up is not timed):
    # a step is one Markov step of one chain on every host core
    _, per_step, procs, _ = oracle_parallel(args.warmup + args.steps, cfg=workload(args))
    timed = per_step[args.warmup:]
    total_t = sum(timed)
    value = procs * args.steps / total_t
    line = {"metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": dict(workload_config(args, args.chains), precision="fp64 (CPU oracle)"),
            "cpu_baseline": {"value": value, "unit": "samples/s", "cores": procs, "kind": "oracle",
                             "sample": "per timed step one Markov step of one chain on each of %d host cores "
                                       "(numpy/LAPACK FP64, 1 thread per process)" % procs},
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_serve(args):
    """The serving form on one GPU: requests drawn like the fifth workload
    (Lx in {8, 16, 32}, 2W in {4, 8}, beta log-uniform in [0.5, 16], chi in
    {128, 256, 512}, 100-2000 samples scaled by --serve-samples) arrive as a
    Poisson stream; the server admits them by arena bytes, advances every
    resident chain by <= --tick-ops two-site ops per tick (a request's
    samples spread over --serve-chains chains) and reports served
    samples/s and per-sample latency.  One JSON line, not the headline."""
    import torch
    from paper_1910_09142_gb300 import binding as b, build, serve
    if not os.path.exists(build.LIB):
        build.build()
    torch.cuda.set_device(0)
    prec = {"mixed": b.HM_MIXED, "mixed32": b.HM_MIXED32, "fp64": b.HM_FP64}[args.precision]
    reqs = synth.poisson_requests(args.serve_rate, args.serve_duration, seed=0)
    free, _ = torch.cuda.mem_get_info(0)
    arena = int(min(free * 0.8, 180e9))
    stream = torch.cuda.Stream(0)
    ctx = b.Context(arena, device=0, stream=stream)
    srv = serve.Server(ctx, arena, tick_ops=args.tick_ops, chains_per_job=args.serve_chains)
    stream_reqs = []
    for i, (t, cfg, n) in enumerate(reqs):
        n = max(1, int(round(n * args.serve_samples)))
        stream_reqs.append((t, b.params(**cfg, precision=prec, seed=1, chain_id=i, susceptibility=False), n, 0))
    t0 = time.perf_counter()
    st = srv.run_stream(stream_reqs, horizon_s=args.serve_horizon)
    wall = time.perf_counter() - t0
    line = {"metric": "served hybrid-METTS samples/s and per-sample latency (Poisson stream)", "mode": "serve",
            "value": st["samples"] / wall if wall > 0 else None, "unit": "samples/s",
            "latency_p50_s": st["latency_p50_s"], "latency_p99_s": st["latency_p99_s"],
            "queue_wait_p50_s": st["queue_wait_p50_s"], "queue_wait_p99_s": st["queue_wait_p99_s"],
            "samples": st["samples"], "ticks": st["ticks"], "busy_s": st["busy_s"], "wall_s": wall,
            "requests": len(stream_reqs), "jobs_finished": st["jobs_finished"],
            "jobs_resident": st["jobs_resident"], "chains_resident": st["chains_resident"],
            "jobs_queued": st["jobs_queued"],
            "config": {"rate_per_s": args.serve_rate, "arrival_window_s": args.serve_duration,
                       "horizon_s": args.serve_horizon, "samples_scale": args.serve_samples,
                       "tick_ops": args.tick_ops, "chains_per_request": args.serve_chains,
                       "precision": args.precision, "arena_gb": arena / 1e9,
                       "mix": {k: v for k, v in synth.SERVE_MIX.items()}},
            "data": "synthetic"}
    print(json.dumps(line), flush=True)
    ctx.close()


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "serve":
        return run_serve(args)
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1910_09142_gb300 import binding, build
    if not os.path.exists(build.LIB):
        build.build()
    b = binding
    cfg = workload(args)
    prec = {"mixed": b.HM_MIXED, "mixed32": b.HM_MIXED32, "fp64": b.HM_FP64}[args.precision]
    n = args.chains
    ps = [b.params(**cfg, precision=prec, seed=0, chain_id=c) for c in rank_chain_ids(rank, n)]
    per = b.query_memory(ps[0])
    stream = torch.cuda.Stream(local)
    ctx = b.Context(per * n + (512 << 20), device=local, stream=stream)
    ids = [ctx.init_chain(p) for p in ps]
    n_obs, n_env = b.num_obs(ps[0]), b.num_env(ps[0])
    obs = torch.empty((n, n_obs), dtype=torch.float64, device="cuda:%d" % local)
    env = torch.empty((n, n_env), dtype=torch.int8, device="cuda:%d" % local)
    logp = torch.empty((n,), dtype=torch.float64, device="cuda:%d" % local)
    max_ops = len(b.plan(ps[0]))
    batches = (n + 447) // 448
    launches_per_step = batches * ((max_ops + 4095) // 4096 + 3)

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps + 2)]

    def step(i=None):
        if i is not None:
            ev[2 + 2 * i].record(stream)
        ctx.evolve(ids)
        if i is not None:
            ev[3 + 2 * i].record(stream)
        ctx.measure_device(ids, obs)
        ctx.collapse_device(ids, env, logp)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    stats0 = np.array([ctx.stats(c) for c in ids])

    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    step_ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    step_ev[0].record(stream)
    for i in range(args.steps):
        step(i)
        step_ev[i + 1].record(stream)
    ev[1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    t_ms = ev[0].elapsed_time(ev[1])
    evolve_ms = [ev[2 + 2 * i].elapsed_time(ev[3 + 2 * i]) for i in range(args.steps)]
    lat = [step_ev[i].elapsed_time(step_ev[i + 1]) for i in range(args.steps)]
    stats1 = np.array([ctx.stats(c) for c in ids])
    d = stats1 - stats0
    flops_alg = float(d[:, 0].sum() + d[:, 1].sum() + d[:, 2].sum())
    t_ms = max_over_ranks(t_ms, dist, "cuda:%d" % local)
    value = world * n * args.steps / (t_ms / 1e3)

    e2e = None
    if not args.no_e2e:
        torch.cuda.synchronize()
        e2e_steps = 1
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            ctx.evolve(ids)
            ctx.measure(ids, n_obs)            # host output (D2H inside)
            ctx.collapse(ids, n_env)           # host outputs (D2H inside)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        e2e_s = max_over_ranks(e2e_s, dist, "cuda:%d" % local)
        e2e = {"value": world * n * e2e_steps / e2e_s, "unit": "samples/s", "steps": e2e_steps,
               "h2d_bytes_per_step": 8 * n,                      # chain handles
               "d2h_bytes_per_step": n * (8 * n_obs + n_env + 8)}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    evolve_s = sum(evolve_ms) / 1e3
    achieved = flops_alg / evolve_s / 1e12
    peak = FP32_ALU_PEAK / 1e12 if prec != b.HM_FP64 else FP64_ALU_PEAK / 1e12
    line = {"metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == b.HM_FP64 else "f32+f64", "data": "synthetic",
            "config": workload_config(args, n, per),
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "note": "per-sample latency = step time (all chains of a step finish together)"},
            "roofline": {"bound": "alu", "kernel": "evolve (two-site ops)", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                         "flops_per_step": flops_alg / args.steps,
                         "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz" if prec != b.HM_FP64
                         else "nominal GB300 FP64 rate"},
            "evolve_share": sum(evolve_ms) / t_ms,
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clk}
    if e2e:
        line["e2e"] = e2e
    if args.susceptibility:
        ctx.evolve(ids)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sus = ctx.susceptibility(ids)                 # host output, synchronised
        sus_s = time.perf_counter() - t0
        line["susceptibility"] = {"ms_per_call": 1e3 * sus_s, "chains": n,
                                  "chi_mean": float(sus[:, 0].mean()), "kernel": "susceptibility_fp64_kernel"}
        ctx.collapse(ids, n_env)
    if not args.no_cpu_baseline and world == 1:
        rate, dt, procs = oracle_sample_rate(1)
        line["cpu_baseline"] = {"value": rate, "unit": "samples/s", "cores": procs, "kind": "oracle",
                                "sample": "one Markov step of one chain on each of %d host cores (%.1f s wall, "
                                          "numpy/LAPACK FP64, 1 thread per process)" % (procs, dt)}
    print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
