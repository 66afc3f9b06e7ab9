"""Seeded synthetic inputs shared by the tests and the benchmark.

This module holds no arithmetic of the method: only workload parameter sets
(S=1 Heisenberg ladders, Hamiltonian-defined, so there is no dataset) and
seeded random tensors for kernel-level parity cases.  Both the oracle-side and
the CUDA-side of a test draw their inputs from here.
"""
import numpy as np

# Workloads.  cutoff = 1e-7 is the truncation error cutoff the paper uses for
# its hybrid samples (Sec. II.A); the small case keeps the tighter 1e-12.
SMALL = dict(Lx=4, two_W=4, J_leg=1.0, J_rung=1.0, beta=2.0, tau=0.1,
             chi_max=64, cutoff=1e-12)
LADDER16 = dict(Lx=16, two_W=8, J_leg=1.0, J_rung=1.0, beta=1.0, tau=0.05,
                chi_max=256, cutoff=1e-7)
LADDER32 = dict(Lx=32, two_W=8, J_leg=1.0, J_rung=1.0, beta=4.0, tau=0.05,
                chi_max=512, cutoff=1e-7)


def ladder(name, **over):
    """Copy of a named workload with overrides."""
    base = {"small": SMALL, "ladder16": LADDER16, "ladder32": LADDER32}[name]
    out = dict(base)
    out.update(over)
    return out


def random_mps(n_sites, dims, seed, d=3):
    """Random real tensors with bond dims ``dims`` (len n_sites + 1, ends 1)."""
    rng = np.random.default_rng(seed)
    assert len(dims) == n_sites + 1 and dims[0] == 1 and dims[-1] == 1
    return [rng.standard_normal((dims[k], d, dims[k + 1])) for k in range(n_sites)]


def random_matrix(m, n, seed, decay=None):
    """Random m x n matrix; with ``decay`` its singular values fall as decay**i."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((m, n))
    if decay is None:
        return a
    u, _, vt = np.linalg.svd(a, full_matrices=False)
    s = decay ** np.arange(min(m, n))
    return (u * s) @ vt


def env_draws(n_env, seed):
    """Seeded environment outcomes in {0, 1, 2} for explicit initial states."""
    return np.random.default_rng(seed).integers(0, 3, size=n_env).astype(np.int8)


# Uneven batch: chains of mixed ladder length, cluster size, temperature and
# bond cap in one batch.
UNEVEN_MIX = dict(Lx=(8, 16, 24, 32), two_W=(4, 8), beta=(0.5, 16.0), chi_max=(64, 128, 256, 512),
                  tau=0.05, cutoff=1e-7, J_leg=1.0, J_rung=1.0)


def uneven_batch(n, seed, mix=None):
    """Seeded list of n ladder parameter dicts: Lx, two_W and chi_max
    uniform over the mix's choices, beta log-uniform over its range."""
    mix = dict(UNEVEN_MIX if mix is None else mix)
    rng = np.random.default_rng(seed)
    lo, hi = mix["beta"]
    return [dict(Lx=int(rng.choice(mix["Lx"])), two_W=int(rng.choice(mix["two_W"])),
                 beta=float(np.exp(rng.uniform(np.log(lo), np.log(hi)))), tau=mix["tau"],
                 chi_max=int(rng.choice(mix["chi_max"])), cutoff=mix["cutoff"],
                 J_leg=mix["J_leg"], J_rung=mix["J_rung"]) for _ in range(n)]


# Serving workload: a Poisson stream of sampling requests of mixed sizes.
SERVE_MIX = dict(Lx=(8, 16, 32), two_W=(4, 8), beta=(0.5, 16.0), chi_max=(128, 256, 512),
                 samples=(100, 2000), tau=0.05, cutoff=1e-7, J_leg=1.0, J_rung=1.0)


def poisson_requests(rate, duration_s, seed, mix=None):
    """Seeded request stream: exponential inter-arrival times of mean 1/rate
    over [0, duration_s).  Each request draws Lx, two_W and chi_max uniformly
    from the mix's choices, beta log-uniformly from its range, and the
    sample count uniformly from its integer range.

    Returns a list of (t_s, ladder parameter dict, n_samples)."""
    mix = dict(SERVE_MIX if mix is None else mix)
    rng = np.random.default_rng(seed)
    out, t = [], 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration_s:
            return out
        lo, hi = mix["beta"]
        cfg = dict(Lx=int(rng.choice(mix["Lx"])), two_W=int(rng.choice(mix["two_W"])),
                   beta=float(np.exp(rng.uniform(np.log(lo), np.log(hi)))), tau=mix["tau"],
                   chi_max=int(rng.choice(mix["chi_max"])), cutoff=mix["cutoff"],
                   J_leg=mix["J_leg"], J_rung=mix["J_rung"])
        n = int(rng.integers(mix["samples"][0], mix["samples"][1] + 1))
        out.append((t, cfg, n))
