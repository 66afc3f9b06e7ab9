"""The hybrid METTS-ancilla Markov chain, steps 1-4 of Sec. I.C.1 (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

One call of ``HybridChain.sample`` is one Markov step n:
  1. initial state |i_n>_E |B>_C (product environment, Bell-paired cluster);
  2. evolve by beta/2 with second-order Trotter gates on the physical legs;
  3. measure the cluster observables <<A>>_n;
  4. collapse the environment to |i_{n+1}>_E (basis of sample n) and reset
     the cluster to Bell pairs (the next call rebuilds it from the outcomes).
Pins: ``tests/test_oracle_chain.py`` (pure-ancilla limit: zero variance and
exact diagonalisation; beta = 0; thermal averages against exact
diagonalisation within 3 sigma).
"""
import numpy as np

from . import model, mps as mpsmod, measure as measmod, collapse as colmod


class HybridChain:
    def __init__(self, Lx, two_W, J_leg=1.0, J_rung=1.0, beta=1.0, tau=0.05,
                 chi_max=64, cutoff=1e-12, seed=0, chain_id=0,
                 basis_zx=True, meas_cols=None, schedule=model.SCHEDULE_PLAIN):
        self.ladder = model.Ladder(Lx, two_W, J_leg, J_rung)
        self.beta, self.chi_max, self.cutoff = beta, chi_max, cutoff
        self.seed, self.chain_id, self.basis_zx = seed, chain_id, basis_zx
        self.n_steps, self.tau_eff = model.trotter_steps(beta, tau)
        self.ops, self.gates = model.schedule(self.ladder, self.n_steps, self.tau_eff, schedule)
        if meas_cols is None:
            self.meas_bonds = self.ladder.measured_bonds()
        else:
            self.meas_bonds = self.ladder.measured_bonds(*meas_cols)
        self.env = colmod.initial_env(len(self.ladder.env), seed, chain_id)
        self.env_basis = colmod.BASIS_Z
        self.n = 0
        self.last_mps = None

    def initial_mps(self):
        return mpsmod.MPS(colmod.product_state(self.ladder, self.env, self.env_basis), 0)

    def evolve(self, log=None):
        st = self.initial_mps()
        return mpsmod.evolve(st, self.ops, self.gates, self.chi_max, self.cutoff, log)

    def sample(self, log=None):
        """One Markov step; returns dict(obs, env_out, basis, logp, n)."""
        st = self.evolve(log)
        obs = measmod.measure(st, self.meas_bonds)
        basis = colmod.sample_basis(self.n, self.basis_zx)
        out, logp, _ = colmod.collapse(st, self.ladder, basis, self.seed, self.chain_id, self.n)
        rec = dict(obs=obs, env_out=list(out), basis=basis, logp=logp, n=self.n,
                   env_in=list(self.env), basis_in=self.env_basis)
        self.env, self.env_basis = out, basis
        self.n += 1
        self.last_mps = st
        return rec


def binned_error(x, n_bins=10):
    """Mean and binning standard error of an autocorrelated series."""
    x = np.asarray(x, dtype=np.float64)
    m = len(x) // n_bins
    if m == 0:
        raise ValueError("series shorter than the number of bins")
    bins = x[: m * n_bins].reshape(n_bins, m).mean(axis=1)
    return float(x.mean()), float(bins.std(ddof=1) / np.sqrt(n_bins))
