"""Thermal averages from many chains, and their merge across ranks.

The Markov chain of Sec. I.C.1 estimates <A> = Tr[e^{-beta H} A]/Z by the
plain mean of the per-sample values <<A>>_n (Sec. I.C.1 step 3).  One
chain's samples are correlated, so the error bar comes from binning: the
chain's series is cut into consecutive bins of ``bin_size`` samples, and the
bin means are treated as independent.  Different chains are independent.

``Estimator`` keeps, per observable:
* the sum, the sum of squares and the count of every accepted sample;
* the sum, the sum of squares and the count of the completed bin means.
Each chain's incomplete bin is kept apart until it fills.  All sums are
additive, so estimators of disjoint chains merge by addition.  Across the
ranks of a multi-GPU run that addition is one all-reduce of a float64
vector: chains are independent, so this is the only exchange the
statistics need (Sec. III).  Samples a chain yields before ``n_warmup``
are discarded.
"""
import numpy as np


class Estimator:
    """Per-observable sums of the accepted samples of any number of chains."""

    def __init__(self, n_obs, bin_size=10, n_warmup=0):
        if n_obs < 1 or bin_size < 1 or n_warmup < 0:
            raise ValueError("n_obs >= 1, bin_size >= 1 and n_warmup >= 0 required")
        self.n_obs, self.bin_size, self.n_warmup = int(n_obs), int(bin_size), int(n_warmup)
        self.sums = np.zeros((6, self.n_obs))    # sum x, sum x^2, n, sum b, sum b^2, n_bins
        self._open = {}                          # chain -> [seen, partial bin sum, partial count]

    # -- accumulation -------------------------------------------------------------
    def add(self, chain, values):
        """Append the next samples of ``chain`` (shape (n_obs,) or (k, n_obs))."""
        x = np.asarray(values, dtype=np.float64).reshape(-1, self.n_obs)
        st = self._open.setdefault(chain, [0, np.zeros(self.n_obs), 0])
        for row in x:
            st[0] += 1
            if st[0] <= self.n_warmup:
                continue
            self.sums[0] += row
            self.sums[1] += row * row
            self.sums[2] += 1.0
            st[1] = st[1] + row
            st[2] += 1
            if st[2] == self.bin_size:
                b = st[1] / self.bin_size
                self.sums[3] += b
                self.sums[4] += b * b
                self.sums[5] += 1.0
                st[1], st[2] = np.zeros(self.n_obs), 0

    # -- merging --------------------------------------------------------------------
    def merge(self, other):
        """Add the completed sums of another estimator of disjoint chains."""
        if (other.n_obs, other.bin_size) != (self.n_obs, self.bin_size):
            raise ValueError("estimators differ in observables or bin size")
        self.sums += other.sums
        return self

    def to_vector(self):
        return self.sums.reshape(-1).copy()

    def load_vector(self, v):
        self.sums = np.asarray(v, dtype=np.float64).reshape(6, self.n_obs).copy()

    def all_reduce(self, dist, device=None):
        """Sum the completed sums of every rank (a no-op without a process group).

        ``device``: where the reduction tensor lives ("cpu" for gloo, the
        rank's CUDA device for NCCL)."""
        if not (dist.is_available() and dist.is_initialized()):
            return self
        import torch
        t = torch.tensor(self.to_vector(), dtype=torch.float64, device=device or "cpu")
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        self.load_vector(t.cpu().numpy())
        return self

    # -- results --------------------------------------------------------------------
    @property
    def count(self):
        return int(self.sums[2][0])

    def mean(self):
        n = self.sums[2]
        if n[0] == 0:
            raise ValueError("no accepted samples")
        return self.sums[0] / n

    def stderr(self):
        """Standard error of the mean from the completed bin means."""
        nb = self.sums[5][0]
        if nb < 2:
            raise ValueError("fewer than two completed bins")
        mb = self.sums[3] / nb
        var = (self.sums[4] - nb * mb * mb) / (nb - 1.0)
        return np.sqrt(np.maximum(var, 0.0) / nb)

    def naive_stderr(self):
        """Standard error ignoring autocorrelation (a lower bound for one chain)."""
        n = self.sums[2][0]
        if n < 2:
            raise ValueError("fewer than two samples")
        m = self.sums[0] / n
        var = (self.sums[1] - n * m * m) / (n - 1.0)
        return np.sqrt(np.maximum(var, 0.0) / n)
