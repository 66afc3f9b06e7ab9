"""Counter-based RNG, projective collapse of the environment, Bell-pair reset.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper passages followed:
* Sec. I.C.1 step 4: the environment sites are collapsed to a new product
  state by projective measurements of each site in turn, then every cluster
  physical site is re-paired with its ancilla in a Bell pair.
* Sec. I.C, Bell pair |B_j> = d^{-1/2} sum_s |s>_P |s>_A.
* Sec. I.C.2, Eq. detailbalance1: the probability of the new environment state
  j is <psi_i| Pi_j |psi_i> with Pi_j = |j><j|_E (x) 1_C, i.e. the cluster is
  traced out, which is why a density matrix is carried past the cluster.

Readings where the paper is silent:
* measurement basis of sample n: S^z eigenbasis for even n, S^x eigenbasis for
  odd n (or S^z always); x eigenvectors (m=+1,0,-1 components):
  v+ = (1/2, 1/sqrt2, 1/2), v0 = (1/sqrt2, 0, -1/sqrt2), v- = (1/2, -1/sqrt2, 1/2);
* random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key =
  (seed mod 2^32, chain id), counter = (n mod 2^32, env ordinal, seed >> 32, 0);
  u = ((x0 >> 5) 2^26 + (x1 >> 6)) 2^-53; the outcome is the first b with
  u < cumulative p_b (else the last b with p_b > 0).  The initial environment
  is drawn in the S^z basis with p = 1/3 each and n = -1.

Pins: ``tests/test_oracle_collapse.py`` (Philox against cuRAND's host
generator of the same kind, brute force enumeration of collapse
probabilities, detailed balance).
"""
import math

import numpy as np

from .model import D

BASIS_Z = 0
BASIS_X = 1

_M0, _M1 = 0xD2511F53, 0xCD9E8D57
_W0, _W1 = 0x9E3779B9, 0xBB67AE85
_MASK = 0xFFFFFFFF


def philox4x32_10(counter, key):
    """Philox4x32 with 10 rounds; counter = 4 words, key = 2 words."""
    c0, c1, c2, c3 = (int(x) & _MASK for x in counter)
    k0, k1 = (int(x) & _MASK for x in key)
    for r in range(10):
        if r:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> 32, p0 & _MASK
        hi1, lo1 = p1 >> 32, p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def uniform(seed, chain, n, ordinal):
    """The uniform draw in [0, 1) for env ordinal ``ordinal`` of sample ``n``."""
    x = philox4x32_10((n & _MASK, ordinal, (seed >> 32) & _MASK, 0),
                      (seed & _MASK, chain & _MASK))
    return ((x[0] >> 5) * 67108864 + (x[1] >> 6)) / 9007199254740992.0


def choose(p, u):
    """First b with u < sum_{q<=b} p_q; else the last b with p_b > 0."""
    acc = 0.0
    for b, pb in enumerate(p):
        acc += pb
        if u < acc:
            return b
    for b in range(len(p) - 1, -1, -1):
        if p[b] > 0.0:
            return b
    raise FloatingPointError("all collapse probabilities are zero")


def basis_matrix(basis):
    """Rows are the basis vectors (components in m = +1, 0, -1 order)."""
    if basis == BASIS_Z:
        return np.eye(D)
    r = 1.0 / math.sqrt(2.0)
    return np.array([[0.5, r, 0.5], [r, 0.0, -r], [0.5, -r, 0.5]])


def sample_basis(n, schedule_zx=True):
    """Basis used to collapse after sample n (Sz for even n, Sx for odd n)."""
    return BASIS_X if (schedule_zx and n % 2 == 1) else BASIS_Z


def initial_env(n_env, seed, chain):
    """Environment outcomes of the first initial state (S^z basis, n = -1)."""
    third = 1.0 / 3.0
    return [choose([third, third, third], uniform(seed, chain, -1, e)) for e in range(n_env)]


def product_state(ladder, env_outcomes, basis):
    """Site tensors of |i>_E |B>_C (Sec. I.C.1 step 1, Sec. I.C Bell pair).

    Environment site: basis vector of its outcome, shape (1, d, 1).  Cluster
    physical site: delta(s, alpha)/sqrt(d), shape (1, d, d); its ancilla:
    delta(alpha, a), shape (d, d, 1).  Every tensor is right-orthonormal, so
    the state is in right-canonical form with the centre on site 0.
    """
    bm = basis_matrix(basis)
    env_pos = {k: e for e, k in enumerate(ladder.env)}
    tensors = []
    for k, (kind, _, _) in enumerate(ladder.sites):
        if k in env_pos:
            tensors.append(bm[env_outcomes[env_pos[k]]].reshape(1, D, 1).copy())
        elif kind == "P":
            tensors.append(np.eye(D).reshape(1, D, D) / math.sqrt(D))
        else:
            tensors.append(np.eye(D).reshape(D, D, 1))
    return tensors


def collapse(mps, ladder, basis, seed, chain, n, forced=None):
    """Sequential projective measurement of the environment, left to right.

    Requires the centre on site 0 (sites 1.. right-orthonormal), so that the
    conditional probabilities only need the left boundary.  Before the first
    cluster site the boundary is a vector v (p_b = |v A~^b|^2); from the first
    cluster site on it is a density rho = v v^T, cluster sites are traced
    (rho <- sum_s A^sT rho A^s) and environment sites use p_b = Tr[A~^bT rho A~^b].
    A~^b = sum_s <b|s> A^s.  Returns (outcomes, log_p, conditional p vectors).
    ``forced`` replaces the draws by given outcomes (for brute-force checks).
    """
    if mps.centre != 0:
        raise RuntimeError("collapse needs the orthogonality centre on site 0")
    bm = basis_matrix(basis)
    env_pos = {k: e for e, k in enumerate(ladder.env)}
    v = np.ones(1)
    rho = None
    outcomes, conds, logp = [], [], 0.0
    for k, a in enumerate(mps.tensors):
        if k in env_pos:
            e = env_pos[k]
            arot = np.einsum("bs,lsr->blr", bm, a)
            if rho is None:
                w = [v @ arot[b] for b in range(D)]
                q = np.array([float(x @ x) for x in w])
            else:
                w = [rho @ arot[b] for b in range(D)]
                q = np.array([float(np.sum(arot[b] * w[b])) for b in range(D)])
            p = q / np.sum(q)
            b = forced[e] if forced is not None else choose(p, uniform(seed, chain, n, e))
            if rho is None:
                v = w[b] / math.sqrt(q[b])
            else:
                rho = (arot[b].T @ w[b]) / q[b]
            outcomes.append(b)
            conds.append(p)
            logp += math.log(p[b])
        else:
            if rho is None:
                rho = np.outer(v, v)
            rho = np.einsum("ij,isk,jsl->kl", rho, a, a, optimize=True)
    return outcomes, logp, conds
