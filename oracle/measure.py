"""Cluster observables of one sample: <<A>>_n = <psi|A|psi> (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper passages followed:
* Sec. I.C.1 step 3: the Monte Carlo estimator of an observable is its
  expectation value in the evolved, normalised state.
* Sec. II.A: observables are taken on physical sites of the cluster; the
  energy estimator is the sum over measured bonds of J_b <S_i . S_j>.
* Sec. II, Eq. H: S_i . S_j = Sz Sz + (S+ S- + S- S+)/2.

The contraction makes no canonical-form assumption: left and right
environments are built over all sites and every value is divided by <psi|psi>.

Output layout of ``measure`` (also the layout of the CUDA library's output):
  [0]               E_est = sum_b J_b <S_i . S_j>_b over measured bonds
  [1 + 2 b]         <S_i . S_j> of measured bond b (bonds in sorted order)
  [2 + 2 b]         <Sz_i Sz_j> of measured bond b
``susceptibility`` follows Eq. sus (Sec. II.A): chi = (beta/3) sum_i <S_c . S_i>,
averaged over the centre sites c of the measured region.
Pins: ``tests/test_oracle_measure.py`` (dense expectation values, SU(2)
relation in the pure-ancilla limit, beta = 0 values).
"""
import numpy as np

from .model import spin1_operators


def _left(L, a, op=None):
    # L'[k,l] = sum L[i,j] A[i,s,k] O[s,t] A[j,t,l]   (bra index s, ket index t)
    if op is None:
        return np.einsum("ij,isk,jsl->kl", L, a, a, optimize=True)
    return np.einsum("ij,isk,st,jtl->kl", L, a, op, a, optimize=True)


def _right(R, a):
    return np.einsum("isk,kl,jsl->ij", a, R, a, optimize=True)


def environments(mps):
    """Plain left environments L[k] (sites < k) and right R[k] (sites > k)."""
    n = mps.n_sites
    left = [np.ones((1, 1))]
    for k in range(n):
        left.append(_left(left[-1], mps.tensors[k]))
    right = [None] * n
    r = np.ones((1, 1))
    for k in range(n - 1, -1, -1):
        right[k] = r
        r = _right(r, mps.tensors[k])
    return left, right


def two_point(mps, envs, i, j, op_i, op_j):
    """<psi| op_i op_j |psi> / <psi|psi> for MPS sites i < j."""
    left, right = envs
    norm = float(np.trace(left[mps.n_sites]))
    L = _left(left[i], mps.tensors[i], op_i)
    for k in range(i + 1, j):
        L = _left(L, mps.tensors[k])
    L = _left(L, mps.tensors[j], op_j)
    return float(np.sum(L * right[j])) / norm


def bond_values(mps, envs, i, j):
    """(<S_i . S_j>, <Sz_i Sz_j>) for MPS sites i < j."""
    sz, sp, sm = spin1_operators()
    zz = two_point(mps, envs, i, j, sz, sz)
    pm = two_point(mps, envs, i, j, sp, sm)
    mp = two_point(mps, envs, i, j, sm, sp)
    return zz + 0.5 * (pm + mp), zz


def measure(mps, bonds):
    """Observable vector of one sample for measured bonds [(i, j, J), ...]."""
    envs = environments(mps)
    out = np.zeros(1 + 2 * len(bonds))
    for b, (i, j, J) in enumerate(bonds):
        ss, zz = bond_values(mps, envs, i, j)
        out[1 + 2 * b] = ss
        out[2 + 2 * b] = zz
        out[0] += J * ss
    return out


def susceptibility(mps, ladder, region_sites, beta):
    """Estimator of the uniform susceptibility of Eq. sus for one sample.

    chi_M = (beta / 3) (1 / |M|) sum_{j in M} sum_{i physical} <S_j . S_i>, with
    M = ``region_sites`` (MPS indices of physical sites; the paper averages j
    over the central 6 x 2 block) and i running over every physical site of the
    ladder, environment included (<S_j . S_j> = s(s+1) = 2).  Returns
    (chi_M, raw sum).  Written directly from Eq. sus with two-point functions.
    """
    envs = environments(mps)
    phys = [k for k, (kind, _, _) in enumerate(ladder.sites) if kind == "P"]
    total = 0.0
    for j in region_sites:
        for i in phys:
            if i == j:
                total += 2.0
            else:
                a, b = min(i, j), max(i, j)
                total += bond_values(mps, envs, a, b)[0]
    return beta / 3.0 * total / len(region_sites), total
