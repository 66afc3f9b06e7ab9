"""MPS state, truncated two-site splits and exact centre moves (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper passages followed:
* Sec. I.A: the state is an MPS, evolved with Trotter gates acting on the
  physical legs only.
* Sec. II (third source of error): after each gate the two-site tensor is
  split by an SVD truncated so that the discarded weight, sum of discarded
  s^2 over sum of all s^2, stays at or below a fixed cutoff.
* Eq. psi and the P_i definition: the state is kept at unit norm, so the kept
  singular values are renormalised after every truncation.

Readings where the paper is silent: the kept count is additionally capped at
chi_max, and is lowered to the nearest gap so that a (near-)degenerate
multiplet, s_{k+1} >= s_k (1 - 1e-8), is never split.

Library primitives used as steps: numpy SVD (LAPACK gesdd, with gesvd when
gesdd does not converge) and QR (geqrf).
Pins: ``tests/test_oracle_mps.py`` (dense Trotter evolver, single-rung closed
form, pure-ancilla limit against exact diagonalisation).
"""
import numpy as np

from .model import D, SPLIT, MOVE_R, MOVE_L, ABSORB_L

GAP_REL = 1e-8  # degenerate-multiplet guard of the truncation rule


class MPS:
    """Site tensors A[k] of shape (chi_{k-1}, d, chi_k), real FP64."""

    def __init__(self, tensors, centre=0):
        self.tensors = [np.asarray(t, dtype=np.float64) for t in tensors]
        self.centre = centre

    @property
    def n_sites(self):
        return len(self.tensors)

    def bond_dims(self):
        return [t.shape[2] for t in self.tensors[:-1]]

    def to_dense(self):
        """Contract to a dense vector (tiny systems only)."""
        psi = self.tensors[0]
        for t in self.tensors[1:]:
            psi = np.tensordot(psi, t, axes=(psi.ndim - 1, 0))
        return psi.reshape(-1)


def truncation_rank(s, chi_max, cutoff):
    """Kept count k for singular values s sorted in descending order.

    k is the smallest k >= 1 whose discarded weight sum_{q>k} s_q^2 / sum s^2 is
    at most ``cutoff`` (Sec. II); then k <- min(k, chi_max); then, while the next
    value s_{k+1} >= s_k (1 - 1e-8), k is lowered (never below 1).
    """
    n = len(s)
    w = s * s
    # tail[q] = sum_{p >= q} w_p, accumulated from the smallest value upwards
    tail = np.zeros(n + 1)
    for q in range(n - 1, -1, -1):
        tail[q] = tail[q + 1] + w[q]
    total = float(tail[0])
    if not np.isfinite(total) or total <= 0.0:
        raise FloatingPointError("zero or non-finite two-site tensor")
    k = n
    for kk in range(1, n + 1):
        if tail[kk] <= cutoff * total:
            k = kk
            break
    k = min(k, chi_max)
    while 1 < k < n and s[k] >= s[k - 1] * (1.0 - GAP_REL):
        k -= 1
    return k


def thin_svd(m):
    """Thin SVD, a library step: LAPACK gesdd, or gesvd when gesdd does not
    converge.  That happens on strongly rank-deficient two-site tensors, for
    example a fully polarised environment around a small cluster.  Both
    drivers compute the same decomposition."""
    try:
        return np.linalg.svd(m, full_matrices=False)
    except np.linalg.LinAlgError:
        import scipy.linalg
        return scipy.linalg.svd(m, full_matrices=False, lapack_driver="gesvd")


def split(mps, k, gate, absorb, chi_max, cutoff):
    """Apply a 9x9 gate to sites (k, k+1) and split by a truncated SVD.

    gate[(a b), (s1 s2)] acts on the physical legs (Sec. I.A).  Returns the
    discarded weight.  Absorb left: A_k <- U S, A_{k+1} <- V^T; absorb right:
    A_k <- U, A_{k+1} <- S V^T.
    """
    if mps.centre not in (k, k + 1):
        raise RuntimeError("split away from the orthogonality centre")
    a, b = mps.tensors[k], mps.tensors[k + 1]
    chil, chir = a.shape[0], b.shape[2]
    theta = np.tensordot(a, b, axes=(2, 0))                     # (l, s1, s2, r)
    g = np.asarray(gate).reshape(D, D, D, D)                     # (a, b, s1, s2)
    theta = np.einsum("abst,lstr->labr", g, theta)
    u, s, vt = thin_svd(theta.reshape(chil * D, D * chir))
    kk = truncation_rank(s, chi_max, cutoff)
    w = s * s
    discarded = float(np.sum(w[kk:]) / np.sum(w))
    sk = s[:kk] / np.sqrt(np.sum(w[:kk]))
    u, vt = u[:, :kk], vt[:kk, :]
    if absorb == ABSORB_L:
        left, right = u * sk[None, :], vt
        mps.centre = k
    else:
        left, right = u, sk[:, None] * vt
        mps.centre = k + 1
    mps.tensors[k] = left.reshape(chil, D, kk)
    mps.tensors[k + 1] = right.reshape(kk, D, chir)
    return discarded


def move_right(mps, c):
    """Exact centre move c -> c+1: QR of A_c as (chi_l d) x chi_r."""
    a = mps.tensors[c]
    chil, _, chir = a.shape
    q, r = np.linalg.qr(a.reshape(chil * D, chir))
    mps.tensors[c] = q.reshape(chil, D, q.shape[1])
    mps.tensors[c + 1] = np.tensordot(r, mps.tensors[c + 1], axes=(1, 0))
    mps.centre = c + 1


def move_left(mps, c):
    """Exact centre move c -> c-1: LQ of A_c as chi_l x (d chi_r)."""
    a = mps.tensors[c]
    chil, _, chir = a.shape
    q, r = np.linalg.qr(a.reshape(chil, D * chir).T)           # A^T = Q R
    mps.tensors[c] = q.T.reshape(q.shape[1], D, chir)
    mps.tensors[c - 1] = np.tensordot(mps.tensors[c - 1], r.T, axes=(2, 0))
    mps.centre = c - 1


def evolve(mps, ops, gates, chi_max, cutoff, log=None):
    """Run an op list from ``model.plan_ops`` (Sec. I.C.1 step 2).

    If ``log`` is a list, one (kind, k, chi_l, chi_m, chi_r, kept, discarded)
    tuple is appended per op (chi_m = inner bond before the op).
    """
    for kind, k, gi, absorb in ops:
        if kind == SPLIT:
            chil, chim = mps.tensors[k].shape[0], mps.tensors[k].shape[2]
            chir = mps.tensors[k + 1].shape[2]
            disc = split(mps, k, gates[gi], absorb, chi_max, cutoff)
            if log is not None:
                log.append((kind, k, chil, chim, chir, mps.tensors[k].shape[2], disc))
        elif kind == MOVE_R:
            if mps.centre != k:
                raise RuntimeError("move_right from a site that is not the centre")
            move_right(mps, k)
        elif kind == MOVE_L:
            if mps.centre != k:
                raise RuntimeError("move_left from a site that is not the centre")
            move_left(mps, k)
        else:
            raise ValueError("unknown op kind")
    return mps
