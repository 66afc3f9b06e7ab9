"""Total-S^z (U(1)) block-sparse evolution of the hybrid state, Sec. II.C.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper passages followed (Sec. II.C, "Exploiting Conserved Quantum Numbers",
and Fig. qn):
* the ancilla legs carry flipped quantum numbers, so every Bell pair of the
  restored cluster has total S^z = 0;
* with the environment collapsed in the S^z basis, the next initial state
  |i>_E |B>_C has a definite total S^z, Q = sum of the environment outcomes'
  m values, which can change from sample to sample;
* the gates (Sec. I.A: exp(-tau J S_i.S_j) on physical legs, which conserves
  S^z_i + S^z_j) keep Q fixed during the evolution, so every MPS tensor is
  block sparse;
* METTS (no cluster) collapses every site, which keeps Q, so it stays in one
  sector.

Charge rule: A[l, s, r] = 0 unless q(l) + c(s) = q(r).  Here c(s) = m(s) =
+1, 0, -1 on physical legs and c(a) = -m(a) on ancilla legs.  The left edge
bond has charge 0 and the right edge bond has charge Q.  A SWAP moves a
site's content, and its leg charges with it, to the neighbouring position,
so each position's leg charges are tracked through the schedule.

Here every bond index carries its charge.  A two-site split groups the rows
(l, s1) of theta by q(l) + c(s1) and the columns (s2, r) by q(r) - c(s2).
theta is block diagonal in that charge, and each block is decomposed on its
own.  The singular values of a block-diagonal matrix are the union of its
blocks' values.  The truncation rule of ``mps.truncation_rank`` (Sec. II,
with the same readings) therefore runs on that union, sorted, and keeps the
set a dense SVD keeps.  Each kept value's block charge labels its new bond
index.  Exact centre moves are QR (or LQ) block by block.  The two-site
contraction and the gate are dense library steps, since their result does
not depend on blocking.  The decompositions, where the cost is, are the
blocked part.

Library primitives used as steps: numpy SVD and QR on each block.
Pins: ``tests/test_oracle_u1.py``:
* block evolution vs the dense oracle (state to 1e-12 without truncation,
  per-sample observables and collapse outcomes with truncation);
* the charge rule on every tensor;
* Q equal to the environment's S^z;
* METTS stuck in one sector while the hybrid chain's Q fluctuates (Fig. qn).
"""
import numpy as np

from . import chain as chainmod
from . import collapse as colmod
from . import model
from . import mps as mpsmod

M_OF = np.array([1, 0, -1])   # m of local basis index s (order +1, 0, -1)


def leg_charges(ladder):
    """Charge c(s) of every site's local leg: m(s) physical, -m(s) ancilla."""
    return [M_OF.copy() if kind == "P" else -M_OF for kind, _, _ in ladder.sites]


def right_charges(a, q_left, c, tol=0.0):
    """Charges of the right bond of a tensor, read off its nonzero entries."""
    chil, _, chir = a.shape
    out = np.zeros(chir, dtype=np.int64)
    for r in range(chir):
        nz = np.argwhere(np.abs(a[:, :, r]) > tol)
        if len(nz) == 0:
            raise ValueError("empty bond index has no charge")
        qs = {int(q_left[l] + c[s]) for l, s in nz}
        if len(qs) != 1:
            raise ValueError("tensor mixes charges on one bond index")
        out[r] = qs.pop()
    return out


class U1MPS(mpsmod.MPS):
    """MPS whose bond indices carry S^z charges: q[k] labels bond k (0..n)."""

    def __init__(self, tensors, charges, legs, centre=0):
        super().__init__(tensors, centre)
        self.q = [np.asarray(x, dtype=np.int64) for x in charges]
        self.legs = legs

    @property
    def total_charge(self):
        return int(self.q[-1][0])

    def violation(self):
        """Largest |A[l, s, r]| with q(l) + c(s) != q(r), over all tensors."""
        worst = 0.0
        for k, a in enumerate(self.tensors):
            bad = (self.q[k][:, None, None] + self.legs[k][None, :, None]) != self.q[k + 1][None, None, :]
            if bad.any():
                worst = max(worst, float(np.abs(a[bad]).max()))
        return worst


def product_state(ladder, env_outcomes):
    """|i>_E |B>_C in the S^z basis with charge labels (Sec. II.C)."""
    tensors = colmod.product_state(ladder, env_outcomes, colmod.BASIS_Z)
    legs = leg_charges(ladder)
    q = [np.zeros(1, dtype=np.int64)]
    for k, a in enumerate(tensors):
        q.append(right_charges(a, q[k], legs[k]))
    return U1MPS(tensors, q, legs, 0)


def _blocks(row_q, col_q):
    """Charges present on both sides, with their row and column indices."""
    out = []
    for q in sorted(set(row_q.tolist()) & set(col_q.tolist())):
        out.append((q, np.flatnonzero(row_q == q), np.flatnonzero(col_q == q)))
    return out


def output_legs(gate, c1, c2, tol=1e-14):
    """Leg charges after a two-site gate: (c1, c2), or (c2, c1) if it moves
    the site contents across (a SWAP, or a product with an odd number of
    them).  A gate that conserves neither way breaks the symmetry."""
    g = np.asarray(gate).reshape(model.D, model.D, model.D, model.D)     # (a, b, s1, s2)
    q_in = c1[None, None, :, None] + c2[None, None, None, :]
    scale = float(np.abs(g).max())
    for o1, o2 in ((c1, c2), (c2, c1)):
        bad = (o1[:, None, None, None] + o2[None, :, None, None]) != q_in
        if not bad.any() or float(np.abs(g[bad]).max()) <= tol * scale:
            return o1, o2
    raise FloatingPointError("gate does not conserve S^z")


def split(st, k, gate, absorb, chi_max, cutoff, sizes=None):
    """Block-sparse version of ``mps.split`` (gate on (k, k+1), truncated SVD).

    ``sizes``: if a list, the (rows, cols) of every block are appended.
    Returns the discarded weight.
    """
    if st.centre not in (k, k + 1):
        raise RuntimeError("split away from the orthogonality centre")
    a, b = st.tensors[k], st.tensors[k + 1]
    chil, chir = a.shape[0], b.shape[2]
    theta = np.tensordot(a, b, axes=(2, 0))
    g = np.asarray(gate).reshape(model.D, model.D, model.D, model.D)
    theta = np.einsum("abst,lstr->labr", g, theta).reshape(chil * model.D, model.D * chir)
    st.legs[k], st.legs[k + 1] = output_legs(gate, st.legs[k], st.legs[k + 1])
    row_q = (st.q[k][:, None] + st.legs[k][None, :]).reshape(-1)
    col_q = (st.q[k + 2][None, :] - st.legs[k + 1][:, None]).reshape(-1)
    off = row_q[:, None] != col_q[None, :]
    scale = float(np.abs(theta).max())
    if off.any() and float(np.abs(theta[off]).max()) > 1e-12 * scale:
        raise FloatingPointError("two-site tensor breaks S^z conservation")
    parts = []
    for q, rows, cols in _blocks(row_q, col_q):
        u, s, vt = mpsmod.thin_svd(theta[np.ix_(rows, cols)])
        parts.append((q, rows, cols, u, s, vt))
        if sizes is not None:
            sizes.append((len(rows), len(cols)))
    s_all = np.concatenate([p[4] for p in parts])
    owner = np.concatenate([np.full(len(p[4]), i) for i, p in enumerate(parts)])
    local = np.concatenate([np.arange(len(p[4])) for p in parts])
    order = np.argsort(-s_all, kind="stable")
    kk = mpsmod.truncation_rank(s_all[order], chi_max, cutoff)
    w = s_all * s_all
    discarded = float(np.sum(w[order[kk:]]) / np.sum(w))
    keep = order[:kk]
    sk = s_all[keep] / np.sqrt(np.sum(w[keep]))
    U = np.zeros((chil * model.D, kk))
    Vt = np.zeros((kk, model.D * chir))
    qnew = np.zeros(kk, dtype=np.int64)
    for j, idx in enumerate(keep):
        q, rows, cols, u, _, vt = parts[owner[idx]]
        U[rows, j] = u[:, local[idx]]
        Vt[j, cols] = vt[local[idx], :]
        qnew[j] = q
    if absorb == model.ABSORB_L:
        left, right = U * sk[None, :], Vt
        st.centre = k
    else:
        left, right = U, sk[:, None] * Vt
        st.centre = k + 1
    st.tensors[k] = left.reshape(chil, model.D, kk)
    st.tensors[k + 1] = right.reshape(kk, model.D, chir)
    st.q[k + 1] = qnew
    return discarded


def move_right(st, c):
    """Exact centre move c -> c+1: QR of each charge block of A_c."""
    a = st.tensors[c]
    chil, _, chir = a.shape
    m = a.reshape(chil * model.D, chir)
    row_q = (st.q[c][:, None] + st.legs[c][None, :]).reshape(-1)
    Qs, Rs, qs = [], [], []
    for q, rows, cols in _blocks(row_q, st.q[c + 1]):
        qq, rr = np.linalg.qr(m[np.ix_(rows, cols)])
        Qs.append((rows, qq))
        Rs.append((cols, rr))
        qs += [q] * qq.shape[1]
    n = len(qs)
    Q = np.zeros((chil * model.D, n))
    R = np.zeros((n, chir))
    j = 0
    for (rows, qq), (cols, rr) in zip(Qs, Rs):
        Q[rows, j:j + qq.shape[1]] = qq
        R[j:j + qq.shape[1]][:, cols] = rr
        j += qq.shape[1]
    st.tensors[c] = Q.reshape(chil, model.D, n)
    st.tensors[c + 1] = np.tensordot(R, st.tensors[c + 1], axes=(1, 0))
    st.q[c + 1] = np.array(qs, dtype=np.int64)
    st.centre = c + 1


def move_left(st, c):
    """Exact centre move c -> c-1: LQ of each charge block of A_c."""
    a = st.tensors[c]
    chil, _, chir = a.shape
    m = a.reshape(chil, model.D * chir)
    col_q = (st.q[c + 1][None, :] - st.legs[c][:, None]).reshape(-1)
    Ls, Qs, qs = [], [], []
    for q, rows, cols in _blocks(st.q[c], col_q):
        qq, rr = np.linalg.qr(m[np.ix_(rows, cols)].T)          # block^T = Q R
        Ls.append((rows, rr.T))
        Qs.append((cols, qq.T))
        qs += [q] * qq.shape[1]
    n = len(qs)
    L = np.zeros((chil, n))
    Qt = np.zeros((n, model.D * chir))
    j = 0
    for (rows, ll), (cols, qt) in zip(Ls, Qs):
        L[rows, j:j + ll.shape[1]] = ll
        Qt[j:j + qt.shape[0]][:, cols] = qt
        j += qt.shape[0]
    st.tensors[c] = Qt.reshape(n, model.D, chir)
    st.tensors[c - 1] = np.tensordot(st.tensors[c - 1], L, axes=(2, 0))
    st.q[c] = np.array(qs, dtype=np.int64)
    st.centre = c - 1


def evolve(st, ops, gates, chi_max, cutoff, sizes=None):
    """Run an op list (``model.plan_ops`` / ``model.schedule``) block by block.

    ``sizes``: if a list, one list of block (rows, cols) per split is appended.
    """
    for kind, k, gi, absorb in ops:
        if kind == model.SPLIT:
            blk = [] if sizes is not None else None
            split(st, k, gates[gi], absorb, chi_max, cutoff, blk)
            if sizes is not None:
                sizes.append(blk)
        elif kind == model.MOVE_R:
            if st.centre != k:
                raise RuntimeError("move_right from a site that is not the centre")
            move_right(st, k)
        elif kind == model.MOVE_L:
            if st.centre != k:
                raise RuntimeError("move_left from a site that is not the centre")
            move_left(st, k)
        else:
            raise ValueError("unknown op kind")
    return st


class U1Chain(chainmod.HybridChain):
    """The hybrid chain with S^z-basis collapses and block-sparse evolution.

    Identical to ``HybridChain(basis_zx=False)`` sample by sample (same
    draws, same kept singular values); each record also carries the initial
    state's total S^z, ``Q`` (Fig. qn)."""

    def __init__(self, *args, **kw):
        if kw.get("basis_zx", False):
            raise ValueError("the S^z sectors need S^z-basis collapses (basis_zx=False)")
        kw["basis_zx"] = False
        super().__init__(*args, **kw)

    def initial_mps(self):
        return product_state(self.ladder, self.env)

    def evolve(self, sizes=None):
        st = self.initial_mps()
        return evolve(st, self.ops, self.gates, self.chi_max, self.cutoff, sizes)

    def sample(self, sizes=None):
        q = int(sum(M_OF[s] for s in self.env))
        rec = super().sample(sizes)
        rec["Q"] = q
        return rec


def svd_cost(m, n):
    """Dense-SVD flop count 4 M^2 N + 8 M N^2 + 9 N^3 of an m x n matrix (M >= N)."""
    M, N = max(m, n), min(m, n)
    return 4.0 * M * M * N + 8.0 * M * N * N + 9.0 * N ** 3
