"""Spin-1 ladder model, hybrid site map, Trotter gates and the op schedule.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper passages followed:
* Sec. II, Eq. H: S=1 Heisenberg two-leg ladder, open boundaries, leg coupling
  J, rung coupling J_perp.
* Sec. I.A: local dimension d=3, M steps of size tau = beta/(2M), gates act on
  the physical sites only.
* Sec. I.C and Fig. 4: a contiguous central cluster of physical sites, each
  paired with an ancilla; every other physical site is an environment site.
* Sec. II ("Trotter-Suzuki decomposition", second order, error O(tau^3) per
  step).

Readings where the paper is silent (both the oracle and the CUDA planner
implement exactly these, independently):
* cluster = columns [x0, x0+Wc) with Wc = two_W/2, x0 = floor((Lx-Wc)/2);
* 1D order: column-major, (x,0) then (x,1); a cluster physical site is
  immediately followed by its ancilla;
* bonds sorted by (lower MPS index, upper MPS index); one second-order step is
  the forward sweep over that list with exp(-(tau/2) J h) followed by the
  reversed sweep with the same gates; in the plain schedule consecutive half
  steps are not merged (the fused schedule, ``fuse_ops``, merges every run of
  splits on one site pair, half-step turning points included);
* a gate on MPS sites i<j is applied with swap gates.  In a forward half step
  the centre is brought to i, site i is swapped right up to j-1, the gate acts
  on (j-1, j) and the site is swapped back; in a reverse half step the mirror
  image (centre at j, site j swapped left to i+1, gate on (i, i+1), swapped
  back).  Every two-site split truncates.  The final split of each gate leaves
  the centre on the side of the next gate's start; exact (untruncated) centre
  moves cover any remaining distance; after the last gate the centre is moved
  to site 0.
"""
import math

import numpy as np

D = 3  # spin-1 local dimension (Sec. I.A)

# Op kinds of the schedule.
SPLIT = 0    # theta = A_k A_{k+1}, gate, truncated SVD, absorb S left or right
MOVE_R = 1   # exact centre move k -> k+1 (QR of A_k)
MOVE_L = 2   # exact centre move k -> k-1 (LQ of A_k)

ABSORB_L = 0  # A_k <- U S, A_{k+1} <- V^T  (centre ends on k)
ABSORB_R = 1  # A_k <- U,   A_{k+1} <- S V^T (centre ends on k+1)

GATE_SWAP = 0  # gate table index 0 is the SWAP of the two physical legs


def spin1_operators():
    """S^z, S^+, S^- for S=1 in the basis m = +1, 0, -1 (all real)."""
    sz = np.diag([1.0, 0.0, -1.0])
    sp = np.zeros((D, D))
    sp[0, 1] = np.sqrt(2.0)
    sp[1, 2] = np.sqrt(2.0)
    sm = sp.T.copy()
    return sz, sp, sm


def bond_operator():
    """h = S_i . S_j = Sz Sz + (S+ S- + S- S+)/2 as a 9x9 matrix.

    Row index 3*s_i' + s_j', column index 3*s_i + s_j (s_i on the lower MPS
    index).  Sec. II, Eq. H.
    """
    sz, sp, sm = spin1_operators()
    return np.kron(sz, sz) + 0.5 * (np.kron(sp, sm) + np.kron(sm, sp))


def bond_gate(coef):
    """exp(-coef * h) for the 9x9 bond operator h (library eigensolver)."""
    h = bond_operator()
    w, v = np.linalg.eigh(h)
    return (v * np.exp(-coef * w)) @ v.T


def swap_gate():
    """Permutation P[(a b), (s1 s2)] = delta(a, s2) delta(b, s1)."""
    p = np.zeros((D * D, D * D))
    for s1 in range(D):
        for s2 in range(D):
            p[D * s2 + s1, D * s1 + s2] = 1.0
    return p


class Ladder:
    """Site map of the hybrid state for an Lx x 2 ladder (Sec. I.C, Fig. 4).

    Attributes
    ----------
    sites : list of (kind, x, y), kind 'P' (physical) or 'A' (ancilla)
    phys  : dict (x, y) -> MPS index of the physical site
    env   : MPS indices of environment physical sites, in MPS order
    cluster_cols : columns paired with ancillas
    bonds : list of (i, j, J) with MPS indices i < j, sorted by (i, j)
    """

    def __init__(self, Lx, two_W, J_leg=1.0, J_rung=1.0):
        if Lx < 1 or two_W < 0 or two_W % 2 or two_W > 2 * Lx:
            raise ValueError("need Lx >= 1 and even 0 <= two_W <= 2*Lx")
        self.Lx, self.two_W = Lx, two_W
        self.J_leg, self.J_rung = float(J_leg), float(J_rung)
        wc = two_W // 2
        x0 = (Lx - wc) // 2
        self.cluster_cols = list(range(x0, x0 + wc))
        self.sites, self.phys = [], {}
        for x in range(Lx):
            for y in (0, 1):
                self.phys[(x, y)] = len(self.sites)
                self.sites.append(("P", x, y))
                if x in self.cluster_cols:
                    self.sites.append(("A", x, y))
        self.n_sites = len(self.sites)
        self.env = [k for k, (kind, x, _) in enumerate(self.sites)
                    if kind == "P" and x not in self.cluster_cols]
        self.cluster_sites = [k for k, (_, x, _) in enumerate(self.sites)
                              if x in self.cluster_cols]
        bonds = []
        for x in range(Lx):
            bonds.append((self.phys[(x, 0)], self.phys[(x, 1)], self.J_rung))
        for x in range(Lx - 1):
            for y in (0, 1):
                bonds.append((self.phys[(x, y)], self.phys[(x + 1, y)], self.J_leg))
        bonds.sort(key=lambda b: (b[0], b[1]))
        self.bonds = bonds

    def measured_bonds(self, col_lo=None, col_hi=None):
        """Bonds (i, j, J) with both ends in columns [col_lo, col_hi).

        Default region: the cluster (Sec. II.A measures inside the cluster);
        with no cluster, the whole ladder.
        """
        if col_lo is None or col_hi is None:
            if self.cluster_cols:
                col_lo, col_hi = self.cluster_cols[0], self.cluster_cols[-1] + 1
            else:
                col_lo, col_hi = 0, self.Lx
        inside = {self.phys[(x, y)] for x in range(col_lo, col_hi) for y in (0, 1)}
        return [b for b in self.bonds if b[0] in inside and b[1] in inside]


def trotter_steps(beta, tau):
    """Number of steps M and the step tau_eff = beta/(2M) (Sec. I.A).

    M = floor(beta/(2 tau) + 1/2) (halves round up), at least 1 for beta > 0.
    """
    if beta < 0 or tau <= 0:
        raise ValueError("beta >= 0 and tau > 0 required")
    if beta == 0:
        return 0, tau
    m = max(1, int(math.floor(beta / (2.0 * tau) + 0.5)))
    return m, beta / (2.0 * m)


def gate_table(ladder, tau_eff):
    """Gate table: index 0 = SWAP, index 1 + b = exp(-(tau/2) J_b h) for bond b."""
    gates = [swap_gate()]
    for (_, _, J) in ladder.bonds:
        gates.append(bond_gate(0.5 * tau_eff * J))
    return gates


def plan_ops(ladder, n_steps):
    """Op list of one evolution by beta/2: n_steps second-order Trotter steps.

    Returns a list of tuples (kind, k, gate, absorb): SPLIT at (k, k+1) with
    gate index ``gate`` and absorb side; MOVE_R / MOVE_L at site k (gate and
    absorb are -1).  The centre starts and ends at site 0.
    """
    nb = len(ladder.bonds)
    seq = []
    for _ in range(n_steps):
        seq += [(b, "F") for b in range(nb)]
        seq += [(b, "R") for b in reversed(range(nb))]

    def target(entry):
        b, mode = entry
        i, j, _ = ladder.bonds[b]
        return i if mode == "F" else j

    ops, c = [], 0
    for t, (b, mode) in enumerate(seq):
        i, j, _ = ladder.bonds[b]
        tgt = target((b, mode))
        while c < tgt:
            ops.append((MOVE_R, c, -1, -1))
            c += 1
        while c > tgt:
            ops.append((MOVE_L, c, -1, -1))
            c -= 1
        g = 1 + b
        if mode == "F":
            for k in range(i, j - 1):
                ops.append((SPLIT, k, GATE_SWAP, ABSORB_R))
            ops.append((SPLIT, j - 1, g, ABSORB_L))
            for k in range(j - 2, i - 1, -1):
                ops.append((SPLIT, k, GATE_SWAP, ABSORB_L))
        else:
            for k in range(j - 1, i, -1):
                ops.append((SPLIT, k, GATE_SWAP, ABSORB_L))
            ops.append((SPLIT, i, g, ABSORB_R))
            for k in range(i + 1, j):
                ops.append((SPLIT, k, GATE_SWAP, ABSORB_R))
        # The last split leaves the centre towards the next gate's start.
        nxt = target(seq[t + 1]) if t + 1 < len(seq) else 0
        kind, k, gi, _ = ops[-1]
        absorb = ABSORB_L if nxt <= k else ABSORB_R
        ops[-1] = (kind, k, gi, absorb)
        c = k if absorb == ABSORB_L else k + 1
    while c > 0:
        ops.append((MOVE_L, c, -1, -1))
        c -= 1
    return ops


SCHEDULE_PLAIN = "plain"   # the op list of plan_ops as it stands
SCHEDULE_FUSED = "fused"   # plan_ops followed by fuse_ops


def _centre_after(op, c):
    kind, k, _, absorb = op
    if kind == SPLIT:
        return k if absorb == ABSORB_L else k + 1
    return k + 1 if kind == MOVE_R else k - 1


def fuse_ops(ops, gates):
    """Merge consecutive truncated splits that act on the same pair of sites.

    Sec. I.A applies a product of two-site gates; Sec. II's second-order
    step is palindromic.  Two gates applied one after the other to the same
    MPS pair (k, k+1) are one gate, their matrix product: the reverse sweep's
    first bond meets the forward sweep's last one (exp(-(tau/2)J h) twice =
    exp(-tau J h), the merged half steps of a second-order product), and a
    bond gate meets the SWAP that starts or ends a neighbouring bond's swap
    path.  A SWAP followed by a SWAP on the same pair is the identity; both
    drop out.  If they moved the centre, an exact move takes their place.
    The evolved state is the same product of gates applied to the same state,
    so without truncation it is unchanged.  With truncation, one SVD
    replaces two or more.

    ``ops`` come from ``plan_ops`` and ``gates`` from ``gate_table``.
    Returns ``(ops, gates)``.  New gate entries hold the products and are
    appended in order of first use.  A fused op keeps the absorb side of the
    last op it replaces.
    """
    # stack entries: [op, centre before it, word of base gate indices]
    out = []
    c = 0
    for op in ops:
        kind, k, g, absorb = op
        c_next = _centre_after(op, c)
        top = out[-1] if out else None
        if kind == SPLIT and top is not None and top[0][0] == SPLIT and top[0][1] == k:
            out.pop()
            word = top[2] + [g]
            if len(word) >= 2 and word[-1] == GATE_SWAP and word[-2] == GATE_SWAP:
                word = word[:-2]
            if word:
                out.append([(SPLIT, k, None, absorb), top[1], word])
            elif top[1] != c_next:
                move = MOVE_R if c_next > top[1] else MOVE_L
                out.append([(move, top[1], -1, -1), top[1], None])
            c = c_next
            continue
        out.append([op, c, [g] if kind == SPLIT else None])
        c = c_next
    table = list(gates)
    index = {}
    fused = []
    for op, _, word in out:
        if op[0] != SPLIT:
            fused.append(op)
            continue
        if len(word) == 1:
            gi = word[0]
        else:
            key = tuple(word)
            if key not in index:
                m = gates[word[0]]
                for w in word[1:]:
                    m = gates[w] @ m
                index[key] = len(table)
                table.append(m)
            gi = index[key]
        fused.append((SPLIT, op[1], gi, op[3]))
    return fused, table


def schedule(ladder, n_steps, tau_eff, kind=SCHEDULE_PLAIN):
    """Op list and gate table of one evolution by beta/2, plain or fused."""
    ops, gates = plan_ops(ladder, n_steps), gate_table(ladder, tau_eff)
    if kind == SCHEDULE_FUSED:
        return fuse_ops(ops, gates)
    if kind != SCHEDULE_PLAIN:
        raise ValueError("unknown schedule %r" % (kind,))
    return ops, gates
