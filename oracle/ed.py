"""Exact diagonalisation and dense (untruncated) evolution, tiny systems only.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* ``LadderED``: the Hamiltonian of Sec. II (Eq. H) built by applying S^z, S^+,
  S^- to explicit basis states, block-diagonalised by total S^z; thermal
  averages <A> = Tr[e^{-beta H} A]/Z (Sec. I, Eq. sqrtrho).  Its own site
  labels p = 2x + y; it does not use the MPS site map.
* ``trotter_thermal``: <A>_T = Tr[T A T]/Tr[T T] with T the dense second-order
  Trotter product for beta/2 (palindromic, hence symmetric): the exact target
  of the sampler before truncation.
* ``dense_evolve``: the hybrid initial state |i>_E|B>_C as a dense vector over
  physical and ancilla sites, with the same gate sequence applied directly to
  the two physical legs (no swaps, no SVD): the untruncated MPS evolution.
Pins: ``tests/test_oracle_ed.py`` (two-site closed form, traceless H, SU(2)
relation, high-temperature series, library matrix exponential).
"""
import math

import numpy as np

from .model import D, bond_gate, bond_operator, swap_gate  # noqa: F401


def _cp(m):   # <m+1|S+|m>
    return math.sqrt(2.0 - m * (m + 1))


def _cm(m):   # <m-1|S-|m>
    return math.sqrt(2.0 - m * (m - 1))


def ladder_bonds_xy(Lx, J_leg, J_rung):
    """Bonds of Eq. H as ((x, y), (x', y'), J)."""
    out = [((x, 0), (x, 1), J_rung) for x in range(Lx)]
    for x in range(Lx - 1):
        for y in (0, 1):
            out.append(((x, y), (x + 1, y), J_leg))
    return out


class LadderED:
    """Sz-sector exact diagonalisation of the Lx x 2 spin-1 ladder."""

    def __init__(self, Lx, J_leg=1.0, J_rung=1.0):
        self.Lx = Lx
        self.N = 2 * Lx
        self.bonds = [((2 * a[0] + a[1]), (2 * b[0] + b[1]), J)
                      for a, b, J in ladder_bonds_xy(Lx, J_leg, J_rung)]
        N = self.N
        states = np.array(np.unravel_index(np.arange(D ** N), (D,) * N)).T  # digits
        self.m = 1 - states                               # m = +1, 0, -1
        tot = self.m.sum(axis=1)
        self.sectors = {}
        for q in range(-N, N + 1):
            idx = np.nonzero(tot == q)[0]
            if len(idx):
                self.sectors[q] = idx
        self._eig = {}

    def _index(self, mvec):
        return int(np.ravel_multi_index(tuple(1 - np.asarray(mvec)), (D,) * self.N))

    def operator_block(self, q, terms):
        """Dense matrix of sum_t c_t * (op1_p op2_q) in sector q.

        ``terms`` = [(c, p, r, kind)], kind 'zz' (Sz_p Sz_r) or 'ss' (S_p . S_r).
        """
        idx = self.sectors[q]
        pos = {int(s): a for a, s in enumerate(idx)}
        M = np.zeros((len(idx), len(idx)))
        for col, s in enumerate(idx):
            mv = self.m[s]
            for c, p, r, kind in terms:
                mp, mr = mv[p], mv[r]
                M[col, col] += c * mp * mr
                if kind == "zz":
                    continue
                if mp < 1 and mr > -1:     # (1/2) S+_p S-_r
                    nv = mv.copy(); nv[p] += 1; nv[r] -= 1
                    M[pos[self._index(nv)], col] += 0.5 * c * _cp(mp) * _cm(mr)
                if mp > -1 and mr < 1:     # (1/2) S-_p S+_r
                    nv = mv.copy(); nv[p] -= 1; nv[r] += 1
                    M[pos[self._index(nv)], col] += 0.5 * c * _cm(mp) * _cp(mr)
        return M

    def hamiltonian_terms(self):
        return [(J, p, r, "ss") for p, r, J in self.bonds]

    def eig(self, q):
        if q not in self._eig:
            self._eig[q] = np.linalg.eigh(self.operator_block(q, self.hamiltonian_terms()))
        return self._eig[q]

    def thermal(self, beta, terms_list):
        """Thermal averages <O_t> for each O_t = terms_list[t]; also <H>."""
        e_min = min(self.eig(q)[0][0] for q in self.sectors)
        z = 0.0
        acc = np.zeros(len(terms_list) + 1)
        for q in self.sectors:
            w, v = self.eig(q)
            boltz = np.exp(-beta * (w - e_min))
            z += boltz.sum()
            acc[-1] += float(boltz @ w)
            for t, terms in enumerate(terms_list):
                o = self.operator_block(q, terms)
                acc[t] += float(boltz @ np.einsum("in,ij,jn->n", v, o, v))
        return acc / z

    def bond_thermal(self, beta, xy_pairs):
        """[(<S.S>, <SzSz>) for each ((x,y),(x',y'))] and <H>."""
        terms = []
        for a, b in xy_pairs:
            p, r = 2 * a[0] + a[1], 2 * b[0] + b[1]
            terms.append([(1.0, p, r, "ss")])
            terms.append([(1.0, p, r, "zz")])
        vals = self.thermal(beta, terms)
        return [(vals[2 * t], vals[2 * t + 1]) for t in range(len(xy_pairs))], vals[-1]


def _apply_two(psi, gate, i, j):
    """Apply a 9x9 gate to legs i, j of a dense tensor (gate rows (a b))."""
    g = gate.reshape(D, D, D, D)
    out = np.tensordot(g, psi, axes=([2, 3], [i, j]))
    return np.moveaxis(out, [0, 1], [i, j])


def gate_sequence(ladder, n_steps, tau_eff):
    """(i, j, gate) per gate: forward sweep then reversed sweep, per step."""
    seq = []
    gates = [bond_gate(0.5 * tau_eff * J) for (_, _, J) in ladder.bonds]
    for _ in range(n_steps):
        for b, (i, j, _) in enumerate(ladder.bonds):
            seq.append((i, j, gates[b]))
        for b in reversed(range(len(ladder.bonds))):
            i, j, _ = ladder.bonds[b]
            seq.append((i, j, gates[b]))
    return seq


def dense_initial(ladder, env_outcomes, basis_rows):
    """|i>_E |B>_C as a dense tensor over all MPS sites (tiny systems)."""
    env_pos = {k: e for e, k in enumerate(ladder.env)}
    psi = np.ones(())
    k = 0
    n = ladder.n_sites
    while k < n:
        kind = ladder.sites[k][0]
        if k in env_pos:
            psi = np.multiply.outer(psi, basis_rows[env_outcomes[env_pos[k]]])
            k += 1
        else:
            assert kind == "P" and ladder.sites[k + 1][0] == "A"
            psi = np.multiply.outer(psi, np.eye(D) / math.sqrt(D))
            k += 2
    return psi


def dense_evolve(ladder, env_outcomes, basis_rows, n_steps, tau_eff):
    """Unnormalised e^{-beta H/2}|i>_E|B>_C (Trotterised); returns (phi, |phi|^2)."""
    psi = dense_initial(ladder, env_outcomes, basis_rows)
    for i, j, g in gate_sequence(ladder, n_steps, tau_eff):
        psi = _apply_two(psi, g, i, j)
    return psi, float(np.sum(psi * psi))


def dense_expect(psi, i, j, op_i, op_j):
    """<psi| op_i op_j |psi> / <psi|psi> on legs i != j of a dense tensor."""
    phi = np.moveaxis(np.tensordot(op_i, psi, axes=([1], [i])), 0, i)
    phi = np.moveaxis(np.tensordot(op_j, phi, axes=([1], [j])), 0, j)
    return float(np.sum(psi * phi) / np.sum(psi * psi))


def trotter_operator(Lx, bonds_xy_ordered, n_steps, tau_eff):
    """Dense Trotter product T for beta/2 on the physical sites (N <= 6)."""
    N = 2 * Lx
    dim = D ** N
    t = np.eye(dim).reshape((D,) * N + (dim,))
    gates = [bond_gate(0.5 * tau_eff * J) for (_, _, J) in bonds_xy_ordered]
    lab = [(2 * a[0] + a[1], 2 * b[0] + b[1]) for a, b, _ in bonds_xy_ordered]
    for _ in range(n_steps):
        order = list(range(len(lab))) + list(reversed(range(len(lab))))
        for b in order:
            t = _apply_two(t, gates[b], lab[b][0], lab[b][1])
    return t.reshape(dim, dim)


def trotter_thermal(Lx, bonds_xy_ordered, n_steps, tau_eff, op_mats):
    """Tr[T O T]/Tr[T T] for dense physical-space operators O."""
    t = trotter_operator(Lx, bonds_xy_ordered, n_steps, tau_eff)
    tt = t @ t.T
    z = np.trace(tt)
    return [float(np.sum(o * tt.T) / z) for o in op_mats]


def dense_bond_operator(Lx, a, b, kind):
    """Dense S_a . S_b ('ss') or Sz_a Sz_b ('zz') on 2*Lx spin-1 sites."""
    from .model import spin1_operators
    sz, sp, sm = spin1_operators()
    N = 2 * Lx
    p, r = 2 * a[0] + a[1], 2 * b[0] + b[1]

    def embed(op1, op2):
        mats = [np.eye(D)] * N
        mats = list(mats)
        mats[p], mats[r] = op1, op2
        out = np.ones((1, 1))
        for m in mats:
            out = np.kron(out, m)
        return out
    if kind == "zz":
        return embed(sz, sz)
    return embed(sz, sz) + 0.5 * (embed(sp, sm) + embed(sm, sp))


def total_sz_squared(ed, beta):
    """<(S^z_tot)^2> = sum_q q^2 Z_q / Z from the S^z-sector spectra (no S.S operators)."""
    e_min = min(ed.eig(q)[0][0] for q in ed.sectors)
    z = acc = 0.0
    for q in ed.sectors:
        w = np.exp(-beta * (ed.eig(q)[0] - e_min)).sum()
        z += w
        acc += q * q * w
    return acc / z
