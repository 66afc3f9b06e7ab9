"""Writes the stored expected values under tests/golden/ (calls only oracle/).

small_ladder_exact.json: exact thermal values of the small workload
(Lx = 4 two-leg S=1 Heisenberg ladder, J_leg = J_rung = 1, beta = 2,
tau = 0.1, cluster of 2W = 4 sites). Per bond of the cluster it holds
<S_i.S_j> and <Sz_i Sz_j> of Tr[e^{-beta H} O]/Z (Eq. sqrtrho), by
diagonalising the 3^8-dimensional ladder in S^z sectors. It also holds
the cluster energy of the same expression with e^{-beta H/2} replaced by
the second-order Trotter product the sampler applies (Sec. I.A, Sec. II).

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import ed, model  # noqa: E402

CFG = dict(Lx=4, two_W=4, J_leg=1.0, J_rung=1.0, beta=2.0, tau=0.1)


def exact_values(with_trotter=True):
    lad = model.Ladder(CFG["Lx"], CFG["two_W"], CFG["J_leg"], CFG["J_rung"])
    inv = {k: xy for xy, k in lad.phys.items()}
    bonds = lad.measured_bonds()
    vals, h = ed.LadderED(CFG["Lx"], CFG["J_leg"], CFG["J_rung"]).bond_thermal(
        CFG["beta"], [(inv[i], inv[j]) for i, j, _ in bonds])
    out = dict(config=CFG,
               bonds=[dict(i=int(i), j=int(j), J=J, ss=v[0], zz=v[1]) for (i, j, J), v in zip(bonds, vals)],
               H_ed=h, E_cluster_ed=sum(J * v[0] for (_, _, J), v in zip(bonds, vals)))
    if with_trotter:
        n, teff = model.trotter_steps(CFG["beta"], CFG["tau"])
        bonds_xy = [(inv[i], inv[j], J) for i, j, J in lad.bonds]
        hm = sum(J * ed.dense_bond_operator(CFG["Lx"], inv[i], inv[j], "ss") for i, j, J in bonds)
        (out["E_cluster_trotter"],) = ed.trotter_thermal(CFG["Lx"], bonds_xy, n, teff, [hm])
    return out


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "small_ladder_exact.json")
    with open(path, "w") as f:
        json.dump(exact_values(), f, indent=1)
    print("wrote", path)
