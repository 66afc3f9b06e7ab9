"""Pins of oracle/ed.py: closed forms, traceless H, SU(2), high-T series."""
import math

import numpy as np
import pytest

from oracle import ed, model


def two_site_energy(beta, J=1.0):
    """Two coupled spin-1: S.S eigenvalues -2 (x1), -1 (x3), +1 (x5)."""
    num = J * (-2 * math.exp(2 * beta * J) - 3 * math.exp(beta * J) + 5 * math.exp(-beta * J))
    den = math.exp(2 * beta * J) + 3 * math.exp(beta * J) + 5 * math.exp(-beta * J)
    return num / den


@pytest.mark.parametrize("beta", [0.0, 0.3, 1.0, 4.0])
def test_single_rung_closed_form(beta):
    e = ed.LadderED(1, J_leg=1.0, J_rung=1.0)
    vals, H = e.bond_thermal(beta, [((0, 0), (0, 1))])
    assert abs(H - two_site_energy(beta)) < 1e-13
    assert abs(vals[0][0] - two_site_energy(beta)) < 1e-13


def test_ground_state_two_sites():
    e = ed.LadderED(1)
    assert abs(min(e.eig(q)[0][0] for q in e.sectors) + 2.0) < 1e-13


def test_sector_dimensions():
    e = ed.LadderED(4)
    assert sum(len(v) for v in e.sectors.values()) == 3 ** 8
    assert len(e.sectors[0]) == 1107


@pytest.mark.parametrize("Lx", [2, 3])
def test_infinite_temperature_and_su2(Lx):
    e = ed.LadderED(Lx, J_leg=1.0, J_rung=0.5)
    pairs = [((0, 0), (0, 1)), ((0, 1), (1, 1))]
    vals, H = e.bond_thermal(0.0, pairs)
    assert abs(H) < 1e-12                        # Tr H = 0
    for ss, zz in vals:
        assert abs(ss) < 1e-13 and abs(zz) < 1e-13
    vals, _ = e.bond_thermal(1.3, pairs)
    for ss, zz in vals:                           # SU(2): <S.S> = 3 <Sz Sz>
        assert abs(ss - 3 * zz) < 1e-12
        assert ss < 0                             # antiferromagnetic


def test_high_temperature_series():
    # <H> = -beta Tr(H^2)/3^N + O(beta^2), Tr(H^2)/3^N = (4/3) sum_b J_b^2
    Lx, Jl, Jr = 3, 1.0, 0.5
    e = ed.LadderED(Lx, Jl, Jr)
    m2 = 4.0 / 3.0 * (Lx * Jr ** 2 + 2 * (Lx - 1) * Jl ** 2)
    beta = 1e-4
    _, H = e.bond_thermal(beta, [])
    assert abs(H / beta + m2) < 1e-3 * m2


def test_trotter_thermal_converges_to_ed():
    # second order: error of <H> at fixed beta scales as tau^2
    Lx = 2
    lad = model.Ladder(Lx, 0)
    bonds_xy = []
    inv = {k: (x, y) for (x, y), k in lad.phys.items()}
    for i, j, J in lad.bonds:
        bonds_xy.append((inv[i], inv[j], J))
    beta = 2.0
    hmat = sum(J * ed.dense_bond_operator(Lx, a, b, "ss") for a, b, J in bonds_xy)
    e = ed.LadderED(Lx)
    _, exact = e.bond_thermal(beta, [])
    errs = []
    for m in (5, 10, 20):
        tau = beta / (2 * m)
        (val,) = ed.trotter_thermal(Lx, bonds_xy, m, tau, [hmat])
        errs.append(abs(val - exact))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.8 < r2 < 4.2


def test_dense_bond_operator_matches_sector_blocks():
    Lx = 2
    e = ed.LadderED(Lx)
    full = ed.dense_bond_operator(Lx, (0, 1), (1, 1), "ss")
    for q, idx in e.sectors.items():
        blk = e.operator_block(q, [(1.0, 1, 3, "ss")])
        assert np.allclose(full[np.ix_(idx, idx)], blk, atol=1e-14)
