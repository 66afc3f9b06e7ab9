"""Stored exact values of the small workload (tests/golden/, written by
tests/golden/make_golden.py, which calls only the oracle).

Pins other than the oracle itself:
* SU(2) symmetry of e^{-beta H}, bond by bond: <S.S> = 3 <Sz Sz>;
* reflection symmetry of the ladder: bonds mapped onto each other by
  x -> Lx-1-x or by exchanging the legs have equal values;
* the Trotter product differs from e^{-beta H/2} by O(tau^2): the
  Trotterised cluster energy is within 1e-3 of the exact one.
The regeneration check guards the stored ED numbers against drift in the
oracle's exact diagonalisation. The Trotterised value takes minutes to
recompute; ``python tests/golden/make_golden.py`` does it.
"""
import json
import os
import sys

import pytest

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, HERE)
import make_golden  # noqa: E402


@pytest.fixture(scope="module")
def gold():
    with open(os.path.join(HERE, "small_ladder_exact.json")) as f:
        return json.load(f)


def test_su2_and_reflection_symmetry(gold):
    vals = {(b["i"], b["j"]): b for b in gold["bonds"]}
    for b in gold["bonds"]:
        assert abs(b["ss"] - 3 * b["zz"]) < 1e-12
    from oracle import model
    lad = model.Ladder(4, 4)
    xy = {k: v for v, k in lad.phys.items()}
    idx = lad.phys
    for (i, j), b in vals.items():
        (x1, y1), (x2, y2) = xy[i], xy[j]
        for m1, m2 in (((3 - x1, y1), (3 - x2, y2)), ((x1, 1 - y1), (x2, 1 - y2))):
            key = tuple(sorted((idx[m1], idx[m2])))
            assert abs(vals[key]["ss"] - b["ss"]) < 1e-12


def test_trotter_bias_is_small(gold):
    assert abs(gold["E_cluster_trotter"] - gold["E_cluster_ed"]) < 1e-3
    assert abs(gold["E_cluster_ed"] - sum(b["J"] * b["ss"] for b in gold["bonds"])) < 1e-12


def test_exact_values_regenerate(gold):
    now = make_golden.exact_values(with_trotter=False)
    assert abs(now["E_cluster_ed"] - gold["E_cluster_ed"]) < 1e-12
    assert abs(now["H_ed"] - gold["H_ed"]) < 1e-11
