"""Brute-force collapse probabilities and detailed balance (tiny systems).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* ``joint_probabilities``: for a dense state, the probability of every
  environment outcome j, ||Pi_j psi||^2 with Pi_j = |j><j|_E (x) 1_C
  (Sec. I.C.2, Eq. detailbalance1), by direct enumeration.
* ``transition_matrix``: P_i and p(i -> j) for all environment states i, j of
  a tiny system, built from the dense Trotterised evolver; detailed balance
  (Sec. I.C.2) says P_i p(i -> j) is symmetric.
"""
import itertools

import numpy as np

from .model import D
from .ed import dense_evolve


def joint_probabilities(psi, ladder, basis_rows):
    """dict outcome-tuple -> ||Pi_j psi||^2 / ||psi||^2 over all env outcomes."""
    env = ladder.env
    norm = float(np.sum(psi * psi))
    out = {}
    for js in itertools.product(range(D), repeat=len(env)):
        phi = psi
        # contract environment legs from the highest index down so the
        # remaining leg positions stay valid
        for k, j in sorted(zip(env, js), reverse=True):
            phi = np.tensordot(phi, basis_rows[j], axes=([k], [0]))
        out[js] = float(np.sum(phi * phi)) / norm
    return out


def transition_matrix(ladder, n_steps, tau_eff, rows_in, rows_out):
    """(P, T): P_i = |e^{-beta H/2}|i>|B>|^2 (up to a constant), T_ij = p(i -> j).

    i runs over environment product states in the basis ``rows_in``, j over
    those in the basis ``rows_out``.
    """
    env_states = list(itertools.product(range(D), repeat=len(ladder.env)))
    P = np.zeros(len(env_states))
    T = np.zeros((len(env_states), len(env_states)))
    for a, i in enumerate(env_states):
        psi, nrm = dense_evolve(ladder, list(i), rows_in, n_steps, tau_eff)
        P[a] = nrm
        joint = joint_probabilities(psi, ladder, rows_out)
        for b, j in enumerate(env_states):
            T[a, b] = joint[j]
    return P, T
