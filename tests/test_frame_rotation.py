"""The S^x-basis frame of the GPU path, pinned on the oracle (CPU).

An S^x-basis sample is evolved in charge blocks by storing it rotated by R,
the matrix whose rows are the S^x eigenvectors.  That rests on facts of the
spin-1 algebra and of the Heisenberg ladder (Eq. H is SU(2) invariant), each
checked here independently of the CUDA code:
* R is real, symmetric and its own inverse, R S^z R = S^x, R e_b = v_b;
* every bond gate exp(-(tau/2) J S_i.S_j) commutes with R (x) R, and the
  Bell pair sum_s |s s> (Sec. I.C) is invariant under it;
* so evolving the S^x-product state equals rotating, evolving the S^z-product
  state with the same outcome indices, and rotating back (dense vectors, no
  truncation), and the energy and <Sx Sx> of one are <Sz Sz> of the other;
* for a state of definite total S^z, <Sx_i Sx_j> = (<S+_i S-_j> + <S-_i S+_j>)/4.
"""
import numpy as np

from oracle import chain, collapse, model
from oracle import mps as omps

R = collapse.basis_matrix(collapse.BASIS_X)


def _ops():
    r2 = np.sqrt(2.0)
    sz = np.diag([1.0, 0.0, -1.0])
    sp = np.array([[0, r2, 0], [0, 0, r2], [0, 0, 0]])
    return sz, sp, sp.T


def test_rotation_exchanges_sx_and_sz():
    sz, sp, sm = _ops()
    sx = 0.5 * (sp + sm)
    assert np.allclose(R, R.T, atol=1e-15)
    assert np.allclose(R @ R, np.eye(3), atol=1e-15)
    assert np.allclose(R @ sz @ R, sx, atol=1e-15)
    assert np.allclose(R @ sx @ R, sz, atol=1e-15)
    for b in range(3):                       # R maps the S^z basis to the S^x basis
        assert np.allclose(R @ np.eye(3)[b], R[b], atol=1e-15)


def test_gates_and_bell_pairs_are_invariant():
    rr = np.kron(R, R)
    for coef in (0.025, 0.05, -0.3, 1.7):
        g = model.bond_gate(coef)
        assert np.abs(rr @ g @ rr - g).max() < 1e-13 * np.abs(g).max()
    sw = model.swap_gate()
    assert np.allclose(rr @ sw @ rr, sw, atol=1e-15)
    bell = np.eye(3).reshape(-1)
    assert np.allclose(rr @ bell, bell, atol=1e-15)


def _rotate(tensors):
    return [np.einsum("st,ltr->lsr", R, t) for t in tensors]


def test_rotated_sx_sample_equals_sz_sample():
    """Lx=3, 2W=2, beta=0.6: no truncation (chi 729), dense vectors at 1e-12."""
    cfg = dict(Lx=3, two_W=2, J_leg=1.0, J_rung=0.7, beta=0.6, tau=0.1, chi_max=729, cutoff=0.0)
    ch = chain.HybridChain(seed=1, chain_id=0, **cfg)
    env = [0, 2, 1, 0]
    x_state = omps.MPS(collapse.product_state(ch.ladder, env, collapse.BASIS_X), 0)
    z_state = omps.MPS(collapse.product_state(ch.ladder, env, collapse.BASIS_Z), 0)
    assert np.allclose(omps.MPS(_rotate(x_state.tensors)).to_dense(), z_state.to_dense(), atol=1e-15)
    x_ev = omps.evolve(x_state, ch.ops, ch.gates, 729, 0.0)
    z_ev = omps.evolve(z_state, ch.ops, ch.gates, 729, 0.0)
    a = omps.MPS(_rotate(x_ev.tensors)).to_dense()
    b = z_ev.to_dense()
    assert np.abs(a - np.sign(a @ b) * b).max() < 1e-12


def test_sx_sx_from_raising_and_lowering_at_definite_sz():
    """A random state of total S^z = 0 on three spin-1 sites: <Sx_0 Sx_2> equals
    (<S+_0 S-_2> + <S-_0 S+_2>)/4, and <S+_0 S+_2> vanishes."""
    sz, sp, sm = _ops()
    sx = 0.5 * (sp + sm)
    rng = np.random.default_rng(3)
    m = np.array([1, 0, -1])
    tot = (m[:, None, None] + m[None, :, None] + m[None, None, :]).reshape(-1)
    psi = rng.standard_normal(27) * (tot == 0)
    psi /= np.linalg.norm(psi)

    def ev(a, b):
        op = np.kron(np.kron(a, np.eye(3)), b)
        return psi @ op @ psi

    assert abs(ev(sx, sx) - 0.25 * (ev(sp, sm) + ev(sm, sp))) < 1e-14
    assert abs(ev(sp, sp)) < 1e-14
