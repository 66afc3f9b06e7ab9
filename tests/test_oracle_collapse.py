"""Pins of oracle/collapse.py and oracle/brute.py.

* Philox4x32-10 against a library implementation of the same generator:
  cuRAND's host-side CURAND_RNG_PSEUDO_PHILOX4_32_10, whose output stream for
  seed s is the blocks philox4x32_10((0, 0, j, 0), (s mod 2^32, s >> 32)),
  j = 0, 1, ...  This covers the round function, multipliers, key schedule
  and round count for keys with every bit pattern tried.  Counter words 0, 1
  and 3, which that stream leaves at zero, must each change the output;
* collapse: the product of the sequential conditional probabilities equals the
  brute-force joint probability ||Pi_j psi||^2 of every outcome (Sec. I.C.2);
* detailed balance P_i p(i->j) = P_j p(j->i) and stationarity across a change
  of measurement basis, by brute force on a tiny ladder (Sec. I.C.2).
"""
import ctypes
import ctypes.util
import glob
import itertools
import math
import os

import numpy as np
import pytest

from oracle import brute, collapse, ed, model, mps

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161      # curandRngType_t of cuRAND's public header


def _curand():
    """cuRAND from the CUDA toolkit (host generator only; no GPU needed)."""
    paths = sorted(glob.glob(os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib*", "libcurand.so*")))
    name = ctypes.util.find_library("curand")
    for path in paths + ([name] if name else []):
        try:
            return ctypes.CDLL(path)
        except OSError:
            continue
    pytest.skip("cuRAND not found")


def _curand_stream(lib, seed, n_blocks):
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        buf = (ctypes.c_uint32 * (4 * n_blocks))()
        assert lib.curandGenerate(gen, buf, ctypes.c_size_t(4 * n_blocks)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return [tuple(buf[4 * j:4 * j + 4]) for j in range(n_blocks)]


@pytest.mark.parametrize("seed", [0, 1, 0x0123456789ABCDEF, 0xFEDCBA9876543210, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_the_curand_host_generator(seed):
    lib = _curand()
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for j, block in enumerate(_curand_stream(lib, seed, 300)):
        assert collapse.philox4x32_10((0, 0, j, 0), key) == block, j


def test_philox_uses_every_counter_word():
    key = (0x9E3779B9, 0x7F4A7C15)
    outs = {}
    for c in itertools.product((0, 1, 0xFFFFFFFF), repeat=4):
        outs[c] = collapse.philox4x32_10(c, key)
    assert len(set(outs.values())) == len(outs)               # a bijection of the counter
    base = outs[(0, 0, 0, 0)]
    for w in range(4):
        c = [0, 0, 0, 0]
        c[w] = 1
        x = np.array(outs[tuple(c)], dtype=np.uint64) ^ np.array(base, dtype=np.uint64)
        # one flipped input bit changes about half of the 128 output bits
        assert 40 < sum(bin(int(v)).count("1") for v in x) < 88, w


def test_uniform_range_and_moments():
    u = np.array([collapse.uniform(7, 3, n, e) for n in range(40) for e in range(50)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.02 and abs(u.var() - 1 / 12) < 0.01


def test_choose_rule():
    p = [0.2, 0.0, 0.8]
    assert collapse.choose(p, 0.0) == 0
    assert collapse.choose(p, 0.1999) == 0
    assert collapse.choose(p, 0.2) == 2
    assert collapse.choose([0.5, 0.5, 0.0], 1.0) == 1   # rounding overflow -> last p>0


def test_x_basis_is_sx_eigenbasis():
    sz, sp, sm = model.spin1_operators()
    sx = 0.5 * (sp + sm)
    rows = collapse.basis_matrix(collapse.BASIS_X)
    assert np.allclose(rows @ rows.T, np.eye(3), atol=1e-15)
    for r, m in zip(rows, (1.0, 0.0, -1.0)):
        assert np.allclose(sx @ r, m * r, atol=1e-15)


def _evolved(Lx, two_W, beta, basis_in, seed=2):
    lad = model.Ladder(Lx, two_W, 1.0, 0.8)
    n, teff = model.trotter_steps(beta, 0.1)
    env = collapse.initial_env(len(lad.env), seed, 0)
    st = mps.MPS(collapse.product_state(lad, env, basis_in))
    mps.evolve(st, model.plan_ops(lad, n), model.gate_table(lad, teff), 3 ** lad.n_sites, 0.0)
    return lad, st


@pytest.mark.parametrize("Lx,two_W,basis", [(3, 2, collapse.BASIS_Z), (3, 2, collapse.BASIS_X),
                                             (2, 0, collapse.BASIS_X), (3, 4, collapse.BASIS_Z)])
def test_collapse_conditionals_match_brute_force(Lx, two_W, basis):
    lad, st = _evolved(Lx, two_W, 0.8, collapse.BASIS_Z)
    rows = collapse.basis_matrix(basis)
    joint = brute.joint_probabilities(st.to_dense().reshape((3,) * lad.n_sites), lad, rows)
    assert abs(sum(joint.values()) - 1.0) < 1e-12
    for js in itertools.product(range(3), repeat=len(lad.env)):
        _, logp, conds = collapse.collapse(st, lad, basis, 0, 0, 0, forced=list(js))
        prod = math.prod(c[j] for c, j in zip(conds, js))
        assert abs(prod - joint[js]) < 1e-12


def test_collapse_sampling_uses_the_rng_stream():
    lad, st = _evolved(3, 2, 0.8, collapse.BASIS_Z)
    out, logp, conds = collapse.collapse(st, lad, collapse.BASIS_Z, 11, 4, 9)
    for e, (b, p) in enumerate(zip(out, conds)):
        assert b == collapse.choose(p, collapse.uniform(11, 4, 9, e))
    assert abs(logp - sum(math.log(c[b]) for c, b in zip(conds, out))) < 1e-14


def test_detailed_balance_same_basis():
    lad = model.Ladder(2, 2, 1.0, 0.6)
    n, teff = model.trotter_steps(1.0, 0.1)
    z = collapse.basis_matrix(collapse.BASIS_Z)
    P, T = brute.transition_matrix(lad, n, teff, z, z)
    assert np.allclose(T.sum(axis=1), 1.0, atol=1e-12)
    flux = P[:, None] * T
    assert np.abs(flux - flux.T).max() < 1e-12 * flux.max()


def test_stationarity_across_basis_change():
    # collapsing in x maps the z-basis weights P^z onto the x-basis weights P^x
    lad = model.Ladder(2, 2, 1.0, 0.6)
    n, teff = model.trotter_steps(1.0, 0.1)
    z = collapse.basis_matrix(collapse.BASIS_Z)
    x = collapse.basis_matrix(collapse.BASIS_X)
    Pz, Tzx = brute.transition_matrix(lad, n, teff, z, x)
    Px, _ = brute.transition_matrix(lad, n, teff, x, x)
    assert np.allclose(Pz @ Tzx, Px, rtol=1e-11, atol=0)


def test_initial_env_draws():
    out = collapse.initial_env(6, 5, 2)
    third = 1.0 / 3.0
    assert out == [collapse.choose([third] * 3, collapse.uniform(5, 2, -1, e)) for e in range(6)]
    assert set(out) <= {0, 1, 2}


def test_product_state_norm_and_canonical_form():
    lad = model.Ladder(4, 4)
    ts = collapse.product_state(lad, [0, 1, 2, 0], collapse.BASIS_X)
    st = mps.MPS(ts)
    assert abs(np.linalg.norm(st.to_dense()) - 1.0) < 1e-14
    for t in ts:
        m = t.reshape(t.shape[0], -1)
        assert np.allclose(m @ m.T, np.eye(t.shape[0]), atol=1e-15)
    _ = ed  # dense helpers are pinned in test_oracle_ed
