"""FP64 CPU oracle for the hybrid purification-METTS sampler (arXiv:1910.09142).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link
or execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` use it.  It shares no code with
the CUDA library (``paper_1910_09142_gb300``) and imports nothing from it.

Contents (each function cites the passage of the paper it follows):

* ``model``    spin-1 operators, the two-leg ladder Hamiltonian (Sec. II, Eq. H),
               the cluster/environment site map (Sec. I.C, Fig. 4), Trotter gates
               and the swap-gate op schedule (Sec. I.A, Sec. II "Trotter-Suzuki").
* ``mps``      the MPS state, two-site gate application with truncated SVD
               (Sec. II, truncation error), exact centre moves (QR / LQ).
* ``measure``  cluster observables <<A>>_n (Sec. I.C.1 step 3, Sec. II.A).
* ``collapse`` Philox4x32-10 counter RNG, projective collapse of the environment
               and the Bell-pair reset (Sec. I.C.1 step 4, Eq. detailbalance1).
* ``chain``    the hybrid Markov chain, steps 1-4 of Sec. I.C.1.
* ``ed``       exact diagonalisation by S^z sectors, thermal averages
               (Eq. sqrtrho) and a dense Trotterised state-vector evolver.
* ``brute``    brute-force collapse enumeration and detailed balance
               (Sec. I.C.2) on tiny systems.
* ``u1``       total-S^z block-sparse evolution with S^z-basis collapses
               (Sec. II.C, Fig. qn).

Pins: every function here is checked by ``tests/test_oracle_*.py`` against
closed forms, exact diagonalisation, library routines or brute force; see the
header of each module for which pin covers it.
"""
