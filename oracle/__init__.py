"""CPU oracle for MPS-PT (Sharma & Chan, "A flexible multi-reference
perturbation theory by minimizing the Hylleraas functional with matrix
product states").

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, float64 NumPy
restatement of the method, written to be checked against the paper by eye.
It is imported only by ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The GPU
library never imports it, and it never imports the GPU library; the two
share only the seeded inputs of ``synthetic/``.

Modules
  fermion    local site basis, Jordan-Wigner conventions, QN labels
  operators  integral preprocessing (Eq. 1 inputs) and second-quantised
             term lists for H, H0 (Fock / Dyall) and the RHS part of V
  brute      determinant-space operators, exact (uncontracted) E2 / E3
  mpo        matrix product operators (Eq. 4) built from term lists
  mps        QN-labelled MPS (Eq. 3) and the two-site Hylleraas sweep
  mp2        closed-form MP2 (pin for the single-determinant limit)

Parity status: every function is pinned by a test in ``tests/`` against a
value the mathematics fixes (brute force, closed form, invariants); see the
module headers.
"""
