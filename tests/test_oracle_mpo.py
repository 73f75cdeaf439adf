"""Oracle MPO (Eq. 4) == brute-force determinant operator on small chains.

The brute force applies each elementary operator to bit strings with the
Jordan-Wigner sign taken literally, so any error in the site factors, the
parity strings, the prefix/suffix sharing or the centre coefficients shows
up as a mismatch in some (N, Sz) sector."""
import numpy as np
import pytest

import synthetic
from oracle.brute import DetSpace, dets_to_site_index, operator_matrix
from oracle.mpo import build_mpo
from oracle.operators import Problem


def _problem(h0):
    h, L = synthetic.integrals(7, 2, 3, 5)
    ci, _ = synthetic.fci_reference(h, L, 2, 2)
    return Problem(h, L, 2, 2, ci, h0=h0)


def _max_err(terms, prob):
    mpo = build_mpo(terms, prob.k, k_split=prob.k_act)
    dense = mpo.to_dense()
    err = 0.0
    for N in range(2 * prob.k + 1):
        for sz in range(-N, N + 1, 2):
            S = DetSpace.sector(prob.k, N, sz)
            if len(S) == 0:
                continue
            B = operator_matrix(terms, S).toarray()
            idx = dets_to_site_index(S.dets, prob.k)
            err = max(err, float(np.abs(dense[np.ix_(idx, idx)] - B).max()))
    # nothing outside the N/Sz-conserving blocks
    return err, mpo


@pytest.mark.parametrize("h0", ["fock", "dyall"])
def test_h0_mpo_matches_brute_force(h0):
    p = _problem(h0)
    err, mpo = _max_err(p.h0_terms(), p)
    assert err < 1e-12
    # the virtual region carries only "identity" and "complete" states
    assert max(mpo.dims[p.k_act + 1:-1]) == 2


def test_rhs_mpo_matches_brute_force():
    p = _problem("fock")
    err, _ = _max_err(p.rhs_terms(), p)
    assert err < 1e-12


def test_full_hamiltonian_mpo_matches_brute_force():
    p = _problem("fock")
    err, _ = _max_err(p.hamiltonian_terms(), p)
    assert err < 1e-12


def test_planted_sign_error_is_caught():
    """Dropping the Jordan-Wigner parity on pass-through sites must fail."""
    import oracle.mpo as m
    p = _problem("fock")
    saved = m.PARITY
    try:
        m.PARITY = m.IDENT
        err, _ = _max_err(p.rhs_terms(), p)
    finally:
        m.PARITY = saved
    assert err > 1e-3
