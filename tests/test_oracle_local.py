"""The oracle's local operators at a bond (Fig. 1C: the two-site sigma,
right-hand side and diagonal built from renormalised environments) equal the
brute-force operators projected on the two-site space of the MPS:
A_loc = Phi^T (H0 - E0) Phi and g = Phi^T V Psi0, with Phi the orthonormal
embedding given by the left- and right-canonical sites.  The determinant
operators apply each elementary operator to bit strings (no MPO), and Psi0 is
the CI vector placed on the empty virtual sites, so neither side shares the
oracle's MPS code.

A transposed environment block, a dropped or sign-flipped MPO term in sigma,
or a transposed block inside a transfer each fail this test.  The systems
have three and four active sites, so active sites also enter the right
environments and their transfers; virtual sites alone give diagonal H0
blocks (sum_a eps_a n_a), where a transposition cannot show."""
import numpy as np
import pytest

import synthetic
from oracle.brute import DetSpace, dets_to_site_index, operator_matrix
from oracle.mps import HylleraasSweep
from oracle.operators import Problem


def _dense_operator(terms, k):
    H = np.zeros((4 ** k, 4 ** k))
    for N in range(2 * k + 1):
        for sz in range(-N, N + 1, 2):
            S = DetSpace.sector(k, N, sz)
            if len(S) == 0:
                continue
            idx = dets_to_site_index(S.dets, k)
            H[np.ix_(idx, idx)] = operator_matrix(terms, S).toarray()
    return H


def _embedding(mps, i):
    k = mps.nsite
    Lb = np.ones((1, 1))
    for c in range(i):
        Lb = np.einsum("xl,lsr->xsr", Lb, mps.A[c]).reshape(-1, mps.A[c].shape[2])
    Rb = np.ones((1, 1))
    for c in range(k - 1, i + 1, -1):
        Rb = np.einsum("lsr,rx->lsx", mps.A[c], Rb).reshape(mps.A[c].shape[0], -1)
    return np.kron(np.kron(Lb, np.eye(16)), Rb.T)


@pytest.mark.parametrize("k_act,k_virt", [(3, 2), (4, 1)])
@pytest.mark.parametrize("h0", ["fock", "dyall"])
def test_local_operators_equal_projected_brute_force(h0, k_act, k_virt):
    h, L = synthetic.integrals(7, k_act, k_virt, 5)
    ci, _ = synthetic.fci_reference(h, L, k_act, 4)
    p = Problem(h, L, k_act, 4, ci, h0=h0)
    k = p.k
    Hd = _dense_operator(p.h0_terms(), k)
    Vd = _dense_operator(p.rhs_terms(), k)
    psi0 = np.kron(ci, np.eye(4 ** p.k_virt)[0])       # virtual sites empty
    sw = HylleraasSweep(p, 4, seed=5)
    rng = np.random.default_rng(2)
    checked = 0
    order = [(i, "LR") for i in range(k - 1)] + [(i, "RL") for i in range(k - 2, -1, -1)]
    for i, direction in order:                           # one full sweep; every bond twice
        x0, g, apply, diag, mask = sw.local_problem(i)
        Phi = _embedding(sw.psi1, i)
        assert np.abs(Phi.T @ Phi - np.eye(Phi.shape[1])).max() < 1e-12
        Aloc = Phi.T @ Hd @ Phi
        m = mask.ravel().astype(bool)
        x = rng.normal(size=x0.shape) * mask
        got = (apply(x) * mask).ravel()[m]
        want = (Aloc @ x.ravel())[m]
        assert np.abs(got - want).max() < 1e-11 * max(1.0, np.abs(want).max()), i
        assert np.abs(g.ravel()[m] - (Phi.T @ (Vd @ psi0))[m]).max() < 1e-12, i
        assert np.abs(diag.ravel()[m] - np.diag(Aloc)[m]).max() < 1e-11, i
        checked += int(m.sum() > 0)
        sw.step(i, direction)
    assert checked >= 2 * (k - 2)


@pytest.mark.parametrize("h0", ["fock", "dyall"])
def test_third_order_transfer_equals_dense_formula_at_truncating_m(h0):
    """Eq. 5 by MPO transfers on a truncated Psi1 (M = 4) equals the same
    formula on the dense Psi1 with brute-force operators:
    E3 = <H> - <H0 - E0> - (E0 + E1) <1>."""
    from oracle.mps import third_order
    h, L = synthetic.integrals(7, 3, 2, 5)
    ci, _ = synthetic.fci_reference(h, L, 3, 4)
    p = Problem(h, L, 3, 4, ci, h0=h0)
    sw = HylleraasSweep(p, 4, seed=5, max_sweeps=2)
    sw.run()
    psi = sw.psi1.to_dense()
    Hd = _dense_operator(p.hamiltonian_terms(), p.k)
    Ad = _dense_operator(p.h0_terms(), p.k)
    want = psi @ Hd @ psi - psi @ Ad @ psi - (p.E0 + p.E1) * (psi @ psi)
    assert abs(third_order(sw) - want) < 1e-12 * max(1.0, abs(want))
    assert abs(psi @ psi - 1.0) > 1e-6          # Psi1 is not normalised: the <1> term matters
