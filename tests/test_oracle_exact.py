"""Pins of the exact (uncontracted) first-order quantities (Eqs. 1, 2, 5)."""
import numpy as np
import pytest

import synthetic
from oracle.brute import DetSpace, ExactFirstOrder, apply_terms, ci_to_dets, operator_matrix
from oracle.mp2 import mp2_closed_form
from oracle.mps import HylleraasSweep
from oracle.operators import Problem


def test_reference_is_lowest_singlet_eigenvector_of_h_act():
    h, L, c = synthetic.config_integrals("tiny")
    ci, e = synthetic.fci_reference(h, L, c["k_act"], c["n_elec"])
    p = Problem(h, L, c["k_act"], c["n_elec"], ci, h0="dyall")
    space = DetSpace.sector(c["k_act"], c["n_elec"], 0)
    d, v = ci_to_dets(ci, c["k_act"])
    psi = np.zeros(len(space))
    psi[space.index(d)] = v
    hp = apply_terms(p.h_act_terms(), space, psi, space)
    assert np.linalg.norm(hp - e * psi) < 1e-10
    assert abs(p.E_ref - e) < 1e-12
    assert p.E1 == 0.0          # Dyall: E1 = 0 exactly with no core


def test_mp2_closed_form_single_determinant():
    """Fock H0 + closed-shell determinant: Hylleraas minimum == MP2 (with singles)."""
    h, L = synthetic.integrals(11, 2, 6, 10)
    ci, _ = synthetic.fci_reference(h, L, 2, 4)
    assert np.count_nonzero(ci) == 1
    p = Problem(h, L, 2, 4, ci, h0="fock")
    ex = ExactFirstOrder(p)
    ref = mp2_closed_form(h, L, 2)
    assert abs(ex.e2() - ref) < 1e-12
    sw = HylleraasSweep(p, max(ex.schmidt_ranks()))
    assert abs(sw.run() - ref) < 1e-10


@pytest.mark.parametrize("h0", ["fock", "dyall"])
def test_perturbation_series_coefficients(h0):
    """E(lam) of H0 + lam V on span{Psi0} + X has Taylor coefficients
    E0, E1, E2*, E3* (Rayleigh-Schroedinger; E3 by Wigner's 2n+1 rule)."""
    h, L = synthetic.integrals(3, 3, 3, 8)
    ci, _ = synthetic.fci_reference(h, L, 3, 4)
    p = Problem(h, L, 3, 4, ci, h0=h0)
    ex = ExactFirstOrder(p)
    Hx = operator_matrix(p.hamiltonian_terms(), ex.X).toarray()
    n = len(ex.X) + 1
    H = np.zeros((n, n))
    H[0, 0] = p.E_ref
    H[1:, 0] = H[0, 1:] = ex.g
    H[1:, 1:] = Hx
    H0 = np.zeros((n, n))
    H0[0, 0] = p.E0
    H0[1:, 1:] = ex.A.toarray() + p.E0 * np.eye(n - 1)
    V = H - H0
    lams = np.arange(-4, 5) * 0.02
    E = [np.linalg.eigvalsh(H0 + lam * V)[0] for lam in lams]
    coef = np.polynomial.polynomial.polyfit(lams, E, 8)
    assert abs(coef[0] - p.E0) < 1e-10
    assert abs(coef[1] - p.E1) < 1e-9
    assert abs(coef[2] - ex.e2()) < 1e-8
    assert abs(coef[3] - ex.e3()) < 1e-6


def test_e2_invariant_under_virtual_rotation():
    h, L = synthetic.integrals(5, 3, 4, 8)
    ci, _ = synthetic.fci_reference(h, L, 3, 4)
    e = ExactFirstOrder(Problem(h, L, 3, 4, ci, h0="fock")).e2()
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.normal(size=(4, 4)))
    C = np.eye(7)
    C[3:, 3:] = Q
    h2 = C.T @ h @ C
    L2 = np.einsum("pi,Qpq,qj->Qij", C, L, C)
    e2 = ExactFirstOrder(Problem(h2, L2, 3, 4, ci, h0="fock")).e2()
    assert abs(e - e2) < 1e-12


@pytest.mark.parametrize("h0", ["fock", "dyall"])
def test_hylleraas_functional_is_the_quadratic_with_minimum_e2(h0):
    """Eq. 1 on X is J(x) = x^T A x + 2 x^T g with A = H0 - E0 symmetric:
    J(x* + d) - J(x*) = d^T A d exactly, J(x*) = g^T x* = E2*, and (A > 0)
    J(x) >= E2* for every x."""
    h, L = synthetic.integrals(3, 3, 3, 8)
    ci, _ = synthetic.fci_reference(h, L, 3, 4)
    ex = ExactFirstOrder(Problem(h, L, 3, 4, ci, h0=h0))
    A = ex.A.toarray()
    assert np.abs(A - A.T).max() < 1e-14
    lam = np.linalg.eigvalsh(A)
    assert lam.min() > 0.0
    e2 = ex.e2()
    xs = ex.psi1
    assert abs(ex.hylleraas(xs) - e2) < 1e-12
    assert np.linalg.norm(A @ xs + ex.g) < 1e-10 * np.linalg.norm(ex.g)
    rng = np.random.default_rng(11)
    for _ in range(5):
        d = rng.normal(size=xs.shape) * 0.1
        dJ = ex.hylleraas(xs + d) - e2
        assert abs(dJ - d @ (A @ d)) < 1e-10 * max(1.0, abs(dJ))
        assert dJ > 0.0
        x = rng.normal(size=xs.shape)
        assert ex.hylleraas(x) >= e2


def test_preprocessing_invariants():
    """Reading R5 and the active 1-RDM: gamma is symmetric with trace N and
    occupations in [0, 2]; the semicanonical rotation is orthogonal, acts on
    the virtual block only, makes f_vv diagonal in ascending order, and gives
    every virtual orbital a positive largest-magnitude coefficient."""
    h, L = synthetic.integrals(5, 3, 4, 8)
    ci, _ = synthetic.fci_reference(h, L, 3, 4)
    p = Problem(h, L, 3, 4, ci, h0="fock")
    g = p.gamma
    assert np.abs(g - g.T).max() < 1e-13
    assert abs(np.trace(g) - 4) < 1e-12
    occ = np.linalg.eigvalsh(g)
    assert occ.min() > -1e-12 and occ.max() < 2 + 1e-12
    C = p.rotation
    assert np.abs(C.T @ C - np.eye(7)).max() < 1e-13
    assert np.array_equal(C[:3, :3], np.eye(3)) and not C[:3, 3:].any() and not C[3:, :3].any()
    fv = p.f[3:, 3:]
    assert np.abs(fv - np.diag(np.diag(fv))).max() < 1e-12
    assert np.all(np.diff(np.diag(fv)) >= 0)
    U = C[3:, 3:]
    for j in range(4):
        assert U[int(np.argmax(np.abs(U[:, j]))), j] > 0
    # the integrals are those of the rotated orbitals
    assert np.abs(p.h - C.T @ h @ C).max() < 1e-13
