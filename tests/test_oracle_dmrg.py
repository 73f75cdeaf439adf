"""Ground-state DMRG oracle (the reference Psi0 as a DMRG state): pinned to
the brute-force determinant Hamiltonian (literal Jordan-Wigner action on bit
strings, no MPS code) and to the variational principle."""
import numpy as np
import pytest

import synthetic
from oracle.brute import DetSpace, operator_matrix
from oracle.dmrg import GroundStateSweep, active_hamiltonian_terms, spin_squared_terms
from oracle.mps import expectation, overlap


def _sector_ground(h, L, k_act, n_elec):
    space = DetSpace.sector(k_act, n_elec, 0)
    H = operator_matrix(active_hamiltonian_terms(h, L, k_act), space)
    H = H.toarray() if hasattr(H, "toarray") else np.asarray(H)
    return float(np.linalg.eigvalsh(0.5 * (H + H.T))[0])


@pytest.fixture(scope="module")
def tiny():
    h, L, c = synthetic.config_integrals("tiny")
    return h, L, c["k_act"], c["n_elec"]


def test_exact_at_full_bond_dimension(tiny):
    """4 active orbitals: M = 16 = 4^2 holds every Schmidt state, so the sweep
    reaches the lowest (N, Sz = 0) eigenvalue of the brute-force H_act; the
    final MPS's <H_act> by MPO transfer is that value."""
    h, L, ka, n = tiny
    e_bf = _sector_ground(h, L, ka, n)
    gs = GroundStateSweep(h, L, ka, n, 16, keep_rel=1e-14)
    e = gs.run()
    assert abs(e - e_bf) < 1e-10, (e, e_bf)
    psi = gs.psi
    assert abs(expectation(psi, gs.W, psi) / overlap(psi, psi) - e_bf) < 1e-10


def test_truncated_runs_are_variational_and_monotone():
    """5 active orbitals, 4 electrons: energies at M = 2, 4, 6 lie above the
    brute-force ground energy and decrease with M; M = 16 (every Schmidt
    state) reaches it."""
    h, L = synthetic.integrals(11, 5, 0, 10)
    e_bf = _sector_ground(h, L, 5, 4)
    es = [GroundStateSweep(h, L, 5, 4, M, max_sweeps=12, keep_rel=1e-14).run() for M in (2, 4, 6, 16)]
    assert es[0] >= es[1] - 1e-10 and es[1] >= es[2] - 1e-10, es
    assert es[2] > e_bf + 1e-8, es              # M = 6 really truncates
    assert abs(es[3] - e_bf) < 1e-9, (es[3], e_bf)


def test_agrees_with_the_fci_singlet_of_the_synthetic_reference(tiny):
    """The synthetic reference (string-based FCI, independent code) picks the
    lowest singlet; on this draw it is the sector's lowest state, so the DMRG
    energy at full bond dimension equals it."""
    h, L, ka, n = tiny
    _, e_fci = synthetic.fci_reference(h, L, ka, n)
    assert abs(GroundStateSweep(h, L, ka, n, 16).run() - e_fci) < 1e-9


def _near_degenerate(seed=11, k=5, n=4):
    """Seeded draw with the one-body diagonal replaced by nearly degenerate
    frontier orbitals (0, 0.001 for the highest occupied pair, 1..2 above)
    and the off-diagonal scaled by 0.1: exchange then puts a triplet lowest."""
    h, L = synthetic.integrals(seed, k, 0, 10)
    h = 0.1 * (h - np.diag(np.diag(h)))
    occ = n // 2
    h = h + np.diag(np.r_[np.zeros(occ - 1), 0.0, 0.001, np.linspace(1, 2, k - occ - 1)])
    return h, L


def test_spin_penalty_selects_the_lowest_singlet():
    """With lam S^2 added, the sweep at full bond dimension reaches the lowest
    singlet; without it, the sector's lowest state.  Pin: brute-force H_act
    eigenvectors in the (N, Sz = 0) sector, each classified by <S^2> from the
    brute-force S- S+ matrix.  On this draw the lowest state is a triplet, so
    the penalty changes the answer."""
    h, L = _near_degenerate()
    space = DetSpace.sector(5, 4, 0)
    H = operator_matrix(active_hamiltonian_terms(h, L, 5), space)
    S2 = operator_matrix(spin_squared_terms(5, 1.0), space)
    H = H.toarray() if hasattr(H, "toarray") else np.asarray(H)
    S2 = S2.toarray() if hasattr(S2, "toarray") else np.asarray(S2)
    w, v = np.linalg.eigh(0.5 * (H + H.T))
    s2 = np.einsum("ij,ik,kj->j", v, S2, v)
    assert np.all(np.abs(s2 - np.round(s2)) < 1e-8)      # exact multiplets S(S+1)
    assert s2[0] > 1.5                                   # a triplet is lowest
    e_singlet = min(w[j] for j in range(len(w)) if abs(s2[j]) < 1e-8)
    e = GroundStateSweep(h, L, 5, 4, 16, keep_rel=1e-14, s2_penalty=1.0).run()
    assert abs(e - e_singlet) < 1e-9, (e, e_singlet)
    e0 = GroundStateSweep(h, L, 5, 4, 16, keep_rel=1e-14).run()
    assert abs(e0 - w[0]) < 1e-9, (e0, w[0])
