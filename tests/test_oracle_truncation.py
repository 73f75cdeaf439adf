"""The renormalisation step of the oracle sweep: state selection by reading
R7 (M largest density-matrix eigenvalues above 1e-10 tr rho, a tied group at
the cut dropped whole) and the split of a two-site tensor, checked against
the Eckart-Young identity: the squared error of the kept projection equals
the discarded eigenvalue sum exactly."""
import numpy as np
import pytest

import synthetic
from oracle.mps import HylleraasSweep, select_states, truncate
from oracle.operators import Problem


def _kept(evals, M):
    kept, disc = select_states(evals, M, sum(float(np.sum(l)) for _, l in evals))
    return sorted(kept), disc


def test_select_keeps_the_m_largest_above_the_threshold():
    ev = [((3, 1), np.array([0.5, 0.2, 1e-15])), ((3, -1), np.array([0.25, 0.05]))]
    tr = 0.5 + 0.2 + 1e-15 + 0.25 + 0.05
    kept, disc = _kept(ev, 3)
    assert kept == [((3, -1), 0), ((3, 1), 0), ((3, 1), 1)]
    assert disc == pytest.approx((0.05 + 1e-15) / tr, rel=1e-12)
    # M above the number of states: everything above 1e-10 tr rho, nothing else
    kept, disc = _kept(ev, 10)
    assert len(kept) == 4 and ((3, 1), 2) not in kept
    assert disc == pytest.approx(1e-15 / tr, rel=1e-6)


def test_select_drops_a_tied_group_at_the_cut():
    ev = [((2, 0), np.array([0.4, 0.2])), ((2, 2), np.array([0.2])), ((2, -2), np.array([0.2 * (1 + 1e-10)]))]
    kept, _ = _kept(ev, 2)
    assert kept == [((2, 0), 0)]              # the three-fold 0.2 group straddles the cut
    kept, _ = _kept(ev, 4)
    assert len(kept) == 4                      # cut below the group: all kept
    # a group with nothing above it is kept up to M instead of emptied
    ev = [((1, 1), np.array([0.3])), ((1, -1), np.array([0.3]))]
    kept, _ = _kept(ev, 1)
    assert len(kept) == 1


@pytest.mark.parametrize("direction", ["LR", "RL"])
def test_split_error_equals_discarded_weight(direction):
    h, L = synthetic.integrals(7, 3, 2, 5)
    ci, _ = synthetic.fci_reference(h, L, 3, 4)
    p = Problem(h, L, 3, 4, ci, h0="fock")
    sw = HylleraasSweep(p, 16, seed=9)
    rng = np.random.default_rng(4)
    for i in range(p.k - 1):                    # left to right, so every environment exists
        x0, _, _, _, mask = sw.local_problem(i)
        x = rng.normal(size=x0.shape) * mask    # respects the bond QN labels and the X filter
        ps = sw.psi1
        for M in (1, 2, 4, 64):
            Al, Ar, lab, w = truncate(x, ps.q[i], ps.q[i + 2], M, direction, sw.allowed.get(i + 1))
            Dn = Al.shape[2]
            assert Dn <= M and lab.shape == (Dn, 2)
            rec = np.einsum("lsm,mtr->lstr", Al, Ar)
            err = np.sum((x - rec) ** 2) / np.sum(x ** 2)
            assert abs(err - w) < 1e-12, (i, M, err, w)
            # and what is dropped is the smallest part of the spectrum of the dense rho
            X = x.reshape(x.shape[0] * 4, -1)
            lam = np.sort(np.linalg.eigvalsh(X @ X.T if direction == "LR" else X.T @ X))[::-1]
            if Dn == M:
                assert abs(w * np.sum(x ** 2) - np.sum(lam[M:])) < 1e-12 * np.sum(x ** 2), (i, M)
            # the kept basis is orthonormal on its side of the bond
            if direction == "LR":
                U = Al.reshape(-1, Dn)
            else:
                U = Ar.reshape(Dn, -1).T
            assert np.abs(U.T @ U - np.eye(Dn)).max() < 1e-12
            # every kept vector carries one QN: rows of other sectors are zero
            rowq = ((ps.q[i][:, None, :] + np.array([[0, 0], [1, 1], [1, -1], [2, 0]])[None]).reshape(-1, 2)
                    if direction == "LR" else
                    (ps.q[i + 2][None, :, :] - np.array([[0, 0], [1, 1], [1, -1], [2, 0]])[:, None, :]).reshape(-1, 2))
            for n in range(Dn):
                off = np.any(rowq != lab[n], axis=1)
                assert np.abs(U[off, n]).max(initial=0.0) == 0.0
        sw.step(i, "LR")
