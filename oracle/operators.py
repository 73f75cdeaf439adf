"""Integral preprocessing and operator term lists (Eq. 1 ingredients).

Hamiltonian (no core, no nuclear term):
  H = sum_pq h_pq sum_s c+_ps c_qs
      + 1/2 sum_pqrs (pq|rs) sum_st c+_ps c+_rt c_st c_qs.
Zeroth-order Hamiltonians on the first-order space X (1-2 virtual electrons):
  Dyall:  H0 = H_act + sum_a eps_a n_a,  E0 = <Psi0|H_act|Psi0>, E1 = 0;
  Fock:   H0 = sum_tu f_tu E_tu + sum_a eps_a n_a,  E0 = sum_tu f_tu gamma_tu,
          E1 = E_ref - E0  (generalised Fock with the active-virtual block
          projected out, the "one-body Fock operator times many-body
          projectors" of the CASPT2-like choice).
  f_pq = h_pq + sum_tu gamma_tu [(pq|tu) - 1/2 (pu|tq)];  eps_a from
  diagonalising f_vv (semicanonical virtuals, ascending; each orbital's sign
  fixed by making its largest-magnitude coefficient positive).
RHS: since Psi0 has no virtual electrons and Psi1 lies in X (Q = 1 there),
  -Q V Psi0 = -P_X H Psi0, i.e. only the terms of H with at least one virtual
  creator and no virtual annihilator contribute (the "<= 2 external indices"
  restriction of the cost analysis).

Pinned by: MP2 closed form (single determinant, Fock H0), E1 = 0 for Dyall,
Psi0 being an eigenvector of H_act (tests/test_oracle_exact.py).
"""
import numpy as np

from .brute import DetSpace, apply_terms, ci_to_dets


def eri_from_cholesky(L):
    return np.einsum("Qpq,Qrs->pqrs", L, L, optimize=True)


def one_body_terms(t, P, Q):
    """sum_{p in P, q in Q} t_pq sum_s c+_ps c_qs."""
    out = []
    for p in P:
        for q in Q:
            v = float(t[p, q])
            if v == 0.0:
                continue
            for s in (0, 1):
                out.append((v, ((2 * p + s, True), (2 * q + s, False))))
    return out


def two_body_terms(eri, P, Q, R, S, keep=None):
    """1/2 sum (pq|rs) sum_st c+_ps c+_rt c_st c_qs over the given index sets.

    When the (p,q) and (r,s) index sets coincide, the two equal halves
    c+_ps c+_rt c_st c_qs = c+_rt c+_ps c_qs c_st are merged: one term with
    coefficient (pq|rs) per unordered pair of (orbital, orbital, spin)."""
    P, Q, R, S = list(P), list(Q), list(R), list(S)
    sym = P == R and Q == S
    out = []
    for p in P:
        for q in Q:
            for r in R:
                for s in S:
                    if keep is not None and not keep(p, q, r, s):
                        continue
                    v = 0.5 * float(eri[p, q, r, s])
                    if v == 0.0:
                        continue
                    for a in (0, 1):
                        for b in (0, 1):
                            if a == b and (p == r or q == s):
                                continue
                            if sym:
                                k1, k2 = (p, q, a), (r, s, b)
                                if k1 > k2:
                                    continue
                                c = 2.0 * v if k1 < k2 else v
                            else:
                                c = v
                            out.append((c, ((2 * p + a, True), (2 * r + b, True),
                                            (2 * s + b, False), (2 * q + a, False))))
    return out


def number_terms(eps, orbitals):
    out = []
    for a in orbitals:
        v = float(eps[a])
        if v == 0.0:
            continue
        for s in (0, 1):
            out.append((v, ((2 * a + s, True), (2 * a + s, False))))
    return out


def active_expectation(terms, ci, k_act, n_elec):
    space = DetSpace.sector(k_act, n_elec, 0)
    d, c = ci_to_dets(ci, k_act)
    psi = np.zeros(len(space))
    idx = space.index(d)
    if np.any(idx < 0):
        raise ValueError("reference outside the (N, Sz=0) active sector")
    psi[idx] = c
    return float(psi @ apply_terms(terms, space, psi, space))


class Problem:
    """Preprocessed MPS-PT problem (paper Eqs. 1-2, 5 inputs).

    h, L: integrals in the original basis; ci: active CI vector of Psi0;
    h0: 'fock' or 'dyall'.  After construction the integrals are expressed
    in the semicanonical virtual basis (active orbitals untouched).
    """

    def __init__(self, h, L, k_act, n_elec, ci, h0="fock", semicanonical=True):
        self.k = h.shape[0]
        self.k_act = k_act
        self.k_virt = self.k - k_act
        self.n_elec = n_elec
        self.ci = np.asarray(ci, dtype=np.float64)
        self.h0 = h0
        act = range(k_act)
        eri = eri_from_cholesky(L)
        g = np.zeros((k_act, k_act))
        for t in act:
            for u in act:
                g[t, u] = active_expectation(one_body_terms(_unit(self.k, t, u), [t], [u]),
                                             self.ci, k_act, n_elec)
        self.gamma = g
        f = self._fock(h, eri, g)
        if semicanonical and self.k_virt > 0:
            eps, U = np.linalg.eigh(f[k_act:, k_act:])
            # each semicanonical orbital is defined up to sign: make its
            # largest-magnitude coefficient positive (first one on ties)
            for j in range(U.shape[1]):
                i = int(np.argmax(np.abs(U[:, j])))
                if U[i, j] < 0:
                    U[:, j] = -U[:, j]
            C = np.eye(self.k)
            C[k_act:, k_act:] = U
            h = C.T @ h @ C
            L = np.einsum("pi,Qpq,qj->Qij", C, L, C, optimize=True)
            eri = eri_from_cholesky(L)
            f = C.T @ f @ C
            self.rotation = C
        self.h = h
        self.L = L
        self.eri = eri
        self.f = f
        self.eps = np.diag(f).copy()
        self.E_ref = active_expectation(self.h_act_terms(), self.ci, k_act, n_elec)
        if h0 == "dyall":
            self.E0 = self.E_ref
        elif h0 == "fock":
            self.E0 = float(np.sum(f[:k_act, :k_act] * g))
        else:
            raise ValueError(h0)
        self.E1 = self.E_ref - self.E0

    def _fock(self, h, eri, g):
        ka = self.k_act
        ea = eri[:, :, :ka, :ka]
        f = h + np.einsum("tu,pqtu->pq", g, ea, optimize=True)
        f -= 0.5 * np.einsum("tu,putq->pq", g, eri[:, :ka, :ka, :], optimize=True)
        return f

    # ---- term lists -------------------------------------------------------
    def h_act_terms(self):
        act = range(self.k_act)
        return one_body_terms(self.h, act, act) + two_body_terms(self.eri, act, act, act, act)

    def h0_terms(self, shift=True):
        """Terms of A = H0 - E0 (the constant is a term with no operators)."""
        act = range(self.k_act)
        virt = range(self.k_act, self.k)
        if self.h0 == "dyall":
            t = self.h_act_terms()
        else:
            t = one_body_terms(self.f, act, act)
        t = t + number_terms(self.eps, virt)
        if shift:
            t.append((-self.E0, ()))
        return t

    def rhs_terms(self):
        """Terms of H with >= 1 virtual creator and no virtual annihilator."""
        act = range(self.k_act)
        virt = range(self.k_act, self.k)
        allo = range(self.k)
        ka = self.k_act
        out = one_body_terms(self.h, virt, act)
        out += two_body_terms(self.eri, allo, act, allo, act,
                              keep=lambda p, q, r, s: p >= ka or r >= ka)
        return out

    def hamiltonian_terms(self):
        allo = range(self.k)
        return one_body_terms(self.h, allo, allo) + two_body_terms(self.eri, allo, allo, allo, allo)


def _unit(k, t, u):
    m = np.zeros((k, k))
    m[t, u] = 1.0
    return m
