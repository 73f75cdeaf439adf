"""Ground-state DMRG for the reference Psi0 (TEST INFRASTRUCTURE ONLY).

The paper takes Psi0 from a DMRG calculation of the active space and notes
that its Hylleraas sweep is the standard DMRG sweep with a linear equation in
place of the eigenvalue problem.  This module is that standard sweep, built
from the same pieces as ``mps.HylleraasSweep``:

* H_act = the terms of H whose indices are all active, as an MPO on the
  k_act active sites, optionally plus lam S^2 (every spin-S state raised by
  lam S(S+1), so the lowest singlet becomes the ground state: reading A3 of
  the reference wants a singlet);
* the initial state is the first-order sweep's seeded rule (reading R8):
  ``random_mps`` in the (n_elec, Sz = 0) sector, made right-canonical by
  density-matrix splits;
* at bond (i, i+1) the two-site tensor x minimises the Rayleigh quotient
  x.H_loc x / x.x with H_loc = L_i W_i W_{i+1} R_{i+2} (the Fig. 1C
  contraction of H_act): its lowest eigenvector, found by a dense ``eigh`` of
  H_loc built column by column on small local spaces and by ARPACK
  (``eigsh``, Lanczos) started from the current two-site product on larger
  ones;
* x is split by the renormalisation step (``mps.truncate``: density matrix,
  QN sectors, reading R7's keep rule) and the environment is updated;
* sweeps alternate left-to-right and right-to-left until the energy changes
  by less than tol_e between full sweeps.

Pinned by tests/test_oracle_dmrg.py: at a bond dimension that represents the
state exactly the energy equals the lowest (N, Sz = 0) eigenvalue of the
brute-force determinant Hamiltonian; truncated runs lie above it and
decrease with M; the final MPS's <H_act> by MPO transfer equals the last
local eigenvalue when nothing is truncated.
"""
import numpy as np

from .mpo import build_mpo
from .mps import (KEEP_REL, canonicalize_by_splits, env_left, env_right, random_mps, truncate,
                  two_site_apply, two_site_mask)
from .operators import eri_from_cholesky, one_body_terms, two_body_terms


def active_hamiltonian_terms(h, L, k_act):
    """H_act: one- and two-electron terms with every index active."""
    act = range(k_act)
    eri = eri_from_cholesky(L[:, :k_act, :k_act])
    return one_body_terms(h, act, act) + two_body_terms(eri, act, act, act, act)


def spin_squared_terms(k_act, lam):
    """lam S^2 on Sz = 0 states: lam S- S+ with S+ = sum_p c+_pa c_pb and
    S- = sum_q c+_qb c_qa, as the literal operator products."""
    out = []
    for q in range(k_act):
        for p in range(k_act):
            out.append((lam, ((2 * q + 1, True), (2 * q, False), (2 * p, True), (2 * p + 1, False))))
    return out


class GroundStateSweep:
    def __init__(self, h, L, k_act, n_elec, M, seed=1408, tol_e=1e-10, max_sweeps=30, keep_rel=None,
                 dense_max=300, s2_penalty=0.0):
        self.k = k_act
        self.M = M
        self.tol_e = tol_e
        self.max_sweeps = max_sweeps
        self.keep_rel = KEEP_REL if keep_rel is None else keep_rel
        self.dense_max = dense_max
        terms = active_hamiltonian_terms(h, L, k_act)
        if s2_penalty > 0.0:
            terms = terms + spin_squared_terms(k_act, s2_penalty)
        self.W = build_mpo(terms, k_act)
        self.psi = canonicalize_by_splits(random_mps(k_act, (n_elec, 0), {}, M, seed), {}, self.keep_rel)
        k = k_act
        one = np.ones((1, 1, 1))
        self.L = [None] * (k + 1)
        self.R = [None] * (k + 1)
        self.L[0] = one
        self.R[k] = one
        for c in range(k - 1, 0, -1):
            self.R[c] = env_right(self.R[c + 1], self.psi.A[c], self.W.W[c], self.psi.A[c], self.W.dims[c])
        self.history = []
        self.discarded = []

    def local_eigen(self, i):
        ps = self.psi
        x0 = np.einsum("lsm,mtr->lstr", ps.A[i], ps.A[i + 1])
        mask = two_site_mask(ps.q[i], ps.q[i + 2], None)
        idx = np.flatnonzero(mask)
        Li, Ri = self.L[i], self.R[i + 2]
        W1, W2, Dm = self.W.W[i], self.W.W[i + 1], self.W.dims[i + 1]

        def apply(v):
            full = np.zeros(x0.size)
            full[idx] = v
            return two_site_apply(Li, W1, W2, Ri, full.reshape(x0.shape), Dm).reshape(-1)[idx]

        n = len(idx)
        if n <= self.dense_max:
            H = np.column_stack([apply(e) for e in np.eye(n)])
            w, v = np.linalg.eigh(0.5 * (H + H.T))
            e, y = float(w[0]), v[:, 0]
        else:
            from scipy.sparse.linalg import LinearOperator, eigsh
            op = LinearOperator((n, n), matvec=apply, dtype=np.float64)
            w, v = eigsh(op, k=1, which="SA", v0=x0.reshape(-1)[idx], tol=1e-14, maxiter=100000)
            e, y = float(w[0]), v[:, 0]
        x = np.zeros(x0.size)
        x[idx] = y
        return e, x.reshape(x0.shape)

    def step(self, i, direction):
        e, x = self.local_eigen(i)
        ps = self.psi
        Al, Ar, lab, w = truncate(x, ps.q[i], ps.q[i + 2], self.M, direction, None, self.keep_rel)
        ps.A[i], ps.A[i + 1] = Al, Ar
        ps.q[i + 1] = lab
        self.discarded.append(w)
        if direction == "LR":
            self.L[i + 1] = env_left(self.L[i], Al, self.W.W[i], Al, self.W.dims[i + 1])
        else:
            self.R[i + 1] = env_right(self.R[i + 2], Ar, self.W.W[i + 1], Ar, self.W.dims[i + 1])
        return e

    def sweep(self):
        e = None
        for i in range(self.k - 1):
            e = self.step(i, "LR")
        for i in range(self.k - 2, -1, -1):
            e = self.step(i, "RL")
        return e

    def run(self):
        prev = None
        for _ in range(self.max_sweeps):
            self.discarded = []
            e = self.sweep()
            self.history.append(e)
            if prev is not None and abs(e - prev) < self.tol_e:
                break
            prev = e
        self.energy = self.history[-1]
        return self.energy
