"""Partitioned first-order problem (the "embarrassing" parallelism over
virtual-orbital pairs mentioned with the paper's parallelisation).

H0 (Fock or Dyall) conserves the occupation of every semicanonical virtual
orbital, so A = P_X (H0 - E0) P_X is block-diagonal over virtual occupation
patterns and E2* = sum_P E2*_P exactly.  Pairs are read as a <= b:
  P = (a, b), a < b : one electron in a and one in b;
  P = (a, a)        : one or two electrons in a (the single-virtual sector of
                      a is folded into (a, a)).
That gives k_v (k_v + 1) / 2 partitions (1830 for k_v = 60).

Each partition is an MPS-PT problem of its own on the chain
  active orbitals (in order), then a, then b (a < b),
with the occupation constraints imposed on the bonds after the active
block and after a.  The sub-problems reuse the full-space machinery:
operators are the full H0 and the RHS part of H restricted to these
orbitals, written in the sub-chain's site order (which keeps the relative
orbital order, so Jordan-Wigner signs agree with the full chain).
Pinned by tests/test_oracle_partition.py: sum of partition E2* equals the
full brute-force E2*, and the MPS sweep of each partition at its exact bond
dimension reproduces its E2*_P.
"""
import numpy as np

from .brute import DetSpace, ExactFirstOrder, apply_terms, ci_to_dets, operator_matrix
from .operators import number_terms, one_body_terms, two_body_terms


def partitions(k_virt):
    """(a, b) virtual indices (0-based within the virtual block), a <= b,
    ordered by a then b (the summation order of E2)."""
    return [(a, b) for a in range(k_virt) for b in range(a, k_virt)]


class SubProblem:
    """MPS-PT problem of one partition, with the interface HylleraasSweep uses."""

    def __init__(self, prob, a, b):
        ka = prob.k_act
        self.parent = prob
        self.pair = (a, b)
        orbs = list(range(ka)) + ([ka + a] if a == b else [ka + a, ka + b])
        self.orbs = orbs
        self.k = len(orbs)
        self.k_act = ka
        self.k_virt = self.k - ka
        self.n_elec = prob.n_elec
        self.ci = prob.ci
        self.h0 = prob.h0
        ix = np.array(orbs)
        self.h = prob.h[np.ix_(ix, ix)]
        self.f = prob.f[np.ix_(ix, ix)]
        self.eri = prob.eri[np.ix_(ix, ix, ix, ix)]
        self.eps = np.diag(self.f).copy()
        self.E0, self.E1, self.E_ref = prob.E0, prob.E1, prob.E_ref
        N = prob.n_elec
        if a == b:
            self.allowed = {ka: {N - 1, N - 2}}
        else:
            self.allowed = {ka: {N - 2}, ka + 1: {N - 1}}

    def h_act_terms(self):
        act = range(self.k_act)
        return one_body_terms(self.h, act, act) + two_body_terms(self.eri, act, act, act, act)

    def h0_terms(self, shift=True):
        act = range(self.k_act)
        virt = range(self.k_act, self.k)
        t = self.h_act_terms() if self.h0 == "dyall" else one_body_terms(self.f, act, act)
        t = t + number_terms(self.eps, virt)
        if shift:
            t.append((-self.E0, ()))
        return t

    def rhs_terms(self):
        act = range(self.k_act)
        virt = range(self.k_act, self.k)
        allo = range(self.k)
        ka = self.k_act
        out = one_body_terms(self.h, virt, act)
        out += two_body_terms(self.eri, allo, act, allo, act, keep=lambda p, q, r, s: p >= ka or r >= ka)
        return out

    def x_mask(self, space):
        """Determinants of the sub-chain that belong to this partition."""
        ka = self.k_act
        occ_a = ((space.dets >> np.uint64(2 * ka)) & np.uint64(3))
        na = np.bitwise_count(occ_a).astype(int)
        if self.pair[0] == self.pair[1]:
            return (na == 1) | (na == 2)
        occ_b = ((space.dets >> np.uint64(2 * ka + 2)) & np.uint64(3))
        nb = np.bitwise_count(occ_b).astype(int)
        return (na == 1) & (nb == 1)


class ExactPartition:
    """Uncontracted E2*_P of one partition (dense solve on its X_P)."""

    def __init__(self, sub):
        full = DetSpace.sector(sub.k, sub.n_elec, 0)
        self.X = full.subset(sub.x_mask(full))
        d0, c0 = ci_to_dets(sub.ci, sub.k_act)
        ref = DetSpace(d0)
        order = np.argsort(d0)
        self.A = operator_matrix(sub.h0_terms(), self.X)
        self.g = apply_terms(sub.rhs_terms(), ref, c0[order], self.X)

    def e2(self):
        if len(self.X) == 0:
            return 0.0
        x = np.linalg.solve(self.A.toarray(), self.g)
        return -float(self.g @ x)


def partition_e2(prob, M_of, sweep_kwargs=None):
    """Sum of MPS-PT2 partition energies (FP64, partition order a, then b).

    M_of: callable (a, b) -> bond dimension of that partition."""
    from .mps import HylleraasSweep
    total = 0.0
    parts = []
    for a, b in partitions(prob.k_virt):
        sub = SubProblem(prob, a, b)
        sw = HylleraasSweep(sub, M_of(a, b), allowed=sub.allowed, **(sweep_kwargs or {}))
        e = sw.run()
        parts.append(((a, b), e))
        total += e
    return total, parts
