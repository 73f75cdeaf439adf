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

E3 over partitions (Eq. 5 for Psi1 = sum_P Psi1^P).  Partitions live on
disjoint virtual-occupation patterns and H0 keeps every pattern, so for
P != P' both <Psi1^P|Psi1^P'> and <Psi1^P|H0|Psi1^P'> vanish, while V (which
moves up to two electrons between orbitals) does not:
  E3 = sum_P E3(Psi1^P) + sum_{P != P'} <Psi1^P|H|Psi1^P'>.
Two routes: the plain definition (every Psi1^P written as a vector on the
full determinant space X and Eq. 5 applied to the sum; small systems), and
transfers of embedded MPSs (every Psi1^P written on the full chain, empty
virtual sites passing the bond through).  Pinned by
tests/test_oracle_partition.py: at exact partitions the sum of the embedded
vectors is the full-space Psi1* and the E3 of the sum is the full-space E3*;
the two routes agree on truncated MPSs.
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

    def solve(self):
        """Exact Psi1*_P on X_P (Eq. 2 restricted to the partition)."""
        if len(self.X) == 0:
            return np.zeros(0)
        return -np.linalg.solve(self.A.toarray(), self.g)

    def e2(self):
        if len(self.X) == 0:
            return 0.0
        return float(self.g @ self.solve())


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


# ------------------------------------------------------- E3 over partitions
def sub_dets_to_full(sub, dets):
    """Bit strings over a partition chain's orbitals -> bit strings over all
    orbitals (chain orbital i is orbital sub.orbs[i]).  The chain keeps the
    orbitals' relative order, so a determinant's sign convention (creators in
    ascending spin-orbital order) is unchanged."""
    out = np.zeros(len(dets), dtype=np.uint64)
    for i, p in enumerate(sub.orbs):
        out |= ((dets >> np.uint64(2 * i)) & np.uint64(3)) << np.uint64(2 * p)
    return out


def embed_vector(sub, dets, coefs, X):
    """Psi1^P given on sub-chain determinants -> vector on the full space X."""
    x = np.zeros(len(X))
    if len(dets) == 0:
        return x
    idx = X.index(sub_dets_to_full(sub, dets))
    if np.any(idx < 0):
        raise ValueError("partition determinant outside the first-order space")
    x[idx] = coefs
    return x


def mps_vector(sub, mps, X):
    """An MPS on a partition chain -> its vector on the full space X."""
    d, c = ci_to_dets(mps.to_dense(), sub.k)
    return embed_vector(sub, d, c, X)


def e3_split(prob, X, A, xs):
    """Eq. 5 for x = sum(xs) on X by its plain definition:
    E3 = <x|H|x> - <x|A|x> - (E0 + E1) <x|x>   (A = H0 - E0).
    Returns (E3 of the sum, [E3 of each x_P], sum of the cross terms); the
    cross sum is E3 of the sum minus the diagonal terms."""
    H = operator_matrix(prob.hamiltonian_terms(), X)

    def e3(x):
        return float(x @ (H @ x) - x @ (A @ x) - (prob.E0 + prob.E1) * (x @ x))

    diag = [e3(x) for x in xs]
    tot = e3(np.sum(xs, axis=0)) if xs else 0.0
    return tot, diag, tot - sum(diag)


def embed_mps(prob, sub, mps):
    """Psi1^P (MPS on its partition chain) written on the full chain: active
    sites and the partition's virtual sites keep their tensors; every other
    virtual orbital becomes an empty site that passes the bond through
    (identity on the bond, local state |0>, even parity)."""
    from .mps import MPS
    ka = prob.k_act
    A = [t.copy() for t in mps.A[:ka]]
    q = [l.copy() for l in mps.q[:ka + 1]]
    j = ka
    for v in range(prob.k_virt):
        if j < sub.k and sub.orbs[j] == ka + v:
            A.append(mps.A[j].copy())
            q.append(mps.q[j + 1].copy())
            j += 1
        else:
            D = len(q[-1])
            T = np.zeros((D, 4, D))
            T[np.arange(D), 0, np.arange(D)] = 1.0
            A.append(T)
            q.append(q[-1].copy())
    return MPS(A, q)


def partition_psi1(prob, pairs, M_of, sweep_kwargs=None):
    """MPS-PT2 sweep of every listed partition: [(sub, E2_P, Psi1^P MPS)]."""
    from .mps import HylleraasSweep
    out = []
    for a, b in pairs:
        sub = SubProblem(prob, a, b)
        sw = HylleraasSweep(sub, M_of(a, b), allowed=sub.allowed, **(sweep_kwargs or {}))
        out.append((sub, sw.run(), sw.psi1))
    return out


def partition_e3_mps(prob, subs_psis, WH=None, WA=None):
    """E3 of Psi1 = sum of the listed partitions' MPSs by transfers on the
    full chain: E3(Psi1^P) = <H> - <A> - (E0 + E1)<1> for each P, and
    2 <Psi1^P|H|Psi1^P'> for each pair P < P' (pairs in list order).
    Returns (total, [E3 of each], cross sum, {(i, j): <P_i|H|P_j>})."""
    from .mpo import build_mpo
    from .mps import expectation, overlap
    k, ka = prob.k, prob.k_act
    WH = WH or build_mpo(prob.hamiltonian_terms(), k, k_split=ka)
    WA = WA or build_mpo(prob.h0_terms(), k, k_split=ka)
    emb = [embed_mps(prob, sub, psi) for sub, psi in subs_psis]
    diag = [expectation(e, WH, e) - expectation(e, WA, e) - (prob.E0 + prob.E1) * overlap(e, e) for e in emb]
    h = {}
    cross = 0.0
    for i in range(len(emb)):
        for j in range(i + 1, len(emb)):
            h[(i, j)] = expectation(emb[i], WH, emb[j])
            cross += 2.0 * h[(i, j)]
    return sum(diag) + cross, diag, cross, h
