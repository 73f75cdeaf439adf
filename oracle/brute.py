"""Determinant-space brute force: the uncontracted first-order problem.

A second-quantised term (coef, ops) with ops = ((j, dagger), ...) in product
order is applied to bit strings literally: operators act right to left, each
c_j / c+_j picks up (-1)^{#occupied j' < j} (the Jordan-Wigner string) and
kills the state when the occupation forbids it.  No Slater rules are used.

On top of that this module states the exact (uncontracted, M -> infinity)
quantities of the paper:
  A  = P_X (H0 - E0) P_X,  g = P_X V Psi0          (Eq. 2, Q = 1 on X)
  E2* = min H[Psi1] = -g^T A^{-1} g                 (Eq. 1 at its minimum)
  E3* = <Psi1|V|Psi1> - E1 <Psi1|Psi1>              (Eq. 5)
where X is the span of determinants with one or two electrons in virtual
orbitals (no core orbitals).  Pinned by the MP2 closed form
(tests/test_oracle_exact.py) and by the Sz-flip / orbital-rotation
invariances of E2*.
"""
import itertools
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def _bitcount(x):
    return np.bitwise_count(x).astype(np.int64)


class DetSpace:
    """Sorted uint64 bit strings over 2*n_orb spin-orbitals (j = 2p + s)."""

    def __init__(self, dets):
        self.dets = np.unique(np.asarray(dets, dtype=np.uint64))

    @classmethod
    def sector(cls, n_orb, n_elec, two_sz=0):
        na = (n_elec + two_sz) // 2
        nb = n_elec - na
        out = []
        for occa in itertools.combinations(range(n_orb), na):
            ba = 0
            for p in occa:
                ba |= 1 << (2 * p)
            for occb in itertools.combinations(range(n_orb), nb):
                bb = 0
                for p in occb:
                    bb |= 1 << (2 * p + 1)
                out.append(ba | bb)
        return cls(out)

    def __len__(self):
        return len(self.dets)

    def index(self, d):
        pos = np.searchsorted(self.dets, d)
        pos = np.minimum(pos, len(self.dets) - 1)
        found = self.dets[pos] == d
        return np.where(found, pos, -1)

    def subset(self, mask):
        return DetSpace(self.dets[mask])

    def n_virtual(self, k_act):
        """Number of electrons in spin-orbitals of spatial orbitals >= k_act."""
        low = np.uint64((1 << (2 * k_act)) - 1)
        return _bitcount(self.dets & ~low)


def apply_ops(dets, ops):
    """Apply a product of elementary operators to every bit string.

    Returns (new_dets, sign, alive)."""
    cur = dets.copy()
    sign = np.ones(len(dets), dtype=np.int64)
    alive = np.ones(len(dets), dtype=bool)
    for j, dag in reversed(ops):
        bit = (cur >> np.uint64(j)) & np.uint64(1)
        alive &= (bit == 0) if dag else (bit == 1)
        below = _bitcount(cur & np.uint64((1 << j) - 1))
        sign *= 1 - 2 * (below & 1)
        cur = cur ^ np.uint64(1 << j)
    return cur, sign, alive


def operator_matrix(terms, space_in, space_out=None):
    """Sparse matrix <out| sum_terms |in> (projected onto space_out)."""
    space_out = space_in if space_out is None else space_out
    rows, cols, vals = [], [], []
    ar = np.arange(len(space_in))
    for coef, ops in terms:
        if coef == 0.0:
            continue
        new, sign, alive = apply_ops(space_in.dets, ops)
        idx = space_out.index(new)
        keep = alive & (idx >= 0)
        rows.append(idx[keep])
        cols.append(ar[keep])
        vals.append(coef * sign[keep])
    if not rows:
        return sp.csr_matrix((len(space_out), len(space_in)))
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals).astype(np.float64)
    return sp.csr_matrix((v, (r, c)), shape=(len(space_out), len(space_in)))


def apply_terms(terms, space_in, vec, space_out=None):
    """sum_terms applied to a vector on space_in, projected onto space_out."""
    space_out = space_in if space_out is None else space_out
    out = np.zeros(len(space_out))
    nz = np.nonzero(vec)[0]
    dets = space_in.dets[nz]
    x = vec[nz]
    for coef, ops in terms:
        if coef == 0.0:
            continue
        new, sign, alive = apply_ops(dets, ops)
        idx = space_out.index(new)
        keep = alive & (idx >= 0)
        np.add.at(out, idx[keep], coef * sign[keep] * x[keep])
    return out


def ci_to_dets(ci, k_act):
    """Active-space CI vector (4**k_act site-occupation basis) -> (dets, coefs)."""
    nz = np.nonzero(ci)[0]
    dets = np.zeros(len(nz), dtype=np.uint64)
    for n, idx in enumerate(nz):
        b = 0
        rem = int(idx)
        for p in range(k_act - 1, -1, -1):
            code = rem % 4
            rem //= 4
            if code & 1:
                b |= 1 << (2 * p)
            if code & 2:
                b |= 1 << (2 * p + 1)
        dets[n] = b
    return dets, ci[nz]


def dets_to_site_index(dets, n_orb):
    """Bit strings -> index in the 4**n_orb site-occupation basis."""
    out = np.zeros(len(dets), dtype=np.int64)
    for p in range(n_orb):
        code = ((dets >> np.uint64(2 * p)) & np.uint64(1)) + 2 * ((dets >> np.uint64(2 * p + 1)) & np.uint64(1))
        out = out * 4 + code.astype(np.int64)
    return out


class ExactFirstOrder:
    """Uncontracted first-order problem on X (1 or 2 virtual electrons)."""

    def __init__(self, prob):
        k = prob.k
        self.prob = prob
        full = DetSpace.sector(k, prob.n_elec, 0)
        nv = full.n_virtual(prob.k_act)
        self.X = full.subset((nv == 1) | (nv == 2))
        d0, c0 = ci_to_dets(prob.ci, prob.k_act)
        self.ref_space = DetSpace(d0)
        order = np.argsort(d0)
        self.psi0 = c0[order]
        self.A = operator_matrix(prob.h0_terms(), self.X)
        self.g = apply_terms(prob.rhs_terms(), self.ref_space, self.psi0, self.X)

    def solve(self):
        A = self.A.toarray() if len(self.X) <= 6000 else None
        if A is not None:
            self.psi1 = -np.linalg.solve(A, self.g)
        else:
            self.psi1 = -spla.spsolve(self.A.tocsc(), self.g)
        return self.psi1

    def e2(self):
        if not hasattr(self, "psi1"):
            self.solve()
        return float(self.g @ self.psi1)

    def hylleraas(self, psi1):
        """Eq. 1 on X: <psi1|H0-E0|psi1> + 2 <psi1|V|psi0>."""
        return float(psi1 @ (self.A @ psi1) + 2.0 * psi1 @ self.g)

    def e3(self):
        """Eq. 5 with V = H - H0 on X; <psi1|H0|psi1> = <psi1|A|psi1> + E0 |psi1|^2."""
        if not hasattr(self, "psi1"):
            self.solve()
        p = self.prob
        x = self.psi1
        Hx = apply_terms(p.hamiltonian_terms(), self.X, x)
        n2 = float(x @ x)
        vxx = float(x @ Hx) - float(x @ (self.A @ x)) - p.E0 * n2
        return vxx - p.E1 * n2

    def schmidt_ranks(self):
        """QN-blocked Schmidt rank of psi1* at every cut (sets M_exact)."""
        if not hasattr(self, "psi1"):
            self.solve()
        k = self.prob.k
        site_idx = dets_to_site_index(self.X.dets, k)
        ranks = []
        for c in range(1, k):
            left = site_idx // (4 ** (k - c))
            right = site_idx % (4 ** (k - c))
            # group by left QN (N, 2Sz) of the left part
            lq = {}
            for n, (li, ri) in enumerate(zip(left, right)):
                lq.setdefault(_left_qn(int(li), c), []).append(n)
            rank = 0
            for q, members in lq.items():
                members = np.array(members)
                lu, linv = np.unique(left[members], return_inverse=True)
                ru, rinv = np.unique(right[members], return_inverse=True)
                m = np.zeros((len(lu), len(ru)))
                m[linv, rinv] = self.psi1[members]
                s = np.linalg.svd(m, compute_uv=False)
                rank += int(np.sum(s > 1e-12 * max(1.0, s[0] if len(s) else 0.0)))
            ranks.append(rank)
        return ranks


def _left_qn(left_index, c):
    n = 0
    sz = 0
    for _ in range(c):
        code = left_index % 4
        left_index //= 4
        n += (code & 1) + ((code >> 1) & 1)
        sz += (code & 1) - ((code >> 1) & 1)
    return (n, sz)
