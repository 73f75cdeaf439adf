"""Matrix product operators (Eq. 4) from second-quantised term lists.

Each term c * o_1 o_2 ... o_n (elementary c / c+ operators) is first brought
to site order (stable sort, sign of the permutation; operators on one site
keep their order).  Under the Jordan-Wigner string every operator on site q
acts as the parity P on every site p < q, so the term is the product over
sites p of  F_p = (product of the term's local operators on p) * P^{n_>p},
n_>p = number of its operators on sites > p.

The MPO is the finite-state machine that applies these factors site by site:
a bond state at cut c (between sites c-1 and c) is
  'I'                  nothing applied yet,
  ('P', prefix)        factors already applied on sites < c (coefficient not
                       yet applied; shared by all terms with that prefix),
  ('S', suffix)        coefficient applied, factors on sites >= c still to
                       apply (a complementary operator; shared by all terms
                       with that suffix),
  'F'                  term complete.
The coefficient is applied at one "centre" site of each term.  With the
centre chosen so that the open side carries at most two sites, the bond
dimension is O(k^2) (and O(k_a^2 + k_v) for the RHS operator), the
complementary-operator structure the paper relies on.
Pinned by tests/test_oracle_mpo.py: the contracted MPO equals the
brute-force determinant operator on small chains.
"""
import numpy as np

from .fermion import IDENT, PARITY, local_op, op_qn


class MPO:
    def __init__(self, nsite, W, qn, keys):
        self.nsite = nsite
        self.W = W            # W[p] = {(a, b): 4x4 matrix}
        self.qn = qn          # qn[c] = int array (D_c, 2) of (dN, d2Sz)
        self.keys = keys      # keys[c] = list of state keys
        self.dims = [len(k) for k in keys]

    def dense_site(self, p):
        Da, Db = self.dims[p], self.dims[p + 1]
        out = np.zeros((Da, Db, 4, 4))
        for (a, b), m in self.W[p].items():
            out[a, b] = m
        return out

    def to_dense(self):
        """Full 4^n x 4^n matrix (site 0 = most significant digit)."""
        T = {0: np.ones((1, 1))}
        for p in range(self.nsite):
            new = {}
            for (a, b), m in self.W[p].items():
                if a in T:
                    v = np.kron(T[a], m)
                    new[b] = new[b] + v if b in new else v
            T = new
        return T[0]


def _canonical(ops):
    """Stable sort by site; returns (sign, sorted ops)."""
    n = len(ops)
    inv = 0
    for i in range(n):
        for j in range(i + 1, n):
            if ops[i][0] // 2 > ops[j][0] // 2:
                inv += 1
    srt = sorted(range(n), key=lambda i: (ops[i][0] // 2, i))
    return (-1) ** inv, [ops[i] for i in srt]


class _FactorTable:
    def __init__(self):
        self.ids = {}
        self.mats = []

    def get(self, m):
        key = np.round(m, 12).tobytes()
        if key not in self.ids:
            self.ids[key] = len(self.mats)
            self.mats.append(m.copy())
        return self.ids[key]


def default_center(sites, k_split, nsite):
    """Centre site for a term with sorted distinct op sites."""
    m = len(sites)
    if m == 0:
        return 0
    if m == 1:
        return sites[0]
    if sites[-1] >= k_split:
        return sites[m - 2]
    mid2 = k_split - 1  # twice the midpoint of the active region
    if m == 2:
        return sites[1] if sites[0] + sites[1] <= mid2 else sites[0]
    if m == 3:
        return sites[1]
    return sites[2] if sites[1] + sites[2] <= mid2 else sites[1]


def build_mpo(terms, nsite, k_split=None, center=None):
    k_split = nsite if k_split is None else k_split
    center = center or (lambda S: default_center(S, k_split, nsite))
    ft = _FactorTable()
    I_id = ft.get(IDENT)
    P_id = ft.get(PARITY)
    entries = [dict() for _ in range(nsite)]   # (in_key, out_key) -> [fid, coef or None]
    qn_of = {"I": (0, 0), "F": (0, 0)}
    pass_range = {}                            # key -> [lo_site, hi_site] of pass-throughs
    parity_of = {}

    def set_entry(p, a, b, fid):
        e = entries[p].get((a, b))
        if e is None:
            entries[p][(a, b)] = [fid, None]
        elif e[1] is not None or e[0] != fid:
            raise AssertionError("inconsistent shared MPO transition")

    def add_entry(p, a, b, fid, coef):
        m = ft.mats[fid] * coef
        e = entries[p].get((a, b))
        if e is None:
            entries[p][(a, b)] = [None, m]
        elif e[1] is None:
            raise AssertionError("centre entry collides with a shared transition")
        else:
            e[1] = e[1] + m

    for coef, ops in terms:
        if coef == 0.0:
            continue
        if len(ops) % 2:
            raise ValueError("only fermion-parity-even terms are supported")
        sign, ops_s = _canonical(list(ops))
        c = coef * sign
        if not ops_s:
            s0 = center([])
            add_entry(s0, "I", "F", I_id, c)
            continue
        sites = sorted({j // 2 for j, _ in ops_s})
        fac = {}
        qn_site = {}
        for p in sites:
            m = IDENT
            dn = dsz = 0
            n_right = 0
            for j, dag in ops_s:
                q = j // 2
                if q == p:
                    m = m @ local_op(j % 2, dag)
                    a, b = op_qn(j % 2, dag)
                    dn += a
                    dsz += b
                elif q > p:
                    n_right += 1
            if n_right % 2:
                m = m @ PARITY
            fac[p] = ft.get(m)
            qn_site[p] = (dn, dsz)
        tot = (sum(v[0] for v in qn_site.values()), sum(v[1] for v in qn_site.values()))
        if tot != (0, 0):
            raise ValueError("terms must conserve N and Sz")
        s_c = center(sites)
        # state at each cut c in [sites[0]+1, sites[-1]]
        def state(cut):
            if cut <= sites[0]:
                return "I"
            if cut > sites[-1]:
                return "F"
            if cut <= s_c:
                pre = tuple((p, fac[p]) for p in sites if p < cut)
                return ("P", pre)
            suf = tuple((p, fac[p]) for p in sites if p >= cut)
            return ("S", suf)

        for idx, p in enumerate(sites):
            a = state(p)
            b = state(p + 1)
            if p == s_c:
                add_entry(p, a, b, fac[p], c)
            else:
                set_entry(p, a, b, fac[p])
            # QN / parity of the outgoing state and its pass-through range
            if b not in ("I", "F"):
                if b[0] == "P":
                    ops_in = [q for q in sites if q <= p]
                    dq = (sum(qn_site[q][0] for q in ops_in), sum(qn_site[q][1] for q in ops_in))
                else:
                    ops_in = [q for q in sites if q > p]
                    dq = (-sum(qn_site[q][0] for q in ops_in), -sum(qn_site[q][1] for q in ops_in))
                qn_of[b] = dq
                nxt = sites[idx + 1]
                lo, hi = p + 1, nxt - 1
                if lo <= hi:
                    r = pass_range.get(b)
                    pass_range[b] = [lo, hi] if r is None else [min(r[0], lo), max(r[1], hi)]
                nops = sum(1 for j, _ in ops_s if (j // 2 <= p) == (b[0] == "P"))
                parity_of[b] = nops % 2

    for key, (lo, hi) in pass_range.items():
        fid = P_id if parity_of[key] else I_id
        for p in range(lo, hi + 1):
            set_entry(p, key, key, fid)
    for p in range(nsite):
        entries[p][("I", "I")] = [I_id, None]
        entries[p][("F", "F")] = [I_id, None]

    # prune states not connected to I at cut 0 and F at cut nsite
    alive = [set() for _ in range(nsite + 1)]
    alive[0].add("I")
    for p in range(nsite):
        for (a, b) in entries[p]:
            if a in alive[p]:
                alive[p + 1].add(b)
    back = [set() for _ in range(nsite + 1)]
    back[nsite].add("F")
    for p in range(nsite - 1, -1, -1):
        for (a, b) in entries[p]:
            if b in back[p + 1]:
                back[p].add(a)
    keys = []
    for c in range(nsite + 1):
        ks = alive[c] & back[c]
        keys.append(sorted(ks, key=_sort_key))
    index = [{k: i for i, k in enumerate(ks)} for ks in keys]
    W = []
    for p in range(nsite):
        Wp = {}
        for (a, b), (fid, m) in entries[p].items():
            if a in index[p] and b in index[p + 1]:
                mat = ft.mats[fid] if m is None else m
                Wp[(index[p][a], index[p + 1][b])] = mat
        W.append(Wp)
    qn = [np.array([qn_of[k] for k in ks], dtype=np.int64).reshape(-1, 2) for ks in keys]
    return MPO(nsite, W, qn, keys)


def _sort_key(k):
    if k == "I":
        return (0, ())
    if k == "F":
        return (3, ())
    return (1 if k[0] == "P" else 2, k[1])
