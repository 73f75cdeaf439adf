"""MPS (Eq. 3) and the two-site sweep that minimises the Hylleraas functional.

Plain dense NumPy with QN labels: every bond index carries the (N, 2Sz) of
the part of the chain to its left; tensor entries that violate the labels
are zero.  Steps follow the paper's description of the sweep:

* at bond (i, i+1) the Hylleraas functional restricted to the two-site
  tensor x (all other tensors fixed, mixed-canonical gauge) is
      h(x) = x.A_loc x + 2 x.g_loc                              (Eq. 1)
  with A_loc the projection of H0 - E0 (L_A W W R_A, Fig. 1C first term)
  and g_loc the projection of V Psi0 (L_V W W R_V applied to Psi0's
  two-site tensor, Fig. 1C second term; the third, Q-projection term
  vanishes because Psi1 lies in X, orthogonal to Psi0);
* its stationarity condition A_loc x = -g_loc (Fig. 1C) is solved by
  Jacobi-preconditioned conjugate gradient, warm-started from the current
  two-site tensor;
* x is split by the density matrix rho = X X^T (left-to-right) or X^T X
  (right-to-left), eigen-decomposed per QN sector in float64, keeping the M
  largest eigenvalues; the discarded weight is recorded;
* the renormalised operators (environments) of <Psi1|H0-E0|Psi1> and
  <Psi1|V|Psi0> are updated;
* sweeps alternate left-to-right and right-to-left until the energy changes
  by less than tol_e between full sweeps.  E2(M) is h at the last bond.

The first-order space X (1 or 2 virtual electrons) is imposed by allowing
only N_left in {N-1, N-2} on the bond between the last active and the first
virtual site.

Initial Psi1 (a documented rule shared with the GPU library):
  * sector dimensions at cut c: w_q = min(nL_c(q), nR_c(q), M) where nL/nR
    count the occupation strings left / right of the cut compatible with the
    target and the sector filter; if sum w > M, dim_q = min(w_q,
    max(1, floor(M w_q / sum w)));  sectors sorted by (N, 2Sz);
  * entry (l, s, r) of site c: u = splitmix64((seed << 48) + ((4c + s) << 38)
    + (l << 19) + r) >> 11, value = u * 2^-53 - 0.5 (l, r = positions in the
    sorted bond bases);
  * then brought to right-canonical form by the renormalisation step
    itself: for i = nsite-2 .. 0 the two-site product A_i A_{i+1} is split
    right-to-left by its density matrix (truncate with no M cap: every
    eigenvector above 1e-10 tr rho is kept, the sector filter applies), so
    the initial state is the random MPS with its negligible directions
    removed by the same rule the sweep uses.
"""
import numpy as np

from .fermion import QN_N, QN_SZ

QN_SITE = np.stack([QN_N, QN_SZ], axis=1)

# Reading R7: density-matrix eigenvectors with eigenvalue <= KEEP_REL tr(rho)
# are never kept.  The paper leaves the threshold open.  At 1e-10 the
# smallest kept eigenvalues lie six decades above the rounding level of a
# float64 eigensolver (~1e-16 |rho|), so which states are kept, and the
# energies that follow, do not depend on how an eigensolver rounds.
KEEP_REL = 1e-10
MASK64 = (1 << 64) - 1


def splitmix64(x):
    """SplitMix64 finaliser (Steele, Lea, Flood 2014) on a 64-bit integer."""
    z = (x + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def init_value(seed, c, s, l, r):
    x = ((seed << 48) + ((4 * c + s) << 38) + (l << 19) + r) & MASK64
    return (splitmix64(x) >> 11) * 2.0 ** -53 - 0.5


# ---------------------------------------------------------------- structure
def sector_counts(nsite, target, allowed_n):
    """nL[c], nR[c]: dict q -> number of compatible strings (exact ints)."""
    nL = [dict() for _ in range(nsite + 1)]
    nL[0][(0, 0)] = 1
    for c in range(nsite):
        for q, n in nL[c].items():
            for s in range(4):
                q2 = (q[0] + int(QN_N[s]), q[1] + int(QN_SZ[s]))
                nL[c + 1][q2] = nL[c + 1].get(q2, 0) + n
        if allowed_n.get(c + 1) is not None:
            nL[c + 1] = {q: n for q, n in nL[c + 1].items() if q[0] in allowed_n[c + 1]}
    nR = [dict() for _ in range(nsite + 1)]
    nR[nsite][tuple(target)] = 1
    for c in range(nsite - 1, -1, -1):
        for q, n in nR[c + 1].items():
            for s in range(4):
                q2 = (q[0] - int(QN_N[s]), q[1] - int(QN_SZ[s]))
                nR[c][q2] = nR[c].get(q2, 0) + n
        if allowed_n.get(c) is not None:
            nR[c] = {q: n for q, n in nR[c].items() if q[0] in allowed_n[c]}
    return nL, nR


def initial_sectors(nsite, target, allowed_n, M):
    nL, nR = sector_counts(nsite, target, allowed_n)
    out = []
    for c in range(nsite + 1):
        w = {}
        for q in nL[c]:
            if q in nR[c]:
                v = min(nL[c][q], nR[c][q], M)
                if v > 0:
                    w[q] = v
        tot = sum(w.values())
        if tot > M:
            w = {q: min(v, max(1, (M * v) // tot)) for q, v in w.items()}
        out.append(sorted(w.items()))
    return out


def _labels(sectors):
    lab = []
    for q, d in sectors:
        lab.extend([q] * d)
    return np.array(lab, dtype=np.int64).reshape(-1, 2)


def _block_mask(ql, qr):
    """mask[l, s, r] of QN-consistent entries of a site tensor."""
    comp = ql[:, None, :] + QN_SITE[None, :, :]
    return np.all(comp[:, :, None, :] == qr[None, None, :, :], axis=-1)


class MPS:
    def __init__(self, tensors, labels):
        self.A = tensors       # A[c]: (D_c, 4, D_{c+1})
        self.q = labels        # q[c]: (D_c, 2) left-cumulative (N, 2Sz)

    @property
    def nsite(self):
        return len(self.A)

    def dims(self):
        return [len(x) for x in self.q]

    def to_dense(self):
        v = np.ones((1, 1))
        for A in self.A:
            v = np.einsum("xl,lsr->xsr", v, A).reshape(-1, A.shape[2])
        return v[:, 0]


def random_mps(nsite, target, allowed_n, M, seed):
    secs = initial_sectors(nsite, target, allowed_n, M)
    labels = [_labels(s) for s in secs]
    A = []
    for c in range(nsite):
        ql, qr = labels[c], labels[c + 1]
        mask = _block_mask(ql, qr)
        T = np.zeros((len(ql), 4, len(qr)))
        for l, s, r in zip(*np.nonzero(mask)):
            T[l, s, r] = init_value(seed, c, int(s), int(l), int(r))
        A.append(T)
    return MPS(A, labels)


def canonicalize_by_splits(mps, allowed, keep_rel=KEEP_REL):
    """Right-canonical form by right-to-left density-matrix splits of the
    two-site products (the sweep's renormalisation step without an M cap);
    the norm ends up in A[0]."""
    for i in range(mps.nsite - 2, -1, -1):
        x = np.einsum("lsm,mtr->lstr", mps.A[i], mps.A[i + 1])
        Al, Ar, lab, _ = truncate(x, mps.q[i], mps.q[i + 2], 1 << 30, "RL", allowed.get(i + 1),
                                  keep_rel)
        mps.A[i], mps.A[i + 1], mps.q[i + 1] = Al, Ar, lab
    return mps


def right_canonicalize(mps, tol=1e-14):
    """Sweep right to left making A[c] (c >= 1) right-orthonormal (SVD per
    left sector); the norm ends up in A[0]."""
    for c in range(mps.nsite - 1, 0, -1):
        A = mps.A[c]
        ql = mps.q[c]
        Dl, _, Dr = A.shape
        X = A.reshape(Dl, 4 * Dr)
        keys = sorted({tuple(q) for q in ql})
        newB, newLab, Cmat = [], [], np.zeros((Dl, 0))
        blocks = []
        for q in keys:
            rows = np.nonzero(np.all(ql == q, axis=1))[0]
            U, S, Vt = np.linalg.svd(X[rows], full_matrices=False)
            keep = S > tol * max(S[0], 1e-300) if len(S) else np.zeros(0, bool)
            keep &= S > 0
            blocks.append((q, rows, U[:, keep] * S[keep], Vt[keep]))
        Dn = sum(b[3].shape[0] for b in blocks)
        B = np.zeros((Dn, 4 * Dr))
        C = np.zeros((Dl, Dn))
        lab = []
        o = 0
        for q, rows, US, Vt in blocks:
            n = Vt.shape[0]
            B[o:o + n] = Vt
            C[np.ix_(rows, np.arange(o, o + n))] = US
            lab.extend([q] * n)
            o += n
        mps.A[c] = B.reshape(Dn, 4, Dr)
        mps.q[c] = np.array(lab, dtype=np.int64).reshape(-1, 2)
        mps.A[c - 1] = np.einsum("lsm,mn->lsn", mps.A[c - 1], C)
    return mps


def mps_from_vector(vec, nsite, tol=1e-14):
    """Exact left-to-right QN-blocked SVD of a vector on the 4^nsite space."""
    site_q = QN_SITE
    T = vec.reshape(1, -1)
    ql = np.zeros((1, 2), dtype=np.int64)
    A = []
    labels = [ql]
    for c in range(nsite - 1):
        Dl = T.shape[0]
        X = T.reshape(Dl * 4, -1)
        rq = (ql[:, None, :] + site_q[None, :, :]).reshape(-1, 2)
        keys = sorted({tuple(q) for q in rq})
        Us, rest, lab = [], [], []
        for q in keys:
            rows = np.nonzero(np.all(rq == q, axis=1))[0]
            U, S, Vt = np.linalg.svd(X[rows], full_matrices=False)
            keep = S > tol * max(S[0], 1e-300) if len(S) else np.zeros(0, bool)
            keep &= S > 0
            Us.append((rows, U[:, keep]))
            rest.append(S[keep, None] * Vt[keep])
            lab.extend([q] * int(keep.sum()))
        Dn = len(lab)
        U_full = np.zeros((Dl * 4, Dn))
        o = 0
        for rows, U in Us:
            U_full[np.ix_(rows, np.arange(o, o + U.shape[1]))] = U
            o += U.shape[1]
        A.append(U_full.reshape(Dl, 4, Dn))
        T = np.concatenate(rest, axis=0) if rest else np.zeros((0, X.shape[1]))
        ql = np.array(lab, dtype=np.int64).reshape(-1, 2)
        labels.append(ql)
    Dl = T.shape[0]
    rq = (ql[:, None, :] + site_q[None, :, :]).reshape(-1, 2)
    tot = rq[np.argmax(np.abs(T.reshape(-1)))]
    last = T.reshape(Dl, 4, 1).copy()
    last[~np.all(rq == tot, axis=1).reshape(Dl, 4)] = 0.0
    A.append(last)
    labels.append(tot.reshape(1, 2).copy())
    return MPS(A, labels)


def reference_mps(ci, k_act, k_virt):
    """Psi0 on the full chain: active FCI as an MPS, then empty virtual sites."""
    m = mps_from_vector(ci, k_act)
    tot = m.q[-1]
    for _ in range(k_virt):
        T = np.zeros((1, 4, 1))
        T[0, 0, 0] = 1.0
        m.A.append(T)
        m.q.append(tot.copy())
    return m


# ------------------------------------------------------------- contractions
def env_left(Lc, bra, W, ket, Dout):
    """L_{c+1}[b] = sum_a bra^T (W_ab x L_c[a]) ket  (transfer, O(M^3))."""
    Y = np.einsum("alr,rts->alts", Lc, ket, optimize=True)
    out = np.zeros((Dout, bra.shape[2], ket.shape[2]))
    Dl = bra.shape[0]
    Bm = bra.reshape(Dl * 4, -1)
    for (a, b), w in W.items():
        Z = np.einsum("st,ltr->lsr", w, Y[a], optimize=True)
        out[b] += Bm.T @ Z.reshape(Dl * 4, -1)
    return out


def env_right(Rc, bra, W, ket, Dout):
    """R_c[a] = sum_b bra (W_ab x R_{c+1}[b]) ket^T."""
    Y = np.einsum("rts,bls->brtl", ket, Rc, optimize=True)
    out = np.zeros((Dout, bra.shape[0], ket.shape[0]))
    Dr = bra.shape[2]
    Bm = bra.reshape(bra.shape[0], 4 * Dr)
    for (a, b), w in W.items():
        Z = np.einsum("st,rtl->rsl", w, Y[b], optimize=True)
        out[a] += Bm @ Z.reshape(Z.shape[0], 4 * Dr).T
    return out


def two_site_apply(L, W1, W2, R, x, Dmid):
    """sum_abc L_a (W1_ab x W2_bc) R_c applied to a two-site tensor (Fig. 1C)."""
    Y = np.einsum("alm,mtur->altur", L, x, optimize=True)
    Z = {}
    for (a, b), w in W1.items():
        v = np.einsum("st,ltur->lsur", w, Y[a], optimize=True)
        Z[b] = Z[b] + v if b in Z else v
    U = {}
    for (b, c), w in W2.items():
        if b not in Z:
            continue
        v = np.einsum("ut,lstr->lsur", w, Z[b], optimize=True)
        U[c] = U[c] + v if c in U else v
    out = np.zeros((L.shape[1],) + x.shape[1:3] + (R.shape[1],))
    for c, v in U.items():
        out += np.einsum("lsur,qr->lsuq", v, R[c], optimize=True)
    return out


def two_site_diag(L, W1, W2, R, shape, Dmid):
    dL = np.einsum("all->al", L)
    dR = np.einsum("crr->cr", R)
    D1 = np.zeros((Dmid, L.shape[1], 4))
    for (a, b), w in W1.items():
        D1[b] += dL[a][:, None] * np.diag(w)[None, :]
    out = np.zeros(shape)
    D2 = {}
    for (b, c), w in W2.items():
        v = np.diag(w)[:, None] * dR[c][None, :]
        D2[b] = D2[b] + v if b in D2 else v
    for b, v in D2.items():
        out += D1[b][:, :, None, None] * v[None, None, :, :]
    return out


def two_site_mask(ql, qr, allowed_mid):
    mid = ql[:, None, :] + QN_SITE[None, :, :]                     # (Dl, 4, 2)
    tot = mid[:, :, None, :] + QN_SITE[None, None, :, :]           # (Dl, 4, 4, 2)
    ok = np.all(tot[:, :, :, None, :] == qr[None, None, None, :, :], axis=-1)
    if allowed_mid is not None:
        okm = np.isin(mid[:, :, 0], list(allowed_mid))
        ok &= okm[:, :, None, None]
    return ok


# --------------------------------------------------------------------- CG
class NotSPD(RuntimeError):
    pass


def pcg(apply, b, x0, diag, mask, tol, maxit):
    """Jacobi-preconditioned CG for A x = b on the masked entries."""
    m = mask.astype(np.float64)
    inv = np.where(mask & (diag > 0), 1.0 / np.where(diag > 0, diag, 1.0), 0.0)
    x = x0 * m
    r = (b - apply(x)) * m
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return np.zeros_like(b), 0
    z = inv * r
    p = z.copy()
    rz = float(np.vdot(r, z))
    it = 0
    while np.linalg.norm(r) > tol * bn and it < maxit:
        Ap = apply(p) * m
        pAp = float(np.vdot(p, Ap))
        if pAp <= 0.0:
            raise NotSPD("p^T A p <= 0")
        alpha = rz / pAp
        x = x + alpha * p
        r = r - alpha * Ap
        z = inv * r
        rz_new = float(np.vdot(r, z))
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
    return x, it


# --------------------------------------------------------------- truncation
def select_states(evals, M, tr, keep_rel=None, tie_rel=1e-8):
    """Indices (sector, index) of kept density-matrix eigenvectors.

    evals: list of (qkey, eigenvalues descending).  Keeps the M largest
    eigenvalues above keep_rel * tr; if the M-th and (M+1)-th agree to
    tie_rel, the whole tied group at the cut is dropped (so degenerate
    multiplets are never split).  Ties of equal value order by QN key."""
    keep_rel = KEEP_REL if keep_rel is None else keep_rel
    cand = []
    for qkey, lam in evals:
        for i, v in enumerate(lam):
            if v > keep_rel * tr:
                cand.append((-float(v), qkey, i))
    cand.sort()
    m = min(M, len(cand))
    if m < len(cand):
        m0 = m
        while m > 0 and -cand[m - 1][0] <= -cand[m][0] * (1.0 + tie_rel):
            m -= 1
        if m == 0:
            m = m0
    kept = cand[:m]
    disc = tr - sum(-c[0] for c in kept)
    return [(c[1], c[2]) for c in kept], max(disc, 0.0) / tr if tr > 0 else 0.0


def truncate(x, ql, qr, M, direction, allowed_mid, keep_rel=None):
    """Split a two-site tensor.  Returns (A_left, A_right, labels_mid, w)."""
    Dl, _, _, Dr = x.shape
    if direction == "LR":
        X = x.reshape(Dl * 4, 4 * Dr)
        lab = (ql[:, None, :] + QN_SITE[None, :, :]).reshape(-1, 2)
        rho = X @ X.T
    else:
        X = x.reshape(Dl * 4, 4 * Dr)
        lab = (qr[None, :, :] - QN_SITE[:, None, :]).reshape(-1, 2)
        rho = X.T @ X
    keys = sorted({tuple(q) for q in lab})
    if allowed_mid is not None:
        keys = [q for q in keys if q[0] in allowed_mid]
    eig = {}
    evals = []
    tr = 0.0
    for q in keys:
        idx = np.nonzero(np.all(lab == q, axis=1))[0]
        w, v = np.linalg.eigh(rho[np.ix_(idx, idx)])
        w, v = w[::-1], v[:, ::-1]
        eig[q] = (idx, w, v)
        evals.append((q, w))
        tr += float(np.sum(w))
    kept, disc = select_states(evals, M, tr, keep_rel)
    kept.sort(key=lambda t: (t[0], t[1]))
    Dn = len(kept)
    U = np.zeros((X.shape[0] if direction == "LR" else X.shape[1], Dn))
    labn = np.zeros((Dn, 2), dtype=np.int64)
    for n, (q, i) in enumerate(kept):
        idx, w, v = eig[q]
        U[idx, n] = v[:, i]
        labn[n] = q
    if direction == "LR":
        Aleft = U.reshape(Dl, 4, Dn)
        Aright = (U.T @ X).reshape(Dn, 4, Dr)
    else:
        Aright = U.T.reshape(Dn, 4, Dr)
        Aleft = (X @ U).reshape(Dl, 4, Dn)
    return Aleft, Aright, labn, disc


# ------------------------------------------------------------------- sweep
class HylleraasSweep:
    """Two-site MPS-PT2 sweep on the full chain (active sites, then virtual)."""

    def __init__(self, prob, M, seed=1408, tol_cg=1e-10, tol_e=1e-10,
                 max_sweeps=30, cg_maxit=1000, mpo_A=None, mpo_V=None, verbose=False,
                 allowed=None, keep_rel=None):
        from .mpo import build_mpo
        self.prob = prob
        self.M = M
        self.k = prob.k
        self.tol_cg = tol_cg
        self.tol_e = tol_e
        self.max_sweeps = max_sweeps
        self.cg_maxit = cg_maxit
        self.verbose = verbose
        self.keep_rel = KEEP_REL if keep_rel is None else keep_rel
        N = prob.n_elec
        # bond filters: N_left allowed on given cuts (default: first-order space X)
        self.allowed = allowed if allowed is not None else {prob.k_act: {N - 1, N - 2}}
        self.WA = mpo_A or build_mpo(prob.h0_terms(), self.k, k_split=prob.k_act)
        self.WV = mpo_V or build_mpo(prob.rhs_terms(), self.k, k_split=prob.k_act)
        self.psi0 = reference_mps(prob.ci, prob.k_act, prob.k_virt)
        self.psi1 = canonicalize_by_splits(random_mps(self.k, (N, 0), self.allowed, M, seed), self.allowed,
                                           self.keep_rel)
        k = self.k
        self.LA = [None] * (k + 1)
        self.LV = [None] * (k + 1)
        self.RA = [None] * (k + 1)
        self.RV = [None] * (k + 1)
        one = np.ones((1, 1, 1))
        self.LA[0] = one
        self.LV[0] = one
        self.RA[k] = one
        self.RV[k] = one
        for c in range(k - 1, 0, -1):
            self._update_right(c)
        self.history = []
        self.discarded = []
        self.cg_iters = 0

    def _update_left(self, c):
        A = self.psi1.A[c]
        self.LA[c + 1] = env_left(self.LA[c], A, self.WA.W[c], A, self.WA.dims[c + 1])
        self.LV[c + 1] = env_left(self.LV[c], A, self.WV.W[c], self.psi0.A[c], self.WV.dims[c + 1])

    def _update_right(self, c):
        A = self.psi1.A[c]
        self.RA[c] = env_right(self.RA[c + 1], A, self.WA.W[c], A, self.WA.dims[c])
        self.RV[c] = env_right(self.RV[c + 1], A, self.WV.W[c], self.psi0.A[c], self.WV.dims[c])

    def local_problem(self, i):
        ps = self.psi1
        x0 = np.einsum("lsm,mtr->lstr", ps.A[i], ps.A[i + 1])
        ql, qr = ps.q[i], ps.q[i + 2]
        mask = two_site_mask(ql, qr, self.allowed.get(i + 1))
        p0 = np.einsum("lsm,mtr->lstr", self.psi0.A[i], self.psi0.A[i + 1])
        g = two_site_apply(self.LV[i], self.WV.W[i], self.WV.W[i + 1], self.RV[i + 2], p0,
                           self.WV.dims[i + 1]) * mask
        LA, RA = self.LA[i], self.RA[i + 2]
        W1, W2, Dm = self.WA.W[i], self.WA.W[i + 1], self.WA.dims[i + 1]

        def apply(v):
            return two_site_apply(LA, W1, W2, RA, v, Dm)

        diag = two_site_diag(LA, W1, W2, RA, x0.shape, Dm)
        return x0 * mask, g, apply, diag, mask

    def step(self, i, direction):
        x0, g, apply, diag, mask = self.local_problem(i)
        x, it = pcg(apply, -g, x0, diag, mask, self.tol_cg, self.cg_maxit)
        self.cg_iters += it
        h = float(np.vdot(x, apply(x) * mask) + 2.0 * np.vdot(x, g))
        ps = self.psi1
        Al, Ar, lab, w = truncate(x, ps.q[i], ps.q[i + 2], self.M, direction,
                                  self.allowed.get(i + 1), self.keep_rel)
        ps.A[i], ps.A[i + 1] = Al, Ar
        ps.q[i + 1] = lab
        self.discarded.append(w)
        if direction == "LR":
            self._update_left(i)
        else:
            self._update_right(i + 1)
        return h

    def sweep(self):
        k = self.k
        h = None
        for i in range(k - 1):
            h = self.step(i, "LR")
        for i in range(k - 2, -1, -1):
            h = self.step(i, "RL")
        return h

    def run(self):
        prev = None
        for n in range(self.max_sweeps):
            self.discarded = []
            e = self.sweep()
            self.history.append(e)
            if self.verbose:
                print(f"sweep {n}: E2 = {e:.12f}  max discarded {max(self.discarded):.3e}")
            if prev is not None and abs(e - prev) < self.tol_e:
                break
            prev = e
        self.e2 = self.history[-1]
        return self.e2


def expectation(bra, mpo, ket):
    """<bra|O|ket> by one left-to-right transfer (O(M^3) per site)."""
    L = np.ones((1, 1, 1))
    for c in range(bra.nsite):
        L = env_left(L, bra.A[c], mpo.W[c], ket.A[c], mpo.dims[c + 1])
    return float(L[0, 0, 0])


def overlap(bra, ket):
    L = np.ones((1, 1))
    for A, B in zip(bra.A, ket.A):
        L = np.einsum("lr,lsx,rsy->xy", L, A, B, optimize=True)
    return float(L[0, 0])


def third_order(sweep, mpo_H=None):
    """Eq. 5: E3 = <Psi1|V|Psi1> - E1 <Psi1|Psi1>, V = H - H0 on X.

    <Psi1|H0|Psi1> = <Psi1|A|Psi1> + E0 <Psi1|Psi1>, so
    E3 = <H> - <A> - (E0 + E1) <1> with the final bond-M Psi1."""
    from .mpo import build_mpo
    p = sweep.prob
    WH = mpo_H or build_mpo(p.hamiltonian_terms(), p.k, k_split=p.k_act)
    psi = sweep.psi1
    n2 = overlap(psi, psi)
    return expectation(psi, WH, psi) - expectation(psi, sweep.WA, psi) - (p.E0 + p.E1) * n2
