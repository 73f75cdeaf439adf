"""Reference wavefunction Psi0: lowest singlet of the active-space Hamiltonian.

The paper takes Psi0 as an input (a CASSCF/DMRG reference).  Here it is the
exact active-space FCI ground state of the seeded integrals, restricted to
<S^2> = 0.  The FCI uses an alpha-string x beta-string determinant basis and
spin-adapted excitation operators E_pq; it shares nothing with the oracle's
spin-orbital operator code, so the oracle can check it independently.
"""
import itertools
import os

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def _strings(norb, nel):
    out = []
    for occ in itertools.combinations(range(norb), nel):
        s = 0
        for p in occ:
            s |= 1 << p
        out.append(s)
    return np.array(sorted(out), dtype=np.int64)


def _popcount_below(s, p):
    return bin(s & ((1 << p) - 1)).count("1")


def _excitation_matrices(strings, norb):
    """E[p][q] = sparse matrix of a+_p a_q on one spin's string space."""
    index = {int(s): i for i, s in enumerate(strings)}
    n = len(strings)
    E = [[None] * norb for _ in range(norb)]
    for p in range(norb):
        for q in range(norb):
            rows, cols, vals = [], [], []
            for i, s in enumerate(strings):
                s = int(s)
                if not (s >> q) & 1:
                    continue
                sign = _popcount_below(s, q)
                t = s & ~(1 << q)
                if (t >> p) & 1:
                    continue
                sign += _popcount_below(t, p)
                t |= 1 << p
                rows.append(index[t])
                cols.append(i)
                vals.append(-1.0 if sign & 1 else 1.0)
            E[p][q] = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    return E


def _s_plus_norm2(vec, astr, bstr, norb):
    """<S^2> = |S+ psi|^2 for an Sz = 0 state (alpha-then-beta ordering)."""
    na = bin(int(astr[0])).count("1")
    acc = {}
    nb_str = len(bstr)
    for ia, sa in enumerate(astr):
        sa = int(sa)
        for ib, sb in enumerate(bstr):
            c = vec[ia * nb_str + ib]
            if c == 0.0:
                continue
            sb = int(sb)
            for p in range(norb):
                if not (sb >> p) & 1 or (sa >> p) & 1:
                    continue
                sign = na + _popcount_below(sb, p) + _popcount_below(sa, p)
                key = (sa | (1 << p), sb & ~(1 << p))
                acc[key] = acc.get(key, 0.0) + (-c if sign & 1 else c)
    return float(sum(v * v for v in acc.values()))


def fci_reference(h, L, k_act, n_elec, n_roots=8, s2_tol=1e-8):
    """Lowest singlet FCI state of the active block of (h, L).

    Returns (ci, energy) with ``ci`` a float64 vector of length 4**k_act in
    the site-occupation basis described in the package docstring.  No core
    orbitals: the active one-body operator is h restricted to the active
    block.
    """
    if n_elec % 2:
        raise ValueError("singlet reference needs an even electron count")
    nal = nbe = n_elec // 2
    h_a = h[:k_act, :k_act]
    L_a = L[:, :k_act, :k_act]
    eri = np.einsum("Qpq,Qrs->pqrs", L_a, L_a)
    astr = _strings(k_act, nal)
    bstr = _strings(k_act, nbe)
    Ea = _excitation_matrices(astr, k_act)
    Eb = _excitation_matrices(bstr, k_act)
    Ia = sp.identity(len(astr), format="csr")
    Ib = sp.identity(len(bstr), format="csr")
    E = [[sp.kron(Ea[p][q], Ib, format="csr") + sp.kron(Ia, Eb[p][q], format="csr")
          for q in range(k_act)] for p in range(k_act)]
    dim = len(astr) * len(bstr)
    H = sp.csr_matrix((dim, dim))
    # one-body part, with the two-body normal-ordering correction
    #   1/2 sum (pq|rs) (E_pq E_rs - delta_qr E_ps)
    k1 = h_a - 0.5 * np.einsum("pqqs->ps", eri)
    for p in range(k_act):
        for q in range(k_act):
            K = sp.csr_matrix((dim, dim))
            for r in range(k_act):
                for s in range(k_act):
                    if eri[p, q, r, s] != 0.0:
                        K = K + eri[p, q, r, s] * E[r][s]
            H = H + 0.5 * (E[p][q] @ K) + k1[p, q] * E[p][q]
    H = 0.5 * (H + H.T)
    if dim <= 3000:
        w, v = np.linalg.eigh(H.toarray())
    else:
        nr = min(n_roots, dim - 2)
        # seeded start vector: ARPACK otherwise draws a random one, and the
        # converged vector then differs between runs at the 1e-14 level
        v0 = np.random.Generator(np.random.PCG64(0)).normal(size=dim)
        w, v = spla.eigsh(H, k=nr, which="SA", tol=1e-14, maxiter=20000, v0=v0)
        order = np.argsort(w)
        w, v = w[order], v[:, order]
    chosen = None
    for i in range(min(n_roots, len(w))):
        if _s_plus_norm2(v[:, i], astr, bstr, k_act) < s2_tol:
            chosen = i
            break
    if chosen is None:
        raise RuntimeError("no singlet among the lowest roots; reseed")
    vec = v[:, chosen].copy()
    energy = float(w[chosen])
    # convert to the site-occupation basis, interleaved spin-orbital order
    ci = np.zeros(4 ** k_act)
    nb_str = len(bstr)
    for ia, sa in enumerate(astr):
        sa = int(sa)
        for ib, sb in enumerate(bstr):
            c = vec[ia * nb_str + ib]
            sb = int(sb)
            idx = 0
            for p in range(k_act):
                code = ((sa >> p) & 1) + 2 * ((sb >> p) & 1)
                idx = idx * 4 + code
            swaps = 0
            for p in range(k_act):
                if (sb >> p) & 1:
                    swaps += bin(sa >> (p + 1)).count("1")
            ci[idx] = -c if swaps & 1 else c
    ci /= np.linalg.norm(ci)
    imax = int(np.argmax(np.abs(ci)))
    if ci[imax] < 0:
        ci = -ci
    return ci, energy


_DATA = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")


def stored_reference_path(name, seed):
    return os.path.join(_DATA, f"{name}_seed{seed}_psi0.npz")


def config_reference(name, seed=None):
    """(h, L, config, ci) of a named workload.

    The reference vector is read from ``synthetic/data`` when a stored copy
    of (name, seed) exists (written by ``python -m synthetic.store_reference``
    from fci_reference).  LAPACK/ARPACK round differently on different
    machines and BLAS builds, and sweep energies at medium size respond to
    1e-14 changes of Psi0 at the 1e-9 level, so every machine that compares
    against stored oracle values must start from the same bits."""
    from .integrals import EVAL_SEED, config_integrals
    seed = EVAL_SEED if seed is None else seed
    h, L, c = config_integrals(name, seed=seed)
    path = stored_reference_path(name, seed)
    if os.path.exists(path):
        z = np.load(path)
        ci = np.zeros(4 ** c["k_act"])
        ci[z["idx"]] = z["val"]
    else:
        ci, _ = fci_reference(h, L, c["k_act"], c["n_elec"])
    return h, L, c, ci
