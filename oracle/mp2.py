"""Closed-form second-order energy of a closed-shell single determinant.

With Psi0 a single determinant (all active orbitals doubly occupied) and the
Fock H0, the Hylleraas minimum (Eq. 1) is the textbook MP2 energy in the
semicanonical basis, plus a singles term because random orbitals break
Brillouin's theorem:
  E2 = sum_ijab (ia|jb)[2(ia|jb) - (ib|ja)] / (e_i + e_j - e_a - e_b)
       + 2 sum_ia f_ia^2 / (e_i - e_a).
This is a pin for the brute-force and MPS oracles, not part of the method.
"""
import numpy as np


def mp2_closed_form(h, L, n_occ):
    k = h.shape[0]
    eri = np.einsum("Qpq,Qrs->pqrs", L, L, optimize=True)
    o = slice(0, n_occ)
    f = h + 2.0 * np.einsum("pqjj->pq", eri[:, :, o, o]) - np.einsum("pjjq->pq", eri[:, o, o, :])
    eo, Uo = np.linalg.eigh(f[o, o])
    ev, Uv = np.linalg.eigh(f[n_occ:, n_occ:])
    C = np.zeros((k, k))
    C[o, o] = Uo
    C[n_occ:, n_occ:] = Uv
    f = C.T @ f @ C
    Lr = np.einsum("pi,Qpq,qj->Qij", C, L, C, optimize=True)
    ov = Lr[:, o, n_occ:]
    iajb = np.einsum("Qia,Qjb->iajb", ov, ov)
    denom = eo[:, None, None, None] - ev[None, :, None, None] + eo[None, None, :, None] - ev[None, None, None, :]
    e_d = np.sum(iajb * (2.0 * iajb - iajb.transpose(0, 3, 2, 1)) / denom)
    fia = f[o, n_occ:]
    e_s = 2.0 * np.sum(fia ** 2 / (eo[:, None] - ev[None, :]))
    return float(e_d + e_s)
