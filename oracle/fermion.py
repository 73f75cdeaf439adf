"""Site basis and Jordan-Wigner conventions (Fig. 1A: d = 4 per orbital).

Local states of one spatial orbital: 0 = |0>, 1 = |a>, 2 = |b>, 3 = |ab>,
with |ab> = c+_a c+_b |0>.  Spin-orbital index j = 2p + s (s = 0 alpha,
1 beta); many-body basis states are creators in ascending j applied to the
vacuum, so c_j carries the string prod_{i<j} (-1)^{n_i}.

Quantum numbers (N, 2Sz) per local state: (0,0), (1,1), (1,-1), (2,0).
Pinned by tests/test_oracle_mpo.py (MPO of a term list == brute-force
determinant operator, which applies the string definition literally).
"""
import numpy as np

D = 4
QN_N = np.array([0, 1, 1, 2])
QN_SZ = np.array([0, 1, -1, 0])

IDENT = np.eye(4)
PARITY = np.diag([1.0, -1.0, -1.0, 1.0])

_CRE = np.zeros((2, 4, 4))
# alpha creator: |0> -> |a>, |b> -> |ab>
_CRE[0][1, 0] = 1.0
_CRE[0][3, 2] = 1.0
# beta creator: |0> -> |b>, |a> -> c+_b c+_a|0> = -|ab>
_CRE[1][2, 0] = 1.0
_CRE[1][3, 1] = -1.0


def local_op(spin, dagger):
    """4x4 matrix of c+_{s} (dagger) or c_{s} on one site (site-internal sign)."""
    m = _CRE[spin]
    return m.copy() if dagger else m.T.copy()


def op_qn(spin, dagger):
    """(dN, d2Sz) of one elementary operator."""
    sgn = 1 if dagger else -1
    return sgn, sgn * (1 if spin == 0 else -1)
