"""E2 against the truncation error (TEST INFRASTRUCTURE ONLY).

The paper studies the convergence of the MPS-PT2 energy with the bond
dimension M and extrapolates it linearly in the discarded weight of the
renormalisation step (Figs. 3-4 and the surrounding text).  This restates
that study: one HylleraasSweep per M (same seeded start, reading R8), w(M) =
the largest discarded weight of the last sweep, and the least-squares line
E2 = a + b w (numpy.polyfit, degree 1); a is the extrapolated E2.

Pinned by tests/test_oracle_extrapolate.py: every point is an upper bound to
the uncontracted E2*, w vanishes at the exact bond dimension where E2 = E2*,
and the line through the points recovers E2* within the spread of the
points about it.
"""
import numpy as np

from .mps import HylleraasSweep


def extrapolate_e2(prob, Ms, **sweep_kwargs):
    e2, w = [], []
    for M in Ms:
        sw = HylleraasSweep(prob, M, **sweep_kwargs)
        e2.append(sw.run())
        w.append(max(sw.discarded))
    b, a = np.polyfit(np.array(w), np.array(e2), 1)
    return float(a), float(b), e2, w
