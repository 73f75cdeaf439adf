"""E2(M) and its extrapolation in the discarded weight (oracle): upper bounds,
a bounded slope, and the line's intercept against the uncontracted E2*
(the exact limit itself is pinned in test_oracle_sweep.py)."""
import numpy as np
import pytest

import synthetic
from oracle.brute import ExactFirstOrder
from oracle.extrapolate import extrapolate_e2
from oracle.operators import Problem


@pytest.mark.parametrize("h0", ["fock"])
def test_points_bound_e2_star_and_the_line_recovers_it(h0):
    h, L, c = synthetic.config_integrals("tiny")
    ci, _ = synthetic.fci_reference(h, L, c["k_act"], c["n_elec"])
    p = Problem(h, L, c["k_act"], c["n_elec"], ci, h0=h0)
    ex = ExactFirstOrder(p)
    e_star = ex.e2()
    # the small-truncation regime (discarded weight 1e-6 .. 3e-4 here), where
    # the paper finds E2 linear in the discarded weight
    Ms = (20, 26, 32, 36)
    a, b, e2, w = extrapolate_e2(p, Ms)
    assert all(e >= e_star - 1e-10 for e in e2)                 # Eq. 1 minimum: upper bounds
    assert all(x > 0 for x in w) and w[0] > w[-1]
    assert b > 0                                                # more truncation, higher E2
    ratio = (np.array(e2) - e_star) / np.array(w)               # roughly linear: a bounded slope
    assert ratio.min() > 0.2 and ratio.max() < 10, ratio
    # the intercept moves towards E2*: well inside the first point's error
    assert abs(a - e_star) < 0.2 * (e2[0] - e_star), (a - e_star, e2[0] - e_star)
