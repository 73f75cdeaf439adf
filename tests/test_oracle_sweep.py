"""MPS-PT2 sweep oracle: upper bound and exactness at the exact bond dimension
(the large-M limit recovers the uncontracted energy), E3 by Eq. 5."""
import numpy as np
import pytest

import synthetic
from oracle.brute import ExactFirstOrder
from oracle.mps import HylleraasSweep, third_order
from oracle.operators import Problem


@pytest.fixture(scope="module")
def tiny():
    h, L, c = synthetic.config_integrals("tiny")
    ci, _ = synthetic.fci_reference(h, L, c["k_act"], c["n_elec"])
    out = {}
    for h0 in ("fock", "dyall"):
        p = Problem(h, L, c["k_act"], c["n_elec"], ci, h0=h0)
        ex = ExactFirstOrder(p)
        out[h0] = (p, ex, max(ex.schmidt_ranks()))
    return out


@pytest.mark.parametrize("h0", ["fock", "dyall"])
def test_exact_at_full_bond_dimension(tiny, h0):
    p, ex, m_exact = tiny[h0]
    sw = HylleraasSweep(p, m_exact)
    assert abs(sw.run() - ex.e2()) < 1e-9
    if h0 == "fock":
        assert abs(third_order(sw) - ex.e3()) < 1e-9


def test_upper_bound_and_monotone_in_m(tiny):
    p, ex, _ = tiny["fock"]
    e16 = HylleraasSweep(p, 16).run()
    e32 = HylleraasSweep(p, 32).run()
    assert e16 >= e32 - 1e-10
    assert e32 >= ex.e2() - 1e-10
    assert e16 - ex.e2() > 1e-4      # M = 16 really truncates
