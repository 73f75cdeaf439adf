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
    # keep threshold at the rounding level: the sweep reproduces the
    # uncontracted E2* and E3* (the large-M limit of the paper)
    sw = HylleraasSweep(p, m_exact, keep_rel=1e-13)
    assert abs(sw.run() - ex.e2()) < 1e-9
    assert abs(third_order(sw) - ex.e3()) < 1e-9
    # reading R7's threshold (1e-10 tr rho) drops Schmidt states of weight
    # below it: E2 stays an upper bound and moves by O(weight) (Eq. 1 is
    # quadratic about its minimum), E3 by O(sqrt(weight)) (Eq. 5 is not
    # stationary)
    sw = HylleraasSweep(p, m_exact)
    e2 = sw.run()
    assert -1e-12 <= e2 - ex.e2() < 1e-9
    assert abs(third_order(sw) - ex.e3()) < 1e-7


def test_upper_bound_and_monotone_in_m(tiny):
    p, ex, _ = tiny["fock"]
    e16 = HylleraasSweep(p, 16).run()
    e32 = HylleraasSweep(p, 32).run()
    assert e16 >= e32 - 1e-10
    assert e32 >= ex.e2() - 1e-10
    assert e16 - ex.e2() > 1e-4      # M = 16 really truncates


def test_initial_state_canonicalisation():
    """Reading R8: the seeded random MPS is made right-canonical by
    right-to-left density-matrix splits (no M cap, states above 1e-10 tr rho
    kept).  The state changes only by the dropped directions (relative norm
    below sqrt of their weight), every site but the first is right-
    orthonormal, and no bond grows."""
    import numpy as np
    from oracle.mps import canonicalize_by_splits, random_mps
    k, N = 8, 4
    allowed = {4: {N - 1, N - 2}}
    m0 = random_mps(k, (N, 0), allowed, 12, 1408)
    before = m0.to_dense().copy()
    dims0 = m0.dims()
    m1 = canonicalize_by_splits(random_mps(k, (N, 0), allowed, 12, 1408), allowed)
    after = m1.to_dense()
    rel = np.linalg.norm(after - before) / np.linalg.norm(before)
    assert rel < 1e-6, rel
    for A in m1.A[1:]:
        X = A.reshape(A.shape[0], -1)
        assert np.abs(X @ X.T - np.eye(A.shape[0])).max() < 1e-12
    assert all(d1 <= d0 for d0, d1 in zip(dims0, m1.dims()))


def test_partition_bond_dims_are_seeded_and_in_range():
    import synthetic
    a = synthetic.partition_bond_dims(1830)
    b = synthetic.partition_bond_dims(1830)
    assert a == b and len(a) == 1830
    assert set(a) <= {32, 64, 128, 256, 512} and len(set(a)) == 5


def test_splitmix64_reproduces_the_published_stream():
    """Reading R8 keys the initial Psi1 entries by SplitMix64 (Steele, Lea,
    Flood 2014).  The generator's first outputs from state 0 are its
    published reference values; the oracle's function maps the state
    before the increment to the output."""
    from oracle.mps import init_value, splitmix64
    gamma = 0x9E3779B97F4A7C15
    mask = (1 << 64) - 1
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    assert [splitmix64((i * gamma) & mask) for i in range(4)] == want
    # entries are u * 2^-53 - 0.5 with u the top 53 bits: in [-0.5, 0.5)
    v = [init_value(1408, c, s, l, r) for c in range(3) for s in range(4) for l in range(3) for r in range(3)]
    assert min(v) >= -0.5 and max(v) < 0.5 and len(set(v)) == len(v)
    assert init_value(1408, 0, 0, 0, 0) == (splitmix64(1408 << 48) >> 11) * 2.0 ** -53 - 0.5
