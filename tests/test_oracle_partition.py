"""Partitioned first-order problem: E2* = sum over virtual-pair partitions
(exact, because H0 conserves every virtual occupation), and the MPS sweep of
a partition at its exact bond dimension reproduces E2*_P."""
import numpy as np
import pytest

import synthetic
from oracle.brute import ExactFirstOrder
from oracle.mps import HylleraasSweep
from oracle.operators import Problem
from oracle.partition import ExactPartition, SubProblem, partitions


@pytest.fixture(scope="module")
def tiny():
    h, L, c = synthetic.config_integrals("tiny")
    ci, _ = synthetic.fci_reference(h, L, c["k_act"], c["n_elec"])
    return h, L, c, ci


def test_partition_count():
    assert len(partitions(60)) == 1830
    assert len(partitions(160)) == 12880
    assert len(partitions(8)) == 36


@pytest.mark.parametrize("h0", ["fock", "dyall"])
def test_partition_sum_is_exact(tiny, h0):
    h, L, c, ci = tiny
    p = Problem(h, L, c["k_act"], c["n_elec"], ci, h0=h0)
    full = ExactFirstOrder(p).e2()
    tot = 0.0
    for a, b in partitions(p.k_virt):
        tot += ExactPartition(SubProblem(p, a, b)).e2()
    assert abs(tot - full) < 1e-12


@pytest.mark.parametrize("pair", [(0, 0), (1, 5), (7, 7)])
def test_partition_sweep_reaches_exact(tiny, pair):
    h, L, c, ci = tiny
    p = Problem(h, L, c["k_act"], c["n_elec"], ci, h0="fock")
    sub = SubProblem(p, *pair)
    e_ex = ExactPartition(sub).e2()
    sw = HylleraasSweep(sub, 40, allowed=sub.allowed)
    assert abs(sw.run() - e_ex) < 1e-10


@pytest.mark.parametrize("h0", ["fock", "dyall"])
def test_partition_e3_exact_limit_is_the_full_space_e3(tiny, h0):
    """Eq. 5 for the sum of the exact partition solutions: the embedded
    vectors add up to the full-space Psi1*, their E3 is the full-space E3*,
    the cross-partition part is a sizeable share of it (so a dropped cross
    term fails), and distinct partitions are orthogonal with no H0 coupling."""
    from oracle.partition import e3_split, embed_vector
    h, L, c, ci = tiny
    p = Problem(h, L, c["k_act"], c["n_elec"], ci, h0=h0)
    ex = ExactFirstOrder(p)
    ex.solve()
    xs = []
    for a, b in partitions(p.k_virt):
        sub = SubProblem(p, a, b)
        ep = ExactPartition(sub)
        xs.append(embed_vector(sub, ep.X.dets, ep.solve(), ex.X))
    assert np.abs(np.sum(xs, axis=0) - ex.psi1).max() < 1e-13
    tot, diag, cross = e3_split(p, ex.X, ex.A, xs)
    e3 = ex.e3()
    assert abs(tot - e3) < 1e-12
    assert abs(cross) > 0.1 * abs(e3)
    for i, j in [(0, 1), (0, 8), (3, 20), (35, 34)]:
        assert xs[i] @ xs[j] == 0.0
        assert abs(xs[i] @ (ex.A @ xs[j])) < 1e-15


def test_partition_e3_transfer_route_equals_plain_definition(tiny):
    """The transfer route (partition MPSs written on the full chain, one MPO
    transfer per term) against Eq. 5 applied to the dense sum, on truncated
    partition MPSs (Dyall H0): total, each E3(Psi1^P) and each
    <Psi1^P|H|Psi1^P'>."""
    from oracle.brute import operator_matrix
    from oracle.partition import e3_split, mps_vector, partition_e3_mps, partition_psi1
    h, L, c, ci = tiny
    p = Problem(h, L, c["k_act"], c["n_elec"], ci, h0="dyall")
    ex = ExactFirstOrder(p)
    pairs = [(0, 0), (0, 1), (1, 3), (3, 3)]
    sp = partition_psi1(p, pairs, lambda a, b: 4 + (3 * a + 5 * b) % 5)
    tot, diag, cross, hh = partition_e3_mps(p, [(s, m) for s, _, m in sp])
    xs = [mps_vector(s, m, ex.X) for s, _, m in sp]
    tot_d, diag_d, cross_d = e3_split(p, ex.X, ex.A, xs)
    assert abs(tot - tot_d) < 1e-12
    assert np.abs(np.array(diag) - np.array(diag_d)).max() < 1e-12
    assert abs(cross - cross_d) < 1e-12
    H = operator_matrix(p.hamiltonian_terms(), ex.X)
    for (i, j), v in hh.items():
        assert abs(v - xs[i] @ (H @ xs[j])) < 1e-12
    assert max(abs(v) for v in hh.values()) > 1e-4
