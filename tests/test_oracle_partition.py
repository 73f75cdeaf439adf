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
