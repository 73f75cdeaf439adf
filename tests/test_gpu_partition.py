"""Partitioned E2 on the GPU (virtual-pair partitions run concurrently on
several streams) against the oracle's partition sweeps, and the exact limit
against the brute-force sum."""
import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny():
    h, L, c = synthetic.config_integrals("tiny")
    ci, _ = synthetic.fci_reference(h, L, c["k_act"], c["n_elec"])
    return h, L, c, ci


def _ctx(L, tiny, prec="fp64"):
    h, Lc, c, ci = tiny
    o = L.mpspt_default_options()
    o.prec = L.PREC[prec]
    ctx = L.mpspt_create(o)
    L.mpspt_set_integrals(ctx, c["k_act"], h.shape[0] - c["k_act"], c["n_elec"], h, Lc)
    L.mpspt_set_reference_ci(ctx, ci)
    return ctx


@pytest.mark.parametrize("h0", ["fock", "dyall"])
def test_partitioned_e2_matches_oracle(tiny, h0):
    from oracle.mps import HylleraasSweep
    from oracle.operators import Problem
    from oracle.partition import SubProblem, partitions
    from paper_1408_5092_gb300 import _lib as L
    h, Lc, c, ci = tiny
    p = Problem(h, Lc, c["k_act"], c["n_elec"], ci, h0=h0)
    pairs = partitions(p.k_virt)
    Ms = [4 + (3 * a + 5 * b) % 9 for a, b in pairs]     # uneven, some truncating
    ref = []
    for (a, b), M in zip(pairs, Ms):
        sub = SubProblem(p, a, b)
        ref.append(HylleraasSweep(sub, M, allowed=sub.allowed).run())
    ctx = _ctx(L, tiny)
    tot, ep, rep = L.mpspt_minimize_partitioned(ctx, h0, pairs, Ms, n_streams=4)
    assert np.max(np.abs(ep - np.array(ref))) < 1e-8
    assert abs(tot - sum(ref)) < 1e-8
    L.mpspt_destroy(ctx)


def test_partitioned_exact_limit_equals_brute_force(tiny):
    from oracle.brute import ExactFirstOrder
    from oracle.operators import Problem
    from oracle.partition import partitions
    from paper_1408_5092_gb300 import _lib as L
    h, Lc, c, ci = tiny
    p = Problem(h, Lc, c["k_act"], c["n_elec"], ci, h0="fock")
    e_ex = ExactFirstOrder(p).e2()
    pairs = partitions(p.k_virt)
    for prec in ("fp64", "mixed"):
        ctx = _ctx(L, tiny, prec)
        tot, ep, rep = L.mpspt_minimize_partitioned(ctx, "fock", pairs, [64] * len(pairs), n_streams=8)
        assert abs(tot - e_ex) < (1e-9 if prec == "fp64" else 1e-6), (prec, tot, e_ex)
        L.mpspt_destroy(ctx)


def test_medium_partitions_match_oracle():
    """Virtual-pair partitions of the medium system (8e/8o + 24 virtual; the
    sub-chains carry the exact M0 = 256 reference) at M_P = 16 against the
    oracle's partition sweeps (tests/golden/oracle_medium_partitions_fock_M16.json),
    run concurrently on four streams."""
    import json
    import os
    from paper_1408_5092_gb300 import _lib as L
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "oracle_medium_partitions_fock_M16.json")))
    h, Lc, c, ci = synthetic.config_reference("medium")
    o = L.mpspt_default_options()
    ctx = L.mpspt_create(o)
    L.mpspt_set_integrals(ctx, c["k_act"], h.shape[0] - c["k_act"], c["n_elec"], h, Lc)
    L.mpspt_set_reference_ci(ctx, ci)
    pairs = [(p["a"], p["b"]) for p in gold["parts"]]
    tot, ep, rep = L.mpspt_minimize_partitioned(ctx, "fock", pairs, [gold["M"]] * len(pairs), n_streams=4)
    ref = np.array([p["E2"] for p in gold["parts"]])
    assert np.max(np.abs(ep - ref)) < 1e-8, (ep, ref)
    L.mpspt_destroy(ctx)
