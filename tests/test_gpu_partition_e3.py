"""E3 over virtual-pair partitions on the GPU (every partition solved, written
on the full chain, Eq. 5 with the cross-partition pair elements) against the
oracle: Eq. 5 applied to the dense sum of the partition solutions on the tiny
system, the exact limit (the full-space E3*), and the transfer route on a
medium subset (tests/golden/oracle_medium_partition_e3_fock_M16.json)."""
import json
import os

import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny():
    h, L, c = synthetic.config_integrals("tiny")
    ci, _ = synthetic.fci_reference(h, L, c["k_act"], c["n_elec"])
    return h, L, c, ci


def _ctx(L, sysm, prec="fp64", keep_rel=None):
    h, Lc, c, ci = sysm
    o = L.mpspt_default_options()
    o.prec = L.PREC[prec]
    if keep_rel is not None:
        o.keep_rel = keep_rel
    ctx = L.mpspt_create(o)
    L.mpspt_set_integrals(ctx, c["k_act"], h.shape[0] - c["k_act"], c["n_elec"], h, Lc)
    L.mpspt_set_reference_ci(ctx, ci)
    return ctx


@pytest.mark.parametrize("h0", ["fock", "dyall"])
def test_partition_e3_matches_oracle_tiny(tiny, h0):
    """All 36 partitions of the tiny system at uneven, partly truncating M_P:
    E2 and E3 of every partition, every pair element <Psi1^i|H|Psi1^j> and
    the totals against the oracle's sweeps with Eq. 5 applied to the dense
    vectors; the result does not depend on the number of streams."""
    from oracle.brute import ExactFirstOrder, operator_matrix
    from oracle.operators import Problem
    from oracle.partition import e3_split, mps_vector, partition_psi1, partitions
    from paper_1408_5092_gb300 import _lib as L
    h, Lc, c, ci = tiny
    p = Problem(h, Lc, c["k_act"], c["n_elec"], ci, h0=h0)
    pairs = partitions(p.k_virt)
    Mof = {(a, b): 4 + (3 * a + 5 * b) % 9 for a, b in pairs}
    Ms = [Mof[x] for x in pairs]
    sp = partition_psi1(p, pairs, lambda a, b: Mof[(a, b)])
    ex = ExactFirstOrder(p)
    xs = [mps_vector(s, m, ex.X) for s, _, m in sp]
    tot, diag, cross = e3_split(p, ex.X, ex.A, xs)
    H = operator_matrix(p.hamiltonian_terms(), ex.X)
    G = np.array([[xi @ (H @ xj) for xj in xs] for xi in xs])
    np.fill_diagonal(G, 0.0)
    ctx = _ctx(L, tiny)
    e2, e3, e3x, e2p, e3p, hp, rep = L.mpspt_third_order_partitioned(ctx, h0, pairs, Ms, n_streams=4)
    n = len(pairs)
    assert np.max(np.abs(e2p - np.array([e for _, e, _ in sp]))) < 1e-8
    assert np.max(np.abs(e3p - np.array(diag))) < 1e-8
    assert np.max(np.abs(hp - G)) < 1e-8
    assert abs(e3x - cross) < 1e-8 and abs(e3 - tot) < 1e-8, (e3, tot, e3x, cross)
    assert abs(cross) > 1e-4
    assert rep.e3_transfers == 3 * n + n * (n - 1) // 2 and rep.e3_ms > 0.0
    _, e3b, _, _, _, hpb, _ = L.mpspt_third_order_partitioned(ctx, h0, pairs, Ms, n_streams=1)
    assert abs(e3b - e3) < 1e-13 and np.max(np.abs(hpb - hp)) < 1e-13
    L.mpspt_destroy(ctx)


def test_partition_e3_exact_limit_is_the_full_space_e3(tiny):
    """All partitions at their exact bond dimensions (keep threshold 1e-13):
    E2 and E3 of the partition sum equal the brute-force full-space E2*, E3*
    (float64 partition solves 1e-8, mixed 1e-6)."""
    from oracle.brute import ExactFirstOrder
    from oracle.operators import Problem
    from oracle.partition import partitions
    from paper_1408_5092_gb300 import _lib as L
    h, Lc, c, ci = tiny
    p = Problem(h, Lc, c["k_act"], c["n_elec"], ci, h0="fock")
    ex = ExactFirstOrder(p)
    e2_ex, e3_ex = ex.e2(), ex.e3()
    pairs = partitions(p.k_virt)
    for prec, tol in (("fp64", 1e-8), ("mixed", 1e-6)):
        ctx = _ctx(L, tiny, prec, keep_rel=1e-13)
        e2, e3, e3x, *_ = L.mpspt_third_order_partitioned(ctx, "fock", pairs, [64] * len(pairs), n_streams=8)
        assert abs(e2 - e2_ex) < tol and abs(e3 - e3_ex) < tol, (prec, e2, e2_ex, e3, e3_ex)
        L.mpspt_destroy(ctx)


def test_medium_partition_e3_matches_oracle():
    """Five partitions of the medium system (8e/8o + 24 virtual) at M_P = 16:
    E2, E3 of each, the ten pair elements and the totals against the oracle's
    transfer route (stored values)."""
    from paper_1408_5092_gb300 import _lib as L
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "oracle_medium_partition_e3_fock_M16.json")))
    pairs = [tuple(x) for x in gold["pairs"]]
    ctx = _ctx(L, synthetic.config_reference("medium"))
    e2, e3, e3x, e2p, e3p, hp, rep = L.mpspt_third_order_partitioned(ctx, gold["h0"], pairs,
                                                                     [gold["M"]] * len(pairs), n_streams=4)
    assert np.max(np.abs(e2p - np.array(gold["E2_part"]))) < 1e-8
    assert np.max(np.abs(e3p - np.array(gold["E3_part"]))) < 1e-8
    for i, j, v in gold["H_pair"]:
        assert abs(hp[i, j] - v) < 1e-8 and hp[i, j] == hp[j, i], (i, j, hp[i, j], v)
    assert abs(e3x - gold["E3_cross"]) < 1e-8 and abs(e3 - gold["E3"]) < 1e-8
    L.mpspt_destroy(ctx)
