"""GPU library vs the CPU oracle on the same seeded inputs.

Local operators (Fig. 1C terms) are compared element by element on a shared
Psi1; energies (E2, E3) at equal bond dimension against stored oracle values
(tests/golden/make_golden.py) to 1e-8 Eh (float64 path)."""
import json
import os

import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "oracle_tiny.json")


@pytest.fixture(scope="module")
def L():
    from paper_1408_5092_gb300 import _lib
    _lib.load()
    return _lib


@pytest.fixture(scope="module")
def tiny():
    h, Lc, c = synthetic.config_integrals("tiny")
    ci, _ = synthetic.fci_reference(h, Lc, c["k_act"], c["n_elec"])
    return h, Lc, c, ci


@pytest.fixture(scope="module")
def gold():
    with open(GOLD) as f:
        return json.load(f)


def _session(L, tiny, **opts):
    h, Lc, c, ci = tiny
    o = L.mpspt_default_options()
    for k, v in opts.items():
        setattr(o, k, v)
    ctx = L.mpspt_create(o)
    L.mpspt_set_integrals(ctx, c["k_act"], h.shape[0] - c["k_act"], c["n_elec"], h, Lc)
    L.mpspt_set_reference_ci(ctx, ci)
    return ctx


@pytest.mark.parametrize("h0", ["fock", "dyall"])
def test_reference_energies(L, tiny, gold, h0):
    ctx = _session(L, tiny)
    e0, e1, eref = L.mpspt_energies(ctx, h0)
    g = gold["h0"][h0]
    assert abs(eref - g["E_ref"]) < 1e-11
    assert abs(e0 - g["E0"]) < 1e-11
    assert abs(e1 - g["E1"]) < 1e-11
    L.mpspt_destroy(ctx)


@pytest.mark.parametrize("h0", ["fock", "dyall"])
def test_local_operators_match_oracle(L, tiny, h0):
    from oracle.mps import HylleraasSweep, two_site_apply, two_site_diag, two_site_mask
    from oracle.operators import Problem
    h, Lc, c, ci = tiny
    p = Problem(h, Lc, c["k_act"], c["n_elec"], ci, h0=h0)
    sw = HylleraasSweep(p, 24, seed=7)
    ctx = _session(L, tiny)
    psi = L.mpspt_mps_import(ctx, sw.psi1.A, sw.psi1.q)
    rng = np.random.default_rng(3)
    for i in range(p.k - 1):
        # oracle environments for bond i from the shared Psi1
        for s in range(i):
            sw._update_left(s)
        ql, qr = sw.psi1.q[i], sw.psi1.q[i + 2]
        mask = two_site_mask(ql, qr, sw.allowed.get(i + 1))
        x = rng.normal(size=mask.shape) * mask
        ref_sig = two_site_apply(sw.LA[i], sw.WA.W[i], sw.WA.W[i + 1], sw.RA[i + 2], x, sw.WA.dims[i + 1]) * mask
        p0 = np.einsum("lsm,mtr->lstr", sw.psi0.A[i], sw.psi0.A[i + 1])
        ref_g = two_site_apply(sw.LV[i], sw.WV.W[i], sw.WV.W[i + 1], sw.RV[i + 2], p0, sw.WV.dims[i + 1]) * mask
        ref_d = two_site_diag(sw.LA[i], sw.WA.W[i], sw.WA.W[i + 1], sw.RA[i + 2], x.shape, sw.WA.dims[i + 1]) * mask
        got_sig = L.mpspt_local_apply(ctx, h0, psi, i, L.MPSPT_LOCAL_SIGMA, x, x.shape)
        got_g = L.mpspt_local_apply(ctx, h0, psi, i, L.MPSPT_LOCAL_RHS, None, x.shape)
        got_d = L.mpspt_local_apply(ctx, h0, psi, i, L.MPSPT_LOCAL_DIAG, None, x.shape)
        scale = max(1.0, np.abs(ref_sig).max())
        assert np.abs(got_sig - ref_sig).max() < 1e-12 * scale, i
        assert np.abs(got_g - ref_g).max() < 1e-12 * max(1.0, np.abs(ref_g).max()), i
        assert np.abs(got_d - ref_d).max() < 1e-12 * max(1.0, np.abs(ref_d).max()), i
        # reset the oracle's left environments for the next bond
        sw.LA[1:] = [None] * (len(sw.LA) - 1)
        sw.LV[1:] = [None] * (len(sw.LV) - 1)
    L.mpspt_mps_free(psi)
    L.mpspt_destroy(ctx)


@pytest.mark.parametrize("h0", ["fock", "dyall"])
@pytest.mark.parametrize("which", ["16", "32", "exact"])
def test_e2_e3_match_oracle(L, tiny, gold, h0, which):
    g = gold["h0"][h0]
    M = g["M_exact"] if which == "exact" else int(which)
    run = g["runs"][str(M)]
    ctx = _session(L, tiny)
    e2, psi, rep = L.mpspt_minimize_hylleraas(ctx, h0, M)
    assert abs(e2 - run["E2"]) < 1e-8, (e2, run["E2"])
    assert e2 >= g["E2_exact"] - 1e-10          # upper bound (Eq. 1 minimum)
    e3 = L.mpspt_third_order(ctx, h0, psi)
    assert abs(e3 - run["E3"]) < 1e-8, (e3, run["E3"])
    if which == "exact":
        # reading R7 drops Schmidt states below 1e-10 tr rho: E2 moves by
        # O(weight), E3 by O(sqrt(weight)); at a rounding-level threshold the
        # uncontracted E2*, E3* are reproduced
        assert abs(e2 - g["E2_exact"]) < 1e-9
        assert abs(e3 - g["E3_exact"]) < 1e-7
    assert rep.max_bond_dim <= M
    L.mpspt_mps_free(psi)
    L.mpspt_destroy(ctx)
    if which == "exact":
        ctx = _session(L, tiny, keep_rel=1e-13)
        e2, psi, rep = L.mpspt_minimize_hylleraas(ctx, h0, M)
        assert abs(e2 - g["E2_exact"]) < 1e-9, (e2, g["E2_exact"])
        assert abs(L.mpspt_third_order(ctx, h0, psi) - g["E3_exact"]) < 1e-9
        L.mpspt_mps_free(psi)
        L.mpspt_destroy(ctx)


@pytest.mark.parametrize("h0", ["fock", "dyall"])
def test_eigensolver_paths_agree(L, tiny, gold, h0):
    """The truncation's eigen-decomposition (Eq. 6 density matrix) has two
    paths: float32 Jacobi + float64 Newton-Schulz + float64 Jacobi polish
    (default), and float64 Jacobi from the identity.  Both give the oracle's
    E2, and the kept states are orthonormal: after the closing right-to-left
    half sweep every site but the first is right-orthonormal."""
    run = gold["h0"][h0]["runs"]["16"]
    e2s = []
    for fp64_only in (0, 1):
        ctx = _session(L, tiny, eig_fp64_only=fp64_only)
        e2, psi, rep = L.mpspt_minimize_hylleraas(ctx, h0, 16)
        assert abs(e2 - run["E2"]) < 1e-8, (fp64_only, e2, run["E2"])
        ts, _ = L.mpspt_mps_export(psi)
        for A in ts[1:]:
            m = A.reshape(A.shape[0], -1)
            assert np.abs(m @ m.T - np.eye(A.shape[0])).max() < 1e-12
        e2s.append(e2)
        L.mpspt_mps_free(psi)
        L.mpspt_destroy(ctx)
    assert abs(e2s[0] - e2s[1]) < 1e-10, e2s


def test_errors_are_statuses_not_crashes(L, tiny):
    h, Lc, c, ci = tiny
    ctx = L.mpspt_create()
    with pytest.raises(L.MpsptError) as e:
        L.mpspt_minimize_hylleraas(ctx, "fock", 16)
    assert e.value.status == -7                 # STATE: no integrals / reference
    L.mpspt_set_integrals(ctx, c["k_act"], h.shape[0] - c["k_act"], c["n_elec"], h, Lc)
    with pytest.raises(L.MpsptError) as e:
        L.mpspt_set_reference_ci(ctx, ci[:-1])
    assert e.value.status == -1
    bad = ci.copy()
    bad[np.argmax(np.abs(bad))] = np.nan
    with pytest.raises(L.MpsptError):
        L.mpspt_set_reference_ci(ctx, bad)
    L.mpspt_set_reference_ci(ctx, ci)
    with pytest.raises(L.MpsptError) as e:
        L.mpspt_minimize_hylleraas(ctx, "fock", 0)
    assert e.value.status == -1
    L.mpspt_destroy(ctx)


def test_bond_dimension_one_is_an_upper_bound(L, tiny, gold):
    """Degenerate M = 1: a valid (poor) variational state, still above E2*."""
    ctx = _session(L, tiny, max_sweeps=4)
    e2, psi, rep = L.mpspt_minimize_hylleraas(ctx, "fock", 1)
    assert e2 >= gold["h0"]["fock"]["E2_exact"] - 1e-10
    assert rep.max_bond_dim == 1
    L.mpspt_mps_free(psi)
    L.mpspt_destroy(ctx)


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("mixed", 2e-4)])
def test_low_precision_sigma_matches_oracle(L, tiny, prec, tol):
    """Inner operator of the refined CG: float32 CUDA cores / split-bf16
    tensor cores.  Relative max-norm error bounded by the arithmetic:
    float32 keeps 24 bits (2^-24 ~ 6e-8 per product, summed over the
    K-lists); the three-term bf16 split keeps about 16 bits
    (3 x 2^-17 ~ 2.3e-5 per product).  The environments here come from a
    right-canonical state, so left environments are not normalised: their
    entries span many decades, which float32 and bfloat16 exponents cover."""
    from oracle.mps import HylleraasSweep, two_site_apply, two_site_mask
    from oracle.operators import Problem
    h, Lc, c, ci = tiny
    p = Problem(h, Lc, c["k_act"], c["n_elec"], ci, h0="dyall")
    sw = HylleraasSweep(p, 32, seed=11)
    ctx = _session(L, tiny, prec=L.PREC[prec])
    psi = L.mpspt_mps_import(ctx, sw.psi1.A, sw.psi1.q)
    rng = np.random.default_rng(5)
    worst = 0.0
    for i in (0, 2, 3, 4, 6, 10):
        for s in range(i):
            sw._update_left(s)
        mask = two_site_mask(sw.psi1.q[i], sw.psi1.q[i + 2], sw.allowed.get(i + 1))
        x = rng.normal(size=mask.shape) * mask
        ref = two_site_apply(sw.LA[i], sw.WA.W[i], sw.WA.W[i + 1], sw.RA[i + 2], x, sw.WA.dims[i + 1]) * mask
        got = L.mpspt_local_apply(ctx, "dyall", psi, i, L.MPSPT_LOCAL_SIGMA, x, x.shape)
        err = np.abs(got - ref).max() / np.abs(ref).max()
        worst = max(worst, err)
        sw.LA[1:] = [None] * (len(sw.LA) - 1)
        sw.LV[1:] = [None] * (len(sw.LV) - 1)
    assert worst < tol, worst
    L.mpspt_mps_free(psi)
    L.mpspt_destroy(ctx)


def test_fp16_sigma_on_the_sweep_environments(L, tiny):
    """Split-f16 sigma (11-bit significands, three products ~ 22 bits) at the
    environments the sweep itself uses: mixed-canonical at the bond (left
    sites left-orthonormal, right sites right-orthonormal), whose entries
    stay inside the f16 exponent range.  Relative max-norm error against the
    float64 oracle below 2e-5 (about 2^-22 per product summed over the
    K-lists, an order above the bf16 split's 2e-4)."""
    from oracle.mps import HylleraasSweep, two_site_apply, two_site_mask
    from oracle.operators import Problem
    h, Lc, c, ci = tiny
    p = Problem(h, Lc, c["k_act"], c["n_elec"], ci, h0="dyall")
    sw = HylleraasSweep(p, 32, seed=11)
    for i in range(p.k - 1):            # left-to-right half sweep: all sites left-orthonormal
        sw.step(i, "LR")
    ctx = _session(L, tiny, prec=L.MPSPT_MIXED_FP16)
    rng = np.random.default_rng(5)
    worst = 0.0
    for i in range(p.k - 2, -1, -1):    # right-to-left: bond i is mixed-canonical before its step
        if i in (9, 6, 4, 2, 0):
            psi = L.mpspt_mps_import(ctx, sw.psi1.A, sw.psi1.q)
            mask = two_site_mask(sw.psi1.q[i], sw.psi1.q[i + 2], sw.allowed.get(i + 1))
            x = rng.normal(size=mask.shape) * mask
            ref = two_site_apply(sw.LA[i], sw.WA.W[i], sw.WA.W[i + 1], sw.RA[i + 2], x, sw.WA.dims[i + 1]) * mask
            got = L.mpspt_local_apply(ctx, "dyall", psi, i, L.MPSPT_LOCAL_SIGMA, x, x.shape)
            worst = max(worst, np.abs(got - ref).max() / np.abs(ref).max())
            L.mpspt_mps_free(psi)
        sw.step(i, "RL")
    assert worst < 2e-5, worst
    L.mpspt_destroy(ctx)


@pytest.mark.parametrize("prec", ["fp32", "mixed", "mixed_fp16"])
@pytest.mark.parametrize("h0", ["fock", "dyall"])
def test_refined_e2_matches_oracle(L, tiny, gold, prec, h0):
    """Float64-refined CG with a low-precision inner operator: E2 and E3 to
    1e-6 Eh of the float64 oracle at equal M (the Hylleraas value itself is
    evaluated with a float64 sigma)."""
    g = gold["h0"][h0]
    run = g["runs"]["32"]
    ctx = _session(L, tiny, prec=L.PREC[prec])
    e2, psi, rep = L.mpspt_minimize_hylleraas(ctx, h0, 32)
    assert abs(e2 - run["E2"]) < 1e-6, (e2, run["E2"])
    assert e2 >= g["E2_exact"] - 1e-10
    e3 = L.mpspt_third_order(ctx, h0, psi)
    assert abs(e3 - run["E3"]) < 1e-6, (e3, run["E3"])
    assert rep.sigma_calls > 0 and rep.sigma64_calls > 0
    L.mpspt_mps_free(psi)
    L.mpspt_destroy(ctx)


def test_iteration_caps_are_reported(L, tiny):
    """A local CG that reaches cg_max_iter, and float64 refinement whose inner
    solves are cut to one iteration, return MPSPT_ERR_NOT_CONVERGED; a run
    ended by max_sweeps returns OK with report.converged = 0."""
    ctx = _session(L, tiny, cg_max_iter=2)
    with pytest.raises(L.MpsptError) as e:
        L.mpspt_minimize_hylleraas(ctx, "fock", 16, want_psi1=False)
    assert e.value.status == L.MPSPT_ERR_NOT_CONVERGED
    L.mpspt_destroy(ctx)
    ctx = _session(L, tiny, cg_max_iter=1, prec=L.MPSPT_MIXED_BF16)
    with pytest.raises(L.MpsptError) as e:
        L.mpspt_minimize_hylleraas(ctx, "fock", 16, want_psi1=False)
    assert e.value.status == L.MPSPT_ERR_NOT_CONVERGED
    L.mpspt_destroy(ctx)
    ctx = _session(L, tiny, max_sweeps=1)
    e2, _, rep = L.mpspt_minimize_hylleraas(ctx, "fock", 16, want_psi1=False)
    assert rep.n_sweeps == 1 and rep.converged == 0 and np.isfinite(e2)
    assert rep.max_discarded_per_sweep[0] == rep.max_discarded_weight
    L.mpspt_destroy(ctx)
    ctx = _session(L, tiny)
    _, _, rep = L.mpspt_minimize_hylleraas(ctx, "fock", 16, want_psi1=False)
    assert rep.converged == 1
    L.mpspt_destroy(ctx)


@pytest.mark.parametrize("h0", ["fock", "dyall"])
def test_extrapolation_matches_oracle(L, tiny, h0):
    """E2(M), the last sweep's discarded weight and the least-squares
    intercept in the discarded weight (the paper's extrapolation) against the
    oracle's (tests/golden/oracle_tiny_extrapolation.json)."""
    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_tiny_extrapolation.json")
    g = json.load(open(path))
    ref = g["h0"][h0]
    ctx = _session(L, tiny)
    a, b, e2, w = L.mpspt_extrapolate_e2(ctx, h0, g["Ms"])
    assert np.abs(e2 - np.array(ref["E2"])).max() < 1e-8, (e2, ref["E2"])
    assert np.abs(w - np.array(ref["w"])).max() < 1e-8 * max(1.0, max(ref["w"])), (w, ref["w"])
    assert abs(a - ref["E2_extrap"]) < 1e-7 and abs(b - ref["slope"]) < 1e-4 * abs(ref["slope"])
    L.mpspt_destroy(ctx)
