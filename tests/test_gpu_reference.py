"""The reference Psi0 as an MPS (the form a DMRG calculation gives) and the
library's own ground-state DMRG, against the CPU oracle and the
string-based FCI of the synthetic inputs.

* mpspt_set_reference (QN-blocked MPS) and mpspt_set_reference_ci (dense CI
  vector) describe the same state: E_ref, E0, E1 and the E2 sweep agree.
* mpspt_ground_state at a bond dimension that holds every Schmidt state
  reproduces the FCI energy; at a truncating one it follows the oracle's
  DMRG sweep (same seeded start, reading R8) sweep by sweep."""
import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1408_5092_gb300 import _lib
    _lib.load()
    return _lib


def _ctx(L, h, Lc, k_act, n_elec, **opts):
    o = L.mpspt_default_options()
    for k, v in opts.items():
        setattr(o, k, v)
    ctx = L.mpspt_create(o)
    L.mpspt_set_integrals(ctx, k_act, h.shape[0] - k_act, n_elec, h, Lc)
    return ctx


@pytest.mark.parametrize("name", ["tiny", "medium"])
def test_mps_reference_equals_ci_reference(L, name):
    from oracle.mps import mps_from_vector
    h, Lc, c, ci = synthetic.config_reference(name)
    ka, n = c["k_act"], c["n_elec"]
    m = mps_from_vector(ci, ka)
    a = _ctx(L, h, Lc, ka, n, max_sweeps=2, e_tol=1e-14)
    L.mpspt_set_reference_ci(a, ci)
    b = _ctx(L, h, Lc, ka, n, max_sweeps=2, e_tol=1e-14)
    # any norm is accepted: scale the first tensor
    L.mpspt_set_reference(b, [m.A[0] * 3.0] + m.A[1:], m.q)
    for h0 in ("fock", "dyall"):
        ea, eb = L.mpspt_energies(a, h0), L.mpspt_energies(b, h0)
        assert np.abs(np.array(ea) - np.array(eb)).max() < 1e-11, (h0, ea, eb)
    if name == "tiny":
        e2a, _, _ = L.mpspt_minimize_hylleraas(a, "fock", 16, want_psi1=False)
        e2b, _, _ = L.mpspt_minimize_hylleraas(b, "fock", 16, want_psi1=False)
        assert abs(e2a - e2b) < 1e-10, (e2a, e2b)
    L.mpspt_destroy(a)
    L.mpspt_destroy(b)


def test_mps_reference_rejects_bad_blocks(L):
    from oracle.mps import mps_from_vector
    h, Lc, c, ci = synthetic.config_reference("tiny")
    ka, n = c["k_act"], c["n_elec"]
    m = mps_from_vector(ci, ka)
    ctx = _ctx(L, h, Lc, ka, n)
    bad = [q.copy() for q in m.q]
    bad[-1][:] = (n + 2, 0)                        # last bond is not (n_elec, 0)
    with pytest.raises(L.MpsptError) as e:
        L.mpspt_set_reference(ctx, m.A, bad)
    assert e.value.status == L.MPSPT_ERR_INVALID
    with pytest.raises(L.MpsptError) as e:
        L.mpspt_set_reference(ctx, m.A[:-1], m.q[:-1])   # wrong site count
    assert e.value.status == L.MPSPT_ERR_INVALID
    L.mpspt_destroy(ctx)


@pytest.mark.parametrize("name,M0", [("tiny", 16), ("medium", 256)])
def test_ground_state_reaches_fci(L, name, M0):
    """4^(k_act/2) states at the middle cut hold the exact state: with the
    S^2 penalty the DMRG energy equals the FCI singlet of the synthetic
    reference (on the medium draw the lowest Sz = 0 state is not a singlet),
    and the installed reference gives it back as E_ref = <Psi0|H|Psi0>."""
    h, Lc, c = synthetic.config_integrals(name)
    ka, n = c["k_act"], c["n_elec"]
    _, e_fci = synthetic.fci_reference(h, Lc, ka, n)
    ctx = _ctx(L, h, Lc, ka, n, keep_rel=1e-14)
    e, psi, rep = L.mpspt_ground_state(ctx, M0, s2_penalty=1.0, want_psi0=True)
    assert abs(e - e_fci) < 1e-9, (e, e_fci)
    _, _, eref = L.mpspt_energies(ctx, "dyall")
    assert abs(eref - e_fci) < 1e-9, (eref, e_fci)
    nsite, dims = L.mpspt_mps_shape(psi)
    assert nsite == ka and dims.max() <= M0
    L.mpspt_mps_free(psi)
    L.mpspt_destroy(ctx)


def test_ground_state_follows_the_oracle_when_truncating(L):
    """5 active orbitals, 4 electrons, M0 = 4 (truncating): per-sweep DMRG
    energies equal the oracle's from the same seeded start."""
    from oracle.dmrg import GroundStateSweep
    h, Lc = synthetic.integrals(11, 5, 0, 10)
    gs = GroundStateSweep(h, Lc, 5, 4, 4, max_sweeps=6, tol_e=1e-12)
    gs.run()
    ctx = _ctx(L, h, Lc, 5, 4, max_sweeps=len(gs.history), e_tol=1e-12)
    e, _, rep = L.mpspt_ground_state(ctx, 4)
    hist = [rep.e2_per_sweep[s] for s in range(rep.n_sweeps)]
    assert len(hist) == len(gs.history)
    assert np.abs(np.array(hist) - np.array(gs.history)).max() < 1e-9, (hist, gs.history)
    L.mpspt_destroy(ctx)


def test_spin_penalty_matches_the_oracle(L):
    """Near-degenerate 5-orbital draw whose lowest Sz = 0 state is a triplet
    (the oracle's pin): the library's DMRG without the penalty finds the
    triplet, with it the singlet, each at the oracle's energy."""
    from oracle.dmrg import GroundStateSweep
    h, Lc = synthetic.integrals(11, 5, 0, 10)
    h = 0.1 * (h - np.diag(np.diag(h)))
    h = h + np.diag(np.r_[0.0, 0.0, 0.001, np.linspace(1, 2, 2)])
    for lam in (0.0, 1.0):
        ref = GroundStateSweep(h, Lc, 5, 4, 16, keep_rel=1e-14, s2_penalty=lam).run()
        ctx = _ctx(L, h, Lc, 5, 4, keep_rel=1e-14)
        e, _, rep = L.mpspt_ground_state(ctx, 16, s2_penalty=lam)
        last = rep.e2_per_sweep[rep.n_sweeps - 1]
        assert abs(last - ref) < 1e-9, (lam, last, ref)
        L.mpspt_destroy(ctx)


def test_e2_from_the_dmrg_reference(L):
    """Tiny system: MPS-PT on the DMRG reference (exact at M0 = 16) gives the
    E2 of the FCI reference."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_tiny.json")))
    h, Lc, c = synthetic.config_integrals("tiny")
    ctx = _ctx(L, h, Lc, c["k_act"], c["n_elec"], keep_rel=1e-14)
    L.mpspt_ground_state(ctx, 16, s2_penalty=1.0)
    e2, _, _ = L.mpspt_minimize_hylleraas(ctx, "fock", 16, want_psi1=False)
    assert abs(e2 - gold["h0"]["fock"]["runs"]["16"]["E2"]) < 1e-7
    L.mpspt_destroy(ctx)
