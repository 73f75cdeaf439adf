"""Medium workload (8e/8o + 24 virtual, the benchmark's system) at full bond
dimension on sampled outputs: the Fig. 1C local operators at bonds in the
active and the virtual region, for a shared random right-canonical Psi1,
against the oracle element by element."""
import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def medium():
    h, L, c = synthetic.config_integrals("medium")
    ci, _ = synthetic.fci_reference(h, L, c["k_act"], c["n_elec"])
    return h, L, c, ci


@pytest.mark.parametrize("h0", ["fock", "dyall"])
def test_medium_local_operators(medium, h0):
    from oracle.mps import HylleraasSweep, two_site_apply, two_site_diag, two_site_mask
    from oracle.operators import Problem
    from paper_1408_5092_gb300 import _lib as L
    h, Lc, c, ci = medium
    p = Problem(h, Lc, c["k_act"], c["n_elec"], ci, h0=h0)
    sw = HylleraasSweep(p, 128, seed=3)
    o = L.mpspt_default_options()
    ctx = L.mpspt_create(o)
    L.mpspt_set_integrals(ctx, c["k_act"], h.shape[0] - c["k_act"], c["n_elec"], h, Lc)
    L.mpspt_set_reference(ctx, ci)
    psi = L.mpspt_mps_import(ctx, sw.psi1.A, sw.psi1.q)
    rng = np.random.default_rng(9)
    done = 0
    for i in range(p.k - 1):
        if i not in (5, 7, 20):
            if i < 20:
                sw._update_left(i)
            continue
        mask = two_site_mask(sw.psi1.q[i], sw.psi1.q[i + 2], sw.allowed.get(i + 1))
        x = rng.normal(size=mask.shape) * mask
        ref_s = two_site_apply(sw.LA[i], sw.WA.W[i], sw.WA.W[i + 1], sw.RA[i + 2], x, sw.WA.dims[i + 1]) * mask
        p0 = np.einsum("lsm,mtr->lstr", sw.psi0.A[i], sw.psi0.A[i + 1])
        ref_g = two_site_apply(sw.LV[i], sw.WV.W[i], sw.WV.W[i + 1], sw.RV[i + 2], p0, sw.WV.dims[i + 1]) * mask
        ref_d = two_site_diag(sw.LA[i], sw.WA.W[i], sw.WA.W[i + 1], sw.RA[i + 2], x.shape, sw.WA.dims[i + 1]) * mask
        got_s = L.mpspt_local_apply(ctx, h0, psi, i, L.MPSPT_LOCAL_SIGMA, x, x.shape)
        got_g = L.mpspt_local_apply(ctx, h0, psi, i, L.MPSPT_LOCAL_RHS, None, x.shape)
        got_d = L.mpspt_local_apply(ctx, h0, psi, i, L.MPSPT_LOCAL_DIAG, None, x.shape)
        # a-priori float64 bound: rounding <= eps * K * (same contraction on |.|)
        absW = lambda W: {k: np.abs(v) for k, v in W.items()}
        bnd_s = two_site_apply(np.abs(sw.LA[i]), absW(sw.WA.W[i]), absW(sw.WA.W[i + 1]), np.abs(sw.RA[i + 2]),
                               np.abs(x), sw.WA.dims[i + 1]) * mask
        bnd_g = two_site_apply(np.abs(sw.LV[i]), absW(sw.WV.W[i]), absW(sw.WV.W[i + 1]), np.abs(sw.RV[i + 2]),
                               np.abs(p0), sw.WV.dims[i + 1]) * mask
        bnd_d = two_site_diag(np.abs(sw.LA[i]), absW(sw.WA.W[i]), absW(sw.WA.W[i + 1]), np.abs(sw.RA[i + 2]),
                              x.shape, sw.WA.dims[i + 1]) * mask
        for got, ref, bnd in ((got_s, ref_s, bnd_s), (got_g, ref_g, bnd_g), (got_d, ref_d, bnd_d)):
            assert np.all(np.abs(got - ref) <= 1e-12 * bnd + 1e-300), i
        done += 1
        if i < 20:
            sw._update_left(i)
    assert done == 3
    L.mpspt_mps_free(psi)
    L.mpspt_destroy(ctx)
