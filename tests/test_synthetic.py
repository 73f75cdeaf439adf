"""The seeded input generator: the stated recipe (ranges, symmetries, rank)
and determinism.  It holds none of the method's arithmetic; both the oracle
and the GPU path take their inputs from it."""
import numpy as np

import synthetic


def test_recipe_shapes_symmetries_and_ranges():
    for name, c in synthetic.CONFIGS.items():
        if name in ("partitions", "large"):
            continue   # same code path; these are large to hold in a CPU test
        h, L, cc = synthetic.config_integrals(name)
        k = c["k_act"] + c["k_virt"]
        assert cc is c
        assert h.shape == (k, k) and L.shape == (c["n_chol"], k, k)
        assert h.dtype == np.float64 and L.dtype == np.float64
        assert np.array_equal(h, h.T)
        assert np.array_equal(L, L.transpose(0, 2, 1))
        # orbital energies sit on the diagonal on top of N(0, 0.1^2) noise
        d = np.diag(h)
        ka = c["k_act"]
        assert d[:ka].min() > -0.5 - 0.6 and d[:ka].max() < 0.5 + 0.6
        assert d[ka:].min() > 0.5 - 0.6 and d[ka:].max() < 3.0 + 0.6
        off = h[np.triu_indices(k, 1)]
        assert abs(off.std() - 0.1) < 0.02 and abs(off.mean()) < 0.02
        lv = L[:, np.triu_indices(k)[0], np.triu_indices(k)[1]].ravel()
        sd = 0.05 * c.get("l_scale", 1.0)
        assert abs(lv.std() - sd) < 0.1 * sd


def test_eri_is_positive_semidefinite_with_cholesky_rank():
    h, L = synthetic.integrals(3, 3, 4, 6)
    k = h.shape[0]
    eri = np.einsum("Qpq,Qrs->pqrs", L, L)
    # 8-fold permutational symmetry of real orbitals
    assert np.allclose(eri, eri.transpose(1, 0, 2, 3))
    assert np.allclose(eri, eri.transpose(2, 3, 0, 1))
    assert np.allclose(eri, eri.transpose(0, 1, 3, 2))
    G = eri.reshape(k * k, k * k)
    w = np.linalg.eigvalsh(G)
    assert w.min() > -1e-12
    assert int(np.sum(w > 1e-10 * w.max())) == 6


def test_seeded_and_deterministic():
    a = synthetic.integrals(11, 2, 3, 4)
    b = synthetic.integrals(11, 2, 3, 4)
    c = synthetic.integrals(12, 2, 3, 4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not np.array_equal(a[0], c[0])
    assert synthetic.EVAL_SEED != synthetic.TRAIN_SEED


def test_stored_medium_reference_is_the_fci_singlet():
    """The stored medium Psi0 (read by config_reference so that every machine
    starts from the same bits) is the string-based FCI singlet: same vector
    to 1e-10, unit norm, Sz = 0 / N = 8 strings only."""
    import numpy as np
    h, L, c, ci = synthetic.config_reference("medium")
    ref, _ = synthetic.fci_reference(h, L, c["k_act"], c["n_elec"])
    assert abs(np.linalg.norm(ci) - 1.0) < 1e-14
    assert np.abs(ci - ref).max() < 1e-10
