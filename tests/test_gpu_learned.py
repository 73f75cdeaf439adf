"""Learned block preconditioner: the GPU network's forward pass and
gradients (hand-written training kernels) against the float64 oracle
network with the same bfloat16 weights, and the trained network in the sweep:
E2 unchanged (Jacobi-PCG still converges to the same tolerance) and the CG
iteration count with and without it recorded."""
import json
import os

import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu


def test_network_forward_and_gradients_match_oracle():
    from oracle.mlp import backward, forward, init_params
    from paper_1408_5092_gb300 import _lib as L
    p = init_params(16, 256, 2, seed=3)
    p = {k: v.astype(np.float32).astype(np.float64) for k, v in p.items()}
    rng = np.random.default_rng(4)
    p["b1"] = rng.normal(0, 0.1, 256)
    p["b2"] = rng.normal(0, 0.1, 256)
    p = {k: v.astype(np.float32).astype(np.float64) for k, v in p.items()}
    x = rng.normal(size=(300, 16)).astype(np.float32).astype(np.float64)
    t = rng.normal(size=(300, 2)).astype(np.float32).astype(np.float64)
    net = L.mpspt_mlp_create(0, 256, 1)
    L.mpspt_mlp_set_params(net, p)
    y_ref, _ = forward(p, x)
    y = L.mpspt_mlp_forward(net, x)
    assert np.max(np.abs(y - y_ref)) < 1e-4 * max(1.0, np.abs(y_ref).max())
    loss, g = L.mpspt_mlp_gradient(net, x, t)
    g_ref = backward(p, x, t)
    assert abs(loss - 0.5 * np.sum((y_ref - t) ** 2) / 300) < 1e-4
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        scale = max(1e-6, np.abs(g_ref[k]).max())
        assert np.max(np.abs(g[k] - g_ref[k])) < 1e-4 * scale, k
    L.mpspt_mlp_free(net)


def _ctx(L, seed, use_learned=0):
    h, Lc, c = synthetic.config_integrals("tiny", seed=seed)
    ci, _ = synthetic.fci_reference(h, Lc, c["k_act"], c["n_elec"])
    o = L.mpspt_default_options()
    o.use_learned = use_learned
    ctx = L.mpspt_create(o)
    L.mpspt_set_integrals(ctx, c["k_act"], h.shape[0] - c["k_act"], c["n_elec"], h, Lc)
    L.mpspt_set_reference_ci(ctx, ci)
    return ctx


def test_trained_network_in_the_sweep():
    from paper_1408_5092_gb300 import _lib as L
    # harvest on the training draw, train on the GPU
    ctx = _ctx(L, synthetic.TRAIN_SEED)
    x, t = L.mpspt_harvest(ctx, "dyall", 32, 20000)
    L.mpspt_destroy(ctx)
    assert len(x) > 1000
    perm = np.random.default_rng(0).permutation(len(x))
    x, t = x[perm], t[perm]
    net = L.mpspt_mlp_create(0, 256, 5092)
    l0, _ = L.mpspt_mlp_gradient(net, x[:2000], t[:2000])
    loss = L.mpspt_mlp_train(net, x, t, epochs=30, batch=256, lr=1e-3)
    assert loss < l0
    # evaluate on the evaluation draw: plain vs learned
    ctx = _ctx(L, 1408, use_learned=0)
    e_plain, psi, r_plain = L.mpspt_minimize_hylleraas(ctx, "dyall", 32)
    L.mpspt_mps_free(psi)
    L.mpspt_destroy(ctx)
    ctx = _ctx(L, 1408, use_learned=1)
    L.mpspt_set_preconditioner(ctx, net)
    e_learn, psi, r_learn = L.mpspt_minimize_hylleraas(ctx, "dyall", 32)
    L.mpspt_mps_free(psi)
    L.mpspt_destroy(ctx)
    L.mpspt_mlp_free(net)
    assert abs(e_learn - e_plain) < 1e-8
    assert r_learn.learned_used + r_learn.learned_rejected > 0
    rec = {"train_samples": int(len(x)), "train_loss_initial": float(l0), "train_loss_final": float(loss),
           "cg_iters_jacobi": int(r_plain.cg_iters), "cg_iters_learned": int(r_learn.cg_iters),
           "learned_used": int(r_learn.learned_used), "learned_rejected": int(r_learn.learned_rejected),
           "sweeps_jacobi": int(r_plain.n_sweeps), "sweeps_learned": int(r_learn.n_sweeps),
           "E2_jacobi": e_plain, "E2_learned": e_learn}
    out = os.environ.get("MPSPT_LEARNED_REPORT")
    if out:
        with open(out, "w") as f:
            json.dump(rec, f, indent=1)
    print("learned preconditioner:", rec)


def test_train_preconditioner_end_to_end(tmp_path):
    """mpspt_train_preconditioner: harvest on the context's problem, train on
    the GPU, attach; the harvest file is written, and a second context trains
    from the file instead of sweeping.  With the network attached the sweep
    reaches the plain sweep's E2."""
    from paper_1408_5092_gb300 import _lib as L
    path = str(tmp_path / "pairs.bin")
    ctx = _ctx(L, synthetic.TRAIN_SEED, use_learned=1)
    loss = L.mpspt_train_preconditioner(ctx, "dyall", 16, max_samples=4000, epochs=5, harvest_path=path)
    assert np.isfinite(loss) and os.path.getsize(path) > 4
    n = int(np.fromfile(path, dtype=np.int32, count=1)[0])
    assert 0 < n <= 4000 and os.path.getsize(path) == 4 + 4 * n * 18
    L.mpspt_destroy(ctx)
    ctx = _ctx(L, 1408, use_learned=1)
    L.mpspt_train_preconditioner(ctx, "dyall", 16, max_samples=4000, epochs=5, harvest_path=path)
    e_learn, _, r = L.mpspt_minimize_hylleraas(ctx, "dyall", 16, want_psi1=False)
    L.mpspt_destroy(ctx)
    ctx = _ctx(L, 1408)
    e_plain, _, _ = L.mpspt_minimize_hylleraas(ctx, "dyall", 16, want_psi1=False)
    L.mpspt_destroy(ctx)
    assert abs(e_learn - e_plain) < 1e-8
    assert r.learned_used + r.learned_rejected > 0
