"""Batching machinery of the sweep on the GPU: CUDA graphs of CG chunks,
persistent grouped GEMMs and the tile-shape autotuner change how work is
launched, never what is computed.

* The CUDA-core grouped GEMM sums every output element over K in the same
  order for any tile shape, so tuned tiles reproduce the default run bit for
  bit; the tuned table is written to the cache file and read back.
* A graph replays the same kernels in the same order as the direct
  launches, so graph runs reproduce the direct run bit for bit, with fewer
  host launches."""
import os

import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1408_5092_gb300 import _lib
    _lib.load()
    return _lib


def _run(L, name, h0, M, **opts):
    h, Lc, c, ci = synthetic.config_reference(name)
    o = L.mpspt_default_options()
    for k, v in opts.items():
        setattr(o, k, v)
    ctx = L.mpspt_create(o)
    L.mpspt_set_integrals(ctx, c["k_act"], h.shape[0] - c["k_act"], c["n_elec"], h, Lc)
    L.mpspt_set_reference_ci(ctx, ci)
    e2, _, rep = L.mpspt_minimize_hylleraas(ctx, h0, M, want_psi1=False)
    hist = [rep.e2_per_sweep[s] for s in range(rep.n_sweeps)]
    L.mpspt_destroy(ctx)
    return hist, rep


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_autotuned_tiles_reproduce_the_default_run(L, tmp_path, prec):
    cache = str(tmp_path / "tiles.txt")
    base, _ = _run(L, "medium", "fock", 32, prec=L.PREC[prec], max_sweeps=2, e_tol=1e-14)
    tuned, _ = _run(L, "medium", "fock", 32, prec=L.PREC[prec], max_sweeps=2, e_tol=1e-14, autotune=1,
                    autotune_cache=cache.encode())
    assert tuned == base
    rows = [l.split() for l in open(cache) if l.strip()]
    assert rows and all(len(r) == 8 for r in rows)
    tiles = {(int(r[6]), int(r[7])) for r in rows}
    assert tiles <= {(64, 64), (32, 64), (64, 32), (16, 128), (32, 32)}
    again, _ = _run(L, "medium", "fock", 32, prec=L.PREC[prec], max_sweeps=2, e_tol=1e-14, autotune=1,
                    autotune_cache=cache.encode())
    assert again == base


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_graph_chunks_reproduce_direct_launches(L, prec):
    """Graphs are captured on a created stream (the legacy default stream
    cannot be captured; there the option has no effect)."""
    import torch
    st = torch.cuda.Stream()
    base, rb = _run(L, "tiny", "fock", 24, prec=L.PREC[prec], stream=st.cuda_stream)
    graph, rg = _run(L, "tiny", "fock", 24, prec=L.PREC[prec], cuda_graphs=1, stream=st.cuda_stream)
    same, rs = _run(L, "tiny", "fock", 24, prec=L.PREC[prec], cuda_graphs=1)     # stream 0: direct launches
    assert same == base
    assert graph == base
    assert rg.cg_iters == rb.cg_iters
    assert rg.kernel_launches < rb.kernel_launches


def test_partitions_with_graphs(L):
    """Medium virtual-pair partitions on 4 streams with graph chunks: the
    energies of the direct run, bit for bit, with fewer host launches."""
    h, Lc, c, ci = synthetic.config_reference("medium")
    pairs = [(0, 0), (0, 5), (3, 17), (23, 23)]
    out = []
    for graphs in (0, 1):
        o = L.mpspt_default_options()
        o.cuda_graphs = graphs
        ctx = L.mpspt_create(o)
        L.mpspt_set_integrals(ctx, c["k_act"], h.shape[0] - c["k_act"], c["n_elec"], h, Lc)
        L.mpspt_set_reference_ci(ctx, ci)
        tot, ep, rep = L.mpspt_minimize_partitioned(ctx, "fock", pairs, [16] * len(pairs), n_streams=4)
        out.append((tot, ep.copy(), rep.kernel_launches))
        L.mpspt_destroy(ctx)
    assert np.array_equal(out[0][1], out[1][1]) and out[0][0] == out[1][0]
    assert out[1][2] < out[0][2]


def test_partitions_with_autotune_and_graphs(L, tmp_path):
    """Partition lanes share the context's tile tuner (its timing buffers
    outlive the lanes' streams): tuned and untuned partition energies agree
    bit for bit, the context is destroyed cleanly after the lanes are gone,
    and a second context reads the tuned table back."""
    h, Lc, c, ci = synthetic.config_reference("medium")
    pairs = [(0, 0), (0, 5), (3, 17), (23, 23)]
    cache = str(tmp_path / "tiles.txt")
    out = []
    for tune in (0, 1, 1):
        o = L.mpspt_default_options()
        o.cuda_graphs = 1
        o.autotune = tune
        if tune:
            o.autotune_cache = cache.encode()
        ctx = L.mpspt_create(o)
        L.mpspt_set_integrals(ctx, c["k_act"], h.shape[0] - c["k_act"], c["n_elec"], h, Lc)
        L.mpspt_set_reference_ci(ctx, ci)
        tot, ep, _ = L.mpspt_minimize_partitioned(ctx, "fock", pairs, [16] * len(pairs), n_streams=4)
        out.append(ep.copy())
        L.mpspt_destroy(ctx)
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])
    assert os.path.getsize(cache) > 0
