"""Batched float64 Jacobi eigensolver of the truncation step, through the C
ABI on device data, against numpy.linalg.eigh: eigenvalues to 1e-12 of the
spectral radius, eigenvectors orthonormal and A V = V diag(w)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _batch(rng, sizes):
    mats = []
    for n in sizes:
        X = rng.normal(size=(n, n + 3))
        X[:, : n // 3] *= 1e-4            # graded spectrum, like a density matrix
        mats.append(X @ X.T)
    return mats


def test_eigh_batched_matches_numpy():
    import torch
    from paper_1408_5092_gb300 import _lib as L
    rng = np.random.default_rng(1)
    sizes = [1, 2, 7, 64, 112, 113, 180]
    mats = _batch(rng, sizes)
    A = torch.tensor(np.concatenate([m.ravel() for m in mats]), device="cuda", dtype=torch.float64)
    V = torch.zeros_like(A)
    w = torch.zeros(sum(sizes), device="cuda", dtype=torch.float64)
    L.mpspt_eigh_batched(0, torch.cuda.current_stream().cuda_stream, sizes, A.data_ptr(), V.data_ptr(), w.data_ptr())
    torch.cuda.synchronize()
    Vh, wh = V.cpu().numpy(), w.cpu().numpy()
    o = ow = 0
    for n, m in zip(sizes, mats):
        v = Vh[o:o + n * n].reshape(n, n)
        e = wh[ow:ow + n]
        ref = np.linalg.eigvalsh(m)
        scale = np.abs(ref).max()
        assert np.max(np.abs(np.sort(e) - ref)) < 1e-12 * scale
        assert np.max(np.abs(v.T @ v - np.eye(n))) < 1e-12
        assert np.max(np.abs(m @ v - v * e[None, :])) < 1e-12 * scale
        o += n * n
        ow += n
    # the input is not modified
    assert np.array_equal(A.cpu().numpy(), np.concatenate([m.ravel() for m in mats]))
