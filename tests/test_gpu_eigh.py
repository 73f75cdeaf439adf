"""Batched eigensolvers of the truncation step (Eq. 6 density matrices),
through the C ABI on device data, against numpy.linalg.eigh: eigenvalues to
1e-12 of the spectral radius, eigenvectors orthonormal and A V = V diag(w).
Three solvers are held to the same float64 bounds: the single-launch
float64 Jacobi (mpspt_eigh_batched) and the sweep-per-launch solver of the
truncation step, from float64 sweeps alone or from a float32 start with a
float64 polish (mpspt_eigh_batched_ex).  The sizes straddle the kernels'
placement limits (single launch: A and V in shared memory up to n = 112, A
alone up to 158; sweep-per-launch: packed A in shared memory of one CTA up to
n = 218 in float64 and 308 in float32, float64 sweeps of n >= 48 on 8-CTA
clusters up to n = 594, larger ones on one CTA with A in global memory).
The float64 polish after the float32 start uses the large-diagonal-first
pair schedule; the others the round-robin one."""

ENTRIES = [("mpspt_eigh_batched", ()), ("mpspt_eigh_batched_ex", (0,)), ("mpspt_eigh_batched_ex", (1,))]
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


@pytest.mark.parametrize("entry,extra", ENTRIES)
def test_eigh_batched_matches_numpy(entry, extra):
    import torch
    from paper_1408_5092_gb300 import _lib as L
    rng = np.random.default_rng(1)
    sizes = [1, 2, 7, 47, 48, 64, 112, 113, 158, 159, 184, 218, 219, 308, 309, 400, 600]
    mats = _batch(rng, sizes)
    A = torch.tensor(np.concatenate([m.ravel() for m in mats]), device="cuda", dtype=torch.float64)
    V = torch.zeros_like(A)
    w = torch.zeros(sum(sizes), device="cuda", dtype=torch.float64)
    getattr(L, entry)(0, torch.cuda.current_stream().cuda_stream, sizes, A.data_ptr(), V.data_ptr(), w.data_ptr(),
                      *extra)
    torch.cuda.synchronize()
    Vh, wh = V.cpu().numpy(), w.cpu().numpy()
    o = ow = 0
    for n, m in zip(sizes, mats):
        v = Vh[o:o + n * n].reshape(n, n)
        e = wh[ow:ow + n]
        ref = np.linalg.eigvalsh(m)
        scale = np.abs(ref).max()
        assert np.max(np.abs(np.sort(e) - ref)) < 1e-12 * scale, n
        assert np.max(np.abs(v.T @ v - np.eye(n))) < 1e-12
        assert np.max(np.abs(m @ v - v * e[None, :])) < 1e-12 * scale
        o += n * n
        ow += n
    # the input is not modified
    assert np.array_equal(A.cpu().numpy(), np.concatenate([m.ravel() for m in mats]))


@pytest.mark.parametrize("entry,extra", ENTRIES)
def test_eigh_degenerate_and_zero(entry, extra):
    """Exactly repeated eigenvalues (a density matrix of a spin multiplet) and
    the zero matrix: any orthonormal basis of each eigenspace is valid, so the
    test checks the eigenvalues, orthonormality and the residual only."""
    import torch
    from paper_1408_5092_gb300 import _lib as L
    rng = np.random.default_rng(2)
    mats = []
    for n in (12, 130, 170):
        Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
        lam = np.repeat(rng.uniform(0.0, 1.0, size=(n + 2) // 3), 3)[:n]
        mats.append((Q * lam) @ Q.T)
    mats.append(np.zeros((9, 9)))
    sizes = [m.shape[0] for m in mats]
    A = torch.tensor(np.concatenate([m.ravel() for m in mats]), device="cuda", dtype=torch.float64)
    V = torch.zeros_like(A)
    w = torch.zeros(sum(sizes), device="cuda", dtype=torch.float64)
    getattr(L, entry)(0, torch.cuda.current_stream().cuda_stream, sizes, A.data_ptr(), V.data_ptr(), w.data_ptr(),
                      *extra)
    torch.cuda.synchronize()
    Vh, wh = V.cpu().numpy(), w.cpu().numpy()
    o = ow = 0
    for n, m in zip(sizes, mats):
        v = Vh[o:o + n * n].reshape(n, n)
        e = wh[ow:ow + n]
        ref = np.linalg.eigvalsh(m)
        scale = max(np.abs(ref).max(), 1.0)
        assert np.max(np.abs(np.sort(e) - ref)) < 1e-12 * scale, n
        assert np.max(np.abs(v.T @ v - np.eye(n))) < 1e-12, n
        assert np.max(np.abs(m @ v - v * e[None, :])) < 1e-12 * scale, n
        o += n * n
        ow += n
