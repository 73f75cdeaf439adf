"""The allocation-free eigensolver entry point (for callers that cannot
allocate device memory during the call) against the allocating one, through
the C ABI on device data, on two calls in a row with different inputs.

Collected last on purpose: if it fails, a run that stops at the first
failure has already run every other test.  It must pass alone in a fresh
process (the first call performs the per-device set-up) and after the
other tests."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _mats(seed, sizes):
    rng = np.random.default_rng(seed)
    out = []
    for n in sizes:
        X = rng.normal(size=(n, n + 2))
        X[:, : n // 4] *= 1e-3
        out.append(X @ X.T)
    return np.concatenate([m.ravel() for m in out])


def _run(fn, sizes, A):
    import torch
    Ad = torch.tensor(A, device="cuda", dtype=torch.float64)
    V = torch.zeros_like(Ad)
    w = torch.zeros(sum(sizes), device="cuda", dtype=torch.float64)
    dev = torch.cuda.current_device()
    fn(0, torch.cuda.current_stream().cuda_stream, sizes, Ad.data_ptr(), V.data_ptr(), w.data_ptr())
    assert torch.cuda.current_device() == dev      # the caller's current device is left as it was
    torch.cuda.synchronize()
    return V.cpu().numpy(), w.cpu().numpy()


def test_noalloc_matches_allocating_entry_point_twice():
    from paper_1408_5092_gb300 import _lib as L
    for call, (seed, sizes) in enumerate([(11, [3, 64, 150, 1, 97]), (12, [200, 5, 33])]):
        A = _mats(seed, sizes)
        V1, w1 = _run(L.mpspt_eigh_batched, sizes, A)
        V2, w2 = _run(L.mpspt_eigh_batched_noalloc, sizes, A)
        o = ow = 0
        for n in sizes:
            a = A[o:o + n * n].reshape(n, n)
            scale = max(1.0, np.abs(a).max())
            e1, e2 = w1[ow:ow + n], w2[ow:ow + n]
            v1, v2 = V1[o:o + n * n].reshape(n, n), V2[o:o + n * n].reshape(n, n)
            assert np.max(np.abs(np.sort(e1) - np.sort(e2))) < 1e-12 * scale, call
            # same eigen-decomposition: projector onto each eigenvector agrees
            assert np.max(np.abs(v1 @ np.diag(e1) @ v1.T - v2 @ np.diag(e2) @ v2.T)) < 1e-11 * scale, call
            assert np.max(np.abs(a @ v2 - v2 * e2[None, :])) < 1e-12 * scale, call
            o += n * n
            ow += n


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_1408_5092_gb300 import _lib as L
    d = torch.zeros(8, device="cuda", dtype=torch.float64)
    with pytest.raises(L.MpsptError) as e:
        # 3 x 2048^2 doubles exceed the fixed 2^21-double scratch: rejected on the host
        L.mpspt_eigh_batched_noalloc(0, 0, [2048, 2048, 2048], d.data_ptr(), d.data_ptr(), d.data_ptr())
    assert e.value.status == -1
