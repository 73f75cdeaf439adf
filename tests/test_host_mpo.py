"""Host logic of the GPU library without a GPU: its MPO builder (compiled with
g++ from the library sources) contracted to a dense matrix equals the
oracle's brute-force determinant operator, for every operator the sweep uses."""
import os
import subprocess
import tempfile

import numpy as np
import pytest

import synthetic
from oracle.brute import DetSpace, dets_to_site_index, operator_matrix
from oracle.operators import Problem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    out = tmp_path_factory.mktemp("mpo") / "mpo_dense"
    src = [os.path.join(ROOT, "tests", "cpp", "mpo_dense.cpp"),
           os.path.join(ROOT, "paper_1408_5092_gb300", "csrc", "mpo.cpp")]
    r = subprocess.run(["g++", "-O2", "-std=c++17", "-I/usr/local/cuda/include", *src, "-o", str(out)],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail(r.stderr)
    return str(out)


def _dense(exe, p, which, tmp):
    k = p.k
    one = p.f if which == 0 else p.h
    fin, fout = os.path.join(tmp, "in.bin"), os.path.join(tmp, "out.bin")
    with open(fin, "wb") as f:
        np.array([k, p.k_act, which], dtype=np.int32).tofile(f)
        p.eps.astype(np.float64).tofile(f)
        np.ascontiguousarray(one, dtype=np.float64).tofile(f)
        np.ascontiguousarray(p.eri, dtype=np.float64).tofile(f)
        np.array([p.E0], dtype=np.float64).tofile(f)
    subprocess.run([exe, fin, fout], check=True)
    with open(fout, "rb") as f:
        dim, nd = np.fromfile(f, dtype=np.int32, count=2)
        dims = np.fromfile(f, dtype=np.int32, count=nd)
        M = np.fromfile(f, dtype=np.float64, count=dim * dim).reshape(dim, dim)
    return M, dims


@pytest.mark.parametrize("h0,which", [("fock", 0), ("dyall", 1), ("fock", 2), ("fock", 3)])
def test_library_mpo_matches_brute_force(exe, h0, which, tmp_path):
    h, L = synthetic.integrals(7, 2, 3, 5)
    ci, _ = synthetic.fci_reference(h, L, 2, 2)
    p = Problem(h, L, 2, 2, ci, h0=h0)
    terms = {0: p.h0_terms, 1: p.h0_terms, 2: p.rhs_terms, 3: p.hamiltonian_terms}[which]()
    M, dims = _dense(exe, p, which, str(tmp_path))
    err = 0.0
    for N in range(2 * p.k + 1):
        for sz in range(-N, N + 1, 2):
            S = DetSpace.sector(p.k, N, sz)
            if len(S) == 0:
                continue
            B = operator_matrix(terms, S).toarray()
            idx = dets_to_site_index(S.dets, p.k)
            err = max(err, float(np.abs(M[np.ix_(idx, idx)] - B).max()))
    assert err < 1e-12
    if which in (0, 1):
        assert max(dims[p.k_act + 1:-1]) == 2


def _compress(dets, keep):
    """Bit strings over all orbitals -> bit strings over the kept orbitals
    (the dropped orbitals are empty, so no sign changes)."""
    out = np.zeros(len(dets), dtype=np.uint64)
    for i, p in enumerate(keep):
        out |= ((dets >> np.uint64(2 * p)) & np.uint64(3)) << np.uint64(2 * i)
    return out


@pytest.mark.parametrize("which,mask", [(3, "00101"), (3, "00111"), (3, "00010"), (1, "00110")])
def test_run_maps_match_brute_force_on_empty_sites(exe, which, mask, tmp_path):
    """The library's run maps (a run of sites held empty applied as one
    sparse map of MPO states) reproduce the brute-force operator on the
    determinants whose masked orbitals are empty."""
    h, L = synthetic.integrals(7, 2, 3, 5)
    ci, _ = synthetic.fci_reference(h, L, 2, 2)
    p = Problem(h, L, 2, 2, ci, h0="dyall" if which == 1 else "fock")
    terms = p.h0_terms() if which == 1 else p.hamiltonian_terms()
    k = p.k
    fin, fout = os.path.join(str(tmp_path), "in.bin"), os.path.join(str(tmp_path), "out.bin")
    one = p.h
    with open(fin, "wb") as f:
        np.array([k, p.k_act, which], dtype=np.int32).tofile(f)
        p.eps.astype(np.float64).tofile(f)
        np.ascontiguousarray(one, dtype=np.float64).tofile(f)
        np.ascontiguousarray(p.eri, dtype=np.float64).tofile(f)
        np.array([p.E0], dtype=np.float64).tofile(f)
    subprocess.run([exe, fin, fout, mask], check=True)
    with open(fout, "rb") as f:
        dim, nd = np.fromfile(f, dtype=np.int32, count=2)
        np.fromfile(f, dtype=np.int32, count=nd)
        M = np.fromfile(f, dtype=np.float64, count=dim * dim).reshape(dim, dim)
    keep = [q for q in range(k) if mask[q] == "0"]
    assert dim == 4 ** len(keep)
    empty_bits = np.uint64(sum(3 << (2 * q) for q in range(k) if mask[q] == "1"))
    err, seen = 0.0, 0
    for N in range(2 * k + 1):
        for sz in range(-N, N + 1, 2):
            S = DetSpace.sector(k, N, sz)
            if len(S) == 0:
                continue
            S = S.subset((S.dets & empty_bits) == 0)
            if len(S) == 0:
                continue
            B = operator_matrix(terms, S).toarray()
            idx = dets_to_site_index(_compress(S.dets, keep), len(keep))
            err = max(err, float(np.abs(M[np.ix_(idx, idx)] - B).max()))
            seen += len(S)
    assert seen == dim
    assert err < 1e-12
