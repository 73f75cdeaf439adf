"""ctypes binding of include/mpspt.h (argument marshalling only).

Every function here has the name of the C entry point it wraps.  Arrays are
numpy float64 / int32 on the host; the library copies them.  The product path
has no CPU fallback: if libmpspt.so is missing or no CUDA device is present,
the calls fail.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmpspt.so")

MPSPT_OK = 0
MPSPT_H0_FOCK = 0
MPSPT_H0_DYALL = 1
MPSPT_FP64 = 0
MPSPT_FP32 = 1
MPSPT_MIXED_BF16 = 2
MPSPT_MIXED_FP16 = 3
MPSPT_LOCAL_SIGMA = 0
MPSPT_LOCAL_RHS = 1
MPSPT_LOCAL_DIAG = 2
H0 = {"fock": MPSPT_H0_FOCK, "dyall": MPSPT_H0_DYALL}
PREC = {"fp64": MPSPT_FP64, "fp32": MPSPT_FP32, "mixed": MPSPT_MIXED_BF16, "mixed_fp16": MPSPT_MIXED_FP16}
STATUS = {0: "OK", -1: "INVALID", -2: "OOM", -3: "NOT_SPD", -4: "NOT_CONVERGED",
          -5: "TIMEOUT", -6: "CUDA", -7: "STATE"}
# mpspt_status values of include/mpspt.h
MPSPT_OK, MPSPT_ERR_INVALID, MPSPT_ERR_OOM, MPSPT_ERR_NOT_SPD = 0, -1, -2, -3
MPSPT_ERR_NOT_CONVERGED, MPSPT_ERR_TIMEOUT, MPSPT_ERR_CUDA, MPSPT_ERR_STATE = -4, -5, -6, -7


class mpspt_options(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("stream", ctypes.c_void_p), ("prec", ctypes.c_int),
                ("max_sweeps", ctypes.c_int), ("e_tol", ctypes.c_double), ("cg_tol", ctypes.c_double),
                ("cg_max_iter", ctypes.c_int), ("seed", ctypes.c_ulonglong),
                ("use_learned", ctypes.c_int), ("verbose", ctypes.c_int),
                ("eig_fp64_only", ctypes.c_int), ("keep_rel", ctypes.c_double),
                ("autotune", ctypes.c_int), ("autotune_cache", ctypes.c_char_p), ("cuda_graphs", ctypes.c_int)]


class mpspt_report(ctypes.Structure):
    _fields_ = [("n_sweeps", ctypes.c_int), ("e2_per_sweep", ctypes.c_double * 64),
                ("max_discarded_weight", ctypes.c_double), ("cg_iters", ctypes.c_longlong),
                ("sigma_calls", ctypes.c_longlong), ("sigma_flops", ctypes.c_double),
                ("sigma_ms", ctypes.c_double), ("wall_ms", ctypes.c_double),
                ("max_bond_dim", ctypes.c_int), ("sweep_ms", ctypes.c_double * 64),
                ("kernel_launches", ctypes.c_longlong), ("sigma64_calls", ctypes.c_longlong),
                ("sigma64_flops", ctypes.c_double), ("sigma64_ms", ctypes.c_double),
                ("learned_used", ctypes.c_longlong), ("learned_rejected", ctypes.c_longlong),
                ("converged", ctypes.c_int), ("max_discarded_per_sweep", ctypes.c_double * 64),
                ("sigma_calls_cum", ctypes.c_longlong * 64), ("host_wait_ms", ctypes.c_double),
                ("e3_ms", ctypes.c_double), ("e3_transfers", ctypes.c_longlong), ("e3_wait_ms", ctypes.c_double),
                ("e3_flops", ctypes.c_double), ("e3_plan_bytes", ctypes.c_double),
                ("e3_setup_ms", ctypes.c_double)]


class MpsptError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"mpspt status {status} ({STATUS.get(status, '?')}): {msg}")
        self.status = status


_lib = None


def load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_1408_5092_gb300.build.build()")
        lib = ctypes.CDLL(LIB_PATH)
        vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
        fp = ctypes.POINTER(ctypes.c_float)
        sig = {
            "mpspt_default_options": (None, [ctypes.POINTER(mpspt_options)]),
            "mpspt_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.POINTER(mpspt_options)]),
            "mpspt_destroy": (None, [vp]),
            "mpspt_set_integrals": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int]),
            "mpspt_set_reference_ci": (ctypes.c_int, [vp, dp, ctypes.c_longlong]),
            "mpspt_set_reference": (ctypes.c_int, [vp, ctypes.c_int, ip, ip, ctypes.POINTER(dp)]),
            "mpspt_ground_state": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_double, dp, ctypes.POINTER(vp),
                                                  ctypes.POINTER(mpspt_report)]),
            "mpspt_energies": (ctypes.c_int, [vp, ctypes.c_int, dp, dp, dp]),
            "mpspt_minimize_hylleraas": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, dp, ctypes.POINTER(vp),
                                                        ctypes.POINTER(mpspt_report)]),
            "mpspt_third_order": (ctypes.c_int, [vp, ctypes.c_int, vp, dp]),
            "mpspt_extrapolate_e2": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ip, dp, dp, dp, dp]),
            "mpspt_minimize_partitioned": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ip, ip, ctypes.c_int, dp, dp,
                                                          ctypes.POINTER(mpspt_report)]),
            "mpspt_third_order_partitioned": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ip, ip, ctypes.c_int,
                                                             dp, dp, dp, dp, dp, dp, ctypes.POINTER(mpspt_report)]),
            "mpspt_mps_free": (None, [vp]),
            "mpspt_mps_import": (ctypes.c_int, [vp, ctypes.c_int, ip, ip, ctypes.POINTER(dp), ctypes.POINTER(vp)]),
            "mpspt_mps_shape": (ctypes.c_int, [vp, ip, ip]),
            "mpspt_mps_export": (ctypes.c_int, [vp, ip, ctypes.POINTER(dp)]),
            "mpspt_local_apply": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, dp, dp]),
            "mpspt_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "mpspt_eigh_batched": (ctypes.c_int, [ctypes.c_int, vp, ctypes.c_int, ip, vp, vp, vp]),
            "mpspt_eigh_batched_noalloc": (ctypes.c_int, [ctypes.c_int, vp, ctypes.c_int, ip, vp, vp, vp]),
            "mpspt_eigh_batched_ex": (ctypes.c_int, [ctypes.c_int, vp, ctypes.c_int, ip, vp, vp, vp, ctypes.c_int]),
            "mpspt_mlp_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_ulonglong, ctypes.POINTER(vp)]),
            "mpspt_mlp_free": (None, [vp]),
            "mpspt_mlp_set_params": (ctypes.c_int, [vp] + [fp] * 6),
            "mpspt_mlp_get_params": (ctypes.c_int, [vp] + [fp] * 6),
            "mpspt_mlp_forward": (ctypes.c_int, [vp, ctypes.c_int, fp, fp]),
            "mpspt_mlp_gradient": (ctypes.c_int, [vp, ctypes.c_int, fp, fp, fp] + [fp] * 6),
            "mpspt_mlp_train": (ctypes.c_int, [vp, ctypes.c_int, fp, fp, ctypes.c_int, ctypes.c_int, ctypes.c_float, fp]),
            "mpspt_harvest": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, fp, fp, ip]),
            "mpspt_set_preconditioner": (ctypes.c_int, [vp, vp]),
            "mpspt_train_preconditioner": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                          ctypes.c_char_p, fp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def declared_symbols():
    """Entry points declared in include/mpspt.h (parsed from the header)."""
    import re
    hdr = os.path.join(os.path.dirname(HERE), "include", "mpspt.h")
    text = open(hdr).read()
    pat = r"^\s*(?:mpspt_status|void|const char\s*\*)\s+(mpspt_[a-z0-9_]+)\s*\("
    return sorted(set(re.findall(pat, text, flags=re.M)))


def _check(st):
    if st != MPSPT_OK:
        msg = load().mpspt_status_string(st)
        raise MpsptError(st, msg.decode() if msg else "")


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def mpspt_default_options():
    o = mpspt_options()
    load().mpspt_default_options(ctypes.byref(o))
    return o


def mpspt_create(opt=None):
    o = opt if opt is not None else mpspt_default_options()
    h = ctypes.c_void_p()
    _check(load().mpspt_create(ctypes.byref(h), ctypes.byref(o)))
    return h


def mpspt_destroy(ctx):
    load().mpspt_destroy(ctx)


def mpspt_set_integrals(ctx, k_act, k_virt, n_elec, h, L):
    h = _f64(h)
    L = _f64(L)
    _check(load().mpspt_set_integrals(ctx, k_act, k_virt, n_elec, _dp(h), _dp(L), L.shape[0]))


def mpspt_set_reference_ci(ctx, ci):
    ci = _f64(ci)
    _check(load().mpspt_set_reference_ci(ctx, _dp(ci), ci.size))


def mpspt_set_reference(ctx, tensors, labels):
    """Reference as an active-space MPS: tensors[c] dense (D_c, 4, D_{c+1}),
    labels[c] (D_c, 2) the (N, 2Sz) of every bond index (contiguous,
    ascending sectors).  Marshalled into the header's block list: one block
    per (left sector, local state) with a nonzero QN-allowed right sector."""
    qsite = [(0, 0), (1, 1), (1, -1), (2, 0)]
    counts, meta, blocks = [], [], []
    for c, T in enumerate(tensors):
        T = _f64(T)
        ql, qr = np.asarray(labels[c]).reshape(-1, 2), np.asarray(labels[c + 1]).reshape(-1, 2)

        def sectors(q):
            out, i = [], 0
            while i < len(q):
                j = i
                while j < len(q) and tuple(q[j]) == tuple(q[i]):
                    j += 1
                out.append((tuple(int(x) for x in q[i]), i, j))
                i = j
            return out
        sl_, sr_ = sectors(ql), sectors(qr)
        rmap = {q: (a, b) for q, a, b in sr_}
        n = 0
        for q, a, b in sl_:
            for s_ in range(4):
                q2 = (q[0] + qsite[s_][0], q[1] + qsite[s_][1])
                if q2 not in rmap:
                    continue
                ra, rb = rmap[q2]
                blk = np.ascontiguousarray(T[a:b, s_, ra:rb])
                meta.extend([q[0], q[1], s_, q2[0], q2[1], b - a, rb - ra])
                blocks.append(blk)
                n += 1
        counts.append(n)
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    meta = np.ascontiguousarray(meta, dtype=np.int32)
    arr = (ctypes.POINTER(ctypes.c_double) * max(1, len(blocks)))(*[_dp(b) for b in blocks])
    ipp = ctypes.POINTER(ctypes.c_int)
    _check(load().mpspt_set_reference(ctx, len(tensors), counts.ctypes.data_as(ipp), meta.ctypes.data_as(ipp), arr))


def mpspt_ground_state(ctx, M0, s2_penalty=0.0, want_psi0=False):
    e = ctypes.c_double()
    psi = ctypes.c_void_p()
    rep = mpspt_report()
    _check(load().mpspt_ground_state(ctx, M0, float(s2_penalty), ctypes.byref(e),
                                     ctypes.byref(psi) if want_psi0 else None, ctypes.byref(rep)))
    return e.value, (psi if want_psi0 else None), rep


def mpspt_energies(ctx, h0):
    e = [ctypes.c_double() for _ in range(3)]
    _check(load().mpspt_energies(ctx, H0.get(h0, h0), *[ctypes.byref(x) for x in e]))
    return tuple(x.value for x in e)


def mpspt_minimize_hylleraas(ctx, h0, M, want_psi1=True):
    e2 = ctypes.c_double()
    psi = ctypes.c_void_p()
    rep = mpspt_report()
    _check(load().mpspt_minimize_hylleraas(ctx, H0.get(h0, h0), M, ctypes.byref(e2),
                                           ctypes.byref(psi) if want_psi1 else None, ctypes.byref(rep)))
    return e2.value, (psi if want_psi1 else None), rep


def mpspt_minimize_partitioned(ctx, h0, pairs, Ms, n_streams=0):
    pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    Ms = np.ascontiguousarray(np.asarray(Ms, dtype=np.int32).reshape(-1))
    n = len(Ms)
    e2 = ctypes.c_double()
    ep = np.zeros(n)
    rep = mpspt_report()
    ipp = ctypes.POINTER(ctypes.c_int)
    _check(load().mpspt_minimize_partitioned(ctx, H0.get(h0, h0), n, pairs.ctypes.data_as(ipp),
                                             Ms.ctypes.data_as(ipp), n_streams, ctypes.byref(e2), _dp(ep),
                                             ctypes.byref(rep)))
    return e2.value, ep, rep


def mpspt_third_order_partitioned(ctx, h0, pairs, Ms, n_streams=0):
    """Returns (E2, E3, E3 cross sum, E2 per partition, E3 per partition,
    <Psi1^i|H|Psi1^j> matrix, report)."""
    pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    Ms = np.ascontiguousarray(np.asarray(Ms, dtype=np.int32).reshape(-1))
    n = len(Ms)
    e2, e3, ex = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    e2p, e3p, hp = np.zeros(n), np.zeros(n), np.zeros((n, n))
    rep = mpspt_report()
    ipp = ctypes.POINTER(ctypes.c_int)
    _check(load().mpspt_third_order_partitioned(ctx, H0.get(h0, h0), n, pairs.ctypes.data_as(ipp),
                                                Ms.ctypes.data_as(ipp), n_streams, ctypes.byref(e2),
                                                ctypes.byref(e3), ctypes.byref(ex), _dp(e2p), _dp(e3p), _dp(hp),
                                                ctypes.byref(rep)))
    return e2.value, e3.value, ex.value, e2p, e3p, hp, rep


def mpspt_extrapolate_e2(ctx, h0, Ms):
    Ms = np.ascontiguousarray(np.asarray(Ms, dtype=np.int32))
    e2 = np.zeros(len(Ms))
    w = np.zeros(len(Ms))
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load().mpspt_extrapolate_e2(ctx, H0.get(h0, h0), len(Ms), Ms.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                       _dp(e2), _dp(w), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value, e2, w


def mpspt_third_order(ctx, h0, psi1):
    e3 = ctypes.c_double()
    _check(load().mpspt_third_order(ctx, H0.get(h0, h0), psi1, ctypes.byref(e3)))
    return e3.value


def mpspt_mps_free(psi):
    load().mpspt_mps_free(psi)


def mpspt_mps_import(ctx, tensors, labels):
    """tensors: list of (D_l, 4, D_r) arrays; labels: list of (D_c, 2) int arrays."""
    n = len(tensors)
    dims = np.array([len(q) for q in labels], dtype=np.int32)
    qn = np.ascontiguousarray(np.concatenate([np.asarray(q).reshape(-1, 2) for q in labels]), dtype=np.int32)
    ts = [_f64(t) for t in tensors]
    arr = (ctypes.POINTER(ctypes.c_double) * n)(*[_dp(t) for t in ts])
    out = ctypes.c_void_p()
    _check(load().mpspt_mps_import(ctx, n, dims.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                   qn.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), arr, ctypes.byref(out)))
    return out


def mpspt_mps_shape(psi):
    n = ctypes.c_int()
    _check(load().mpspt_mps_shape(psi, ctypes.byref(n), None))
    dims = np.zeros(n.value + 1, dtype=np.int32)
    _check(load().mpspt_mps_shape(psi, ctypes.byref(n), dims.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
    return n.value, dims


def mpspt_mps_export(psi):
    n, dims = mpspt_mps_shape(psi)
    qn = np.zeros((int(dims.sum()), 2), dtype=np.int32)
    ts = [np.zeros((dims[c], 4, dims[c + 1])) for c in range(n)]
    arr = (ctypes.POINTER(ctypes.c_double) * n)(*[_dp(t) for t in ts])
    _check(load().mpspt_mps_export(psi, qn.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), arr))
    labels = np.split(qn, np.cumsum(dims)[:-1])
    return ts, labels


def mpspt_local_apply(ctx, h0, psi1, i, op, x=None, shape=None):
    out = np.zeros(shape)
    xp = _dp(_f64(x)) if x is not None else None
    xa = _f64(x) if x is not None else None
    if xa is not None:
        xp = _dp(xa)
    _check(load().mpspt_local_apply(ctx, H0.get(h0, h0), psi1, i, op, xp, _dp(out)))
    return out


def mpspt_eigh_batched(device, stream, n, A_ptr, V_ptr, w_ptr):
    """Device pointers (ints, e.g. torch tensor .data_ptr()); n: host sizes."""
    n = np.ascontiguousarray(np.asarray(n, dtype=np.int32))
    _check(load().mpspt_eigh_batched(device, stream, len(n), n.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                     A_ptr, V_ptr, w_ptr))


def mpspt_eigh_batched_ex(device, stream, n, A_ptr, V_ptr, w_ptr, f32_start=1):
    """As mpspt_eigh_batched, with the truncation step's sweep-per-launch solver."""
    n = np.ascontiguousarray(np.asarray(n, dtype=np.int32))
    _check(load().mpspt_eigh_batched_ex(device, stream, len(n), n.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                        A_ptr, V_ptr, w_ptr, int(f32_start)))


def mpspt_eigh_batched_noalloc(device, stream, n, A_ptr, V_ptr, w_ptr):
    """As mpspt_eigh_batched, with no device allocation (fixed 16 MiB scratch)."""
    n = np.ascontiguousarray(np.asarray(n, dtype=np.int32))
    _check(load().mpspt_eigh_batched_noalloc(device, stream, len(n), n.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                             A_ptr, V_ptr, w_ptr))


MLP_NF = 16


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _fpp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def mpspt_mlp_create(device=0, width=256, seed=5092):
    h = ctypes.c_void_p()
    _check(load().mpspt_mlp_create(device, width, seed, ctypes.byref(h)))
    return h


def mpspt_mlp_free(net):
    load().mpspt_mlp_free(net)


def mpspt_mlp_set_params(net, p):
    arrs = [_f32(p[k]) for k in ("W1", "b1", "W2", "b2", "W3", "b3")]
    _check(load().mpspt_mlp_set_params(net, *[_fpp(a) for a in arrs]))


def mpspt_mlp_get_params(net, width=256):
    shapes = {"W1": (width, MLP_NF), "b1": (width,), "W2": (width, width), "b2": (width,), "W3": (2, width), "b3": (2,)}
    out = {k: np.zeros(v, dtype=np.float32) for k, v in shapes.items()}
    _check(load().mpspt_mlp_get_params(net, *[_fpp(out[k]) for k in ("W1", "b1", "W2", "b2", "W3", "b3")]))
    return out


def mpspt_mlp_forward(net, x):
    x = _f32(x)
    y = np.zeros((x.shape[0], 2), dtype=np.float32)
    _check(load().mpspt_mlp_forward(net, x.shape[0], _fpp(x), _fpp(y)))
    return y


def mpspt_mlp_gradient(net, x, t, width=256):
    x, t = _f32(x), _f32(t)
    loss = ctypes.c_float()
    shapes = {"W1": (width, MLP_NF), "b1": (width,), "W2": (width, width), "b2": (width,), "W3": (2, width), "b3": (2,)}
    g = {k: np.zeros(v, dtype=np.float32) for k, v in shapes.items()}
    _check(load().mpspt_mlp_gradient(net, x.shape[0], _fpp(x), _fpp(t), ctypes.byref(loss),
                                     *[_fpp(g[k]) for k in ("W1", "b1", "W2", "b2", "W3", "b3")]))
    return loss.value, g


def mpspt_mlp_train(net, x, t, epochs=10, batch=256, lr=1e-3):
    x, t = _f32(x), _f32(t)
    loss = ctypes.c_float()
    _check(load().mpspt_mlp_train(net, x.shape[0], _fpp(x), _fpp(t), epochs, batch, lr, ctypes.byref(loss)))
    return loss.value


def mpspt_harvest(ctx, h0, M, max_samples):
    x = np.zeros((max_samples, MLP_NF), dtype=np.float32)
    t = np.zeros((max_samples, 2), dtype=np.float32)
    n = ctypes.c_int()
    _check(load().mpspt_harvest(ctx, H0.get(h0, h0), M, max_samples, _fpp(x), _fpp(t), ctypes.byref(n)))
    return x[: n.value].copy(), t[: n.value].copy()


def mpspt_train_preconditioner(ctx, h0, M, max_samples=20000, epochs=30, harvest_path=None):
    loss = ctypes.c_float()
    _check(load().mpspt_train_preconditioner(ctx, H0.get(h0, h0), M, max_samples, epochs,
                                             harvest_path.encode() if harvest_path else None, ctypes.byref(loss)))
    return loss.value


def mpspt_set_preconditioner(ctx, net):
    _check(load().mpspt_set_preconditioner(ctx, net))


def mpspt_status_string(st):
    return load().mpspt_status_string(st).decode()
