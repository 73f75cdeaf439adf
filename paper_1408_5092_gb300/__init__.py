"""GB300 MPS-PT: the Hylleraas-functional sweep of matrix product state
perturbation theory (Sharma & Chan) as a CUDA library for sm_103a.

The compute path is ``libmpspt.so`` (C ABI in ``include/mpspt.h``); this
package only builds it and marshals arguments.  ``Session`` wraps one context.
"""
from . import _lib
from ._lib import *  # noqa: F401,F403  (C-ABI names)


class Session:
    """One mpspt context with integrals and a reference loaded."""

    def __init__(self, h, L, k_act, n_elec, ci, prec="fp64", device=0, stream=None, **opts):
        o = _lib.mpspt_default_options()
        o.device = device
        o.prec = _lib.PREC.get(prec, prec)
        if stream is not None:
            o.stream = stream
        for k, v in opts.items():
            setattr(o, k, v)
        self.ctx = _lib.mpspt_create(o)
        k = h.shape[0]
        _lib.mpspt_set_integrals(self.ctx, k_act, k - k_act, n_elec, h, L)
        _lib.mpspt_set_reference_ci(self.ctx, ci)

    def energies(self, h0):
        return _lib.mpspt_energies(self.ctx, h0)

    def minimize(self, h0, M):
        return _lib.mpspt_minimize_hylleraas(self.ctx, h0, M)

    def third_order(self, h0, psi1):
        return _lib.mpspt_third_order(self.ctx, h0, psi1)

    def close(self):
        if self.ctx:
            _lib.mpspt_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
