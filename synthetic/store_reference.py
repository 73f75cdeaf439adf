"""Stores the reference vector Psi0 of a named workload (sparse: indices and
values of the nonzero CI coefficients) under synthetic/data, so that every
machine reads the same bits.  Run from the repository root:
    python -m synthetic.store_reference medium [seed]
"""
import os
import sys

import numpy as np

from .integrals import EVAL_SEED, config_integrals
from .reference import fci_reference, stored_reference_path


def store(name, seed=EVAL_SEED):
    h, L, c = config_integrals(name, seed=seed)
    ci, energy = fci_reference(h, L, c["k_act"], c["n_elec"])
    idx = np.nonzero(ci)[0].astype(np.int64)
    path = stored_reference_path(name, seed)
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.savez(path, idx=idx, val=ci[idx], energy=np.float64(energy))
    return path


if __name__ == "__main__":
    name = sys.argv[1] if len(sys.argv) > 1 else "medium"
    seed = int(sys.argv[2]) if len(sys.argv) > 2 else EVAL_SEED
    print("wrote", store(name, seed))
