"""Seeded synthetic inputs for MPS-PT.

This module is the only code shared by the CPU oracle (``oracle/``) and the
GPU library (``paper_1408_5092_gb300``).  It holds no arithmetic of the
perturbation method itself: it draws integrals from a seeded generator and
produces the reference wavefunction Psi0, which the method takes as given
(Sharma & Chan, Eq. 1: "E0 and Psi0 are the zeroth order energy and
wavefunction").  The paper's N2/cc-pVXZ integrals are not available; these
draws stand in for them with the shapes of the paper's workloads.

Conventions (shared by every consumer):

* spatial orbitals p = 0..k-1, active orbitals first (0..k_act-1), then
  virtual orbitals;
* one-electron integrals ``h`` (k x k, symmetric) and a symmetric Cholesky-like
  factor ``L`` (n_chol x k x k) with (pq|rs) = sum_Q L[Q,p,q] L[Q,r,s];
* the reference is returned as a dense vector over the 4**k_act occupation
  strings of the active sites.  Site p holds one of |0>, |a>, |b>, |ab>
  (codes 0,1,2,3), the string index is sum_p code_p * 4**(k_act-1-p), and the
  basis state is the product of creators in ascending spin-orbital order
  (p0a, p0b, p1a, p1b, ...) applied to the vacuum.
"""
from .integrals import integrals, config_integrals, partition_bond_dims, CONFIGS, EVAL_SEED, TRAIN_SEED
from .reference import config_reference, fci_reference

__all__ = ["integrals", "config_integrals", "partition_bond_dims", "CONFIGS", "EVAL_SEED", "TRAIN_SEED",
           "fci_reference", "config_reference"]
