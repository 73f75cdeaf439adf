"""Seeded integral generator.

h_pq = S_pq + delta_pq eps_p with S symmetric, S_pq ~ N(0, 0.1^2) drawn for
p <= q; eps_act ~ U[-0.5, 0.5] (sorted), eps_virt ~ U[0.5, 3] (sorted).
L[Q,p,q] = L[Q,q,p] ~ N(0, 0.05^2) drawn for p <= q, Q < n_chol.
Draw order: eps_act, eps_virt, S (upper triangle, row-major), L (Q-major,
upper triangle row-major).  numpy PCG64 bit generator.
"""
import numpy as np

# Workload shapes: (k_act, k_virt, n_elec, n_chol).  The electron count is the
# number of active electrons of the reference; every orbital beyond the
# active ones is a virtual (no core orbitals).
CONFIGS = {
    "tiny": dict(k_act=4, k_virt=8, n_elec=4, n_chol=20),
    "medium": dict(k_act=8, k_virt=24, n_elec=8, n_chol=60),
    "partitions": dict(k_act=12, k_virt=60, n_elec=12, n_chol=150),
    "large": dict(k_act=16, k_virt=160, n_elec=16, n_chol=400),
}

EVAL_SEED = 1408
TRAIN_SEED = 5092


def integrals(seed, k_act, k_virt, n_chol, l_scale=1.0):
    """Return (h, L) for a seeded synthetic Hamiltonian (float64); the
    Cholesky entries are drawn with standard deviation 0.05 * l_scale."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = k_act + k_virt
    eps_act = np.sort(rng.uniform(-0.5, 0.5, size=k_act))
    eps_virt = np.sort(rng.uniform(0.5, 3.0, size=k_virt))
    iu = np.triu_indices(k)
    S = np.zeros((k, k))
    S[iu] = rng.normal(0.0, 0.1, size=iu[0].size)
    S = S + np.triu(S, 1).T
    h = S + np.diag(np.concatenate([eps_act, eps_virt]))
    L = np.zeros((n_chol, k, k))
    for Q in range(n_chol):
        M = np.zeros((k, k))
        M[iu] = rng.normal(0.0, 0.05 * l_scale, size=iu[0].size)
        L[Q] = M + np.triu(M, 1).T
    return np.ascontiguousarray(h), np.ascontiguousarray(L)


def config_integrals(name, seed=EVAL_SEED):
    c = CONFIGS[name]
    h, L = integrals(seed, c["k_act"], c["k_virt"], c["n_chol"], c.get("l_scale", 1.0))
    return h, L, c


def partition_bond_dims(n_part, seed=20140819, choices=(32, 64, 128, 256, 512)):
    """Uneven bond dimensions of the virtual-pair partitions: drawn uniformly
    from `choices` with numpy PCG64(seed), in partition order."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [int(choices[i]) for i in rng.integers(0, len(choices), size=n_part)]
