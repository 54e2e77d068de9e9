"""Shared helpers of the GPU parity tests: layout maps between the oracle's
unknown order and the library's block order, and relative errors."""
import numpy as np


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def oracle_to_gpu_perm(oprob, gprob):
    """Index array q with gpu_vector = oracle_vector[q] for the full unknown vector."""
    interior = oprob.grid.interior_nodes          # lattice ids, sorted (oracle order)
    ids = gprob.interior_nodes()                  # lattice ids in the library's order
    rank = np.searchsorted(interior, ids)
    assert np.array_equal(interior[rank], ids)
    uq = (2 * rank[:, None] + np.arange(2)[None, :]).ravel()
    n_u = uq.size
    rest = np.arange(n_u, oprob.I.size + 3 * oprob.N ** 2 + 4 * oprob.ref_xy.shape[0])
    return np.concatenate([uq, rest])
