"""All-core evaluation of the oracle's sparse products (test infrastructure, CPU baseline only).

The oracle's V-cycle and PCG spend their time in sparse matrix-vector products (A_l x, P e,
P^T r).  ``threaded(H, A, nthreads)`` returns the same hierarchy and fine matrix with every
sparse operator replaced by ``RowSplit``: the rows are cut into `nthreads` contiguous blocks
and the blocks' products run on a thread pool (scipy's sparse kernels release the GIL).  Each
row's sum is formed exactly as in the single-threaded product (same entries, same order), so
the results are the same bits; only the wall time changes.  Nothing else of the oracle changes.
"""
from __future__ import annotations

from concurrent.futures import ThreadPoolExecutor
from dataclasses import replace

import numpy as np
import scipy.sparse as sp


class RowSplit:
    """A CSR matrix whose products run on row blocks in parallel threads."""

    def __init__(self, M, pool: ThreadPoolExecutor, nthreads: int):
        self.M = sp.csr_matrix(M)
        self.shape = self.M.shape
        self.dtype = self.M.dtype
        self.pool = pool
        self.nthreads = nthreads
        cut = np.linspace(0, self.shape[0], nthreads + 1).astype(np.int64)
        self.blocks = [self.M[cut[i]:cut[i + 1]] for i in range(nthreads) if cut[i + 1] > cut[i]]
        self._T = None

    def __matmul__(self, x):
        parts = list(self.pool.map(lambda B: B @ x, self.blocks))
        return np.concatenate(parts)

    @property
    def T(self):
        if self._T is None:
            self._T = RowSplit(self.M.T.tocsr(), self.pool, self.nthreads)
        return self._T

    def diagonal(self):
        return self.M.diagonal()

    def toarray(self):
        return self.M.toarray()


def threaded(H, A, nthreads: int):
    """(H', A'): the hierarchy and fine matrix with row-split parallel sparse products."""
    pool = ThreadPoolExecutor(max(1, nthreads))
    wrap = lambda M: RowSplit(M, pool, max(1, nthreads))
    Hp = replace(H, A=[wrap(M) for M in H.A], P=[wrap(M) for M in H.P])
    return Hp, wrap(A)
