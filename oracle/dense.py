"""TEST INFRASTRUCTURE ONLY: the paper's matrix formulation, dense and tiny.

Alg. 3 (Sec. 3.3, after Azad, Buluc and Gilbert): order the rows of the
adjacency matrix A by increasing number of nonzeros, split A = L + U into its
strictly lower and strictly upper triangles, form B = L U (B[i][j] counts the
wedges i-k-j with k before both i and j), take the Hadamard product C = A o B
and return half the sum of C.  The printed last line of Alg. 3 sums A; the
Fig. 3 caption sums C, which is the reading taken here.

This is a second formulation of the same count (Sec. 4.3 cites Schank and
Wagner for the equivalence), so tests use it to cross-check the forward
oracle.  It uses numpy's integer matmul as its only library step.
"""
from __future__ import annotations

import numpy as np


def alg3_matrices(A: np.ndarray, permute: bool = True):
    """Return (order, L, U, B, C, T) for a dense symmetric 0/1 matrix A.

    With ``permute`` the rows/columns are first ordered by increasing nonzero
    count (ties by index), as Alg. 3 step 1 states.  Fig. 3 prints L, U, B and
    C of the example in its given vertex order, i.e. with ``permute=False``.
    """
    A = np.asarray(A, dtype=np.int64)
    n = A.shape[0]
    if permute:
        nnz = A.sum(axis=1)
        order = np.lexsort((np.arange(n), nnz))
    else:
        order = np.arange(n)
    P = A[np.ix_(order, order)]
    L = np.tril(P, -1)
    U = np.triu(P, 1)
    B = L @ U
    C = P * B
    total = int(C.sum())
    assert total % 2 == 0
    return order, L, U, B, C, total // 2


def alg3_count(A: np.ndarray, permute: bool = True) -> int:
    return alg3_matrices(A, permute)[-1]
