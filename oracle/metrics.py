"""TEST INFRASTRUCTURE ONLY: triangle-derived metrics by definition (numpy).

The paper names clustering coefficient and transitivity as the immediate use
of the counts (Sec. 5).  With d(v) the undirected degree:
  wedges(v) = d(v)(d(v)-1)/2, c(v) = t(v)/wedges(v) (0 when d(v) < 2),
  transitivity = 3T / sum_v wedges(v) (0 without wedges).
Each ratio is one float64 division of exact integers.  Pinned in
tests/test_oracle_metrics.py against networkx and closed forms.
"""
from __future__ import annotations

import numpy as np


def wedges(row_ptr) -> np.ndarray:
    d = np.diff(np.asarray(row_ptr, dtype=np.int64))
    return d * (d - 1) // 2


def local_clustering(row_ptr, t) -> np.ndarray:
    w = wedges(row_ptr)
    t = np.asarray(t, dtype=np.int64)
    out = np.zeros(w.shape[0], dtype=np.float64)
    nz = w > 0
    out[nz] = t[nz].astype(np.float64) / w[nz].astype(np.float64)
    return out


def transitivity(T: int, row_ptr) -> float:
    W = int(wedges(row_ptr).sum())
    return float(3 * int(T)) / float(W) if W else 0.0
