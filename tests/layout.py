"""Test helper: map between the oracle's de-duplicated numbering and the library's
per-diamond node / wedge layouts (the layouts are documented in include/terra_wedge.h)."""
import numpy as np


class LayoutMap:
    def __init__(self, info, omesh):
        N, n_r, P = info["N"], info["n_r"], info["pitch"]
        assert N == omesh.N and n_r == omesh.n_r
        self.info, self.omesh = info, omesh
        self.n_layout = info["n_layout"]
        d, k, i, j = np.meshgrid(np.arange(10), np.arange(n_r), np.arange(N + 1), np.arange(N + 1), indexing="ij")
        d, k, i, j = (a.ravel() for a in (d, k, i, j))
        self.idx = ((d * n_r + k) * (N + 1) + i) * P + j
        self.node = omesh.lat_id[d, i, j] * n_r + k
        # wedges
        d, k, i, j, w = np.meshgrid(np.arange(10), np.arange(n_r - 1), np.arange(N), np.arange(N), np.arange(2),
                                    indexing="ij")
        d, k, i, j, w = (a.ravel() for a in (d, k, i, j, w))
        self.widx = (((d * (n_r - 1) + k) * N + i) * N + j) * 2 + w
        t = ((d * N + i) * N + j) * 2 + w
        self.wedge = t * (n_r - 1) + k

    def to_layout(self, vals):
        """Oracle node values (n_nodes,) -> layout array (n_layout,), zero padding."""
        out = np.zeros(self.n_layout)
        out[self.idx] = vals[self.node]
        return out

    def from_layout(self, arr, check_copies=True):
        """Layout array -> oracle node values; every copy of a node must hold the same bits."""
        arr = np.asarray(arr)
        out = np.full(self.omesh.n_nodes, np.nan)
        out[self.node] = arr[self.idx]
        if check_copies:
            assert np.array_equal(out[self.node], arr[self.idx]), "copies of a shared node differ"
        return out

    def wedges_to_layout(self, vals):
        out = np.zeros(self.info["n_wedges"])
        out[self.widx] = vals[self.wedge]
        return out

    def wedges_from_layout(self, arr):
        out = np.empty(self.omesh.n_wedges)
        out[self.wedge] = np.asarray(arr)[self.widx]
        return out


def max_rel(got, want):
    """Normwise max-relative error max|got - want| / max|want|."""
    got, want = np.asarray(got), np.asarray(want)
    return float(np.abs(got - want).max() / np.abs(want).max())
