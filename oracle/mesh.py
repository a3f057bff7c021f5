"""Oracle mesh: radially extruded icosahedral shell (paper Sec. 2, Fig. 1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Construction, step by step as Sec. 2 describes it:

1. Icosahedral base grid with 12 vertices: north pole N, an upper ring U_k at
   latitude +atan(1/2), longitude 72 k degrees, a lower ring L_k at latitude
   -atan(1/2), longitude 36 + 72 k degrees, and the south pole S (k = 0..4).
2. Ten diamonds, each the union of two spherical triangles, IDs 0-4 north and
   5-9 south (Fig. 1a).  A diamond is stored as the lattice corners
   (c00, c10, c01, c11); its two triangles are (c00, c10, c01) and
   (c11, c01, c10), sharing the edge c10-c01.  Reading (Fig. 1a shows only the
   unfolded picture): north d = k is (N, U_k, U_k+1, L_k); south d = 5 + k is
   (U_k+1, L_k, L_k+1, S).
3. Recursive lateral midpoint refinement: every refinement halves the lattice
   spacing and places the new point of each lattice edge (i-, j- and
   anti-diagonal direction) at the normalised sum of its two end points, which
   yields 2^l x 2^l quadrilateral cells per diamond at level l.
4. Radial extrusion through N_r node layers with uniform spacing (reading of
   the paper's "flexible spacing": the configurations use uniform radii).
5. Each hexahedral cell (d, i, j, k) is split implicitly into two wedges,
   W0 = lateral (i,j), (i+1,j), (i,j+1) and W1 = (i+1,j+1), (i,j+1), (i+1,j)
   (reading of "split diagonally": the diagonal is parallel to the diamond's
   inner edge, so both wedges are midpoint-refined icosahedral triangles).
   Wedge node order follows Eq. (wedgebasis): lateral nodes 0-2 on the bottom
   layer k, then the same three on layer k+1.

Global numbering comes from de-duplicating lateral coordinates (diamond-edge
points are generated from the same end points and coincide bitwise); the node
id of lateral point L on layer k is ``L * n_r + k``.
"""
import numpy as np


def icosahedron():
    """Return the 12 base vertices as a dict of arrays (step 1)."""
    lat = np.arctan(0.5)
    north = np.array([0.0, 0.0, 1.0])
    south = np.array([0.0, 0.0, -1.0])
    upper = np.empty((5, 3))
    lower = np.empty((5, 3))
    for k in range(5):
        lon_u = 2.0 * np.pi * k / 5.0
        lon_l = np.pi / 5.0 + 2.0 * np.pi * k / 5.0
        upper[k] = [np.cos(lat) * np.cos(lon_u), np.cos(lat) * np.sin(lon_u), np.sin(lat)]
        lower[k] = [np.cos(-lat) * np.cos(lon_l), np.cos(-lat) * np.sin(lon_l), np.sin(-lat)]
    return {"N": north, "S": south, "U": upper, "L": lower}


def diamond_corners():
    """Corners (c00, c10, c01, c11) of the 10 diamonds, shape (10, 4, 3) (step 2)."""
    ico = icosahedron()
    U, L = ico["U"], ico["L"]
    out = np.empty((10, 4, 3))
    for k in range(5):
        k1 = (k + 1) % 5
        out[k] = [ico["N"], U[k], U[k1], L[k]]
        out[5 + k] = [U[k1], L[k], L[k1], ico["S"]]
    return out


def normalized_sum(p, q):
    """normalise(p + q), written out so the rounding is fixed: (x^2 + y^2) + z^2."""
    v = p + q
    nrm = np.sqrt((v[..., 0] * v[..., 0] + v[..., 1] * v[..., 1]) + v[..., 2] * v[..., 2])
    return v / nrm[..., None]


def lateral_points(level):
    """Unit-sphere lattice points of the 10 diamonds, shape (10, N+1, N+1, 3), N = 2^level (step 3)."""
    n = 1 << level
    pts = np.full((10, n + 1, n + 1, 3), np.nan)
    c = diamond_corners()
    pts[:, 0, 0] = c[:, 0]
    pts[:, n, 0] = c[:, 1]
    pts[:, 0, n] = c[:, 2]
    pts[:, n, n] = c[:, 3]
    s = n
    while s > 1:
        h = s // 2
        # i-direction edges (i, j)-(i+s, j) for lattice i, j multiples of s
        pts[:, h::s, 0::s] = normalized_sum(pts[:, 0:n:s, 0::s], pts[:, s::s, 0::s])
        # j-direction edges (i, j)-(i, j+s)
        pts[:, 0::s, h::s] = normalized_sum(pts[:, 0::s, 0:n:s], pts[:, 0::s, s::s])
        # anti-diagonal edges (i+s, j)-(i, j+s); midpoint at (i+h, j+h)
        pts[:, h::s, h::s] = normalized_sum(pts[:, s::s, 0:n:s], pts[:, 0:n:s, s::s])
        s = h
    assert not np.isnan(pts).any()
    return pts


def dedup_lateral(pts):
    """Global lateral ids by exact coordinate de-duplication.

    Returns (ids of shape (10, N+1, N+1), unique points of shape (n_lat, 3)),
    with unique points ordered lexicographically by coordinate."""
    flat = np.ascontiguousarray(pts.reshape(-1, 3))
    uniq, inv = np.unique(flat, axis=0, return_inverse=True)
    return inv.reshape(pts.shape[:3]), uniq


def uniform_radii(r_in, r_out, n_r):
    """Node radii r_k = r_in + ((r_out - r_in) * k) / (n_r - 1), k = 0..n_r-1 (step 4)."""
    k = np.arange(n_r, dtype=np.float64)
    return r_in + ((r_out - r_in) * k) / (n_r - 1)


def lateral_triangles(level):
    """Lateral wedge triangles as lattice positions (step 5).

    Returns an int array (10*N*N*2, 3, 2) of (i, j) lattice positions and an
    int array (10*N*N*2, 4) of (d, i, j, w) labels, ordered d, i, j, w."""
    n = 1 << level
    d, i, j, w = np.meshgrid(np.arange(10), np.arange(n), np.arange(n), np.arange(2), indexing="ij")
    d, i, j, w = (a.ravel() for a in (d, i, j, w))
    pos = np.empty((d.size, 3, 2), dtype=np.int64)
    # W0: (i,j), (i+1,j), (i,j+1);  W1: (i+1,j+1), (i,j+1), (i+1,j)
    w0 = w == 0
    pos[:, 0, 0] = np.where(w0, i, i + 1)
    pos[:, 0, 1] = np.where(w0, j, j + 1)
    pos[:, 1, 0] = np.where(w0, i + 1, i)
    pos[:, 1, 1] = np.where(w0, j, j + 1)
    pos[:, 2, 0] = np.where(w0, i, i + 1)
    pos[:, 2, 1] = np.where(w0, j + 1, j)
    return pos, np.stack([d, i, j, w], axis=1)


class ShellMesh:
    """Oracle shell mesh at lateral level ``level`` with ``n_r`` radial node layers.

    Attributes
    ----------
    lat_pts  : (10, N+1, N+1, 3) per-diamond lattice points
    lat_id   : (10, N+1, N+1) global lateral id of each lattice point
    lat_xyz  : (n_lat, 3) unique unit-sphere points
    radii    : (n_r,) node radii
    tri      : (n_tri, 3) global lateral ids of the wedge triangles (node order 0-2)
    tri_lab  : (n_tri, 4) (d, i, j, w) label of each triangle
    Wedge (t, k) -- triangle t extruded between layers k and k+1 -- has wedge id
    ``t * (n_r - 1) + k`` and nodes ``tri[t] * n_r + k`` then ``tri[t] * n_r + k + 1``.
    """

    def __init__(self, level, n_r, r_in, r_out):
        assert level >= 0 and n_r >= 2
        self.level, self.n_r, self.r_in, self.r_out = level, n_r, float(r_in), float(r_out)
        self.N = 1 << level
        self.lat_pts = lateral_points(level)
        self.lat_id, self.lat_xyz = dedup_lateral(self.lat_pts)
        self.n_lat = self.lat_xyz.shape[0]
        self.radii = uniform_radii(r_in, r_out, n_r)
        pos, self.tri_lab = lateral_triangles(level)
        d = self.tri_lab[:, 0]
        self.tri = self.lat_id[d[:, None], pos[:, :, 0], pos[:, :, 1]]
        self.n_tri = self.tri.shape[0]
        self.n_nodes = self.n_lat * n_r
        self.n_wedges = self.n_tri * (n_r - 1)

    # ---- node helpers -------------------------------------------------------------
    def node_xyz(self, nodes=None):
        """Coordinates x = r_k * s_L of the given global nodes (all if None)."""
        if nodes is None:
            nodes = np.arange(self.n_nodes)
        lat, k = np.divmod(np.asarray(nodes), self.n_r)
        return self.radii[k][:, None] * self.lat_xyz[lat]

    def boundary_nodes(self):
        """Boolean masks (inner, outer) over global nodes: layer 0 and layer n_r-1."""
        k = np.arange(self.n_nodes) % self.n_r
        return k == 0, k == self.n_r - 1

    # ---- wedge helpers ------------------------------------------------------------
    def wedge_nodes(self, wedges=None):
        """Global node ids (n, 6) of the given wedge ids (all if None)."""
        if wedges is None:
            wedges = np.arange(self.n_wedges)
        t, k = np.divmod(np.asarray(wedges), self.n_r - 1)
        base = self.tri[t] * self.n_r + k[:, None]
        return np.concatenate([base, base + 1], axis=1)

    def wedge_labels(self, wedges=None):
        """(d, i, j, w, k) label of each wedge id (all if None), shape (n, 5)."""
        if wedges is None:
            wedges = np.arange(self.n_wedges)
        t, k = np.divmod(np.asarray(wedges), self.n_r - 1)
        return np.concatenate([self.tri_lab[t], k[:, None]], axis=1)

    def wedges_of_nodes(self, nodes):
        """Sorted ids of all wedges that contain at least one of the given global nodes.

        A node (L, k) lies in the wedges (t, k-1) and (t, k) of every lateral
        triangle t that has L as a vertex."""
        lat, k = np.divmod(np.asarray(nodes, dtype=np.int64), self.n_r)
        if not hasattr(self, "_lat_tris"):
            rows = self.tri.ravel()
            cols = np.repeat(np.arange(self.n_tri), 3)
            order = np.argsort(rows, kind="stable")
            self._lat_tri_ptr = np.searchsorted(rows[order], np.arange(self.n_lat + 1))
            self._lat_tris = cols[order]
        out = []
        for L, kk in zip(lat.tolist(), k.tolist()):
            tris = self._lat_tris[self._lat_tri_ptr[L]:self._lat_tri_ptr[L + 1]]
            for layer in (kk - 1, kk):
                if 0 <= layer < self.n_r - 1:
                    out.append(tris * (self.n_r - 1) + layer)
        return np.unique(np.concatenate(out)) if out else np.zeros(0, dtype=np.int64)

    def node_of_layout(self, d, i, j, k):
        """Global node id of per-diamond lattice position (d, i, j) on layer k."""
        return self.lat_id[d, i, j] * self.n_r + k
