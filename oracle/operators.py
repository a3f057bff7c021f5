"""Oracle global operators of the W1-iso-W2 / W1 wedge Stokes discretisation.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Velocity DoFs are numbered component-major: dof(c, node) = c * n_nodes + node.
Vectors are arrays of shape (3, n_nodes) (velocity) or (n_pnodes,) (pressure).

* A   -- viscous block, y = sum_e I_e^T A_e I_e x (Eq. matfree, Eq. elemmat),
         assembled (CSR) or applied element by element.
* B   -- divergence.  Pressure lives on the grid one level coarser in both
         the lateral and the radial direction (Sec. 3): p in W1 on level l-1.
         Reading of "iso": the pressure function on the fine mesh is the fine
         W1 interpolant of P p, P the nested iso-interpolation (weight 1 at
         coincident nodes, 1/2 at lateral or radial edge midpoints, 1/4 where
         both apply).  With the one-point rule,
             B[k, (j, d)] = - sum_e V_e psi_k(q_c^e) dN_j/dx_d (q_c^e),
             psi_k(q_c^e) = (1/6) sum_{fine nodes n of e} P[n, k].
         The minus sign makes the saddle matrix [[A, B^T], [B, 0]] (Sec. 7).
* Constraints (reading: the paper names free-slip, not how it is imposed):
  at boundary nodes P_j = I - s_j s_j^T (free-slip, s_j the unit radial
  direction) or P_j = 0 (no-slip); the constrained blocks are
  P A P + (I - P), B P and P B^T.
* diag(M_{1/eta}) -- Eq. (pmass), one-point rule on the fine wedges:
  sum_e V_e / eta_e psi_k(q_c^e)^2.
"""
import numpy as np
import scipy.sparse as sp

from .element import (geometry, hourglass_base_vectors, hourglass_stabilised, quadrature_rule,
                      viscous_element_matrix, viscous_element_matrix_rule)
from .mesh import ShellMesh

FREE, NOSLIP = "free", "noslip"


# ----------------------------------------------------------------------------- geometry
def wedge_geometry(mesh, wedges=None):
    """grad N_j(q_c) (n, 6, 3) and V_e (n,) of the given wedges (all if None)."""
    nodes = mesh.wedge_nodes(wedges)
    x = mesh.node_xyz(nodes.ravel()).reshape(-1, 6, 3)
    _, _, grad, V = geometry(x)
    return grad, V


def element_matrices(mesh, eta, wedges, div_term=True, kappa=0.0, quad=1):
    """Element matrices (n, 18, 18) of the given wedges: Eq. (elemmat) under the one-point rule
    (quad = 1) or with a second radial point (quad = 2), plus the hourglass control of
    Eq. (hgstab) when kappa > 0 (see ``oracle.element``)."""
    nodes = mesh.wedge_nodes(wedges)
    x = mesh.node_xyz(nodes.ravel()).reshape(-1, 6, 3)
    _, _, grad, V = geometry(x)
    if quad == 1:
        A = viscous_element_matrix(grad, V, eta, div_term)
    else:
        A = viscous_element_matrix_rule(x, eta, quadrature_rule(quad), div_term)
    if kappa > 0.0:
        A = hourglass_stabilised(A, hourglass_base_vectors(x, grad), kappa)
    return A


def _chunks(ids, size):
    for s in range(0, len(ids), size):
        yield ids[s:s + size]


# ----------------------------------------------------------------------------- viscous block A
def assemble_A(mesh, eta, div_term=True, kappa=0.0, quad=1):
    """Assembled A (3n x 3n CSR) from the element matrices, Eq. (matfree); kappa > 0 adds the
    hourglass control of Eq. (hgstab), quad = 2 takes the second radial quadrature point."""
    n = mesh.n_nodes
    nodes = mesh.wedge_nodes()
    Ae = element_matrices(mesh, eta, np.arange(mesh.n_wedges), div_term, kappa, quad)   # a = 3 j + d
    dof = (np.arange(3)[None, None, :] * n + nodes[:, :, None]).reshape(-1, 18)
    rows = np.repeat(dof, 18, axis=1).ravel()
    cols = np.tile(dof, (1, 18)).ravel()
    return sp.csr_matrix((Ae.ravel(), (rows, cols)), shape=(3 * n, 3 * n))


def apply_A(mesh, eta, u, wedges=None, div_term=True, chunk=50000, kappa=0.0, quad=1):
    """Matrix-free y = sum_e I_e^T A_e I_e u over the given wedges (all if None).

    u: (3, n_nodes).  Element matrices are formed explicitly per wedge."""
    n = mesh.n_nodes
    y = np.zeros((3, n))
    ids = np.arange(mesh.n_wedges) if wedges is None else np.asarray(wedges)
    for ch in _chunks(ids, chunk):
        nodes = mesh.wedge_nodes(ch)
        Ae = element_matrices(mesh, eta[ch], ch, div_term, kappa, quad)
        ue = np.transpose(u[:, nodes], (1, 2, 0)).reshape(-1, 18)   # ue[e, 3 j + d]
        ye = np.einsum("eab,eb->ea", Ae, ue).reshape(-1, 6, 3)
        for d in range(3):
            y[d] += np.bincount(nodes.ravel(), weights=ye[:, :, d].ravel(), minlength=n)
    return y


# ----------------------------------------------------------------------------- constraints
def boundary_projectors(mesh, bc=(FREE, FREE)):
    """Per-node 3x3 projectors P_j (n, 3, 3): identity in the interior,
    I - s s^T (free-slip) or 0 (no-slip) on layer 0 (bc[0]) and layer n_r-1 (bc[1])."""
    n = mesh.n_nodes
    P = np.broadcast_to(np.eye(3), (n, 3, 3)).copy()
    inner, outer = mesh.boundary_nodes()
    lat = np.arange(n) // mesh.n_r
    for mask, kind in ((inner, bc[0]), (outer, bc[1])):
        s = mesh.lat_xyz[lat[mask]]
        if kind == FREE:
            P[mask] = np.eye(3)[None] - np.einsum("nc,nd->ncd", s, s)
        elif kind == NOSLIP:
            P[mask] = 0.0
        else:
            raise ValueError(kind)
    return P


def projector_matrix(P):
    """Sparse (3n x 3n) matrix of the node-wise projectors in component-major numbering."""
    n = P.shape[0]
    rows, cols, vals = [], [], []
    for c in range(3):
        for d in range(3):
            rows.append(c * n + np.arange(n))
            cols.append(d * n + np.arange(n))
            vals.append(P[:, c, d])
    M = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(3 * n, 3 * n))
    M.eliminate_zeros()
    return M


def project(P, u):
    """Apply node-wise projectors P (n,3,3) to a velocity field u (3, n)."""
    return np.einsum("ncd,dn->cn", P, u)


def constrain_A(Amat, Pm):
    """P A P + (I - P) for assembled matrices."""
    I = sp.identity(Amat.shape[0], format="csr")
    return (Pm @ Amat @ Pm + (I - Pm)).tocsr()


def apply_A_constrained(mesh, eta, u, P, wedges=None, div_term=True, kappa=0.0, quad=1):
    """Matrix-free (P A P + (I - P)) u; complete at every node whose wedges are all in ``wedges``."""
    pu = project(P, u)
    return project(P, apply_A(mesh, eta, pu, wedges, div_term, kappa=kappa, quad=quad)) + (u - pu)


# ----------------------------------------------------------------------------- pressure space
def pressure_mesh(mesh):
    """Pressure mesh: one level coarser laterally and radially, Sec. 3."""
    assert mesh.level >= 1 and (mesh.n_r - 1) % 2 == 0
    return ShellMesh(mesh.level - 1, (mesh.n_r - 1) // 2 + 1, mesh.r_in, mesh.r_out)


def _lateral_parents(i, j):
    """Coarse lattice parents and weights of fine lattice position (i, j) under nested
    midpoint refinement: returns list of ((I, J), w)."""
    if i % 2 == 0 and j % 2 == 0:
        return [((i // 2, j // 2), 1.0)]
    if i % 2 == 1 and j % 2 == 0:
        return [(((i - 1) // 2, j // 2), 0.5), (((i + 1) // 2, j // 2), 0.5)]
    if i % 2 == 0 and j % 2 == 1:
        return [((i // 2, (j - 1) // 2), 0.5), ((i // 2, (j + 1) // 2), 0.5)]
    # midpoint of the coarse anti-diagonal edge (I+1, J)-(I, J+1)
    return [(((i + 1) // 2, (j - 1) // 2), 0.5), (((i - 1) // 2, (j + 1) // 2), 0.5)]


def lateral_prolongation(fine, coarse):
    """Sparse (n_lat_fine x n_lat_coarse) nested lateral interpolation."""
    N = fine.N
    first = np.unique(fine.lat_id.ravel(), return_index=True)[1]
    d_all, i_all, j_all = np.unravel_index(first, fine.lat_id.shape)
    rows, cols, vals = [], [], []
    for d, i, j in zip(d_all.tolist(), i_all.tolist(), j_all.tolist()):
        r = fine.lat_id[d, i, j]
        for (I, J), w in _lateral_parents(i, j):
            rows.append(r)
            cols.append(coarse.lat_id[d, I, J])
            vals.append(w)
    assert N == 2 * coarse.N
    return sp.csr_matrix((vals, (rows, cols)), shape=(fine.n_lat, coarse.n_lat))


def radial_prolongation(n_r_fine, n_r_coarse):
    """Sparse (n_r_fine x n_r_coarse) radial interpolation (1 / (1/2, 1/2))."""
    assert n_r_fine == 2 * (n_r_coarse - 1) + 1
    rows, cols, vals = [], [], []
    for k in range(n_r_fine):
        if k % 2 == 0:
            rows.append(k); cols.append(k // 2); vals.append(1.0)
        else:
            rows += [k, k]; cols += [(k - 1) // 2, (k + 1) // 2]; vals += [0.5, 0.5]
    return sp.csr_matrix((vals, (rows, cols)), shape=(n_r_fine, n_r_coarse))


def prolongation(fine, coarse):
    """Nested iso-interpolation between node sets (n_fine x n_coarse), node = L * n_r + k."""
    return sp.kron(lateral_prolongation(fine, coarse), radial_prolongation(fine.n_r, coarse.n_r), format="csr")


def wedge_incidence(mesh, wedges=None):
    """Sparse (n_wedges x n_nodes) incidence, 1 at the six nodes of each wedge."""
    ids = np.arange(mesh.n_wedges) if wedges is None else np.asarray(wedges)
    nodes = mesh.wedge_nodes(ids)
    rows = np.repeat(np.arange(len(ids)), 6)
    return sp.csr_matrix((np.ones(nodes.size), (rows, nodes.ravel())), shape=(len(ids), mesh.n_nodes))


def psi_at_centroids(mesh, Pp, wedges=None):
    """Psi[e, k] = psi_k(q_c^e) = (1/6) sum_{n in e} P[n, k]  (n_wedges x n_pnodes)."""
    return (wedge_incidence(mesh, wedges) @ Pp / 6.0).tocsr()


def assemble_B(mesh, Pp, wedges=None, rho=None):
    """Assembled B (n_p x 3 n): B[k, (j,d)] = - sum_e V_e psi_k(q_c^e) dN_j/dx_d (q_c^e).

    With a reference density rho (one value per node layer, rho[k] at r_k) this is the divergence
    of Eq. (mass), div(rho u) (TALA, Sec. 1).  Reading (the paper states the continuous equation
    only): the product rule at the quadrature point,
        div(rho u)(q_c) = rho(q_c) div u_h(q_c) + rho'(q_c) r_hat(q_c) . u_h(q_c),
    with rho(q_c) = (rho_k + rho_k+1) / 2 and rho'(q_c) = (rho_k+1 - rho_k) / (r_k+1 - r_k) of the
    radial P1 interpolant, r_hat(q_c) = x(q_c) / |x(q_c)| and u_h(q_c) the mean of the six nodal
    values (N_j(q_c) = 1/6), so B[k, (j,d)] = - sum_e V_e psi_k(q_c) (rho_e dN_j/dx_d + rho'_e
    r_hat_d / 6).  Rigid rotations keep div(rho u) = 0 exactly: their discrete divergence vanishes
    per wedge and u_h(q_c) = omega x x(q_c) is orthogonal to r_hat(q_c)."""
    n = mesh.n_nodes
    ids = np.arange(mesh.n_wedges) if wedges is None else np.asarray(wedges)
    nodes = mesh.wedge_nodes(ids)
    grad, V = wedge_geometry(mesh, ids)
    Psi = psi_at_centroids(mesh, Pp, ids)                          # (m, n_p)
    # D[e, d*n + node_j] = -V_e dN_j/dx_d  (times rho_e, plus the rho' r_hat term with a reference state)
    rows = np.repeat(np.arange(len(ids)), 18)
    cols = (np.arange(3)[None, None, :] * n + nodes[:, :, None]).ravel()
    if rho is None:
        vals = (-V[:, None, None] * grad).ravel()
    else:
        rho = np.asarray(rho, dtype=np.float64)
        k = ids % (mesh.n_r - 1)
        rho_e = 0.5 * (rho[k] + rho[k + 1])
        drho_e = (rho[k + 1] - rho[k]) / (mesh.radii[k + 1] - mesh.radii[k])
        xc = mesh.node_xyz(nodes.ravel()).reshape(-1, 6, 3).mean(axis=1)
        rhat = xc / np.linalg.norm(xc, axis=1)[:, None]
        term = rho_e[:, None, None] * grad + (drho_e[:, None] * rhat / 6.0)[:, None, :]
        vals = (-V[:, None, None] * term).ravel()
    D = sp.csr_matrix((vals, (rows, cols)), shape=(len(ids), 3 * n))
    return (Psi.T @ D).tocsr()


def diag_pressure_mass(mesh, Pp, eta):
    """diag(M_{1/eta})_k = sum_e V_e eta_e^{-1} psi_k(q_c^e)^2, Eq. (pmass), one-point rule."""
    _, V = wedge_geometry(mesh)
    Psi = psi_at_centroids(mesh, Pp)
    return np.asarray(Psi.multiply(Psi).T @ (V / eta)).ravel()


# ----------------------------------------------------------------------------- diagonal of A
def diag_A_constrained(mesh, eta, P, div_term=True, chunk=50000, wedges=None, kappa=0.0, quad=1):
    """Diagonal of P A P + (I - P), shape (3, n), from the 3x3 node blocks of A.

    The node block A_jj is accumulated element by element from the explicit
    element matrices (over the given wedges, all if None); the constrained
    block is P_j A_jj P_j + I - P_j."""
    n = mesh.n_nodes
    blocks = np.zeros((n, 3, 3))
    ids = np.arange(mesh.n_wedges) if wedges is None else np.asarray(wedges)
    for ch in _chunks(ids, chunk):
        nodes = mesh.wedge_nodes(ch)
        Ae = element_matrices(mesh, eta[ch], ch, div_term, kappa, quad).reshape(-1, 6, 3, 6, 3)
        for j in range(6):
            blk = Ae[:, j, :, j, :]
            for c in range(3):
                for d in range(3):
                    blocks[:, c, d] += np.bincount(nodes[:, j], weights=blk[:, c, d], minlength=n)
    cb = np.einsum("nab,nbc,ncd->nad", P, blocks, P) + (np.eye(3)[None] - P)
    return np.stack([cb[:, c, c] for c in range(3)])
