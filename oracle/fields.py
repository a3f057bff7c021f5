"""Oracle coefficient fields: per-wedge viscosity and the buoyancy right-hand side.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* Viscosity: one value per wedge, evaluated at the quadrature point q_c
  (Sec. 4, "eta(q_c)" in Eq. oneptenergy).  At q_c every basis function equals
  1/6, so T(q_c) is the mean of the six nodal temperatures.  Law (Sec. 8,
  Frank-Kamenetskii, eta = exp(-E (T - 1/2))), optionally multiplied by a
  radial jump factor on wedges whose mid-radius lies below r_jump (reading of
  the radial-jump configuration).
* Coarse-level viscosity (reading: the paper re-discretises on coarse grids
  without saying how eta is restricted): mean of the 8 child wedges.
* Buoyancy: f = P_bc sum_e V_e Ra T(q_c) r_hat(q_c) N_j(q_c), N_j(q_c) = 1/6,
  r_hat(q_c) = x(q_c) / |x(q_c)| with x(q_c) the mean of the six node
  coordinates (Eq. stokes with the Boussinesq buoyancy Ra T r_hat; reading:
  full T, as in the spherical benchmark setup of Sec. 8).
"""
import numpy as np

from .operators import wedge_geometry


def wedge_temperature(mesh, T_nodes, wedges=None):
    """T(q_c) per wedge = mean of the six nodal temperatures."""
    nodes = mesh.wedge_nodes(wedges)
    return T_nodes[nodes].sum(axis=1) / 6.0


def wedge_mid_radius(mesh, wedges=None):
    """(r_k + r_{k+1}) / 2 of each wedge."""
    ids = np.arange(mesh.n_wedges) if wedges is None else np.asarray(wedges)
    k = ids % (mesh.n_r - 1)
    return 0.5 * (mesh.radii[k] + mesh.radii[k + 1])


def viscosity(mesh, T_nodes, E, jump_r=None, jump_factor=1.0, wedges=None):
    """eta_e = (jump_factor if r_mid < jump_r else 1) * exp(E * (0.5 - T(q_c)))."""
    Te = wedge_temperature(mesh, T_nodes, wedges)
    eta = np.exp(E * (0.5 - Te))
    if jump_r is not None:
        eta = np.where(wedge_mid_radius(mesh, wedges) < jump_r, jump_factor * eta, eta)
    return eta


def coarsen_viscosity(fine, coarse, eta_fine):
    """Mean of the 8 child wedges (4 lateral sub-triangles x 2 radial layers).

    Children of coarse cell (I, J): for W0 the fine cells (2I,2J) W0, (2I+1,2J) W0,
    (2I,2J+1) W0 and (2I,2J) W1 (the middle triangle); for W1 the fine cells
    (2I+1,2J+1) W1, (2I,2J+1) W1, (2I+1,2J) W1 and (2I+1,2J+1) W0."""
    lab = coarse.wedge_labels()            # (d, I, J, w, K)
    d, I, J, w, K = lab.T
    Nf, nkf = fine.N, fine.n_r - 1

    def fid(d, i, j, ww, k):
        t = ((d * Nf + i) * Nf + j) * 2 + ww
        return t * nkf + k

    kids0 = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    kids1 = [(1, 1, 1), (0, 1, 1), (1, 0, 1), (1, 1, 0)]
    acc = np.zeros(coarse.n_wedges)
    for (a0, b0, w0), (a1, b1, w1) in zip(kids0, kids1):
        di = np.where(w == 0, a0, a1)
        dj = np.where(w == 0, b0, b1)
        ww = np.where(w == 0, w0, w1)
        for dk in (0, 1):
            acc += eta_fine[fid(d, 2 * I + di, 2 * J + dj, ww, 2 * K + dk)]
    return acc / 8.0


def reference_weight(mesh, rho, alpha, wedges=None):
    """rho(q_c) alpha(q_c) per wedge for reference profiles given at the node layers (rho[k],
    alpha[k] at r_k): each is the mean of its six nodal values at q_c (all N_j(q_c) = 1/6), the
    layer mean, and the buoyancy of Eq. (stokes) takes their product."""
    ids = np.arange(mesh.n_wedges) if wedges is None else np.asarray(wedges)
    k = ids % (mesh.n_r - 1)
    rho, alpha = np.asarray(rho, dtype=np.float64), np.asarray(alpha, dtype=np.float64)
    return (0.5 * (rho[k] + rho[k + 1])) * (0.5 * (alpha[k] + alpha[k + 1]))


def buoyancy_rhs(mesh, T_nodes, Ra, P=None, wedges=None, rho=None, alpha=None):
    """Right-hand side f (3, n): sum_e V_e Ra T(q_c) r_hat(q_c) / 6, projected by P if given;
    with reference profiles rho, alpha (TALA, Eq. stokes: Ra rho alpha T' r_hat, T_nodes then
    the perturbation T') each wedge's term is weighted by rho(q_c) alpha(q_c).

    Summed over the given wedges (all if None): complete at every node whose wedges are all in
    ``wedges``."""
    n = mesh.n_nodes
    nodes = mesh.wedge_nodes(wedges)
    _, V = wedge_geometry(mesh, wedges)
    Te = wedge_temperature(mesh, T_nodes, wedges)
    if rho is not None:
        Te = Te * reference_weight(mesh, rho, alpha, wedges)
    xc = mesh.node_xyz(nodes.ravel()).reshape(-1, 6, 3).sum(axis=1) / 6.0
    rhat = xc / np.linalg.norm(xc, axis=1)[:, None]
    f = np.zeros((3, n))
    for d in range(3):
        w = V * Ra * Te * rhat[:, d] / 6.0
        f[d] = np.bincount(nodes.ravel(), weights=np.repeat(w, 6), minlength=n)
    if P is not None:
        f = np.einsum("ncd,dn->cn", P, f)
    return f
