"""Oracle element kernels: W1 wedge basis and one-point quadrature.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* Basis, Eq. (wedgebasis): N_j = N^lat_{j mod 3}(xi, eta) N^rad_{floor(j/3)}(zeta)
  with N^lat = (1 - xi - eta, xi, eta), N^rad = ((1 - zeta)/2, (1 + zeta)/2) on
  the reference wedge xi, eta >= 0, xi + eta <= 1, zeta in [-1, 1].
* One quadrature point at the barycentre q_c = (1/3, 1/3, 0) with weight
  w_q = 1 (the reference wedge's volume), Sec. 4, Eq. (oneptenergy).
* Geometry (reading: the paper does not state the map): isoparametric,
  x(xi, eta, zeta) = sum_j N_j x_j; J = dx/d(xi, eta, zeta) at q_c;
  V_e = w_q |det J(q_c)|; grad N_j(q_c) = J^{-T} grad_ref N_j(q_c).
* Viscous element matrix, Eq. (elemmat) under the one-point rule:
  (A_e)_{ab} = V_e eta_e [2 eps(phi_a) : eps(phi_b) - 2/3 div(phi_a) div(phi_b)]
  for vector basis functions phi_a = N_j e_d, a = 3 j + d.
* Hourglass control, Eq. (hgstab): A_e + eps_e sum_m sum_d (g_m x e_d)(g_m x e_d)^T.
  Readings (the paper leaves both open): g_m are the nodal hourglass vectors w_m of
  Eq. (hourglass) with their physical linear part removed, g_m = w_m - sum_c (w_m . X_c) dN/dx_c,
  the hourglass base vectors of Flanagan & Belytschko (1981) -- so that rigid motions and every
  linear field keep zero stabilisation energy; eps_e = kappa tr(A_e) / 18, kappa times the mean
  diagonal entry of the element matrix ("scaled with the local stiffness").
* Second radial quadrature point, the other remedy of Sec. 4 for the one-point hourglass modes.
  Reading (the paper names the variant only): the two-point Gauss-Legendre rule in zeta at the
  lateral barycentre, points (1/3, 1/3, -/+ 1/sqrt 3), weight 1/2 each (triangle area 1/2 times
  the Gauss weight 1), so the weights still sum to the reference wedge's volume; eta_e is the same
  at both points (one viscosity per wedge, as for the one-point rule).  A_e is then
  sum_q w_q |det J_q| eta_e [2 eps_q(phi_a) : eps_q(phi_b) - 2/3 div_q(phi_a) div_q(phi_b)].
"""
import numpy as np

QC = (1.0 / 3.0, 1.0 / 3.0, 0.0)


def basis(xi, eta, zeta):
    """The six basis values N_j(xi, eta, zeta), Eq. (wedgebasis)."""
    lat = np.array([1.0 - xi - eta, xi, eta])
    rad = np.array([0.5 * (1.0 - zeta), 0.5 * (1.0 + zeta)])
    return np.array([lat[j % 3] * rad[j // 3] for j in range(6)])


def basis_ref_gradients(xi, eta, zeta):
    """Reference gradients dN_j/d(xi, eta, zeta), shape (6, 3), differentiated by hand
    from Eq. (wedgebasis)."""
    lat = np.array([1.0 - xi - eta, xi, eta])
    dlat = np.array([[-1.0, -1.0], [1.0, 0.0], [0.0, 1.0]])
    rad = np.array([0.5 * (1.0 - zeta), 0.5 * (1.0 + zeta)])
    drad = np.array([-0.5, 0.5])
    g = np.empty((6, 3))
    for j in range(6):
        a, b = j % 3, j // 3
        g[j] = [dlat[a, 0] * rad[b], dlat[a, 1] * rad[b], lat[a] * drad[b]]
    return g


GHAT = basis_ref_gradients(*QC)


def quadrature_rule(radial_points=1):
    """Quadrature points and weights of the reference wedge: the barycentre with weight 1
    (radial_points = 1), or the two-point Gauss-Legendre rule in zeta at the lateral barycentre
    with weights 1/2 (radial_points = 2)."""
    if radial_points == 1:
        return [(QC, 1.0)]
    if radial_points == 2:
        z = 1.0 / np.sqrt(3.0)
        return [((1.0 / 3.0, 1.0 / 3.0, -z), 0.5), ((1.0 / 3.0, 1.0 / 3.0, z), 0.5)]
    raise ValueError(radial_points)


def geometry(x):
    """One-point geometry of wedges with node coordinates ``x`` (n, 6, 3).

    Returns (J (n,3,3), detJ (n,), grad (n,6,3) = grad N_j(q_c), V (n,))."""
    J = np.einsum("njc,jm->ncm", x, GHAT)          # J[c, m] = sum_j x_j[c] dN_j/dref_m
    detJ = np.linalg.det(J)
    Jinv = np.linalg.inv(J)
    grad = np.einsum("jm,nmc->njc", GHAT, Jinv)    # grad N_j = J^{-T} ghat_j
    V = 1.0 * np.abs(detJ)                          # w_q = 1
    return J, detJ, grad, V


def geometry_at(x, point, weight):
    """Geometry of wedges with node coordinates ``x`` (n, 6, 3) at one quadrature point.

    Returns (grad (n,6,3) = grad N_j(point), V (n,) = weight |det J(point)|)."""
    g = basis_ref_gradients(*point)
    J = np.einsum("njc,jm->ncm", x, g)
    grad = np.einsum("jm,nmc->njc", g, np.linalg.inv(J))
    return grad, weight * np.abs(np.linalg.det(J))


def vector_basis_strain(grad):
    """eps(phi_a) and div(phi_a) for phi_a = N_j e_d, a = 3 j + d.

    Returns (eps (n, 18, 3, 3), div (n, 18))."""
    n = grad.shape[0]
    gradphi = np.zeros((n, 18, 3, 3))               # gradphi[a][c, m] = d(phi_a)_c / dx_m
    for j in range(6):
        for d in range(3):
            gradphi[:, 3 * j + d, d, :] = grad[:, j, :]
    eps = 0.5 * (gradphi + np.swapaxes(gradphi, 2, 3))
    div = np.trace(gradphi, axis1=2, axis2=3)
    return eps, div


def viscous_element_matrix(grad, V, eta, div_term=True):
    """(A_e) of Eq. (elemmat) with one-point quadrature, shape (n, 18, 18).

    ``div_term=False`` drops the -2/3 div div term (incompressible form)."""
    eps, div = vector_basis_strain(grad)
    A = 2.0 * np.einsum("nacm,nbcm->nab", eps, eps)
    if div_term:
        A = A - (2.0 / 3.0) * np.einsum("na,nb->nab", div, div)
    return (V * eta)[:, None, None] * A


def viscous_element_matrix_rule(x, eta, rule, div_term=True):
    """(A_e) of Eq. (elemmat) under a quadrature rule [(point, weight), ...], shape (n, 18, 18),
    with one viscosity per wedge."""
    A = 0.0
    for point, weight in rule:
        grad, V = geometry_at(x, point, weight)
        A = A + viscous_element_matrix(grad, V, eta, div_term)
    return A


def hourglass_vectors():
    """Nodal values of w1 = (xi - 1/3) zeta and w2 = (eta - 1/3) zeta, Eq. (hourglass), shape (2, 6)."""
    nodes = [(0.0, 0.0, -1.0), (1.0, 0.0, -1.0), (0.0, 1.0, -1.0),
             (0.0, 0.0, 1.0), (1.0, 0.0, 1.0), (0.0, 1.0, 1.0)]
    w1 = np.array([(xi - 1.0 / 3.0) * z for xi, _, z in nodes])
    w2 = np.array([(et - 1.0 / 3.0) * z for _, et, z in nodes])
    return np.stack([w1, w2])


def hourglass_base_vectors(x, grad):
    """g_m = w_m - sum_c (w_m . X_c) grad N(q_c)[:, c] per wedge, shape (n, 2, 6), from node
    coordinates ``x`` (n, 6, 3) and gradients ``grad`` (n, 6, 3) (Flanagan & Belytschko 1981)."""
    w = hourglass_vectors()
    wX = np.einsum("mj,njc->nmc", w, x)
    return w[None] - np.einsum("nmc,njc->nmj", wX, grad)


def hourglass_stabilised(A, g, kappa):
    """Eq. (hgstab) on element matrices A (n, 18, 18) with base vectors g (n, 2, 6) and
    eps_e = kappa tr(A_e) / 18; DoF a = 3 j + d."""
    eps = kappa * np.einsum("naa->n", A) / 18.0
    S = np.zeros_like(A)
    for m in range(2):
        G = np.einsum("ni,nj->nij", g[:, m], g[:, m])
        for d in range(3):
            S[:, d::3, d::3] += G
    return A + eps[:, None, None] * S
