"""Oracle energy update: explicit advection-diffusion of the temperature on the wedge mesh.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Eq. (energy) in the nondimensional Boussinesq form of the spherical benchmark runs (Sec. 8:
rho c_p = k = 1, no shear, adiabatic or internal heating), dT/dt + u . grad T = lap T, with the
temperature held at its values on both surfaces (T = 1 at r_in, 0 at r_out for the benchmark
family).  Readings (the paper names its schemes -- SUPG, entropy viscosity, MMOC -- without the
discrete forms):

* space: W1 wedges with the one-point rule of Sec. 4 for every integral, lumped mass
  m_j = sum_e V_e / 6;
* residual R = K T + C(u) T + S(u) T with the diffusion K_jk = sum_e V_e gradN_j . gradN_k, the
  Galerkin advection C_jk = sum_e V_e N_j(q_c) ubar_e . gradN_k (N_j(q_c) = 1/6, ubar_e the mean of
  the six nodal velocities) and the streamline-upwind term of SUPG (Brooks and Hughes 1982)
  S_jk = sum_e V_e tau_e (ubar_e . gradN_j)(ubar_e . gradN_k), all gradients at q_c;
  tau_e = h_e / (2 |ubar_e|) (coth Pe_e - 1 / Pe_e), Pe_e = |ubar_e| h_e / 2, h_e = (2 V_e)^(1/3)
  (the cube root of the hexahedral cell volume); the SUPG weight of the time derivative is dropped
  with the lumped mass;
* time: Heun's method (explicit trapezoid), T* = T - dt M^-1 R(T), T_new = (T + T* - dt M^-1 R(T*)) / 2,
  at interior nodes; surface nodes keep their values;
* Nu_top: the consistent boundary flux -- the diffusion residual (K T)_j summed over the outer
  surface nodes -- divided by the same sum for the conductive profile; V_rms with the lumped mass.
"""
import numpy as np
import scipy.sparse as sp

from .operators import wedge_geometry


def wedge_velocity(mesh, u, wedges=None):
    """ubar_e: mean of the six nodal velocities, (n, 3)."""
    nodes = mesh.wedge_nodes(wedges)
    return np.stack([u[c][nodes].mean(axis=1) for c in range(3)], axis=1)


def supg_tau(V, ubar):
    """tau_e = h / (2 |ubar|) (coth Pe - 1 / Pe), Pe = |ubar| h / 2, h = (2 V)^(1/3); 0 where ubar = 0."""
    h = np.cbrt(2.0 * V)
    un = np.linalg.norm(ubar, axis=1)
    pe = un * h / 2.0
    tau = np.zeros_like(V)
    big = pe > 1e-3
    tau[big] = h[big] / (2.0 * un[big]) * (1.0 / np.tanh(pe[big]) - 1.0 / pe[big])
    # small Pe: coth(x) - 1/x = x/3 - x^3/45 + ..., so tau = h^2 / 12 (1 - Pe^2 / 15)
    small = ~big
    tau[small] = h[small] ** 2 / 12.0 * (1.0 - pe[small] ** 2 / 15.0)
    return tau


def lumped_mass(mesh):
    _, V = wedge_geometry(mesh)
    return np.bincount(mesh.wedge_nodes().ravel(), weights=np.repeat(V / 6.0, 6), minlength=mesh.n_nodes)


def assemble_energy(mesh, u=None, supg=True):
    """(K, C + S) as sparse n x n matrices for the velocity u (3, n) (C + S = 0 without u)."""
    n = mesh.n_nodes
    nodes = mesh.wedge_nodes()
    grad, V = wedge_geometry(mesh)                        # grad (m, 6, 3)
    rows = np.repeat(nodes, 6, axis=1).ravel()
    cols = np.tile(nodes, (1, 6)).ravel()
    Ke = V[:, None, None] * np.einsum("ejx,ekx->ejk", grad, grad)
    K = sp.csr_matrix((Ke.ravel(), (rows, cols)), shape=(n, n))
    if u is None:
        return K, sp.csr_matrix((n, n))
    ub = wedge_velocity(mesh, u)
    ug = np.einsum("ex,ekx->ek", ub, grad)                # ubar . gradN_k
    Ce = (V / 6.0)[:, None, None] * np.broadcast_to(ug[:, None, :], (len(V), 6, 6))
    if supg:
        tau = supg_tau(V, ub)
        Ce = Ce + (V * tau)[:, None, None] * ug[:, :, None] * ug[:, None, :]
    C = sp.csr_matrix((Ce.ravel(), (rows, cols)), shape=(n, n))
    return K, C


def heun_steps(mesh, T, u, dt, n_steps, supg=True):
    """n_steps Heun steps of size dt with fixed velocity u; surface nodes keep their values."""
    K, C = assemble_energy(mesh, u, supg)
    R = (K + C).tocsr()
    m = lumped_mass(mesh)
    inner, outer = mesh.boundary_nodes()
    free = ~(inner | outer)
    T = np.array(T, dtype=np.float64)
    for _ in range(n_steps):
        t1 = T.copy()
        t1[free] -= dt * (R @ T)[free] / m[free]
        t2 = T.copy()
        t2[free] = 0.5 * (T[free] + t1[free] - dt * (R @ t1)[free] / m[free])
        T = t2
    return T


def nusselt_top(mesh, T, T_conductive):
    """Consistent heat flux through the outer surface, relative to the conductive profile's."""
    K, _ = assemble_energy(mesh)
    _, outer = mesh.boundary_nodes()
    return float((K @ T)[outer].sum() / (K @ T_conductive)[outer].sum())


def v_rms(mesh, u):
    m = lumped_mass(mesh)
    return float(np.sqrt(np.sum(m * np.sum(np.asarray(u) ** 2, axis=0)) / m.sum()))
