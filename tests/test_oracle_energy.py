"""Pins of the oracle's energy update (Eq. energy, nondimensional Boussinesq form; CPU only)."""
import numpy as np

from oracle import energy as E
from oracle.mesh import ShellMesh
from paper_2609_21633_gb300 import inputs

R_IN, R_OUT = 0.55, 1.0


def rotation(m, om):
    return np.cross(om[None, :], m.node_xyz()).T


def test_operators_leave_constants_and_conserve():
    m = ShellMesh(3, 9, R_IN, R_OUT)
    u = rotation(m, np.array([0.2, -0.5, 1.0])) + 0.1 * inputs.normal((3, m.n_nodes), 1)
    K, C = E.assemble_energy(m, u)
    one = np.ones(m.n_nodes)
    assert np.abs(K @ one).max() <= 1e-13 * abs(K).max()              # grad 1 = 0
    assert np.abs(C @ one).max() <= 1e-13 * abs(C).max()
    assert abs(K - K.T).max() <= 1e-15 * abs(K).max()
    T = inputs.normal(m.n_nodes, 2)
    assert T @ (K @ T) > 0
    # diffusion and the streamline term conserve sum_j: 1^T K = 0 and 1^T S = 0 (sum_j gradN_j = 0)
    assert abs(one @ (K @ T)) <= 1e-12 * np.abs(K @ T).sum()
    _, C0 = E.assemble_energy(m, u, supg=False)
    S = C - C0
    assert abs(one @ (S @ T)) <= 1e-12 * np.abs(S @ T).sum()


def test_radial_dirichlet_mode_rayleigh_quotient_converges():
    """phi = sin(pi (r - r_in) / d) / r is an eigenfunction of -lap with zero values on both
    surfaces, eigenvalue (pi / d)^2; the discrete Rayleigh quotient phi^T K phi / phi^T M phi of its
    interpolant converges to it at second order (a wrong gradient scale or a dropped V_e moves it)."""
    d = R_OUT - R_IN
    lam = (np.pi / d) ** 2
    errs = []
    for level, n_r in ((2, 5), (3, 9), (4, 17)):
        m = ShellMesh(level, n_r, R_IN, R_OUT)
        r = np.linalg.norm(m.node_xyz(), axis=1)
        phi = np.sin(np.pi * (r - R_IN) / d) / r
        K, _ = E.assemble_energy(m)
        errs.append(abs((phi @ (K @ phi)) / (phi @ (E.lumped_mass(m) * phi)) / lam - 1))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 2e-2 and np.all(orders > 1.7), (errs, orders)


def test_advection_of_a_linear_field_by_a_rotation():
    """For T = a . x the one-point gradient is exact and ubar_e = omega x xbar_e exactly, so
    (C T)_j / m_j (Galerkin part) is (omega x xhat_j) . a with xhat_j the volume-weighted mean of the
    centroids of the wedges around node j: it converges to (omega x x_j) . a pointwise at first order
    on the icosahedral lattice (a wrong weight, e.g. a dropped N_j(q_c) = 1/6, does not converge)."""
    om, a = np.array([0.3, -0.7, 0.5]), np.array([1.0, 2.0, -0.5])
    errs = []
    for level, n_r in ((2, 5), (3, 9), (4, 17)):
        m = ShellMesh(level, n_r, R_IN, R_OUT)
        x = m.node_xyz()
        _, C = E.assemble_energy(m, rotation(m, om), supg=False)
        got = (C @ (x @ a)) / E.lumped_mass(m)
        want = np.cross(om[None, :], x) @ a
        inner = ~(m.boundary_nodes()[0] | m.boundary_nodes()[1])
        errs.append(np.abs(got - want)[inner].max() / np.abs(want).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 1e-2 and np.all(orders > 0.9), (errs, orders)


def test_supg_tau_limits():
    V = np.array([0.5, 0.5, 0.5])
    h = np.cbrt(2 * 0.5)
    ub = np.array([[1e-9, 0, 0], [0, 0, 1e4], [0, 3.0, 0]])
    tau = E.supg_tau(V, ub)
    assert abs(tau[0] / (h * h / 12) - 1) < 1e-9                 # diffusion-dominated: h^2 / 12
    assert abs(tau[1] / (h / 2e4) - 1) < 1e-3                    # advection-dominated: h / (2 |u|)
    pe = 3.0 * h / 2
    assert abs(tau[2] - h / 6.0 * (1 / np.tanh(pe) - 1 / pe)) < 1e-15


def test_nusselt_of_a_perturbed_conductive_profile():
    """T = T_c + 0.1 sin(pi (r - r_in) / d): the exact top flux ratio is 1 - 0.1 (pi / d) / T_c'(r_out),
    T_c' = r_in / ((r_in - r_out) r_out) at r_out; the consistent flux converges to it (first order:
    the top layer's volume term), and the conductive profile itself gives 1."""
    d = R_OUT - R_IN
    tc_slope = R_IN / ((R_IN - R_OUT) * R_OUT)
    exact = 1.0 - 0.1 * (np.pi / d) / tc_slope
    errs = []
    for level, n_r in ((2, 5), (3, 9), (4, 17)):
        m = ShellMesh(level, n_r, R_IN, R_OUT)
        r = np.linalg.norm(m.node_xyz(), axis=1)
        Tc = R_IN * (r - R_OUT) / (r * (R_IN - R_OUT))
        T = Tc + 0.1 * np.sin(np.pi * (r - R_IN) / d)
        assert abs(E.nusselt_top(m, Tc, Tc) - 1) < 1e-14
        errs.append(abs(E.nusselt_top(m, T, Tc) - exact))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 0.9), (errs, orders)


def test_heun_step_decays_the_radial_mode_at_the_discrete_rate():
    """Without velocity, the radial eigenmode decays by exp(-lam t) up to the O(h^2) eigenvalue and
    O(dt^2) Heun errors."""
    d = R_OUT - R_IN
    lam = (np.pi / d) ** 2
    m = ShellMesh(3, 17, R_IN, R_OUT)
    r = np.linalg.norm(m.node_xyz(), axis=1)
    phi = np.sin(np.pi * (r - R_IN) / d) / r
    t, n = 0.01, 40
    T = E.heun_steps(m, phi, np.zeros((3, m.n_nodes)), t / n, n)
    w = E.lumped_mass(m)
    ratio = (w * T) @ phi / ((w * phi) @ phi)
    assert abs(ratio / np.exp(-lam * t) - 1) < 0.02, ratio
