"""Pins of the oracle's global operators (CPU only).

Invariants fixed by the paper's definitions: symmetric bilinear form (Eq. elemmat),
zero strain of rigid motions (Eq. stress), div of rigid rotations and constants is
zero, the discrete consistency of constant stress at interior nodes, and the
block structure [[A, B^T], [B, 0]] (Sec. 7)."""
import numpy as np
import pytest

from oracle.fields import buoyancy_rhs, coarsen_viscosity, viscosity, wedge_temperature
from oracle.mesh import ShellMesh
from oracle.operators import (FREE, NOSLIP, apply_A, apply_A_constrained, assemble_A, assemble_B,
                              boundary_projectors, constrain_A, diag_A_constrained, diag_pressure_mass,
                              pressure_mesh, project, projector_matrix, prolongation, psi_at_centroids,
                              wedge_geometry)


@pytest.fixture(scope="module")
def small():
    m = ShellMesh(2, 5, 0.55, 1.0)
    rng = np.random.default_rng(11)
    eta = np.exp(rng.normal(size=m.n_wedges))
    pm = pressure_mesh(m)
    Pp = prolongation(m, pm)
    return m, eta, pm, Pp, rng


def rotation_field(m, om):
    X = m.node_xyz()
    return np.cross(om[None, :], X).T


def test_A_symmetric_and_matrix_free_equals_assembled(small):
    m, eta, _, _, rng = small
    A = assemble_A(m, eta)
    u, v = rng.normal(size=(2, 3, m.n_nodes))
    Au = A @ u.ravel()
    assert abs(v.ravel() @ Au - u.ravel() @ (A @ v.ravel())) <= 1e-14 * abs(u.ravel() @ Au)
    np.testing.assert_allclose(apply_A(m, eta, u).ravel(), Au, atol=1e-14 * np.abs(Au).max())
    # positive semi-definite
    assert u.ravel() @ Au > 0


def test_A_kills_rigid_motions(small):
    m, eta, _, _, rng = small
    u = rng.normal(size=(3, m.n_nodes))
    ref = np.abs(apply_A(m, eta, u)).max()
    for om in np.eye(3):
        assert np.abs(apply_A(m, eta, rotation_field(m, om))).max() <= 1e-14 * ref
    t = np.zeros((3, m.n_nodes)); t[1] = 1.0
    assert np.abs(apply_A(m, eta, t)).max() <= 1e-14 * ref
    # rotations are tangential at the boundary, so the free-slip operator kills them too
    P = boundary_projectors(m, (FREE, FREE))
    rot = rotation_field(m, np.array([0.3, -1.0, 0.7]))
    assert np.abs(apply_A_constrained(m, eta, rot, P)).max() <= 1e-14 * ref


def test_A_constant_stress_balances_at_interior_nodes(small):
    """For constant eta and an affine field u = G x the stress is constant, and with
    uniform radial spacing the element contributions cancel at every interior node."""
    m, _, _, _, rng = small
    G = rng.normal(size=(3, 3))
    u = G @ m.node_xyz().T
    y = apply_A(m, np.ones(m.n_wedges), u)
    inner, outer = m.boundary_nodes()
    assert np.abs(y[:, ~(inner | outer)]).max() <= 1e-13 * np.abs(y).max()
    assert np.abs(y[:, inner | outer]).max() > 1e-3 * np.abs(y).max()


def test_B_properties(small):
    m, _, pm, Pp, rng = small
    B = assemble_B(m, Pp)
    scale = np.abs(B).max()
    for om in np.eye(3):
        assert np.abs(B @ rotation_field(m, om).ravel()).max() <= 1e-14 * scale
    assert np.abs(B @ np.ones(3 * m.n_nodes)).max() <= 1e-14 * scale
    # B^T 1 = 0 at interior nodes (telescoping with uniform radial spacing), not at the boundary
    BT1 = (B.T @ np.ones(pm.n_nodes)).reshape(3, -1)
    inner, outer = m.boundary_nodes()
    assert np.abs(BT1[:, ~(inner | outer)]).max() <= 1e-14 * scale
    assert np.abs(BT1[:, inner | outer]).max() > 1e-3 * scale
    # B of an affine field equals -trace(G) times the pressure-space integral of psi_k
    G = rng.normal(size=(3, 3))
    u = G @ m.node_xyz().T
    _, V = wedge_geometry(m)
    Psi = psi_at_centroids(m, Pp)
    np.testing.assert_allclose(B @ u.ravel(), -np.trace(G) * (Psi.T @ V), atol=1e-13 * scale)


def test_B_iso_structure(small):
    """B = P^T B_fine with B_fine the fine-level W1/W1 divergence (psi_n(q_c) = 1/6)."""
    m, _, pm, Pp, _ = small
    B = assemble_B(m, Pp)
    import scipy.sparse as sp
    Bf = assemble_B(m, sp.identity(m.n_nodes, format="csr"))
    assert abs(B - (Pp.T @ Bf)).max() <= 1e-15 * abs(B).max()


def test_diag_matches_assembled(small):
    m, eta, _, _, _ = small
    for bc in ((FREE, FREE), (NOSLIP, FREE)):
        P = boundary_projectors(m, bc)
        K = constrain_A(assemble_A(m, eta), projector_matrix(P))
        d = diag_A_constrained(m, eta, P)
        np.testing.assert_allclose(d.ravel(), K.diagonal(), rtol=1e-13)


def test_constrained_matrix_free_equals_assembled(small):
    m, eta, _, _, rng = small
    for bc in ((FREE, FREE), (NOSLIP, FREE), (NOSLIP, NOSLIP)):
        P = boundary_projectors(m, bc)
        K = constrain_A(assemble_A(m, eta), projector_matrix(P))
        u = rng.normal(size=(3, m.n_nodes))
        y = apply_A_constrained(m, eta, u, P)
        np.testing.assert_allclose(y.ravel(), K @ u.ravel(), atol=1e-14 * np.abs(y).max())
        # K is symmetric
        assert abs(K - K.T).max() <= 1e-15 * abs(K).max()


def test_pressure_mass_diag(small):
    """One-point diag(M_{1/eta}); for eta = 1 its sum equals sum_e V_e (psi sums to 1) weighted by psi."""
    m, eta, pm, Pp, _ = small
    d = diag_pressure_mass(m, Pp, eta)
    assert d.shape == (pm.n_nodes,) and d.min() > 0
    _, V = wedge_geometry(m)
    Psi = psi_at_centroids(m, Pp)
    np.testing.assert_allclose(np.asarray(Psi.sum(axis=1)).ravel(), 1.0, atol=1e-15)
    # brute force over wedges for a few pressure nodes
    dense = Psi.toarray()
    for k in (0, 7, pm.n_nodes - 1):
        assert abs(d[k] - sum(V[e] / eta[e] * dense[e, k] ** 2 for e in range(m.n_wedges))) <= 1e-14 * d[k]


def test_buoyancy_rhs_orthogonal_to_rotations(small):
    m, _, _, _, rng = small
    T = rng.random(m.n_nodes)
    P = boundary_projectors(m, (FREE, FREE))
    f = buoyancy_rhs(m, T, 7e3, P)
    for om in np.eye(3):
        assert abs(np.sum(f * rotation_field(m, om))) <= 1e-13 * np.abs(f).sum()
    # with T = 1 the net force vanishes up to the mesh's central symmetry
    f1 = buoyancy_rhs(m, np.ones(m.n_nodes), 1.0)
    assert np.abs(f1.sum(axis=1)).max() <= 1e-12 * np.abs(f1).sum()


def test_viscosity_law_and_coarsening():
    f = ShellMesh(3, 9, 0.55, 1.0)
    c = ShellMesh(2, 5, 0.55, 1.0)
    rng = np.random.default_rng(2)
    T = rng.random(f.n_nodes)
    eta = viscosity(f, T, np.log(1e3), jump_r=0.9, jump_factor=30.0)
    Te = wedge_temperature(f, T)
    rmid = 0.5 * (f.radii[np.arange(f.n_wedges) % 8] + f.radii[np.arange(f.n_wedges) % 8 + 1])
    np.testing.assert_allclose(eta, np.where(rmid < 0.9, 30.0, 1.0) * np.exp(np.log(1e3) * (0.5 - Te)), rtol=1e-15)
    np.testing.assert_allclose(coarsen_viscosity(f, c, np.full(f.n_wedges, 2.5)), 2.5, rtol=1e-15)
    # each coarse wedge's children lie inside it: child centroids average to the parent centroid
    # (the 4 lateral children tile the parent triangle; their lattice centroids average to the parent's)
    xf = f.node_xyz(f.wedge_nodes().ravel()).reshape(-1, 6, 3).mean(axis=1)
    xc = c.node_xyz(c.wedge_nodes().ravel()).reshape(-1, 6, 3).mean(axis=1)
    for ax in range(3):
        got = coarsen_viscosity(f, c, xf[:, ax])
        assert np.abs(got - xc[:, ax]).max() < 0.05
    # and picking the wrong children would move the average by about a cell width
    wrong = coarsen_viscosity(f, c, np.roll(xf[:, 0], 2))
    assert np.abs(wrong - xc[:, 0]).max() > 0.05


def test_buoyancy_rhs_magnitude_converges_to_the_shell_integral():
    """Scale of the Boussinesq load of Eq. (stokes), f_j = sum_e V_e Ra T(q_c) r_hat(q_c) N_j(q_c).

    With T = 1 and no projection, sum_j f_j . x_j = Ra sum_e V_e r_hat_e . (sum_j N_j(q_c) x_j)
    = Ra sum_e V_e |x(q_c)|, the one-point rule for Ra times the integral of r over the shell,
    Ra pi (r_out^4 - r_in^4).  The mesh and the rule are both second order, so the relative error
    must fall by ~4 per refinement; a dropped 1/6 (N_j(q_c)), a dropped V_e or a doubled Ra
    changes the limit itself."""
    r_in, r_out, Ra = 0.55, 1.0, 2.5
    exact = Ra * np.pi * (r_out ** 4 - r_in ** 4)
    errs = []
    for level, n_r in ((2, 3), (3, 5), (4, 9)):
        m = ShellMesh(level, n_r, r_in, r_out)
        f = buoyancy_rhs(m, np.ones(m.n_nodes), Ra)
        errs.append(abs(np.sum(f * m.node_xyz().T) - exact) / exact)
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 5e-3, errs
    assert np.all((orders > 1.9) & (orders < 2.1)), orders
