"""Pins of the oracle's multigrid and Stokes-system code (CPU only)."""
import numpy as np
import pytest

from oracle import operators as O
from oracle.mesh import ShellMesh
from oracle.multigrid import Hierarchy, rotation_basis
from oracle.solver import StokesSystem
from paper_2609_21633_gb300 import inputs


@pytest.fixture(scope="module")
def hier():
    m = ShellMesh(3, 9, 0.55, 1.0)
    eta = inputs.lognormal_viscosity(m.n_wedges, 3, 0.5)
    H = Hierarchy(3, 9, 0.55, 1.0, eta, bc=(O.NOSLIP, O.FREE))
    H.setup(inputs.normal(3 * m.n_nodes, 4))
    return H


def test_chebyshev_step_is_the_scaled_chebyshev_polynomial(hier):
    """One step from x = 0 leaves the error e = T_2((theta - D^-1 K)/delta) / T_2(theta/delta) K^-1 b
    (two Chebyshev-acceleration iterations = the degree-2 Chebyshev polynomial)."""
    h = hier.nlev - 1
    K = hier.K[h].toarray()
    Dinv = hier.Dinv[h].toarray()
    lam = np.max(np.abs(np.linalg.eigvals(Dinv @ K)))
    hier.lam[h] = lam
    b = inputs.normal(K.shape[0], 5)
    x = hier.chebyshev(h, np.zeros_like(b), b, True)
    a, bb = hier.lo * lam, hier.hi * lam
    theta, delta = (a + bb) / 2, (bb - a) / 2
    Z = (theta * np.eye(K.shape[0]) - Dinv @ K) / delta
    T2 = 2 * Z @ Z - np.eye(K.shape[0])
    E = T2 / (2 * (theta / delta) ** 2 - 1)
    xs = np.linalg.solve(K, b)
    np.testing.assert_allclose(x, xs - E @ xs, atol=1e-10 * np.abs(xs).max())


def test_power_iteration_estimates_the_largest_eigenvalue(hier):
    for h in range(hier.nlev - 1):
        ev = np.linalg.eigvals(hier.Dinv[h].toarray() @ hier.K[h].toarray()) if hier.K[h].shape[0] < 6000 else None
        if ev is None:
            continue
        lmax = np.max(np.abs(ev))
        assert 0.8 * lmax <= hier.lam[h] <= lmax * (1 + 1e-12)


def test_coarse_cg_solves_the_coarsest_system(hier):
    h = hier.nlev - 1
    save = hier.coarse_rtol, hier.coarse_max_iters
    hier.coarse_rtol, hier.coarse_max_iters = 1e-14, 2000
    b = inputs.normal(hier.K[h].shape[0], 6)
    x = hier.coarse_cg(b)
    hier.coarse_rtol, hier.coarse_max_iters = save
    np.testing.assert_allclose(hier.K[h] @ x, b, atol=1e-9 * np.abs(b).max())


def test_vcycle_is_a_convergent_iteration(hier):
    """Stand-alone V-cycle iteration converges.  With the one-point rule its rate is slow
    (point Jacobi: about 0.8 here, also with an exact coarse solve and eta = 1): the hourglass
    modes of Sec. 4 degrade stand-alone multigrid, as Fig. 2 (left) reports."""
    K = hier.K[0]
    b = inputs.normal(K.shape[0], 7)
    x = np.zeros_like(b)
    norms = [np.linalg.norm(b)]
    for _ in range(8):
        x = x + hier.vcycle(b - K @ x)
        norms.append(np.linalg.norm(b - K @ x))
    rates = np.array(norms[1:]) / np.array(norms[:-1])
    assert np.all(rates < 0.9), rates


def test_hourglass_control_restores_vcycle_contraction():
    """Eq. (hgstab): with hourglass control, and with a second radial quadrature point, the
    stand-alone V-cycle contracts far faster than with the plain one-point rule (Fig. 2, left),
    on the same shell and viscosity."""
    m = ShellMesh(3, 9, 0.55, 1.0)
    eta = inputs.lognormal_viscosity(m.n_wedges, 3, 0.0)
    rates = {}
    for kappa, quad in ((0.0, 1), (0.1, 1), (0.0, 2)):
        H = Hierarchy(3, 9, 0.55, 1.0, eta, bc=(O.NOSLIP, O.FREE), coarse_rtol=1e-12, coarse_max_iters=1000,
                      kappa=kappa, quad=quad)
        H.setup(inputs.normal(3 * m.n_nodes, 4))
        K = H.K[0]
        b = inputs.normal(K.shape[0], 7)
        x = np.zeros_like(b)
        norms = [np.linalg.norm(b)]
        for _ in range(8):
            x = x + H.vcycle(b - K @ x)
            norms.append(np.linalg.norm(b - K @ x))
        rates[(kappa, quad)] = norms[-1] / norms[-2]
    assert rates[(0.0, 1)] > 0.6 and rates[(0.1, 1)] < 0.45 and rates[(0.0, 2)] < 0.45, rates


def test_direct_solve_and_invariants():
    m = ShellMesh(2, 5, 0.55, 1.0)
    T = inputs.temperature(m.node_xyz(), 0.55, 1.0)
    from oracle.fields import viscosity
    eta = viscosity(m, T, np.log(10.0))
    S = StokesSystem(m, eta)
    b = S.rhs(T, 7e3)
    u, p = S.direct_solve(b)
    assert S.residual(b, u, p) < 1e-10
    # zero net rotation (the bordered constraint) and a nonzero flow
    R = rotation_basis(m)
    assert np.abs(R.T @ u.ravel()).max() < 1e-10 * np.abs(u).max() * np.sqrt(m.n_nodes)
    assert np.abs(u).max() > 1e-3
    # free-slip: zero normal velocity at the boundary nodes
    inner, outer = m.boundary_nodes()
    s = m.lat_xyz[np.arange(m.n_nodes) // m.n_r]
    un = np.einsum("cn,nc->n", u, s)
    assert np.abs(un[inner | outer]).max() < 1e-10 * np.abs(u).max()
