"""Pins of the oracle's TALA pieces (Sec. 1, Eq. stokes and Eq. mass; CPU only).

The reference profiles rho(r), alpha(r) are given at the node layers.  The constraint
div(rho u) = 0 is discretised by the product rule at the quadrature point,
rho(q_c) div u_h(q_c) + rho'(q_c) r_hat . u_h(q_c), and the buoyancy of Eq. (stokes) is
Ra rho alpha T' r_hat with rho, alpha taken at the wedge's quadrature point."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import operators as O
from oracle.fields import buoyancy_rhs
from oracle.mesh import ShellMesh

sympy = pytest.importorskip("sympy")

R_IN, R_OUT = 0.55, 1.0


def rotation_field(m, om):
    return np.cross(om[None, :], m.node_xyz()).T


def test_unit_density_gives_the_boussinesq_divergence_and_rotations_stay_free():
    m = ShellMesh(3, 9, R_IN, R_OUT)
    Pp = O.prolongation(m, O.pressure_mesh(m))
    B = O.assemble_B(m, Pp)
    assert abs(O.assemble_B(m, Pp, rho=np.ones(m.n_r)) - B).max() == 0.0
    rho = np.exp(1.5 * (R_OUT - m.radii))
    Br = O.assemble_B(m, Pp, rho=rho)
    # rigid rotations stay an exact null space of the weighted divergence (div(rho omega x x) = 0)
    u = rotation_field(m, np.array([0.3, -1.2, 0.8]))
    scale = np.abs(Br).max() * np.abs(u).max()
    assert np.abs(Br @ u.ravel()).max() <= 1e-14 * scale
    # a constant density is a scaled B (rho' = 0)
    assert abs(O.assemble_B(m, Pp, rho=np.full(m.n_r, 2.5)) - 2.5 * B).max() <= 1e-15 * np.abs(B).max()
    # the radial field u = r_hat / (rho r^2) has div(rho u) = 0 in the continuum: second-order small
    errs = []
    for level, n_r in ((2, 5), (3, 9)):
        mm = ShellMesh(level, n_r, R_IN, R_OUT)
        rr = np.exp(1.5 * (R_OUT - mm.radii))
        X = mm.node_xyz()
        rn = np.linalg.norm(X, axis=1)
        v = (X / (rn ** 3 * rr[np.arange(mm.n_nodes) % mm.n_r])[:, None]).T
        Bm = O.assemble_B(mm, O.prolongation(mm, O.pressure_mesh(mm)), rho=rr)
        errs.append(np.abs(Bm @ v.ravel()).max() / (np.abs(Bm).max() * np.abs(v).max()))
    assert errs[1] < errs[0] / 3, errs
    # the weighting is not a no-op: on a generic field B_rho differs from B
    w = np.random.default_rng(4).normal(size=3 * m.n_nodes)
    assert np.abs(Br @ w - B @ w).max() > 0.1 * np.abs(B @ w).max()


def test_weighted_buoyancy_magnitude_converges_to_the_shell_integral():
    """With T' = 1: sum_j f_j . x_j = Ra sum_e V_e rho alpha(q_c) |x(q_c)|, the one-point rule for
    Ra times the integral of rho alpha r over the shell; rho = 2 - r, alpha = 1/2 + r."""
    r = sympy.symbols("r")
    exact = float(sympy.integrate(4 * sympy.pi * (2 - r) * (sympy.Rational(1, 2) + r) * r ** 3, (r, R_IN, R_OUT)))
    Ra, errs = 3.0, []
    for level, n_r in ((2, 3), (3, 5), (4, 9)):
        m = ShellMesh(level, n_r, R_IN, R_OUT)
        f = buoyancy_rhs(m, np.ones(m.n_nodes), Ra, rho=2 - m.radii, alpha=0.5 + m.radii)
        errs.append(abs(np.sum(f * m.node_xyz().T) / Ra - exact) / exact)
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 5e-3 and np.all((orders > 1.8) & (orders < 2.2)), (errs, orders)


def _tala_fields(beta, p_scale):
    X, Y, Z = sympy.symbols("x y z", real=True)
    V = (X, Y, Z)
    rr = sympy.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    rho = sympy.exp(beta * (R_OUT - rr))
    phi = sympy.sin(sympy.pi * (rr - R_IN) / (R_OUT - R_IN)) ** 2
    pw = [phi * (Y * Z + X), phi * (X * X - Z), phi * (Z * X + Y * Y)]
    m = [sympy.diff(pw[2], Y) - sympy.diff(pw[1], Z), sympy.diff(pw[0], Z) - sympy.diff(pw[2], X),
         sympy.diff(pw[1], X) - sympy.diff(pw[0], Y)]          # rho u, divergence-free
    u = [c / rho for c in m]
    eta = sympy.exp(rr)
    p = p_scale * (X * Y * Z + X * X - Z)
    div = sum(sympy.diff(u[i], V[i]) for i in range(3))
    tau = [[eta * (sympy.diff(u[i], V[j]) + sympy.diff(u[j], V[i])) - (sympy.Rational(2, 3) * eta * div if i == j else 0)
            for j in range(3)] for i in range(3)]
    f = [-sum(sympy.diff(tau[i][j], V[j]) for j in range(3)) + sympy.diff(p, V[i]) for i in range(3)]
    lam = lambda e: sympy.lambdify(V, e, "numpy")
    rs = sympy.symbols("r", positive=True)
    return lam(u), lam(f), lam(p), lam(eta), sympy.lambdify(rs, sympy.exp(beta * (R_OUT - rs)), "numpy")


def _tala_errors(level, n_r, fu, ff, fp, feta, frho):
    m = ShellMesh(level, n_r, R_IN, R_OUT)
    pm = O.pressure_mesh(m)
    xyz = m.node_xyz()
    nodes = m.wedge_nodes()
    eta = feta(*xyz[nodes.ravel()].reshape(-1, 6, 3).mean(axis=1).T)
    P = O.boundary_projectors(m, (O.NOSLIP, O.NOSLIP))
    Pm = O.projector_matrix(P)
    Pp = O.prolongation(m, pm)
    A = O.constrain_A(O.assemble_A(m, eta), Pm)
    BT = (O.assemble_B(m, Pp) @ Pm).T
    Br = O.assemble_B(m, Pp, rho=frho(m.radii)) @ Pm
    _, Vw = O.wedge_geometry(m)
    mass = np.bincount(nodes.ravel(), weights=np.repeat(Vw / 6.0, 6), minlength=m.n_nodes)
    full = lambda vals, n: np.array([np.broadcast_to(c, (n,)) for c in vals])
    F = O.project(P, full(ff(*xyz.T), m.n_nodes) * mass)
    ones = sp.csr_matrix(np.ones((1, pm.n_nodes)))
    K = sp.bmat([[A, BT, None], [Br, None, ones.T], [None, ones, None]], format="csc")
    x = spla.spsolve(K, np.concatenate([F.ravel(), np.zeros(pm.n_nodes + 1)]))
    nu = 3 * m.n_nodes
    uh, ph = x[:nu].reshape(3, -1), x[nu:nu + pm.n_nodes]
    ue = full(fu(*xyz.T), m.n_nodes)
    _, Vp = O.wedge_geometry(pm)
    pmass = np.bincount(pm.wedge_nodes().ravel(), weights=np.repeat(Vp / 6.0, 6), minlength=pm.n_nodes)
    pe = fp(*pm.node_xyz().T)
    pe, ph = pe - pmass @ pe / pmass.sum(), ph - pmass @ ph / pmass.sum()
    return (np.sqrt(np.sum(mass * (uh - ue) ** 2) / np.sum(mass * ue ** 2)),
            np.sqrt(np.sum(pmass * (ph - pe) ** 2) / np.sum(pmass * pe ** 2)))


def test_tala_manufactured_solution_orders():
    """div(rho u) = 0 with rho = exp(1.5 (r_out - r)) (density rising with depth, div u != 0, so
    the -2/3 div term of Eq. stress is active), no-slip, eta = exp(r): velocity order >= 1.8 and
    pressure order >= 1.4 from level 2 / 5 layers to level 3 / 9 layers, as for the Boussinesq
    system; dropping the density weighting in B stops the velocity from converging to this u."""
    fu, ff, fp, feta, frho = _tala_fields(1.5, 100.0)
    eu2, ep2 = _tala_errors(2, 5, fu, ff, fp, feta, frho)
    eu3, ep3 = _tala_errors(3, 9, fu, ff, fp, feta, frho)
    ou, op = np.log2(eu2 / eu3), np.log2(ep2 / ep3)
    print(f"TALA velocity {eu2:.3e} -> {eu3:.3e} (order {ou:.2f}); pressure {ep2:.3e} -> {ep3:.3e} (order {op:.2f})")
    assert eu3 < 0.08 and ep3 < 0.2, (eu3, ep3)  # without the weighting: 0.108 at level 3
    assert 1.8 <= ou <= 2.6 and 1.4 <= op <= 2.8, (ou, op)
