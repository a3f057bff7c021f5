"""Manufactured-solution convergence of the oracle's viscous block (CPU only).

u = sin(pi (r - r_in) / (r_out - r_in)) v(x) vanishes on both surfaces (no-slip); with eta = 1
the strong operator of Eq. (stokes) with the -2/3 div term is -div(2 eps(u) - 2/3 div u I) =
-(Lap u + 1/3 grad div u), computed symbolically.  The load is lumped (f at the nodes times
sum_e V_e / 6), and the discrete L2 error at the nodes must fall with second order under uniform
refinement (lateral and radial), for the plain one-point rule, with hourglass control, whose
error the paper reports unchanged (Sec. 4, Fig. 2 right), and with a second radial quadrature
point."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import operators as O
from oracle.mesh import ShellMesh

sympy = pytest.importorskip("sympy")

R_IN, R_OUT = 0.55, 1.0


def _fields():
    X, Y, Z = sympy.symbols("x y z", real=True)
    r = sympy.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    phi = sympy.sin(sympy.pi * (r - R_IN) / (R_OUT - R_IN))
    u = [phi * (Y + Z * Z), phi * (X * Z - Y), phi * (X * Y + 1)]
    div = sum(sympy.diff(u[i], v) for i, v in enumerate((X, Y, Z)))
    f = [-sum(sympy.diff(u[i], v, 2) for v in (X, Y, Z)) - sympy.diff(div, w) / 3 for i, w in enumerate((X, Y, Z))]
    return sympy.lambdify((X, Y, Z), u, "numpy"), sympy.lambdify((X, Y, Z), f, "numpy")


def _error(level, n_r, kappa, fu, ff, quad=1):
    m = ShellMesh(level, n_r, R_IN, R_OUT)
    xyz = m.node_xyz()
    P = O.boundary_projectors(m, (O.NOSLIP, O.NOSLIP))
    K = O.constrain_A(O.assemble_A(m, np.ones(m.n_wedges), True, kappa, quad), O.projector_matrix(P))
    _, V = O.wedge_geometry(m)
    mass = np.bincount(m.wedge_nodes().ravel(), weights=np.repeat(V / 6.0, 6), minlength=m.n_nodes)
    F = O.project(P, np.array([np.broadcast_to(c, (m.n_nodes,)) for c in ff(*xyz.T)]) * mass)
    uh = spla.spsolve(K.tocsc(), F.ravel()).reshape(3, -1)
    ue = np.array([np.broadcast_to(c, (m.n_nodes,)) for c in fu(*xyz.T)])
    return np.sqrt(np.sum(mass * (uh - ue) ** 2) / np.sum(mass * ue ** 2))


@pytest.mark.parametrize("kappa,quad", [(0.0, 1), (0.1, 1), (0.0, 2)])
def test_second_order_convergence(kappa, quad):
    fu, ff = _fields()
    e2 = _error(2, 5, kappa, fu, ff, quad)
    e3 = _error(3, 9, kappa, fu, ff, quad)
    order = np.log2(e2 / e3)
    print(f"kappa {kappa}, radial points {quad}: errors {e2:.3e} {e3:.3e}, order {order:.2f}")
    assert 1.8 <= order <= 2.4, order


def _stokes_fields(p_scale):
    """A divergence-free velocity u = curl(phi(r) w(x)) with phi = sin^2(pi (r - r_in)/(r_out - r_in)),
    so u and its radial derivative vanish on both surfaces (no-slip), a viscosity eta = exp(r) and a
    pressure p = p_scale (x y z + x^2 - z).  The load is the strong form of Eq. (stokes),
    f = -div(eta (grad u + grad u^T)) + grad p (div u = 0, so the -2/3 div term drops out)."""
    X, Y, Z = sympy.symbols("x y z", real=True)
    V = (X, Y, Z)
    r = sympy.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    phi = sympy.sin(sympy.pi * (r - R_IN) / (R_OUT - R_IN)) ** 2
    pw = [phi * (Y * Z + X), phi * (X * X - Z), phi * (Z * X + Y * Y)]
    u = [sympy.diff(pw[2], Y) - sympy.diff(pw[1], Z), sympy.diff(pw[0], Z) - sympy.diff(pw[2], X),
         sympy.diff(pw[1], X) - sympy.diff(pw[0], Y)]
    eta = sympy.exp(r)
    p = p_scale * (X * Y * Z + X * X - Z)
    grad = [[sympy.diff(u[i], V[j]) for j in range(3)] for i in range(3)]
    f = [-sum(sympy.diff(eta * (grad[i][j] + grad[j][i]), V[j]) for j in range(3)) + sympy.diff(p, V[i])
         for i in range(3)]
    lam = lambda e: sympy.lambdify(V, e, "numpy")
    return lam(u), lam(f), lam(p), lam(eta)


def _stokes_errors(level, n_r, fu, ff, fp, feta):
    """Relative discrete L2 errors of velocity (fine nodes) and pressure (coarse nodes, mean removed)
    of the no-slip saddle system [[P A P + I - P, P B^T], [B P, 0]] with the lumped load, bordered by
    the constant-pressure constraint (an exact null vector under no-slip)."""
    import scipy.sparse as sp
    m = ShellMesh(level, n_r, R_IN, R_OUT)
    pm = O.pressure_mesh(m)
    xyz = m.node_xyz()
    nodes = m.wedge_nodes()
    eta = feta(*xyz[nodes.ravel()].reshape(-1, 6, 3).mean(axis=1).T)
    P = O.boundary_projectors(m, (O.NOSLIP, O.NOSLIP))
    Pm = O.projector_matrix(P)
    A = O.constrain_A(O.assemble_A(m, eta), Pm)
    B = O.assemble_B(m, O.prolongation(m, pm)) @ Pm
    _, V = O.wedge_geometry(m)
    mass = np.bincount(nodes.ravel(), weights=np.repeat(V / 6.0, 6), minlength=m.n_nodes)
    full = lambda vals, n: np.array([np.broadcast_to(c, (n,)) for c in vals])
    F = O.project(P, full(ff(*xyz.T), m.n_nodes) * mass)
    ones = sp.csr_matrix(np.ones((1, pm.n_nodes)))
    K = sp.bmat([[A, B.T, None], [B, None, ones.T], [None, ones, None]], format="csc")
    x = spla.spsolve(K, np.concatenate([F.ravel(), np.zeros(pm.n_nodes + 1)]))
    nu = 3 * m.n_nodes
    uh, ph = x[:nu].reshape(3, -1), x[nu:nu + pm.n_nodes]
    ue = full(fu(*xyz.T), m.n_nodes)
    _, Vp = O.wedge_geometry(pm)
    pmass = np.bincount(pm.wedge_nodes().ravel(), weights=np.repeat(Vp / 6.0, 6), minlength=pm.n_nodes)
    pe = fp(*pm.node_xyz().T)
    pe, ph = pe - pmass @ pe / pmass.sum(), ph - pmass @ ph / pmass.sum()
    eu = np.sqrt(np.sum(mass * (uh - ue) ** 2) / np.sum(mass * ue ** 2))
    ep = np.sqrt(np.sum(pmass * (ph - pe) ** 2) / np.sum(pmass * pe ** 2))
    return eu, ep


def test_stokes_manufactured_solution_orders():
    """Coupled Stokes convergence (Sec. 3 pairs W1-iso-W2 velocity with W1 pressure one level coarser;
    Sec. 4 / Fig. 2 claim optimal order for the one-point rule): from level 2 / 5 layers to level 3 /
    9 layers the velocity error must fall with order >= 1.8 and the pressure error with order >= 1.4.
    The pressure scale (100) balances grad p against the viscous force, so neither part of the load
    dominates; a wrong sign or scale of B or B^T, or a wrong pressure basis, stops the pressure from
    converging."""
    fu, ff, fp, feta = _stokes_fields(100.0)
    eu2, ep2 = _stokes_errors(2, 5, fu, ff, fp, feta)
    eu3, ep3 = _stokes_errors(3, 9, fu, ff, fp, feta)
    ou, op = np.log2(eu2 / eu3), np.log2(ep2 / ep3)
    print(f"velocity {eu2:.3e} -> {eu3:.3e} (order {ou:.2f}); pressure {ep2:.3e} -> {ep3:.3e} (order {op:.2f})")
    assert eu3 < 0.1 and ep3 < 0.2, (eu3, ep3)
    assert 1.8 <= ou <= 2.6, ou
    assert 1.4 <= op <= 2.8, op
