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
