"""Oracle Stokes system: the constrained saddle matrix, right-hand side, residual and a direct solve.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

K = [[P A P + (I - P), P B^T], [B P, 0]] (Sec. 7 block form, free-slip / no-slip by nodal
projection), b = (P f, 0) with the Boussinesq buoyancy f.  The relative residual is
||b - K x||_2 / ||b||_2 over the unique DoFs (velocity components, then pressure).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import operators as O
from .fields import buoyancy_rhs
from .multigrid import rotation_basis


class StokesSystem:
    def __init__(self, mesh, eta, bc=(O.FREE, O.FREE), div_term=True, kappa=0.0, quad=1):
        self.mesh, self.bc = mesh, bc
        self.pmesh = O.pressure_mesh(mesh)
        P = O.boundary_projectors(mesh, bc)
        self.P = P
        Pm = O.projector_matrix(P)
        A = O.constrain_A(O.assemble_A(mesh, eta, div_term, kappa, quad), Pm)
        B = O.assemble_B(mesh, O.prolongation(mesh, self.pmesh)) @ Pm
        self.nu, self.np_ = 3 * mesh.n_nodes, self.pmesh.n_nodes
        self.K = sp.bmat([[A, B.T], [B, None]], format="csr")

    def rhs(self, T, Ra):
        f = buoyancy_rhs(self.mesh, T, Ra, self.P)
        return np.concatenate([f.ravel(), np.zeros(self.np_)])

    def residual(self, b, u, p):
        """Relative residual of a solution given as u (3, n) and p (n_p,)."""
        x = np.concatenate([np.asarray(u).ravel(), np.asarray(p).ravel()])
        return np.linalg.norm(b - self.K @ x) / np.linalg.norm(b)

    def direct_solve(self, b):
        """Sparse direct solve; with free-slip on both surfaces the three rigid rotations are a
        null space, removed by bordering the system with the constraint R^T u = 0."""
        K = self.K
        if self.bc == (O.FREE, O.FREE):
            R = rotation_basis(self.mesh)
            C = sp.csr_matrix(np.vstack([R, np.zeros((self.np_, 3))]))
            K = sp.bmat([[K, C], [C.T, None]], format="csc")
            b = np.concatenate([b, np.zeros(3)])
        x = spla.spsolve(K.tocsc(), b)
        return x[: self.nu].reshape(3, -1), x[self.nu: self.nu + self.np_]
