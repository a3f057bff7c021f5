"""Oracle Stokes system: the constrained saddle matrix, right-hand side, residual and two solves.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

K = [[P A P + (I - P), P B^T], [B P, 0]] (Sec. 7 block form, free-slip / no-slip by nodal
projection), b = (P f, 0) with the Boussinesq buoyancy f.  The relative residual is
||b - K x||_2 / ||b||_2 over the unique DoFs (velocity components, then pressure).

Solves: a sparse direct solve (small meshes), and flexible GMRES (Saad 1993) without restarts,
right-preconditioned by the block upper-triangular preconditioner of Sec. 7 (Eq. block-precond)
with one oracle V-cycle for A^-1 and -diag(M_1/eta)^-1 (Eq. pmass) for the Schur complement, for
meshes the direct solve cannot factor in reasonable time.  Either way the returned solution is
only trusted through ``residual``, evaluated with the assembled K.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import operators as O
from .fields import buoyancy_rhs
from .multigrid import Hierarchy, rotation_basis


class StokesSystem:
    """With reference profiles rho, alpha (one value per node layer) the system is the TALA one of
    Sec. 1: the momentum block and its pressure gradient P B^T are unchanged, the constraint is
    Eq. (mass) with the density-weighted B_rho of ``oracle.operators.assemble_B``, so K is no
    longer symmetric, and the load is Ra rho alpha T' r_hat."""

    def __init__(self, mesh, eta, bc=(O.FREE, O.FREE), div_term=True, kappa=0.0, quad=1, rho=None, alpha=None):
        self.mesh, self.bc = mesh, bc
        self.rho, self.alpha = rho, alpha
        self.pmesh = O.pressure_mesh(mesh)
        P = O.boundary_projectors(mesh, bc)
        self.P = P
        Pm = O.projector_matrix(P)
        A = O.constrain_A(O.assemble_A(mesh, eta, div_term, kappa, quad), Pm)
        Pp = O.prolongation(mesh, self.pmesh)
        BT = (O.assemble_B(mesh, Pp) @ Pm).T
        B = O.assemble_B(mesh, Pp, rho=rho) @ Pm
        self.nu, self.np_ = 3 * mesh.n_nodes, self.pmesh.n_nodes
        self.K = sp.bmat([[A, BT], [B, None]], format="csr")

    def rhs(self, T, Ra):
        f = buoyancy_rhs(self.mesh, T, Ra, self.P, rho=self.rho, alpha=self.alpha)
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

    def fgmres_solve(self, b, eta, tol=1e-11, max_iters=600, seed=4):
        """Flexible GMRES from x = 0 with z = P^-1 v: z_p = -v_p / diag(M_1/eta),
        z_u = V(v_u - P B^T z_p) (V one V-cycle of ``oracle.multigrid.Hierarchy`` on this mesh's
        viscosity and boundary conditions); with free-slip on both surfaces the rigid rotations are
        removed from z_u (an exact null space of K).  Arnoldi with modified Gram-Schmidt; stops when
        the least-squares residual falls below tol ||b||.  Returns (u, p, iterations); the returned
        u has no rigid-rotation component when that null space exists."""
        m = self.mesh
        H = Hierarchy(m.level, m.n_r, m.r_in, m.r_out, eta, bc=self.bc)
        H.setup(np.random.default_rng(seed).normal(size=self.nu))
        mdiag = O.diag_pressure_mass(m, O.prolongation(m, self.pmesh), eta)
        PBt = self.K[: self.nu, self.nu:]
        Q = np.linalg.qr(rotation_basis(m))[0] if self.bc == (O.FREE, O.FREE) else None

        def prec(v):
            zp = -v[self.nu:] / mdiag
            zu = H.vcycle(v[: self.nu] - PBt @ zp)
            if Q is not None:
                zu = zu - Q @ (Q.T @ zu)
            return np.concatenate([zu, zp])

        beta = np.linalg.norm(b)
        V = [b / beta]
        Z, Hm = [], np.zeros((max_iters + 1, max_iters))
        for j in range(max_iters):
            Z.append(prec(V[j]))
            w = self.K @ Z[j]
            for i in range(j + 1):
                Hm[i, j] = V[i] @ w
                w = w - Hm[i, j] * V[i]
            Hm[j + 1, j] = np.linalg.norm(w)
            V.append(w / Hm[j + 1, j])
            e1 = np.zeros(j + 2)
            e1[0] = beta
            y, *_ = np.linalg.lstsq(Hm[: j + 2, : j + 1], e1, rcond=None)
            if np.linalg.norm(e1 - Hm[: j + 2, : j + 1] @ y) <= tol * beta:
                break
        x = np.stack(Z, axis=1) @ y
        u = x[: self.nu]
        if Q is not None:
            u = u - Q @ (Q.T @ u)
        return u.reshape(3, -1), x[self.nu:], j + 1

    def lumped_mass(self):
        """Nodal quadrature weights sum_e V_e / 6 (one-point rule, N_j(q_c) = 1/6)."""
        _, V = O.wedge_geometry(self.mesh)
        return np.bincount(self.mesh.wedge_nodes().ravel(), weights=np.repeat(V / 6.0, 6),
                           minlength=self.mesh.n_nodes)

    def v_rms(self, u):
        """Root-mean-square velocity sqrt(int |u|^2 dV / V) with the lumped nodal quadrature."""
        w = self.lumped_mass()
        return float(np.sqrt(np.sum(w * np.sum(np.asarray(u) ** 2, axis=0)) / w.sum()))
