"""Oracle geometric multigrid: the V-cycle of Sec. 7 on explicitly assembled level operators.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Algorithm (the paper gives the structure: two pre- and two post-smoothing steps of a
degree-2 Chebyshev smoother per level, conjugate gradients on the coarsest level; the
remaining choices are readings):
* level operators K_h = P_h A_h P_h + (I - P_h), re-discretised with the coarse viscosity
  (mean of the 8 children) and, with kappa > 0 or quad = 2, the same hourglass control or
  radial quadrature on every level; D_h = the 3x3 node-block diagonal of K_h (block Jacobi; reading:
  the paper does not say which diagonal its Chebyshev smoother uses);
* level shapes: each coarser level halves the lateral and / or radial resolution according
  to the cells' radial / lateral size ratio q (semi-coarsening where the cells are
  anisotropic; see ``mg_shapes``, a reading: the paper states no coarsening rule);
* transfers: prolongation P_h T_h (nested iso-interpolation in the coarsened directions,
  identity in a direction that is not coarsened, then the fine boundary projector),
  restriction P_{h+1} T_h^T;
* Chebyshev acceleration (Saad, Iterative Methods for Sparse Linear Systems, Alg. 12.1) with
  D^-1 preconditioning, two iterations per smoothing step, on [lo, hi] x lambda_h;
  lambda_h from power iterations on D^-1 K_h started from the restricted start vector;
* coarsest level: D-preconditioned CG from zero, stopping when
  (r, D^-1 r) <= rtol^2 (r0, D^-1 r0) or after max_iters; with free-slip on both surfaces
  the rigid rotations are projected out of its right-hand side and solution.
Vectors are component-major flat arrays (3 n_nodes).
"""
import numpy as np
import scipy.sparse as sp

from . import operators as O
from .fields import coarsen_viscosity
from .mesh import ShellMesh


def mg_shapes(level, n_r, r_in, r_out):
    """(lateral level, node layers) of every multigrid level.  q = radial / lateral cell size
    = (r_out - r_in) 2^l / (atan(2) r_mid (n_r - 1)); q >= 2: coarsen laterally only,
    q <= 1/2: radially only, otherwise both (or the one still possible); stop when the
    preferred direction cannot coarsen (lateral needs l >= 2, radial an even cell count)."""
    out = [(level, n_r)]
    edge = 1.1071487177940904
    while True:
        l, nr = out[-1]
        R = nr - 1
        can_lat, can_rad = l >= 2, R % 2 == 0 and R >= 2
        q = (r_out - r_in) * float(1 << l) / (edge * (0.5 * (r_in + r_out)) * float(R))
        if q >= 2.0:
            if not can_lat:
                break
            nxt = (l - 1, nr)
        elif q <= 0.5:
            if not can_rad:
                break
            nxt = (l, R // 2 + 1)
        elif can_lat and can_rad:
            nxt = (l - 1, R // 2 + 1)
        elif can_lat:
            nxt = (l - 1, nr)
        elif can_rad:
            nxt = (l, R // 2 + 1)
        else:
            break
        out.append(nxt)
    return out


def vec_prolongation(fine, coarse):
    """Nested interpolation for 3-component fields in component-major numbering; identity in a
    direction the pair does not coarsen."""
    if fine.N == coarse.N:
        Pl = sp.identity(fine.n_lat, format="csr")
    else:
        Pl = O.lateral_prolongation(fine, coarse)
    if fine.n_r == coarse.n_r:
        Pr = sp.identity(fine.n_r, format="csr")
    else:
        Pr = O.radial_prolongation(fine.n_r, coarse.n_r)
    T = sp.kron(Pl, Pr, format="csr")
    return sp.block_diag([T, T, T], format="csr")


def coarsen_viscosity_semi(fine, coarse, eta_fine):
    """Mean of the child wedges: 8 for full coarsening, 4 (lateral only) or 2 (radial only)."""
    if fine.N != coarse.N and fine.n_r != coarse.n_r:
        return coarsen_viscosity(fine, coarse, eta_fine)
    lab = coarse.wedge_labels()
    d, I, J, w, K = lab.T
    Nf, nkf = fine.N, fine.n_r - 1

    def fid(d, i, j, ww, k):
        return (((d * Nf + i) * Nf + j) * 2 + ww) * nkf + k

    if fine.N == coarse.N:  # radial only: the two layers 2K, 2K+1
        return 0.5 * (eta_fine[fid(d, I, J, w, 2 * K)] + eta_fine[fid(d, I, J, w, 2 * K + 1)])
    kids0 = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    kids1 = [(1, 1, 1), (0, 1, 1), (1, 0, 1), (1, 1, 0)]
    acc = np.zeros(coarse.n_wedges)
    for (a0, b0, w0), (a1, b1, w1) in zip(kids0, kids1):
        di = np.where(w == 0, a0, a1)
        dj = np.where(w == 0, b0, b1)
        ww = np.where(w == 0, w0, w1)
        acc += eta_fine[fid(d, 2 * I + di, 2 * J + dj, ww, K)]
    return acc / 4.0


def block_jacobi_inverse(K):
    """Sparse inverse of the 3x3 node-block diagonal of K (component-major numbering)."""
    K = K.tocsr()
    n = K.shape[0] // 3
    idx = np.arange(n)
    Bk = np.zeros((n, 3, 3))
    for a in range(3):
        for c in range(3):
            Bk[:, a, c] = np.asarray(K[a * n + idx, c * n + idx]).ravel()
    Bi = np.linalg.inv(Bk)
    rows = [a * n + idx for a in range(3) for c in range(3)]
    cols = [c * n + idx for a in range(3) for c in range(3)]
    vals = [Bi[:, a, c] for a in range(3) for c in range(3)]
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=K.shape)


def rotation_basis(mesh):
    """The three rigid rotations e_i x x as columns (3 n x 3)."""
    X = mesh.node_xyz()
    cols = []
    for om in np.eye(3):
        cols.append(np.cross(om[None, :], X).T.ravel())
    return np.stack(cols, axis=1)


class Hierarchy:
    def __init__(self, level, n_r, r_in, r_out, eta0, bc=(O.FREE, O.FREE), nlev=None, div_term=True,
                 lo=0.1, hi=1.1, power_iters=15, pre=2, post=2, coarse_max_iters=50, coarse_rtol=1e-3,
                 kappa=0.0, quad=1):
        self.meshes = [ShellMesh(l, nr, r_in, r_out) for l, nr in mg_shapes(level, n_r, r_in, r_out)]
        if nlev is not None:
            self.meshes = self.meshes[:nlev]
        self.nlev = len(self.meshes)
        self.bc = bc
        self.eta = [np.asarray(eta0, dtype=np.float64)]
        for h in range(1, self.nlev):
            self.eta.append(coarsen_viscosity_semi(self.meshes[h - 1], self.meshes[h], self.eta[h - 1]))
        self.Pb = [O.projector_matrix(O.boundary_projectors(m, bc)) for m in self.meshes]
        self.K = [O.constrain_A(O.assemble_A(m, e, div_term, kappa, quad), Pb)
                  for m, e, Pb in zip(self.meshes, self.eta, self.Pb)]
        self.Dinv = [block_jacobi_inverse(K) for K in self.K]
        self.T = [vec_prolongation(self.meshes[h], self.meshes[h + 1]) for h in range(self.nlev - 1)]
        self.lo, self.hi, self.power_iters = lo, hi, power_iters
        self.pre, self.post = pre, post
        self.coarse_max_iters, self.coarse_rtol = coarse_max_iters, coarse_rtol
        self.singular = bc == (O.FREE, O.FREE)
        R = rotation_basis(self.meshes[-1])
        self.rotQ = np.linalg.qr(R)[0] if self.singular else None
        self.lam = [None] * self.nlev

    def prolong(self, h, xc):
        return self.Pb[h] @ (self.T[h] @ xc)

    def restrict(self, h, xf):
        return self.Pb[h + 1] @ (self.T[h].T @ xf)

    def setup(self, v0):
        """Power iterations on D^-1 K_h from v0 (level 0) and its restrictions."""
        v = np.asarray(v0, dtype=np.float64)
        for h in range(self.nlev):
            if h > 0:
                v = self.restrict(h - 1, v)
            if h == self.nlev - 1:
                break
            w = v / np.linalg.norm(v)
            lam = None
            for _ in range(self.power_iters):
                z = self.Dinv[h] @ (self.K[h] @ w)
                lam = np.linalg.norm(z)
                w = z / lam
            self.lam[h] = lam

    def chebyshev(self, h, x, b, zero_x):
        a, bb = self.lo * self.lam[h], self.hi * self.lam[h]
        theta, delta = 0.5 * (bb + a), 0.5 * (bb - a)
        sigma = theta / delta
        rho0 = 1.0 / sigma
        rho1 = 1.0 / (2.0 * sigma - rho0)
        r = b.copy() if zero_x else b - self.K[h] @ x
        d = (self.Dinv[h] @ r) / theta
        x = d.copy() if zero_x else x + d
        r = r - self.K[h] @ d
        d = rho1 * rho0 * d + (2.0 * rho1 / delta) * (self.Dinv[h] @ r)
        return x + d

    def coarse_cg(self, b):
        h = self.nlev - 1
        K, Dinv = self.K[h], self.Dinv[h]
        if self.singular:
            b = b - self.rotQ @ (self.rotQ.T @ b)
        x = np.zeros_like(b)
        r = b.copy()
        z = Dinv @ r
        p = z.copy()
        rz0 = rz = r @ z
        if rz0 > 0:
            for it in range(self.coarse_max_iters):
                q = K @ p
                alpha = rz / (p @ q)
                x = x + alpha * p
                r = r - alpha * q
                z = Dinv @ r
                rzn = r @ z
                beta = rzn / rz
                rz = rzn
                if not (rzn > self.coarse_rtol ** 2 * rz0) or it == self.coarse_max_iters - 1:
                    break
                p = z + beta * p
        if self.singular:
            x = x - self.rotQ @ (self.rotQ.T @ x)
        return x

    def vcycle(self, b, h=0):
        if h == self.nlev - 1:
            return self.coarse_cg(b)
        x = np.zeros_like(b)
        for s in range(self.pre):
            x = self.chebyshev(h, x, b, s == 0)
        r = b - self.K[h] @ x
        xc = self.vcycle(self.restrict(h, r), h + 1)
        x = x + self.prolong(h, xc)
        for s in range(self.post):
            x = self.chebyshev(h, x, b, False)
        return x
