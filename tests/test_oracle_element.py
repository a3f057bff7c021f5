"""Pins of the oracle's wedge element against closed forms from the paper (CPU only)."""
import numpy as np
import pytest

from oracle.element import (GHAT, QC, basis, basis_ref_gradients, geometry, geometry_at, hourglass_base_vectors,
                            hourglass_stabilised, hourglass_vectors, quadrature_rule, viscous_element_matrix,
                            viscous_element_matrix_rule)
from oracle.mesh import ShellMesh

REF_NODES = [(0.0, 0.0, -1.0), (1.0, 0.0, -1.0), (0.0, 1.0, -1.0),
             (0.0, 0.0, 1.0), (1.0, 0.0, 1.0), (0.0, 1.0, 1.0)]


def random_wedges(n=6, seed=1):
    """Wedges of a real shell mesh (one per diamond region), plus random nodal viscosity."""
    m = ShellMesh(3, 5, 0.55, 1.0)
    rng = np.random.default_rng(seed)
    ids = rng.choice(m.n_wedges, size=n, replace=False)
    x = m.node_xyz(m.wedge_nodes(ids).ravel()).reshape(-1, 6, 3)
    return x, np.exp(rng.normal(size=n))


def test_basis_nodal_and_partition_of_unity():
    for a, p in enumerate(REF_NODES):
        np.testing.assert_allclose(basis(*p), np.eye(6)[a], atol=1e-15)
    rng = np.random.default_rng(0)
    for _ in range(20):
        xi, eta = rng.random(2) * 0.5
        z = rng.uniform(-1, 1)
        assert abs(basis(xi, eta, z).sum() - 1.0) < 1e-15
    np.testing.assert_allclose(basis(*QC), 1.0 / 6.0, atol=1e-16)


def test_reference_gradients_match_finite_differences():
    """Central differences of the (at most bilinear) basis are exact up to rounding."""
    h = 1e-4
    for q in (QC, (0.2, 0.1, 0.3), (0.05, 0.7, -0.6)):
        g = basis_ref_gradients(*q)
        for m in range(3):
            e = np.zeros(3); e[m] = h
            fd = (basis(*(np.array(q) + e)) - basis(*(np.array(q) - e))) / (2 * h)
            np.testing.assert_allclose(g[:, m], fd, atol=1e-11)
    # closed form at q_c
    np.testing.assert_allclose(GHAT[:, 2], [-1 / 6] * 3 + [1 / 6] * 3, atol=1e-16)
    np.testing.assert_allclose(GHAT.sum(axis=0), 0.0, atol=1e-16)


def test_gradients_reproduce_linear_fields():
    """sum_j f(x_j) grad N_j(q_c) = grad f for every affine f (isoparametric map)."""
    x, _ = random_wedges()
    _, _, grad, _ = geometry(x)
    rng = np.random.default_rng(3)
    for _ in range(5):
        a, b = rng.normal(size=3), rng.normal()
        got = np.einsum("nj,njc->nc", x @ a + b, grad)
        np.testing.assert_allclose(got, np.broadcast_to(a, got.shape), atol=1e-12)


def _energy_by_finite_differences(xe, ue, eta, q0=QC, w=1.0):
    """Eq. (oneptenergy) at point q0 with weight w, evaluated from the interpolants x(q), u(q)
    by central differences."""
    h = 1e-4

    def interp(vals, q):
        return basis(*q) @ vals

    dx = np.empty((3, 3)); du = np.empty((3, 3))
    for m in range(3):
        e = np.zeros(3); e[m] = h
        qp, qm = np.array(q0) + e, np.array(q0) - e
        dx[:, m] = (interp(xe, qp) - interp(xe, qm)) / (2 * h)
        du[:, m] = (interp(ue, qp) - interp(ue, qm)) / (2 * h)
    gradu = du @ np.linalg.inv(dx)              # d u_c / d x_m
    eps = 0.5 * (gradu + gradu.T)
    V = abs(np.linalg.det(dx)) * w              # w_q = 1 (reference wedge volume) for q_c
    return V * eta * (2.0 * np.sum(eps * eps) - 2.0 / 3.0 * np.trace(gradu) ** 2)


def test_element_matrix_equals_one_point_energy():
    """u^T A_e u = E_e(u) of Eq. (oneptenergy), computed independently by finite differences."""
    x, eta = random_wedges()
    _, _, grad, V = geometry(x)
    A = viscous_element_matrix(grad, V, eta)
    rng = np.random.default_rng(5)
    for e in range(x.shape[0]):
        for _ in range(3):
            u = rng.normal(size=(6, 3))
            E = _energy_by_finite_differences(x[e], u, eta[e])
            assert abs(u.ravel() @ A[e] @ u.ravel() - E) <= 1e-7 * abs(E)


def test_element_matrix_rank_and_kernel():
    """Symmetric; rank 5 (deviatoric strain only); rank 6 without the -2/3 term; kernel holds
    translations, rotations, the dilatation x and the six hourglass modes (Eq. hourglass)."""
    x, eta = random_wedges()
    _, _, grad, V = geometry(x)
    A = viscous_element_matrix(grad, V, eta)
    A0 = viscous_element_matrix(grad, V, eta, div_term=False)
    for e in range(x.shape[0]):
        scale = np.abs(A[e]).max()
        np.testing.assert_array_equal(A[e], A[e].T)
        assert np.linalg.matrix_rank(A[e], tol=1e-10 * scale) == 5
        assert np.linalg.matrix_rank(A0[e], tol=1e-10 * scale) == 6
        kernel = []
        for d in range(3):
            t = np.zeros((6, 3)); t[:, d] = 1.0
            kernel.append(t)
        for om in np.eye(3):
            kernel.append(np.cross(om[None, :], x[e]))
        kernel.append(x[e].copy())
        for w in hourglass_vectors():
            for d in range(3):
                v = np.zeros((6, 3)); v[:, d] = w
                kernel.append(v)
        K = np.stack([k.ravel() for k in kernel])
        assert np.linalg.matrix_rank(K) == 13
        assert np.abs(A[e] @ K.T).max() <= 1e-13 * scale
    # nodal values of the hourglass modes, Eq. (hourglass)
    np.testing.assert_allclose(hourglass_vectors()[0], [1 / 3, -2 / 3, 1 / 3, -1 / 3, 2 / 3, -1 / 3], atol=1e-16)
    np.testing.assert_allclose(hourglass_vectors()[1], [1 / 3, 1 / 3, -2 / 3, -1 / 3, -1 / 3, 2 / 3], atol=1e-16)


def test_diagonal_closed_form():
    """(A_e)_{(j,d),(j,d)} = V eta (|grad N_j|^2 + 1/3 (d_d N_j)^2)."""
    x, eta = random_wedges()
    _, _, grad, V = geometry(x)
    A = viscous_element_matrix(grad, V, eta)
    for e in range(x.shape[0]):
        for j in range(6):
            for d in range(3):
                g = grad[e, j]
                want = V[e] * eta[e] * (g @ g + g[d] ** 2 / 3.0)
                assert abs(A[e, 3 * j + d, 3 * j + d] - want) <= 1e-13 * abs(want)


def _linear_fields(xe):
    """Nodal values (6, 3) of the 12 physical linear fields u_d = x_c (and the 3 constants)."""
    out = []
    for d in range(3):
        t = np.zeros((6, 3)); t[:, d] = 1.0
        out.append(t)
        for c in range(3):
            v = np.zeros((6, 3)); v[:, d] = xe[:, c]
            out.append(v)
    return out


def test_hourglass_base_vectors():
    """Eq. (hgstab) with Flanagan-Belytschko base vectors: g_m is orthogonal to every physical
    linear field and to the constants, and keeps the hourglass part: g_m . w_m' = w_m . w_m' on
    the reference-linear part's complement (g - w is a combination of gradient columns)."""
    x, _ = random_wedges()
    _, _, grad, _ = geometry(x)
    g = hourglass_base_vectors(x, grad)
    w = hourglass_vectors()
    for e in range(x.shape[0]):
        for m in range(2):
            assert abs(g[e, m].sum()) <= 1e-14
            for c in range(3):
                assert abs(g[e, m] @ x[e, :, c]) <= 1e-14
            # g_m - w_m lies in the span of the gradient columns dN/dx_c
            coef, *_ = np.linalg.lstsq(grad[e], g[e, m] - w[m], rcond=None)
            np.testing.assert_allclose(grad[e] @ coef, g[e, m] - w[m], atol=1e-13)


def test_stabilised_element_matrix():
    """A_e + eps sum (g_m x e_d)(g_m x e_d)^T: symmetric, rank 11 (5 + 6: every hourglass mode
    now has energy), equal to A_e on all linear fields, eps = kappa tr(A_e) / 18, and the added
    energy of the unit reference hourglass mode w_m x e_d is eps sum_m' (g_m' . w_m)^2."""
    x, eta = random_wedges()
    _, _, grad, V = geometry(x)
    A = viscous_element_matrix(grad, V, eta)
    g = hourglass_base_vectors(x, grad)
    kappa = 0.25
    As = hourglass_stabilised(A, g, kappa)
    w = hourglass_vectors()
    for e in range(x.shape[0]):
        scale = np.abs(As[e]).max()
        np.testing.assert_array_equal(As[e], As[e].T)
        assert np.linalg.matrix_rank(As[e], tol=1e-10 * scale) == 11
        assert np.linalg.eigvalsh(As[e]).min() >= -1e-12 * scale
        for u in _linear_fields(x[e]):
            np.testing.assert_allclose(As[e] @ u.ravel(), A[e] @ u.ravel(), atol=1e-13 * scale)
        eps = kappa * np.trace(A[e]) / 18.0
        for m in range(2):
            for d in range(3):
                v = np.zeros((6, 3)); v[:, d] = w[m]
                got = v.ravel() @ (As[e] - A[e]) @ v.ravel()
                want = eps * sum((g[e, mm] @ w[m]) ** 2 for mm in range(2))
                assert abs(got - want) <= 1e-12 * abs(want)


# --------------------------------------------------------------- second radial quadrature point
def test_two_point_rule_energy_and_volume():
    """Two radial points: u^T A_e u is the sum of Eq. (oneptenergy) at (1/3, 1/3, -/+ 1/sqrt 3)
    with weights 1/2 (finite differences of the interpolants), and the weights times |det J|
    add up to |det M| (r_t^3 - r_b^3) / 6: the exact integral of |det J| = rho^2 h |det M| along
    the wedge's centre line (M = [s1 - s0, s2 - s0, (s0 + s1 + s2) / 3] from the unit directions)."""
    x, eta = random_wedges()
    rule = quadrature_rule(2)
    z = 1.0 / np.sqrt(3.0)
    assert [p for p, _ in rule] == [(1 / 3, 1 / 3, -z), (1 / 3, 1 / 3, z)] and [w for _, w in rule] == [0.5, 0.5]
    A2 = viscous_element_matrix_rule(x, eta, rule)
    rng = np.random.default_rng(6)
    for e in range(x.shape[0]):
        for _ in range(3):
            u = rng.normal(size=(6, 3))
            E = sum(_energy_by_finite_differences(x[e], u, eta[e], p, w) for p, w in rule)
            assert abs(u.ravel() @ A2[e] @ u.ravel() - E) <= 1e-7 * abs(E)
        rb, rt = np.linalg.norm(x[e, 0]), np.linalg.norm(x[e, 3])
        s = x[e, :3] / rb
        M = np.stack([s[1] - s[0], s[2] - s[0], s.mean(axis=0)], axis=1)
        V = sum(geometry_at(x[e:e + 1], p, w)[1][0] for p, w in rule)
        want = abs(np.linalg.det(M)) * (rt ** 3 - rb ** 3) / 6.0
        assert abs(V - want) <= 1e-13 * want


def test_two_point_rule_is_exact_in_zeta():
    """On the wedge's centre line the integrand is a quadratic in zeta (rho^2 from |det J| against
    1 / rho^2, 1 / rho or 1 from the gradients, times the radial basis), so the two-point rule
    equals a six-point Gauss-Legendre rule in zeta to rounding; the one-point rule does not."""
    x, eta = random_wedges()
    zg, wg = np.polynomial.legendre.leggauss(6)
    rule6 = [((1 / 3, 1 / 3, z), 0.5 * w) for z, w in zip(zg, wg)]
    for div_term in (True, False):
        A6 = viscous_element_matrix_rule(x, eta, rule6, div_term)
        A2 = viscous_element_matrix_rule(x, eta, quadrature_rule(2), div_term)
        A1 = viscous_element_matrix_rule(x, eta, quadrature_rule(1), div_term)
        scale = np.abs(A6).max()
        assert np.abs(A2 - A6).max() <= 1e-13 * scale
        assert np.abs(A1 - A6).max() >= 1e-3 * scale


def test_two_point_rank_and_kernel():
    """With two radial points five of the six hourglass modes of Eq. (hourglass) get energy.  The
    one left is the twist u = zeta (sbar x s(xi, eta)) / 2 (top layer turned about the wedge axis
    sbar, bottom layer back): its lateral gradient is skew and its radial derivative vanishes on
    the centre line, where the rule samples.  So the element matrix is symmetric positive
    semi-definite of rank 11 without the -2/3 term (18 - 6 rigid motions - the twist) and 10 with
    it (the dilatation x too), and on the hourglass span it has rank 5."""
    x, eta = random_wedges()
    A = viscous_element_matrix_rule(x, eta, quadrature_rule(2))
    A0 = viscous_element_matrix_rule(x, eta, quadrature_rule(2), div_term=False)
    w = hourglass_vectors()
    for e in range(x.shape[0]):
        scale = np.abs(A[e]).max()
        np.testing.assert_allclose(A[e], A[e].T, atol=1e-15 * scale)
        assert np.linalg.matrix_rank(A[e], tol=1e-10 * scale) == 10
        assert np.linalg.matrix_rank(A0[e], tol=1e-10 * scale) == 11
        assert np.linalg.eigvalsh(A0[e]).min() >= -1e-12 * scale
        kernel = []
        for d in range(3):
            t = np.zeros((6, 3)); t[:, d] = 1.0
            kernel.append(t.ravel())
        for om in np.eye(3):
            kernel.append(np.cross(om[None, :], x[e]).ravel())
        su = x[e, :3] / np.linalg.norm(x[e, 0])
        tw = 0.5 * np.cross(su.mean(axis=0)[None, :], su)
        kernel.append(np.concatenate([-tw, tw]).ravel())
        K = np.stack(kernel)
        assert np.linalg.matrix_rank(K) == 7
        assert np.abs(A0[e] @ K.T).max() <= 1e-13 * scale
        assert np.abs(A[e] @ K.T).max() <= 1e-13 * scale
        assert np.abs(A[e] @ x[e].ravel()).max() <= 1e-13 * scale
        Hs = []
        for m in range(2):
            for d in range(3):
                v = np.zeros((6, 3)); v[:, d] = w[m]
                Hs.append(v.ravel())
        Hs = np.stack(Hs)
        assert np.linalg.matrix_rank(Hs @ A0[e] @ Hs.T, tol=1e-10 * scale) == 5
