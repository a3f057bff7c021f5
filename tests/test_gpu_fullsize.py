"""Parity at the full benchmark size: level 7 (129 x 129 nodes per diamond), 129 radial layers,
63.4 M velocity DoFs, in the launch configuration the benchmark times.

The oracle cannot evaluate the whole shell quickly, so the GPU results are compared on sampled
nodes: the oracle applies its element matrices over exactly the wedges around the sampled nodes,
which makes its values there complete.  Samples cover both boundary layers, interior layers,
diamond edges, the two poles and a diamond corner.  Properties that hold at any size are checked
on the whole field: symmetry of A and adjointness of B and B^T (inner products over unique
nodes), and B of a rigid rotation vanishing.
"""
import numpy as np
import pytest

from oracle import operators as O
from oracle.mesh import ShellMesh
from paper_2609_21633_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LEVEL, NR, R_IN, R_OUT = 7, 129, 0.55, 1.0
TOL64, TOL32 = 1e-12, 2e-5


@pytest.fixture(scope="module")
def tn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_21633_gb300 as tn
    tn.lib()
    return tn


class FullShell:
    """The full-size mesh on both sides; only per-sample index maps are built on the host."""

    def __init__(self, tn, kappa, quad=1):
        self.tn = tn
        self.m = tn.tn_mesh_create(LEVEL, NR, R_IN, R_OUT, hg_kappa=kappa, radial_quad_points=quad)
        self.info = tn.tn_mesh_info(self.m, 0)
        self.om = ShellMesh(LEVEL, NR, R_IN, R_OUT)
        N, P = self.info["N"], self.info["pitch"]
        # one (d, i, j) position of every de-duplicated lateral point
        d, i, j = np.meshgrid(np.arange(10), np.arange(N + 1), np.arange(N + 1), indexing="ij")
        self.lat_dij = np.zeros((self.om.n_lat, 3), dtype=np.int64)
        self.lat_dij[self.om.lat_id.ravel()] = np.stack([d.ravel(), i.ravel(), j.ravel()], axis=1)
        self.N, self.P = N, P
        canon = tn.tn_mesh_canonical_index(self.m, 0)
        self.canon = canon
        self.unique = torch.tensor(canon == np.arange(canon.size), device="cuda", dtype=torch.float64)

    def layout_of_nodes(self, nodes):
        lat, k = np.divmod(np.asarray(nodes, dtype=np.int64), NR)
        d, i, j = self.lat_dij[lat].T
        return ((d * NR + k) * (self.N + 1) + i) * self.P + j

    def layout_of_wedges(self, wedges):
        d, i, j, w, k = self.om.wedge_labels(wedges).T
        return (((d * (NR - 1) + k) * self.N + i) * self.N + j) * 2 + w

    def field(self, seed, n=None):
        """Seeded layout field with equal values on the copies of a node, zero padding."""
        n = n or self.info["n_layout"]
        canon = self.canon if n == self.info["n_layout"] else self.tn.tn_mesh_canonical_index(self.m, 1)
        v = inputs.normal(n, seed)
        return np.where(canon >= 0, v[np.maximum(canon, 0)], 0.0)

    def samples(self, seed=5, n=120):
        rng = np.random.default_rng(seed)
        N = self.N
        pos = [(int(rng.integers(10)), int(rng.integers(NR)), int(rng.integers(N + 1)), int(rng.integers(N + 1)))
               for _ in range(n)]
        pos += [(0, 0, 0, 0), (5, NR - 1, N, N), (3, 64, 0, 17), (7, 0, 40, N), (2, NR - 1, N, 0),
                (9, 1, 64, 64), (4, NR - 2, 0, N)]
        return np.array([self.om.node_of_layout(d, i, j, k) for d, k, i, j in pos], dtype=np.int64)

    def close(self):
        self.tn.tn_mesh_destroy(self.m)


@pytest.fixture(scope="module", params=[(0.0, 1), (0.3, 1), (0.0, 2)], ids=["plain", "hg0.3", "quad2"])
def shell(tn, request):
    s = FullShell(tn, *request.param)
    s.kappa, s.quad = request.param
    yield s
    s.close()


def test_sampled_A_and_diag_at_full_size(tn, shell):
    s, om = shell, shell.om
    n_w = s.info["n_wedges"]
    eta_l = inputs.lognormal_viscosity(n_w, 11)
    tn.tn_set_viscosity(s.m, torch.tensor(eta_l, device="cuda"))
    u_l = [s.field(20 + c) for c in range(3)]
    nodes = s.samples()
    wedges = om.wedges_of_nodes(nodes)
    near = np.unique(om.wedge_nodes(wedges).ravel())
    # oracle inputs on the nodes / wedges it touches (the rest stays zero and is never read)
    eta = np.zeros(om.n_wedges)
    eta[wedges] = eta_l[s.layout_of_wedges(wedges)]
    u = np.zeros((3, om.n_nodes))
    for c in range(3):
        u[c, near] = u_l[c][s.layout_of_nodes(near)]
    P = O.boundary_projectors(om)
    want = O.apply_A_constrained(om, eta, u, P, wedges=wedges, kappa=s.kappa, quad=s.quad)[:, nodes]
    want_d = O.diag_A_constrained(om, eta, P, wedges=wedges, kappa=s.kappa, quad=s.quad)[:, nodes]
    idx = s.layout_of_nodes(nodes)
    for dtype, tol in ((torch.float64, TOL64), (torch.float32, TOL32)):
        y = [torch.zeros(s.info["n_layout"], device="cuda", dtype=dtype) for _ in range(3)]
        tn.tn_apply_A(s.m, 0, [torch.tensor(v, device="cuda", dtype=dtype) for v in u_l], y)
        got = np.stack([t.double().cpu().numpy()[idx] for t in y])
        err = np.abs(got - want).max() / np.abs(want).max()
        print(f"kappa {s.kappa} {dtype}: A sampled max-rel {err:.2e}")
        assert err <= tol, (dtype, err)
    d = [torch.zeros(s.info["n_layout"], device="cuda", dtype=torch.float64) for _ in range(3)]
    tn.tn_diag_A(s.m, 0, d)
    got_d = np.stack([t.cpu().numpy()[idx] for t in d])
    err = np.abs(got_d - want_d).max() / np.abs(want_d).max()
    print(f"kappa {s.kappa}: diag sampled max-rel {err:.2e}")
    assert err <= TOL64


def test_symmetry_and_adjointness_at_full_size(tn, shell):
    s = shell
    if s.kappa != 0.0 or s.quad != 1:
        pytest.skip("the B blocks do not depend on the hourglass control or the quadrature of A")
    n = s.info["n_layout"]
    pinfo = tn.tn_mesh_info(s.m, 1)
    tn.tn_set_viscosity(s.m, torch.tensor(inputs.lognormal_viscosity(s.info["n_wedges"], 12), device="cuda"))
    w = s.unique
    wp = torch.tensor(tn.tn_mesh_canonical_index(s.m, 1) == np.arange(pinfo["n_layout"]), device="cuda",
                      dtype=torch.float64)
    u = [torch.tensor(s.field(30 + c), device="cuda") for c in range(3)]
    v = [torch.tensor(s.field(40 + c), device="cuda") for c in range(3)]
    p = torch.tensor(s.field(50, pinfo["n_layout"]), device="cuda")

    def dot(a, b, wt):
        return float(sum(torch.dot(x * wt, y) for x, y in zip(a, b)))

    Au, Av = [[torch.zeros(n, device="cuda", dtype=torch.float64) for _ in range(3)] for _ in range(2)]
    tn.tn_apply_A(s.m, 0, u, Au)
    tn.tn_apply_A(s.m, 0, v, Av)
    a1, a2 = dot(Au, v, w), dot(u, Av, w)
    assert abs(a1 - a2) <= 1e-12 * (abs(a1) + dot(Au, Au, w) ** 0.5 * dot(v, v, w) ** 0.5)
    q = torch.zeros(pinfo["n_layout"], device="cuda", dtype=torch.float64)
    tn.tn_apply_B(s.m, 0, u, q)
    BTp = [torch.zeros(n, device="cuda", dtype=torch.float64) for _ in range(3)]
    tn.tn_apply_BT(s.m, 0, p, BTp)
    b1, b2 = float(torch.dot(q * wp, p)), dot(u, BTp, w)
    scale = float(torch.dot(q * wp, q)) ** 0.5 * float(torch.dot(p * wp, p)) ** 0.5
    assert abs(b1 - b2) <= 1e-12 * scale, (b1, b2)
    # B of a rigid rotation (tangential at both surfaces, divergence-free) vanishes
    xyz = tn.tn_mesh_lateral_points(s.m, 0).reshape(10, s.N + 1, s.N + 1, 3)
    radii = R_IN + (R_OUT - R_IN) * np.arange(NR) / (NR - 1)
    om_ = np.array([0.3, -1.1, 0.7])
    rot = np.cross(om_[None, :], xyz.reshape(-1, 3)).reshape(10, 1, s.N + 1, s.N + 1, 3) * radii[None, :, None, None,
                                                                                                 None]
    rl = np.zeros((3, 10, NR, s.N + 1, s.P))
    rl[:, :, :, :, :s.N + 1] = np.moveaxis(rot, -1, 0)
    r_dev = [torch.tensor(rl[c].ravel(), device="cuda") for c in range(3)]
    tn.tn_apply_B(s.m, 0, r_dev, q)
    qr = float(torch.abs(q * wp).max())
    tn.tn_apply_B(s.m, 0, u, q)
    qu = float(torch.abs(q * wp).max())
    ur = max(float(torch.abs(t).max()) for t in r_dev)
    uu = max(float(torch.abs(t).max()) for t in u)
    assert qr <= 1e-12 * qu * ur / uu, (qr, qu)
