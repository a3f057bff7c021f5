"""GPU parity of the wedge Stokes operators against the CPU FP64 oracle.

Every call goes through the C ABI (ctypes binding).  FP64 bar: normwise max-relative
error <= 1e-12 (max |y_gpu - y_oracle| / max |y_oracle|); the FP32 path is checked
against a bound derived from single-precision rounding."""
import numpy as np
import pytest

from oracle import operators as O
from oracle.fields import buoyancy_rhs, coarsen_viscosity, viscosity
from oracle.mesh import ShellMesh
from paper_2609_21633_gb300 import inputs
from tests.layout import LayoutMap, max_rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5

BCS = {"free/free": (0, 0), "noslip/free": (1, 0), "noslip/noslip": (1, 1)}
ORACLE_BC = {0: O.FREE, 1: O.NOSLIP}


@pytest.fixture(scope="module")
def tn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_21633_gb300 as tn
    tn.lib()
    return tn


class Case:
    """One mesh on both sides with random fields (seeded)."""

    def __init__(self, tn, level, n_r, bc=(0, 0), div_term=True, seed=0, r_in=0.55, r_out=1.0, eta_storage=0,
                 hg_kappa=0.0, quad=1, fp64_element=0):
        self.tn = tn
        self.m = tn.tn_mesh_create(level, n_r, r_in, r_out, bc[0], bc[1], div_term, eta_storage=eta_storage,
                                   hg_kappa=hg_kappa, radial_quad_points=quad, fp64_element=fp64_element)
        self.info = tn.tn_mesh_info(self.m, 0)
        self.om = ShellMesh(level, n_r, r_in, r_out)
        self.map = LayoutMap(self.info, self.om)
        self.P = O.boundary_projectors(self.om, (ORACLE_BC[bc[0]], ORACLE_BC[bc[1]]))
        self.eta = inputs.lognormal_viscosity(self.om.n_wedges, seed + 1)
        self.div_term = div_term
        self.eta_dev = torch.tensor(self.map.wedges_to_layout(self.eta), device="cuda")
        tn.tn_set_viscosity(self.m, self.eta_dev)
        self.rng_seed = seed

    def vec(self, seed, n=None):
        return inputs.normal((3, self.om.n_nodes) if n is None else n, seed)

    def dev(self, vals, dtype=torch.float64):
        return torch.tensor(self.map.to_layout(vals), device="cuda", dtype=dtype)

    def zeros(self, n=3, dtype=torch.float64, info=None):
        info = info or self.info
        return [torch.zeros(info["n_layout"], device="cuda", dtype=dtype) for _ in range(n)]

    def host(self, t, mp=None):
        return (mp or self.map).from_layout(t.double().cpu().numpy())

    def close(self):
        self.tn.tn_mesh_destroy(self.m)


def test_mesh_matches_oracle(tn):
    for level in (1, 3, 5):
        c = Case(tn, level, 3)
        pts = tn.tn_mesh_lateral_points(c.m, 0)
        assert np.abs(pts - c.om.lat_pts).max() <= 2e-16
        canon = tn.tn_mesh_canonical_index(c.m, 0)
        # two layout entries are copies of one node exactly when the oracle de-duplicates them together
        assert np.array_equal(c.map.node[np.searchsorted(c.map.idx, canon[c.map.idx])], c.map.node)
        groups = np.unique(canon[c.map.idx]).size
        assert groups == c.om.n_nodes
        c.close()


@pytest.mark.parametrize("level,n_r", [(1, 3), (2, 5), (3, 9), (4, 17), (4, 27), (4, 33), (5, 9)])
@pytest.mark.parametrize("bc", ["free/free", "noslip/free"])
def test_apply_A_f64(tn, level, n_r, bc):
    c = Case(tn, level, n_r, BCS[bc])
    u = c.vec(10)
    want = O.apply_A_constrained(c.om, c.eta, u, c.P)
    ud = [c.dev(u[i]) for i in range(3)]
    y = c.zeros()
    tn.tn_apply_A(c.m, 0, ud, y)
    got = np.stack([c.host(t) for t in y])
    assert max_rel(got, want) <= TOL64
    # deterministic: a second apply is bitwise identical
    y2 = c.zeros()
    tn.tn_apply_A(c.m, 0, ud, y2)
    assert all(torch.equal(a, b) for a, b in zip(y, y2))
    c.close()


@pytest.mark.parametrize("level,n_r,bc,kappa,div_term", [
    (5, 9, "free/free", 0.0, True), (5, 17, "noslip/free", 0.0, True), (6, 9, "free/free", 0.0, True),
    (5, 9, "free/free", 0.3, True), (5, 9, "noslip/noslip", 0.0, False)])
def test_apply_A_f64_element_arithmetics(tn, level, n_r, bc, kappa, div_term):
    """Levels with N >= 32 evaluate the FP64 element op in double-float by default
    (TN_FP64_ELEM_DOUBLE_FLOAT) or in binary64 (TN_FP64_ELEM_BINARY64): both meet the FP64 bar
    against the oracle, and they agree with each other to it."""
    got = {}
    for elem in (tn.TN_FP64_ELEM_DOUBLE_FLOAT, tn.TN_FP64_ELEM_BINARY64):
        c = Case(tn, level, n_r, BCS[bc], div_term=div_term, hg_kappa=kappa, fp64_element=elem)
        u = c.vec(31)
        want = O.apply_A_constrained(c.om, c.eta, u, c.P, div_term=div_term, kappa=kappa)
        y = c.zeros()
        tn.tn_apply_A(c.m, 0, [c.dev(u[i]) for i in range(3)], y)
        got[elem] = np.stack([c.host(t) for t in y])
        err = max_rel(got[elem], want)
        print(f"level {level} / {n_r} {bc} kappa {kappa} element arithmetic {elem}: max-rel {err:.2e}")
        assert err <= TOL64, (elem, err)
        c.close()
    assert max_rel(got[0], got[1]) <= TOL64


def test_apply_A_without_div_term(tn):
    c = Case(tn, 3, 9, div_term=False)
    u = c.vec(11)
    want = O.apply_A_constrained(c.om, c.eta, u, c.P, div_term=False)
    y = c.zeros()
    tn.tn_apply_A(c.m, 0, [c.dev(u[i]) for i in range(3)], y)
    assert max_rel(np.stack([c.host(t) for t in y]), want) <= TOL64
    c.close()


def test_apply_A_f32(tn):
    c = Case(tn, 4, 17)
    u = c.vec(12)
    want = O.apply_A_constrained(c.om, c.eta, u, c.P)
    y = c.zeros(dtype=torch.float32)
    tn.tn_apply_A(c.m, 0, [c.dev(u[i], torch.float32) for i in range(3)], y)
    got = np.stack([c.host(t) for t in y])
    assert max_rel(got, want) <= TOL32
    c.close()


@pytest.mark.parametrize("level,n_r,bc,div_term", [(3, 9, "noslip/free", True), (4, 17, "free/free", True),
                                                  (4, 9, "free/free", False), (5, 9, "free/free", True),
                                                  (5, 9, "noslip/noslip", False)])
def test_hourglass_control_apply_and_diag(tn, level, n_r, bc, div_term):
    """Eq. (hgstab) with kappa = 0.3: FP64 apply and diagonal at the FP64 bar, FP32 apply at the
    FP32 bar, against the oracle's explicit element matrices with Flanagan-Belytschko vectors."""
    kappa = 0.3
    c = Case(tn, level, n_r, BCS[bc], div_term=div_term, hg_kappa=kappa)
    u = c.vec(21)
    want = O.apply_A_constrained(c.om, c.eta, u, c.P, div_term=div_term, kappa=kappa)
    plain = O.apply_A_constrained(c.om, c.eta, u, c.P, div_term=div_term)
    assert max_rel(plain, want) > 1e-3  # the control changes the result
    for dtype, tol in ((torch.float64, TOL64), (torch.float32, TOL32)):
        y = c.zeros(dtype=dtype)
        tn.tn_apply_A(c.m, 0, [c.dev(u[i], dtype) for i in range(3)], y)
        assert max_rel(np.stack([c.host(t) for t in y]), want) <= tol, dtype
    d = c.zeros()
    tn.tn_diag_A(c.m, 0, d)
    want_d = O.diag_A_constrained(c.om, c.eta, c.P, div_term=div_term, kappa=kappa)
    assert max_rel(np.stack([c.host(t) for t in d]), want_d) <= TOL64
    c.close()


@pytest.mark.parametrize("level,n_r,bc,div_term", [(2, 5, "free/free", True), (3, 9, "noslip/free", True),
                                                  (4, 17, "free/free", True), (4, 9, "free/free", False),
                                                  (5, 9, "noslip/noslip", True), (5, 5, "free/free", True)])
def test_second_radial_point_apply_and_diag(tn, level, n_r, bc, div_term):
    """The A block with the second radial quadrature point (two-point Gauss rule in zeta): FP64
    apply and diagonal at the FP64 bar, FP32 apply at the FP32 bar, against the oracle's element
    matrices summed over the two points.  Level 5 runs the 16 x 32 halo-free FP64 tiles."""
    c = Case(tn, level, n_r, BCS[bc], div_term=div_term, quad=2)
    u = c.vec(23)
    want = O.apply_A_constrained(c.om, c.eta, u, c.P, div_term=div_term, quad=2)
    plain = O.apply_A_constrained(c.om, c.eta, u, c.P, div_term=div_term)
    assert max_rel(plain, want) > 1e-3  # the rule changes the result
    for dtype, tol in ((torch.float64, TOL64), (torch.float32, TOL32)):
        y = c.zeros(dtype=dtype)
        tn.tn_apply_A(c.m, 0, [c.dev(u[i], dtype) for i in range(3)], y)
        err = max_rel(np.stack([c.host(t) for t in y]), want)
        print(f"l{level} n_r {n_r} {bc} div {div_term} {dtype}: {err:.2e}")
        assert err <= tol, dtype
    want_d = O.diag_A_constrained(c.om, c.eta, c.P, div_term=div_term, quad=2)
    for dtype, tol in ((torch.float64, TOL64), (torch.float32, TOL32)):
        d = c.zeros(dtype=dtype)
        tn.tn_diag_A(c.m, 0, d)
        assert max_rel(np.stack([c.host(t) for t in d]), want_d) <= tol, dtype
    c.close()


def test_second_radial_point_options(tn):
    """radial_quad_points is 1 or 2 (0 means 1) and excludes hourglass control."""
    for q, kappa in ((3, 0.0), (-1, 0.0), (2, 0.3)):
        with pytest.raises(tn.TnError):
            tn.tn_mesh_create(2, 5, 0.55, 1.0, radial_quad_points=q, hg_kappa=kappa)
    tn.tn_mesh_destroy(tn.tn_mesh_create(2, 5, 0.55, 1.0, radial_quad_points=0))


def _bf16_round(x32):
    """float32 -> bfloat16 (round to nearest even), returned as float32."""
    b = x32.view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16).astype(np.uint32)
    return (b << 16).view(np.float32)


def stored_viscosity(eta_layout, N, n_r, kind):
    """The viscosity the FP32 kernels see under 16-bit storage, from the format the header
    states: per radial column of wedges c = fp32(sqrt(min max)), value = 16-bit(fp32(eta / c)) * c."""
    e = eta_layout.reshape(10, n_r - 1, 2 * N * N)
    c = np.sqrt(e.min(axis=1) * e.max(axis=1)).astype(np.float32)
    r = (e / c[:, None, :].astype(np.float64)).astype(np.float32)
    q = _bf16_round(r) if kind == 1 else r.astype(np.float16).astype(np.float32)
    return (q.astype(np.float64) * c[:, None, :].astype(np.float64)).reshape(-1)


@pytest.mark.parametrize("kind,unit", [(1, 2.0 ** -8), (2, 2.0 ** -11)])
def test_apply_A_and_diag_f32_with_16bit_viscosity(tn, kind, unit):
    c = Case(tn, 4, 17, eta_storage=kind)
    eta_q = c.map.wedges_from_layout(stored_viscosity(c.map.wedges_to_layout(c.eta), 16, 17, kind))
    # rounding to nearest: relative change at most the unit roundoff (plus the FP32 steps)
    assert np.abs(eta_q / c.eta - 1).max() <= unit * (1 + 1e-3) + 2e-7
    u = c.vec(12)
    y = c.zeros(dtype=torch.float32)
    tn.tn_apply_A(c.m, 0, [c.dev(u[i], torch.float32) for i in range(3)], y)
    got = np.stack([c.host(t) for t in y])
    err_q = max_rel(got, O.apply_A_constrained(c.om, eta_q, u, c.P))
    err_full = max_rel(got, O.apply_A_constrained(c.om, c.eta, u, c.P))
    print(f"kind {kind}: vs stored eta {err_q:.2e}, vs FP64 eta {err_full:.2e}")
    assert err_q <= TOL32
    assert err_full > 10 * err_q  # the kernel really read the 16-bit values
    d = c.zeros(dtype=torch.float32)
    tn.tn_diag_A(c.m, 0, d)
    assert max_rel(np.stack([c.host(t) for t in d]), O.diag_A_constrained(c.om, eta_q, c.P)) <= TOL32
    c.close()


@pytest.mark.parametrize("level,n_r,bc,kappa,div_term,kind", [
    (5, 17, "free/free", 0.0, True, 0), (5, 27, "noslip/free", 0.0, True, 0), (6, 9, "noslip/noslip", 0.0, False, 0),
    (5, 17, "free/free", 0.3, True, 0), (6, 11, "noslip/free", 0.3, False, 0), (5, 9, "free/free", 0.0, True, 1),
    (5, 19, "noslip/free", 0.3, True, 2)])
def test_apply_A_f32_paired_tiles(tn, level, n_r, bc, kappa, div_term, kind):
    """FP32 A on levels with N >= 32 (two cells per thread, tile lines through the ring buffer,
    radial chunks with a ragged last one when n_r - 1 is not a multiple of the chunk) against the
    oracle; inputs moved off the 16-byte boundary take the square tiles, which agree to FP32
    rounding."""
    c = Case(tn, level, n_r, BCS[bc], div_term=div_term, eta_storage=kind, hg_kappa=kappa)
    N = 2 ** level
    eta = c.eta if kind == 0 else c.map.wedges_from_layout(
        stored_viscosity(c.map.wedges_to_layout(c.eta), N, n_r, kind))
    u = c.vec(31)
    want = O.apply_A_constrained(c.om, eta, u, c.P, div_term=div_term, kappa=kappa)
    ud = [c.dev(u[i], torch.float32) for i in range(3)]
    y = c.zeros(dtype=torch.float32)
    tn.tn_apply_A(c.m, 0, ud, y)
    got = np.stack([c.host(t) for t in y])
    err = max_rel(got, want)
    # the same input one element past a 16-byte boundary
    n = c.info["n_layout"]
    buf = [torch.zeros(n + 4, device="cuda", dtype=torch.float32) for _ in range(3)]
    for b, x in zip(buf, ud):
        b[1:n + 1] = x
    y2 = c.zeros(dtype=torch.float32)
    tn.tn_apply_A(c.m, 0, [b[1:n + 1] for b in buf], y2)
    got2 = np.stack([c.host(t) for t in y2])
    print(f"level {level} / {n_r} kappa {kappa} kind {kind}: paired {err:.2e}, square tiles {max_rel(got2, want):.2e}")
    assert err <= TOL32
    assert max_rel(got2, want) <= TOL32
    assert max_rel(got, got2) <= TOL32
    c.close()


@pytest.mark.parametrize("level,n_r,bc", [(2, 5, "free/free"), (3, 9, "noslip/free"), (4, 27, "free/free"),
                                          (5, 9, "free/free"), (5, 17, "noslip/free")])
def test_apply_B_and_BT_f64(tn, level, n_r, bc):
    c = Case(tn, level, n_r, BCS[bc])
    pm = O.pressure_mesh(c.om)
    Pp = O.prolongation(c.om, pm)
    B = O.assemble_B(c.om, Pp)
    Pm = O.projector_matrix(c.P)
    pinfo = tn.tn_mesh_info(c.m, 1)
    pmap = LayoutMap(pinfo, pm)
    u = c.vec(20)
    q = torch.zeros(pinfo["n_layout"], device="cuda", dtype=torch.float64)
    tn.tn_apply_B(c.m, 0, [c.dev(u[i]) for i in range(3)], q)
    want_q = B @ (Pm @ u.ravel())
    assert max_rel(pmap.from_layout(q.cpu().numpy()), want_q) <= TOL64
    p = inputs.normal(pm.n_nodes, 21)
    y = c.zeros()
    tn.tn_apply_BT(c.m, 0, torch.tensor(pmap.to_layout(p), device="cuda"), y)
    want_y = (Pm @ (B.T @ p)).reshape(3, -1)
    assert max_rel(np.stack([c.host(t) for t in y]), want_y) <= TOL64
    c.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_operator_steps_from_host_memory(tn, dtype):
    """tn_operator_steps_host: five pipelined steps with distinct pinned host inputs return, bitwise,
    what the device-side calls return (steps 0, 2, 4 share one device buffer set, 1 and 3 the
    other, so a missing wait between the streams would mix steps), and A u matches the oracle."""
    c = Case(tn, 5, 9, BCS["free/free"])
    pm = O.pressure_mesh(c.om)
    pinfo = tn.tn_mesh_info(c.m, 1)
    pmap = LayoutMap(pinfo, pm)
    n, npr = c.info["n_layout"], pinfo["n_layout"]
    steps = 5
    u_h = [[torch.tensor(c.map.to_layout(c.vec(60 + i)[k]), dtype=dtype).pin_memory() for k in range(3)]
           for i in range(steps)]
    p_h = [torch.tensor(pmap.to_layout(inputs.normal(pm.n_nodes, 70 + i)), dtype=dtype).pin_memory()
           for i in range(steps)]
    sizes = [n, n, n, npr, n, n, n, n, n, n]
    out_h = [[torch.full((m,), float("nan"), dtype=dtype).pin_memory() for m in sizes] for _ in range(steps)]
    # real layout entries (the row padding j > N is never written by the kernels)
    real0 = torch.from_numpy(tn.tn_mesh_canonical_index(c.m, 0) >= 0)
    real1 = torch.from_numpy(tn.tn_mesh_canonical_index(c.m, 1) >= 0)
    tn.tn_operator_steps_host(c.m, u_h, p_h, out_h)
    torch.cuda.synchronize()
    for i in range(steps):
        u = [t.cuda() for t in u_h[i]]
        yA = [torch.empty(n, device="cuda", dtype=dtype) for _ in range(3)]
        q = torch.empty(npr, device="cuda", dtype=dtype)
        yBT = [torch.empty(n, device="cuda", dtype=dtype) for _ in range(3)]
        d = [torch.empty(n, device="cuda", dtype=dtype) for _ in range(3)]
        tn.tn_apply_A(c.m, 0, u, yA)
        tn.tn_apply_B(c.m, 0, u, q)
        tn.tn_apply_BT(c.m, 0, p_h[i].cuda(), yBT)
        tn.tn_diag_A(c.m, 0, d)
        for k, t in enumerate(yA + [q] + yBT + d):
            real = real1 if k == 3 else real0
            assert torch.equal(out_h[i][k][real], t.cpu()[real]), (i, k)
            assert not torch.any(out_h[i][k][~real]), (i, k)  # padding comes back as 0
        want = O.apply_A_constrained(c.om, c.eta, c.vec(60 + i), c.P)
        tol = TOL64 if dtype == torch.float64 else TOL32
        assert max_rel(np.stack([c.map.from_layout(out_h[i][k].double().numpy()) for k in range(3)]), want) <= tol
    c.close()


@pytest.mark.parametrize("level,n_r,bc", [(2, 5, "free/free"), (3, 9, "noslip/free"),
                                          (4, 17, "free/free"), (5, 9, "noslip/noslip")])
def test_diagonals_f64(tn, level, n_r, bc):
    c = Case(tn, level, n_r, BCS[bc])
    want = O.diag_A_constrained(c.om, c.eta, c.P)
    d = c.zeros()
    tn.tn_diag_A(c.m, 0, d)
    assert max_rel(np.stack([c.host(t) for t in d]), want) <= TOL64
    pm = O.pressure_mesh(c.om)
    pinfo = tn.tn_mesh_info(c.m, 1)
    pmap = LayoutMap(pinfo, pm)
    mm = torch.zeros(pinfo["n_layout"], device="cuda", dtype=torch.float64)
    tn.tn_diag_pmass(c.m, 0, mm)
    want_m = O.diag_pressure_mass(c.om, O.prolongation(c.om, pm), c.eta)
    assert max_rel(pmap.from_layout(mm.cpu().numpy()), want_m) <= TOL64
    c.close()


@pytest.mark.parametrize("level,n_r", [(3, 9), (4, 17)])
def test_transfers_f64(tn, level, n_r):
    c = Case(tn, level, n_r, BCS["noslip/free"])
    cm = O.pressure_mesh(c.om)
    cinfo = tn.tn_mesh_info(c.m, 1)
    cmap = LayoutMap(cinfo, cm)
    Pt = O.prolongation(c.om, cm)
    Pc = O.boundary_projectors(cm, (O.NOSLIP, O.FREE))
    # scalar prolongation / restriction
    x = inputs.normal(cm.n_nodes, 30)
    f = torch.zeros(c.info["n_layout"], device="cuda", dtype=torch.float64)
    tn.tn_prolong(c.m, 0, [torch.tensor(cmap.to_layout(x), device="cuda")], [f])
    assert max_rel(c.host(f), Pt @ x) <= 1e-15
    z = inputs.normal(c.om.n_nodes, 31)
    g = torch.zeros(cinfo["n_layout"], device="cuda", dtype=torch.float64)
    tn.tn_restrict(c.m, 0, [c.dev(z)], [g])
    assert max_rel(cmap.from_layout(g.cpu().numpy()), Pt.T @ z) <= 1e-14
    # velocity with boundary projection
    v = inputs.normal((3, cm.n_nodes), 32)
    fv = c.zeros()
    tn.tn_prolong(c.m, 0, [torch.tensor(cmap.to_layout(v[i]), device="cuda") for i in range(3)], fv, apply_bc=True)
    want = O.project(c.P, np.stack([Pt @ v[i] for i in range(3)]))
    assert max_rel(np.stack([c.host(t) for t in fv]), want) <= 1e-15
    w = c.vec(33)
    gv = [torch.zeros(cinfo["n_layout"], device="cuda", dtype=torch.float64) for _ in range(3)]
    tn.tn_restrict(c.m, 0, [c.dev(w[i]) for i in range(3)], gv, apply_bc=True)
    want = O.project(Pc, np.stack([Pt.T @ w[i] for i in range(3)]))
    assert max_rel(np.stack([cmap.from_layout(t.cpu().numpy()) for t in gv]), want) <= 1e-14
    c.close()


def test_temperature_viscosity_and_buoyancy(tn):
    c = Case(tn, 4, 17)
    T = inputs.temperature(c.om.node_xyz(), 0.55, 1.0) + inputs.normal(c.om.n_nodes, 40, 0.01)
    Td = c.dev(T)
    tn.tn_set_temperature(c.m, Td, np.log(1e3), 0.9, 30.0)
    eta_want = viscosity(c.om, T, np.log(1e3), jump_r=0.9, jump_factor=30.0)
    got = torch.zeros(c.info["n_wedges"], device="cuda", dtype=torch.float64)
    tn.tn_get_viscosity(c.m, 0, got)
    assert np.abs(c.map.wedges_from_layout(got.cpu().numpy()) / eta_want - 1).max() <= 1e-14
    # coarse level = mean of the 8 children
    cm = ShellMesh(3, 9, 0.55, 1.0)
    cinfo = tn.tn_mesh_info(c.m, 1)
    cmap = LayoutMap(cinfo, cm)
    gc = torch.zeros(cinfo["n_wedges"], device="cuda", dtype=torch.float64)
    tn.tn_get_viscosity(c.m, 1, gc)
    assert np.abs(cmap.wedges_from_layout(gc.cpu().numpy()) / coarsen_viscosity(c.om, cm, eta_want) - 1).max() <= 1e-14
    f = c.zeros()
    tn.tn_buoyancy(c.m, Td, 7e3, f)
    want = buoyancy_rhs(c.om, T, 7e3, c.P)
    assert max_rel(np.stack([c.host(t) for t in f]), want) <= TOL64
    c.close()


def test_argument_errors(tn):
    c = Case(tn, 2, 5)
    u = [c.dev(c.vec(1)[i]) for i in range(3)]
    with pytest.raises(tn.TnError) as e:
        tn.tn_apply_A(c.m, 0, u, [u[0], c.zeros(1)[0], c.zeros(1)[0]])
    assert e.value.status == tn.TN_EINVAL
    with pytest.raises(tn.TnError):
        tn.tn_apply_A(c.m, 7, u, c.zeros())
    with pytest.raises(tn.TnError):
        tn.tn_apply_B(c.m, c.info["depth"] - 1, u, c.zeros(1)[0])
    m2 = tn.tn_mesh_create(2, 5, 0.55, 1.0)
    with pytest.raises(tn.TnError) as e:
        tn.tn_apply_A(m2, 0, u, c.zeros())
    assert e.value.status == tn.TN_ESTATE
    tn.tn_mesh_destroy(m2)
    c.close()


def test_operator_steps_host_rejects_bad_buffers(tn):
    """The binding checks every host buffer before the call: device, contiguity, one dtype and the
    layout size of its slot (the C side copies n_layout elements on trust)."""
    c = Case(tn, 3, 9, BCS["free/free"])
    n, npr = c.info["n_layout"], tn.tn_mesh_info(c.m, 1)["n_layout"]
    u = [torch.zeros(n, dtype=torch.float64) for _ in range(3)]
    p = torch.zeros(npr, dtype=torch.float64)
    good = [torch.zeros(m, dtype=torch.float64) for m in [n, n, n, npr, n, n, n, n, n, n]]
    tn.tn_operator_steps_host(c.m, [u], [p], [good])
    torch.cuda.synchronize()
    bad_cases = [
        [good[0][:-1]] + good[1:],                                   # undersized output
        good[:3] + [torch.zeros(n, dtype=torch.float64)] + good[4:],  # q slot with the velocity size
        [good[0].float()] + good[1:],                                # mixed dtypes
        [good[0].cuda()] + good[1:],                                 # device tensor as a host buffer
        [torch.zeros(2 * n, dtype=torch.float64)[::2]] + good[1:],   # not contiguous
    ]
    for outs in bad_cases:
        with pytest.raises(ValueError):
            tn.tn_operator_steps_host(c.m, [u], [p], [outs])
