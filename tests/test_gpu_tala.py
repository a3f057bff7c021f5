"""TALA operators (Sec. 1, Eq. stokes and Eq. mass) on the GPU against the oracle, through the C ABI.

Reference profiles at the node radii: rho(r) = exp(1.5 (r_out - r)), alpha(r) = 1/2 + r.  The
divergence of Eq. (mass) is B applied to the nodal rho_k u_j, the load Ra rho alpha T' r_hat; the
saddle system is non-symmetric and FGMRES must still reach 1e-8, with the residual evaluated by
the oracle's assembled TALA system."""
import math

import numpy as np
import pytest

from oracle import operators as O
from oracle.fields import buoyancy_rhs, viscosity
from oracle.mesh import ShellMesh
from oracle.solver import StokesSystem
from paper_2609_21633_gb300 import inputs
from tests.layout import LayoutMap, max_rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

R_IN, R_OUT = 0.55, 1.0


@pytest.fixture(scope="module")
def tn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_21633_gb300 as tn
    tn.lib()
    return tn


def profiles(om):
    return np.exp(1.5 * (R_OUT - om.radii)), 0.5 + om.radii


@pytest.mark.parametrize("level,n_r", [(3, 9), (5, 9)])
def test_tala_divergence_and_buoyancy(tn, level, n_r):
    om = ShellMesh(level, n_r, R_IN, R_OUT)
    m = tn.tn_mesh_create(level, n_r, R_IN, R_OUT)
    try:
        info, pinfo = tn.tn_mesh_info(m, 0), tn.tn_mesh_info(m, 1)
        mp, pmap = LayoutMap(info, om), LayoutMap(pinfo, O.pressure_mesh(om))
        rho, alpha = profiles(om)
        tn.tn_set_viscosity(m, torch.tensor(mp.wedges_to_layout(inputs.lognormal_viscosity(om.n_wedges, 1)),
                                            device="cuda"))
        tn.tn_set_reference_state(m, rho, alpha)
        P = O.boundary_projectors(om)
        Pm = O.projector_matrix(P)
        Pp = O.prolongation(om, O.pressure_mesh(om))
        u = inputs.normal((3, om.n_nodes), 3)
        want = O.assemble_B(om, Pp, rho=rho) @ (Pm @ u.ravel())
        for dtype, tol in ((torch.float64, 1e-12), (torch.float32, 2e-5)):
            q = torch.zeros(pinfo["n_layout"], device="cuda", dtype=dtype)
            tn.tn_apply_B(m, 0, [torch.tensor(mp.to_layout(u[c]), device="cuda", dtype=dtype) for c in range(3)], q)
            err = max_rel(pmap.from_layout(q.double().cpu().numpy()), want)
            assert err <= tol, (dtype, err)
        T = inputs.temperature(om.node_xyz(), R_IN, R_OUT)
        f = [torch.zeros(info["n_layout"], device="cuda", dtype=torch.float64) for _ in range(3)]
        tn.tn_buoyancy(m, torch.tensor(mp.to_layout(T), device="cuda"), 7e3, f)
        want_f = buoyancy_rhs(om, T, 7e3, P, rho=rho, alpha=alpha)
        assert max_rel(np.stack([mp.from_layout(t.cpu().numpy()) for t in f]), want_f) <= 1e-12
        # removing the reference state restores the Boussinesq divergence
        tn.tn_set_reference_state(m, None)
        q = torch.zeros(pinfo["n_layout"], device="cuda", dtype=torch.float64)
        tn.tn_apply_B(m, 0, [torch.tensor(mp.to_layout(u[c]), device="cuda") for c in range(3)], q)
        assert max_rel(pmap.from_layout(q.cpu().numpy()), O.assemble_B(om, Pp) @ (Pm @ u.ravel())) <= 1e-12
        with pytest.raises(tn.TnError):
            tn.tn_set_reference_state(m, -rho, alpha)
    finally:
        tn.tn_mesh_destroy(m)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_tala_solve_reaches_1e8_by_the_oracle(tn, mode):
    level, n_r = 3, 9
    om = ShellMesh(level, n_r, R_IN, R_OUT)
    m = tn.tn_mesh_create(level, n_r, R_IN, R_OUT, hg_kappa=0.3)
    try:
        info, pinfo = tn.tn_mesh_info(m, 0), tn.tn_mesh_info(m, 1)
        mp, pmap = LayoutMap(info, om), LayoutMap(pinfo, O.pressure_mesh(om))
        xyz = om.node_xyz()
        T = inputs.temperature(xyz, R_IN, R_OUT)
        Tp = T - inputs.temperature(xyz, R_IN, R_OUT, amp=0.0)
        rho, alpha = profiles(om)
        tn.tn_set_temperature(m, torch.tensor(mp.to_layout(T), device="cuda"), math.log(100.0))
        tn.tn_set_reference_state(m, rho, alpha)
        f = [torch.zeros(info["n_layout"], device="cuda", dtype=torch.float64) for _ in range(3)]
        tn.tn_buoyancy(m, torch.tensor(mp.to_layout(Tp), device="cuda"), 1e5, f)
        u = [torch.zeros_like(f[0]) for _ in range(3)]
        p = torch.zeros(pinfo["n_layout"], device="cuda", dtype=torch.float64)
        st = tn.tn_stokes_solve(m, f, None, u, p, tn.tn_solve_default_opts(mode=mode))
        S = StokesSystem(om, viscosity(om, T, math.log(100.0)), kappa=0.3, rho=rho, alpha=alpha)
        b = S.rhs(Tp, 1e5)
        res = S.residual(b, np.stack([mp.from_layout(t.cpu().numpy()) for t in u]), pmap.from_layout(p.cpu().numpy()))
        print(f"TALA mode {mode}: {st['iterations']} iterations, GPU residual {st['rel_residual']:.2e}, oracle {res:.2e}")
        assert st["converged"] == 1 and res <= 1e-8 * (1 + 1e-3), (st, res)
        # a different system than the Boussinesq one: its residual with the plain divergence is large
        S0 = StokesSystem(om, viscosity(om, T, math.log(100.0)), kappa=0.3)
        assert S0.residual(b, np.stack([mp.from_layout(t.cpu().numpy()) for t in u]),
                           pmap.from_layout(p.cpu().numpy())) > 1e-6
    finally:
        tn.tn_mesh_destroy(m)
