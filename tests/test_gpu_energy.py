"""Energy equation (Eq. energy) and the coupled Stokes-energy loop on the GPU against the oracle,
through the C ABI."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import energy as E
from oracle import operators as O
from oracle.fields import viscosity
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


class Shell:
    def __init__(self, tn, level, n_r):
        self.tn, self.om = tn, ShellMesh(level, n_r, R_IN, R_OUT)
        self.m = tn.tn_mesh_create(level, n_r, R_IN, R_OUT)
        self.info = tn.tn_mesh_info(self.m, 0)
        self.mp = LayoutMap(self.info, self.om)
        xyz = self.om.node_xyz()
        self.T = inputs.temperature(xyz, R_IN, R_OUT, amp=0.05)
        self.u = np.cross(np.array([0.2, -0.4, 1.0])[None, :], xyz).T * 30 + 5 * inputs.normal((3, self.om.n_nodes), 7)

    def dev(self, v):
        return torch.tensor(self.mp.to_layout(v), device="cuda")

    def host(self, t):
        return self.mp.from_layout(t.cpu().numpy())

    def close(self):
        self.tn.tn_mesh_destroy(self.m)


@pytest.mark.parametrize("level,n_r", [(3, 9), (5, 9)])
def test_energy_residual_matches_oracle(tn, level, n_r):
    """Halo tiles (level 3) and halo-free tiles (level 5); with and without the streamline term, and
    diffusion only."""
    s = Shell(tn, level, n_r)
    try:
        Td = s.dev(s.T)
        ud = [s.dev(s.u[c]) for c in range(3)]
        R = torch.zeros_like(Td)
        for supg in (True, False):
            K, C = E.assemble_energy(s.om, s.u, supg)
            tn.tn_energy_residual(s.m, Td, ud, R, supg)
            err = max_rel(s.host(R), (K + C) @ s.T)
            print(f"level {level} supg {supg}: max-rel {err:.2e}")
            assert err <= 1e-12, (supg, err)
        tn.tn_energy_residual(s.m, Td, None, R, True)
        assert max_rel(s.host(R), K @ s.T) <= 1e-12
    finally:
        s.close()


def test_heun_steps_diagnostics_and_stable_dt(tn):
    s = Shell(tn, 3, 9)
    try:
        # the stable substep: power iteration on M^-1 K against the exact largest eigenvalue
        K, _ = E.assemble_energy(s.om)
        inner = ~(s.om.boundary_nodes()[0] | s.om.boundary_nodes()[1])
        w = 1.0 / np.sqrt(E.lumped_mass(s.om)[inner])
        Ki = sp.diags(w) @ K[inner][:, inner] @ sp.diags(w)
        lam = spla.eigsh(Ki, k=1, which="LA", return_eigenvectors=False)[0]
        dt = tn.tn_energy_stable_dt(s.m)
        assert 1.5 / (1.1 * lam) * (1 - 1e-9) <= dt <= 1.5 / (1.1 * 0.8 * lam), (dt, lam)
        # Heun steps with a velocity
        Td = s.dev(s.T)
        ud = [s.dev(s.u[c]) for c in range(3)]
        tn.tn_energy_steps(s.m, Td, ud, dt, 6)
        want = E.heun_steps(s.om, s.T, s.u, dt, 6)
        assert np.abs(s.host(Td) - want).max() <= 1e-12 * np.abs(want).max()
        assert np.abs(s.host(Td) - s.T).max() > 1e-6          # it moved
        # diagnostics
        nu, vr = tn.tn_energy_diagnostics(s.m, Td, ud)
        r = np.linalg.norm(s.om.node_xyz(), axis=1)
        Tc = R_IN * (r - R_OUT) / (r * (R_IN - R_OUT))
        assert abs(nu / E.nusselt_top(s.om, want, Tc) - 1) <= 1e-12
        assert abs(vr / E.v_rms(s.om, s.u) - 1) <= 1e-12
    finally:
        s.close()


def test_convection_loop_matches_the_oracle(tn):
    """Three coupled steps at level 3 / 9 layers (Ra 1e5, contrast 100, fixed dt and substeps): every
    step's viscosity, load, Stokes solve (FP64, 1e-10) and Heun update replayed by the oracle; the
    temperatures agree to the solve tolerance, the per-step Nu_top and V_rms likewise."""
    level, n_r, Ra, Econ, dt, nsub, steps = 3, 9, 1e5, math.log(100.0), 2e-4, 4, 3
    s = Shell(tn, level, n_r)
    try:
        T0 = inputs.temperature(s.om.node_xyz(), R_IN, R_OUT, amp=0.05)
        Td = s.dev(T0)
        u = [torch.zeros_like(Td) for _ in range(3)]
        p = torch.zeros(tn.tn_mesh_info(s.m, 1)["n_layout"], device="cuda", dtype=torch.float64)
        opts = tn.tn_convection_default_opts(Ra=Ra, E=Econ, mode=tn.TN_SOLVE_F64, rtol=1e-10, dt=dt, substeps=nsub)
        stats = tn.tn_convection_steps(s.m, Td, u, p, steps, opts)
        T = T0.copy()
        r = np.linalg.norm(s.om.node_xyz(), axis=1)
        Tc = R_IN * (r - R_OUT) / (r * (R_IN - R_OUT))
        for k in range(steps):
            eta = viscosity(s.om, T, Econ)
            S = StokesSystem(s.om, eta)
            b = S.rhs(T, Ra)
            uo, po, _ = S.fgmres_solve(b, eta, tol=1e-11)
            nu, vr = E.nusselt_top(s.om, T, Tc), E.v_rms(s.om, uo)
            print(f"step {k}: GPU Nu {stats[k]['nu_top']:.9f} V_rms {stats[k]['v_rms']:.6f} "
                  f"({stats[k]['stokes_iterations']} its) / oracle Nu {nu:.9f} V_rms {vr:.6f}")
            assert abs(stats[k]["nu_top"] / nu - 1) <= 1e-9 and abs(stats[k]["v_rms"] / vr - 1) <= 1e-7
            T = E.heun_steps(s.om, T, uo, dt / nsub, nsub)
        err = np.abs(s.host(Td) - T).max()
        assert err <= 1e-7 * np.abs(T - T0).max() + 1e-12, err
        assert np.abs(T - T0).max() > 1e-4                    # the field evolved
    finally:
        s.close()


def test_stable_substep_scales_with_the_mesh(tn):
    """The diffusion bound dt ~ h^2: from level 3 / 9 to 5 / 33 to 7 / 129 layers the spacing halves
    twice per pair, so the stable substep shrinks by about 16 each time (the largest eigenvalue of
    M^-1 K reaches ~1e6 at level 7, where an unnormalised power iteration would overflow)."""
    dts = []
    for level, n_r in ((3, 9), (5, 33), (7, 129)):
        m = tn.tn_mesh_create(level, n_r, R_IN, R_OUT, max_levels=2)
        try:
            dts.append(tn.tn_energy_stable_dt(m))
        finally:
            tn.tn_mesh_destroy(m)
    ratios = [dts[0] / dts[1], dts[1] / dts[2]]
    print("stable substeps", dts, "ratios", ratios)
    assert all(8.0 <= q <= 32.0 for q in ratios), (dts, ratios)
