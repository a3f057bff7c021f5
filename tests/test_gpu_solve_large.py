"""The config-2 Stokes solves (level 6, 65 layers, viscosity contrast 1e4, 8.3 M DoFs) checked by
the oracle.  The oracle cannot assemble this system quickly, so it evaluates the residual
b - K x of the GPU solution row by row on sampled nodes: for a velocity node it applies its element
matrices (Eq. elemmat, one-point rule) and its B^T over exactly the wedges around the node, and its
buoyancy load over the same wedges; for a pressure node it applies B (Sec. 7) over every fine
wedge in the support of the node's basis function.  Those rows are complete, so they must equal
the GPU's own b - K x (its FP64 applies) there, and stay below the residual bound the solve reports
(|r_i| <= ||r||_2 <= rtol ||b||_2).  Modes: FP64, FP64 FGMRES with the FP32 preconditioner and BF16
viscosity, and FP32 inner solves inside FP64 refinement with BF16 viscosity."""
import math

import numpy as np
import pytest

from oracle import operators as O
from oracle.fields import buoyancy_rhs, viscosity
from oracle.mesh import ShellMesh
from paper_2609_21633_gb300 import inputs
from tests.layout import LayoutMap

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LEVEL, NR, R_IN, R_OUT = 6, 65, 0.55, 1.0
E, RA, RTOL = math.log(1e4), 7e3, 1e-8


@pytest.fixture(scope="module")
def tn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_21633_gb300 as tn
    tn.lib()
    return tn


@pytest.fixture(scope="module")
def shell():
    om = ShellMesh(LEVEL, NR, R_IN, R_OUT)
    pm = O.pressure_mesh(om)
    T = inputs.temperature(om.node_xyz(), R_IN, R_OUT)
    rng = np.random.default_rng(3)
    vel = rng.integers(0, om.n_nodes, 200)
    vel = np.concatenate([vel, [om.node_of_layout(0, 0, 0, 0), om.node_of_layout(5, 2 ** LEVEL, 2 ** LEVEL, NR - 1),
                                om.node_of_layout(3, 0, 17, 32), om.node_of_layout(7, 40, 2 ** LEVEL, 0)]])
    pres = rng.integers(0, pm.n_nodes, 60)
    return dict(om=om, pm=pm, T=T, Pp=O.prolongation(om, pm), vel=vel, pres=pres)


def first_layout(mp):
    """Layout index of one copy of every oracle node (indexed by node id)."""
    nodes, first = np.unique(mp.node, return_index=True)
    out = np.empty(nodes.size, dtype=np.int64)
    out[nodes] = mp.idx[first]
    return out


def oracle_rows(sh, u, p):
    """Oracle residual rows (b - K x) at the sampled velocity nodes (3, n_v) and pressure nodes."""
    om, pm, T, Pp = sh["om"], sh["pm"], sh["T"], sh["Pp"]
    P = O.boundary_projectors(om)
    Pm = O.projector_matrix(P)
    wv = om.wedges_of_nodes(sh["vel"])
    eta = np.zeros(om.n_wedges)
    eta[wv] = viscosity(om, T, E, wedges=wv)
    Ku = O.apply_A_constrained(om, eta, u, P, wedges=wv)
    BT = O.project(P, (O.assemble_B(om, Pp, wedges=wv).T @ p).reshape(3, -1))
    f = buoyancy_rhs(om, T, RA, P, wedges=wv)
    r_u = (f - Ku - BT)[:, sh["vel"]]
    # pressure rows: every fine wedge that touches a fine node in the support of the coarse basis
    Pc = Pp.tocsc()
    fine = np.unique(np.concatenate([Pc.indices[Pc.indptr[k]:Pc.indptr[k + 1]] for k in sh["pres"]]))
    wp = om.wedges_of_nodes(fine)
    Bu = O.assemble_B(om, Pp, wedges=wp) @ (Pm @ u.ravel())
    r_p = -Bu[sh["pres"]]
    return r_u, r_p, f[:, sh["vel"]]


@pytest.mark.parametrize("mode,eta_storage", [(0, 0), (2, 1), (1, 1)], ids=["fp64", "fp64_prec32_bf16", "mixed_bf16"])
def test_config2_solve_residual_checked_by_the_oracle(tn, shell, mode, eta_storage):
    om, pm = shell["om"], shell["pm"]
    m = tn.tn_mesh_create(LEVEL, NR, R_IN, R_OUT, eta_storage=eta_storage)
    try:
        info, pinfo = tn.tn_mesh_info(m, 0), tn.tn_mesh_info(m, 1)
        mp, pmap = LayoutMap(info, om), LayoutMap(pinfo, pm)
        Td = torch.tensor(mp.to_layout(shell["T"]), device="cuda")
        tn.tn_set_temperature(m, Td, E)
        f = [torch.zeros(info["n_layout"], device="cuda", dtype=torch.float64) for _ in range(3)]
        tn.tn_buoyancy(m, Td, RA, f)
        u = [torch.zeros_like(f[0]) for _ in range(3)]
        p = torch.zeros(pinfo["n_layout"], device="cuda", dtype=torch.float64)
        st = tn.tn_stokes_solve(m, f, None, u, p, tn.tn_solve_default_opts(mode=mode, rtol=RTOL))
        assert st["converged"] == 1 and st["rel_residual"] <= RTOL, st
        # the GPU's own b - K x with its FP64 applies
        Au = [torch.zeros_like(f[0]) for _ in range(3)]
        BTp = [torch.zeros_like(f[0]) for _ in range(3)]
        q = torch.zeros_like(p)
        tn.tn_apply_A(m, 0, u, Au)
        tn.tn_apply_BT(m, 0, p, BTp)
        tn.tn_apply_B(m, 0, u, q)
        r_gpu = [(f[c] - Au[c] - BTp[c]).cpu().numpy() for c in range(3)]
        rp_gpu = (-q).cpu().numpy()
        wu = torch.tensor(tn.tn_mesh_canonical_index(m, 0) == np.arange(info["n_layout"]), device="cuda",
                          dtype=torch.float64)
        wp = torch.tensor(tn.tn_mesh_canonical_index(m, 1) == np.arange(pinfo["n_layout"]), device="cuda",
                          dtype=torch.float64)
        bnorm = math.sqrt(sum(float(torch.dot(t * wu, t)) for t in f))
        rnorm = math.sqrt(sum(float(np.dot(r * wu.cpu().numpy(), r)) for r in r_gpu) +
                          float(np.dot(rp_gpu * wp.cpu().numpy(), rp_gpu)))
        assert abs(rnorm / bnorm - st["rel_residual"]) <= 1e-3 * st["rel_residual"], (rnorm / bnorm, st)
        # oracle rows at the sampled nodes
        u_o = np.stack([mp.from_layout(t.cpu().numpy()) for t in u])
        p_o = pmap.from_layout(p.cpu().numpy())
        r_u, r_p, f_o = oracle_rows(shell, u_o, p_o)
        vl = first_layout(mp)[shell["vel"]]
        pl = first_layout(pmap)[shell["pres"]]
        fmax = max(float(torch.abs(t).max()) for t in f)
        f_gpu = np.stack([t.cpu().numpy()[vl] for t in f])
        assert np.abs(f_gpu - f_o).max() <= 1e-12 * fmax
        ru_gpu = np.stack([r[vl] for r in r_gpu])
        err_u = np.abs(ru_gpu - r_u).max() / fmax
        err_p = np.abs(rp_gpu[pl] - r_p).max() / fmax
        print(f"mode {mode}: rel_residual {st['rel_residual']:.2e} ({st['iterations']} its); sampled oracle rows: "
              f"max |r_u| {np.abs(r_u).max() / bnorm:.2e} ||b||, max |r_p| {np.abs(r_p).max() / bnorm:.2e} ||b||; "
              f"oracle vs GPU rows {err_u:.1e} / {err_p:.1e} of max |f|")
        assert err_u <= 1e-10 and err_p <= 1e-10, (err_u, err_p)
        assert np.abs(r_u).max() <= RTOL * bnorm and np.abs(r_p).max() <= RTOL * bnorm
    finally:
        tn.tn_mesh_destroy(m)


def test_vrms_matches_the_oracle_and_keeps_converging(tn):
    """First-solve V_rms of the config-0 shell family driven by the lateral temperature perturbation
    (viscosity from the full T): the GPU FP64 solves at levels 3, 4, 5 reproduce the oracle's stored
    values (tests/golden/vrms_config0.txt), and level 6, beyond the oracle, continues the
    second-order self-convergence ((V5 - V4) / (V6 - V5) near 4; Sec. 8 reports V_rms)."""
    from tests.test_oracle_vrms import golden
    g = golden()
    v = {}
    for level in (3, 4, 5, 6):
        n_r = 2 ** level + 1
        om = ShellMesh(level, n_r, R_IN, R_OUT)
        m = tn.tn_mesh_create(level, n_r, R_IN, R_OUT)
        try:
            info, pinfo = tn.tn_mesh_info(m, 0), tn.tn_mesh_info(m, 1)
            mp = LayoutMap(info, om)
            xyz = om.node_xyz()
            T = inputs.temperature(xyz, R_IN, R_OUT)
            Tp = T - inputs.temperature(xyz, R_IN, R_OUT, amp=0.0)
            tn.tn_set_temperature(m, torch.tensor(mp.to_layout(T), device="cuda"), math.log(10.0))
            f = [torch.zeros(info["n_layout"], device="cuda", dtype=torch.float64) for _ in range(3)]
            tn.tn_buoyancy(m, torch.tensor(mp.to_layout(Tp), device="cuda"), RA, f)
            u = [torch.zeros_like(f[0]) for _ in range(3)]
            p = torch.zeros(pinfo["n_layout"], device="cuda", dtype=torch.float64)
            st = tn.tn_stokes_solve(m, f, None, u, p, tn.tn_solve_default_opts(rtol=1e-10), check=False)
            assert st["rel_residual"] <= 1e-9, st
            uo = np.stack([mp.from_layout(t.cpu().numpy()) for t in u])
            _, V = O.wedge_geometry(om)  # lumped one-point quadrature, as the oracle's v_rms
            mass = np.bincount(om.wedge_nodes().ravel(), weights=np.repeat(V / 6.0, 6), minlength=om.n_nodes)
            v[level] = float(np.sqrt(np.sum(mass * np.sum(uo ** 2, axis=0)) / mass.sum()))
            print(f"level {level}: V_rms {v[level]:.9f} ({st['iterations']} its, residual {st['rel_residual']:.1e})")
        finally:
            tn.tn_mesh_destroy(m)
        if level <= 5:
            assert abs(v[level] / g[(level, "perturbation")] - 1) <= 1e-7, (level, v[level])
    ratio = (v[5] - v[4]) / (v[6] - v[5])
    print(f"(V5 - V4) / (V6 - V5) = {ratio:.3f}, order {np.log2(ratio):.2f}")
    assert 3.0 <= ratio <= 5.3, ratio
