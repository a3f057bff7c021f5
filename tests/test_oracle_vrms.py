"""Self-convergence of the first-solve V_rms (CPU only).

Sec. 8 reports V_rms beside Nu_top for the spherical-shell benchmark runs; here the first solve of
the config-0 shell family (levels 3, 4, 5 with 2^l + 1 node layers, free-slip, viscosity contrast
10, Ra = 7e3) is solved by the oracle and its V_rms must converge with second order (Richardson):
with the lateral temperature perturbation as the load the ratio of successive differences is
(V4 - V3) / (V5 - V4) = 4 for order 2.  With the full temperature the conductive part adds a radial
load Ra T_c(r) r_hat, a gradient that pressure balances exactly in the continuum; the discrete
balance is not exact, so the full-load V_rms carries a spurious flow at coarse levels, which must
vanish fast under refinement (the two V_rms approach each other).

The level-4 and level-5 solves take about 20 minutes, so their values are stored in
tests/golden/vrms_config0.txt by tests/golden/make_vrms_config0.py (oracle only); the level-3 value
is recomputed here and must equal the stored one."""
import os

import numpy as np

from oracle.fields import viscosity
from oracle.mesh import ShellMesh
from oracle.solver import StokesSystem
from paper_2609_21633_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "vrms_config0.txt")


def golden():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        level, n_r, load, v, res, its = line.split()
        assert float(res) <= 1e-10
        out[(int(level), load)] = float(v)
    return out


def test_vrms_converges_at_second_order():
    g = golden()
    v = [g[(l, "perturbation")] for l in (3, 4, 5)]
    ratio = (v[1] - v[0]) / (v[2] - v[1])
    order = np.log2(ratio)
    extrapolated = v[2] + (v[2] - v[1]) / 3.0
    print(f"V_rms {v}, ratio {ratio:.3f}, order {order:.2f}, Richardson limit {extrapolated:.6f}")
    assert 1.7 <= order <= 2.3, order
    # the spurious flow of the radial load vanishes fast: full and perturbation V_rms converge together
    gaps = [abs(g[(l, "full")] - g[(l, "perturbation")]) for l in (3, 4, 5)]
    assert gaps[1] < gaps[0] / 10 and gaps[2] < gaps[1] / 10, gaps
    assert abs(g[(5, "full")] - extrapolated) < 3 * abs(v[2] - v[1])


def test_stored_vrms_is_the_oracles():
    m = ShellMesh(3, 9, 0.55, 1.0)
    xyz = m.node_xyz()
    T = inputs.temperature(xyz, 0.55, 1.0)
    Tc = inputs.temperature(xyz, 0.55, 1.0, amp=0.0)
    eta = viscosity(m, T, np.log(10.0))
    S = StokesSystem(m, eta)
    b = S.rhs(T - Tc, 7e3)
    u, p, its = S.fgmres_solve(b, eta, tol=1e-10)
    assert S.residual(b, u, p) <= 1e-10
    assert abs(S.v_rms(u) / golden()[(3, "perturbation")] - 1) <= 1e-9
