"""Write vrms_config0.txt: first-solve V_rms of the level-l / (2^l + 1)-layer shell, l = 3, 4, 5, from
the oracle alone (oracle/ and the seeded input module; nothing from the CUDA path).

Problem (the config-0 family): r in [0.55, 1], free-slip on both surfaces, T = conductive profile
plus 0.01 cos(2 phi) P_3^2(cos theta) sin(pi (r - r_in) / (r_out - r_in)), viscosity exp(ln 10 (1/2 - T))
per wedge, Ra = 7e3, Boussinesq load Ra T r_hat (Eq. stokes).  Two loads: the full T, and the
lateral perturbation T' = T - T_conductive alone (the conductive part is a radial function, so its
load Ra T_c(r) r_hat is a gradient that pressure balances exactly in the continuum).  Solved by the
oracle's flexible GMRES to a relative residual of 1e-10; V_rms = sqrt(int |u|^2 dV / V) with the
lumped one-point quadrature (Sec. 8 reports V_rms beside Nu for the spherical benchmark runs).

    python tests/golden/make_vrms_config0.py      # about 20 minutes on one core
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.fields import viscosity  # noqa: E402
from oracle.mesh import ShellMesh  # noqa: E402
from oracle.solver import StokesSystem  # noqa: E402
from paper_2609_21633_gb300 import inputs  # noqa: E402

R_IN, R_OUT, RA = 0.55, 1.0, 7e3


def main():
    rows = []
    for level in (3, 4, 5):
        n_r = 2 ** level + 1
        m = ShellMesh(level, n_r, R_IN, R_OUT)
        xyz = m.node_xyz()
        T = inputs.temperature(xyz, R_IN, R_OUT)
        Tc = inputs.temperature(xyz, R_IN, R_OUT, amp=0.0)
        eta = viscosity(m, T, np.log(10.0))
        S = StokesSystem(m, eta)
        for load, Tl in (("full", T), ("perturbation", T - Tc)):
            b = S.rhs(Tl, RA)
            u, p, its = S.fgmres_solve(b, eta, tol=1e-10)
            rows.append((level, n_r, load, S.v_rms(u), S.residual(b, u, p), its))
            print(rows[-1], flush=True)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "vrms_config0.txt")
    with open(out, "w") as f:
        f.write("# First-solve V_rms of the config-0 shell family (written by make_vrms_config0.py from the oracle).\n")
        f.write("# level n_r load v_rms oracle_rel_residual fgmres_iterations\n")
        for level, n_r, load, v, res, its in rows:
            f.write(f"{level} {n_r} {load} {v:.15e} {res:.3e} {its}\n")


if __name__ == "__main__":
    main()
