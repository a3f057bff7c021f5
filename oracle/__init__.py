"""CPU FP64 oracle for the wedge Stokes operator of TERRA-NG (arxiv 2609.21633).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

It is a plain, slow, obviously-correct restatement of what the paper defines,
written with numpy / scipy library primitives and no blocking, fusion or
reordering beyond what the definitions state:

* ``mesh``      -- icosahedral base grid, 10 diamonds, recursive normalised
                   midpoint refinement, radial extrusion, implicit hex -> 2
                   wedge split, global numbering by coordinate de-duplication
                   (Sec. 2 "Grid and Parallelization", Fig. 1).
* ``element``   -- W1 wedge basis (Eq. wedgebasis), one-point quadrature at the
                   barycentre (Sec. 4, Eq. oneptenergy), element matrices of the
                   viscous block (Eq. elemmat) and of the divergence.
* ``operators`` -- global assembled (CSR) and matrix-free (element loop)
                   operators A, B, B^T, diag(A), diag(M_{1/eta}); iso-interpolation
                   between nested levels; free-slip / no-slip constraints.
* ``fields``    -- temperature -> per-wedge viscosity law and buoyancy RHS.
* ``solver``    -- reference Stokes solves and residuals (Sec. 7).

Where the paper is silent the readings are the ones stated in each function's
docstring; each is also listed in the repository's design notes.
"""
