"""Plain FP64 CPU oracle of the TUfRG Lambda-flow right-hand side.

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path and never calls it; the product path never calls it either.

The oracle follows the paper (Lichtenstein et al., "High-performance
functional renormalization group calculations for interacting fermions",
arXiv:1604.06296) step by step, in numpy float64:

* ``model``        -- dispersion (Eq. hubb-disp), grids, chemical potential.
* ``formfactors``  -- bond form factors adapted to C4v (Sec. 3, App. C).
* ``loops``        -- Omega-cutoff loops chi^pp, chi^ph and their scale
                      derivatives (Eq. chis) with the frequency integral done
                      in closed form.
* ``projections``  -- V^P, V^C, V^D (Eqs. proj_VP/VC/VD) by the literal
                      definition (Eqs. proj-P/C/D) and by a position-space
                      route (Eq. proj_pos) checked term by term against it.
* ``rhs``          -- the products of Eqs. matmul-P/C/D.
* ``flow``         -- Dormand-Prince 5(4) / RK4 integration of the flow,
                      critical scale and classification (Sec. 4).

Parity status of every function is stated in its module header.
"""
