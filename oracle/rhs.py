"""Right-hand side of the TUfRG flow (oracle; test infrastructure).

Eqs. (matmul-P/C/D), Sec. 2.4, for every bosonic momentum l:
    dP/dL =  V^P chi_dot^pp V^P
    dC/dL = -V^C chi_dot^ph V^C
    dD/dL =  2 V^D chi_dot^ph V^D - V^C chi_dot^ph V^D - V^D chi_dot^ph V^C
computed in the paper's three steps (Sec. 2.4): i) projections,
ii) loops, iii) products.

Pins: with projections switched off the flow reduces to single-channel
ladders with closed forms V^P = (V0^-1 + Dchi^pp)^-1, V^C = (V0^-1 + Dchi^ph)^-1,
2 V^D - V^C = (V0^-1 - Dchi^ph)^-1 (tests/test_oracle_flow.py).
"""
from __future__ import annotations

import numpy as np

from . import loops, projections


def products(V, chi_pp, chi_ph):
    """Step iii: Eqs. (matmul-P/C/D).  V = (V^P, V^C, V^D) [3][Nl][Nff][Nff]."""
    VP, VC, VD = V
    dP = VP @ chi_pp @ VP
    dC = -(VC @ chi_ph @ VC)
    dD = 2.0 * (VD @ chi_ph @ VD) - VC @ chi_ph @ VD - VD @ chi_ph @ VC
    return np.stack([dP, dC, dD])


def rhs(prob, lam, y):
    """dy/dLambda for y = (P, C, D) [3][Nl][Nff][Nff] at scale lam."""
    V = projections.project(prob, y)          # step i
    chi_pp, chi_ph = loops.chi_dot(prob, lam)  # step ii
    return products(V, chi_pp, chi_ph)        # step iii
