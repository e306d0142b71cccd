"""Pins of the oracle's Fermi-surface-refined loop integration (Sec. 3: the
adaptive cubature's role; the refinement rule is a reading).

* every cell refined (any kappa large enough) = the uniform rule on s nf
  points per direction, to rounding (the sub-points tile the finer grid);
* no cell refined (Lambda >= Lambda_on, or kappa = 0) = the uniform rule;
* at a scale the coarse grid under-resolves, the refined loops are far
  closer to a much finer uniform grid than the unrefined ones;
* the refined loops keep the symmetry in (m, n), the parity selection of the
  particle-particle loop and C4v covariance (App. C) inside the zone;
* the flags: cells that straddle the Fermi surface are always refined.
"""
import numpy as np
import pytest

from oracle import formfactors as ffm
from oracle import loops as lp
from oracle import refine as rf
from tests.conftest import make_problem


@pytest.mark.parametrize("s", [3, 5])
def test_every_cell_refined_is_the_finer_uniform_grid(s):
    om = 0.2
    p = make_problem(shells=2, nc=4, nf=16, tp=-0.3)
    fine = make_problem(shells=2, nc=4, nf=16 * s, tp=-0.3)
    got = rf.chi_dot_refined(p, om, s=s, kappa=1e30)
    ref = lp.chi_dot(fine, om)
    for g, r in zip(got, ref):
        assert np.abs(g - r).max() <= 1e-13 * np.abs(r).max()


def test_no_cell_refined_is_the_uniform_grid():
    om = 0.05
    p = make_problem(shells=1, nc=4, nf=16)
    ref = lp.chi_dot(p, om)
    for got in (rf.chi_dot_refined(p, om, s=3, kappa=8.0, lam_on=0.04),
                rf.chi_dot_refined(p, om, s=3, kappa=0.0),
                rf.chi_dot_refined(p, om, s=1, kappa=8.0)):
        for g, r in zip(got, ref):
            assert np.array_equal(g, r)


def test_refinement_converges_where_the_grid_under_resolves():
    om = 0.1
    p = make_problem(shells=1, nc=4, nf=32, tp=-0.25)
    fine = make_problem(shells=1, nc=4, nf=32 * 15, tp=-0.25)
    ref = lp.chi_dot(fine, om)[0]
    sc = np.abs(ref).max()
    plain = np.abs(lp.chi_dot(p, om)[0] - ref).max() / sc
    refined = np.abs(rf.chi_dot_refined(p, om, s=5, kappa=10.0)[0] - ref).max() / sc
    assert plain > 1e-2
    assert refined < 0.05 * plain


def test_refined_loops_keep_the_symmetries():
    om = 0.08
    p = make_problem(shells=2, nc=6, nf=24, tp=-0.3)
    pp, ph = rf.chi_dot_refined(p, om, s=3, kappa=6.0)
    sc = max(np.abs(pp).max(), np.abs(ph).max())
    for X in (pp, ph):
        assert np.abs(X - np.swapaxes(X, 1, 2)).max() <= 1e-14 * sc
    par = p.basis.parity
    odd = (par[:, None] * par[None, :]) < 0
    assert np.abs(pp[:, odd]).max() <= 1e-14 * sc
    lu = p.l_units
    index = {tuple(u): i for i, u in enumerate(lu)}
    inner = np.nonzero(np.all(np.abs(lu) < p.ncx, axis=1))[0]
    for S in ffm.POINT_GROUP:
        C = p.basis.rep_matrix(S)
        for li in inner:
            lj = index[tuple(S @ lu[li])]
            for X in (pp, ph):
                assert np.abs(X[lj] - C @ X[li] @ C.T).max() <= 1e-13 * sc


def test_cells_on_the_fermi_surface_are_refined():
    om = 1e-3
    p = make_problem(shells=1, nc=4, nf=32, tp=-0.25)
    flags = rf.refine_flags(p, om, [0], 1.0, np.inf)[0]
    half = 0.5 * p.l_values[0]
    hx = np.pi / p.nfx
    q = p.p_values
    for sgn in (1, -1):
        c = [p.xi(q[:, 0] + dx + sgn * half[0], q[:, 1] + dy + sgn * half[1])
             for dx in (-hx, hx) for dy in (-hx, hx)]
        straddle = (np.min(c, axis=0) < 0) & (np.max(c, axis=0) > 0)
        assert straddle.any()
        assert flags[straddle].all()
