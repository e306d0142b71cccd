"""Pins of the oracle's non-uniform, channel-specific bosonic meshes (Sec. 4;
the mesh construction and the quadrature of the source propagators are
readings).

* the uniform coarse mesh (m = 1) reproduces projections.project and rhs.rhs;
* a mesh refined everywhere is the uniform grid of nc m points: projections
  and right-hand side equal those of that grid, on coarse grids whose bond
  sums do not alias (so that both use the same term lists);
* each channel's quadrature weights sum to one; the refined cells carry m^2
  points; entries off a channel's mesh get no derivative;
* the loops at mesh points equal the grid loops where the points coincide.
"""
import numpy as np
import pytest

import workloads as W
from oracle import loops as lp
from oracle import mesh as ms
from oracle import projections as pj
from oracle import rhs as orhs
from tests.conftest import make_problem

PI = np.pi


def test_uniform_mesh_is_the_coarse_grid():
    prob = make_problem(shells=2, nc=6, nf=24, tp=-0.3, U=2.8)
    mesh = ms.refined_mesh(6, 1, [], [], 0.0)
    assert mesh.n == prob.nl
    assert np.allclose(mesh.l_values, prob.l_values, atol=1e-15)
    y = W.random_state(4, prob.nl, prob.nff, 0.3)
    ref = pj.project(prob, y)
    got = ms.project_mesh(prob, mesh, y)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    ref = orhs.rhs(prob, 0.2, y)
    got = ms.rhs_mesh(prob, mesh, 0.2, y)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("shells,nc,m", [(1, 10, 3), (2, 12, 3)])
def test_mesh_refined_everywhere_is_the_finer_grid(shells, nc, m):
    fine = make_problem(shells=shells, nc=nc * m, nf=2 * nc * m, tp=-0.3, U=2.8)
    coarse = make_problem(shells=shells, nc=nc, nf=2 * nc * m, tp=-0.3, U=2.8)
    for sig in pj.SIGNATURES.values():      # no aliasing: the same term lists
        a, b = pj._terms(coarse, sig)[0], pj._terms(fine, sig)[0]
        assert a.shape == b.shape and np.array_equal(a, b)
    mesh = ms.refined_mesh(nc, m, [(0.0, 0.0)], [(PI, PI)], 10.0)
    assert mesh.n == fine.nl
    order = np.lexsort((mesh.points[:, 1], mesh.points[:, 0]))
    idx = mesh.points[order, 0] * (nc * m) + mesh.points[order, 1]
    assert np.array_equal(idx, np.arange(fine.nl))
    y = W.random_state(6, fine.nl, fine.nff, 0.3)
    ym = np.empty_like(y)
    ym[:, order] = y
    ref = pj.project(fine, y)
    got = ms.project_mesh(coarse, mesh, ym)[:, order]
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    ref = orhs.rhs(fine, 0.15, y)
    got = ms.rhs_mesh(coarse, mesh, 0.15, ym)[:, order]
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_weights_points_and_masks():
    nc, m = 8, 3
    mesh = ms.refined_mesh(nc, m, [(0.0, 0.0)], [(PI, PI), (PI, 0.0), (0.0, PI)], 0.9)
    assert abs(mesh.w_p.sum() - 1.0) < 1e-14 and abs(mesh.w_cd.sum() - 1.0) < 1e-14
    fine_w = 1.0 / (nc * nc * m * m)
    n_fine_p = int(np.sum(np.isclose(mesh.w_p, fine_w)))
    n_coarse_p = int(np.sum(np.isclose(mesh.w_p, 1.0 / (nc * nc))))
    assert n_fine_p % (m * m) == 0 and n_fine_p // (m * m) + n_coarse_p == nc * nc
    assert 0 < n_fine_p and mesh.n > nc * nc
    prob = make_problem(shells=1, nc=nc, nf=2 * nc * m, tp=-0.3)
    y = W.random_state(8, mesh.n, prob.nff, 0.3)
    y[0][mesh.w_p == 0] = 0.0
    y[1:, mesh.w_cd == 0] = 0.0
    dy = ms.rhs_mesh(prob, mesh, 0.3, y)
    assert np.all(dy[0][mesh.w_p == 0] == 0.0)
    assert np.all(dy[1:, mesh.w_cd == 0] == 0.0)
    assert np.abs(dy[0][mesh.w_p > 0]).max() > 0 and np.abs(dy[1][mesh.w_cd > 0]).max() > 0


def test_loops_at_mesh_points_equal_grid_loops():
    prob = make_problem(shells=1, nc=4, nf=24, tp=-0.3)
    mesh = ms.refined_mesh(4, 3, [(0.0, 0.0)], [], 1.0)
    coarse = mesh.points % 3 == 0
    on = np.nonzero(coarse.all(axis=1))[0]
    pp, ph = ms.chi_dot_at(prob, 0.2, mesh.l_values[on])
    gi = (mesh.points[on, 0] // 3) * 4 + mesh.points[on, 1] // 3
    rpp, rph = lp.chi_dot(prob, 0.2, gi)
    assert np.abs(pp - rpp).max() <= 1e-14 * np.abs(rpp).max()
    assert np.abs(ph - rph).max() <= 1e-14 * np.abs(rph).max()


@pytest.mark.parametrize("nc,m,radius", [(8, 3, 0.9), (6, 5, 1.2), (24, 5, 0.6)])
def test_workload_mesh_generator_agrees_with_the_oracle(nc, m, radius):
    cp, ccd = [(0.0, 0.0)], [(PI, PI), (0.0, 0.0)]
    mesh = ms.refined_mesh(nc, m, cp, ccd, radius)
    pts, wp, wc = W.channel_mesh(nc, m, (cp, radius), (ccd, radius))
    assert np.array_equal(pts, mesh.points)
    assert np.abs(wp - mesh.w_p).max() <= 1e-18 and np.abs(wc - mesh.w_cd).max() <= 1e-18


def test_production_mesh_sizes():
    M = W.PRODUCTION_MESH
    pts, wp, wc = W.channel_mesh(M["nc"], M["m"], M["p"], M["cd"])
    # about the paper's 992 (P) and 6632 (C, D) points
    assert (wp > 0).sum() == 1080 and (wc > 0).sum() == 6384 and len(pts) == 6384
    assert abs(wp.sum() - 1) < 1e-13 and abs(wc.sum() - 1) < 1e-13


def test_symmetric_mesh_flow_is_covariant_where_the_mesh_is():
    """On a point-group symmetric mesh the flowing state, its projections and
    its right-hand side satisfy X(g l) = C^g X(l) C^g^T for every (l, g)
    whose image g l lies in the zone without a fold and is a mesh point with
    the same two weights (the relation the GPU's wedge rows use); images that
    need a fold do not (the half momentum moves by pi)."""
    from oracle import flow as fl
    from oracle import formfactors as ffm
    nc, m = 6, 3
    prob = make_problem(shells=1, nc=nc, nf=36, tp=-0.3, U=3.0)
    mesh = ms.refined_mesh(nc, m, [(0.0, 0.0)], [(PI, PI), (PI, 0.0), (0.0, PI)], 0.9)

    def f(s, y):
        lam = np.exp(s)
        return lam * ms.rhs_mesh(prob, mesh, lam, y)

    _, y = fl.rk4(f, np.log(4.0), np.zeros((3, mesh.n, prob.nff, prob.nff)),
                  np.log(0.5 / 4.0) / 3, 3)
    V = ms.project_mesh(prob, mesh, y)
    dy = ms.rhs_mesh(prob, mesh, 0.5, y)
    div, hd = nc * m, nc * m // 2
    at = {tuple(p): i for i, p in enumerate(mesh.points)}
    u = mesh.points - hd
    for X in (y, V, dy):
        sc = np.abs(X).max()
        assert sc > 0.05
        held, broken = 0, 0.0
        for S in ffm.POINT_GROUP:
            C = prob.basis.rep_matrix(S)
            for li in range(mesh.n):
                v = S @ u[li]
                lj = at.get(tuple((v + hd) % div))
                if lj is None or mesh.w_p[lj] != mesh.w_p[li] or mesh.w_cd[lj] != mesh.w_cd[li]:
                    continue
                err = np.abs(X[:, lj] - C @ X[:, li] @ C.T).max() / sc
                if np.all((v >= -hd) & (v < hd)):
                    assert err <= 1e-13
                    held += 1
                else:
                    broken = max(broken, err)
        assert held > 6 * mesh.n
        assert broken > 1e-7          # far above rounding: the fold is a real break


@pytest.mark.parametrize("feedback", [True, False])
def test_rhs_at_selected_points_equals_the_full_rhs(feedback):
    nc, m = 6, 3
    prob = make_problem(shells=2, nc=nc, nf=36, tp=-0.3, U=2.8, feedback=feedback)
    mesh = ms.refined_mesh(nc, m, [(0.0, 0.0)], [(PI, PI), (PI, 0.0)], 0.9)
    y = W.random_state(12, mesh.n, prob.nff, 0.3)
    y[0][mesh.w_p == 0] = 0.0
    y[1:, mesh.w_cd == 0] = 0.0
    full = ms.rhs_mesh(prob, mesh, 0.25, y)
    out = np.array([0, 3, mesh.n // 2, mesh.n - 1, 7])
    got = ms.rhs_mesh_at(prob, mesh, 0.25, y, out)
    assert np.abs(got - full[:, out]).max() <= 1e-13 * np.abs(full).max()
