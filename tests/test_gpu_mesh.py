"""Non-uniform, channel-specific bosonic meshes on the GPU (Sec. 4) against
the oracle's mesh functions, through the C ABI: the loops at the mesh points,
the projections with the source channels' quadratures, the right-hand side
with each channel's derivative confined to its own mesh, a fixed-step flow,
the uniform mesh against a coarse-grid context, and invalid meshes."""
import numpy as np
import pytest

import workloads as W
from tests.conftest import make_problem

pytestmark = pytest.mark.gpu

PI = np.pi
BOUND = {"fp64": 1e-10, "bf16x3": 2e-5}
T, TP, MU, U = 1.0, -0.3, -1.2, 3.0


@pytest.fixture(scope="module")
def torch():
    import torch as t
    from paper_1604_06296_gb300 import build
    build.build()
    return t


def _mesh(nc, m, radius=0.9):
    from oracle import mesh as ms
    return ms.refined_mesh(nc, m, [(0.0, 0.0)], [(-PI, -PI), (-PI, 0.0), (0.0, -PI)], radius)


def _pair(shells, nc, m, nf, prec, feedback=True, radius=0.9):
    from paper_1604_06296_gb300 import Solver
    mesh = _mesh(nc, m, radius)
    prob = make_problem(shells=shells, nc=nc, nf=nf, t=T, tp=TP, mu=MU, U=U, feedback=feedback)
    sv = Solver(T, TP, MU, U, W.bonds_for_shells(shells), nc, nf, precision=prec,
                feedback=feedback, mesh=(m, mesh.points, mesh.w_p, mesh.w_cd))
    assert sv.nl == mesh.n
    return prob, mesh, sv


def _state(seed, mesh, nff, amp=0.3):
    y = W.random_state(seed, mesh.n, nff, amp)
    y[0][mesh.w_p == 0] = 0.0
    y[1:, mesh.w_cd == 0] = 0.0
    return y


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


CASES = [  # shells, nc, m, nf, precision
    (1, 6, 3, 36, "fp64"),
    (2, 8, 3, 48, "fp64"),
    (1, 4, 5, 40, "fp64"),
    (1, 8, 3, 48, "bf16x3"),
    (2, 6, 3, 36, "bf16x3"),
]


@pytest.mark.parametrize("shells,nc,m,nf,prec", CASES)
def test_mesh_loops_match_oracle(torch, shells, nc, m, nf, prec):
    from oracle import mesh as ms
    prob, mesh, sv = _pair(shells, nc, m, nf, prec)
    assert mesh.n > nc * nc
    for om in (0.9, 0.08):
        got = sv.loops(om).cpu().numpy()
        ref = np.stack(ms.chi_dot_at(prob, om, mesh.l_values))
        for ch in range(2):
            assert _rel(got[ch], ref[ch]) <= BOUND[prec]
    sv.close()


@pytest.mark.parametrize("shells,nc,m,nf,prec", CASES)
def test_mesh_projections_match_oracle(torch, shells, nc, m, nf, prec):
    from oracle import mesh as ms
    prob, mesh, sv = _pair(shells, nc, m, nf, prec)
    for seed in (3, 4):
        y = _state(seed, mesh, prob.nff)
        got = sv.project(torch.from_numpy(y).cuda()).cpu().numpy()
        ref = ms.project_mesh(prob, mesh, y)
        assert _rel(got, ref) <= BOUND[prec]
    sv.close()


@pytest.mark.parametrize("shells,nc,m,nf,prec", CASES)
def test_mesh_rhs_matches_oracle_and_stays_on_each_mesh(torch, shells, nc, m, nf, prec):
    from oracle import mesh as ms
    prob, mesh, sv = _pair(shells, nc, m, nf, prec)
    y = _state(5, mesh, prob.nff)
    got = sv.rhs(0.15, torch.from_numpy(y).cuda()).cpu().numpy()
    ref = ms.rhs_mesh(prob, mesh, 0.15, y)
    assert _rel(got, ref) <= BOUND[prec]
    assert np.all(got[0][mesh.w_p == 0] == 0.0)
    assert np.all(got[1:, mesh.w_cd == 0] == 0.0)
    assert np.abs(got[0][mesh.w_p > 0]).max() > 0 and np.abs(got[1][mesh.w_cd > 0]).max() > 0
    sv.close()


def test_mesh_without_feedback(torch):
    from oracle import mesh as ms
    prob, mesh, sv = _pair(1, 6, 3, 36, "fp64", feedback=False)
    y = _state(7, mesh, prob.nff)
    got = sv.rhs(0.2, torch.from_numpy(y).cuda()).cpu().numpy()
    assert _rel(got, ms.rhs_mesh(prob, mesh, 0.2, y)) <= 1e-10
    sv.close()


def test_uniform_mesh_equals_the_coarse_grid_context(torch):
    from paper_1604_06296_gb300 import Solver
    nc, nf = 8, 32
    mesh = _mesh(nc, 1, radius=0.0)
    assert mesh.n == nc * nc
    sv_m = Solver(T, TP, MU, U, W.bonds_for_shells(2), nc, nf,
                  mesh=(1, mesh.points, mesh.w_p, mesh.w_cd))
    sv_c = Solver(T, TP, MU, U, W.bonds_for_shells(2), nc, nf)
    y = torch.from_numpy(W.random_state(11, nc * nc, sv_c.nff, 0.3)).cuda()
    a = sv_m.rhs(0.3, y).cpu().numpy()
    b = sv_c.rhs(0.3, y).cpu().numpy()
    assert _rel(a, b) <= 1e-12
    sv_m.close()
    sv_c.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_mesh_rk4_flow_matches_oracle(torch, prec):
    from oracle import flow as ofl
    from oracle import mesh as ms
    prob, mesh, sv = _pair(1, 6, 3, 36, prec)
    lam0, lam1, steps = 4.0, 0.8, 4
    h = (np.log(lam1) - np.log(lam0)) / steps
    y, res, _ = sv.flow(lambda0=lam0, lambda_min=lam1, threshold=1e9, h0=abs(h), method="rk4")

    def f(s, yy):
        lam = np.exp(s)
        return lam * ms.rhs_mesh(prob, mesh, lam, yy)

    _, yref = ofl.rk4(f, np.log(lam0), np.zeros((3, mesh.n, prob.nff, prob.nff)), h, steps)
    got = y.cpu().numpy()
    assert res["n_accepted"] == steps and not res["diverged"]
    assert _rel(got, yref) <= (1e-9 if prec == "fp64" else 1e-4)
    assert np.all(got[0][mesh.w_p == 0] == 0.0)
    assert np.all(got[1:, mesh.w_cd == 0] == 0.0)
    sv.close()


def test_mesh_dopri5_flow_stays_on_each_mesh(torch):
    prob, mesh, sv = _pair(1, 6, 3, 36, "bf16x3")
    y, res, _ = sv.flow(lambda0=10.0, lambda_min=0.05, threshold=30.0, rtol=1e-6, atol=1e-8,
                        max_steps=400)
    got = y.cpu().numpy()
    assert np.isfinite(got).all() and res["n_accepted"] > 0
    assert np.all(got[0][mesh.w_p == 0] == 0.0)
    assert np.all(got[1:, mesh.w_cd == 0] == 0.0)
    sv.close()


def test_invalid_meshes_and_refused_features(torch):
    from paper_1604_06296_gb300 import Solver, TufrgError
    nc, m, nf = 6, 3, 36
    mesh = _mesh(nc, m)
    b = W.bonds_for_shells(1)
    pts, wp, wc = mesh.points, mesh.w_p, mesh.w_cd

    def bad(m_, pts_, wp_, wc_, nf_=nf, ncy=None):
        with pytest.raises(TufrgError) as e:
            Solver(T, TP, MU, U, b, nc, nf_, ncy=ncy, mesh=(m_, pts_, wp_, wc_))
        assert e.value.status == -1

    bad(2, pts, wp, wc)                                  # even m
    bad(m, pts, wp, wc, nf_=24)                          # nf not a multiple of 2 nc m
    bad(m, pts, wp, wc, ncy=8)                           # rectangular coarse grid
    taken = {tuple(q) for q in pts.tolist()}
    free = next((x, y) for x in range(nc * m) for y in range(nc * m) if (x, y) not in taken)
    bad(m, np.vstack([pts, [free]]), np.append(wp, 0.0), np.append(wc, 0.0))  # in no mesh
    dup = pts.copy()
    dup[1] = dup[0]
    bad(m, dup, wp, wc)                                  # a point twice
    out = pts.copy()
    out[0, 0] = nc * m
    bad(m, out, wp, wc)                                  # outside the lattice
    bad(m, pts, 2 * wp, wc)                              # weights not summing to one
    neg = wc.copy()
    neg[np.argmax(neg)] *= -1
    bad(m, pts, wp, neg)                                 # negative weight
    sv = Solver(T, TP, MU, U, b, nc, nf, precision="bf16x3", mesh=(m, pts, wp, wc))
    from paper_1604_06296_gb300 import _abi
    for call in (lambda: sv.set_refinement(s=3), lambda: sv.atensor_build(),
                 lambda: _abi.tufrg_shard_rows(sv.ctx, 0, 1)):
        with pytest.raises(TufrgError) as e:
            call()
        assert e.value.status == -7
    sv.close()


def _mesh_classes(nc, m, pts, wp, wc):
    """Loop rows of a mesh: classes of l under the point-group elements whose
    image lies in the zone without a fold and is a mesh point with the same
    two weights (union-find over the pairs)."""
    div, hd = nc * m, nc * m // 2
    at = {tuple(p): i for i, p in enumerate(np.asarray(pts).tolist())}
    parent = list(range(len(pts)))

    def find(i):
        while parent[i] != i:
            parent[i] = parent[parent[i]]
            i = parent[i]
        return i

    group = [((1, 0), (0, 1)), ((0, -1), (1, 0)), ((-1, 0), (0, -1)), ((0, 1), (-1, 0)),
             ((1, 0), (0, -1)), ((-1, 0), (0, 1)), ((0, 1), (1, 0)), ((0, -1), (-1, 0))]
    for i, (jx, jy) in enumerate(np.asarray(pts).tolist()):
        ux, uy = jx - hd, jy - hd
        for (a, b), (c, d) in group:
            vx, vy = a * ux + b * uy, c * ux + d * uy
            if not (-hd <= vx < hd and -hd <= vy < hd):
                continue
            j = at.get((vx + hd, vy + hd))
            if j is not None and wp[j] == wp[i] and wc[j] == wc[i]:
                parent[find(j)] = find(i)
    return len({find(i) for i in range(len(pts))})


def test_symmetric_meshes_get_point_group_rows(torch):
    from paper_1604_06296_gb300 import Solver, _abi
    for nc, m, nf, radius in ((6, 3, 36, 0.9), (8, 3, 48, 1.3), (4, 5, 40, 0.9)):
        mesh = _mesh(nc, m, radius)
        sv = Solver(T, TP, MU, U, W.bonds_for_shells(1), nc, nf,
                    mesh=(m, mesh.points, mesh.w_p, mesh.w_cd))
        nrow, _ = _abi.tufrg_row_info(sv.ctx)
        assert nrow == _mesh_classes(nc, m, mesh.points, mesh.w_p, mesh.w_cd)
        assert 3 * nrow < mesh.n
        sv.close()
    M = W.PRODUCTION_MESH
    pts, wp, wc = W.channel_mesh(M["nc"], M["m"], M["p"], M["cd"])
    sv = Solver(T, TP, MU, U, W.bonds_for_shells(3), M["nc"], 480, precision="bf16x3",
                mesh=(M["m"], pts, wp, wc))
    nrow, _ = _abi.tufrg_row_info(sv.ctx)
    assert nrow == _mesh_classes(M["nc"], M["m"], pts, wp, wc) and 6 * nrow < len(pts)
    sv.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_mesh_rk4_flow_from_a_non_covariant_state(torch, prec):
    """A random start is not covariant: the flow runs on every mesh point."""
    from oracle import flow as ofl
    from oracle import mesh as ms
    prob, mesh, sv = _pair(1, 6, 3, 36, prec)
    y0 = _state(13, mesh, prob.nff, 0.2)
    lam0, lam1, steps = 4.0, 1.0, 3
    h = (np.log(lam1) - np.log(lam0)) / steps
    y, res, _ = sv.flow(torch.from_numpy(y0).cuda(), lambda0=lam0, lambda_min=lam1,
                        threshold=1e9, h0=abs(h), method="rk4")

    def f(s, yy):
        lam = np.exp(s)
        return lam * ms.rhs_mesh(prob, mesh, lam, yy)

    _, yref = ofl.rk4(f, np.log(lam0), y0, h, steps)
    assert res["n_accepted"] == steps
    assert _rel(y.cpu().numpy(), yref) <= (1e-9 if prec == "fp64" else 1e-4)
    sv.close()


@pytest.mark.parametrize("prec", ["bf16x3", "fp64"])
def test_production_mesh_rhs_sampled(torch, prec):
    """The production-sized meshes (mesh_P 1080, mesh_CD 6384 points, coarse
    24x24, Nff 13, fine 480x480): one right-hand side on every mesh point,
    checked against the oracle at 12 points spread over the mesh (zone
    boundary, refined and coarse cells, points off mesh_P).  BF16x3 runs the
    key quadrature on the tensor cores, FP64 on the CUDA cores."""
    from oracle import mesh as ms
    from paper_1604_06296_gb300 import Solver
    c = W.config("cfg2")
    M = W.PRODUCTION_MESH
    pts, wp, wc = W.channel_mesh(M["nc"], M["m"], M["p"], M["cd"])
    mesh = ms.Mesh(M["nc"], M["m"], pts.astype(np.int64), wp, wc)
    tp = c["tp"]
    prob = make_problem(shells=c["shells"], nc=c["nc"], nf=c["nf"], t=c["t"], tp=tp, mu=4 * tp,
                        U=c["U"])
    sv = Solver(c["t"], tp, 4 * tp, c["U"], W.bonds_for_shells(c["shells"]), c["nc"], c["nf"],
                precision=prec, mesh=(M["m"], pts, wp, wc))
    y = W.random_state(21, mesh.n, prob.nff, 0.1)
    y[0][wp == 0] = 0.0
    y[1:, wc == 0] = 0.0
    got = sv.rhs(0.3, torch.from_numpy(y).cuda()).cpu().numpy()
    out = np.linspace(0, mesh.n - 1, 12).astype(int)
    assert (wp[out] == 0).any() and (wp[out] > 0).any()
    ref = ms.rhs_mesh_at(prob, mesh, 0.3, y, out)
    assert _rel(got[:, out], ref) <= (1e-10 if prec == "fp64" else 2e-5)
    sv.close()
