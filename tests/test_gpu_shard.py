"""The loop contraction split over loop rows (the multi-GPU path) on one GPU:
two contexts of the same point compute the two halves of the rows, and the
right-hand side from the combined row loops equals the one-context
right-hand side; a split context refuses the calls that need every row."""
import numpy as np
import pytest

import workloads as W
from tests.conftest import make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as T
    from paper_1604_06296_gb300 import build
    build.build()
    assert T.cuda.is_available()
    return T


def _solver(shells, nc, nf, precision="bf16x3"):
    from paper_1604_06296_gb300 import Solver
    return Solver(1.0, -0.3, -1.2, 3.0, W.bonds_for_shells(shells), nc, nf, precision=precision)


@pytest.mark.parametrize("shells,nc,nf", [(2, 8, 32), (3, 12, 48)])
def test_row_halves_on_two_contexts_give_the_full_rhs(torch, shells, nc, nf):
    from paper_1604_06296_gb300 import _abi, _stream
    full = _solver(shells, nc, nf)
    y = torch.from_numpy(W.random_state(3, full.nl, full.nff, 0.3)).cuda()
    ref = full.rhs(0.4, y).cpu().numpy()
    a, b = _solver(shells, nc, nf), _solver(shells, nc, nf)
    nrow, npair = _abi.tufrg_row_info(a.ctx)
    assert (nrow, npair) == _abi.tufrg_row_info(full.ctx)
    half = nrow // 2
    _abi.tufrg_shard_rows(a.ctx, 0, half, _stream())
    _abi.tufrg_shard_rows(b.ctx, half, nrow, _stream())
    rows = torch.full((2, nrow, npair), float("nan"), dtype=torch.float64, device="cuda")
    _abi.tufrg_loop_rows(a.ctx, 0.4, rows.data_ptr(), _stream())
    _abi.tufrg_loop_rows(b.ctx, 0.4, rows.data_ptr(), _stream())
    assert torch.isfinite(rows).all()
    dy = a.empty(3)
    _abi.tufrg_rhs_from_rows(a.ctx, 0.4, rows.data_ptr(), y.data_ptr(), dy.data_ptr(), _stream())
    got = dy.cpu().numpy()
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-6
    for s in (full, a, b):
        s.close()


def test_split_context_refuses_whole_row_calls(torch):
    from paper_1604_06296_gb300 import TufrgError, _abi, _stream
    s = _solver(2, 8, 32)
    y = s.zeros(3)
    nrow, _ = _abi.tufrg_row_info(s.ctx)
    _abi.tufrg_shard_rows(s.ctx, 1, nrow, _stream())
    with pytest.raises(TufrgError) as e:
        s.rhs(0.5, y)
    assert e.value.status == -7
    with pytest.raises(TufrgError):
        _abi.tufrg_shard_rows(s.ctx, 3, 3, _stream())       # empty range
    _abi.tufrg_shard_rows(s.ctx, 0, nrow, _stream())        # whole range: usable again
    assert np.isfinite(s.rhs(0.5, y).cpu().numpy()).all()
    fp = _solver(2, 8, 32, precision="fp64")
    with pytest.raises(TufrgError):
        _abi.tufrg_shard_rows(fp.ctx, 0, 1, _stream())
    s.close()
    fp.close()


def test_sharded_solver_single_rank_equals_rhs(torch):
    from paper_1604_06296_gb300.sharded import ShardedSolver
    s = _solver(2, 8, 32)
    y = torch.from_numpy(W.random_state(5, s.nl, s.nff, 0.3)).cuda()
    ref = s.rhs(0.7, y).cpu().numpy()
    sh = ShardedSolver(_solver(2, 8, 32), 0, 1)
    got = sh.rhs(0.7, y).cpu().numpy()
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-6
    s.close()
    sh.s.close()


def test_wedge_flow_matches_the_oracle_flow_and_a_noncovariant_start_runs_in_full(torch):
    """A flow from zeros runs its projections and products at the rows'
    representatives (the state stays covariant); a flow from a state that
    is not covariant runs them at every l.  Both agree with the oracle's
    right-hand side of their states at the first stage."""
    from oracle import rhs as orhs
    prob = make_problem(shells=2, nc=8, nf=32, tp=-0.3, mu=-1.2)
    s = _solver(2, 8, 32, precision="fp64")
    for y0 in (np.zeros((3, s.nl, s.nff, s.nff)), W.random_state(9, s.nl, s.nff, 0.2)):
        yd = torch.from_numpy(y0).cuda()
        s.flow_init(yd, lambda0=2.0, lambda_min=1.0, rtol=1e-6, atol=1e-8, method="rk4",
                    h0=0.05)
        r = s.flow_step(1)
        y1 = s.flow_state()[0].cpu().numpy()
        # one RK4 step of the oracle from the same state (the library's step:
        # the interval ln 2 cut into round(ln 2 / h0) equal steps)
        steps = max(1, int(round(np.log(2.0 / 1.0) / 0.05)))
        h = -np.log(2.0) / steps
        def f(sv, yv):
            L = np.exp(sv)
            return L * orhs.rhs(prob, L, yv)
        s0 = np.log(2.0)
        k1 = f(s0, y0)
        k2 = f(s0 + h / 2, y0 + h / 2 * k1)
        k3 = f(s0 + h / 2, y0 + h / 2 * k2)
        k4 = f(s0 + h, y0 + h * k3)
        ref = y0 + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        assert np.abs(y1 - ref).max() / max(np.abs(ref).max(), 1e-300) < 1e-9
        assert r["n_accepted"] >= 1
    s.close()
