"""Batches through the C ABI: uneven phase-diagram points (own t', mu, U,
grids, bond shells, feedback) whose loops, right-hand sides and flows run as
multi-point launches, against the FP64 oracle point by point; batches against
single contexts; the tile autotuner.

Bar as for the tensor-core path: loops and right-hand sides within 1e-5
relative max-norm of the oracle (BF16x3), Lambda_c within 1 % of the FP64
oracle's golden flow.  A batch runs the same kernels as a single context with
another partition of the loop sum into work items, so the two agree to the
FP32 accumulation order.
"""
import os

import numpy as np
import pytest

import workloads as W
from oracle import loops as olo
from oracle import model as omodel
from oracle import rhs as orhs
from oracle.model import Problem
from tests.test_gpu_parity import dev, rel

pytestmark = pytest.mark.gpu

BOUND = 1e-5

SMALL = [
    dict(tp=-0.25, mu=-1.0, U=3.0, shells=1, nc=8, nf=96),
    dict(tp=-0.3, mu=-0.9, U=2.5, shells=2, nc=6, nf=36),
    dict(tp=-0.1, mu=-0.4, U=2.0, shells=3, nc=8, nf=48),
    dict(tp=-0.4, mu=-1.5, U=3.5, shells=4, nc=10, nf=80, feedback=False),
    dict(tp=0.0, mu=-0.2, U=2.2, shells=1, nc=4, nf=24),
]
LAMS = [2.0, 0.5, 0.05, 1.0, 0.01]


@pytest.fixture(scope="module")
def torch():
    import torch as T
    from paper_1604_06296_gb300 import build
    build.build()
    assert T.cuda.is_available()
    return T


def points(cases):
    return [dict(t=1.0, tp=c["tp"], mu=c["mu"], U=c["U"], bonds=W.bonds_for_shells(c["shells"]),
                 nc=c["nc"], nf=c["nf"], feedback=c.get("feedback", True)) for c in cases]


def problem(c):
    return Problem(1.0, c["tp"], c["mu"], c["U"], W.bonds_for_shells(c["shells"]), c["nc"],
                   c["nc"], c["nf"], c["nf"], feedback=c.get("feedback", True)).check()


@pytest.fixture(scope="module")
def small(torch):
    from paper_1604_06296_gb300 import Batch
    b = Batch(points(SMALL), precision="bf16x3")
    yield b
    b.close()


def test_batch_loops_each_point_against_oracle(torch, small):
    chi = small.loops(LAMS)
    small.check()
    for i, c in enumerate(SMALL):
        got = small.view(chi, i, loops=True).cpu().numpy()
        ref = np.stack(olo.chi_dot(problem(c), LAMS[i]))
        err = rel(got, ref)
        print(f"point {i} (Nff {got.shape[-1]}, Nl {got.shape[1]}) lam={LAMS[i]}: {err:.2e}")
        assert err < BOUND
        assert np.array_equal(got, np.swapaxes(got, -1, -2))


def test_batch_rhs_each_point_against_oracle(torch, small):
    y = small.zeros()
    ys = []
    for i, c in enumerate(SMALL):
        nl, nff = c["nc"] ** 2, W.n_ff_for_shells(c["shells"])
        yi = W.random_state(40 + i, nl, nff, 0.5)
        small.view(y, i).copy_(dev(torch, yi))
        ys.append(yi)
    dy = small.rhs(LAMS, y)
    small.check()
    for i, c in enumerate(SMALL):
        err = rel(small.view(dy, i).cpu().numpy(), orhs.rhs(problem(c), LAMS[i], ys[i]))
        print(f"point {i}: rhs rel err {err:.2e}")
        assert err < BOUND


def test_batch_equals_single_contexts(torch, small):
    from paper_1604_06296_gb300 import Solver
    chi = small.loops(LAMS)
    for i, c in enumerate(SMALL):
        s = Solver(1.0, c["tp"], c["mu"], c["U"], W.bonds_for_shells(c["shells"]), c["nc"],
                   c["nf"], precision="bf16x3", feedback=c.get("feedback", True))
        one = s.loops(LAMS[i]).cpu().numpy()
        s.close()
        err = rel(small.view(chi, i, loops=True).cpu().numpy(), one)
        print(f"point {i}: batch vs single context {err:.2e}")
        assert err < 1e-6


def test_batch_flow_against_golden_and_single_contexts(torch):
    from paper_1604_06296_gb300 import Batch, Solver
    g = np.load(os.path.join(os.path.dirname(__file__), "golden", "flow_cfg1.npz"))
    cfg = W.config("cfg1")
    cases = [SMALL[0], SMALL[1], dict(tp=0.0, mu=-1.8, U=1.0, shells=1, nc=4, nf=24)]
    b = Batch(points(cases), precision="bf16x3")
    kw = dict(lambda0=cfg["lambda0"], lambda_min=cfg["lambda_min"],
              threshold=cfg["threshold"], rtol=1e-8, atol=1e-10, h0=0.05)
    y, res, st = b.flow(**kw)
    b.check()
    assert st == [0, 0, 0]
    dl = abs(res[0]["lambda_c"] / float(g["lambda_c"]) - 1)
    print(f"cfg1 in a batch: Lambda_c {res[0]['lambda_c']:.8f} ({dl:.2e} vs the oracle)")
    assert res[0]["diverged"] and dl < 1e-2
    assert (res[0]["channel"], res[0]["l_index"]) == (int(g["channel"]), int(g["l_index"]))
    for i, c in enumerate(cases):
        s = Solver(1.0, c["tp"], c["mu"], c["U"], W.bonds_for_shells(c["shells"]), c["nc"],
                   c["nf"], precision="bf16x3")
        ys, rs, _ = s.flow(**kw)
        s.close()
        d = abs(res[i]["lambda_c"] / rs["lambda_c"] - 1)
        e = rel(b.view(y, i).cpu().numpy(), ys.cpu().numpy())
        print(f"point {i}: batch {res[i]['lambda_c']:.6g} ({res[i]['kind']}) vs single "
              f"{rs['lambda_c']:.6g} ({rs['kind']}): dLc {d:.1e}, state {e:.1e}, "
              f"steps {res[i]['n_accepted']}+{res[i]['n_rejected']} vs "
              f"{rs['n_accepted']}+{rs['n_rejected']}")
        assert res[i]["diverged"] == rs["diverged"] and res[i]["finished"]
        assert (res[i]["channel"], res[i]["l_index"]) == (rs["channel"], rs["l_index"])
        assert d < 5e-4 and e < 5e-3
    assert not res[2]["diverged"] and abs(res[2]["lambda_c"] / cfg["lambda_min"] - 1) < 1e-9
    # the points' skip flags of the flow are cleared for later calls
    chi = b.loops(0.3)
    ref = np.stack(olo.chi_dot(problem(cases[1]), 0.3))
    assert rel(b.view(chi, 1, loops=True).cpu().numpy(), ref) < BOUND
    b.close()


def test_autotune_keeps_results(torch, small):
    rep = small.autotune(0.5)
    print("batch autotune:", rep)
    assert len(rep["kbps"]) >= 3 and rep["kbps_default"] in rep["kbps"]
    assert rep["chosen"] == rep["kbps"][int(np.argmin(rep["ms"]))]
    chi = small.loops(LAMS)
    small.check()
    for i in (0, 3):
        ref = np.stack(olo.chi_dot(problem(SMALL[i]), LAMS[i]))
        assert rel(small.view(chi, i, loops=True).cpu().numpy(), ref) < BOUND


def test_single_context_autotune(torch):
    from tests.test_gpu_parity import make
    s, p = make("cfg1", torch, precision="3xtf32")
    rep = s.autotune(0.7)
    print("context autotune:", rep)
    assert rep["chosen"] == rep["kbps"][int(np.argmin(rep["ms"]))]
    assert rel(s.loops(0.7).cpu().numpy(), np.stack(olo.chi_dot(p, 0.7))) < BOUND
    y, res, _ = s.flow(threshold=50.0, rtol=1e-8, atol=1e-10, h0=0.05)
    assert res["diverged"]


def test_phase_diagram_scan_sampled(torch):
    """Seeded scan points at their own sizes (fine grids up to 480^2, Nff up
    to 21): loops of sampled l per point against the oracle."""
    from paper_1604_06296_gb300 import Batch, tufrg_mu_for_density
    pts = W.batch_points(6)
    for q in pts:
        q["mu"] = tufrg_mu_for_density(1.0, q["tp"], q["density"], q["nf"], q["nf"])
        assert abs(q["mu"] - omodel.mu_for_density(q["density"], 1.0, q["tp"], q["nf"],
                                                   q["nf"])) < 1e-9
        q["bonds"] = W.bonds_for_shells(q["shells"])
    b = Batch(pts, precision="bf16x3")
    lams = [0.5, 0.08, 1.5, 0.2, 0.03, 3.0]
    chi = b.loops(lams)
    b.check()
    for i, q in enumerate(pts):
        p = Problem(1.0, q["tp"], q["mu"], q["U"], q["bonds"], q["nc"], q["nc"], q["nf"],
                    q["nf"]).check()
        got = b.view(chi, i, loops=True).cpu().numpy()
        sel = [0, 1, p.nl // 2 + 3, p.nl - 1]
        err = rel(got[:, sel], np.stack(olo.chi_dot(p, lams[i], sel)))
        print(f"scan point {i} nc={q['nc']} nf={q['nf']} Nff={got.shape[-1]}: {err:.2e}")
        assert err < BOUND
    b.close()


def test_batch_rejects_mixed_or_fp64_precision(torch):
    from paper_1604_06296_gb300 import Batch, TufrgError
    with pytest.raises(TufrgError) as e:
        Batch(points(SMALL[:2]), precision="fp64")
    assert e.value.status == -1
    from paper_1604_06296_gb300 import _abi, make_params
    a, ka = make_params(1.0, -0.25, -1.0, 3.0, W.bonds_for_shells(1), 8, 96, "bf16x3")
    c, kc = make_params(1.0, -0.25, -1.0, 3.0, W.bonds_for_shells(1), 8, 96, "3xtf32")
    arr = (_abi.tufrg_params * 2)(a, c)
    with pytest.raises(TufrgError) as e:
        _abi.tufrg_batch_setup(arr)
    assert e.value.status == -1


def test_batch_profile_loops(torch, small):
    k, g = small.profile_loops(0.5, 2)
    assert 0 < k <= g
