"""Learned loop surrogate through the C ABI: the GPU network (tcgen05 GEMMs
with BF16 hi/lo operands, FP32 accumulation) against the FP64 oracle network
on the same parameters -- forward outputs and the gradient of the loss --;
training on exact loops; flows in which the surrogate gives the loops while
the exact judge accepts them, against the golden FP64 flow.

Bars: outputs within 1e-4 of the oracle's (relative max-norm; the BF16 hi/lo
operands keep ~16 mantissa bits, FP32 accumulation), gradients within 1e-3
per parameter block; a flow with the surrogate reaches Lambda_c within 1 % of
the FP64 oracle's (the bar of the reduced-precision paths) and classifies the
instability the same.
"""
import os

import numpy as np
import pytest

import workloads as W
from oracle import loops as olo
from oracle import mlp as omlp
from oracle.formfactors import Basis
from oracle.model import Problem
from tests.test_gpu_parity import dev, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as T
    from paper_1604_06296_gb300 import build
    build.build()
    assert T.cuda.is_available()
    return T


def rows(torch, n, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, (n, 5)).astype(np.float32)
    return x, dev(torch, x)


@pytest.mark.parametrize("n_out,width,depth,n", [(98, 256, 4, 300), (18, 64, 2, 128),
                                                 (242, 128, 3, 77)])
def test_forward_against_oracle(torch, n_out, width, depth, n):
    from paper_1604_06296_gb300 import Surrogate
    s = Surrogate(n_out, width, depth, seed=7)
    assert s.n_params == omlp.n_params(s.sizes)
    x, xd = rows(torch, n, 1)
    y = s.predict(xd).cpu().numpy()
    ref, _ = omlp.forward(s.params().astype(np.float64), s.sizes, x.astype(np.float64))
    err = rel(y, ref)
    print(f"n_out {n_out} width {width} depth {depth} rows {n}: forward rel err {err:.2e}")
    assert err < 1e-4
    s.close()


@pytest.mark.parametrize("n_out,width,depth,n", [(98, 256, 4, 512), (18, 64, 2, 200)])
def test_gradient_against_oracle(torch, n_out, width, depth, n):
    from paper_1604_06296_gb300 import Surrogate
    s = Surrogate(n_out, width, depth, seed=11)
    x, xd = rows(torch, n, 2)
    rng = np.random.default_rng(3)
    t = rng.standard_normal((n, n_out)).astype(np.float32)
    loss, g = s.loss_grad(xd, dev(torch, t))
    theta = s.params().astype(np.float64)
    L, gref = omlp.loss_and_grad(theta, s.sizes, x.astype(np.float64), t.astype(np.float64))
    print(f"loss {loss:.8g} vs {L:.8g}")
    assert abs(loss / L - 1) < 1e-5
    o = 0
    for i, (k, m) in enumerate(zip(s.sizes[:-1], s.sizes[1:])):
        for name, size in (("W", m * k), ("b", m)):
            err = rel(g[o:o + size], gref[o:o + size])
            print(f"layer {i} {name}: grad rel err {err:.2e}")
            assert err < 1e-3
            o += size
    assert o == len(g)
    s.close()


def cfg1_problem(tp):
    return Problem(1.0, tp, 4 * tp, 3.0, W.bonds_for_shells(1), 8, 8, 96, 96).check()


def make_solver(tp, precision="bf16x3"):
    from paper_1604_06296_gb300 import Solver
    return Solver(1.0, tp, 4 * tp, 3.0, W.bonds_for_shells(1), 8, 96, precision=precision)


TRAIN_TP = tuple(float(tp) for tp in np.linspace(-0.42, -0.02, 15) if abs(tp + 0.25) > 0.01)
HELD_OUT_TP = -0.25


@pytest.fixture(scope="module")
def trained(torch):
    """A surrogate trained on exact loops of cfg1-sized points at 14 t'
    (mu = 4 t'; t' = -0.25 held out), 200 scales log-uniform in [0.02, 12]."""
    from paper_1604_06296_gb300 import Surrogate
    npair = len(omlp.pair_list(Basis.from_bonds(W.bonds_for_shells(1)).parity))
    s = Surrogate(2 * npair, 256, 4, seed=5)
    rng = np.random.default_rng(9)
    xs, ts = [], []
    for tp in TRAIN_TP:
        sol = make_solver(tp)
        for lam in np.exp(rng.uniform(np.log(0.02), np.log(12.0), 200)):
            x, t = s.samples(sol, lam)
            xs.append(x.clone())
            ts.append(t.clone())
        sol.close()
    x = torch.cat(xs)
    t = torch.cat(ts)
    hist = s.train(x, t, epochs=150, batch=2048, lr=1e-3, seed=1)
    print(f"{x.shape[0]} samples; loss {hist[0]:.3e} -> {hist[-1]:.3e}")
    yield s, hist, x[:300].contiguous()
    s.close()


def test_samples_against_oracle(torch):
    from paper_1604_06296_gb300 import Surrogate
    p = cfg1_problem(-0.2)
    pairs = omlp.pair_list(Basis.from_bonds(W.bonds_for_shells(1)).parity)
    s = Surrogate(2 * len(pairs), 64, 1)
    sol = make_solver(-0.2, "fp64")
    x, t = s.samples(sol, 0.4)
    chi = np.stack(olo.chi_dot(p, 0.4))
    lv = p.l_values
    assert np.allclose(x.cpu().numpy(), omlp.features(lv[:, 0], lv[:, 1], 0.4, -0.2, -0.8),
                       atol=1e-6)
    assert rel(t.cpu().numpy(), omlp.targets(chi[0], chi[1], 0.4, pairs)) < 1e-6
    sol.close()
    s.close()


def test_trained_network_against_oracle(torch, trained):
    """Predictions of the trained network equal the oracle network on the
    same parameters and output standardisation."""
    s, _, x = trained
    shift, scale = s.scaling()
    assert np.all(scale > 0) and not np.all(scale == 1)
    y = s.predict(x).cpu().numpy()
    net, _ = omlp.forward(s.params().astype(np.float64), s.sizes, x.cpu().numpy())
    ref = net * scale + shift
    err = rel(y, ref)
    print(f"trained network vs oracle: {err:.2e}")
    assert err < 1e-4


def test_training_fits_held_out_point(torch, trained):
    s, hist, _ = trained
    assert hist[-1] < 0.01 * hist[0]
    p = cfg1_problem(HELD_OUT_TP)
    pairs = omlp.pair_list(Basis.from_bonds(W.bonds_for_shells(1)).parity)
    lv = p.l_values
    for lam in (5.0, 1.0, 0.2):
        x = omlp.features(lv[:, 0], lv[:, 1], lam, HELD_OUT_TP, 4 * HELD_OUT_TP)
        y = s.predict(dev(torch, x.astype(np.float32))).cpu().numpy()
        got = omlp.loops_from_outputs(y, lam, pairs, p.nff)
        err = rel(got, np.stack(olo.chi_dot(p, lam)))
        print(f"held-out t'={HELD_OUT_TP} lam={lam}: loops rel err {err:.2e}")
        assert err < 1e-2


def test_flow_with_surrogate_at_tol_1e2_keeps_lambda_c_with_fewer_exact_loops(torch, trained):
    """At judge tolerance 1e-2 the trained network serves most right-hand
    sides of the held-out flow: the flow computes fewer exact loop
    contractions (those of the RHS it serves not, plus the judgements) than
    the plain flow, and Lambda_c stays within 1 % of the oracle.  (At 1e-3,
    the tolerance of the learned production flows, the judge rejects this
    network at the start: its held-out error is above 1e-3.)"""
    import time
    s, _, _ = trained
    g = np.load(os.path.join(os.path.dirname(__file__), "golden", "flow_cfg1.npz"))
    cfg = W.config("cfg1")
    kw = dict(lambda0=cfg["lambda0"], lambda_min=cfg["lambda_min"], threshold=cfg["threshold"],
              rtol=1e-8, atol=1e-10, h0=0.05)
    sol = make_solver(HELD_OUT_TP)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, plain, _ = sol.flow(**kw)
    t_plain = time.perf_counter() - t0
    sol.attach_surrogate(s, judge_every=8, tol=1e-2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, res, _ = sol.flow(**kw)
    t_sur = time.perf_counter() - t0
    sol.close()
    dl = abs(res["lambda_c"] / float(g["lambda_c"]) - 1)
    print(f"with surrogate: Lambda_c {res['lambda_c']:.6g} ({dl:.2e} vs the oracle), "
          f"{res['n_rhs_surrogate']} of {res['n_rhs']} RHS from the surrogate, "
          f"{res['n_judges']} judgements, off below Lambda={res['lambda_surrogate_off']:.4g}; "
          f"plain flow {plain['n_rhs']} RHS in {t_plain:.3f} s, with surrogate {t_sur:.3f} s")
    assert res["diverged"] and dl < 1e-2
    assert (res["channel"], res["l_index"]) == (int(g["channel"]), int(g["l_index"]))
    assert res["n_rhs_surrogate"] > 0 and res["n_judges"] >= 1
    if res["lambda_surrogate_off"] > 0:
        assert res["lambda_surrogate_off"] > res["lambda_c"]
    exact = res["n_rhs"] - res["n_rhs_surrogate"] + res["n_judges"]
    print(f"exact loop contractions: {exact} with the surrogate, {plain['n_rhs']} without")
    assert exact < plain["n_rhs"]


def test_repeated_flows_with_accepted_surrogate(torch, trained):
    """Flows after one that switched from the surrogate to the exact loops
    (each flow captures its graphs afresh) give the same result."""
    s, _, _ = trained
    sol = make_solver(HELD_OUT_TP)
    sol.attach_surrogate(s, judge_every=8, tol=1e-2)
    kw = dict(threshold=50.0, rtol=1e-6, atol=1e-8, h0=0.05)
    _, a, _ = sol.flow(**kw)
    sol.attach_surrogate(s, judge_every=8, tol=1e-2)
    _, b, _ = sol.flow(**kw)
    _, c, _ = sol.flow(**kw)
    sol.close()
    assert a["n_rhs_surrogate"] > 0
    for r in (b, c):
        assert r["n_rhs_surrogate"] == a["n_rhs_surrogate"] and r["n_rhs"] == a["n_rhs"]
        assert abs(r["lambda_c"] / a["lambda_c"] - 1) < 1e-12


def test_judge_rejects_an_untrained_network(torch):
    from paper_1604_06296_gb300 import Surrogate
    npair = len(omlp.pair_list(Basis.from_bonds(W.bonds_for_shells(1)).parity))
    s = Surrogate(2 * npair, 64, 1, seed=3)
    sol = make_solver(-0.2)
    sol.attach_surrogate(s, judge_every=4, tol=1e-3)
    _, res, _ = sol.flow(threshold=50.0, rtol=1e-8, atol=1e-10, h0=0.05)
    assert res["n_rhs_surrogate"] == 0 and res["n_judges"] == 1
    assert res["lambda_surrogate_off"] == pytest.approx(10.0)
    assert res["diverged"]
    sol.close()
    s.close()
