"""Tensor-core loop contraction (BF16x3 and 3xTF32 on tcgen05) against the FP64
oracle, through the C ABI.

Bar (reduced-precision paths): loops and couplings within 1e-4 relative
max-norm of the FP64 oracle, Lambda_c within 1 %.  The tests assert tighter
per-precision bounds derived from the split arithmetic: BF16x3 keeps ~16
mantissa bits per operand (products ~2^-16 relative), 3xTF32 ~22 bits;
FP32 accumulation in TMEM (the tensor core rounds the accumulator at every
MMA instruction, so the error grows with the chain length: K-blocks go
round-robin to up to four accumulator sets), FP64 across CTAs.  Measured on
GB300: ~2e-6 (BF16x3) and ~3e-7 / 6e-6 (3xTF32, short / production chains).
At the large size (Nff = 25) the BF16x3 loops are checked entry by entry
against the bound the split arithmetic gives, 4 * 2^-16 (1/Nf) sum |f f w|.
"""
import os

import numpy as np
import pytest

import workloads as W
from oracle import loops as olo
from oracle import rhs as orhs
from tests.test_gpu_parity import CASES, dev, make, rel

pytestmark = pytest.mark.gpu

BOUND = {"bf16x3": 1e-5, "3xtf32": 1e-5}


@pytest.fixture(scope="module")
def torch():
    import torch as T
    from paper_1604_06296_gb300 import build
    build.build()
    assert T.cuda.is_available()
    return T


def check_device(s):
    from paper_1604_06296_gb300 import _abi
    _abi.tufrg_check(s.ctx)


@pytest.mark.parametrize("precision", ["bf16x3", "3xtf32"])
@pytest.mark.parametrize("case", ["cfg1", "ragged", "rect"])
@pytest.mark.parametrize("lam", [5.0, 0.3, 0.02])
def test_loops_tensor_core(torch, precision, case, lam):
    s, p = make(case, torch, precision=precision)
    got = s.loops(lam).cpu().numpy()
    check_device(s)
    ref = np.stack(olo.chi_dot(p, lam))
    err = rel(got, ref)
    print(f"{precision} {case} lam={lam}: rel err {err:.2e}")
    assert err < BOUND[precision]


@pytest.mark.parametrize("case", ["cfg1", "rect", "cfg2", "nff25"])
def test_projections_mixed_precision(torch, case):
    # mixed-precision contexts project in FP32 arithmetic (FP64 state and result);
    # Nff = 25 takes the grouped form of the projections, the others the term form
    from oracle import projections as opj
    if case == "cfg2":
        c = W.config("cfg2")
        case = dict(shells=c["shells"], nc=c["nc"], nf=c["nf"], tp=-0.25, mu=-1.0, U=3.0)
    elif case == "nff25":
        case = dict(shells=5, nc=8, nf=16, tp=-0.3, mu=-1.2, U=3.5)
    s, p = make(case, torch, precision="bf16x3")
    y = W.random_state(21, p.nl, p.nff, 0.7)
    err = rel(s.project(dev(torch, y)).cpu().numpy(), opj.project(p, y))
    print(f"FP32 projections {p.nl} l: rel err {err:.2e}")
    assert err < 2e-6


def test_products_mixed_precision(torch):
    s, p = make("rect", torch, precision="bf16x3")
    V = W.random_state(3, p.nl, p.nff)
    chi = W.random_state(4, p.nl, p.nff)[:2]
    err = rel(s.products(dev(torch, V), dev(torch, chi)).cpu().numpy(),
              orhs.products(V, chi[0], chi[1]))
    print(f"FP32 products: rel err {err:.2e}")
    assert err < 1e-6


@pytest.mark.parametrize("precision", ["bf16x3", "3xtf32"])
def test_rhs_tensor_core(torch, precision):
    s, p = make("cfg1", torch, precision=precision)
    y = W.random_state(8, p.nl, p.nff, 0.5)
    got = s.rhs(0.7, dev(torch, y)).cpu().numpy()
    check_device(s)
    assert rel(got, orhs.rhs(p, 0.7, y)) < BOUND[precision]


@pytest.mark.parametrize("precision", ["bf16x3", "3xtf32"])
def test_production_size_loops_sampled(torch, precision):
    c = W.config("cfg2")
    case = dict(shells=c["shells"], nc=c["nc"], nf=c["nf"], tp=-0.25, mu=-1.0, U=3.0)
    s, p = make(case, torch, precision=precision)
    for lam in (1.0, 0.02):
        got = s.loops(lam).cpu().numpy()
        check_device(s)
        sel = [0, 37, 288, 300, 575]
        ref = np.stack(olo.chi_dot(p, lam, sel))
        err = rel(got[:, sel], ref)
        print(f"cfg2 {precision} lam={lam}: rel err {err:.2e}")
        assert err < BOUND[precision]
        # chi(-l) = chi(l) is exact by construction, chi symmetric
        assert np.array_equal(got, np.swapaxes(got, -1, -2))


def test_production_size_rhs_sampled_bf16x3(torch):
    """One whole right-hand side at the production size in the precision the
    bench times (tufrg_rhs: loops on the tensor cores, FP32 projections and
    products), sampled l against the oracle: the projections over all l, the
    loops and products at the sampled l."""
    from oracle import projections as opj
    c = W.config("cfg2")
    case = dict(shells=c["shells"], nc=c["nc"], nf=c["nf"], tp=-0.25, mu=-1.0, U=3.0)
    s, p = make(case, torch, precision="bf16x3")
    y = W.random_state(11, p.nl, p.nff, 0.5)
    got = s.rhs(0.4, dev(torch, y)).cpu().numpy()
    check_device(s)
    sel = [0, 37, 288, 300, 575]
    V = opj.project(p, y)
    chi = olo.chi_dot(p, 0.4, sel)
    ref = orhs.products(V[:, sel], chi[0], chi[1])
    err = rel(got[:, sel], ref)
    print(f"cfg2 bf16x3 RHS (sampled l): rel err {err:.2e}")
    assert err < BOUND["bf16x3"]


def test_large_size_loops_sampled_bf16x3(torch):
    """The large workload (coarse 48x48, Nff = 25: 169 allowed pairs, the
    widest N the two pipeline stages hold; fine 960x960) on the tensor cores,
    sampled l against the oracle: an interior l, its C4v image, a zone-boundary
    l and a general one."""
    c = W.config("cfg5")
    case = dict(shells=c["shells"], nc=c["nc"], nf=c["nf"], tp=c["tp"], mu=c["mu"], U=c["U"])
    s, p = make(case, torch, precision="bf16x3")
    got = s.loops(0.1).cpu().numpy()
    check_device(s)
    ix, iy = 30, 17
    sel = [ix * 48 + iy, iy * 48 + ix, 0 * 48 + 31, 1176]
    ref = np.stack(olo.chi_dot(p, 0.1, sel))
    err = rel(got[:, sel], ref)
    print(f"cfg5 bf16x3: rel err {err:.2e}")
    assert err < 1e-4  # the bar on couplings of the mixed-precision forms
    # Element-wise bound from the arithmetic.  The hi/lo split leaves a
    # relative residual of at most 2^-16 on each of W and F and drops
    # W_lo F_lo (at most 2^-16 |W F|); the FP32 chains and the compensated
    # combination add far less.  So |error_mn| <= 4 * 2^-16 * A_mn with
    # A_mn = (1/Nf) sum_p |f_m(p) f_n(p) w(p)|: with Nff = 25 the sums cancel
    # more than at Nff = 13, and the max-norm error relative to max |chi|
    # grows with them.
    P, F = p.p_values, np.abs(p.f_fine)
    for j, l in enumerate(sel):
        half = 0.5 * p.l_values[l]
        ws = olo.weights(p.xi(P[:, 0] + half[0], P[:, 1] + half[1]),
                         p.xi(P[:, 0] - half[0], P[:, 1] - half[1]), 0.1, True)
        for ch, w in enumerate(ws):
            A = (F * np.abs(w)) @ F.T / p.nf
            d = np.abs(got[ch, l] - ref[ch, j])
            print(f"  l={l} ch={ch}: max |error| / A = {np.max(d / A) * 2 ** 16:.2f} x 2^-16")
            assert np.all(d <= 2.0 ** -14 * A)
    assert np.array_equal(got, np.swapaxes(got, -1, -2))


@pytest.mark.parametrize("precision", ["bf16x3", "3xtf32"])
def test_flow_cfg1_tensor_core_against_oracle(torch, precision):
    g = np.load(os.path.join(os.path.dirname(__file__), "golden", "flow_cfg1.npz"))
    c = W.config("cfg1")
    s, p = make("cfg1", torch, precision=precision)
    y, res, states = s.flow(lambda0=c["lambda0"], lambda_min=c["lambda_min"],
                            threshold=c["threshold"], rtol=1e-8, atol=1e-10, h0=0.05,
                            checkpoints=list(g["checkpoints"]))
    check_device(s)
    dl = abs(res["lambda_c"] / float(g["lambda_c"]) - 1)
    print(f"{precision}: Lambda_c {res['lambda_c']:.8f} vs {float(g['lambda_c']):.8f} ({dl:.2e})")
    assert res["diverged"] and dl < 1e-2
    assert (res["channel"], res["l_index"]) == (int(g["channel"]), int(g["l_index"]))
    for i, lam in enumerate(g["checkpoints"]):
        e = rel(states[i].cpu().numpy(), g["y_checkpoints"][i])
        print(f"  checkpoint {lam}: rel err {e:.2e}")
        assert e < 1e-4


def test_flow_switches_to_fp64_near_the_divergence(torch):
    g = np.load(os.path.join(os.path.dirname(__file__), "golden", "flow_cfg1.npz"))
    c = W.config("cfg1")
    s, p = make("cfg1", torch, precision="bf16x3")
    y, res, _ = s.flow(lambda0=c["lambda0"], lambda_min=c["lambda_min"],
                       threshold=c["threshold"], rtol=1e-8, atol=1e-10, h0=0.05, fp64_above=5.0)
    check_device(s)
    dl = abs(res["lambda_c"] / float(g["lambda_c"]) - 1)
    print(f"bf16x3 -> fp64 above |B| = 5: Lambda_c rel err {dl:.2e}, "
          f"switch at Lambda = {res['lambda_switch']:.5f}")
    assert res["diverged"] and dl < 1e-4
    assert res["lambda_switch"] > res["lambda_c"]
    # the context's own precision is untouched for later calls
    got = s.loops(0.3).cpu().numpy()
    ref = np.stack(olo.chi_dot(p, 0.3))
    assert 1e-9 < rel(got, ref) < BOUND["bf16x3"]


def test_basis_too_large_for_tensor_core_path_rejected(torch):
    from paper_1604_06296_gb300 import TufrgError
    with pytest.raises(TufrgError) as e:
        make(dict(CASES["nff29"]), torch, precision="bf16x3")
    assert e.value.status == -1


@pytest.mark.parametrize("precision", ["bf16x3", "fp64"])
def test_profile_loops(torch, precision):
    s, p = make("cfg1", torch, precision=precision)
    k, g = s.profile_loops(0.4, 3)
    print(f"{precision}: contraction kernel {k * 1e3:.1f} us, loop stage {g * 1e3:.1f} us")
    assert 0 < k <= g
    # the profiled contractions are the real ones: the loops of the last are right
    ref = np.stack(olo.chi_dot(p, 0.4))
    assert rel(s.loops(0.4).cpu().numpy(), ref) < BOUND["bf16x3"]


def test_production_size_loops_every_l_bf16x3(torch):
    """Every l of one production-size loop call (BF16x3, the bench's
    precision): the rows cover every l through the point-group expansion,
    so a tile, queue-order or expansion error at any row shows here."""
    c = W.config("cfg2")
    case = dict(shells=c["shells"], nc=c["nc"], nf=c["nf"], tp=-0.25, mu=-1.0, U=3.0)
    s, p = make(case, torch, precision="bf16x3")
    got = s.loops(0.05).cpu().numpy()
    check_device(s)
    ref = np.stack(olo.chi_dot(p, 0.05))
    err = rel(got, ref)
    worst = np.abs(got - ref).max(axis=(0, 2, 3)) / np.abs(ref).max()
    print(f"cfg2 bf16x3 every l: rel err {err:.2e}, worst l {int(worst.argmax())}")
    assert err < BOUND["bf16x3"]


def test_large_size_rhs_sampled_bf16x3(torch):
    """One whole right-hand side at the large size (coarse 48x48, Nff = 25:
    the grouped projections, tufrg_rhs as the e2e line calls it) on 16
    sampled l: interior l, their C4v images, zone-boundary l of both kinds
    and (-pi, -pi); the oracle's projections over all l, loops and products
    at the sampled l."""
    from oracle import projections as opj
    c = W.config("cfg5")
    case = dict(shells=c["shells"], nc=c["nc"], nf=c["nf"], tp=c["tp"], mu=c["mu"], U=c["U"])
    s, p = make(case, torch, precision="bf16x3")
    y = W.random_state(12, p.nl, p.nff, 0.3)
    got = s.rhs(0.3, dev(torch, y)).cpu().numpy()
    check_device(s)
    n = p.ncx

    def L(ix, iy):
        return ix * n + iy
    sel = [L(30, 17), L(17, 30), L(18, 31), L(31, 18),      # an interior orbit
           L(24, 24), L(5, 40), L(40, 43), L(12, 12),       # l = 0, general, diagonal
           L(0, 31), L(0, 17), L(31, 0), L(17, 0),          # a boundary class
           L(0, 0), L(0, 24), L(24, 0), L(47, 1)]
    V = opj.project(p, y)
    chi = olo.chi_dot(p, 0.3, sel)
    ref = orhs.products(V[:, sel], chi[0], chi[1])
    err = rel(got[:, sel], ref)
    print(f"cfg5 bf16x3 RHS (16 sampled l): rel err {err:.2e}")
    assert err < 1e-4  # the bar on couplings of the mixed-precision forms
