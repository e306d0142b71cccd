"""The C ABI library builds, loads and exports every symbol of include/tufrg.h;
its host-side logic (form-factor basis, filling, argument validation) agrees
with the oracle.  No GPU work is issued here."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads as W
from oracle import formfactors as ffm
from oracle import model

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def abi():
    from paper_1604_06296_gb300 import _abi, build
    build.build()
    return _abi


def header_functions():
    src = open(os.path.join(ROOT, "include", "tufrg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tufrg_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(abi):
    names = header_functions()
    assert len(names) >= 10
    L = ctypes.CDLL(abi.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(abi.SIGNATURES)


@pytest.mark.parametrize("shells", range(7))
def test_basis_matches_oracle(abi, shells):
    bonds = W.bonds_for_shells(shells)
    rng = np.random.default_rng(shells)
    k = rng.uniform(-np.pi, np.pi, (2, 200))
    got = abi.tufrg_eval_formfactors(bonds, k[0], k[1])
    ref = ffm.Basis.from_bonds(bonds).values(k[0], k[1])
    assert got.shape == ref.shape
    assert np.abs(got - ref).max() < 1e-13


def test_basis_is_independent_of_bond_order(abi):
    bonds = W.bonds_for_shells(4)
    perm = np.random.default_rng(0).permutation(len(bonds))
    k = np.linspace(-3, 3, 17)
    a = abi.tufrg_eval_formfactors(bonds, k, k[::-1])
    b = abi.tufrg_eval_formfactors(bonds[perm], k, k[::-1])
    assert np.array_equal(a, b)


@pytest.mark.parametrize("bad", [
    np.array([[0, 0], [1, 0], [0, 1], [-1, 0]]),          # incomplete shell
    np.array([[1, 0], [0, 1], [-1, 0], [0, -1]]),         # shell 0 missing
    np.array([[0, 0], [0, 0]]),                           # duplicate
    np.array([[0, 0], [3, 1]]),                           # unsupported shell
])
def test_invalid_bond_lists_rejected(abi, bad):
    with pytest.raises(abi.TufrgError) as e:
        abi.tufrg_eval_formfactors(bad, np.zeros(1), np.zeros(1))
    assert e.value.status == -1


def test_mu_for_density_matches_oracle(abi):
    for tp, n in [(-0.2, 0.8), (-0.4, 0.65), (0.0, 0.95)]:
        mu = abi.tufrg_mu_for_density(1.0, tp, n, 48, 48)
        assert abs(mu - model.mu_for_density(n, 1.0, tp, 48, 48)) < 1e-12
    with pytest.raises(abi.TufrgError):
        abi.tufrg_mu_for_density(1.0, 0.0, 2.5, 48, 48)


def _params(abi, **over):
    bonds = W.bonds_for_shells(1)
    keep = np.ascontiguousarray(bonds, dtype=np.int32)
    p = abi.tufrg_params()
    p.lattice, p.t, p.tp, p.mu, p.U = 0, 1.0, -0.25, -1.0, 3.0
    p.n_bonds = len(keep)
    p.bonds = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    p.nc_x = p.nc_y = 8
    p.nf_x = p.nf_y = 96
    p.precision, p.feedback = 0, 1
    for k, v in over.items():
        setattr(p, k, v)
    return p, keep


@pytest.mark.parametrize("over", [
    dict(lattice=1), dict(nc_x=7), dict(nf_x=100, precision=2), dict(nf_y=88, precision=1),
    dict(nf_x=98), dict(precision=5),
    dict(feedback=2), dict(t=0.0), dict(U=float("nan")), dict(nc_x=2, nc_y=2, nf_x=8, nf_y=8),
])
def test_setup_rejects_invalid_parameters_before_device_work(abi, over):
    p, keep = _params(abi, **over)
    with pytest.raises(abi.TufrgError) as e:
        abi.tufrg_setup(p, 0)
    assert e.value.status == -1


def test_null_arguments_rejected(abi):
    L = abi.lib()
    assert L.tufrg_rhs(None, 1.0, None, None, None) == -1
    assert L.tufrg_loops(None, 1.0, None, None) == -1
    assert L.tufrg_flow(None, None, None, None, None) == -1
    assert L.tufrg_check(None, None) == -1
    assert L.tufrg_selftest_wait(None, 1000, None) == -1
    assert abi.tufrg_status_string(-3) == "non-finite state"


def test_setup_mesh_rejects_invalid_meshes_before_device_work(abi):
    """tufrg_setup_mesh validates the mesh on the host (odd m, square coarse
    grid, nf a multiple of 2 nc m, points in range and distinct, weights
    non-negative summing to one per channel, every point in a mesh)."""
    p, keep = _params(abi, nc_x=6, nc_y=6, nf_x=36, nf_y=36)
    pts, wp, wc = W.channel_mesh(6, 3, ([(0.0, 0.0)], 0.9), ([(-np.pi, -np.pi)], 0.9))
    bad = []
    bad.append((2, pts, wp, wc))                                   # even m
    out = pts.copy()
    out[0, 0] = 18
    bad.append((3, out, wp, wc))                                   # outside the lattice
    dup = pts.copy()
    dup[1] = dup[0]
    bad.append((3, dup, wp, wc))                                   # a point twice
    bad.append((3, pts, 2 * wp, wc))                               # weights not summing to one
    neg = wc.copy()
    neg[np.argmax(neg)] *= -1
    bad.append((3, pts, wp, neg))                                  # negative weight
    i = int(np.argmax(wp))
    bad.append((3, pts, np.where(np.arange(len(wp)) == i, 0.0, wp), wc))  # sum off by w_i
    for m, q, a, b in bad:
        with pytest.raises(abi.TufrgError) as e:
            abi.tufrg_setup_mesh(p, m, q, a, b)
        assert e.value.status == -1
    p2, keep2 = _params(abi, nc_x=6, nc_y=8, nf_x=36, nf_y=48)
    with pytest.raises(abi.TufrgError) as e:                       # rectangular coarse grid
        abi.tufrg_setup_mesh(p2, 3, pts, wp, wc)
    assert e.value.status == -1
    p3, keep3 = _params(abi, nc_x=6, nc_y=6, nf_x=24, nf_y=24)
    with pytest.raises(abi.TufrgError) as e:                       # nf not a multiple of 2 nc m
        abi.tufrg_setup_mesh(p3, 3, pts, wp, wc)
    assert e.value.status == -1
