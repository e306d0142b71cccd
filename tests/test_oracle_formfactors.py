"""Pins of the form-factor basis (Sec. 3 footnote, App. A counting, App. C)."""
import numpy as np
import pytest

import workloads as W
from oracle import formfactors as ff

SHELL_COUNTS = [1, 5, 9, 13, 21, 25, 29]


@pytest.mark.parametrize("shells", range(7))
def test_counts_and_orthonormality(shells):
    b = ff.Basis.from_bonds(W.bonds_for_shells(shells))
    assert b.nff == SHELL_COUNTS[shells] == len(W.bonds_for_shells(shells))
    n = 2 * b.max_component + 1
    k = -np.pi + 2 * np.pi * np.arange(n) / n
    kx, ky = np.meshgrid(k, k, indexing="ij")
    f = b.values(kx, ky).reshape(b.nff, -1)
    assert np.allclose(f @ f.T / f.shape[1], np.eye(b.nff), atol=1e-13)


def test_smfrg_dimension_fixes_nff_at_fifth_neighbour():
    # App. A: 5th-NN truncation on the 992 + 6632 + 6632 meshes -> ~8.9e6
    nff = ff.Basis.from_bonds(W.bonds_for_shells(5)).nff
    assert (992 + 2 * 6632) * nff ** 2 == 8_910_000


@pytest.mark.parametrize("shells", [3, 6])
def test_parity_and_bond_length(shells):
    b = ff.Basis.from_bonds(W.bonds_for_shells(shells))
    rng = np.random.default_rng(0)
    k = rng.uniform(-np.pi, np.pi, (2, 50))
    assert np.allclose(b.values(-k[0], -k[1]), b.parity[:, None] * b.values(k[0], k[1]))
    c = b.coefficients()
    shell_of_bond = np.array([ff.shell_of(r) for r in b.bonds])
    for m in range(b.nff):
        # every form factor belongs to one bond length (Sec. 3 footnote)
        assert np.all(np.abs(c[m, shell_of_bond != b.shells[m]]) < 1e-14)
        # real function: c(-R) = conj c(R)
        for j, r in enumerate(b.bonds):
            jm = [i for i, q in enumerate(b.bonds) if q[0] == -r[0] and q[1] == -r[1]][0]
            assert abs(c[m, jm] - np.conj(c[m, j])) < 1e-14


def test_point_group_representation():
    b = ff.Basis.from_bonds(W.bonds_for_shells(5))
    mats = [b.rep_matrix(S) for S in ff.POINT_GROUP]
    for Cm in mats:
        assert np.allclose(Cm @ Cm.T, np.eye(b.nff), atol=1e-12)
        # block diagonal in shells
        assert np.all(np.abs(Cm[b.shells[:, None] != b.shells[None, :]]) < 1e-12)
    # homomorphism: f(S1 S2 k) = C^{S1} f(S2 k)  =>  C^{S1 S2} = C^{S1} C^{S2}
    for i, S1 in enumerate(ff.POINT_GROUP):
        for j, S2 in enumerate(ff.POINT_GROUP):
            assert np.allclose(b.rep_matrix(S1 @ S2), mats[i] @ mats[j], atol=1e-12)
    # characters of the 1-d irreps
    for m, irr in enumerate(b.irreps):
        diag = np.array([Cm[m, m] for Cm in mats])
        if irr == "A1":
            assert np.allclose(diag, 1)
        if irr in ("B1", "B2", "A2"):
            assert np.allclose(np.abs(diag), 1) and np.isclose(diag[1], 1 if irr == "A2" else -1)


def test_incomplete_shell_rejected():
    bonds = W.bonds_for_shells(1)[:-1]
    with pytest.raises(ValueError):
        ff.Basis.from_bonds(bonds)
