"""Pins of the oracle's model layer: dispersion (Eq. hubb-disp), grids, filling."""
import numpy as np

from oracle import model


def test_dispersion_high_symmetry_points():
    t, tp, mu = 1.0, -0.3, 0.2
    e = lambda kx, ky: model.dispersion(kx, ky, t, tp, mu)
    assert np.isclose(e(0, 0), -4 * t - 4 * tp - mu)
    assert np.isclose(e(np.pi, np.pi), 4 * t - 4 * tp - mu)
    assert np.isclose(e(np.pi, 0), 4 * tp - mu)


def test_van_hove_filling_puts_saddle_on_fermi_level():
    # Sec. 4: van Hove filling is mu = 4 t'; the saddle point (pi, 0) has eps = 0
    for tp in (-0.1, -0.25, -0.35):
        assert model.dispersion(np.pi, 0.0, 1.0, tp, 4 * tp) == 0.0
        assert model.dispersion(0.0, np.pi, 1.0, tp, 4 * tp) == 0.0


def test_grid_and_fold():
    g = model.grid(8)
    assert np.isclose(g[0], -np.pi) and np.isclose(g[4], 0.0)
    u = np.arange(-20, 21)
    f = model.fold_units(u, 8)
    assert np.all((f >= -8) & (f < 8)) and np.all((f - u) % 16 == 0)


def test_particle_hole_symmetry_of_filling():
    # t' = 0: k -> k + (pi, pi) maps eps0 -> -eps0, so n(mu) + n(-mu) = 2
    for mu in (0.37, 1.3):
        assert model.density(1.0, 0.0, mu, 64, 64) + model.density(1.0, 0.0, -mu, 64, 64) == 2.0
    # bisection hits the target up to one degenerate level (<= 8 points, 2 spins)
    mu = model.mu_for_density(0.8, 1.0, -0.2, 64, 64)
    assert abs(model.density(1.0, -0.2, mu, 64, 64) - 0.8) <= 16.0 / 64 ** 2
