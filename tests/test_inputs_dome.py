"""Pins of the Gaussian-dome initial condition (Sec. 5, Eq. gaussian_bump)
against facts its definition fixes: the chord distance d/a equals
2 sin(theta / 2) for the great-circle angle theta from the spherical law of
cosines (an independent formula), the dome's peak g A sits at the centre
(pi, pi/4), it is mirror-symmetric about the centre's meridian, and its
mean geopotential is g h_bar with h_bar = 29400 m."""
import numpy as np

from paper_1805_07923_gb300 import inputs

G = 9.80616


def test_chord_is_twice_the_half_angle_sine():
    rng = np.random.default_rng(4)
    lam = rng.uniform(0.0, 2.0 * np.pi, 200)
    mu = rng.uniform(-1.0, 1.0, 200)
    lc, pc = inputs.DOME_CENTRE
    cos_theta = mu * np.sin(pc) + np.sqrt(1.0 - mu * mu) * np.cos(pc) * np.cos(lam - lc)
    theta = np.arccos(np.clip(cos_theta, -1.0, 1.0))
    d = np.array([inputs.dome_chord(lam[i], mu[i]) for i in range(lam.size)])
    assert np.max(np.abs(d - 2.0 * np.sin(theta / 2.0))) < 1e-13


def test_peak_symmetry_and_mean():
    lc, pc = inputs.DOME_CENTRE
    phi, phibar = inputs.gaussian_dome_grid(np.array([lc]), np.array([np.sin(pc)]))
    assert abs(phi[0, 0] - G * inputs.DOME_A) < 1e-9
    assert abs(phibar - G * 29400.0) < 1e-9
    lam = np.linspace(0.0, 2.0 * np.pi, 64, endpoint=False)
    mu = np.linspace(-0.99, 0.99, 31)
    f, _ = inputs.gaussian_dome_grid(lam, mu)
    g, _ = inputs.gaussian_dome_grid(2.0 * lc - lam, mu)
    assert np.max(np.abs(f - g)) < 1e-9 * np.max(f)
    assert np.all(f > 0) and np.all(f <= G * inputs.DOME_A * (1 + 1e-15))
    # the far side of the sphere (d = 2 a at the antipode) is flat to exp(-4 alpha)
    anti, _ = inputs.gaussian_dome_grid(np.array([lc - np.pi]), np.array([-np.sin(pc)]))
    assert abs(anti[0, 0] - G * inputs.DOME_A * np.exp(-4.0 * inputs.DOME_ALPHA)) < 1e-12 * G * inputs.DOME_A


def test_dome_spectrum_closed_forms():
    """Through the oracle's analysis: the n = 0 coefficient is sqrt(2) times
    the area mean, which for exp(-alpha (d/a)^2) with (d/a)^2 = 2 (1 - cos
    theta) is (1 - exp(-4 alpha)) / (4 alpha); the mirror symmetry about the
    meridian lambda_c = pi makes every coefficient real."""
    from oracle.sht import Grid
    exact = np.sqrt(2.0) * G * inputs.DOME_A * (1.0 - np.exp(-4.0 * inputs.DOME_ALPHA)) / (4.0 * inputs.DOME_ALPHA)
    for R, I, J in [(21, 64, 32), (42, 128, 64)]:
        grid = Grid(R, I, J)
        phi, _ = inputs.gaussian_dome_grid(grid.lam, grid.mu)
        s = grid.analysis(phi)
        assert abs(s[0] - exact) <= 1e-14 * exact
        assert np.max(np.abs(s.imag)) <= 1e-12 * np.max(np.abs(s))
