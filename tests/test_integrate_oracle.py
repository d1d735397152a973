"""Pins of the time-integration oracle (Sec. 2.2 steps 1, 6, 7; Sec. 2.4, Eq. 6-7), and the
library's host-only helpers against them (no GPU needed)."""
import numpy as np
import pytest

from oracle import integrate as oi


@pytest.mark.parametrize("a0,a1", [(0.02, 0.05), (0.3, 0.31), (0.5, 1.0)])
def test_factors_closed_forms(a0, a1):
    """Einstein-de Sitter (H = H0 a^-3/2): int dt/a = 2(sqrt a1 - sqrt a0)/H0 and
    int dt/a^2 = 2(a0^-1/2 - a1^-1/2)/H0.  de Sitter (H = H0): (1/a0 - 1/a1)/H0 and
    (a0^-2 - a1^-2)/(2 H0)."""
    h0 = 0.7
    k, d = oi.cosmo_factors(a0, a1, 1.0, 0.0, h0)
    assert k == pytest.approx(2 * (np.sqrt(a1) - np.sqrt(a0)) / h0, rel=1e-11)
    assert d == pytest.approx(2 * (a0 ** -0.5 - a1 ** -0.5) / h0, rel=1e-11)
    k, d = oi.cosmo_factors(a0, a1, 0.0, 1.0, h0)
    assert k == pytest.approx((1 / a0 - 1 / a1) / h0, rel=1e-11)
    assert d == pytest.approx((a0 ** -2 - a1 ** -2) / (2 * h0), rel=1e-11)


def test_softening_eq6():
    """Eq. 6: continuous at z_crit, eps_fin below it, and constant in comoving coordinates
    (eps (1+z) = eps_fin (1+z_crit)) above it."""
    ef, zc = 0.01, 5.0
    assert oi.softening(ef, zc, zc) == pytest.approx(ef)
    for z in (0.0, 1.0, 4.999):
        assert oi.softening(ef, zc, z) == ef
    for z in (5.0, 9.0, 99.0):
        assert oi.softening(ef, zc, z) * (1 + z) == pytest.approx(ef * (1 + zc), rel=1e-14)


def test_timestep_eq7_by_hand():
    """|a| = 4 and |v| = 10 at eps = 1: sqrt(1/4) = 0.5 and 1/10 = 0.1, so dt = zeta * 0.1;
    with |v| = 1 the acceleration bound 0.5 wins; zero fields give no bound."""
    v = np.zeros((3, 3), np.float32)
    a = np.zeros((3, 3), np.float32)
    a[1] = [0, 4, 0]
    v[2] = [6, 8, 0]
    assert oi.timestep(v, a, 1.0, 2.0) == pytest.approx(0.2)
    v[2] = [0, 0, 1]
    assert oi.timestep(v, a, 1.0, 1.0) == pytest.approx(0.5)
    assert oi.timestep(np.zeros((2, 3)), np.zeros((2, 3)), 1.0, 1.0) == np.inf


def test_drift_wraps_into_the_box():
    rng = np.random.default_rng(2)
    L = 2.0
    pos = rng.random((1000, 3)) * L
    vel = rng.standard_normal((1000, 3)).astype(np.float32)
    x = oi.drift(pos, vel, L, 0.9)
    assert np.all((x >= 0) & (x < L))
    d = x - pos - 0.9 * vel.astype(np.float64)
    assert np.allclose(d - np.rint(d / L) * L, 0.0, atol=1e-13)


def test_library_host_helpers_match_the_oracle():
    from paper_0910_0121_gb300 import build
    build.build()
    from paper_0910_0121_gb300 import greem
    for z in (0.0, 3.0, 7.0, 30.0):
        assert greem.softening(0.02, 7.0, z) == oi.softening(0.02, 7.0, z)
    for args in ((0.02, 0.05, 0.3, 0.7, 1.0), (0.5, 0.51, 1.0, 0.0, 0.7), (0.1, 1.0, 0.25, 0.7, 2.0)):
        k, d = greem.cosmo_factors(*args)
        kr, dr = oi.cosmo_factors(*args)
        assert k == pytest.approx(kr, rel=1e-12) and d == pytest.approx(dr, rel=1e-12)
    with pytest.raises(greem.GreemError):
        greem.cosmo_factors(0.5, 0.4, 0.3, 0.7, 1.0)
