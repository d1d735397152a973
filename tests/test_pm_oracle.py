"""Pins of the numpy PM oracle (the long-range part of the TreePM split, Sec. 2.1-2.2).

* PP (Eq. 1-2) + PM for a pair equals the exact periodic force, computed by Ewald
  summation as in the paper's accuracy test (Sec. 3.1.2), to the grid accuracy the paper
  works at (its target: 2%).
* A perfect lattice on the grid points feels no force.
* Total momentum of the PM force vanishes for a symmetric configuration.
"""
import numpy as np
import pytest

import oracle
from oracle import pm


def _unit(seed):
    v = np.random.default_rng(seed).standard_normal(3)
    return v / np.linalg.norm(v)


@pytest.mark.parametrize("scheme,tol_near,tol_far", [(pm.TSC, 0.03, 5e-3), (pm.CIC, 0.2, 2e-2)])
def test_pp_plus_pm_equals_ewald_for_a_pair(scheme, tol_near, tol_far):
    L, n = 1.0, 64
    rc = 3.0 / n
    src = np.array([0.37, 0.52, 0.61])
    for k, r in enumerate([0.3 * rc, 0.5 * rc, rc, 2 * rc, 4 * rc, 0.2, 0.35]):
        tp = src + r * _unit(k)
        pos = np.vstack([src, tp])
        m = np.array([1.0, 1e-12], np.float32)
        a = pm.pm_accel(pos, m, L, n, rc, scheme)[1] + oracle.pair_accel(src - tp, 1.0, rc / 2)
        ew = pm.ewald_accel((tp - src)[None, :], L)[0]
        err = np.linalg.norm(a - ew) / np.linalg.norm(ew)
        assert err < (tol_near if r <= rc else tol_far), (r / rc, err)


def test_ewald_is_newton_at_short_range():
    """The Ewald reference itself: a close pair feels m/r^2 up to the image correction."""
    for r in (1e-3, 1e-2):
        ew = pm.ewald_accel(np.array([[r, 0.0, 0.0]]))[0]
        assert ew[0] == pytest.approx(-1.0 / r ** 2, rel=5 * r ** 3 + 1e-9)
        assert abs(ew[1]) < 1e-9 and abs(ew[2]) < 1e-9


def test_lattice_on_grid_points_has_no_force():
    q = np.arange(8) / 8.0
    p = np.stack(np.meshgrid(q, q, q, indexing="ij"), -1).reshape(-1, 3)
    for scheme in (pm.CIC, pm.TSC):
        a = pm.pm_accel(p, np.ones(len(p), np.float32), 1.0, 32, 3.0 / 32, scheme)
        assert np.abs(a).max() < 1e-12


def test_symmetric_pair_momentum():
    """Two equal masses placed symmetrically about a grid point: equal and opposite forces."""
    L, n = 1.0, 32
    c = np.array([0.5, 0.5, 0.5])
    d = np.array([0.0123, -0.031, 0.0207])
    pos = np.vstack([c + d, c - d])
    a = pm.pm_accel(pos, np.ones(2, np.float32), L, n, 3.0 / n, pm.TSC)
    assert np.abs(a[0] + a[1]).max() < 1e-12 * np.abs(a).max()


def test_ewald_field_matches_the_pairwise_ewald_sum():
    """The structure-factor Ewald sum equals the pairwise one (itself pinned to Newton's
    law at short range) on a small random set, sources and targets overlapping."""
    rng = np.random.default_rng(12)
    src = rng.random((40, 3))
    m = rng.uniform(0.5, 1.5, 40)
    tg = np.vstack([rng.random((5, 3)), src[:3]])
    got = pm.ewald_field(tg, src, m)
    ref = np.zeros_like(got)
    for t in range(tg.shape[0]):
        d = tg[t][None, :] - src
        keep = np.linalg.norm(d, axis=1) > 0
        ref[t] = (pm.ewald_accel(d[keep]) * m[keep][:, None]).sum(axis=0)
    assert np.allclose(got, ref, rtol=1e-6, atol=1e-6 * np.abs(ref).max())
