"""The FP32 list-entry checker (tests/listcheck.py) on the CPU: entries formed from the
oracle's own lists and rounded to FP32 pass, and entries with a planted mistake (one
finest cell off, a wrong image shift, a wrong mass) fail, so that the GPU parity test
built on it can tell a misplaced entry from rounding."""
import numpy as np
import pytest

import listcheck
import oracle


def _entries(seed=5):
    rng = np.random.default_rng(seed)
    N = 3000
    pos = rng.random((N, 3))
    pos[: N // 3] = np.mod(0.02 + 0.015 * rng.standard_normal((N // 3, 3)), 1.0)   # clump across a corner
    mass = rng.uniform(0.5, 1.5, N).astype(np.float32) / N
    L, rc = 1.0, 0.09
    T = oracle.Tree(pos, mass, L, rc, n_crit=32)
    T.build_lists(0.5)
    off, kind, idx, sh = T.lists()
    ix = np.concatenate([kind[:, None], idx[:, None], sh], axis=1).astype(np.int64)
    groups = np.arange(len(off) - 1)
    rel, m, k = listcheck.expected_entries(T, L, rc, groups, off, ix)
    f32 = np.concatenate([rel, m[:, None]], axis=1).astype(np.float32)
    return f32, rel, m, k, L, rc, sh


def test_rounded_oracle_entries_pass():
    f32, rel, m, k, *_ = _entries()
    assert (k == 1).sum() > 100 and (k == 0).sum() > 100
    assert listcheck.check_entries(f32, rel, m, k) < 0.5


@pytest.mark.parametrize("mistake", ["finest_cell", "image_shift", "particle_mass", "node_mass"])
def test_planted_mistakes_fail(mistake):
    f32, rel, m, k, L, rc, sh = _entries()
    bad = f32.copy()
    part = np.flatnonzero(k == 0)
    node = np.flatnonzero(k == 1)
    if mistake == "finest_cell":
        bad[part[len(part) // 2], 0] += np.float32(L / 2 ** 21 / rc)
    elif mistake == "image_shift":
        e = np.flatnonzero(np.any(sh != 0, axis=1))[0]
        bad[e, :3] -= (sh[e] * L / rc).astype(np.float32)
    elif mistake == "particle_mass":
        bad[part[7], 3] = np.nextafter(bad[part[7], 3], np.float32(1))
    else:
        bad[node[3], 3] *= np.float32(1.0 + 2e-6)
    with pytest.raises(AssertionError):
        listcheck.check_entries(bad, rel, m, k)
