"""The two facts that let a list walk start below the root (Sec. 3.1.2 walk; the start
table), checked by brute force on random geometries in the walk's integer units
(u = L/2^22, period P = 2^22 u), with the walk's own tests restated here:

  prune:  per axis d = the cell centre's offset from the group cell centre, wrapped to
          [-P/2, P/2); g = max(0, |d - tb| - h - th); pruned iff sum g^2 > T
  accept: e = max(0, |d| - hg) per axis; accepted iff sum e^2 > A

1. A cell of half side h that passes the prune test lies within (sqrt(T) + sqrt(3) h)^2
   of the group cell: sum e^2 <= (sqrt(sum g^2) + sqrt(3) h)^2.  So no node of a level k
   with (sqrt(T) + sqrt(3) h_k)^2 <= A[k] is ever accepted.
2. If L/4 > sqrt(T) + th + |tb| on every axis, every ancestor (half side <= L/4) of a
   cell that passes the prune test passes it too, each tested at its own nearest image.

The bound fails if the prune gap is measured from the group's whole cell instead of its
particle box, or if the accept distance is not wrapped to the nearest image; the third
test shows that the image condition of fact 2 cannot be dropped.  (Whether the kernels
compute these tests as restated here is what the GPU parity tests check: their lists
are compared with the oracle's entry by entry.)
"""
import numpy as np

P = 1 << 22
HALF = P // 2
KMAX = 21


def wrap(d):
    d = np.asarray(d, dtype=np.int64)
    return np.where(d >= HALF, d - P, np.where(d < -HALF, d + P, d))


def gap2(rc, h, tb, th):
    d = wrap(rc)
    g = np.maximum(0, np.abs(d - tb) - h - th)
    return (g * g).sum(axis=-1)


def dist2(rc, hg):
    d = wrap(rc)
    e = np.maximum(0, np.abs(d) - hg)
    return (e * e).sum(axis=-1)


def random_group(rng, n):
    """n groups: cell level kg, corner (finest-cell units), particle box inside the cell."""
    kg = rng.integers(2, 12, n)
    hg = (1 << (KMAX - kg)).astype(np.int64)           # half side (u)
    ncell = 1 << kg
    corner = rng.integers(0, ncell[:, None], (n, 3)) * (2 * hg)[:, None]
    centre = corner + hg[:, None]
    # particle box: a random sub-box of finest cells (2u each) inside the group cell
    lo = rng.integers(0, np.maximum(hg, 1)[:, None], (n, 3)) * 2
    hi = np.minimum(lo + 2 * rng.integers(1, np.maximum(hg, 2)[:, None], (n, 3)), 2 * hg[:, None])
    tb = (lo + hi) // 2 - hg[:, None]                  # box centre minus cell centre
    th = (hi - lo) // 2
    return kg, hg, centre, tb, th


def test_pruned_distance_bounds_the_accept_distance():
    rng = np.random.default_rng(123)
    n = 200000
    kg, hg, gc, tb, th = random_group(rng, n)
    k = rng.integers(1, 22, n)
    h = (1 << (KMAX - k)).astype(np.int64)
    # node cells near the group (and some across the periodic boundary)
    spread = np.maximum(h, hg) * 8
    nc = (gc + rng.integers(-1, 2, (n, 3)) * rng.integers(0, spread[:, None] + 1, (n, 3))) % P
    nc = (nc // (2 * h[:, None])) * (2 * h[:, None]) + h[:, None]   # snap to a level-k cell centre
    rc = nc - gc
    sg = gap2(rc, h[:, None], tb, th)
    sd = dist2(rc, hg[:, None])
    bound = (np.sqrt(sg.astype(np.float64)) + np.sqrt(3.0) * h) ** 2
    assert np.all(sd <= bound * (1 + 1e-12) + 1e-6)
    # the bound is not loose everywhere: some cells come within a factor 2 of it
    assert np.mean(sd > 0.5 * bound) > 0.01


def test_ancestors_of_a_passing_cell_pass_under_the_image_condition():
    rng = np.random.default_rng(7)
    n = 40000
    kg, hg, gc, tb, th = random_group(rng, n)
    # r_cut from a few cells up to nearly L/4 - the particle box reach
    reach = np.abs(tb).max(axis=1) + th.max(axis=1)
    R = rng.integers(1, np.maximum(P // 4 - reach - 1, 2))
    T = R.astype(np.int64) ** 2
    ok = (P // 4 - th - np.abs(tb) > np.ceil(np.sqrt(T))[:, None] + 1).all(axis=1)
    checked = 0
    for k in (6, 7, 9):
        h = 1 << (KMAX - k)
        # a level-k cell within reach of the group (wrapped around the box half the time)
        off = rng.integers(-(R + hg) // (2 * h) - 2, (R + hg) // (2 * h) + 3, (3, n)).T
        cell = ((gc // (2 * h)) + off) % (1 << k)
        rc = cell * 2 * h + h - gc
        passes = (gap2(rc, h, tb, th) <= T) & ok
        for a in range(1, k):
            ha = 1 << (KMAX - a)
            acell = cell >> (k - a)
            arc = acell * 2 * ha + ha - gc
            assert np.all(gap2(arc[passes], ha, tb[passes], th[passes]) <= T[passes]), (k, a)
        checked += int(passes.sum())
    assert checked > 1000


def test_the_image_condition_is_needed():
    """Without it an ancestor can fail where its descendant passes.  A level-2 group cell
    [0, L/4) with its particle box against the +x face and r_cut just above L/4: a
    level-5 cell just past x = L/2 passes (gap L/4 along x), while its level-2 ancestor
    [L/2, 3L/4), whose centre lies exactly L/2 from the group's and wraps to -L/2, has a
    gap of L/2 - 2u there and fails.  Here L/4 - th - |tb| = L/8 < r_cut."""
    hg = P // 8
    gc = np.array([[hg, hg, hg]])
    tb = np.array([[hg - 1, 0, 0]])
    th = np.array([[1, hg, hg]])
    R = P // 4 + 8
    T = R * R
    assert not np.all(P // 4 - th - np.abs(tb) > R)
    k, h = 5, 1 << (KMAX - 5)
    cell = np.array([[(P // 2) // (2 * h), 2, 2]])     # x in [L/2, L/2 + L/32), y, z inside the group's range
    assert gap2(cell * 2 * h + h - gc, h, tb, th)[0] <= T
    a, ha = 2, 1 << (KMAX - 2)
    arc = (cell >> (k - a)) * 2 * ha + ha - gc
    assert wrap(arc)[0, 0] == -HALF
    assert gap2(arc, ha, tb, th)[0] > T
