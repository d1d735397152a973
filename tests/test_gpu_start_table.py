"""The list walk that starts below the root (Sec. 3.1.2 walk): its lists must hold
exactly the entries of the walk from the root, so they are compared with the oracle's
recursive lists bit for bit, and with the GPU's own root walk (start level 0) entry by
entry, FP32 values included.

Each of the first three sets is built to reach one branch of the start (the others are
edge cases: just above the size from which walks start below the root, every particle at
one point, positions outside the box and on its faces):
  coarse -- a dense clump in a sparse background: most of the box's leaves sit above the
            start level, so the table names them and each must be taken once;
  wide   -- r_cut close to L/4: groups whose particle box reaches too far for the image
            argument walk from the root;
  many   -- groups of hundreds of particles at a small r_cut: more level-K cells than
            the start takes, so those groups walk from the root.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0910_0121_gb300 import build as _build  # noqa: E402

_build.build()
from paper_0910_0121_gb300 import greem  # noqa: E402


def _coarse():
    rng = np.random.default_rng(31)
    pos = np.concatenate([np.mod(np.array([0.3, 0.6, 0.2]) + 0.01 * rng.standard_normal((7000, 3)), 1.0),
                          rng.random((1000, 3))])
    return pos, dict(L=1.0, r_cut=0.06, theta=0.5, n_crit=64, n_leaf=10)


def _wide():
    rng = np.random.default_rng(32)
    return rng.random((6000, 3)), dict(L=1.0, r_cut=0.24, theta=0.5, n_crit=128, n_leaf=10)


def _many():
    rng = np.random.default_rng(33)
    return rng.random((40000, 3)), dict(L=1.0, r_cut=0.05, theta=0.5, n_crit=800, n_leaf=10)


def _threshold():
    """One particle above the size from which the walks start below the root."""
    rng = np.random.default_rng(34)
    return rng.random((4097, 3)), dict(L=1.0, r_cut=0.1, theta=0.5, n_crit=32, n_leaf=10)


def _coincident():
    """Every particle at one point: one leaf at the finest level holds them all."""
    return np.tile(np.array([[0.3, 0.7, 0.1]]), (5000, 1)), dict(L=1.0, r_cut=0.1, theta=0.5, n_crit=64, n_leaf=10)


def _wrapped():
    """Positions outside [0, L) (wrapped), on the faces, and a coincident clump."""
    rng = np.random.default_rng(35)
    pos = rng.random((6000, 3))
    pos[:600] += rng.integers(-3, 4, (600, 3))
    pos[600] = [1.0, 0.0, -0.0]
    pos[601] = [np.nextafter(1.0, 0), 0.5, 0.5]
    pos[700:760] = pos[761]
    return pos, dict(L=1.0, r_cut=0.08, theta=0.6, n_crit=48, n_leaf=10)


SETS = {"coarse": _coarse, "wide": _wide, "many": _many, "threshold": _threshold, "coincident": _coincident,
        "wrapped": _wrapped}


def _t(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()


def _run(ctx, pos, mass, prm, start_level):
    ctx.debug_set(greem.DEBUG_START_LEVEL, start_level)
    p = greem.params(L=prm["L"], r_cut=prm["r_cut"], theta=prm["theta"], n_crit=prm["n_crit"],
                     n_leaf=prm["n_leaf"], flags=greem.FLAG_INDEX_LISTS)
    ctx.short_force(_t(pos, np.float64), _t(mass, np.float32), p)
    torch.cuda.synchronize()
    st = ctx.stats()
    off = ctx.dump(greem.DUMP_LIST_OFFSETS)
    lists = ctx.dump(greem.DUMP_LISTS)
    eoff, ent, ix = ctx.dump_group_entries(np.arange(st["n_groups"]), index=True)
    ctx.debug_set(greem.DEBUG_START_LEVEL, -1)
    return st, off, lists, eoff, ent, ix


def _per_group_sorted(eoff, ent, ix):
    """Each group's (index entry, FP32 bits) rows in one canonical order."""
    rows = np.concatenate([ix[:, :5].astype(np.int64), ent.view(np.uint32).astype(np.int64)], axis=1)
    out = []
    for g in range(len(eoff) - 1):
        r = rows[eoff[g]:eoff[g + 1]]
        out.append(r[np.lexsort(r.T[::-1])])
    return out


@pytest.mark.parametrize("name", sorted(SETS))
def test_start_table_lists_equal_root_walk_and_oracle(name):
    pos, prm = SETS[name]()
    mass = np.random.default_rng(7).uniform(0.5, 1.5, len(pos)).astype(np.float32) / len(pos)
    ctx = greem.Context()
    try:
        st, off, lists, eoff, ent, ix = _run(ctx, pos, mass, prm, -1)
        st0, off0, lists0, eoff0, ent0, ix0 = _run(ctx, pos, mass, prm, 0)
    finally:
        ctx.close()
    n_groups = st["n_groups"]
    assert st0["n_start_table"] == 0
    if name == "coarse":
        assert st["n_start_table"] > n_groups // 2 and st["n_start_coarse"] > 0, st
    elif name in ("wide", "many"):
        # the fallback: some (wide: typically all) groups walk from the root
        assert st["n_start_table"] < n_groups, st
    else:
        assert st["n_start_table"] > 0, st
    T = oracle.Tree(pos, mass, prm["L"], prm["r_cut"], n_crit=prm["n_crit"], n_leaf=prm["n_leaf"])
    T.build_lists(prm["theta"])
    toff, kind, idx, sh = T.lists()
    for o, ls in ((off, lists), (off0, lists0)):
        assert np.array_equal(o, toff)
        assert np.array_equal(ls[:, 0], kind.astype(np.int64))
        assert np.array_equal(ls[:, 1], idx)
        assert np.array_equal(ls[:, 2:], sh.astype(np.int64))
    # the same FP32 entries in both walks (their order within a list may differ)
    assert np.array_equal(eoff, eoff0)
    for a, b in zip(_per_group_sorted(eoff, ent, ix), _per_group_sorted(eoff0, ent0, ix0)):
        assert np.array_equal(a, b)
    print(f"{name}: {n_groups} groups, {st['n_start_table']} from the table, "
          f"{st['n_start_coarse']} coarse leaves, {len(ls)} entries")


def test_batched_boxes_each_with_their_own_table():
    """Several boxes in one call, each above the size threshold with its own start level and
    its own table (at its own offset), beside a small box that walks from the root; box
    sides 1, 3 (not a power of two) and 0.5.  Each box's accelerations equal its single-box
    call bit for bit."""
    rng = np.random.default_rng(36)
    specs = [(6000, 1.0, 0.06), (9000, 3.0, 0.2), (700, 1.0, 0.1), (5000, 0.5, 0.03)]
    boxes, prms = [], []
    for n, L, rc in specs:
        boxes.append(rng.random((n, 3)) * L)
        prms.append(dict(L=L, r_cut=rc, theta=0.5, n_crit=48, n_leaf=10))
    masses = [rng.uniform(0.5, 1.5, len(b)).astype(np.float32) / len(b) for b in boxes]
    ctx = greem.Context()
    try:
        singles, starts = [], []
        for p, m, prm in zip(boxes, masses, prms):
            a = ctx.short_force(_t(p, np.float64), _t(m, np.float32), greem.params(**prm))
            torch.cuda.synchronize()
            singles.append(a.cpu().numpy())
            starts.append(ctx.stats()["n_start_table"])
        assert all(s > 0 for s, (n, _, _) in zip(starts, specs) if n > 4096), starts
        assert starts[2] == 0
        off = np.cumsum([0] + [len(b) for b in boxes])
        acc = ctx.short_force_batched(_t(np.concatenate(boxes), np.float64), _t(np.concatenate(masses), np.float32),
                                      off, [greem.params(**q) for q in prms])
        torch.cuda.synchronize()
        assert ctx.stats()["n_start_table"] == sum(starts)
        acc = acc.cpu().numpy()
        for b in range(len(boxes)):
            assert np.array_equal(acc[off[b]:off[b + 1]], singles[b]), b
    finally:
        ctx.close()
