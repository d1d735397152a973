"""GPU path (libgreem.so through the C ABI) against the FP64 CPU oracle.

Integer stages (keys, sort order, tree topology, groups, interaction lists) must be
bit-exact; moments agree to summation order (1e-13); the FP32 force is held to the
bounds median <= 1e-5 and 99.9th percentile <= 1e-4 of the relative error against the
oracle's FP64 force on identical lists; the FP64 form to 1e-11.
"""
import numpy as np
import pytest

import listcheck
import oracle
from paper_0910_0121_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0910_0121_gb300 import build as _build  # noqa: E402

_build.build()
from paper_0910_0121_gb300 import greem  # noqa: E402

MED_BOUND, P999_BOUND = 1e-5, 1e-4


@pytest.fixture(scope="module")
def ctx():
    c = greem.Context()
    yield c
    c.close()


def _t(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()


def gpu_force(ctx, pos, mass, prm, precision=greem.F32_REL, flags=greem.FLAG_INDEX_LISTS, **kw):
    p = greem.params(L=prm["L"], r_cut=prm["r_cut"], theta=prm["theta"], n_crit=prm["n_crit"],
                     n_leaf=prm.get("n_leaf", 10), eps=prm.get("eps", 0.0), precision=precision, flags=flags, **kw)
    acc = ctx.short_force(_t(pos, np.float64), _t(mass, np.float32), p)
    torch.cuda.synchronize()
    return acc.cpu().numpy().astype(np.float64)


def rel_err(a, ref):
    """Per-particle |a - ref| / |ref|; particles with |ref| below 1e-6 of the median
    magnitude are left out (they have no meaningful relative error)."""
    na = np.linalg.norm(ref, axis=1)
    keep = na > 1e-6 * np.median(na[na > 0]) if np.any(na > 0) else na > 0
    return np.linalg.norm(a - ref, axis=1)[keep] / na[keep]


def clustered(N, seed, L=1.0):
    rng = np.random.default_rng(seed)
    pos = rng.random((N, 3)) * L
    k = N // 3
    pos[:k] = np.mod(0.01 * L + 0.02 * L * rng.standard_normal((k, 3)), L)   # clump across a corner
    pos[k:k + 50] = pos[k + 60]                                             # coincident particles
    return pos, rng.uniform(0.5, 1.5, N).astype(np.float32) / N


CASES = {
    "uniform32": lambda: synth.config_uniform32(),
    "clustered": lambda: (*clustered(6000, 4), dict(L=1.0, r_cut=0.08, theta=0.5, n_crit=64, n_leaf=10)),
    "nfw24": lambda: synth.config_nfw128(n_side=24, n_halos=12),
    "boxL3": lambda: (*clustered(3001, 9, L=3.0), dict(L=3.0, r_cut=0.4, theta=0.7, n_crit=40, n_leaf=6)),
    "crit1": lambda: (*clustered(700, 5), dict(L=1.0, r_cut=0.2, theta=0.4, n_crit=1, n_leaf=1)),
    "bigcrit": lambda: (*clustered(4000, 6), dict(L=1.0, r_cut=0.15, theta=0.5, n_crit=700, n_leaf=20)),
    # leaves of up to 99 particles: the tree's window levels beyond the shared-memory
    # halo, and leaf moments in the >= 31-particle bucket
    "bigleaf": lambda: (*clustered(5000, 8), dict(L=1.0, r_cut=0.12, theta=0.5, n_crit=400, n_leaf=100)),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request, ctx):
    pos, mass, prm = CASES[request.param]()
    prm = dict(prm)
    if not prm.get("n_crit"):
        prm["n_crit"] = 64
    acc_plain = gpu_force(ctx, pos, mass, prm, flags=0)   # no index lists: the launch bench.py times
    stats_plain = ctx.stats()
    allg = np.arange(stats_plain["n_groups"])
    ent_plain = ctx.dump_group_entries(allg)              # the FP32 lists of that launch
    acc32 = gpu_force(ctx, pos, mass, prm)
    stats_index = ctx.stats()
    ent_index = ctx.dump_group_entries(allg, index=True)
    dumps = {w: ctx.dump(w) for w in (greem.DUMP_KEYS, greem.DUMP_PERM, greem.DUMP_NODES, greem.DUMP_MOMENTS,
                                      greem.DUMP_GROUPS, greem.DUMP_LIST_OFFSETS, greem.DUMP_LISTS)}
    T = oracle.Tree(pos, mass, prm["L"], prm["r_cut"], n_crit=prm["n_crit"], n_leaf=prm.get("n_leaf", 10))
    T.build_lists(prm["theta"])
    return dict(name=request.param, pos=pos, mass=mass, prm=prm, acc32=acc32, acc_plain=acc_plain, dumps=dumps, T=T,
                stats_plain=stats_plain, stats_index=stats_index, ent_plain=ent_plain, ent_index=ent_index)


def test_keys_and_sort_bit_exact(case):
    key, perm, _, _ = case["T"].sorted()
    assert np.array_equal(case["dumps"][greem.DUMP_KEYS], key)
    assert np.array_equal(case["dumps"][greem.DUMP_PERM].astype(np.int64), perm)


def test_tree_bit_exact(case):
    on = case["T"].nodes()
    gn = case["dumps"][greem.DUMP_NODES]
    assert gn.shape == on.shape
    assert np.array_equal(gn[:, :8], on[:, :8])
    # parent links: each node's parent is the innermost node whose subtree contains it
    par = gn[:, 8]
    assert par[0] == -1
    idx = np.arange(len(gn))
    kids = par >= 0
    assert np.all(par[kids] < idx[kids]) and np.all(gn[par[kids], 6] >= idx[kids] + 1)
    assert np.all(gn[par[kids], 0] == gn[kids, 0] - 1)


def test_moments_to_summation_order(case):
    om = case["T"].moments()
    gm = case["dumps"][greem.DUMP_MOMENTS]
    assert gm.shape == om.shape
    assert np.allclose(gm[:, 0], om[:, 0], rtol=1e-13, atol=0)
    L = case["prm"]["L"]
    assert np.abs(gm[:, 1:] - om[:, 1:]).max() <= 1e-13 * L


def test_groups_bit_exact(case):
    assert np.array_equal(case["dumps"][greem.DUMP_GROUPS], case["T"].groups())


def test_lists_bit_exact(case):
    off, kind, idx, sh = case["T"].lists()
    assert np.array_equal(case["dumps"][greem.DUMP_LIST_OFFSETS], off)
    gl = case["dumps"][greem.DUMP_LISTS]
    assert gl.shape[0] == kind.shape[0]
    assert np.array_equal(gl[:, 0], kind.astype(np.int64))
    assert np.array_equal(gl[:, 1], idx)
    assert np.array_equal(gl[:, 2:], sh.astype(np.int64))


def test_fp32_list_entries(case):
    """The FP32 entries the force kernel reads, element by element.  The list builder
    without index lists (the instantiation the bench times) writes exactly the FP32
    entries of the index-list instantiation, in the same order; those match the oracle's
    FP64 positions relative to the group's cell centre (r_cut units) within a few FP32
    roundings, with the masses, entry by entry in the builder's order."""
    off0, f0, _ = case["ent_plain"]
    off1, f1, ix = case["ent_index"]
    assert np.array_equal(off0, off1)
    assert np.array_equal(f0.view(np.uint32), f1.view(np.uint32))
    prm = case["prm"]
    groups = np.arange(len(off1) - 1)
    rel, mass, kind = listcheck.expected_entries(case["T"], prm["L"], prm["r_cut"], groups, off1, ix)
    worst = listcheck.check_entries(f0, rel, mass, kind)
    print(f"{case['name']}: {len(f0)} entries, worst {worst:.3f} of the tolerance")
    # the builder's order holds the same entries as the oracle's preorder lists
    toff, tkind, tidx, _ = case["T"].lists()
    assert np.array_equal(off1, toff)
    for g in range(len(off1) - 1):
        a = ix[off1[g]:off1[g + 1], :2]
        b = np.stack([tkind[toff[g]:toff[g + 1]], tidx[toff[g]:toff[g + 1]]], axis=1)
        assert np.array_equal(a[np.lexsort(a.T[::-1])], b[np.lexsort(b.T[::-1])])


def test_force_f32_within_bounds(case):
    ref = case["T"].list_force_input_order()
    e = rel_err(case["acc32"], ref)
    assert np.median(e) <= MED_BOUND, np.median(e)
    assert np.quantile(e, 0.999) <= P999_BOUND, np.quantile(e, 0.999)


def test_force_f32_without_index_lists(case):
    """The FP32 call without index lists (the launch bench.py times): the same list
    lengths and interaction counts as the index-list call and as the oracle's lists, and
    the force within the same bounds."""
    si, sp = case["stats_index"], case["stats_plain"]
    off, _, _, _ = case["T"].lists()
    assert sp["n_list_entries"] == si["n_list_entries"] == off[-1]
    assert sp["n_interactions"] == si["n_interactions"]
    ref = case["T"].list_force_input_order()
    e = rel_err(case["acc_plain"], ref)
    assert np.median(e) <= MED_BOUND, np.median(e)
    assert np.quantile(e, 0.999) <= P999_BOUND, np.quantile(e, 0.999)


def test_force_f64_form(case, ctx):
    ref = case["T"].list_force_input_order()
    a = gpu_force(ctx, case["pos"], case["mass"], case["prm"], precision=greem.F64)
    scale = np.abs(ref).max()
    assert np.abs(a - ref).max() <= 1e-11 * scale


# --------------------------------------------------------------------------- plain definition
@pytest.mark.parametrize("precision", [greem.F64, greem.F32_REL])
def test_theta_zero_equals_direct_sum(ctx, precision):
    pos, mass = clustered(3000, 12)
    prm = dict(L=1.0, r_cut=0.1, theta=0.0, n_crit=48)
    ref = oracle.direct(pos, mass, 1.0, 0.1)
    a = gpu_force(ctx, pos, mass, prm, precision=precision, flags=0)
    if precision == greem.F64:
        assert np.abs(a - ref).max() <= 1e-11 * np.abs(ref).max()
    else:
        e = rel_err(a, ref)
        assert np.median(e) <= MED_BOUND and np.quantile(e, 0.999) <= P999_BOUND


def test_uniform32_fp64_against_direct_sum(ctx):
    """32^3 uniform, r_cut = 3/32, theta = 0.5, n_crit = 64, FP64 form vs brute force."""
    pos, mass, prm = synth.config_uniform32()
    ref = oracle.direct(pos, mass, prm["L"], prm["r_cut"])
    a = gpu_force(ctx, pos, mass, prm, precision=greem.F64, flags=0)
    e = rel_err(a, ref)
    # the tree approximation at theta = 0.5 (reported, not a parity bound): most
    # particles' lists open every node within r_cut, a few accept nodes near r_cut
    print(f"uniform32 tree vs direct: median {np.median(e):.2e} p99 {np.quantile(e, 0.99):.2e} "
          f"p99.9 {np.quantile(e, 0.999):.2e}")
    assert np.median(e) < 1e-4
    assert np.quantile(e, 0.99) < 1e-2


# --------------------------------------------------------------------------- edge cases
@pytest.mark.parametrize("N", [1, 2, 9, 10, 11, 3071, 3072, 3073])
def test_small_and_ragged_sizes(ctx, N):
    rng = np.random.default_rng(N)
    pos = rng.random((N, 3))
    if N >= 2:
        pos[1] = pos[0] + [0.01, -0.02, 0.005]
    mass = np.full(N, 1.0 / max(N, 1), np.float32)
    prm = dict(L=1.0, r_cut=0.2, theta=0.5, n_crit=16)
    ref = oracle.short_force(pos, mass, 1.0, 0.2, 0.5, 16)
    for precision in (greem.F64, greem.F32_REL):
        a = gpu_force(ctx, pos, mass, prm, precision=precision, flags=0)
        if N == 1:
            assert np.all(a == 0)
        else:
            e = rel_err(a, ref)
            assert np.median(e) <= MED_BOUND and np.quantile(e, 0.999) <= P999_BOUND


def test_wrapped_and_coincident_positions(ctx):
    rng = np.random.default_rng(3)
    N = 2000
    pos = rng.random((N, 3))
    pos[:200] += rng.integers(-3, 4, (200, 3))      # outside [0, L): wrapped
    pos[200] = [1.0, 0.0, -0.0]                       # exactly L and signed zero
    pos[201] = [np.nextafter(1.0, 0), 0.5, 0.5]
    pos[300:340] = pos[341]                           # 41 coincident particles
    mass = np.full(N, 1.0 / N, np.float32)
    prm = dict(L=1.0, r_cut=0.12, theta=0.6, n_crit=32)
    T = oracle.Tree(pos, mass, 1.0, 0.12, 32)
    T.build_lists(0.6)
    a = gpu_force(ctx, pos, mass, prm)
    key, _, _, _ = T.sorted()
    assert np.array_equal(ctx.dump(greem.DUMP_KEYS), key)
    ref = T.list_force_input_order()
    e = rel_err(a, ref)
    assert np.median(e) <= MED_BOUND and np.quantile(e, 0.999) <= P999_BOUND
    assert np.all(np.isfinite(a))


def test_softening(ctx):
    pos, mass = clustered(3000, 21)
    prm = dict(L=1.0, r_cut=0.1, theta=0.5, n_crit=64, eps=0.1 / 300)
    T = oracle.Tree(pos, mass, 1.0, 0.1, 64)
    T.build_lists(0.5)
    ref = T.list_force_input_order(eps=prm["eps"])
    for precision in (greem.F32_REL, greem.F64):
        a = gpu_force(ctx, pos, mass, prm, precision=precision, flags=0)
        e = rel_err(a, ref)
        assert np.median(e) <= MED_BOUND and np.quantile(e, 0.999) <= P999_BOUND


# --------------------------------------------------------------------------- systems paths
def test_batched_equals_single_boxes(ctx):
    boxes = [clustered(n, 30 + n) for n in (1500, 4097, 777, 2600)]
    prms = [dict(L=1.0, r_cut=rc, theta=th, n_crit=nc) for rc, th, nc in
            ((0.1, 0.5, 64), (0.07, 0.3, 32), (0.2, 0.8, 100), (0.05, 0.5, 48))]
    singles = [gpu_force(ctx, p, m, prm, flags=0) for (p, m), prm in zip(boxes, prms)]
    pos = np.concatenate([b[0] for b in boxes])
    mass = np.concatenate([b[1] for b in boxes])
    off = np.cumsum([0] + [len(b[0]) for b in boxes])
    per = [greem.params(**prm) for prm in prms]
    acc = ctx.short_force_batched(_t(pos, np.float64), _t(mass, np.float32), off, per)
    torch.cuda.synchronize()
    acc = acc.cpu().numpy().astype(np.float64)
    for b in range(len(boxes)):
        assert np.array_equal(acc[off[b]:off[b + 1]], singles[b])


def test_batched_boxes_with_mixed_leaf_sizes(ctx):
    """Boxes with different N_leaf side by side in one call (a block of the tree builder
    then spans boxes with different windows, some beyond the shared-memory halo): the
    tree and the force equal the single-box calls."""
    boxes = [clustered(n, 50 + n) for n in (900, 2100, 1300, 700)]
    prms = [dict(L=1.0, r_cut=0.1, theta=0.5, n_crit=nc, n_leaf=nl) for nc, nl in
            ((64, 6), (300, 100), (64, 10), (200, 70))]
    singles, nodes = [], []
    for (p, m), prm in zip(boxes, prms):
        singles.append(gpu_force(ctx, p, m, prm, flags=0))
        T = oracle.Tree(p, m, prm["L"], prm["r_cut"], n_crit=prm["n_crit"], n_leaf=prm["n_leaf"])
        nodes.append(T.nodes())
        T.build_lists(prm["theta"])
        e = rel_err(singles[-1], T.list_force_input_order())
        assert np.median(e) <= MED_BOUND and np.quantile(e, 0.999) <= P999_BOUND
    # each single-box tree is the oracle's
    for (p, m), prm, on in zip(boxes, prms, nodes):
        gpu_force(ctx, p, m, prm)
        assert np.array_equal(ctx.dump(greem.DUMP_NODES)[:, :8], on[:, :8])
    pos = np.concatenate([b[0] for b in boxes])
    mass = np.concatenate([b[1] for b in boxes])
    off = np.cumsum([0] + [len(b[0]) for b in boxes])
    acc = ctx.short_force_batched(_t(pos, np.float64), _t(mass, np.float32), off, [greem.params(**q) for q in prms])
    torch.cuda.synchronize()
    acc = acc.cpu().numpy().astype(np.float64)
    for b in range(len(boxes)):
        assert np.array_equal(acc[off[b]:off[b + 1]], singles[b])


def test_sort_runs_of_every_size_bit_exact(ctx):
    """The sort orders the top 36 key bits first, then each run of particles sharing a
    level-12 cell by the rest of the key: runs of one, short runs (insertion sort by the
    head), runs of 40 (one warp each), runs of thousands (block sort in shared memory), a
    run beyond that (the one-warp LSD path) and coincident particles (equal keys: input
    order).  Keys and permutation bit-exact."""
    rng = np.random.default_rng(17)
    L = 1.0
    cell = L / 4096
    parts = [rng.random((30000, 3))]                                              # runs of one
    c0 = (np.floor(rng.random((800, 3)) * 4096) + 0.5) * cell
    parts.append((c0[:, None, :] + (rng.random((800, 10, 3)) - 0.5) * cell * 0.98).reshape(-1, 3))  # runs of 10
    c1 = (np.floor(rng.random((300, 3)) * 4096) + 0.5) * cell
    parts.append((c1[:, None, :] + (rng.random((300, 40, 3)) - 0.5) * cell * 0.98).reshape(-1, 3))  # runs of 40
    parts.append(np.array([0.3, 0.6, 0.2]) + rng.random((5000, 3)) * cell * 0.98)                # a run of 5000
    parts.append(np.array([0.71, 0.13, 0.55]) + rng.random((20000, 3)) * cell * 0.98)            # a run of 20000
    parts.append(np.repeat(np.array([[0.9, 0.9, 0.1]]), 300, axis=0))                         # equal keys
    pos = np.concatenate(parts)
    pos = pos[rng.permutation(len(pos))]
    mass = np.full(len(pos), 1.0 / len(pos), np.float32)
    prm = dict(L=L, r_cut=0.01, theta=0.5, n_crit=64)
    ctx.build_tree(_t(pos, np.float64), _t(mass, np.float32), greem.params(**prm))
    key, perm, _, _ = oracle.Tree(pos, mass, L, prm["r_cut"], n_crit=64).sorted()
    assert np.array_equal(ctx.dump(greem.DUMP_KEYS), key)
    assert np.array_equal(ctx.dump(greem.DUMP_PERM).astype(np.int64), perm)


def test_graph_replay_matches_direct_call(ctx):
    pos, mass = clustered(5000, 40)
    prm = dict(L=1.0, r_cut=0.08, theta=0.5, n_crit=64)
    p = greem.params(**prm)
    P, M = _t(pos, np.float64), _t(mass, np.float32)
    acc = torch.zeros((5000, 3), dtype=torch.float32, device="cuda")
    ctx.graph_capture(P, M, p, acc)
    for shift in (0.0, 0.003):
        newpos = np.mod(pos + shift, 1.0)
        P.copy_(_t(newpos, np.float64))
        acc.zero_()
        assert ctx.graph_launch() == greem.OK
        torch.cuda.synchronize()
        ref = gpu_force(ctx, newpos, mass, prm, flags=0)
        assert np.array_equal(acc.cpu().numpy().astype(np.float64), ref)


def test_default_entry_point_matches_ex(ctx):
    pos, mass = clustered(2500, 50)
    acc = greem.short_force(_t(pos, np.float64), _t(mass, np.float32), 1.0, 0.1, 0.5, 64)
    torch.cuda.synchronize()
    ref = gpu_force(ctx, pos, mass, dict(L=1.0, r_cut=0.1, theta=0.5, n_crit=64), flags=0)
    assert np.array_equal(acc.cpu().numpy().astype(np.float64), ref)


def test_invalid_inputs_are_errors(ctx):
    pos, mass = clustered(100, 1)
    bad = pos.copy()
    bad[17, 2] = np.inf
    with pytest.raises(greem.GreemError) as ei:
        gpu_force(ctx, bad, mass, dict(L=1.0, r_cut=0.1, theta=0.5, n_crit=8))
    assert ei.value.code == greem.ERR_INVALID_ARG
    # masses the FP32 force cannot take (NaN, or so large that a particle's zero-distance
    # pair with itself would overflow) are refused too
    for mbad in (np.nan, 2.0 ** 38, -(2.0 ** 39)):
        m2 = mass.copy()
        m2[42] = mbad
        with pytest.raises(greem.GreemError) as ei:
            gpu_force(ctx, pos, m2, dict(L=1.0, r_cut=0.1, theta=0.5, n_crit=8))
        assert ei.value.code == greem.ERR_INVALID_ARG
    for prm in (dict(L=1.0, r_cut=0.5, theta=0.5, n_crit=8), dict(L=1.0, r_cut=0.1, theta=-1.0, n_crit=8),
                dict(L=0.0, r_cut=0.1, theta=0.5, n_crit=8), dict(L=1.0, r_cut=0.1, theta=0.5, n_crit=0)):
        with pytest.raises(greem.GreemError):
            gpu_force(ctx, pos, mass, prm)
    # force-kernel shapes whose chunk buffers exceed a block's shared memory are refused
    # (16 warps x 2 x 1024 entries x 16 bytes = 512 KB); the largest that fits runs
    with pytest.raises(greem.GreemError) as ei:
        gpu_force(ctx, pos, mass, dict(L=1.0, r_cut=0.1, theta=0.5, n_crit=8), list_chunk=1024, block_shape=16)
    assert ei.value.code == greem.ERR_INVALID_ARG
    ok = gpu_force(ctx, pos, mass, dict(L=1.0, r_cut=0.1, theta=0.5, n_crit=8), list_chunk=256, block_shape=16)
    assert np.all(np.isfinite(ok))
    # the context is still usable afterwards
    gpu_force(ctx, pos, mass, dict(L=1.0, r_cut=0.1, theta=0.5, n_crit=8))
    assert greem.lib().greem_pm_force(ctx._h, None, None, 0, 1.0, 32, 0.1, 0, None) == greem.ERR_INVALID_ARG


# --------------------------------------------------------------------------- pairwise error (Sec. 3.1.1)
def test_pairwise_fp32_error_e1(ctx):
    """The pairwise experiment of Sec. 3.1.1 (Fig. 2): r_cut = 5.859375e-3, eps = 1.953125e-5,
    256 x_i x 1024 x_j; the relative error of the FP32 pair force is ~1e-5 beyond eps."""
    rc, eps = 5.859375e-3, 1.953125e-5
    xg, xi, xj, mj = synth.e1_pairs(r_cut=rc)
    a = ctx.pair_force_f32(_t(xg, np.float64), _t(xi, np.float64), _t(xj, np.float64), _t(mj, np.float32), rc, eps)
    torch.cuda.synchronize()
    a = a.cpu().numpy().astype(np.float64)
    d = xj - xi
    r = np.linalg.norm(d, axis=1)
    ref = np.stack([oracle.pair_accel(d[k], 1.0, rc / 2, eps) for k in range(len(r))])
    f = np.linalg.norm(ref, axis=1)
    beyond = (r > eps) & (r < 0.75 * rc)
    err = np.linalg.norm(a - ref, axis=1)[beyond] / f[beyond]
    assert np.median(err) < 1e-5
    assert np.quantile(err, 0.99) < 1e-4
    assert np.all(a[r >= rc] == 0)


# --------------------------------------------------------------------------- Eq. 12 opening angle
@pytest.mark.parametrize("name,theta0,theta_max", [("clustered", 0.2, 0.8), ("nfw24", 0.25, 0.7),
                                                   ("boxL3", 0.3, 1.0)])
def test_eq12_lists_bit_exact_and_force(ctx, name, theta0, theta_max):
    """Distance-dependent opening angle of Sec. 4.1 (Eq. 12), capped at theta_max: the GPU
    applies it through per-level integer distance thresholds, the oracle node by node;
    the lists must be identical and the force within the FP32 bounds."""
    pos, mass, prm = CASES[name]()
    prm = dict(prm, theta=theta_max)
    if not prm.get("n_crit"):
        prm["n_crit"] = 64
    acc = gpu_force(ctx, pos, mass, prm, flags=greem.FLAG_INDEX_LISTS | greem.FLAG_THETA_EQ12, theta0=theta0)
    T = oracle.Tree(pos, mass, prm["L"], prm["r_cut"], n_crit=prm["n_crit"], n_leaf=prm.get("n_leaf", 10))
    T.build_lists(theta_max, theta0=theta0)
    off, kind, idx, sh = T.lists()
    assert np.array_equal(ctx.dump(greem.DUMP_LIST_OFFSETS), off)
    gl = ctx.dump(greem.DUMP_LISTS)
    assert np.array_equal(gl[:, 0], kind.astype(np.int64))
    assert np.array_equal(gl[:, 1], idx)
    assert np.array_equal(gl[:, 2:], sh.astype(np.int64))
    # the variant changes the lists (else this test would not test it)
    T2 = oracle.Tree(pos, mass, prm["L"], prm["r_cut"], n_crit=prm["n_crit"], n_leaf=prm.get("n_leaf", 10))
    T2.build_lists(theta_max)
    assert T2.lists()[0][-1] != off[-1]
    e = rel_err(acc, T.list_force_input_order())
    assert np.median(e) <= MED_BOUND and np.quantile(e, 0.999) <= P999_BOUND


def test_eq12_needs_a_positive_theta0(ctx):
    pos, mass = clustered(300, 3)
    with pytest.raises(greem.GreemError) as ei:
        gpu_force(ctx, pos, mass, dict(L=1.0, r_cut=0.1, theta=0.7, n_crit=16),
                  flags=greem.FLAG_THETA_EQ12, theta0=0.0)
    assert ei.value.code == greem.ERR_INVALID_ARG


# --------------------------------------------------------------------------- second-order terms
@pytest.mark.parametrize("name,theta", [("clustered", 0.7), ("nfw24", 0.6), ("boxL3", 0.7), ("uniform32", 0.8)])
def test_quadrupole_moments_and_force(ctx, name, theta):
    """GREEM_FLAG_QUADRUPOLE (Sec. 4.1): FP32 second moments against the oracle's FP64
    ones (to 2e-5 of M * side^2 per component), and the force with the second-order terms
    against the oracle's on identical lists, within the FP32 bounds."""
    pos, mass, prm = CASES[name]()
    prm = dict(prm, theta=theta)
    if not prm.get("n_crit"):
        prm["n_crit"] = 64
    acc = gpu_force(ctx, pos, mass, prm, flags=greem.FLAG_QUADRUPOLE)
    T = oracle.Tree(pos, mass, prm["L"], prm["r_cut"], n_crit=prm["n_crit"], n_leaf=prm.get("n_leaf", 10))
    T.build_lists(theta)
    gq = ctx.dump(greem.DUMP_QUADRUPOLES)
    oq = T.quadrupoles()
    nodes, mom = T.nodes(), T.moments()
    scale = mom[:, 0] * (prm["L"] / 2.0 ** nodes[:, 0]) ** 2
    assert gq.shape == oq.shape
    assert np.all(np.abs(gq - oq) <= 2e-5 * scale[:, None] + 1e-30)
    ref = T.list_force_input_order(quad=True)
    e = rel_err(acc, ref)
    assert np.median(e) <= MED_BOUND and np.quantile(e, 0.999) <= P999_BOUND, (np.median(e), np.quantile(e, 0.999))
    # the terms matter on these lists: the monopole-only force is farther from the reference
    e0 = rel_err(gpu_force(ctx, pos, mass, prm), ref)
    assert np.quantile(e0, 0.99) > 10 * np.quantile(e, 0.99)


def test_quadrupole_needs_fp32_and_no_softening(ctx):
    pos, mass = clustered(300, 3)
    prm = dict(L=1.0, r_cut=0.1, theta=0.7, n_crit=16)
    for kw in (dict(eps=1e-3), dict(precision=greem.F64)):
        with pytest.raises(greem.GreemError) as ei:
            gpu_force(ctx, pos, mass, dict(prm, **{k: v for k, v in kw.items() if k == "eps"}),
                      precision=kw.get("precision", greem.F32_REL), flags=greem.FLAG_QUADRUPOLE)
        assert ei.value.code == greem.ERR_INVALID_ARG
