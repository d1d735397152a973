"""Parity at the full sizes of the 128^3 NFW-mix and 256^3 Zel'dovich workloads, in the
launch configuration bench.py times (n_crit, list chunk and block shape picked by the
same autotuner over the same candidates).

Whole-array checks where the oracle computes everything cheaply (keys, permutation,
tree nodes, groups: bit-exact; moments to summation order); per-group checks on a
seeded sample of groups for what the oracle computes one group at a time (lists
bit-exact, the FP32 entries of the timed launch entry by entry, FP32 force within
median 1e-5 / 99.9th percentile 1e-4, FP64 form 1e-11).  The sample is at least 2% of
the groups, stratified by interaction count (group size x list length), plus the
heaviest groups (the dense halo cores, whose lists are longest).
"""
import ctypes

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

BENCH_CANDIDATES = [48, 64, 96, 128, 192, 256]   # the candidates bench.py autotunes over
FRAC, NSTRATA, NHEAVY = 0.02, 10, 64


def _list_lengths(ctx, n_groups):
    """Unpadded list length of every group of the last call (offsets only, no entries)."""
    g = np.arange(n_groups, dtype=np.int64)
    off = np.zeros(n_groups + 1, np.int64)
    n = ctypes.c_int64()
    vp = ctypes.c_void_p
    greem.lib().greem_debug_dump_group_entries(ctx._h, g.ctypes.data_as(vp), n_groups, off.ctypes.data_as(vp),
                                               None, None, 0, ctypes.byref(n))
    assert n.value == off[-1]
    return np.diff(off)


def _stratified_sample(weight, rng):
    """FRAC of the groups from each of NSTRATA strata of equal size by weight, plus the
    NHEAVY heaviest; sorted and unique."""
    order = np.argsort(weight, kind="stable")
    parts = [rng.choice(st, size=max(1, int(np.ceil(FRAC * len(st)))), replace=False)
             for st in np.array_split(order, NSTRATA)]
    parts.append(order[-NHEAVY:])
    return np.unique(np.concatenate(parts))


def _rel(a, ref):
    n = np.linalg.norm(ref, axis=1)
    keep = n > 1e-6 * np.median(n[n > 0])
    return np.linalg.norm(a - ref, axis=1)[keep] / n[keep]


@pytest.fixture(scope="module", params=["nfw128", "zel256"])
def full(request):
    if request.param == "nfw128":
        pos, mass, prm = synth.config_nfw128()
    else:
        pos, mass, prm = synth.config_zel256()
    N = len(pos)
    P = torch.from_numpy(pos).cuda()
    M = torch.from_numpy(mass).cuda()
    ctx = greem.Context()
    acc = torch.empty((N, 3), dtype=torch.float32, device="cuda")
    base = greem.params(L=prm["L"], r_cut=prm["r_cut"], theta=prm["theta"], n_crit=128)
    best = ctx.autotune(P, M, base, acc, candidates=BENCH_CANDIDATES)
    p = greem.params(L=best.L, r_cut=best.r_cut, theta=best.theta, n_crit=best.n_crit, n_leaf=best.n_leaf,
                     list_chunk=best.list_chunk, block_shape=best.block_shape, flags=greem.FLAG_INDEX_LISTS)
    # without index lists: exactly the launch bench.py times
    pf = greem.params(L=best.L, r_cut=best.r_cut, theta=best.theta, n_crit=best.n_crit, n_leaf=best.n_leaf,
                      list_chunk=best.list_chunk, block_shape=best.block_shape)
    acc_plain = ctx.short_force(P, M, pf, acc).cpu().numpy().astype(np.float64)
    stats_plain = ctx.stats()
    # the sample, stratified by interaction count, and the FP32 entries of the timed launch
    nodes, grp = ctx.dump(greem.DUMP_NODES), ctx.dump(greem.DUMP_GROUPS)
    count = nodes[grp, 5] - nodes[grp, 4]
    rng = np.random.default_rng(20240 + len(request.param))
    sel = _stratified_sample(count * _list_lengths(ctx, len(grp)), rng)
    ent_plain = ctx.dump_group_entries(sel)
    acc = ctx.short_force(P, M, p, acc)
    torch.cuda.synchronize()
    out = dict(name=request.param, pos=pos, mass=mass, prm=prm, p=p, ctx=ctx, P=P, M=M,
               acc=acc.cpu().numpy().astype(np.float64), acc_plain=acc_plain, stats_plain=stats_plain,
               stats_index=ctx.stats(), ent_plain=ent_plain, ent_index=ctx.dump_group_entries(sel, index=True))
    for w in (greem.DUMP_KEYS, greem.DUMP_PERM, greem.DUMP_NODES, greem.DUMP_MOMENTS, greem.DUMP_GROUPS):
        out[w] = ctx.dump(w)
    T = oracle.Tree(pos, mass, prm["L"], prm["r_cut"], n_crit=p.n_crit, n_leaf=p.n_leaf)
    T.build_lists(prm["theta"], sel)
    out.update(T=T, sel=sel)
    yield out
    ctx.close()


def test_keys_perm_bit_exact(full):
    key, perm, _, _ = full["T"].sorted()
    assert np.array_equal(full[greem.DUMP_KEYS], key)
    assert np.array_equal(full[greem.DUMP_PERM].astype(np.int64), perm)


def test_tree_and_groups_bit_exact(full):
    on = full["T"].nodes()
    gn = full[greem.DUMP_NODES]
    assert gn.shape == on.shape
    assert np.array_equal(gn[:, :8], on[:, :8])
    assert np.array_equal(full[greem.DUMP_GROUPS], full["T"].groups())


def test_moments(full):
    om = full["T"].moments()
    gm = full[greem.DUMP_MOMENTS]
    assert np.allclose(gm[:, 0], om[:, 0], rtol=1e-13, atol=0)
    assert np.abs(gm[:, 1:] - om[:, 1:]).max() <= 1e-13 * full["prm"]["L"]


def test_sampled_lists_bit_exact(full):
    off, kind, idx, sh = full["T"].lists()
    goff, gent = full["ctx"].dump_group_lists(full["sel"])
    assert np.array_equal(goff, off)
    assert np.array_equal(gent[:, 0], kind.astype(np.int64))
    assert np.array_equal(gent[:, 1], idx)
    assert np.array_equal(gent[:, 2:], sh.astype(np.int64))


def test_sample_covers_two_percent_and_the_heaviest_groups(full):
    G = full["stats_plain"]["n_groups"]
    assert len(full["sel"]) >= FRAC * G
    print(f"{full['name']}: {len(full['sel'])} of {G} groups sampled, {len(full['ent_plain'][1])} list entries")


def test_sampled_fp32_entries_of_the_timed_launch(full):
    """The FP32 entries written by the list builder of the launch bench.py times (no
    index lists), entry by entry: bitwise equal to those of the index-list launch, which
    match the oracle-derived positions and masses (tests/listcheck.py)."""
    off0, f0, _ = full["ent_plain"]
    off1, f1, ix = full["ent_index"]
    assert np.array_equal(off0, off1)
    assert np.array_equal(f0.view(np.uint32), f1.view(np.uint32))
    rel, mass, kind = listcheck.expected_entries(full["T"], full["prm"]["L"], full["prm"]["r_cut"], full["sel"],
                                                 off1, ix)
    worst = listcheck.check_entries(f0, rel, mass, kind)
    print(f"{full['name']}: {len(f0)} FP32 entries, worst {worst:.3f} of the tolerance")
    toff = full["T"].lists()[0]
    assert np.array_equal(off1, toff)


def test_sampled_force_fp32_and_fp64(full):
    T = full["T"]
    ref_sorted = T.list_force()
    _, perm, _, _ = T.sorted()
    nodes, grp = T.nodes(), T.groups()
    rows = np.concatenate([np.arange(nodes[grp[g], 4], nodes[grp[g], 5]) for g in full["sel"]])
    ref = ref_sorted[rows]
    for form in ("acc", "acc_plain"):
        got = full[form][perm[rows]]
        e = _rel(got, ref)
        print(f"{full['name']} {form}: n_crit {full['p'].n_crit}, {len(rows)} sampled particles, "
              f"median {np.median(e):.2e}, p99.9 {np.quantile(e, 0.999):.2e}")
        assert np.median(e) <= 1e-5
        assert np.quantile(e, 0.999) <= 1e-4
    p = full["p"]
    p64 = greem.params(L=p.L, r_cut=p.r_cut, theta=p.theta, n_crit=p.n_crit, n_leaf=p.n_leaf, precision=greem.F64)
    a64 = full["ctx"].short_force(full["P"], full["M"], p64)
    torch.cuda.synchronize()
    a64 = a64.cpu().numpy()[perm[rows]]
    assert np.abs(a64 - ref).max() <= 1e-11 * np.abs(ref).max()


def test_counts_without_index_lists_equal_index_lists(full):
    """The launch bench.py times (no index lists) builds the same lists as the index-list
    call: equal list lengths and interaction counts over the whole workload."""
    si, sp = full["stats_index"], full["stats_plain"]
    assert sp["n_groups"] == si["n_groups"]
    assert sp["n_list_entries"] == si["n_list_entries"]
    assert sp["n_interactions"] == si["n_interactions"]
