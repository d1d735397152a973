"""The multi-process pieces on the GPU (Sec. 2.2 steps 3-5 and 7; Sec. 2.3.1):
greem_cell_index, greem_domain_pack and greem_let_export against the oracle, bit-exact
where the oracle's integer decisions fix the result; and the whole parallel step with four
processes emulated as threads of this process on one GPU (each with its own context and
stream; the exchange goes through the host, and no kernel waits on another): at theta = 0
it equals the brute-force sum within the FP32 bounds, at theta = 0.5 its error against the
brute-force sum is that of one process."""
import threading

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0910_0121_gb300 import build as _build  # noqa: E402

_build.build()
from paper_0910_0121_gb300 import domain, greem  # noqa: E402
from oraclecompute import OracleCompute, _cells  # noqa: E402
from threadcomm import World  # noqa: E402

PRM = dict(L=1.0, r_cut=0.06, n_crit=48, n_leaf=10)


def _set(N, seed, L=1.0):
    rng = np.random.default_rng(seed)
    pos = rng.random((N, 3)) * L
    k = N // 3
    pos[:k] = np.mod(0.3 * L + 0.02 * L * rng.standard_normal((k, 3)), L)
    pos[k:k + 30] = pos[k:k + 30] - L          # outside [0, L): wrapped
    pos[k + 30] = [L, 0.0, np.nextafter(L, 0)]
    return pos, rng.uniform(0.5, 1.5, N).astype(np.float32) / N


def _rel(a, ref):
    n = np.linalg.norm(ref, axis=1)
    keep = n > 1e-6 * np.median(n)
    return np.linalg.norm(a - ref, axis=1)[keep] / n[keep]


@pytest.fixture(scope="module")
def ctx():
    c = greem.Context()
    yield c
    c.close()


@pytest.mark.parametrize("L", [1.0, 3.0])
def test_cell_index_is_the_keys_cell(ctx, L):
    pos, _ = _set(5000, 3, L)
    P = torch.from_numpy(pos).cuda()
    got = ctx.cell_index(P, L).cpu().numpy()
    assert np.array_equal(got, _cells(pos, L))
    idx = np.array([4999, 0, 17, 17, 2500])
    got = ctx.cell_index(P, L, torch.from_numpy(idx).cuda()).cpu().numpy()
    assert np.array_equal(got, _cells(pos[idx], L))


def test_domain_pack_is_stable_and_exact(ctx):
    pos, mass = _set(20000, 4)
    rng = np.random.default_rng(1)
    boxes = greem.domain_boxes(_cells(pos[rng.choice(20000, 300, replace=False)], 1.0), (2, 2, 2))
    ids = torch.from_numpy(np.arange(20000, dtype=np.int64) * 7).cuda()
    po, mo, io, counts = ctx.domain_pack(torch.from_numpy(pos).cuda(), torch.from_numpy(mass).cuda(), ids, 1.0, boxes)
    rp, rm, ri, rc = OracleCompute().pack(torch.from_numpy(pos), torch.from_numpy(mass), ids.cpu(), 1.0, boxes)
    assert np.array_equal(counts, rc)
    assert np.array_equal(io.cpu().numpy(), ri.numpy())
    assert np.array_equal(po.cpu().numpy(), rp.numpy())
    assert np.array_equal(mo.cpu().numpy(), rm.numpy())


@pytest.mark.parametrize("theta", [0.0, 0.5, 0.8])
def test_let_export_equals_the_oracle_walk(ctx, theta):
    """Items of the GPU's flat export in the same order as the oracle's recursive walk:
    the same nodes and particles, exact particle positions and masses, node centres of
    mass to summation order."""
    pos, mass = _set(30000, 5)
    boxes = greem.domain_boxes(_cells(pos[::50], 1.0), (2, 2, 1))
    c = _cells(pos, 1.0)
    mine = np.all((c >= boxes[1, 0::2]) & (c < boxes[1, 1::2]), axis=1)   # the particles of box 1
    lp, lm = pos[mine], mass[mine]
    prm = dict(PRM, theta=theta)
    ctx.build_tree(torch.from_numpy(lp).cuda(), torch.from_numpy(lm).cuda(), greem.params(**prm))
    gp, gm, gref, counts = ctx.let_export(boxes, 1, with_refs=True)
    gp, gm, gref = gp.cpu().numpy(), gm.cpu().numpy(), gref.cpu().numpy()
    T = oracle.Tree(lp, lm, 1.0, prm["r_cut"], n_crit=prm["n_crit"], n_leaf=prm["n_leaf"])
    _, _, xyz, ms = T.sorted()
    mom = T.moments()
    o = 0
    assert counts[1] == 0
    for d in range(len(boxes)):
        if d == 1:
            continue
        kind, idx = T.let_export(boxes[d], theta)
        assert counts[d] == len(idx) and len(idx) > 0
        ref = np.where(kind == 1, -1 - idx, idx)
        sl = slice(o, o + len(idx))
        assert np.array_equal(gref[sl], ref)
        part = kind == 0
        assert np.array_equal(gp[sl][part], xyz[idx[part]])
        assert np.array_equal(gm[sl][part], ms[idx[part]])
        if theta == 0.0:
            assert not np.any(kind == 1)
        else:
            assert np.any(kind == 1)
        nd = idx[~part]
        assert np.abs(gp[sl][~part] - mom[nd, 1:]).max(initial=0) <= 1e-13
        m32 = mom[nd, 0].astype(np.float32)
        assert np.all(np.abs(gm[sl][~part] - m32) <= np.spacing(m32))
        o += len(idx)
    assert o == len(gref)


def _emulated(pos, mass, prm, grid, nproc):
    """The parallel step with nproc processes as threads; returns acc [N,3] by id."""
    world = World(nproc)
    N = len(pos)
    out = [None] * nproc
    errs = []

    def rank(r):
        try:
            torch.cuda.set_device(0)
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                c = greem.Context(s)
                step = domain.DomainStep(world.comm(r), domain.GpuCompute(c), prm, grid, rate=0.02, alpha=0.2,
                                         seed=9)
                mine = np.arange(r, N, nproc)
                P = torch.from_numpy(pos[mine].copy()).cuda()
                M = torch.from_numpy(mass[mine].copy()).cuda()
                I = torch.from_numpy(mine.astype(np.int64)).cuda()
                for _ in range(2):
                    P, M, I = step.decompose(P, M, I, N)
                    acc = step.force(P, M)
                s.synchronize()
                out[r] = (I.cpu().numpy(), acc.cpu().numpy().astype(np.float64), dict(step.info), step.boxes)
                c.close()
        except BaseException as e:  # noqa: BLE001 - reported by the caller
            errs.append(e)
            world.barrier.abort()

    th = [threading.Thread(target=rank, args=(r,)) for r in range(nproc)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    if errs:
        raise errs[0]
    acc = np.full((N, 3), np.nan)
    for ids, a, info, _ in out:
        acc[ids] = a
    return acc, out


def test_emulated_four_processes_against_the_direct_sum(ctx):
    N = 20000
    pos, mass = _set(N, 6)
    direct = oracle.direct(pos, mass, 1.0, PRM["r_cut"])
    acc0, out = _emulated(pos, mass, dict(PRM, theta=0.0), (2, 2, 1), 4)
    assert np.all(np.isfinite(acc0))
    ids = np.concatenate([o[0] for o in out])
    assert np.array_equal(np.sort(ids), np.arange(N))
    assert all(o[2]["n_import"] > 0 for o in out)
    e0 = _rel(acc0, direct)
    print(f"theta 0: median {np.median(e0):.2e}, p99.9 {np.quantile(e0, 0.999):.2e}, "
          f"imports {[o[2]['n_import'] for o in out]}")
    assert np.median(e0) <= 1e-5 and np.quantile(e0, 0.999) <= 1e-4
    acc5, out5 = _emulated(pos, mass, dict(PRM, theta=0.5), (2, 2, 1), 4)
    one = ctx.short_force(torch.from_numpy(pos).cuda(), torch.from_numpy(mass).cuda(),
                          greem.params(**dict(PRM, theta=0.5)))
    torch.cuda.synchronize()
    e1 = _rel(one.cpu().numpy().astype(np.float64), direct)
    e4 = _rel(acc5, direct)
    print(f"theta 0.5: split p99 {np.quantile(e4, 0.99):.3e}, one process p99 {np.quantile(e1, 0.99):.3e}")
    assert np.quantile(e4, 0.99) <= 2 * np.quantile(e1, 0.99)
    assert np.quantile(e1, 0.99) <= 2 * np.quantile(e4, 0.99)
    assert np.median(e4) <= 2 * np.median(e1) + 1e-7
