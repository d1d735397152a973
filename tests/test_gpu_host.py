"""greem_short_force_host: independent problems whose inputs and results live in host
memory, with the copies of one problem overlapping the computation of the next.  Each
result must be bit-identical to greem_short_force_ex on device copies of the same inputs
(the same kernels run on the same data), and the FP32 result must meet the force bounds
against the FP64 oracle."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_0910_0121_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0910_0121_gb300 import build as _build  # noqa: E402

_build.build()
from paper_0910_0121_gb300 import greem  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = greem.Context()
    yield c
    c.close()


def _problems():
    """Three boxes of different sizes and structure, all with L = 1."""
    out = []
    pos, mass, prm = synth.config_uniform32()
    out.append((pos, mass))
    rng = np.random.default_rng(91)
    pos2 = rng.random((50000, 3))
    pos2[:20000] = np.mod(0.5 + 0.03 * rng.standard_normal((20000, 3)), 1.0)
    out.append((pos2, np.full(50000, 1.0 / 50000, np.float32)))
    pos3 = rng.random((7001, 3))
    out.append((pos3, rng.uniform(0.5, 1.5, 7001).astype(np.float32) / 7001))
    return out, prm


def _params(prm, **kw):
    return greem.params(L=1.0, r_cut=prm["r_cut"], theta=prm["theta"], n_crit=prm["n_crit"], **kw)


def _device_force(ctx, pos, mass, p):
    acc = ctx.short_force(torch.from_numpy(pos).cuda(), torch.from_numpy(mass).cuda(), p)
    torch.cuda.synchronize()
    return acc.cpu()


@pytest.mark.parametrize("pinned", [True, False])
def test_host_problems_equal_device_calls(ctx, pinned):
    probs, prm = _problems()
    p = _params(prm)
    hp = [torch.from_numpy(np.ascontiguousarray(x)) for x, _ in probs]
    hm = [torch.from_numpy(np.ascontiguousarray(m)) for _, m in probs]
    if pinned:
        hp = [t.pin_memory() for t in hp]
        hm = [t.pin_memory() for t in hm]
        acc = None
    else:
        acc = [torch.full((t.shape[0], 3), np.nan, dtype=torch.float32) for t in hp]
    out = ctx.short_force_host(hp, hm, p, acc)
    for k, (pos, mass) in enumerate(probs):
        ref = _device_force(ctx, pos, mass, p)
        assert torch.equal(out[k], ref), f"problem {k}"


def test_host_problem_meets_force_bounds(ctx):
    probs, prm = _problems()
    pos, mass = probs[0]
    p = _params(prm)
    out = ctx.short_force_host([torch.from_numpy(pos).pin_memory()], [torch.from_numpy(mass).pin_memory()], p)
    ref = oracle.short_force(pos, mass, 1.0, prm["r_cut"], prm["theta"], prm["n_crit"])
    a = out[0].numpy().astype(np.float64)
    na = np.linalg.norm(ref, axis=1)
    keep = na > 1e-6 * np.median(na)
    rel = np.linalg.norm(a - ref, axis=1)[keep] / na[keep]
    assert np.median(rel) <= 1e-5 and np.quantile(rel, 0.999) <= 1e-4


def test_host_f64_precision(ctx):
    probs, prm = _problems()
    p = _params(prm, precision=greem.F64)
    hp = [torch.from_numpy(x).pin_memory() for x, _ in probs[:2]]
    hm = [torch.from_numpy(m).pin_memory() for _, m in probs[:2]]
    out = ctx.short_force_host(hp, hm, p)
    for k in range(2):
        assert out[k].dtype == torch.float64
        assert torch.equal(out[k], _device_force(ctx, probs[k][0], probs[k][1], p))


def test_host_failure_stops_at_the_failing_problem(ctx):
    """Problem 1 holds a NaN position: problem 0 is complete, 1 returns INVALID_ARG, and
    problem 2 is not run (its acc keeps the caller's contents)."""
    probs, prm = _problems()
    p = _params(prm)
    bad = probs[1][0].copy()
    bad[123, 1] = np.nan
    hp = [torch.from_numpy(probs[0][0]), torch.from_numpy(bad), torch.from_numpy(probs[2][0])]
    hm = [torch.from_numpy(m) for _, m in probs]
    acc = [torch.full((t.shape[0], 3), 7.0, dtype=torch.float32) for t in hp]
    with pytest.raises(greem.GreemError) as e:
        ctx.short_force_host(hp, hm, p, acc)
    assert e.value.code == greem.ERR_INVALID_ARG
    assert torch.equal(acc[0], _device_force(ctx, probs[0][0], probs[0][1], p))
    assert bool(torch.all(acc[2] == 7.0))
    # the context stays usable
    out = ctx.short_force_host([hp[2]], [hm[2]], p)
    assert torch.equal(out[0], _device_force(ctx, probs[2][0], probs[2][1], p))


def test_host_rejects_bad_arguments(ctx):
    L = greem.lib()
    probs, prm = _problems()
    p = _params(prm)
    x = torch.from_numpy(probs[2][0])
    m = torch.from_numpy(probs[2][1])
    a = torch.empty((x.shape[0], 3), dtype=torch.float32)
    vp = ctypes.c_void_p
    P = (vp * 1)(x.data_ptr())
    M = (vp * 1)(m.data_ptr())
    A = (vp * 1)(a.data_ptr())
    Ns = (ctypes.c_int64 * 1)(x.shape[0])
    assert L.greem_short_force_host(ctx._h, 0, P, M, Ns, ctypes.byref(p), A) == greem.ERR_INVALID_ARG
    assert L.greem_short_force_host(ctx._h, 1, None, M, Ns, ctypes.byref(p), A) == greem.ERR_INVALID_ARG
    A0 = (vp * 1)(None)
    assert L.greem_short_force_host(ctx._h, 1, P, M, Ns, ctypes.byref(p), A0) == greem.ERR_INVALID_ARG
    N0 = (ctypes.c_int64 * 1)(0)
    assert L.greem_short_force_host(ctx._h, 1, P, M, N0, ctypes.byref(p), A) == greem.ERR_INVALID_ARG
    with pytest.raises(TypeError):
        ctx.short_force_host([x.cuda()], [m], p)
