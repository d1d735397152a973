"""Failure paths of the C ABI, each exercised without a GPU fault, hang or trap:

* a capacity overflow (tree nodes, list pool, traversal stack) grows the buffer and the
  call is retried, with a result identical to that of an unconstrained call;
* the retry bound: a call still overflowing after its attempts returns CAPACITY, and the
  context works afterwards;
* a CUDA-graph replay whose positions need more list space than was captured returns
  CAPACITY, and a direct call on those positions then succeeds;
* a bounded device wait that gives up (the force kernel's list-chunk wait, its poll
  limit lowered to zero through greem_debug_set) returns TIMEOUT, the warps let their
  copies in flight land before leaving, and the next call is correct.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0910_0121_gb300 import build as _build  # noqa: E402

_build.build()
from paper_0910_0121_gb300 import greem  # noqa: E402

DEBUG_WAIT_POLLS, DEBUG_NODE_CAP, DEBUG_STACK_CAP = greem.DEBUG_WAIT_POLLS, greem.DEBUG_NODE_CAP, greem.DEBUG_STACK_CAP
DEBUG_LIST_CAP, DEBUG_MAX_ATTEMPTS = greem.DEBUG_LIST_CAP, greem.DEBUG_MAX_ATTEMPTS


def _t(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()


def _set(ctx, what, value):
    ctx.debug_set(what, value)


def _clustered(N, seed):
    rng = np.random.default_rng(seed)
    pos = rng.random((N, 3))
    k = N // 3
    pos[:k] = np.mod(0.5 + 0.02 * rng.standard_normal((k, 3)), 1.0)
    return pos, rng.uniform(0.5, 1.5, N).astype(np.float32) / N


PRM = dict(L=1.0, r_cut=0.08, theta=0.5, n_crit=64)


def _force(ctx, pos, mass, **kw):
    p = greem.params(**dict(PRM, **kw))
    acc = ctx.short_force(_t(pos, np.float64), _t(mass, np.float32), p)
    torch.cuda.synchronize()
    return acc.cpu().numpy()


@pytest.fixture(scope="module")
def data():
    pos, mass = _clustered(20000, 71)
    ctx = greem.Context()
    ref = _force(ctx, pos, mass)
    st = ctx.stats()
    ctx.close()
    assert st["retries"] == 0
    return pos, mass, ref, st


def test_capacity_overflow_grows_and_retries(data):
    pos, mass, ref, st0 = data
    ctx = greem.Context()
    _set(ctx, DEBUG_NODE_CAP, 64)
    _set(ctx, DEBUG_LIST_CAP, 4096)
    _set(ctx, DEBUG_STACK_CAP, 16)
    got = _force(ctx, pos, mass)
    st = ctx.stats()
    assert st["retries"] >= 2, st["retries"]      # nodes first, then lists and stack
    assert st["n_nodes"] == st0["n_nodes"] and st["n_list_entries"] == st0["n_list_entries"]
    assert np.array_equal(got, ref)
    # the grown capacities stay: the next call needs no retry
    assert np.array_equal(_force(ctx, pos, mass), ref)
    assert ctx.stats()["retries"] == 0
    ctx.close()


def test_retry_bound_returns_capacity_and_the_context_recovers(data):
    pos, mass, ref, _ = data
    ctx = greem.Context()
    _set(ctx, DEBUG_MAX_ATTEMPTS, 1)
    _set(ctx, DEBUG_NODE_CAP, 64)
    with pytest.raises(greem.GreemError) as ei:
        _force(ctx, pos, mass)
    assert ei.value.code == greem.ERR_CAPACITY
    _set(ctx, DEBUG_MAX_ATTEMPTS, -1)
    assert np.array_equal(_force(ctx, pos, mass), ref)
    ctx.close()


def test_graph_replay_that_outgrows_its_capture_is_a_capacity_error():
    """Captured on uniform positions at theta = 0, whose lists are short; replayed on a
    tight cluster, where every group's list holds every particle (2048 x 32768 entries
    and more, beyond the captured pool of about 1.1e7)."""
    N = 32768
    rng = np.random.default_rng(73)
    uni = rng.random((N, 3))
    tight = 0.5 + 0.01 * (rng.random((N, 3)) - 0.5)
    mass = np.full(N, 1.0 / N, np.float32)
    prm = dict(L=1.0, r_cut=0.06, theta=0.0, n_crit=64)
    ctx = greem.Context()
    P, M = _t(uni, np.float64), _t(mass, np.float32)
    acc = torch.zeros((N, 3), dtype=torch.float32, device="cuda")
    ctx.graph_capture(P, M, greem.params(**prm), acc)
    cap = ctx.stats()["list_capacity"]
    assert ctx.graph_launch() == greem.OK
    P.copy_(_t(tight, np.float64))
    assert ctx.graph_launch() == greem.ERR_CAPACITY
    # a direct call grows its buffers and succeeds
    out = ctx.short_force(P, M, greem.params(**prm))
    torch.cuda.synchronize()
    st = ctx.stats()
    assert st["retries"] >= 1 and st["n_list_entries"] > cap
    assert torch.isfinite(out).all()
    ctx.close()


def test_a_wait_that_gives_up_returns_timeout_and_the_context_recovers(data):
    pos, mass, ref, _ = data
    ctx = greem.Context()
    _set(ctx, DEBUG_WAIT_POLLS, 0)
    with pytest.raises(greem.GreemError) as ei:
        _force(ctx, pos, mass)
    assert ei.value.code == greem.ERR_TIMEOUT
    # the pairwise entry point streams its one-entry lists through the same wait
    x = _t(np.full((64, 3), 0.5), np.float64)
    with pytest.raises(greem.GreemError) as ei:
        ctx.pair_force_f32(x, x, _t(np.full((64, 3), 0.5001), np.float64), _t(np.ones(64), np.float32), 0.01)
    assert ei.value.code == greem.ERR_TIMEOUT
    _set(ctx, DEBUG_WAIT_POLLS, -1)
    assert np.array_equal(_force(ctx, pos, mass), ref)
    ctx.close()


def test_debug_controls_reject_bad_values():
    ctx = greem.Context()
    f = greem.lib().greem_debug_set
    assert f(ctx._h, 99, 1) == greem.ERR_INVALID_ARG
    assert f(ctx._h, DEBUG_NODE_CAP, 0) == greem.ERR_INVALID_ARG
    assert f(ctx._h, DEBUG_WAIT_POLLS, 1 << 40) == greem.ERR_INVALID_ARG
    assert f(None, DEBUG_NODE_CAP, 10) == greem.ERR_INVALID_ARG
    ctx.close()
