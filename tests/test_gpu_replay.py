"""greem_short_force_ex replays a CUDA graph of a call that repeats one of the two previous
ones (the same pointers, N and parameters).  A replay must give exactly what the usual call gives,
also when the buffers hold new positions, and must fall back to the usual call when the
new positions need more list space than the graph was captured with."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0910_0121_gb300 import build as _build  # noqa: E402

_build.build()
from paper_0910_0121_gb300 import greem  # noqa: E402

N = 20000


def _uniform(seed):
    return np.random.default_rng(seed).random((N, 3))


def _clump(seed):
    """Every particle within 0.02 of one point: with theta = 0 every group's list holds all
    N particles, far more than the list pool a uniform set needs."""
    rng = np.random.default_rng(seed)
    return np.mod(0.5 + 0.02 * (rng.random((N, 3)) - 0.5), 1.0)


def _direct(pos, mass, p):
    """The same call on a context that never replays."""
    ctx = greem.Context()
    ctx.debug_set(greem.DEBUG_REPLAY, 0)
    try:
        a = ctx.short_force(torch.from_numpy(pos).cuda(), torch.from_numpy(mass).cuda(), p)
        torch.cuda.synchronize()
        assert ctx.stats()["replayed"] == 0
        return a.cpu().numpy()
    finally:
        ctx.close()


@pytest.fixture()
def setup():
    mass = np.random.default_rng(3).uniform(0.5, 1.5, N).astype(np.float32) / N
    P = torch.from_numpy(_uniform(1)).cuda()
    M = torch.from_numpy(mass).cuda()
    acc = torch.empty((N, 3), dtype=torch.float32, device="cuda")
    ctx = greem.Context()
    yield ctx, P, M, acc, mass
    ctx.close()


def _call(ctx, P, M, p, acc):
    ctx.short_force(P, M, p, acc)
    torch.cuda.synchronize()
    return ctx.stats()


def test_replay_equals_the_usual_call_on_old_and_new_positions(setup):
    ctx, P, M, acc, mass = setup
    p = greem.params(L=1.0, r_cut=0.08, theta=0.5, n_crit=64)
    seen = [_call(ctx, P, M, p, acc)["replayed"] for _ in range(4)]
    assert seen == [0, 0, 1, 1]
    assert np.array_equal(acc.cpu().numpy(), _direct(_uniform(1), mass, p))
    # new positions in the same buffers: still a replay, and still exact
    P.copy_(torch.from_numpy(_uniform(2)))
    assert _call(ctx, P, M, p, acc)["replayed"] == 1
    assert np.array_equal(acc.cpu().numpy(), _direct(_uniform(2), mass, p))
    st = ctx.stats()
    assert st["n_groups"] > 0 and st["n_list_entries"] > 0 and st["kernel_launches"] > 0


def test_replay_that_overflows_falls_back_and_grows(setup):
    ctx, P, M, acc, mass = setup
    p = greem.params(L=1.0, r_cut=0.1, theta=0.0, n_crit=64)
    for _ in range(3):
        st = _call(ctx, P, M, p, acc)
    assert st["replayed"] == 1
    cap = st["list_capacity"]
    P.copy_(torch.from_numpy(_clump(5)))
    st = _call(ctx, P, M, p, acc)
    assert st["replayed"] == 0 and st["list_capacity"] > cap, st
    assert st["n_list_entries"] > cap
    assert np.array_equal(acc.cpu().numpy(), _direct(_clump(5), mass, p))
    # the grown buffers are kept, and the calls replay again after two more
    seen = [_call(ctx, P, M, p, acc)["replayed"] for _ in range(3)]
    assert seen == [0, 1, 1]
    assert np.array_equal(acc.cpu().numpy(), _direct(_clump(5), mass, p))


def test_replays_report_stage_times(setup):
    ctx, P, M, acc, _ = setup
    p = greem.params(L=1.0, r_cut=0.08, theta=0.5, n_crit=64, flags=greem.FLAG_STAGE_TIMES)
    for _ in range(3):
        st = _call(ctx, P, M, p, acc)
    assert st["replayed"] == 1
    for k in ("ms_sort", "ms_tree", "ms_lists", "ms_force", "ms_total"):
        assert st[k] > 0, (k, st[k])
    parts = sum(st[k] for k in ("ms_keys", "ms_sort", "ms_tree", "ms_groups", "ms_lists", "ms_force"))
    assert abs(parts - st["ms_total"]) <= 0.05 * st["ms_total"] + 0.05


def test_no_replay_when_off_or_when_the_call_changes(setup):
    ctx, P, M, acc, _ = setup
    p = greem.params(L=1.0, r_cut=0.08, theta=0.5, n_crit=64)
    ctx.debug_set(greem.DEBUG_REPLAY, 0)
    assert [_call(ctx, P, M, p, acc)["replayed"] for _ in range(3)] == [0, 0, 0]
    ctx.debug_set(greem.DEBUG_REPLAY, 1)
    assert [_call(ctx, P, M, p, acc)["replayed"] for _ in range(3)] == [0, 0, 1]
    q = greem.params(L=1.0, r_cut=0.08, theta=0.6, n_crit=64)     # other parameters
    assert _call(ctx, P, M, q, acc)["replayed"] == 0
    other = torch.empty_like(acc)                                  # another result buffer
    assert _call(ctx, P, M, q, other)["replayed"] == 0
    assert _call(ctx, P, M, q, other)["replayed"] == 0
    assert _call(ctx, P, M, q, other)["replayed"] == 1


def test_host_buffer_calls_replay_through_both_staging_slots():
    """greem_short_force_host alternates two device staging slots, so its problems repeat
    two calls: both are captured, and the later problems replay, with the results of a
    context that never replays."""
    mass = np.random.default_rng(4).uniform(0.5, 1.5, N).astype(np.float32) / N
    p = greem.params(L=1.0, r_cut=0.08, theta=0.5, n_crit=64)
    sets = [_uniform(10 + k) for k in range(7)]
    hpos = [torch.from_numpy(x).pin_memory() for x in sets]
    hmass = [torch.from_numpy(mass).pin_memory() for _ in sets]
    outs = {}
    for replay in (0, 1):
        ctx = greem.Context()
        ctx.debug_set(greem.DEBUG_REPLAY, replay)
        try:
            outs[replay] = [a.numpy().copy() for a in ctx.short_force_host(hpos, hmass, p)]
            assert ctx.stats()["replayed"] == replay
        finally:
            ctx.close()
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)
    assert np.array_equal(outs[1][0], _direct(sets[0], mass, p))


@pytest.mark.parametrize("variant", ["quadrupole", "fp64", "softened", "eq12"])
def test_replays_of_every_variant_equal_the_usual_call(setup, variant):
    """The second-order passes, the FP64 form, softening and the Eq. 12 opening angle each
    enqueue other kernels: their replays too equal a context that never replays."""
    ctx, P, M, _, mass = setup
    kw = dict(L=1.0, r_cut=0.08, theta=0.5, n_crit=64)
    if variant == "quadrupole":
        kw.update(flags=greem.FLAG_QUADRUPOLE)
    elif variant == "fp64":
        kw.update(precision=greem.F64)
    elif variant == "softened":
        kw.update(eps=1e-3)
    else:
        kw.update(flags=greem.FLAG_THETA_EQ12, theta0=0.25, theta=0.7)
    p = greem.params(**kw)
    dt = torch.float64 if variant == "fp64" else torch.float32
    out = torch.empty((N, 3), dtype=dt, device="cuda")
    seen = [_call(ctx, P, M, p, out)["replayed"] for _ in range(3)]
    assert seen == [0, 0, 1]
    assert np.array_equal(out.cpu().numpy(), _direct(_uniform(1), mass, p))
