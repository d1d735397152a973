"""The multi-process short-range force (paper_0910_0121_gb300.domain: Sec. 2.2 steps 3-5 and 7,
Sec. 2.3.1) run as world_size 2 and 4 gloo processes on the CPU, each process's
computation done by the FP64 oracle (tests/oraclecompute.py), the decomposition and the
data movement by the product code.

Checked against one process on the same inputs: every particle ends on exactly one
process, inside that process's box; all processes agree on the boxes, which tile the
periodic box and hold about equal numbers of samples; at theta = 0 the split force equals
the brute-force sum over all particles (the LET brings in every particle within r_cut);
at theta = 0.5 its error against the brute-force sum is that of the one-process tree (the
LETs only change which nodes the processes accept near their faces)."""
import os
import socket
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
from paper_0910_0121_gb300 import build as _build  # noqa: E402

_build.build()  # host-only calls of the library (no GPU touched)
from paper_0910_0121_gb300 import domain, greem  # noqa: E402

N = 3000
PRM = dict(L=1.0, r_cut=0.11, n_crit=32, n_leaf=10)


def _set():
    rng = np.random.default_rng(77)
    pos = rng.random((N, 3))
    k = N // 3
    pos[:k] = np.mod(0.25 + 0.03 * rng.standard_normal((k, 3)), 1.0)   # a dense clump
    pos[k:k + 40] = np.mod(pos[k:k + 40] + 1.0, 2.0) - 0.5            # some outside [0, L)
    return pos, rng.uniform(0.5, 1.5, N).astype(np.float32) / N


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, grid, theta, out_dir):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from oraclecompute import OracleCompute, _cells
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    pos, mass = _set()
    mine = np.arange(rank, N, ws)                         # an arbitrary first distribution
    step = domain.DomainStep(domain.TorchComm(), OracleCompute(), dict(PRM, theta=theta), grid, rate=0.05,
                             alpha=0.2, seed=5)
    P, M, I = (torch.from_numpy(pos[mine].copy()), torch.from_numpy(mass[mine].copy()),
               torch.from_numpy(mine.astype(np.int64)))
    first_ok = None
    for it in range(2):   # the second decomposition weighs the samples by the measured times (Eq. 4)
        P, M, I = step.decompose(P, M, I, N)
        if it == 0:       # the first round already puts every particle in its own box
            c = _cells(P.numpy(), PRM["L"])
            first_ok = bool(np.all((c >= step.boxes[rank, 0::2]) & (c < step.boxes[rank, 1::2])))
        acc = step.force(P, M)
    np.savez(os.path.join(out_dir, f"r{rank}.npz"), ids=I.numpy(), acc=acc.numpy(), pos=P.numpy(),
             boxes=step.boxes, n_import=step.info["n_import"], samples=step.info["samples_total"],
             first_ok=first_ok)
    dist.destroy_process_group()


def _run(ws, grid, theta):
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_rank, args=(ws, _free_port(), grid, theta, d), nprocs=ws, join=True)
        return [dict(np.load(os.path.join(d, f"r{r}.npz"))) for r in range(ws)]


def _rel(a, ref):
    n = np.linalg.norm(ref, axis=1)
    keep = n > 1e-6 * np.median(n)
    return np.linalg.norm(a - ref, axis=1)[keep] / n[keep]


@pytest.fixture(scope="module")
def direct():
    pos, mass = _set()
    return oracle.direct(pos, mass, PRM["L"], PRM["r_cut"])


@pytest.mark.parametrize("ws,grid", [(2, (2, 1, 1)), (4, (2, 2, 1))])
def test_split_at_theta_zero_equals_the_direct_sum(ws, grid, direct):
    res = _run(ws, grid, 0.0)
    ids = np.concatenate([r["ids"] for r in res])
    assert np.array_equal(np.sort(ids), np.arange(N))                  # every particle once
    for r in res[1:]:
        assert np.array_equal(r["boxes"], res[0]["boxes"])             # the same boxes everywhere
    boxes = res[0]["boxes"]
    vol = np.prod((boxes[:, 1::2] - boxes[:, 0::2]).astype(np.float64), axis=1)
    assert vol.sum() == float(2 ** 63)                                  # they tile 2^21 cells per axis
    for rank, r in enumerate(res):
        c = np.array([[oracle.cell_index(x, PRM["L"]) for x in p] for p in r["pos"]]).reshape(-1, 3)
        assert np.all((c >= boxes[rank, 0::2]) & (c < boxes[rank, 1::2]))   # inside its own box
        assert bool(r["first_ok"])
        assert r["n_import"] > 0
    acc = np.zeros((N, 3))
    for r in res:
        acc[r["ids"]] = r["acc"]
    scale = np.abs(direct).max()
    assert np.abs(acc - direct).max() <= 1e-12 * scale


def test_split_at_theta_half_has_the_error_of_one_process(direct):
    pos, mass = _set()
    one = oracle.short_force(pos, mass, PRM["L"], PRM["r_cut"], 0.5, PRM["n_crit"])
    e1 = _rel(one, direct)
    res = _run(4, (2, 2, 1), 0.5)
    acc = np.zeros((N, 3))
    for r in res:
        acc[r["ids"]] = r["acc"]
    e4 = _rel(acc, direct)
    # same accuracy class: the medians and tails agree within a factor of two
    assert np.median(e4) <= 2 * np.median(e1) + 1e-12
    assert np.quantile(e4, 0.99) <= 2 * np.quantile(e1, 0.99)
    assert np.quantile(e1, 0.99) <= 2 * np.quantile(e4, 0.99)


def test_decomposition_balances_the_samples():
    """Recursive multisection puts equal numbers of samples in each box (up to ties), and
    the sample counts follow Eq. 3-5."""
    rng = np.random.default_rng(3)
    cells = rng.integers(0, 2 ** 21, (4000, 3))
    cells[:1500] = rng.integers(1000000, 1001000, (1500, 3))           # a dense spot
    boxes = greem.domain_boxes(cells, (2, 3, 2))
    inside = [np.all((cells >= b[0::2]) & (cells < b[1::2]), axis=1).sum() for b in boxes]
    assert sum(inside) == 4000 and max(inside) - min(inside) <= 2
    assert greem.sample_count(10 ** 6, 250000, 4, 4e-4, 0.0, 0.0, 0.2) == 100        # f = 1/p
    assert greem.sample_count(10 ** 6, 250000, 4, 4e-4, 3.0, 4.0, -1) == 300         # Eq. 4
    assert greem.sample_count(10 ** 6, 600000, 4, 4e-4, 0.5, 4.0, 0.2) == 200        # Eq. 5 floor
    assert greem.sample_count(10 ** 6, 10, 4, 4e-4, 3.0, 4.0, 0.2) == 10             # capped at n_local
