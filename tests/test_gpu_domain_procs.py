"""The multi-process step (paper_0910_0121_gb300.domain) as the bench runs it with N > 1:
real processes, torch.distributed and the library on the GPU.  Two processes share this
one GPU through the gloo backend, whose exchange goes through the host, so no kernel of
one process ever waits on another's.  At theta = 0 the split force must match the
brute-force sum within the FP32 bounds."""
import os
import socket
import sys
import tempfile

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
from paper_0910_0121_gb300 import build as _build  # noqa: E402

_build.build()
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N, PRM = 16000, dict(L=1.0, r_cut=0.07, theta=0.0, n_crit=48, n_leaf=10)


def _set():
    rng = np.random.default_rng(23)
    pos = rng.random((N, 3))
    pos[: N // 3] = np.mod(0.6 + 0.03 * rng.standard_normal((N // 3, 3)), 1.0)
    return pos, rng.uniform(0.5, 1.5, N).astype(np.float32) / N


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, ws, port, out_dir):
    sys.path.insert(0, ROOT)
    from paper_0910_0121_gb300 import domain, greem
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    torch.cuda.set_device(0)
    pos, mass = _set()
    mine = np.arange(rank, N, ws)
    ctx = greem.Context()
    step = domain.DomainStep(domain.TorchComm("cpu"), domain.GpuCompute(ctx), PRM, (ws, 1, 1), rate=0.05, seed=3)
    P = torch.from_numpy(pos[mine].copy()).cuda()
    M = torch.from_numpy(mass[mine].copy()).cuda()
    I = torch.from_numpy(mine.astype(np.int64)).cuda()
    for _ in range(2):
        P, M, I = step.decompose(P, M, I, N)
        acc = step.force(P, M)
    torch.cuda.synchronize()
    np.savez(os.path.join(out_dir, f"r{rank}.npz"), ids=I.cpu().numpy(), acc=acc.cpu().numpy().astype(np.float64),
             n_import=step.info["n_import"])
    ctx.close()
    dist.destroy_process_group()


def test_two_processes_on_one_gpu_match_the_direct_sum():
    pos, mass = _set()
    ref = oracle.direct(pos, mass, PRM["L"], PRM["r_cut"])
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_rank, args=(2, _port(), d), nprocs=2, join=True)
        res = [dict(np.load(os.path.join(d, f"r{r}.npz"))) for r in range(2)]
    ids = np.concatenate([r["ids"] for r in res])
    assert np.array_equal(np.sort(ids), np.arange(N))
    assert all(int(r["n_import"]) > 0 for r in res)
    acc = np.zeros((N, 3))
    for r in res:
        acc[r["ids"]] = r["acc"]
    n = np.linalg.norm(ref, axis=1)
    keep = n > 1e-6 * np.median(n)
    e = np.linalg.norm(acc - ref, axis=1)[keep] / n[keep]
    assert np.median(e) <= 1e-5 and np.quantile(e, 0.999) <= 1e-4, (np.median(e), np.quantile(e, 0.999))
