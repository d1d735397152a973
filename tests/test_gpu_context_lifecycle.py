"""A context gives back every byte of device memory it took: its buffers, the list walk's
start table, its captured graphs and events.  Contexts are created, used for replayed
calls at 256^3 (start table 2M cells, 8 MB; list pool several GB) and closed six times;
after the first cycle (which loads the library's kernels) the free device memory must
come back to the same level each time."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0910_0121_gb300 import build as _build  # noqa: E402

_build.build()
from paper_0910_0121_gb300 import greem  # noqa: E402


def test_closed_contexts_release_their_device_memory():
    N = 1 << 24
    rng = np.random.default_rng(5)
    P = torch.from_numpy(rng.random((N, 3))).cuda()
    M = torch.full((N,), 1.0 / N, dtype=torch.float32, device="cuda")
    acc = torch.empty((N, 3), dtype=torch.float32, device="cuda")
    p = greem.params(L=1.0, r_cut=3.0 / 256, theta=0.5, n_crit=192, flags=greem.FLAG_STAGE_TIMES)
    free = []
    for cycle in range(6):
        ctx = greem.Context()
        for _ in range(3):
            ctx.short_force(P, M, p, acc)
        torch.cuda.synchronize()
        st = ctx.stats()
        assert st["replayed"] == 1 and st["n_start_table"] > 0, st
        ctx.close()
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
    drift = max(free[1:]) - min(free[1:])
    assert drift <= 16 << 20, [f >> 20 for f in free]
