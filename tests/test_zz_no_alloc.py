"""greem_pair_force_f32_noalloc: the pairwise force for callers that cannot allocate device
memory.  Called through the C ABI, it must match the allocating entry point
greem_pair_force_f32 on the same pairs, on two calls in a row (the shared scratch array
keeps the previous call's contents, so the second call checks that everything that must
start at zero is cleared).  Collected last so that a run stopping at the first failure
has run every other test first."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0910_0121_gb300 import build as _build  # noqa: E402

_build.build()
from paper_0910_0121_gb300 import greem, synth  # noqa: E402

MAX_PAIRS = 32768


def _noalloc_fn():
    lib = greem.lib()
    f = lib.greem_pair_force_f32_noalloc
    vp = ctypes.c_void_p
    f.argtypes = [vp, vp, vp, vp, ctypes.c_int64, ctypes.c_double, ctypes.c_double, vp, vp]
    f.restype = ctypes.c_int
    return f


def _dev(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()


@pytest.mark.parametrize("eps", [0.0, 1.953125e-5])
def test_noalloc_matches_allocating_entry_point(eps):
    rc = 5.859375e-3
    xg, xi, xj, mj = synth.e1_pairs(n_i=64, n_j=400, r_cut=rc)   # 25600 pairs
    P = xg.shape[0]
    assert P <= MAX_PAIRS
    XG, XI, XJ, MJ = _dev(xg, np.float64), _dev(xi, np.float64), _dev(xj, np.float64), _dev(mj, np.float32)
    ctx = greem.Context()
    ref = ctx.pair_force_f32(XG, XI, XJ, MJ, rc, eps)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy().astype(np.float64)
    ctx.close()
    f = _noalloc_fn()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        acc = torch.full((P, 3), float("nan"), dtype=torch.float32, device="cuda")
        rc_ = f(ctypes.c_void_p(XG.data_ptr()), ctypes.c_void_p(XI.data_ptr()), ctypes.c_void_p(XJ.data_ptr()),
                ctypes.c_void_p(MJ.data_ptr()), P, rc, eps, ctypes.c_void_p(acc.data_ptr()), stream)
        assert rc_ == greem.OK, (call, rc_)
        got = acc.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got))
        n = np.linalg.norm(ref, axis=1)
        nz = n > 0
        rel = np.linalg.norm(got - ref, axis=1)[nz] / n[nz]
        assert np.max(rel) <= 1e-5, (call, np.max(rel))
        assert np.all(got[~nz] == 0)


def test_noalloc_rejects_sizes_beyond_its_limit():
    f = _noalloc_fn()
    x = torch.zeros((MAX_PAIRS + 1, 3), dtype=torch.float64, device="cuda")
    m = torch.ones(MAX_PAIRS + 1, dtype=torch.float32, device="cuda")
    acc = torch.empty((MAX_PAIRS + 1, 3), dtype=torch.float32, device="cuda")
    p = ctypes.c_void_p
    rc_ = f(p(x.data_ptr()), p(x.data_ptr()), p(x.data_ptr()), p(m.data_ptr()), MAX_PAIRS + 1, 0.01, 0.0,
            p(acc.data_ptr()), None)
    assert rc_ == greem.ERR_INVALID_ARG
    rc_ = f(p(x.data_ptr()), p(x.data_ptr()), p(x.data_ptr()), p(m.data_ptr()), 0, 0.01, 0.0, p(acc.data_ptr()), None)
    assert rc_ == greem.ERR_INVALID_ARG
