"""greem_pair_force_f32_noalloc: the pairwise force for callers that cannot allocate device
memory (a library whose allocator policy forbids driver allocations, a caller that must
not be held up by the device-wide synchronisation cudaMalloc/cudaFree can impose, a
process whose free memory belongs to another allocator).  Called through the C ABI, it
must match the allocating entry point greem_pair_force_f32 on the same pairs, on two
calls in a row (the shared scratch array keeps the previous call's contents, so the
second call checks that everything that must start at zero is cleared), at exactly the
array's limit of 32768 pairs, so that the last slot of every piece of the scratch layout
is written and read.  A fresh process that calls it before anything else of the library
(no context exists, so the scratch address is looked up by this call) checks it against
the oracle.  Collected last so that a run stopping at the first failure has run every
other test first."""
import ctypes
import os
import subprocess
import sys
import textwrap

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
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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
    xg, xi, xj, mj = synth.e1_pairs(n_i=64, n_j=512, r_cut=rc)   # 32768 pairs: the limit
    P = xg.shape[0]
    assert P == MAX_PAIRS
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


_FRESH = textwrap.dedent("""
    import ctypes, sys
    import numpy as np
    import torch
    sys.path.insert(0, {root!r})
    import oracle
    from paper_0910_0121_gb300 import greem, synth
    lib = greem.lib()
    f = lib.greem_pair_force_f32_noalloc
    vp = ctypes.c_void_p
    f.argtypes = [vp, vp, vp, vp, ctypes.c_int64, ctypes.c_double, ctypes.c_double, vp, vp]
    f.restype = ctypes.c_int
    rc, eps = 5.859375e-3, 1.953125e-5
    xg, xi, xj, mj = synth.e1_pairs(n_i=64, n_j=512, r_cut=rc)
    P = xg.shape[0]
    dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()
    XG, XI, XJ, MJ = dev(xg, np.float64), dev(xi, np.float64), dev(xj, np.float64), dev(mj, np.float32)
    d = xj - xi
    ref = np.stack([oracle.pair_accel(d[k], float(mj[k]), rc / 2, eps) for k in range(P)])
    r = np.linalg.norm(d, axis=1)
    fref = np.linalg.norm(ref, axis=1)
    beyond = (r > eps) & (r < 0.75 * rc)
    for call in range(2):
        acc = torch.full((P, 3), float("nan"), dtype=torch.float32, device="cuda")
        code = f(vp(XG.data_ptr()), vp(XI.data_ptr()), vp(XJ.data_ptr()), vp(MJ.data_ptr()), P, rc, eps,
                 vp(acc.data_ptr()), None)
        assert code == 0, code
        a = acc.cpu().numpy().astype(np.float64)
        err = np.linalg.norm(a - ref, axis=1)[beyond] / fref[beyond]
        assert np.median(err) < 1e-5 and np.quantile(err, 0.99) < 1e-4, (np.median(err), np.quantile(err, 0.99))
        assert np.all(a[r >= rc] == 0)
    print("fresh-process no-alloc ok", float(np.median(err)))
""")


def test_noalloc_first_call_in_a_fresh_process_against_the_oracle():
    """The first call of the process, before any context: it looks up the scratch address
    itself and sets the force kernel's shared-memory opt-in for this device.  Checked
    against the oracle's FP64 pair force with the Sec. 3.1.1 bounds, on two calls."""
    out = subprocess.run([sys.executable, "-c", _FRESH.format(root=ROOT)], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stdout[-2000:] + out.stderr[-4000:]
    assert "fresh-process no-alloc ok" in out.stdout


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
