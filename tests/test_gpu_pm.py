"""PM part on the GPU (greem_pm_force, GREEM_FLAG_ADD_PM) against the numpy FP64 PM oracle,
and the full TreePM force (PP + PM) against Ewald summation, the paper's exact reference
(Sec. 3.1.2), on a small clustered set."""
import numpy as np
import pytest

import oracle
from oracle import pm as pmo
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


def _t(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()


def clustered(N, seed, L=1.0):
    rng = np.random.default_rng(seed)
    pos = rng.random((N, 3)) * L
    k = N // 3
    pos[:k] = 0.01 * L + 0.03 * L * rng.standard_normal((k, 3))   # across a corner, outside [0, L) too
    return pos, rng.uniform(0.5, 1.5, N).astype(np.float32) / N


@pytest.mark.parametrize("n,scheme,L", [(32, pmo.TSC, 1.0), (64, pmo.TSC, 1.0), (32, pmo.CIC, 1.0),
                                        (48, pmo.TSC, 3.0)])
def test_pm_matches_oracle(ctx, n, scheme, L):
    pos, mass = clustered(20000, n + scheme, L)
    rc = 3.0 * L / n
    ref = pmo.pm_accel(pos, mass, L, n, rc, scheme)
    got = ctx.pm_force(_t(pos, np.float64), _t(mass, np.float32), L, n, rc, scheme)
    torch.cuda.synchronize()
    got = got.cpu().numpy().astype(np.float64)
    rms = np.sqrt(np.mean(np.sum(ref * ref, axis=1)))
    err = np.linalg.norm(got - ref, axis=1)
    assert err.max() <= 2e-4 * rms, err.max() / rms
    assert np.median(err / np.linalg.norm(ref, axis=1)) <= 1e-5


def test_treepm_in_one_call_equals_pp_plus_pm(ctx):
    pos, mass = clustered(30000, 7)
    n, rc = 64, 3.0 / 64
    P, M = _t(pos, np.float64), _t(mass, np.float32)
    pp = ctx.short_force(P, M, greem.params(L=1.0, r_cut=rc, theta=0.5, n_crit=64))
    pmf = ctx.pm_force(P, M, 1.0, n, rc, greem.ASSIGN_TSC)
    both = ctx.short_force(P, M, greem.params(L=1.0, r_cut=rc, theta=0.5, n_crit=64, flags=greem.FLAG_ADD_PM,
                                              n_pm=n, assign=greem.ASSIGN_TSC))
    torch.cuda.synchronize()
    s = (pp + pmf).cpu().numpy().astype(np.float64)
    b = both.cpu().numpy().astype(np.float64)
    scale = np.linalg.norm(s, axis=1)
    # the PM assignment adds with FP32 atomics in no fixed order, so two PM evaluations of
    # the same particles differ at the 1e-7 level of the PM field (up to 4e-7 of its
    # largest value here); where PP and PM nearly cancel that is the whole difference
    pm_rms = float(np.sqrt(np.mean(np.sum(pmf.cpu().numpy().astype(np.float64) ** 2, axis=1))))
    assert np.all(np.linalg.norm(b - s, axis=1) <= 1e-5 * scale + 2e-6 * pm_rms)


def test_treepm_graph_replay_equals_direct_call(ctx):
    """The one-call TreePM step captured as a CUDA graph (the 512^3 benchmark runs it this
    way) replays to the direct call's result on new positions."""
    pos, mass = clustered(20000, 9)
    n, rc = 32, 3.0 / 32
    p = greem.params(L=1.0, r_cut=rc, theta=0.5, n_crit=64, flags=greem.FLAG_ADD_PM, n_pm=n,
                     assign=greem.ASSIGN_TSC)
    P, M = _t(pos, np.float64), _t(mass, np.float32)
    acc = torch.zeros((len(pos), 3), dtype=torch.float32, device="cuda")
    ctx.short_force(P, M, p, acc)   # plans and tables exist before the capture
    ctx.graph_capture(P, M, p, acc)
    newpos = np.mod(pos + 0.0037, 1.0)
    P.copy_(_t(newpos, np.float64))
    acc.zero_()
    assert ctx.graph_launch() == greem.OK
    torch.cuda.synchronize()
    g = acc.cpu().numpy().astype(np.float64)
    d = ctx.short_force(_t(newpos, np.float64), M, p).cpu().numpy().astype(np.float64)
    pmf = ctx.pm_force(P, M, 1.0, n, rc, greem.ASSIGN_TSC).cpu().numpy().astype(np.float64)
    pm_rms = float(np.sqrt(np.mean(np.sum(pmf ** 2, axis=1))))
    # the only difference allowed: the order of the PM assignment's FP32 atomics
    assert np.all(np.linalg.norm(g - d, axis=1) <= 1e-6 * np.linalg.norm(d, axis=1) + 2e-6 * pm_rms)


def test_treepm_total_force_against_ewald(ctx):
    """Total TreePM force vs the Ewald sum (Sec. 3.1.2 method): with TSC and theta = 0.5 the
    error of 90% of the particles stays below 2%, the paper's accuracy goal."""
    N = 1500
    pos, mass = clustered(N, 11)
    pos = np.mod(pos, 1.0)
    n, rc = 32, 3.0 / 32
    a = ctx.short_force(_t(pos, np.float64), _t(mass, np.float32),
                        greem.params(L=1.0, r_cut=rc, theta=0.5, n_crit=32, flags=greem.FLAG_ADD_PM, n_pm=n,
                                     assign=greem.ASSIGN_TSC))
    torch.cuda.synchronize()
    a = a.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(3)
    sample = rng.choice(N, 60, replace=False)
    errs = []
    for i in sample:
        d = pos[i][None, :] - pos        # field point minus sources
        d = np.delete(d, i, axis=0)
        m = np.delete(mass.astype(np.float64), i)
        ref = (pmo.ewald_accel(d) * m[:, None]).sum(axis=0)
        errs.append(np.linalg.norm(a[i] - ref) / np.linalg.norm(ref))
    errs = np.array(errs)
    print(f"TreePM vs Ewald: median {np.median(errs):.2e}, 90th {np.quantile(errs, 0.9):.2e}")
    assert np.quantile(errs, 0.9) < 0.02


def test_pm_invalid_arguments(ctx):
    pos, mass = clustered(100, 1)
    P, M = _t(pos, np.float64), _t(mass, np.float32)
    for args in ((1.0, 4, 0.1, 1), (1.0, 32, 0.6, 1), (0.0, 32, 0.1, 1), (1.0, 32, 0.1, 7)):
        with pytest.raises(greem.GreemError):
            ctx.pm_force(P, M, *args)


def test_treepm_error_distribution_on_a_zeldovich_set(ctx):
    """The accuracy analysis of Sec. 3.1.2 (Figs. 3-5) on a synthetic stand-in for the
    paper's 128^3 LCDM snapshot: 32^3 Zel'dovich particles with NFW halos, total TreePM
    force (PP + TSC PM, r_cut = 3 grid spacings) against the Ewald sum on 1000 particles,
    for N_PM in {16, 32, 64} and theta in {0.3, 0.5, 1.0}.  The paper's goal, 90% of the
    particles below 2% error, holds for theta <= 0.5 at every N_PM."""
    pos, mass = synth.config_zeldovich(32, 0.5 / 32, 40, synth.SEED0 + 21)
    pos = np.mod(pos, 1.0)
    N = len(pos)
    sample = np.random.default_rng(5).choice(N, 1000, replace=False)
    ref = pmo.ewald_field(pos[sample], pos, mass.astype(np.float64))
    nref = np.linalg.norm(ref, axis=1)
    P, M = _t(pos, np.float64), _t(mass, np.float32)
    rows = []
    for n in (16, 32, 64):
        for theta in (0.3, 0.5, 1.0):
            a = ctx.short_force(P, M, greem.params(L=1.0, r_cut=3.0 / n, theta=theta, n_crit=64,
                                                   flags=greem.FLAG_ADD_PM, n_pm=n, assign=greem.ASSIGN_TSC))
            torch.cuda.synchronize()
            a = a.cpu().numpy().astype(np.float64)[sample]
            e = np.linalg.norm(a - ref, axis=1) / nref
            rows.append((n, theta, np.median(e), np.quantile(e, 0.9), np.quantile(e, 0.99)))
    for n, theta, m, p90, p99 in rows:
        print(f"N_PM {n:3d} theta {theta:.1f}: median {m:.2e}  90% {p90:.2e}  99% {p99:.2e}")
    for n, theta, m, p90, p99 in rows:
        if theta <= 0.5:
            assert p90 < 0.02, (n, theta, p90)
