"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

None of these retypes the oracle's own formulas: each compares it with an
independent fact (a Fourier-space derivation of Eq. 2, continuity of the two
branches, Newton's third law, lattice symmetry, a brute-force minimum-image sum,
a bit-by-bit key built from exact rationals, list completeness by brute force).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_0910_0121_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- Eq. 2
def test_g_golden_rationals():
    """Eq. 2 at rational points (tests/golden/g_p3m_eq2.txt, worked from the printed branches)."""
    rows = []
    for line in open(os.path.join(GOLDEN, "g_p3m_eq2.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        r, g = line.split()
        rows.append((Fraction(r), Fraction(g)))
    assert len(rows) >= 6
    for R, g in rows:
        assert oracle.g_p3m(float(R)) == pytest.approx(float(g), rel=1e-15, abs=1e-16)


def _shat(x):
    """Fourier transform of the S2 cloud of radius eta, x = k eta (Hockney & Eastwood)."""
    if x < 1e-2:
        return 1.0 - x * x / 15.0 + x ** 4 / 560.0
    return 12.0 / x ** 4 * (2.0 - 2.0 * math.cos(x) - x * math.sin(x))


def _j1(x):
    if x < 1e-3:
        return x / 3.0
    return math.sin(x) / x ** 2 - math.cos(x) / x


def test_g_equals_s2_cloud_complement():
    """g_P3M(R) = 1 - r^2 F_S2(r): the force between two S2 clouds of radius eta, from
    F(r) = (2/pi) int S(k)^2 k j1(kr) dk, must be the Newtonian force minus the PP part
    (Sec. 2.1: the PP part is Eq. 1 with the cutoff of Eq. 2)."""
    from scipy.integrate import quad

    edges = np.linspace(0.0, 400.0, 2001)
    for R in (0.25, 0.5, 0.75, 1.0, 1.25, 1.5, 1.9, 2.3):
        f = lambda k: _shat(k) ** 2 * k * _j1(k * R)
        tot = sum(quad(f, lo, hi, epsabs=1e-14, epsrel=1e-12, limit=200)[0]
                  for lo, hi in zip(edges[:-1], edges[1:]))
        g_fourier = 1.0 - R * R * 2.0 / math.pi * tot
        assert oracle.g_p3m(R) == pytest.approx(g_fourier, abs=2e-9), R


def test_g_smooth_at_branch_points():
    """Both branches of Eq. 2 meet with equal value, slope and curvature at R=1, and
    g, g', g'' vanish at R=2 (the S2 cutoff is C^2)."""
    h = 1e-4
    for R0 in (1.0, 2.0):
        gl = [oracle.g_p3m(R0 - k * h) for k in range(3)]
        gr = [oracle.g_p3m(R0 + k * h) for k in range(3)] if R0 == 1.0 else None
        # one-sided derivatives from the inner branch
        d1l = (3 * gl[0] - 4 * gl[1] + gl[2]) / (2 * h)
        d2l = (gl[0] - 2 * gl[1] + gl[2]) / h ** 2
        if R0 == 1.0:
            d1r = (-3 * gr[0] + 4 * gr[1] - gr[2]) / (2 * h)
            d2r = (gr[0] - 2 * gr[1] + gr[2]) / h ** 2
            assert abs(d1l - d1r) < 1e-6
            assert abs(d2l - d2r) < 1e-3
        else:
            assert abs(gl[0]) < 1e-15
            assert abs(d1l) < 1e-6
            assert abs(d2l) < 1e-3
    assert oracle.g_p3m(0.0) == 1.0
    assert oracle.g_p3m(1e-3) == pytest.approx(1.0, abs=2e-9)  # Newtonian at r << eta


# --------------------------------------------------------------------------- Eq. 1, two bodies
def test_two_body_direct_sum():
    """Direct sum for two particles: attractive, along the separation, magnitude
    m g(r/eta)/r^2, zero at and beyond r_cut, through the periodic boundary too."""
    L, rc = 1.0, 0.1
    eta = rc / 2
    for r in (1e-4, 0.01, 0.05, 0.07, 0.0999, 0.1, 0.2):
        for x0 in (0.3, 0.99):  # 0.99 puts the partner across the boundary
            pos = np.array([[x0, 0.5, 0.5], [x0 + r, 0.5, 0.5]])
            m = np.array([0.25, 0.5], np.float32)
            a = oracle.direct(pos, m, L, rc)
            mag = 0.5 * oracle.g_p3m(r / eta) / r ** 2
            # g is steep near R = 2, so compare on the Newtonian scale m/r^2 there
            tol = 1e-12 * (0.5 / r ** 2)
            assert a[0, 0] == pytest.approx(mag, rel=1e-12, abs=tol)
            assert a[1, 0] == pytest.approx(-0.25 / 0.5 * mag, rel=1e-12, abs=tol)
            assert np.all(a[:, 1:] == 0)
            if r >= rc:
                assert np.all(a == 0)
    # Newtonian limit
    pos = np.array([[0.2, 0.2, 0.2], [0.2, 0.2 + 1e-6, 0.2]])
    a = oracle.direct(pos, np.ones(2, np.float32), L, rc)
    assert a[0, 1] == pytest.approx(1.0 / 1e-12, rel=1e-9)


def test_momentum_conservation_direct():
    """Pair antisymmetry of Eq. 1: sum_i m_i a_i = 0."""
    rng = np.random.default_rng(5)
    N = 600
    pos = rng.random((N, 3))
    pos[:100] = 0.5 + 0.01 * rng.standard_normal((100, 3))
    m = rng.uniform(0.5, 2.0, N).astype(np.float32)
    a = oracle.direct(pos, m, 1.0, 0.15)
    p = (m[:, None].astype(np.float64) * a).sum(axis=0)
    scale = (m[:, None] * np.abs(a)).sum()
    assert np.all(np.abs(p) < 1e-13 * scale)


def test_direct_sum_at_selected_particles_is_the_direct_sum():
    """direct_at (the O(N)-per-particle sum used for the tree-against-direct error at full
    size) returns exactly the rows of the pinned all-pairs sum, in the order asked."""
    rng = np.random.default_rng(3)
    pos = rng.random((700, 3)) * 2.0 - 0.5          # some outside [0, L): wrapped
    m = rng.uniform(0.5, 1.5, 700).astype(np.float32)
    full = oracle.direct(pos, m, 1.0, 0.2, eps=1e-3)
    idx = np.array([699, 0, 350, 17, 17])
    assert np.array_equal(oracle.direct_at(pos, m, 1.0, 0.2, idx, eps=1e-3), full[idx])
    with pytest.raises(ValueError):
        oracle.direct_at(pos, m, 1.0, 0.2, [700])


def test_lattice_zero_force():
    """A perfect periodic n^3 lattice has zero short-range force by symmetry."""
    n = 10
    q = (np.arange(n) + 0.5) / n
    pos = np.stack(np.meshgrid(q, q, q, indexing="ij"), -1).reshape(-1, 3)
    a = oracle.direct(pos, np.full(n ** 3, 1.0 / n ** 3, np.float32), 1.0, 0.3)
    ref = (1.0 / n ** 3) / (1.0 / n) ** 2
    assert np.abs(a).max() < 1e-12 * ref


def test_softening_reduces_to_plummer_inside():
    """With eps > 0 and r << eta, the pair force is the Plummer form m r/(r^2+eps^2)^1.5."""
    d = np.array([1e-4, 0, 0])
    a = oracle.pair_accel(d, 2.0, eta=0.05, eps=3e-4)
    assert a[0] == pytest.approx(2.0 * 1e-4 / (1e-8 + 9e-8) ** 1.5 * oracle.g_p3m(1e-4 / 0.05), rel=1e-12)


# --------------------------------------------------------------------------- keys and sort
def _key_exact(x, y, z):
    """Reference key from exact rationals: floor(x * 2^21) per axis for L=1, bits
    interleaved with x as the high bit of each triplet, clamped to 2^21-1."""
    ii = []
    for v in (x, y, z):
        f = Fraction(v)
        f = f - math.floor(f)  # periodic wrap into [0,1) on the exact value
        i = math.floor(f * 2 ** 21)
        ii.append(min(i, 2 ** 21 - 1))
    bits = []
    for b in range(20, -1, -1):
        bits += [(ii[0] >> b) & 1, (ii[1] >> b) & 1, (ii[2] >> b) & 1]
    return int("".join(map(str, bits)), 2)


def _interleave(ix, iy, iz, nbits):
    """Bits of three nbits-bit indices interleaved (x high), as a string of digits."""
    if nbits == 0:
        return 0
    s = "".join(f"{(ix >> b) & 1}{(iy >> b) & 1}{(iz >> b) & 1}" for b in range(nbits - 1, -1, -1))
    return int(s, 2)


def test_keys_hand_positions():
    ulp = np.nextafter(1.0, 0.0)
    pts = [(0.0, 0.0, 0.0), (0.5, 0.25, 0.125), (ulp, ulp, ulp), (0.999, 1e-9, 0.5),
           (1.5, -0.25, 2.75), (0.3, 0.7, 0.1), (2 ** -21, 2 ** -22, 3 * 2 ** -21)]
    for p in pts:
        w = [oracle.wrap(v, 1.0) for v in p]
        k = oracle.morton(*[oracle.cell_index(v, 1.0) for v in w])
        assert k == _key_exact(*p), p
    # x == L and tiny negatives wrap to 0
    assert oracle.wrap(1.0, 1.0) == 0.0
    assert oracle.wrap(-1e-20, 1.0) == 0.0
    assert oracle.wrap(-0.25, 1.0) == 0.75
    assert 0.0 <= oracle.wrap(-1e-300, 3.0) < 3.0


def test_sort_is_stable_key_order():
    rng = np.random.default_rng(2)
    N = 3000
    pos = np.floor(rng.random((N, 3)) * 4) / 4 + 0.01  # many equal keys
    t = oracle.Tree(pos, np.ones(N, np.float32), 1.0, 0.1, n_crit=16)
    key, perm, xyz, _ = t.sorted()
    ref = np.array([_key_exact(*p) for p in pos], dtype=np.uint64)
    assert np.array_equal(perm, np.argsort(ref, kind="stable"))
    assert np.array_equal(key, ref[perm])
    assert np.array_equal(xyz, pos[perm])


# --------------------------------------------------------------------------- tree
def _cells_by_definition(keys, n_leaf, lmin):
    """Brute-force node set: the non-empty cells (level, prefix) all of whose proper
    ancestors are split (count >= n_leaf or level < lmin), levels 0..21."""
    keys = [int(k) for k in keys]
    out = set()
    for k in range(22):
        pref = {}
        for key in keys:
            p = key >> (3 * (21 - k))
            pref[p] = pref.get(p, 0) + 1
        for p, c in pref.items():
            ok = True
            for a in range(k):
                pa = p >> (3 * (k - a))
                cnt = sum(1 for key in keys if key >> (3 * (21 - a)) == pa)
                if not (a < lmin or cnt >= n_leaf):
                    ok = False
                    break
            if ok:
                out.add((k, p))
    return out


@pytest.mark.parametrize("seed,N,n_leaf", [(1, 40, 4), (2, 64, 10), (3, 50, 2)])
def test_tree_matches_definition(seed, N, n_leaf):
    rng = np.random.default_rng(seed)
    pos = rng.random((N, 3))
    pos[: N // 3] = 0.3 + 1e-5 * rng.random((N // 3, 3))  # a tight clump -> deep levels
    t = oracle.Tree(pos, np.ones(N, np.float32), 1.0, 0.1, n_crit=8, n_leaf=n_leaf)
    key, _, _, _ = t.sorted()
    nodes = t.nodes()
    got = set()
    for lvl, ix, iy, iz, b, e, skip, leaf, _ in nodes:
        p = _interleave(int(ix), int(iy), int(iz), int(lvl))
        got.add((int(lvl), p))
        # the node's particles are exactly those with that prefix
        pk = [int(k) >> (3 * (21 - lvl)) for k in key]
        assert all(pk[j] == p for j in range(b, e))
        assert (b == 0 or pk[b - 1] != p) and (e == N or pk[e] != p)
        cnt = e - b
        assert leaf == (lvl == 21 or (lvl >= t.lmin and cnt < n_leaf))
    assert got == _cells_by_definition(key, n_leaf, t.lmin)
    # preorder + skip: node n's subtree is (n, skip) and children tile the range
    for n, row in enumerate(nodes):
        lvl, b, e, skip, leaf = row[0], row[4], row[5], row[6], row[7]
        kids = []
        c = n + 1
        while c < skip:
            kids.append(c)
            c = nodes[c, 6]
        if leaf:
            assert skip == n + 1
        else:
            assert kids and nodes[kids[0], 4] == b and nodes[kids[-1], 5] == e
            for c0, c1 in zip(kids[:-1], kids[1:]):
                assert nodes[c0, 5] == nodes[c1, 4]
            assert all(nodes[c, 0] == lvl + 1 for c in kids)


def test_moments_and_groups():
    pos, m, prm = synth.config_uniform32()
    pos, m = pos[:5000], m[:5000] * 7.0
    t = oracle.Tree(pos, m, prm["L"], prm["r_cut"], n_crit=prm["n_crit"])
    _, _, xyz, ms = t.sorted()
    nodes, mom, grp = t.nodes(), t.moments(), t.groups()
    for n in range(0, len(nodes), 7):
        b, e = nodes[n, 4], nodes[n, 5]
        M = ms[b:e].astype(np.float64).sum()
        assert mom[n, 0] == pytest.approx(M, rel=1e-13)
        com = (ms[b:e, None].astype(np.float64) * xyz[b:e]).sum(0) / M
        assert np.allclose(mom[n, 1:], com, rtol=0, atol=1e-13)
    # groups tile [0, N) in order, satisfy the rule, and are maximal
    b = [nodes[g, 4] for g in grp]
    e = [nodes[g, 5] for g in grp]
    assert b[0] == 0 and e[-1] == len(pos) and all(x == y for x, y in zip(e[:-1], b[1:]))
    for g in grp:
        assert nodes[g, 0] >= t.lmin and (nodes[g, 5] - nodes[g, 4] <= 64 or nodes[g, 7])
    # mean group size ~ n_crit/4 (Sec. 3.1.2, after Makino 1991), loosely
    mean = len(pos) / len(grp)
    assert 64 / 8 < mean < 64 / 1.5


# --------------------------------------------------------------------------- lists and force
def _clustered(N, seed):
    rng = np.random.default_rng(seed)
    pos = rng.random((N, 3))
    k = N // 4
    pos[:k] = np.mod(0.02 + 0.01 * rng.standard_normal((k, 3)), 1.0)  # a clump across a corner
    return pos, rng.uniform(0.5, 1.5, N).astype(np.float32) / N


@pytest.mark.parametrize("n_crit", [1, 16, 200])
def test_theta_zero_tree_equals_direct_sum(n_crit):
    """theta = 0 opens every node that is not pruned, so the list force must equal the
    brute-force minimum-image sum (only the summation order differs)."""
    N = 1500
    pos, m = _clustered(N, 11)
    L, rc = 1.0, 0.12
    ref = oracle.direct(pos, m, L, rc)
    got = oracle.short_force(pos, m, L, rc, theta=0.0, n_crit=n_crit)
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() < 1e-12 * scale


def test_list_completeness_and_disjointness():
    """Every particle within r_cut (minimum image) of a group particle is covered by
    exactly one list entry; entries never overlap."""
    N = 800
    pos, m = _clustered(N, 3)
    L, rc = 1.0, 0.15
    t = oracle.Tree(pos, m, L, rc, n_crit=12)
    t.build_lists(0.6)
    off, kind, idx, sh = t.lists()
    nodes = t.nodes()
    _, _, xyz, _ = t.sorted()
    grp = t.groups()
    for gi in range(0, len(grp), 3):
        cov = np.zeros(N, np.int64)
        for e in range(off[gi], off[gi + 1]):
            if kind[e] == 0:
                cov[idx[e]] += 1
            else:
                cov[nodes[idx[e], 4]:nodes[idx[e], 5]] += 1
        assert cov.max() <= 1
        b, e_ = nodes[grp[gi], 4], nodes[grp[gi], 5]
        d = xyz[None, :, :] - xyz[b:e_, None, :]
        d -= np.rint(d / L) * L
        near = (np.sqrt((d * d).sum(-1)) < rc).any(0)
        assert np.all(cov[near] == 1)


def _box_distance(alo, ahi, blo, bhi, L):
    """Distance between two axis-aligned boxes [alo, ahi) and [blo, bhi) in a periodic
    cube of side L: per axis the interval gap minimised over the images -L, 0, +L."""
    g2 = 0.0
    for c in range(3):
        best = np.inf
        for s in (-L, 0.0, L):
            best = np.minimum(best, np.maximum(0.0, np.maximum(alo[..., c] + s - bhi[c], blo[c] - ahi[..., c] - s)))
        g2 = g2 + best * best
    return np.sqrt(g2)


@pytest.mark.parametrize("theta", [0.0, 0.6])
def test_list_entries_lie_within_rcut_of_the_group(theta):
    """Entries are kept iff their cell (a node's cell; a particle's finest cell) comes
    within r_cut of the box of finest cells holding the group's particles.  At theta = 0
    no node is accepted, so the list is exactly that set of particles; anything farther
    adds nothing to the force (Eq. 2 is 0 beyond R = 2)."""
    N = 900
    pos, m = _clustered(N, 5)
    L, rc = 1.0, 0.11
    t = oracle.Tree(pos, m, L, rc, n_crit=14)
    t.build_lists(theta)
    off, kind, idx, sh = t.lists()
    nodes = t.nodes()
    _, _, xyz, _ = t.sorted()
    grp = t.groups()
    c = L / 2 ** 21
    cell = np.floor(xyz / c)
    nontrivial = False
    for gi in range(len(grp)):
        b, e_ = nodes[grp[gi], 4], nodes[grp[gi], 5]
        blo, bhi = cell[b:e_].min(0) * c, (cell[b:e_].max(0) + 1) * c
        ents = slice(off[gi], off[gi + 1])
        if theta == 0.0:
            assert np.all(kind[ents] == 0)
            dist = _box_distance(cell * c, (cell + 1) * c, blo, bhi, L)
            want = np.flatnonzero(dist <= rc)
            assert np.array_equal(np.sort(idx[ents]), want)
            near = np.zeros(N, bool)
            d = xyz[None, :, :] - xyz[b:e_, None, :]
            d -= np.rint(d / L) * L
            near[(np.sqrt((d * d).sum(-1)) < rc).any(0)] = True
            nontrivial |= bool(np.any(~near[want]) or len(want) < N)
        else:
            k, j = kind[ents], idx[ents]
            nj = np.where(k == 1, j, 0)
            side = L / 2.0 ** nodes[nj, 0]
            lo = np.where(k[:, None] == 0, cell[np.where(k == 0, j, 0)] * c, nodes[nj, 1:4] * side[:, None])
            hi = np.where(k[:, None] == 0, lo + c, lo + side[:, None])
            nontrivial |= bool(np.any(k == 1))  # here: some node was accepted
            assert np.all(_box_distance(lo, hi, blo, bhi, L) <= rc)
    assert nontrivial


def test_eq12_with_a_large_theta0_is_the_constant_theta_at_its_cap():
    """Eq. 12 (Sec. 4.1): theta(d) = min(theta_max, theta0 / sqrt(R g(R))).  R g(R) stays
    below 1 on [0, 2), so with theta0 far above theta_max the cap holds everywhere and the
    lists equal those of the constant opening angle theta_max."""
    pos, m = _clustered(1200, 21)
    t = oracle.Tree(pos, m, 1.0, 0.12, n_crit=20)
    for tmax in (0.4, 0.7):
        t.build_lists(tmax)
        ref = t.lists()
        t.build_lists(tmax, theta0=50.0)
        got = t.lists()
        for a, b in zip(ref, got):
            assert np.array_equal(a, b)


def test_eq12_accepted_nodes_meet_the_criterion_and_their_parents_do_not():
    """Brute force over the lists: every accepted node satisfies l < theta(d) d, and its
    parent (which was opened, not accepted) does not, or lies above l_min; d is the
    distance from the node's centre to the nearest point of the group cell, R = d / eta."""
    pos, m = _clustered(1500, 22)
    L, rc, t0, tmax = 1.0, 0.12, 0.2, 0.8
    t = oracle.Tree(pos, m, L, rc, n_crit=16)
    t.build_lists(tmax, theta0=t0)
    off, kind, idx, sh = t.lists()
    nodes, grp = t.nodes(), t.groups()
    # parents from the preorder layout: the innermost earlier node whose subtree holds n
    parent = np.full(len(nodes), -1, np.int64)
    stack = []
    for n in range(len(nodes)):
        while stack and nodes[stack[-1], 6] <= n:
            stack.pop()
        if stack:
            parent[n] = stack[-1]
        stack.append(n)
    lmin = oracle.lmin(L, rc)
    eta = rc / 2

    def theta_d(d):
        R = d / eta
        rg = R * np.array([oracle.g_p3m(r) for r in np.atleast_1d(R)])
        with np.errstate(divide="ignore"):
            th = np.where(rg > 0, t0 / np.sqrt(np.where(rg > 0, rg, 1.0)), np.inf)
        return np.minimum(th, tmax)

    def dist(n, g, shift):
        side_g = L / 2.0 ** nodes[g, 0]
        glo = nodes[g, 1:4] * side_g
        side = L / 2.0 ** nodes[n, 0]
        c = (nodes[n, 1:4] + 0.5) * side + shift * L
        gap = np.maximum(0.0, np.maximum(glo - c, c - (glo + side_g)))
        return np.sqrt((gap * gap).sum()), side

    n_acc = n_par = 0
    for gi in range(len(grp)):
        g = grp[gi]
        for e in range(off[gi], off[gi + 1]):
            if kind[e] != 1:
                continue
            n = idx[e]
            d, side = dist(n, g, sh[e])
            assert side < theta_d(d)[0] * d * (1 + 1e-12)
            n_acc += 1
            p = parent[n]
            if p >= 0 and nodes[p, 0] >= lmin:
                dp, sp = dist(p, g, sh[e])
                assert sp >= theta_d(dp)[0] * dp * (1 - 1e-12)
                n_par += 1
    assert n_acc > 100 and n_par > 100


def test_list_shift_is_min_image_for_near_pairs():
    """The per-entry image shift equals the per-pair minimum image for every pair in range."""
    N = 600
    pos, m = _clustered(N, 8)
    L, rc = 1.0, 0.2
    t = oracle.Tree(pos, m, L, rc, n_crit=10)
    t.build_lists(0.0)
    off, kind, idx, sh = t.lists()
    nodes = t.nodes()
    _, _, xyz, _ = t.sorted()
    grp = t.groups()
    for gi in range(len(grp)):
        b, e_ = nodes[grp[gi], 4], nodes[grp[gi], 5]
        for e in range(off[gi], off[gi + 1]):
            j = idx[e]
            d = xyz[j] + sh[e] * L - xyz[b:e_]
            dm = xyz[j] - xyz[b:e_]
            dm -= np.rint(dm / L) * L
            r = np.sqrt((dm * dm).sum(-1))
            close = r < rc
            assert np.allclose(d[close], dm[close], atol=1e-15)


def test_tree_error_grows_with_theta():
    """The tree-vs-direct error is zero to rounding at theta = 0 and grows with the
    opening angle, roughly as a power near 2 (Sec. 3.1.2 error analysis).  Cell sides are
    powers of two, so on a small set the growth is stepwise; the exponent between
    theta = 0.3 and 0.9 is checked loosely in [1, 5]."""
    N = 12000
    rng = np.random.default_rng(21)
    pos = rng.random((N, 3))
    m = np.full(N, 1.0 / N, np.float32)
    L, rc = 1.0, 0.3
    ref = oracle.direct(pos, m, L, rc)
    ths = (0.0, 0.3, 0.45, 0.6, 0.9)
    errs = []
    for th in ths:
        a = oracle.short_force(pos, m, L, rc, th, n_crit=32)
        errs.append(np.median(np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)))
    assert errs[0] < 1e-13
    assert all(e1 < e2 for e1, e2 in zip(errs[1:-1], errs[2:])), errs
    expo = math.log(errs[-1] / errs[1]) / math.log(ths[-1] / ths[1])
    assert 1.0 <= expo <= 5.0, (errs, expo)


def test_invalid_arguments_rejected():
    pos = np.random.default_rng(0).random((10, 3))
    m = np.ones(10, np.float32)
    with pytest.raises(ValueError):
        oracle.Tree(pos, m, 1.0, 0.5, 8)  # r_cut must be < L/2
    bad = pos.copy()
    bad[3, 1] = np.nan
    with pytest.raises(ValueError):
        oracle.Tree(bad, m, 1.0, 0.1, 8)


def test_eq12_lowers_the_error_tail_at_equal_cost():
    """Sec. 4.1: the tree-force error comes mostly from nodes at distances around eta, and
    Eq. 12 spreads it evenly.  On a 32^3 NFW mix, theta0 = 0.25 capped at 0.7 costs the
    same number of interactions as theta = 0.5 (within 5%) and has a smaller 99th
    percentile and RMS of the relative error against the brute-force sum."""
    from paper_0910_0121_gb300 import synth
    pos, m, prm = synth.config_nfw128(n_side=32, n_halos=30)
    L, rc = 1.0, prm["r_cut"]
    ref = oracle.direct(pos, m, L, rc)
    t = oracle.Tree(pos, m, L, rc, n_crit=64)
    _, perm, _, _ = t.sorted()
    nodes, grp = t.nodes(), t.groups()
    counts = nodes[grp, 5] - nodes[grp, 4]

    def run(**kw):
        t.build_lists(**kw)
        off = t.lists()[0]
        a = np.zeros((len(pos), 3))
        a[perm] = t.list_force()
        n = np.linalg.norm(ref, axis=1)
        keep = n > 1e-6 * np.median(n)
        e = np.linalg.norm(a - ref, axis=1)[keep] / n[keep]
        return np.sum(np.diff(off) * counts) / len(pos), np.quantile(e, 0.99), np.sqrt(np.mean(e * e))

    n_c, p99_c, rms_c = run(theta=0.5)
    n_v, p99_v, rms_v = run(theta=0.7, theta0=0.25)
    assert abs(n_v / n_c - 1) < 0.05, (n_c, n_v)
    assert p99_v < 0.85 * p99_c, (p99_c, p99_v)
    assert rms_v < rms_c, (rms_c, rms_v)


def test_g_derivatives_match_finite_differences():
    """g' and g'' (needed by the second-order terms, Sec. 4.1) against centred differences
    of Eq. 2 itself, on both branches and across R = 1; both vanish at R = 2."""
    for R in np.concatenate([np.linspace(0.01, 0.99, 23), np.linspace(1.01, 1.99, 23)]):
        h = 1e-5
        d1 = (oracle.g_p3m(R + h) - oracle.g_p3m(R - h)) / (2 * h)
        d2 = (oracle.g_p3m(R + h) - 2 * oracle.g_p3m(R) + oracle.g_p3m(R - h)) / (h * h)
        assert oracle.g_p3m_d1(R) == pytest.approx(d1, abs=1e-8)
        assert oracle.g_p3m_d2(R) == pytest.approx(d2, abs=2e-4)
    for R in (1.0 - 1e-12, 1.0 + 1e-12):
        assert oracle.g_p3m_d1(R) == pytest.approx(-1.0, abs=1e-9)
    assert abs(oracle.g_p3m_d1(2.0 - 1e-9)) < 1e-30 and abs(oracle.g_p3m_d2(2.0 - 1e-9)) < 1e-20


@pytest.mark.parametrize("R0", [0.4, 1.0, 1.6])
def test_quadrupole_term_converges_at_third_order(R0):
    """A small cloud of particles at distance R0*eta: the monopole's error against the
    brute-force sum falls as (s/r)^2 with the cloud size s; with the second-order terms
    of Sec. 4.1 it falls as (s/r)^3."""
    rng = np.random.default_rng(int(R0 * 10))
    eta = 0.05
    base = rng.standard_normal((12, 3))
    mass = rng.uniform(0.5, 1.5, 12)
    direction = np.array([0.48, -0.6, 0.64])
    errs_m, errs_q = [], []
    for s in (0.02, 0.01, 0.005):
        off = base * s * eta
        off -= (mass[:, None] * off).sum(0) / mass.sum()
        com = R0 * eta * direction
        pts = com + off
        exact = sum(oracle.pair_accel(p, m, eta) for p, m in zip(pts, mass))
        mono = oracle.pair_accel(com, mass.sum(), eta)
        q = np.array([np.sum(mass * off[:, a] * off[:, b]) for a, b in ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))])
        quad = mono + oracle.quad_accel(com, q, eta)
        errs_m.append(np.linalg.norm(mono - exact))
        errs_q.append(np.linalg.norm(quad - exact))
    for k in range(2):
        assert errs_m[k] / errs_m[k + 1] == pytest.approx(4.0, rel=0.1)
        assert errs_q[k] / errs_q[k + 1] == pytest.approx(8.0, rel=0.15)
    assert errs_q[-1] < 0.05 * errs_m[-1]


def test_quadrupole_lowers_the_tree_error():
    """Sec. 4.1: the second-order terms improve the accuracy a lot.  On a clustered set at
    theta = 0.7 the 99th percentile and the RMS of the relative error against the
    brute-force sum drop by more than 3x with the same lists (most particles' lists hold
    only particles, so the median is at rounding level either way)."""
    pos, m = _clustered(3000, 31)
    L, rc = 1.0, 0.1
    ref = oracle.direct(pos, m, L, rc)
    t = oracle.Tree(pos, m, L, rc, n_crit=24)
    t.build_lists(0.7)

    def err(a):
        n = np.linalg.norm(ref, axis=1)
        keep = n > 1e-6 * np.median(n)
        e = np.linalg.norm(a - ref, axis=1)[keep] / n[keep]
        return np.sqrt(np.mean(e * e)), np.quantile(e, 0.99)

    r0, p0 = err(t.list_force_input_order())
    r1, p1 = err(t.list_force_input_order(quad=True))
    assert r1 < r0 / 3 and p1 < p0 / 3, (r0, r1, p0, p1)


# --------------------------------------------------------------------------- second moments
_QSLOTS = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))


def _qmat(q):
    """3x3 symmetric matrix from the six slots xx, yy, zz, xy, xz, yz."""
    out = np.zeros((3, 3))
    for k, (a, b) in enumerate(_QSLOTS):
        out[a, b] = out[b, a] = q[k]
    return out


def test_second_moments_match_their_definition_on_every_node():
    """Sec. 4.1 second-order terms: Q of each node is sum m (x - COM)(x - COM)^T over the
    node's particles, with the COM recomputed here from the sorted particles (not taken
    from the oracle), on a clustered set whose nodes span every level from the root to
    the leaves."""
    pos, m = _clustered(3000, 41)
    t = oracle.Tree(pos, m, 1.0, 0.1, n_crit=24)
    _, _, xyz, ms = t.sorted()
    nodes, Q = t.nodes(), t.quadrupoles()
    assert Q.shape == (len(nodes), 6)
    mm = ms.astype(np.float64)
    for n in range(len(nodes)):
        b, e = nodes[n, 4], nodes[n, 5]
        w = mm[b:e]
        com = (w[:, None] * xyz[b:e]).sum(0) / w.sum()
        d = xyz[b:e] - com
        ref = np.einsum("i,ia,ib->ab", w, d, d)
        scale = w.sum() * max(np.abs(d).max(), 1e-300) ** 2
        assert np.abs(_qmat(Q[n]) - ref).max() <= 1e-12 * scale, n


def test_second_moments_obey_the_parallel_axis_identity():
    """The second moments of a parent about its COM equal the sum over its children of
    Q_c + M_c (c_c - c_p)(c_c - c_p)^T: holds only if every node's Q is taken about its
    own centre of mass with the slots in the same order."""
    pos, m = _clustered(2500, 43)
    t = oracle.Tree(pos, m, 1.0, 0.1, n_crit=24)
    nodes, mom, Q = t.nodes(), t.moments(), t.quadrupoles()
    checked = 0
    for p in range(len(nodes)):
        if nodes[p, 7]:  # leaf
            continue
        kids, c = [], p + 1
        while c < nodes[p, 6]:
            kids.append(c)
            c = nodes[c, 6]
        acc = np.zeros((3, 3))
        for c in kids:
            d = mom[c, 1:] - mom[p, 1:]
            acc += _qmat(Q[c]) + mom[c, 0] * np.outer(d, d)
        ref = _qmat(Q[p])
        assert np.abs(acc - ref).max() <= 1e-11 * max(np.abs(ref).max(), 1e-300), p
        checked += 1
    assert checked > 50


def test_second_moments_of_a_point_symmetric_cloud_in_closed_form():
    """Four equal masses m at c +- v1 and c +- v2 have their COM at c and second moments
    2 m (v1 v1^T + v2 v2^T).  With v1 = (a, b, 0) and v2 = (0, g, h) every slot differs
    (xy = 2 m a b, xz = 0, yz = 2 m g h), so a swapped slot or a moment taken about the
    cell centre instead of the COM fails.  Exact dyadic inputs: the sums are exact."""
    a, b, g, h = 2.0 ** -6, 3 * 2.0 ** -7, 5 * 2.0 ** -8, 2.0 ** -5
    c = np.array([0.3125, 0.59375, 0.4375])   # not the centre of any cell holding the cloud
    v1, v2 = np.array([a, b, 0.0]), np.array([0.0, g, h])
    pos = np.array([c + v1, c - v1, c + v2, c - v2])
    m = np.full(4, 0.25, np.float32)
    t = oracle.Tree(pos, m, 1.0, 0.1, n_crit=4, n_leaf=10)
    mom, Q = t.moments(), t.quadrupoles()
    assert np.array_equal(mom[0, 1:], c)
    want = 2 * 0.25 * (np.outer(v1, v1) + np.outer(v2, v2))
    assert np.array_equal(_qmat(Q[0]), want)
    assert Q[0, 3] == 2 * 0.25 * a * b and Q[0, 4] == 0.0 and Q[0, 5] == 2 * 0.25 * g * h


# --------------------------------------------------------------------------- local essential trees
def _img_gap2(lo_a, hi_a, lo_b, hi_b, P):
    """Squared distance between boxes [lo_a, hi_a] and [lo_b, hi_b] (per-axis closed
    intervals) in a periodic box of side P: the smallest over the 27 images of b."""
    best = None
    for sx in (-P, 0, P):
        for sy in (-P, 0, P):
            for sz in (-P, 0, P):
                s = np.array([sx, sy, sz])
                g = np.maximum(0, np.maximum(lo_b + s - hi_a, lo_a - (hi_b + s)))
                v = float(np.sum(g.astype(np.float64) ** 2))
                best = v if best is None else min(best, v)
    return best


LET_BOX = np.array([300000, 1300000, 0, 2097152, 900000, 1700000], np.int32)


def test_let_at_theta_zero_is_every_particle_whose_cell_lies_within_rcut():
    """theta = 0 accepts no node, so the LET must be exactly the particles whose finest
    cell lies within r_cut of the box (distance taken over the periodic images)."""
    pos, m = _clustered(2500, 61)
    L, rc = 1.0, 0.11
    T = oracle.Tree(pos, m, L, rc, n_crit=32)
    kind, idx = T.let_export(LET_BOX, 0.0)
    assert np.all(kind == 0) and np.all(np.diff(idx) > 0)
    _, _, xyz, _ = T.sorted()
    f = L / 2 ** 21
    blo, bhi = LET_BOX[0::2] * f, LET_BOX[1::2] * f
    want = []
    for j in range(len(xyz)):
        c = np.array([oracle.cell_index(x, L) for x in xyz[j]])
        if _img_gap2(c * f, (c + 1) * f, blo, bhi, L) <= rc * rc:
            want.append(j)
    assert np.array_equal(idx, np.array(want))


@pytest.mark.parametrize("theta", [0.5, 0.8])
def test_let_covers_every_particle_within_rcut_once_and_accepts_by_the_criterion(theta):
    pos, m = _clustered(2500, 62)
    L, rc = 1.0, 0.2
    T = oracle.Tree(pos, m, L, rc, n_crit=32)
    kind, idx = T.let_export(LET_BOX, theta)
    assert (kind == 1).sum() > 10 and (kind == 0).sum() > 10
    nodes = T.nodes()
    _, _, xyz, _ = T.sorted()
    cover = np.zeros(len(xyz), np.int64)
    f = L / 2 ** 21
    blo, bhi = LET_BOX[0::2] * f, LET_BOX[1::2] * f
    for k, i in zip(kind, idx):
        if k == 0:
            cover[i] += 1
            continue
        lvl = nodes[i, 0]
        side = L / 2 ** lvl
        lo = nodes[i, 1:4] * side
        centre = lo + side / 2
        d2 = _img_gap2(centre, centre, blo, bhi, L)
        assert side * side < theta * theta * d2 * (1 + 1e-12)       # accepted by the criterion
        assert _img_gap2(lo, lo + side, blo, bhi, L) <= rc * rc     # not beyond r_cut
        cover[nodes[i, 4]:nodes[i, 5]] += 1
    assert cover.max() <= 1                                          # disjoint
    near = np.array([_img_gap2(p, p, blo, bhi, L) <= rc * rc for p in xyz])
    assert np.all(cover[near] == 1)                                  # complete within r_cut
    # no accepted node has an accepted ancestor: ancestors were opened
    acc_nodes = set(idx[kind == 1].tolist())
    for i in acc_nodes:
        for a in acc_nodes:
            if a != i:
                assert not (nodes[a, 4] <= nodes[i, 4] and nodes[i, 5] <= nodes[a, 5] and a < i)
