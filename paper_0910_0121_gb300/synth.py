"""Seeded synthetic particle sets that stand in for the paper's GRAFIC LCDM initial
conditions (Sec. 3: 128^3 / 256^3 / 512^3 particles in a periodic box), which are not
available here.

This module draws positions and masses only.  It holds none of the force method's
arithmetic, so both the CUDA path and the CPU oracle may take their inputs from it.

Recipes (box side L = 1, every particle mass 1/N so the mean density is 1):

* ``uniform``      -- positions uniform in [0, 1)^3.
* ``nfw_halos``    -- halo sizes from a power law dN/dn ~ n^-1.9 on [1e2, 1e5] by inverse
  CDF; centres uniform; concentration c ~ U(5, 15); r_200 = (3 n m / (800 pi))^(1/3)
  (mean density 200); radii by inverting mu(x) = ln(1+x) - x/(1+x) at u * mu(c) with
  x = r c / r_200 (truncated at r_200); isotropic directions; wrapped into the box.
* ``zeldovich``    -- a regular n^3 grid displaced by the Zel'dovich field psi_k = i k
  delta_k / k^2 of a Gaussian delta with P(k) ~ k^-2 (k = 0 removed), scaled to a given
  rms |psi| in grid spacings.
* ``config_*``     -- the five workloads (32^3 uniform; 128^3 uniform + 1000 halos;
  256^3 Zel'dovich + 5000 halos; 64 batched boxes; 512^3 Zel'dovich + 20000 halos).
"""
from __future__ import annotations

import math

import numpy as np

SEED0 = 9100121


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def uniform(n: int, rng: np.random.Generator) -> np.ndarray:
    return rng.random((n, 3))


def powerlaw_sizes(nh: int, rng: np.random.Generator, lo: float = 1e2, hi: float = 1e5,
                   slope: float = -1.9) -> np.ndarray:
    """Real-valued halo sizes with pdf ~ n^slope on [lo, hi] (inverse CDF)."""
    a = slope + 1.0
    u = rng.random(nh)
    return (lo ** a + u * (hi ** a - lo ** a)) ** (1.0 / a)


def integer_sizes(real_sizes: np.ndarray, total: int | None) -> np.ndarray:
    """Round sizes to integers >= 1; if ``total`` is given rescale so they sum to it
    exactly, the remainder going to the largest fractional parts."""
    s = np.asarray(real_sizes, dtype=np.float64)
    if total is None:
        return np.maximum(1, np.rint(s)).astype(np.int64)
    f = s * (total / s.sum())
    base = np.floor(f).astype(np.int64)
    rem = int(total - base.sum())
    if rem > 0:
        order = np.argsort(-(f - base), kind="stable")
        base[order[:rem]] += 1
    elif rem < 0:
        order = np.argsort(f - base, kind="stable")
        k = 0
        while rem < 0:
            j = order[k % len(order)]
            if base[j] > 0:
                base[j] -= 1
                rem += 1
            k += 1
    return base


def _nfw_mu(x):
    return np.log1p(x) - x / (1.0 + x)


def nfw_radii(c: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    """x in [0, c] with mu(x) = u mu(c), by bisection (vectorised)."""
    y = rng.random(c.shape[0]) * _nfw_mu(c)
    lo = np.zeros_like(c)
    hi = c.copy()
    for _ in range(64):
        mid = 0.5 * (lo + hi)
        below = _nfw_mu(mid) < y
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    return 0.5 * (lo + hi)


def nfw_halos(sizes: np.ndarray, m_particle: float, rng: np.random.Generator) -> np.ndarray:
    """Particles of NFW halos with the given integer sizes, wrapped into [0,1)^3."""
    sizes = np.asarray(sizes, dtype=np.int64)
    nh = sizes.shape[0]
    centres = rng.random((nh, 3))
    conc = rng.uniform(5.0, 15.0, nh)
    r200 = (3.0 * sizes * m_particle / (800.0 * math.pi)) ** (1.0 / 3.0)
    owner = np.repeat(np.arange(nh), sizes)
    x = nfw_radii(conc[owner], rng)
    r = x * r200[owner] / conc[owner]
    v = rng.standard_normal((owner.shape[0], 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    p = centres[owner] + v * r[:, None]
    return np.mod(p, 1.0)


def zeldovich(n: int, rms_spacing: float, rng: np.random.Generator) -> np.ndarray:
    """n^3 grid at (i+1/2)/n displaced by a Zel'dovich field with P(k) ~ k^-2."""
    k1 = 2.0 * np.pi * np.fft.fftfreq(n, d=1.0 / n)
    kz1 = 2.0 * np.pi * np.fft.rfftfreq(n, d=1.0 / n)
    kx = k1[:, None, None]
    ky = k1[None, :, None]
    kz = kz1[None, None, :]
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    shape = (n, n, n // 2 + 1)
    amp = 1.0 / np.sqrt(k2)  # sqrt(P), P ~ k^-2
    delta = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * amp
    delta[0, 0, 0] = 0.0
    inv = 1.0 / k2
    psi = np.empty((n, n, n, 3), dtype=np.float64)
    for a, ka in enumerate((kx, ky, kz)):
        psi[..., a] = np.fft.irfftn(1j * ka * delta * inv, s=(n, n, n), axes=(0, 1, 2))
    psi = psi.reshape(-1, 3)
    rms = np.sqrt(np.mean(np.sum(psi * psi, axis=1)))
    psi *= (rms_spacing / n) / rms
    q = (np.arange(n) + 0.5) / n
    grid = np.stack(np.meshgrid(q, q, q, indexing="ij"), axis=-1).reshape(-1, 3)
    return np.mod(grid + psi, 1.0)


def _masses(n: int) -> np.ndarray:
    return np.full(n, 1.0 / n, dtype=np.float32)


# --------------------------------------------------------------------------- workloads
def config_uniform32(seed: int = SEED0 + 1):
    """32^3 uniform, r_cut = 3/32, theta = 0.5, n_crit = 64."""
    rng = _rng(seed)
    n = 32 ** 3
    return uniform(n, rng), _masses(n), dict(L=1.0, r_cut=3.0 / 32, theta=0.5, n_crit=64, n_leaf=10)


def config_nfw128(seed: int = SEED0 + 2, n_side: int = 128, n_halos: int = 1000):
    """n_side^3 particles, half uniform, half in power-law NFW halos (default 128^3, 1000 halos)."""
    rng = _rng(seed)
    n = n_side ** 3
    nu = n // 2
    sizes = integer_sizes(powerlaw_sizes(n_halos, rng), n - nu)
    pos = np.concatenate([uniform(nu, rng), nfw_halos(sizes, 1.0 / n, rng)])
    return pos, _masses(n), dict(L=1.0, r_cut=3.0 / n_side, theta=0.5, n_crit=64, n_leaf=10)


def config_zeldovich(n_side: int, rms_spacing: float, n_halos: int, seed: int):
    rng = _rng(seed)
    n = n_side ** 3
    pos = zeldovich(n_side, rms_spacing, rng)
    sizes = integer_sizes(powerlaw_sizes(n_halos, rng), None)
    if sizes.sum() > n // 2:
        sizes = integer_sizes(sizes, n // 2)
    halo = nfw_halos(sizes, 1.0 / n, rng)
    replace = rng.choice(n, size=halo.shape[0], replace=False)
    pos[replace] = halo
    return pos, _masses(n)


def config_zel256(seed: int = SEED0 + 3, theta: float = 0.5):
    """256^3 Zel'dovich (rms 0.5 spacing) + 5000 NFW halos replacing grid particles."""
    pos, m = config_zeldovich(256, 0.5, 5000, seed)
    return pos, m, dict(L=1.0, r_cut=3.0 / 256, theta=theta, n_crit=0, n_leaf=10)


def config_batched(seed: int = SEED0 + 4, nbox: int = 64):
    """nbox boxes, N_b log-uniform in [16^3, 96^3], each half uniform + half halos.
    Returns (pos, mass, offsets[nbox+1], per-box params list)."""
    rng = _rng(seed)
    nb = np.rint(np.exp(rng.uniform(np.log(16 ** 3), np.log(96 ** 3), nbox))).astype(np.int64)
    pos_l, m_l, prm = [], [], []
    for b in range(nbox):
        n = int(nb[b])
        nu = n - n // 2
        nh = max(1, int(round(1000 * n / 128 ** 3)))
        real = np.minimum(powerlaw_sizes(nh, rng), n / 2)
        sizes = integer_sizes(real, n // 2)
        p = np.concatenate([uniform(nu, rng), nfw_halos(sizes, 1.0 / n, rng)]) if n // 2 else uniform(n, rng)
        pos_l.append(p)
        m_l.append(_masses(n))
        prm.append(dict(L=1.0, r_cut=3.0 / n ** (1.0 / 3.0), theta=0.5, n_crit=0, n_leaf=10))
    off = np.zeros(nbox + 1, np.int64)
    off[1:] = np.cumsum(nb)
    return np.concatenate(pos_l), np.concatenate(m_l), off, prm


def config_zel512(seed: int = SEED0 + 5):
    """512^3 Zel'dovich (rms 1.0 spacing) + 20000 NFW halos."""
    pos, m = config_zeldovich(512, 1.0, 20000, seed)
    return pos, m, dict(L=1.0, r_cut=3.0 / 512, theta=0.5, n_crit=0, n_leaf=10)


def e1_pairs(n_i: int = 256, n_j: int = 1024, r_cut: float = 5.859375e-3, seed: int = SEED0 + 11):
    """The pairwise-error experiment of Sec. 3.1.1 (Fig. 2): group centres x_g uniform
    in the unit cube, x_i uniform in a cube of side 1/128 about x_g, x_j at a random
    direction from x_i with log10(distance / r_cut) uniform in [-6, 0].
    Returns xg [P,3], xi [P,3], xj [P,3], m [P] for every (i, j) pair, P = n_i n_j."""
    rng = _rng(seed)
    xg = rng.random((n_i, 3))
    xi = xg + (rng.random((n_i, 3)) - 0.5) / 128.0
    r = r_cut * 10.0 ** rng.uniform(-6.0, 0.0, (n_i, n_j))
    v = rng.standard_normal((n_i, n_j, 3))
    v /= np.linalg.norm(v, axis=2, keepdims=True)
    xj = xi[:, None, :] + v * r[..., None]
    P = n_i * n_j
    return (np.repeat(xg, n_j, axis=0), np.repeat(xi, n_j, axis=0), xj.reshape(P, 3),
            np.ones(P, np.float32))
