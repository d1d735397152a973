"""Plain FP64 numpy oracle for the PM (long-range) part of the TreePM force.

TEST INFRASTRUCTURE ONLY (imported by tests/ and bench.py's CPU legs, never by the
product path).  Written from the paper's statement of the PM step (Sec. 2.2 step 1: mass
assigned to the PM grid with TSC, potential by FFT, forces interpolated back) and from
the force split of Sec. 2.1 (Eq. 1-2: the PP part is Newton's law times g_P3M, so the PM
part must carry the complement).

Readings (the paper gives the scheme only as "same as YTPM"):
  * grid points at x = j*Delta, Delta = L/n_pm (vertex-centred), periodic;
  * CIC: weights (1-f, f) on floor(s), floor(s)+1 with s = x/Delta, f = s - floor(s);
    TSC: nearest point i = round(s), d = s - i, weights 0.5(0.5-d)^2, 0.75-d^2, 0.5(0.5+d)^2
    on i-1, i, i+1 (per axis; products over axes);
  * density rho = sum m w / Delta^3;
  * potential phi_k = G(k) rho_k with G(k) = -4 pi S(k eta)^2 / (k^2 W(k)^2), k = 0 removed:
    S(xi) = 12 (2 - 2 cos xi - xi sin xi) / xi^4 is the transform of the S2 cloud of radius
    eta whose pair force is exactly 1 - g_P3M, and W(k) = prod_a sinc(k_a Delta/2)^p
    (p = 2 CIC, 3 TSC) is divided out once for the assignment and once for the interpolation;
  * acceleration a_k = -i k phi_k (the Nyquist component of each k_a set to 0), back by
    inverse FFT, interpolated at the particles with the assignment weights.
"""
from __future__ import annotations

import numpy as np

CIC, TSC = 0, 1


def _weights(s, scheme):
    """Per-axis cell offsets and weights for scaled coordinates s (shape [N])."""
    if scheme == CIC:
        i0 = np.floor(s)
        f = s - i0
        return [i0.astype(np.int64), i0.astype(np.int64) + 1], [1.0 - f, f]
    i = np.floor(s + 0.5)
    d = s - i
    i = i.astype(np.int64)
    return [i - 1, i, i + 1], [0.5 * (0.5 - d) ** 2, 0.75 - d * d, 0.5 * (0.5 + d) ** 2]


def assign(pos, mass, L, n, scheme):
    """Mass density on the n^3 grid (mass per unit volume)."""
    d = L / n
    s = np.mod(np.asarray(pos, np.float64), L) / d
    rho = np.zeros((n, n, n))
    ix, wx = _weights(s[:, 0], scheme)
    iy, wy = _weights(s[:, 1], scheme)
    iz, wz = _weights(s[:, 2], scheme)
    m = np.asarray(mass, np.float64)
    for a, wa in zip(ix, wx):
        for b, wb in zip(iy, wy):
            for c, wc in zip(iz, wz):
                np.add.at(rho, (a % n, b % n, c % n), m * wa * wb * wc)
    return rho / d ** 3


def s2_transform(xi):
    xi = np.asarray(xi, np.float64)
    out = np.ones_like(xi)
    small = xi < 1e-2
    xs = xi[small]
    out[small] = 1.0 - xs * xs / 15.0 + xs ** 4 / 560.0
    xl = xi[~small]
    out[~small] = 12.0 * (2.0 - 2.0 * np.cos(xl) - xl * np.sin(xl)) / xl ** 4
    return out


def green(L, n, r_cut, scheme):
    """G(k) on the rfft grid [n, n, n//2+1] and the wavenumbers (kx, ky, kz)."""
    eta = 0.5 * r_cut
    d = L / n
    k1 = 2.0 * np.pi * np.fft.fftfreq(n, d=d)
    kz1 = 2.0 * np.pi * np.fft.rfftfreq(n, d=d)
    kx, ky, kz = np.meshgrid(k1, k1, kz1, indexing="ij")
    k2 = kx * kx + ky * ky + kz * kz
    p = 2 if scheme == CIC else 3
    W = (np.sinc(kx * d / (2 * np.pi)) * np.sinc(ky * d / (2 * np.pi)) * np.sinc(kz * d / (2 * np.pi))) ** p
    with np.errstate(divide="ignore", invalid="ignore"):
        G = -4.0 * np.pi * s2_transform(np.sqrt(k2) * eta) ** 2 / (k2 * W * W)
    G[0, 0, 0] = 0.0
    return G, (kx, ky, kz)


def pm_accel(pos, mass, L, n, r_cut, scheme=TSC):
    """PM acceleration [N,3] at the particles (input order), FP64."""
    rho = assign(pos, mass, L, n, scheme)
    rk = np.fft.rfftn(rho)
    G, ks = green(L, n, r_cut, scheme)
    phik = G * rk
    d = L / n
    s = np.mod(np.asarray(pos, np.float64), L) / d
    ix, wx = _weights(s[:, 0], scheme)
    iy, wy = _weights(s[:, 1], scheme)
    iz, wz = _weights(s[:, 2], scheme)
    nyq = np.pi / d
    acc = np.zeros((len(s), 3))
    for a in range(3):
        ka = ks[a].copy()
        ka[np.isclose(np.abs(ka), nyq)] = 0.0
        grid = np.fft.irfftn(-1j * ka * phik, s=(n, n, n), axes=(0, 1, 2))
        for i, wi in zip(ix, wx):
            for j, wj in zip(iy, wy):
                for k, wk in zip(iz, wz):
                    acc[:, a] += wi * wj * wk * grid[i % n, j % n, k % n]
    return acc


def ewald_accel(dr, L=1.0, alpha=None, nreal=3, kmax=7):
    """Acceleration at separations dr [M,3] from a unit mass at the origin with all its
    periodic images and a uniform neutralising background (Ewald summation; the paper's
    exact reference for the total force, Sec. 3.1.2).  G = 1."""
    from scipy.special import erfc
    dr = np.atleast_2d(np.asarray(dr, np.float64))
    if alpha is None:
        alpha = 2.0 / L
    out = np.zeros_like(dr)
    rng = range(-nreal, nreal + 1)
    for a in rng:
        for b in rng:
            for c in rng:
                x = dr - L * np.array([a, b, c])
                r = np.linalg.norm(x, axis=1)
                ok = r < (nreal + 0.6) * L
                f = (erfc(alpha * r) / r ** 2 + 2 * alpha / np.sqrt(np.pi) * np.exp(-alpha * alpha * r * r) / r)
                out[ok] -= (f / r)[ok, None] * x[ok]
    for h in range(-kmax, kmax + 1):
        for i in range(-kmax, kmax + 1):
            for j in range(-kmax, kmax + 1):
                if h == i == j == 0 or h * h + i * i + j * j > kmax * kmax:
                    continue
                k = 2 * np.pi / L * np.array([h, i, j], np.float64)
                k2 = k @ k
                out -= (4 * np.pi / L ** 3) * (np.exp(-k2 / (4 * alpha * alpha)) / k2) * \
                    np.sin(dr @ k)[:, None] * k[None, :]
    return out


def ewald_field(targets, src_pos, src_mass, L=1.0, alpha=None, kmax=None):
    """Ewald-summed acceleration at target points from all source particles, their
    periodic images and a uniform neutralising background (G = 1; Sec. 3.1.2), in the
    structure-factor form, so that every source is visited once per k and once per target:
      real space: each pair at its minimum image, with alpha L/2 = 3.5 so that erfc
        beyond the half box is below 1e-6;
      k space: sum over |n| <= kmax, k = 2 pi n / L, of the same term as ewald_accel,
        with sum_j m_j sin(k.(x_t - x_j)) = sin(k.x_t) C(k) - cos(k.x_t) S(k) from the
        source sums C, S of m cos(k.x), m sin(k.x).
    A source at a target's own position is left out of the real-space sum; its k-space
    share vanishes on its own."""
    from scipy.special import erfc
    tg = np.atleast_2d(np.asarray(targets, np.float64))
    sp = np.asarray(src_pos, np.float64)
    sm = np.asarray(src_mass, np.float64)
    if alpha is None:
        alpha = 7.0 / L
    if kmax is None:
        kmax = int(np.ceil(2.0 * alpha * np.sqrt(16.2) * L / (2 * np.pi)))
    out = np.zeros_like(tg)
    for t in range(tg.shape[0]):
        d = tg[t][None, :] - sp
        d -= np.rint(d / L) * L
        r = np.sqrt(np.sum(d * d, axis=1))
        keep = r > 0
        rk, dk, mk = r[keep], d[keep], sm[keep]
        f = erfc(alpha * rk) / rk ** 2 + 2 * alpha / np.sqrt(np.pi) * np.exp(-alpha * alpha * rk * rk) / rk
        out[t] -= ((mk * f / rk)[:, None] * dk).sum(axis=0)
    rng = np.arange(-kmax, kmax + 1)
    n = np.stack(np.meshgrid(rng, rng, rng, indexing="ij"), -1).reshape(-1, 3)
    n2 = (n * n).sum(1)
    n = n[(n2 > 0) & (n2 <= kmax * kmax)]
    k = 2 * np.pi / L * n.astype(np.float64)
    k2 = (k * k).sum(1)
    w = (4 * np.pi / L ** 3) * np.exp(-k2 / (4 * alpha * alpha)) / k2
    for c0 in range(0, k.shape[0], 256):
        kc = k[c0:c0 + 256]
        ps = sp @ kc.T                                  # [Nsrc, nk]
        C = sm @ np.cos(ps)
        S = sm @ np.sin(ps)
        pt = tg @ kc.T                                  # [Ntg, nk]
        amp = w[c0:c0 + 256] * (np.sin(pt) * C - np.cos(pt) * S)
        out -= amp @ kc
    return out
