"""Plain numpy restatement of the time integration around the force (Sec. 2.2 steps 1, 6
and 7; Sec. 2.4).

TEST INFRASTRUCTURE ONLY (imported by tests/, never by the product path).

  kick:      v <- v + f_kick a, in FP32 (one product, one sum per component);
  drift:     x <- x + f_drift v, in FP64, each coordinate wrapped into [0, L) with
             r = x - L floor(x/L), then r < 0 -> r + L, r >= L -> r - L (the key's rule);
  Eq. 7:     dt = zeta min_i( sqrt(eps/|a_i|), eps/|v_i| ), |.|^2 = (x^2 + y^2) + z^2 in FP32;
  Eq. 6:     physical softening (1+z_crit)/(1+z) eps_fin for z >= z_crit, else eps_fin;
  factors:   int dt/a = int da/(a^2 H), int dt/a^2 = int da/(a^3 H),
             H = H0 sqrt(om a^-3 + (1-om-ol) a^-2 + ol)  (scipy quad).
"""
from __future__ import annotations

import numpy as np


def kick(vel, acc, f_kick):
    v = np.asarray(vel, np.float32)
    return v + np.float32(f_kick) * np.asarray(acc, np.float32)


def wrap(x, L):
    x = np.asarray(x, np.float64)
    r = x - L * np.floor(x / L)
    r = np.where(r < 0.0, r + L, r)
    r = np.where(r >= L, r - L, r)
    return np.where((r >= 0.0) & (r < L), r, 0.0)


def drift(pos, vel, L, f_drift):
    x = np.asarray(pos, np.float64) + np.float64(f_drift) * np.asarray(vel, np.float32).astype(np.float64)
    return wrap(x, L)


def _sq(v):
    v = np.asarray(v, np.float32)
    return (v[:, 0] * v[:, 0] + v[:, 1] * v[:, 1]) + v[:, 2] * v[:, 2]


def timestep(vel, acc, eps, zeta):
    v2, a2 = float(_sq(vel).max()), float(_sq(acc).max())
    dt = np.inf
    if a2 > 0:
        dt = min(dt, np.sqrt(eps / np.sqrt(a2)))
    if v2 > 0:
        dt = min(dt, eps / np.sqrt(v2))
    return zeta * dt


def softening(eps_fin, z_crit, z):
    return (1.0 + z_crit) / (1.0 + z) * eps_fin if z >= z_crit else eps_fin


def cosmo_factors(a0, a1, om, ol, h0):
    from scipy.integrate import quad
    H = lambda a: h0 * np.sqrt(om / a ** 3 + (1.0 - om - ol) / a ** 2 + ol)
    k = quad(lambda a: 1.0 / (a * a * H(a)), a0, a1, epsabs=0, epsrel=1e-13, limit=200)[0]
    d = quad(lambda a: 1.0 / (a ** 3 * H(a)), a0, a1, epsabs=0, epsrel=1e-13, limit=200)[0]
    return k, d
