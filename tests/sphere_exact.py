"""Closed-form Stokes layer potentials on the unit sphere for rigid-body densities.

For f = q = F + Omega x x on the unit sphere centred at the origin (standard results for a
translating / rotating sphere, independent of the paper's method):
  (1/8pi) int S f dS = (2/3) F + (1/3) Omega x y                       for |y| < 1,
                     = 1/2 (F/r + y (y.F)/r^3) + 1/6 (F/r^3 - 3 y (y.F)/r^5)
                       + (1/3) Omega x y / r^3                          for |y| >= 1,
  (1/8pi) int T q n dS = chi(y) (F + Omega x y),  chi = 1, 0, 1/2 inside, outside, on,
which is the identity behind the chi term of Eq. (Stokes_DL1).
"""
import numpy as np

F = np.array([0.3, -0.7, 0.5])
OMEGA = np.array([0.4, 0.2, -0.9])


def rigid(p):
    return F + np.cross(OMEGA, p)


def sl_exact(y):
    r = np.maximum(np.linalg.norm(y, axis=1)[:, None], 1e-3)  # outside branch only used for r >= 1
    yF = (y @ F)[:, None]
    inside = (2 / 3) * F + (1 / 3) * np.cross(OMEGA, y)
    outside = (0.5 * (F / r + y * yF / r**3) + (1 / 6) * (F / r**3 - 3 * y * yF / r**5)
               + (1 / 3) * np.cross(OMEGA, y) / r**3)
    return np.where(r < 1, inside, outside)


def dl_exact(y, b):
    chi = np.where(b < 0, 1.0, np.where(b > 0, 0.0, 0.5))[:, None]
    return chi * rigid(y)
