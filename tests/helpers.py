"""Closed forms used to pin the oracle; none of them calls the oracle."""
import numpy as np
from scipy.integrate import quad


def cap_area(r0, a, kf):
    """Area of a star cap in geodesic polar coordinates:
    int_0^{2pi} int_0^{r(t)} sin(rho) d rho dt = int_0^{2pi} (1 - cos r(t)) dt."""
    val, _ = quad(lambda t: 1.0 - np.cos(r0 * (1.0 + a * np.cos(kf * t))), 0.0, 2.0 * np.pi,
                  epsabs=1e-15, epsrel=1e-14, limit=200)
    return val


def curve_point(c, e1, e2, r0, a, kf, t):
    """A point of a star cap and its first two t-derivatives at any parameter t."""
    r = r0 * (1 + a * np.cos(kf * t))
    rp = -r0 * a * kf * np.sin(kf * t)
    rpp = -r0 * a * kf * kf * np.cos(kf * t)
    u = np.cos(t) * e1 + np.sin(t) * e2
    v = -np.sin(t) * e1 + np.cos(t) * e2
    x = np.cos(r) * c + np.sin(r) * u
    dx = -rp * np.sin(r) * c + rp * np.cos(r) * u + np.sin(r) * v
    d2x = ((-rpp * np.sin(r) - rp ** 2 * np.cos(r)) * c
           + (rpp * np.cos(r) - rp ** 2 * np.sin(r) - np.sin(r)) * u + 2 * rp * np.cos(r) * v)
    return x, dx, d2x


def max_rel(u, ref):
    return float(np.max(np.abs(np.asarray(u) - np.asarray(ref))) / np.max(np.abs(ref)))


def rel_l2(u, ref):
    return float(np.linalg.norm(np.asarray(u) - np.asarray(ref)) / np.linalg.norm(ref))


def planar_nodes(g):
    """xi, xi', xi'' of the projected nodes by the chain rule of xi = z / (1 - x3)
    (Sec. 3), as three N x 2 arrays (re, im)."""
    X, D1, D2 = g.x, g.dx, g.d2x
    z, z1, z2 = (A[:, 0] + 1j * A[:, 1] for A in (X, D1, D2))
    w, w1, w2 = 1 - X[:, 2], -D1[:, 2], -D2[:, 2]
    xi = z / w
    xi1 = z1 / w - z * w1 / w ** 2
    xi2 = z2 / w - 2 * z1 * w1 / w ** 2 - z * w2 / w ** 2 + 2 * z * w1 ** 2 / w ** 3
    return [np.stack([c.real, c.imag], axis=1) for c in (xi, xi1, xi2)]
