"""Density weights (oracle; test infrastructure only).

Sec. 4.1: mu_omega is the Lebesgue measure of the Voronoi region of the
sampling frequency omega.  In 1D, with the frequencies sorted, the cell of
xi_m is [(xi_{m-1}+xi_m)/2, (xi_m+xi_{m+1})/2]; the outer cells are closed by
the bandwidth interval [-K, K] (the region Y_K of App. B in one dimension).
App. B: in 2D the cells partition Y_K = [-K, K]^2 and the weight is the cell's
area; the density delta is the largest distance from a point of Y_K to its
nearest sample.
"""
import numpy as np


def voronoi_1d(xi, K: float) -> np.ndarray:
    xi = np.asarray(xi, dtype=np.float64)
    order = np.argsort(xi, kind="stable")
    s = xi[order]
    mid = (s[1:] + s[:-1]) / 2.0
    lo = np.concatenate([[-K], mid])
    hi = np.concatenate([mid, [K]])
    lo = np.clip(lo, -K, K)
    hi = np.clip(hi, -K, K)
    w = np.empty_like(xi)
    w[order] = hi - lo
    return w


def _clip(poly, a, b, c):
    """The part of convex polygon poly (list of (x, y)) where a x + b y <= c."""
    out = []
    n = len(poly)
    for i in range(n):
        p, q = poly[i], poly[(i + 1) % n]
        fp = a * p[0] + b * p[1] - c
        fq = a * q[0] + b * q[1] - c
        if fp <= 0:
            out.append(p)
        if (fp < 0 < fq) or (fq < 0 < fp):
            t = fp / (fp - fq)
            out.append((p[0] + t * (q[0] - p[0]), p[1] + t * (q[1] - p[1])))
    return out


def _area(poly):
    s = 0.0
    for i in range(len(poly)):
        p, q = poly[i], poly[(i + 1) % len(poly)]
        s += p[0] * q[1] - q[0] * p[1]
    return 0.5 * abs(s)


def voronoi_cell_2d(xi, i: int, K: float):
    """App. B: the Voronoi cell of xi_i within Y_K = [-K, K]^2, written out from its
    definition: the points of Y_K no farther from xi_i than from any other xi_j,
    i.e. Y_K clipped by the half-plane |x - xi_i| <= |x - xi_j| of every j (O(M)).
    Returns its vertex list."""
    xi = np.asarray(xi, dtype=np.float64)
    poly = [(-K, -K), (K, -K), (K, K), (-K, K)]
    pi = xi[i]
    for j in range(xi.shape[0]):
        if j == i or not poly:
            continue
        pj = xi[j]
        # |x - pi|^2 <= |x - pj|^2  <=>  2 (pj - pi) . x <= |pj|^2 - |pi|^2
        a, b = 2.0 * (pj[0] - pi[0]), 2.0 * (pj[1] - pi[1])
        c = pj[0] ** 2 + pj[1] ** 2 - pi[0] ** 2 - pi[1] ** 2
        poly = _clip(poly, a, b, c)
    return poly


def cell_area(poly) -> float:
    return _area(poly) if len(poly) >= 3 else 0.0


def voronoi_cells_2d(xi, K: float):
    """Every cell of voronoi_cell_2d (O(M^2); small inputs only)."""
    return [voronoi_cell_2d(xi, i, K) for i in range(np.asarray(xi).shape[0])]


def voronoi_2d(xi, K: float):
    """(mu, delta): mu_m the area of the Voronoi cell of xi_m in Y_K = [-K, K]^2,
    the density weight of App. B; delta = sup over Y_K of the distance to the
    nearest sample, attained at a vertex of some cell (App. B)."""
    xi = np.asarray(xi, dtype=np.float64)
    cells = voronoi_cells_2d(xi, K)
    mu = np.array([_area(c) if len(c) >= 3 else 0.0 for c in cells])
    delta = 0.0
    for i, c in enumerate(cells):
        for v in c:
            delta = max(delta, float(np.hypot(v[0] - xi[i, 0], v[1] - xi[i, 1])))
    return mu, delta
