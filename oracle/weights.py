"""Density weights (oracle; test infrastructure only).

Sec. 4.1: mu_omega is the Lebesgue measure of the Voronoi region of the
sampling frequency omega.  In 1D, with the frequencies sorted, the cell of
xi_m is [(xi_{m-1}+xi_m)/2, (xi_m+xi_{m+1})/2]; the outer cells are closed by
the bandwidth interval [-K, K] (the region Y_K of App. B in one dimension).
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
