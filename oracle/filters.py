"""Daubechies low-pass filters (oracle; test infrastructure only).

App. A defines m0(xi) = sum_k h_k exp(-2 pi i k xi) with m0(0) = 1 and the
scaling function through phi-hat(xi) = prod m0(2^-j xi).  The paper takes the
filter values from Cohen-Daubechies-Vial without printing them, so they are
derived here from the defining property of the Daubechies family with p
vanishing moments:

    |m0(xi)|^2 = cos(pi xi)^(2p) * P(sin(pi xi)^2),
    P(y) = sum_{k<p} C(p-1+k, k) y^k,

and the extremal-phase spectral factor (largest taps first).  With
z = exp(-2 pi i xi):  m0 = ((1+z)/2)^p * L(z), and every root y_j of P gives a
reciprocal pair of roots of L(z) L(1/z) from z + 1/z = 2 - 4 y_j; the root with
|z| > 1 is kept.  Taps are indexed k = -p+1 .. p so that supp(phi) = [-p+1, p]
(Sec. 3.3).
"""
from math import comb

import numpy as np


def daubechies_filter(p: int) -> tuple[np.ndarray, np.ndarray]:
    """Return (k, h): tap indices k = -p+1..p and real taps h_k with sum h_k = 1.

    p = 1 is Haar: h_0 = h_1 = 1/2.
    """
    if p < 1:
        raise ValueError("p must be >= 1")
    # P(y) coefficients, highest degree first for numpy.roots
    pc = [comb(p - 1 + k, k) for k in range(p)]
    yroots = np.roots(pc[::-1]) if p > 1 else np.array([])
    # polynomial in z, lowest degree first: (1+z)^p
    poly = np.array([1.0 + 0j])
    for _ in range(p):
        poly = np.convolve(poly, np.array([1.0, 1.0]))
    for y in yroots:
        # z^2 - (2 - 4y) z + 1 = 0
        b = 2.0 - 4.0 * y
        disc = np.sqrt(b * b - 4.0 + 0j)
        z1 = (b + disc) / 2.0
        z2 = (b - disc) / 2.0
        z = z1 if abs(z1) > abs(z2) else z2
        poly = np.convolve(poly, np.array([-z, 1.0]))
    h = np.real_if_close(poly, tol=1e6)
    h = np.real(h) / np.real(np.sum(poly))
    k = np.arange(-p + 1, p + 1)
    return k, h.astype(np.float64)


def m0(xi, k: np.ndarray, h: np.ndarray) -> np.ndarray:
    """Low-pass filter symbol m0(xi) = sum_k h_k exp(-2 pi i k xi) (App. A)."""
    xi = np.asarray(xi, dtype=np.float64)
    out = np.zeros(xi.shape, dtype=np.complex128)
    for kk, hh in zip(k, h):
        out += hh * np.exp(-2j * np.pi * kk * xi)
    return out
