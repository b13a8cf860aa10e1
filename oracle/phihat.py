"""Fourier transform of the scaling function (oracle; test infrastructure only).

App. A, eq. Daubechies_Fourier_scaling_function:  phi-hat is the infinite
product of the low-pass symbol m0 at dyadically shrinking arguments.  The
printed product starts at j = 0; with m0(xi) = sum h_k exp(-2 pi i k xi) and
sum h_k = 1 that gives phi-hat(2 xi).  The reading used here starts at j = 1:

    phi-hat(xi) = prod_{j=1}^{K} m0(2^-j xi),   K = 60 + ceil(log2 max(1, |xi|)),

so that |2^-K xi| <= 2^-60 and the neglected tail factor differs from 1 by far
less than the float64 rounding of the product.  The Haar closed form of App. A,
phi-hat(xi) = (1 - exp(-2 pi i xi)) / (2 pi i xi), pins this reading.
"""
import numpy as np

from .filters import m0


def depth(xi) -> np.ndarray:
    """Number of product factors K for each argument."""
    a = np.maximum(1.0, np.abs(np.asarray(xi, dtype=np.float64)))
    return 60 + np.ceil(np.log2(a)).astype(np.int64)


def phihat(xi, k: np.ndarray, h: np.ndarray) -> np.ndarray:
    """phi-hat(xi) by the truncated product, factor by factor."""
    xi = np.asarray(xi, dtype=np.float64)
    K = depth(xi)
    out = np.ones(xi.shape, dtype=np.complex128)
    for j in range(1, int(K.max()) + 1 if K.size else 1):
        f = m0(xi / 2.0**j, k, h)
        out = np.where(j <= K, out * f, out)
    return out


def phihat_haar_closed(xi) -> np.ndarray:
    """App. A closed form for the Haar scaling function 1_[0,1).

    (1 - exp(-2 pi i xi)) / (2 pi i xi) equals exp(-i pi xi) sin(pi xi)/(pi xi)
    exactly; the second form has no cancellation near xi = 0 and gives 1 there.
    """
    xi = np.asarray(xi, dtype=np.float64)
    return np.exp(-1j * np.pi * xi) * np.sinc(xi)
