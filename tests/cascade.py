"""Point values of a refinable function by the cascade algorithm (test helper).

Independent of the oracle's Fourier-side code: phi at the integers is the
eigenvector (eigenvalue 1) of the two-scale relation phi(n) = 2 sum h_k phi(2n-k),
normalised to sum 1, then refined dyadically.  Used only for low-accuracy
(quadrature) cross-checks of Gram entries and Fourier transforms.
"""
import numpy as np


def cascade(k, h, R: int = 12):
    k = np.asarray(k)
    lo, hi = int(k.min()), int(k.max())  # support of phi is [lo, hi]
    ints = np.arange(lo, hi + 1)
    n = ints.size
    A = np.zeros((n, n))
    for a, na in enumerate(ints):
        for kk, hh in zip(k, h):
            m = 2 * na - int(kk)
            if lo <= m <= hi:
                A[a, m - lo] += 2.0 * hh
    w, v = np.linalg.eig(A)
    i = np.argmin(np.abs(w - 1.0))
    cur = np.real(v[:, i])
    cur = cur / cur.sum()
    for r in range(1, R + 1):
        xs = np.arange(lo * 2**r, hi * 2**r + 1)
        new = np.zeros(xs.size)
        base = lo * 2 ** (r - 1)
        top = hi * 2 ** (r - 1)
        for kk, hh in zip(k, h):
            m = xs - int(kk) * 2 ** (r - 1)
            ok = (m >= base) & (m <= top)
            new[ok] += 2.0 * hh * cur[m[ok] - base]
        cur = new
    xs = np.arange(lo * 2**R, hi * 2**R + 1) / 2.0**R
    return xs, cur
