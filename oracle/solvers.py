"""Least-squares solvers (oracle; test infrastructure only).

Sec. 2, eq. least_squares: the coefficients minimise ||T x - w^s||_2; Sec. 6.3
solves it with a conjugate-gradient method whose cost is the products with T
and T^*.  The conjugate-gradient variant is not named; this is textbook CGLS
(CG on the normal equations T^H T x = T^H y, without forming them), stopped on
the normal-equation residual ||T^H (y - T x)|| <= tol * ||T^H y||.
An independent minimiser for small sizes is Householder QR.
"""
import numpy as np


def cgls(apply, adjoint, y, tol=1e-10, maxit=1000, x0=None):
    """Return (x, iterations, history of ||s|| / ||T^H y||)."""
    y = np.asarray(y, dtype=np.complex128)
    bnorm = np.linalg.norm(adjoint(y))
    if x0 is None:
        x = np.zeros_like(adjoint(y))
        r = y.copy()
    else:
        x = np.asarray(x0, dtype=np.complex128).copy()
        r = y - apply(x)
    s = adjoint(r)
    p = s.copy()
    gamma = np.vdot(s, s).real
    hist = [np.sqrt(gamma) / bnorm if bnorm > 0 else 0.0]
    it = 0
    while it < maxit and hist[-1] > tol:
        q = apply(p)
        alpha = gamma / np.vdot(q, q).real
        x = x + alpha * p
        r = r - alpha * q
        s = adjoint(r)
        gamma_new = np.vdot(s, s).real
        beta = gamma_new / gamma
        p = s + beta * p
        gamma = gamma_new
        it += 1
        hist.append(np.sqrt(gamma) / bnorm)
    return x, it, np.array(hist)


def qr_lstsq(T, y):
    """argmin ||T x - y|| by Householder QR (LAPACK geqrf via numpy)."""
    Q, R = np.linalg.qr(np.asarray(T, dtype=np.complex128), mode="reduced")
    rhs = Q.conj().T @ np.asarray(y, dtype=np.complex128)
    return np.linalg.solve(R, rhs) if R.shape[0] == R.shape[1] else None
