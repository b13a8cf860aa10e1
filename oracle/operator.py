"""Change-of-basis matrix T by its entries, and direct products (oracle; test
infrastructure only).

Sec. 4: with N = 2^J, p vanishing moments and b boundary functions per side
(b = p, or b = 0 for Haar, Sec. 3.3), column i = 0..N-1 of T at sample xi is

    left      i <  b    :  2^-J/2 exp(+pi i xi) phi^L_i-hat(xi / 2^J)
    interior  b <= i < N-b :  2^-J/2 exp(-2 pi i (i - N/2) xi / 2^J) phi-hat(xi / 2^J)
    right     i >= N-b  :  2^-J/2 exp(-pi i xi) phi^R_{N-1-i}-hat(xi / 2^J)

(the printed translations tau_{-1}, tau_1 and the interior phase are read as
tau_{-1/2}, tau_{1/2} and exp(-2 pi i k 2^-J xi), per the definition of the
interval basis in Sec. 3.3 and eq. Fourier_transform_of_general_wavelet).
Sec. 4.1: rows (and data) are multiplied by sqrt(mu_m).

Sec. 5 / App. C: in 2D the entry for coefficient (i, j) (i along x, j along y)
is t_x[m, i] * t_y[m, j]; coefficient vectors are stored x-fastest, i + N*j.

The products are direct sums over the entries -- the NDFT of eq. NDFT_def,
never an NFFT.
"""
import numpy as np

from .boundary import EdgeSide
from .filters import daubechies_filter
from .phihat import phihat, phihat_haar_closed


class Basis1D:
    """The interval basis V_J^int of Sec. 3.3 at scale J with p vanishing moments."""

    def __init__(self, p: int, J: int):
        if 2**J < 2 * p:
            raise ValueError("need 2^J >= 2p")
        self.p, self.J, self.N = p, J, 2**J
        self.k, self.h = daubechies_filter(p)
        self.b = 0 if p == 1 else p
        if self.b:
            self.left = EdgeSide(p, "left")
            self.right = EdgeSide(p, "right")

    def phihat(self, eta):
        if self.p == 1:
            return phihat_haar_closed(eta)
        return phihat(eta, self.k, self.h)

    def factors(self, xi, cols=None) -> np.ndarray:
        """t[m, i]: entry of T (without density weight) for samples xi, all N columns,
        or only the columns listed in cols (in that order)."""
        xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
        N, J, b = self.N, self.J, self.b
        cols = np.arange(N) if cols is None else np.asarray(cols, dtype=np.int64)
        s = 2.0 ** (-J / 2.0)
        eta = xi / 2.0**J
        t = np.zeros((xi.size, cols.size), dtype=np.complex128)
        inner = (cols >= b) & (cols < N - b)
        kk = cols[inner] - N // 2
        t[:, inner] = s * np.exp(-2j * np.pi * np.outer(eta, kk)) * self.phihat(eta)[:, None]
        if b:
            vL = self.left.ft(eta)  # (p, M)
            vR = self.right.ft(eta)
            for j, i in enumerate(cols):
                if i < b:
                    t[:, j] = s * np.exp(1j * np.pi * xi) * vL[i]
                elif i >= N - b:
                    t[:, j] = s * np.exp(-1j * np.pi * xi) * vR[N - 1 - i]
        return t


def dense_T_1d(basis: Basis1D, xi, mu=None) -> np.ndarray:
    """The M x N matrix T of eq. CoB_block_1D with rows scaled by sqrt(mu)."""
    t = basis.factors(xi)
    if mu is not None:
        t = np.sqrt(np.asarray(mu, dtype=np.float64))[:, None] * t
    return t


def dense_T_2d(basis: Basis1D, xi2, mu=None) -> np.ndarray:
    """The M x N^2 matrix of Sec. 5, column i + N*j = t_x[:, i] * t_y[:, j]."""
    xi2 = np.asarray(xi2, dtype=np.float64)
    tx = basis.factors(xi2[:, 0])
    ty = basis.factors(xi2[:, 1])
    N = basis.N
    T = (ty[:, :, None] * tx[:, None, :]).reshape(xi2.shape[0], N * N)
    if mu is not None:
        T = np.sqrt(np.asarray(mu, dtype=np.float64))[:, None] * T
    return T


class Operator1D:
    """T and T^H for one 1D sampling pattern, by explicit rows of T."""

    def __init__(self, basis: Basis1D, xi, mu=None):
        self.basis = basis
        self.T = dense_T_1d(basis, xi, mu)

    def apply(self, x):
        return self.T @ np.asarray(x, dtype=np.complex128)

    def adjoint(self, y):
        return self.T.conj().T @ np.asarray(y, dtype=np.complex128)


class Operator2D:
    """T and T^H for one 2D pattern (Sec. 5, App. C), row block by row block.

    y_m = sum_{i,j} t_x[m,i] X[i,j] t_y[m,j]  and
    z[i,j] = sum_m conj(t_x[m,i]) conj(t_y[m,j]) u_m,
    with the per-sample factor rows t_x, t_y kept instead of the M x N^2 matrix.
    """

    def __init__(self, basis: Basis1D, xi2, mu=None, block: int = 8192):
        xi2 = np.asarray(xi2, dtype=np.float64)
        self.basis, self.N, self.M = basis, basis.N, xi2.shape[0]
        self.tx = basis.factors(xi2[:, 0])
        if mu is not None:
            self.tx *= np.sqrt(np.asarray(mu, dtype=np.float64))[:, None]
        self.ty = basis.factors(xi2[:, 1])
        self.block = block

    def apply(self, x):
        N = self.N
        X = np.asarray(x, dtype=np.complex128).reshape(N, N).T  # X[i, j], i along x
        y = np.empty(self.M, dtype=np.complex128)
        for s in range(0, self.M, self.block):
            e = min(self.M, s + self.block)
            y[s:e] = np.sum((self.tx[s:e] @ X) * self.ty[s:e], axis=1)
        return y

    def adjoint(self, u):
        N = self.N
        u = np.asarray(u, dtype=np.complex128)
        Z = np.zeros((N, N), dtype=np.complex128)
        for s in range(0, self.M, self.block):
            e = min(self.M, s + self.block)
            Z += self.tx[s:e].conj().T @ (u[s:e, None] * self.ty[s:e].conj())
        return Z.T.reshape(N * N)  # x-fastest

    def rows(self, idx, x):
        """(T x)[idx] only: the sampled-row form used at full size."""
        N = self.N
        X = np.asarray(x, dtype=np.complex128).reshape(N, N).T
        return np.sum((self.tx[idx] @ X) * self.ty[idx], axis=1)
