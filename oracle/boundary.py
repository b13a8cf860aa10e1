"""Boundary-corrected scaling functions (oracle; test infrastructure only).

Sec. 3.3 uses the Cohen-Daubechies-Vial (CDV) edge functions: p left functions
phi^L_0..phi^L_{p-1} on [0, inf) with phi^L_k nearest the edge for k = 0, the
same number of vanishing moments as the interior, and (App. A.1,
eq. dilation_eq_lphi)

    phi^L_k(x)/sqrt2 = sum_{l<p} H_{k,l} phi^L_l(2x) + sum_{m=p}^{p+2k} h_{k,m} phi(2x-m).

The paper prints neither H nor h, so they are constructed here from the
defining properties (a reading of CDV, not their printed tables):

1. moments mu_a = int x^a phi, from the two-scale relation;
   M[a,l] = int x^a phi(x-l) dx.
2. edge functions phi~_a = sum_{l=-p+1}^{p-1} M[a,l] phi(.-l) 1_[0,inf): the
   part of x^a on [0, inf) that the interior translates (l >= p) do not carry;
   they are orthogonal to every phi(.-l), l >= p.
3. half-line Gram A[a,b] = int_0^inf phi(x-a) phi(x-b) dx, from the two-scale
   relation with A = delta_ab once one translate lies in [0, inf) and A = 0
   once one lies in (-inf, 0].
4. nested flag E_k = {sum c_a phi~_a : coefficient of phi(.-l) is 0 for l > k}
   (support in [0, p+k]); Gram-Schmidt along E_0 c E_1 c ... gives phi^L_k,
   sign fixed by h_{k,p+2k} > 0.
5. H, h from the half-scale expansion: the fine-scale translate coefficients
   d_{k,n}; h_{k,n} = d_{k,n} for n >= p, and the edge part (n <= p-1) is
   H times the coefficient matrix of step 4 (least squares; its residual is
   the nestedness check).
The right functions come from the reflected filter h_rev[k] = h[1-k]
(phi_rev(x) = phi(1-x)) as phi^R_k(x) = phi^L_k[rev](-x); this matches the
right dilation equation of App. A.1 with phi(2x+m+1).

Fourier transforms (App. A.1, eq. Fourier_relation_lphi): with U = H/sqrt2,
V = h/sqrt2,
    v1(xi) ~= U^K v1(0) + sum_{l=0}^{K-1} U^l V v2(xi / 2^(l+1)),
    v1(0)  = (I - U)^-1 V v2(0),
left  v2(eta) = [phi-hat(eta) exp(-2 pi i m eta)]_{m=p}^{3p-2},
right v2(eta) = [phi-hat(eta) exp(+2 pi i (m+1) eta)]_{m=p}^{3p-2}.
"""
from math import comb

import numpy as np

from .filters import daubechies_filter, m0


def moments(k: np.ndarray, h: np.ndarray, p: int) -> np.ndarray:
    """mu_a = int x^a phi(x) dx, a < p, from
    mu_a (1 - 2^-a) = 2^-a sum_{b<a} C(a,b) mu_b sum_k h_k k^(a-b),  mu_0 = 1."""
    mu = np.zeros(p)
    mu[0] = 1.0
    kf = k.astype(np.float64)
    for a in range(1, p):
        s = 0.0
        for b in range(a):
            s += comb(a, b) * mu[b] * np.sum(h * kf ** (a - b))
        mu[a] = 2.0**-a * s / (1.0 - 2.0**-a)
    return mu


def translate_moments(mu: np.ndarray, p: int) -> tuple[np.ndarray, np.ndarray]:
    """M[a, l] = int x^a phi(x - l) dx = sum_b C(a,b) l^(a-b) mu_b for l = -p+1..p-1."""
    ls = np.arange(-p + 1, p)
    M = np.zeros((p, ls.size))
    for a in range(p):
        for j, l in enumerate(ls):
            M[a, j] = sum(comb(a, b) * float(l) ** (a - b) * mu[b] for b in range(a + 1))
    return ls, M


def halfline_gram(k: np.ndarray, h: np.ndarray, p: int) -> np.ndarray:
    """A[a, b] = int_0^inf phi(x-a) phi(x-b) dx for a, b in -p+1..p-1.

    Two-scale relation: A[a,b] = sum_{i,j} hon_i hon_j A[2a+i, 2b+j], hon = sqrt2 h.
    """
    hon = np.sqrt(2.0) * h
    ls = list(range(-p + 1, p))

    def known(a, b):
        if a >= p - 1 or b >= p - 1:
            return 1.0 if a == b else 0.0
        if a <= -p or b <= -p:
            return 0.0
        return None

    unk = [a for a in ls if a <= p - 2]
    idx = {a: i for i, a in enumerate(unk)}
    n = len(unk)
    A = np.zeros((len(ls), len(ls)))
    if n:
        mat = np.eye(n * n)
        rhs = np.zeros(n * n)
        for a in unk:
            for b in unk:
                r = idx[a] * n + idx[b]
                for ki, hi in zip(k, hon):
                    for kj, hj in zip(k, hon):
                        aa, bb = 2 * a + int(ki), 2 * b + int(kj)
                        kv = known(aa, bb)
                        if kv is None:
                            mat[r, idx[aa] * n + idx[bb]] -= hi * hj
                        else:
                            rhs[r] += hi * hj * kv
        sol = np.linalg.solve(mat, rhs)
    for i, a in enumerate(ls):
        for j, b in enumerate(ls):
            kv = known(a, b)
            A[i, j] = kv if kv is not None else sol[idx[a] * n + idx[b]]
    return A


def halfline_integrals(k: np.ndarray, h: np.ndarray, p: int) -> np.ndarray:
    """I_l = int_0^inf phi(x - l) dx for l = -p+1..p-1, from I_l = sum_i h_i I_{2l+i}."""
    ls = list(range(-p + 1, p))

    def known(l):
        if l >= p - 1:
            return 1.0
        if l <= -p:
            return 0.0
        return None

    unk = [l for l in ls if known(l) is None]
    idx = {l: i for i, l in enumerate(unk)}
    n = len(unk)
    vals = {}
    if n:
        mat = np.eye(n)
        rhs = np.zeros(n)
        for l in unk:
            for ki, hi in zip(k, h):
                ll = 2 * l + int(ki)
                kv = known(ll)
                if kv is None:
                    mat[idx[l], idx[ll]] -= hi
                else:
                    rhs[idx[l]] += hi * kv
        sol = np.linalg.solve(mat, rhs)
        vals = {l: sol[idx[l]] for l in unk}
    return np.array([known(l) if known(l) is not None else vals[l] for l in ls])


class EdgeSide:
    """Constants of one edge: filter, CDV coefficients, H, h, U, V, v1(0)."""

    def __init__(self, p: int, side: str):
        if p < 2:
            raise ValueError("Haar has no boundary functions (Sec. 3.3)")
        self.p, self.side = p, side
        k, h = daubechies_filter(p)
        self.k_int, self.h_int = k, h  # interior filter, used by v2
        if side == "left":
            kk, hh = k, h
        elif side == "right":
            # h_rev[k] = h[1-k]; same index range -p+1..p
            kk = k
            hh = np.array([h[list(k).index(1 - int(t))] for t in k])
        else:
            raise ValueError(side)
        self.k, self.h = kk, hh
        hon = np.sqrt(2.0) * hh
        mu = moments(kk, hh, p)
        ls, M = translate_moments(mu, p)
        A = halfline_gram(kk, hh, p)
        G = M @ A @ M.T  # Gram of phi~_a
        self.mu, self.M, self.A, self.G, self.ls = mu, M, A, G, ls

        # step 4: Gram-Schmidt along the nested flag
        rows = []
        for kq in range(p):
            cols = [j for j, l in enumerate(ls) if l > kq]
            if cols:
                con = M[:, cols].T
                _, _, vt = np.linalg.svd(con)
                null = vt[len(cols):].T  # basis of E_kq (dim kq+1)
            else:
                null = np.eye(p)
            # pick the direction of E_kq that leaves E_{kq-1} most
            jk = list(ls).index(kq)
            w = null[:, np.argmax(np.abs(null.T @ M[:, jk]))].copy()
            for v in rows:
                w = w - (v @ G @ w) * v
            w = w / np.sqrt(w @ G @ w)
            rows.append(w)
        Calpha = np.array(rows)  # p x p, over phi~_a
        C = Calpha @ M  # p x (2p-1), over restricted translates phi(.-l), l=-p+1..p-1
        for kq in range(p):
            jk = list(ls).index(kq)
            if C[kq, jk] * hon[-1] < 0:
                C[kq] = -C[kq]
                Calpha[kq] = -Calpha[kq]
        self.Calpha, self.C = Calpha, C

        # step 5: half-scale expansion d_{k,n} = sum_l C[k,l] hon[n-2l]
        # fine translates phi(2x-n) with n <= -p vanish on [0, inf) and drop out
        ns = np.arange(-p + 1, 3 * p - 1)
        D = np.zeros((p, ns.size))
        for kq in range(p):
            for j, l in enumerate(ls):
                for t, hv in zip(kk, hon):
                    n = 2 * int(l) + int(t)
                    if n >= -p + 1:
                        D[kq, n - (-p + 1)] += C[kq, j] * hv
        D_edge = D[:, : 2 * p - 1]  # n = -p+1..p-1
        Hsol, *_ = np.linalg.lstsq(C.T, D_edge.T, rcond=None)
        self.H = Hsol.T
        self.nest_residual = np.max(np.abs(self.H @ C - D_edge))
        self.hb = D[:, 2 * p - 1:]  # h_{k,m}, m = p..3p-2
        self.U = self.H / np.sqrt(2.0)
        self.V = self.hb / np.sqrt(2.0)
        self.v1_0 = np.linalg.solve(np.eye(p) - self.U, self.V @ np.ones(2 * p - 1))

    def v2(self, eta: np.ndarray, phat: np.ndarray) -> np.ndarray:
        """v2(eta) as a (2p-1, n) array; phat = phi-hat(eta) of the interior phi."""
        p = self.p
        ms = np.arange(p, 3 * p - 1)
        if self.side == "left":
            ph = np.exp(-2j * np.pi * np.outer(ms, eta))
        else:
            ph = np.exp(2j * np.pi * np.outer(ms + 1, eta))
        return ph * phat[None, :]

    def ft(self, xi) -> np.ndarray:
        """v1(xi) = [F phi^{L or R}_k (xi)]_k as a (p, n) array (App. A.1)."""
        xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
        K = 60 + np.ceil(np.log2(np.maximum(1.0, np.abs(xi)))).astype(np.int64)
        Kmax = int(K.max())
        # m0(xi / 2^j) for every j that some phi-hat(xi / 2^(l+1)) needs
        jmax = 2 * Kmax + 2
        fac = [None] + [m0(xi / 2.0**j, self.k_int, self.h_int) for j in range(1, jmax + 1)]
        acc = np.zeros((self.p, xi.size), dtype=np.complex128)
        Upow = np.eye(self.p)
        UK = np.zeros((xi.size, self.p, self.p))
        for l in range(Kmax):
            eta = xi / 2.0 ** (l + 1)
            # phi-hat(eta) = prod_{j=1}^{K(eta)} m0(eta/2^j) = prod_{j=l+2}^{l+1+K(eta)} m0(xi/2^j)
            Keta = 60 + np.ceil(np.log2(np.maximum(1.0, np.abs(eta)))).astype(np.int64)
            phat = np.ones(xi.size, dtype=np.complex128)
            for j in range(l + 2, l + 2 + int(Keta.max())):
                phat = np.where(j <= l + 1 + Keta, phat * fac[j], phat)
            term = Upow @ self.V @ self.v2(eta, phat)
            acc += np.where((l < K)[None, :], term, 0.0)
            Upow = Upow @ self.U
            UK[K == l + 1] = Upow
        acc += np.einsum("nij,j->in", UK, self.v1_0)
        return acc
