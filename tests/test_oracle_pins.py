"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each check is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign or index, a transposed operand, the phi-hat product started at the
wrong j) fails at least one of them.  No check here compares the oracle with
itself through a retyped formula.
"""
import numpy as np
import pytest

from oracle.boundary import EdgeSide, halfline_gram, halfline_integrals
from oracle.filters import daubechies_filter, m0
from oracle.operator import Basis1D, Operator1D, Operator2D, dense_T_1d, dense_T_2d
from oracle.phihat import phihat, phihat_haar_closed
from oracle.solvers import cgls, qr_lstsq
from oracle.weights import voronoi_1d
from tests.cascade import cascade

# ------------------------------------------------------------------ filters (App. A)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6])
def test_filter_normalisation_and_qmf(p):
    k, h = daubechies_filter(p)
    assert k[0] == -p + 1 and k[-1] == p  # supp(phi) = [-p+1, p], Sec. 3.3
    assert abs(h.sum() - 1.0) < 1e-14  # m0(0) = 1, App. A
    xi = np.linspace(-1, 1, 37)
    qmf = np.abs(m0(xi, k, h)) ** 2 + np.abs(m0(xi + 0.5, k, h)) ** 2
    assert np.max(np.abs(qmf - 1.0)) < 1e-13
    hon = np.sqrt(2) * h
    for l in range(1, p):  # orthonormal even shifts
        assert abs(np.dot(hon[2 * l:], hon[: hon.size - 2 * l])) < 1e-13


@pytest.mark.parametrize("p", [2, 3, 4])
def test_filter_zero_of_order_p_at_half(p):
    k, h = daubechies_filter(p)
    # m0(1/2 + e) = O(e^p): p vanishing moments
    e1, e2 = 1e-2, 5e-3
    r = abs(m0(0.5 + e1, k, h)) / abs(m0(0.5 + e2, k, h))
    assert abs(np.log2(r) - p) < 0.05


def test_db2_textbook_closed_form():
    k, h = daubechies_filter(2)
    s3 = np.sqrt(3.0)
    ref = np.array([1 + s3, 3 + s3, 3 - s3, 1 - s3]) / 8.0  # orthonormal /(4 sqrt2), times 1/sqrt2
    assert np.max(np.abs(h - ref)) < 1e-15


# ------------------------------------------------------------------ phi-hat (App. A)


def test_phihat_product_equals_haar_closed_form():
    # pins the product start j = 1 (a j = 0 start gives phi-hat(2 xi))
    k, h = daubechies_filter(1)
    xi = np.concatenate([np.linspace(-7.3, 7.3, 41), [0.0, 0.5, 1e-7, 3.0]])
    assert np.max(np.abs(phihat(xi, k, h) - phihat_haar_closed(xi))) < 2e-15
    # the printed form, away from its 0/0 point
    x = np.linspace(-7.3, 7.3, 40)  # excludes 0
    printed = (1.0 - np.exp(-2j * np.pi * x)) / (2j * np.pi * x)
    assert np.max(np.abs(phihat(x, k, h) - printed)) < 2e-15


@pytest.mark.parametrize("p", [2, 4])
def test_phihat_invariants(p):
    k, h = daubechies_filter(p)
    # phi-hat(0) = 1: the product of ~60 factors m0(0) = sum h = 1 (to rounding)
    assert abs(phihat(np.array([0.0]), k, h)[0] - 1.0) < 1e-13
    ints = np.array([-5.0, -3, -2, -1, 1, 2, 4, 7])
    assert np.max(np.abs(phihat(ints, k, h))) < 1e-15
    # orthonormal translates: sum_k |phi-hat(xi + k)|^2 = 1.  For db2 the deficit of
    # the band |k| <= K falls like K^-2 (|phi-hat| ~ |xi|^-1.5), so it is checked to
    # shrink about 25x (at least 15x) from K = 4000 to K = 20000; db4 decays fast
    # enough to reach rounding.
    for xi in [0.13, 0.37, -0.41]:
        s1 = np.sum(np.abs(phihat(xi + np.arange(-4000, 4001), k, h)) ** 2)
        if p == 2:
            s2 = np.sum(np.abs(phihat(xi + np.arange(-20000, 20001), k, h)) ** 2)
            d1, d2 = 1.0 - s1, 1.0 - s2
            assert 0 < d1 < 1e-8 and 0 < d2
            assert d1 / d2 > 15.0
        else:
            assert abs(s1 - 1.0) < 1e-12


@pytest.mark.parametrize("p", [2, 4])
def test_phihat_matches_quadrature_of_cascade(p):
    k, h = daubechies_filter(p)
    xs, ph = cascade(k, h, R=13)
    for xi in [0.0, 0.3, -0.7, 1.6]:
        q = np.trapezoid(np.exp(-2j * np.pi * xi * xs) * ph, xs)
        assert abs(q - phihat(np.array([xi]), k, h)[0]) < 1e-6


# ------------------------------------------------------------------ boundary (Sec. 3.3, App. A.1)


@pytest.mark.parametrize("p", [2, 3, 4])
@pytest.mark.parametrize("side", ["left", "right"])
def test_boundary_filter_invariants(p, side):
    e = EdgeSide(p, side)
    HH = np.hstack([e.H, e.hb])
    # rows of [H | h] orthonormal: phi^L orthonormal and orthogonal to interior translates
    assert np.max(np.abs(HH @ HH.T - np.eye(p))) < 1e-13
    assert e.nest_residual < 1e-11  # edge space is nested: V_0 in V_1
    for kk in range(p):  # h_{k,m} = 0 for m > p + 2k (eq. dilation_eq_lphi)
        assert np.all(np.abs(e.hb[kk, 2 * kk + 1:]) < 1e-13)
        assert e.hb[kk, 2 * kk] > 0  # sign reading h_{k,p+2k} > 0
    # the edge space reproduces x^a on [0, inf): U has eigenvalues 2^(-a-1)
    ev = np.sort(np.linalg.eigvals(e.U).real)[::-1]
    assert np.max(np.abs(ev - 2.0 ** -(np.arange(p) + 1.0))) < 1e-10
    # v1(0) = (I - U)^-1 V 1 equals int phi^L_k from half-line integrals of translates
    I = halfline_integrals(e.k, e.h, p)
    assert np.max(np.abs(e.C @ I - e.v1_0)) < 1e-12


@pytest.mark.parametrize("p", [2, 4])
def test_halfline_gram_matches_quadrature(p):
    k, h = daubechies_filter(p)
    A = halfline_gram(k, h, p)
    xs, ph = cascade(k, h, R=12)
    x = np.arange(0, 3 * p, xs[1] - xs[0])
    ls = list(range(-p + 1, p))
    for i, a in enumerate(ls):
        for j, b in enumerate(ls):
            q = np.trapezoid(np.interp(x - a, xs, ph, 0, 0) * np.interp(x - b, xs, ph, 0, 0), x)
            assert abs(q - A[i, j]) < 1e-5


@pytest.mark.parametrize("p", [2, 4])
def test_boundary_ft_matches_quadrature(p):
    """v1(xi) from the App. A.1 recursion against the transform of the edge
    functions built in the time domain (cascade values, restricted translates)."""
    k, h = daubechies_filter(p)
    for side in ["left", "right"]:
        e = EdgeSide(p, side)
        xs, ph = cascade(e.k, e.h, R=12)  # phi for left, phi_rev(x) = phi(1-x) for right
        dx = xs[1] - xs[0]
        x = np.arange(0, 3 * p, dx)
        fun = np.zeros((p, x.size))
        for kk in range(p):
            for j, l in enumerate(e.ls):
                fun[kk] += e.C[kk, j] * np.interp(x - l, xs, ph, 0, 0)
        for xi in [0.0, 0.45, -1.3]:
            if side == "left":  # phi^L_k on [0, inf)
                q = np.trapezoid(np.exp(-2j * np.pi * xi * x)[None] * fun, x, axis=1)
            else:  # phi^R_k(x) = phi^L_k[rev](-x) on (-inf, 0]
                q = np.trapezoid(np.exp(+2j * np.pi * xi * x)[None] * fun, x, axis=1)
            v = e.ft(np.array([xi]))[:, 0]
            assert np.max(np.abs(q - v)) < 2e-5, (side, xi)


# ------------------------------------------------------------------ operator (Sec. 3.2, 4, 5, App. C)


@pytest.mark.parametrize("p,J", [(1, 4), (2, 4), (4, 4)])
def test_integer_frequencies_give_identity_gram(p, J):
    """For f, g supported in [-1/2, 1/2], sum over integer omega of f-hat(omega)
    conj(g-hat(omega)) = <f, g> (Fourier series); the basis is orthonormal, so
    T^H T -> I as the integer band |omega| < K grows.  Edge functions (and Haar)
    jump at the interval ends, so their transforms decay like 1/omega and the gap
    falls like 1/K: quadrupling K must divide it by about 4."""
    B = Basis1D(p, J)
    errs = []
    for K in [8 * B.N, 32 * B.N]:
        T = dense_T_1d(B, np.arange(-K, K, dtype=np.float64))
        E = T.conj().T @ T - np.eye(B.N)
        errs.append(np.max(np.abs(E)))
    assert errs[0] / errs[1] > 3.5
    assert errs[1] < 0.015


def test_interior_block_is_phase_shifted_dft():
    """Sec. 3.2: on xi_m = eps/N (m-1-M/2) (here N in the formula is N2/q...), the NDFT
    equals a phase times a DFT of a zero-interleaved vector.  Checks the sign and
    index of the interior phase of T against numpy's FFT."""
    B = Basis1D(2, 5)
    N = B.N
    eps = 0.5
    M = 3 * N
    # sample points in units of the reconstruction band: xi = 2^J * nu, nu on the grid
    m = np.arange(1, M + 1)
    nu = eps / N * (m - 1 - M / 2)
    xi = 2.0**B.J * nu
    T = dense_T_1d(B, xi)
    b = B.b
    rng = np.random.default_rng(0)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    x[:b] = 0
    x[N - b:] = 0
    # NDFT with k = n - 1 - N/2, n = 1..N (eq. NDFT_def), via the DFT identity of Sec. 3.2
    q = 1
    while q * N / eps < M:
        q += 1
    N2 = int(q * N / eps)
    z = np.zeros(N2, dtype=np.complex128)
    ell = np.arange(1, N + 1)
    z[q * (ell - 1)] = x * np.exp(1j * np.pi * (ell - 1) * eps * M / N)
    y = np.exp(1j * np.pi * N * nu) * np.fft.fft(z)[:M]
    D = 2.0 ** (-B.J / 2) * B.phihat(nu)
    assert np.max(np.abs(T @ x - D * y)) < 1e-12


def test_2d_operator_matches_dense_and_is_adjoint():
    B = Basis1D(2, 3)
    N = B.N
    rng = np.random.default_rng(1)
    xi2 = rng.uniform(-20, 20, size=(150, 2))
    mu = rng.uniform(0.5, 2, size=150)
    T = dense_T_2d(B, xi2, mu)
    op = Operator2D(B, xi2, mu, block=37)
    x = rng.standard_normal(N * N) + 1j * rng.standard_normal(N * N)
    y = rng.standard_normal(150) + 1j * rng.standard_normal(150)
    assert np.max(np.abs(op.apply(x) - T @ x)) < 1e-12
    assert np.max(np.abs(op.adjoint(y) - T.conj().T @ y)) < 1e-12
    assert abs(np.vdot(op.apply(x), y) - np.vdot(x, op.adjoint(y))) < 1e-11


def test_2d_tensor_grid_is_kronecker_and_app_c_layout():
    """On a tensor grid {(a_s, b_t)} (s fastest) T_2D = T_y kron T_x; a single
    sample row reproduces the App. C layout: entry (i, j) = t_x[i] t_y[j] at
    vec index i + N j (x-fastest, L / I / R blocks along each axis)."""
    B = Basis1D(2, 3)
    N = B.N
    a = np.array([-3.3, 0.7, 5.1, 11.0])
    bb = np.array([-8.2, 2.5, 6.6])
    A, Bg = np.meshgrid(a, bb)  # A varies fastest
    xi2 = np.stack([A.ravel(), Bg.ravel()], axis=1)
    T2 = dense_T_2d(B, xi2)
    Tx = dense_T_1d(B, a)
    Ty = dense_T_1d(B, bb)
    assert np.max(np.abs(T2 - np.kron(Ty, Tx))) < 1e-15
    row = dense_T_2d(B, xi2[:1])[0].reshape(N, N)  # [j, i]
    tx = B.factors(xi2[:1, 0])[0]
    ty = B.factors(xi2[:1, 1])[0]
    for i in range(N):
        for j in range(N):
            assert abs(row[j, i] - tx[i] * ty[j]) <= 1e-15 * abs(tx[i] * ty[j])


def test_uniform_weights_shift_equivalence():
    """[0, 1] versus [-1/2, 1/2]: rows differ by a unit-modulus phase exp(-i pi xi),
    which leaves the weighted least-squares solution unchanged."""
    B = Basis1D(2, 4)
    rng = np.random.default_rng(3)
    xi = np.sort(rng.uniform(-40, 40, 96))
    T = dense_T_1d(B, xi)
    y = rng.standard_normal(96) + 1j * rng.standard_normal(96)
    ph = np.exp(-1j * np.pi * xi)
    x1 = qr_lstsq(T, y)
    x2 = qr_lstsq(ph[:, None] * T, ph * y)
    assert np.max(np.abs(x1 - x2)) < 1e-12


# ------------------------------------------------------------------ weights (Sec. 4.1) and solvers


def test_voronoi_1d():
    xi = np.arange(-10, 10) + 0.5
    assert np.allclose(voronoi_1d(xi, 10.0), 1.0)
    rng = np.random.default_rng(2)
    xi = rng.uniform(-7, 7, 50)
    w = voronoi_1d(xi, 8.0)
    assert abs(w.sum() - 16.0) < 1e-12 and np.all(w > 0)


def test_voronoi_1d_hand_worked_unsorted():
    # Sec. 4.1: the weight of xi_m is the length of its Voronoi cell in [-K, K].
    # Sorted: -4, -1, 0.5, 2, 3, 6; midpoints -2.5, -0.25, 1.25, 2.5, 4.5; cells
    # [-5,-2.5] [-2.5,-0.25] [-0.25,1.25] [1.25,2.5] [2.5,4.5] [4.5,5] (6 lies
    # beyond K = 5: only the part of its cell inside [-K, K] counts).  Listed in
    # the caller's (unsorted) order:
    xi = np.array([3.0, -1.0, 0.5, -4.0, 2.0, 6.0])
    want = np.array([2.0, 2.25, 1.5, 2.5, 1.25, 0.5])
    assert np.array_equal(voronoi_1d(xi, 5.0), want)


def test_voronoi_1d_permutation_equivariant():
    # the weight belongs to the sample, not to its position: w(xi[pi]) = w(xi)[pi]
    g = np.random.default_rng(21)
    xi = g.uniform(-30, 30, 40)
    w = voronoi_1d(xi, 32.0)
    for _ in range(5):
        pi = g.permutation(xi.size)
        assert np.allclose(voronoi_1d(xi[pi], 32.0), w[pi], rtol=0, atol=1e-13)
    # each cell is half the gap to each neighbour (interior samples)
    o = np.argsort(xi)
    s = xi[o]
    assert np.allclose(w[o][1:-1], (s[2:] - s[:-2]) / 2.0, rtol=0, atol=1e-13)


@pytest.mark.parametrize("p,J,M", [(1, 6, 128), (2, 5, 96), (4, 5, 128)])
def test_cgls_recovers_and_matches_qr(p, J, M):
    B = Basis1D(p, J)
    rng = np.random.default_rng(p * 10 + J)
    xi = np.arange(-M // 2, M // 2) + 0.5 + rng.uniform(-0.3, 0.3, M)
    mu = voronoi_1d(xi, M / 2)
    op = Operator1D(B, xi, mu)
    xt = rng.standard_normal(B.N) + 1j * rng.standard_normal(B.N)
    x, it, _ = cgls(op.apply, op.adjoint, op.apply(xt), tol=1e-13, maxit=500)
    assert np.max(np.abs(x - xt)) / np.max(np.abs(xt)) < 1e-10  # exact recovery
    y = op.apply(xt) + 0.05 * (rng.standard_normal(M) + 1j * rng.standard_normal(M))
    x1, _, _ = cgls(op.apply, op.adjoint, y, tol=1e-13, maxit=500)
    x2 = qr_lstsq(op.T, y)
    assert np.max(np.abs(x1 - x2)) / np.max(np.abs(x2)) < 1e-10


def test_cgls_iterates_minimise_over_the_krylov_space():
    """The k-th CGLS iterate from x = 0 is the minimiser of ||y - A x|| over the
    Krylov space span{A^H y, (A^H A) A^H y, ..., (A^H A)^(k-1) A^H y} (Sec. 2: CGLS is
    CG on the normal equations).  Computed here directly: an orthonormal basis of
    that space by QR, then least squares in it.  Pins every iterate of the oracle's
    recurrences, not only their limit (a wrong beta or alpha still converges, more
    slowly, but leaves the Krylov minimisers)."""
    rng = np.random.default_rng(31)
    A = rng.standard_normal((40, 12)) + 1j * rng.standard_normal((40, 12))
    y = rng.standard_normal(40) + 1j * rng.standard_normal(40)
    AH = A.conj().T
    b = AH @ y
    for k in range(1, 8):
        xk, it, _ = cgls(lambda v: A @ v, lambda v: AH @ v, y, tol=0.0, maxit=k)
        assert it == k
        K = np.empty((12, k), dtype=complex)
        v = b.copy()
        for j in range(k):
            K[:, j] = v
            v = AH @ (A @ v)
        Q, _ = np.linalg.qr(K)
        z = np.linalg.lstsq(A @ Q, y, rcond=None)[0]
        xs = Q @ z
        assert np.max(np.abs(xk - xs)) / np.max(np.abs(xs)) < 1e-10, k


@pytest.mark.parametrize("name", ["radial_db4_J8", "grid_db4_J9"])
def test_golden_files_match_their_cases(name):
    # the stored sampled rows are the oracle's T x of the case's seeded inputs
    # (guards the golden files against a drift of the input generators)
    import os

    from oracle.operator import Basis1D, Operator2D
    from tests.golden.cases import CASES

    c = CASES[name]()
    gold = np.load(os.path.join(os.path.dirname(__file__), "golden", name + ".npz"))
    rows = c["rows"][:32]
    op = Operator2D(Basis1D(c["p"], c["J"]), c["xi"][rows], None if c["mu"] is None else c["mu"][rows])
    assert np.max(np.abs(op.apply(c["x"]) - gold["T"][:32])) <= 1e-13 * np.max(np.abs(gold["T"]))
    n = (2 ** c["J"]) ** 2 if c["coefs"] is None else c["coefs"].size
    assert gold["TH"].shape == (n,) and np.all(np.isfinite(gold["TH"]))


# ------------------------------------------------------------------ 2D Voronoi weights (App. B)


def test_voronoi_2d_hand_worked():
    from oracle.weights import voronoi_2d

    # four points at (+-1, +-1) in [-2, 2]^2: each cell is a quadrant of area 4; the
    # farthest point of Y_K from its nearest sample is a corner, at distance sqrt2
    mu, delta = voronoi_2d(np.array([[1.0, 1.0], [-1.0, 1.0], [-1.0, -1.0], [1.0, -1.0]]), 2.0)
    assert np.allclose(mu, 4.0, rtol=0, atol=1e-14) and abs(delta - np.sqrt(2.0)) < 1e-14
    # (0, 0) and (2, 0) in [-2, 2]^2: the bisector x = 1 splits the square 12 : 4;
    # delta = |(-2, 2) - (0, 0)| = 2 sqrt2 (the right cell's farthest vertex is sqrt5 away)
    mu, delta = voronoi_2d(np.array([[0.0, 0.0], [2.0, 0.0]]), 2.0)
    assert np.allclose(mu, [12.0, 4.0], rtol=0, atol=1e-13) and abs(delta - 2.0 * np.sqrt(2.0)) < 1e-13


def test_voronoi_2d_partition_and_equivariance():
    from oracle.weights import voronoi_2d

    g = np.random.default_rng(31)
    xi = g.uniform(-4, 4, size=(120, 2))
    mu, delta = voronoi_2d(xi, 4.5)
    assert abs(mu.sum() - 81.0) < 1e-10 and np.all(mu > 0)  # the cells partition Y_K
    pi = g.permutation(xi.shape[0])
    mu2, delta2 = voronoi_2d(xi[pi], 4.5)
    assert np.allclose(mu2, mu[pi], rtol=0, atol=1e-12) and abs(delta2 - delta) < 1e-12


def test_voronoi_2d_reduces_to_1d_on_a_line():
    # points on the x axis: every cell spans the full height 2K, so the 2D weight is
    # 2K times the 1D Voronoi length of Sec. 4.1 (pinned on its own above)
    from oracle.weights import voronoi_2d

    g = np.random.default_rng(32)
    x = g.uniform(-5, 5, size=25)
    mu, _ = voronoi_2d(np.stack([x, np.zeros_like(x)], axis=1), 6.0)
    assert np.allclose(mu, 12.0 * voronoi_1d(x, 6.0), rtol=0, atol=1e-11)


def test_voronoi_2d_regular_grid():
    from oracle.weights import voronoi_2d

    k = np.arange(-3, 4) * 1.0  # 7 x 7 grid of spacing 1 in [-3.5, 3.5]^2
    X, Y = np.meshgrid(k, k)
    mu, delta = voronoi_2d(np.stack([X.ravel(), Y.ravel()], axis=1), 3.5)
    assert np.allclose(mu, 1.0, rtol=0, atol=1e-13) and abs(delta - np.sqrt(0.5)) < 1e-13


@pytest.mark.parametrize("p", [1, 4])
def test_factor_columns_subset_equals_full_rows(p):
    # the column-subset form of the factor rows (used for sampled T^H at sizes where
    # the full rows do not fit) takes the same entries as the full rows
    B = Basis1D(p, 6)
    xi = np.random.default_rng(41).uniform(-150, 150, 40)
    cols = np.array([0, 3, 5, 31, 32, 58, 60, 63])
    assert np.array_equal(B.factors(xi, cols), B.factors(xi)[:, cols])
