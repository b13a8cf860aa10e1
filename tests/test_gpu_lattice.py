"""The exact lattice path (Sec. 3.2: on a uniform grid the NDFT is a DFT with
phase shifts, no spreading) against the oracle's direct sums.

When sigma xi is an integer for every sample, the plan picks grid values (T)
and folds samples into grid points (T^H) with no Kaiser-Bessel window, so the
float64 applies match the oracle to rounding (1e-12 here, against 1e-10 on the
windowed path).  Cases: the paper's grid(M, eps) with eps = 1/2 in 1D (also the
four-step FFT size of Table 1's "Uniform 1D"), the tensor grid of "Uniform 2D"
at a smaller J, random lattice points with repeats (the folds sum them), and
mixed-precision solves on uniform grids.
"""
import numpy as np
import pytest

from oracle.operator import Basis1D, Operator1D, Operator2D
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1607_04091_gb300 as gs  # noqa: E402


def dev(a, prec):
    dt = torch.complex128 if prec == gs.GS_FP64 else torch.complex64
    return torch.tensor(np.asarray(a), dtype=dt, device="cuda")


def rel(a, b):
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(np.asarray(b)))


def tol_for(prec, n):
    return 1e-12 if prec == gs.GS_FP64 else 1e-6 * (1 + np.log2(n))


def grid_1d(M, eps):
    """The paper's grid(M, eps): xi_m = eps (m - 1 - M/2), m = 1..M."""
    return eps * (np.arange(1, M + 1) - 1 - M / 2)


def rand_c(g, n):
    return g.standard_normal(n) + 1j * g.standard_normal(n)


@pytest.mark.parametrize("prec", [gs.GS_FP64, gs.GS_FP32])
@pytest.mark.parametrize("p", [1, 4])
def test_lattice_1d_uniform_grid(prec, p):
    J = 8
    xi = grid_1d(4 * 2**J, 0.5)  # xi in [-512, 512): wraps twice
    op = Operator1D(Basis1D(p, J), xi)
    plan = gs.Plan.plan_1d(xi, p, J, direct=0, lattice=2)
    g = synth.rng(61)
    x, y = rand_c(g, 2**J), rand_c(g, xi.size)
    assert rel(plan.T(dev(x, prec), prec).cpu().numpy(), op.apply(x)) < tol_for(prec, 2 * 2**J)
    assert rel(plan.TH(dev(y, prec), prec).cpu().numpy(), op.adjoint(y)) < tol_for(prec, 2 * 2**J)


@pytest.mark.parametrize("prec", [gs.GS_FP64, gs.GS_FP32])
def test_lattice_1d_points_with_repeats(prec):
    J = 7
    g = synth.rng(62)
    xi = g.integers(-600, 600, size=900) / 2.0  # lattice points, many repeated
    mu = g.uniform(0.5, 1.5, size=xi.size)
    op = Operator1D(Basis1D(4, J), xi, mu)
    plan = gs.Plan.plan_1d(xi, 4, J, weights=mu, direct=0, lattice=2)
    x, y = rand_c(g, 2**J), rand_c(g, xi.size)
    assert rel(plan.T(dev(x, prec), prec).cpu().numpy(), op.apply(x)) < tol_for(prec, 2 * 2**J)
    assert rel(plan.TH(dev(y, prec), prec).cpu().numpy(), op.adjoint(y)) < tol_for(prec, 2 * 2**J)


@pytest.mark.parametrize("prec", [gs.GS_FP64, gs.GS_FP32])
def test_lattice_1d_four_step_size(prec):
    """Table 1's "Uniform 1D" shape: 8192 samples, 4096 coefficients (n = 8192,
    the four-step FFT); T on sampled rows, T^H on sampled coefficients."""
    J = 12
    xi = grid_1d(8192, 0.5)
    plan = gs.Plan.plan_1d(xi, 4, J, direct=0, lattice=2)
    g = synth.rng(63)
    x, y = rand_c(g, 2**J), rand_c(g, xi.size)
    B = Basis1D(4, J)
    rows = np.sort(g.choice(xi.size, 64, replace=False))
    assert rel(plan.T(dev(x, prec), prec).cpu().numpy()[rows], B.factors(xi[rows]) @ x) < tol_for(prec, 8192)
    z = plan.TH(dev(y, prec), prec).cpu().numpy()
    cols = np.r_[0:4, 4092:4096, np.sort(g.choice(np.arange(4, 4092), 56, replace=False))]
    zref = np.zeros(cols.size, dtype=complex)
    for s in range(0, xi.size, 1024):  # the oracle's factor rows, block by block
        zref += B.factors(xi[s:s + 1024])[:, cols].conj().T @ y[s:s + 1024]
    assert rel(z[cols], zref) < tol_for(prec, 8192)


def uniform_2d(N, eps=0.5):
    k = grid_1d(2 * N, eps)
    X, Y = np.meshgrid(k, k)
    return np.stack([X.ravel(), Y.ravel()], axis=1)


@pytest.mark.parametrize("prec", [gs.GS_FP64, gs.GS_FP32])
@pytest.mark.parametrize("p", [1, 2, 4])
def test_lattice_2d_tensor_grid(prec, p):
    J = 5
    xi = uniform_2d(2**J)  # (2N)^2 samples on the half-integer grid, [-N/2, N/2)^2
    op = Operator2D(Basis1D(p, J), xi)
    plan = gs.Plan.plan_2d(xi, p, J, direct=0, lattice=2)
    g = synth.rng(64 + p)
    x, y = rand_c(g, 4**J), rand_c(g, xi.shape[0])
    assert rel(plan.T(dev(x, prec), prec).cpu().numpy(), op.apply(x)) < tol_for(prec, 2 * 2**J)
    assert rel(plan.TH(dev(y, prec), prec).cpu().numpy(), op.adjoint(y)) < tol_for(prec, 2 * 2**J)


@pytest.mark.parametrize("prec", [gs.GS_FP64, gs.GS_FP32])
def test_lattice_2d_points_with_repeats(prec):
    J = 5
    g = synth.rng(66)
    xi = g.integers(-80, 80, size=(3000, 2)) / 2.0  # wraps, repeats, uneven density
    mu = g.uniform(0.5, 1.5, size=xi.shape[0])
    op = Operator2D(Basis1D(4, J), xi, mu)
    plan = gs.Plan.plan_2d(xi, 4, J, weights=mu, direct=0, lattice=2)
    x, y = rand_c(g, 4**J), rand_c(g, xi.shape[0])
    assert rel(plan.T(dev(x, prec), prec).cpu().numpy(), op.apply(x)) < tol_for(prec, 2 * 2**J)
    assert rel(plan.TH(dev(y, prec), prec).cpu().numpy(), op.adjoint(y)) < tol_for(prec, 2 * 2**J)


def test_lattice_and_windowed_paths_agree():
    """The same uniform 2D grid through the exact path and the Kaiser-Bessel path
    (lattice = 1): equal within the windowed path's float64 tolerance."""
    J = 5
    xi = uniform_2d(2**J)
    pe = gs.Plan.plan_2d(xi, 4, J, direct=0, lattice=2)
    pw = gs.Plan.plan_2d(xi, 4, J, direct=0, lattice=1)
    g = synth.rng(67)
    x = dev(rand_c(g, 4**J), gs.GS_FP64)
    assert rel(pe.T(x).cpu().numpy(), pw.T(x).cpu().numpy()) < 1e-10


@pytest.mark.parametrize("mode", [gs.GS_SOLVE_FP64, gs.GS_SOLVE_MIXED])
def test_lattice_2d_solve(mode):
    J = 5
    N = 2**J
    xi = uniform_2d(N)
    op = Operator2D(Basis1D(4, J), xi)
    g = synth.rng(68)
    xt = synth.ellipse_phantom(N, g) + 0j
    y = op.apply(xt) + 1e-3 * synth.complex_gaussian(xi.shape[0], g)
    plan = gs.Plan.plan_2d(xi, 4, J, direct=0, lattice=2)
    x, info = plan.solve(torch.tensor(y, device="cuda"), tol=1e-6, mode=mode, maxit=2000)
    assert info["status"] == gs.GS_OK, info
    xn = x.cpu().numpy()
    r = np.linalg.norm(op.adjoint(y - op.apply(xn))) / np.linalg.norm(op.adjoint(y))
    assert r <= 1.1e-6, r
