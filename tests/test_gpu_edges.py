"""GPU edge cases against the oracle: a single sample (1D and 2D, NFFT path with
one work item holding one sample), the largest 2D grid (J = 9, n = 1024) and the
largest 1D grid (J = 19, n = 2^20, the four-step FFT at n1 = n2 = 1024).  The
large cases compare T x on sampled rows the oracle evaluates one by one, check
the adjoint identity, and (1D) compare T^H on sampled coefficients (the 2D
J = 9 grid's T^H is compared through golden files, tests/test_gpu_golden.py)."""
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
    return 1e-10 if prec == gs.GS_FP64 else 1e-6 * (1 + np.log2(n))


def rand_c(g, n):
    return g.standard_normal(n) + 1j * g.standard_normal(n)


def adjoint_gap(plan, prec, g):
    x = rand_c(g, plan.ncoef)
    y = rand_c(g, plan.M)
    Tx = plan.T(dev(x, prec), prec).cpu().numpy().astype(np.complex128)
    Thy = plan.TH(dev(y, prec), prec).cpu().numpy().astype(np.complex128)
    a, b = np.vdot(y, Tx), np.vdot(Thy, x)
    return abs(a - b) / abs(a)


@pytest.mark.parametrize("prec", [gs.GS_FP64, gs.GS_FP32])
def test_single_sample_1d(prec):
    g = synth.rng(51)
    xi = np.array([13.7])
    op = Operator1D(Basis1D(4, 6), xi)
    plan = gs.Plan.plan_1d(xi, 4, 6, direct=0)
    x, y = rand_c(g, 64), rand_c(g, 1)
    assert rel(plan.T(dev(x, prec), prec).cpu().numpy(), op.apply(x)) < tol_for(prec, 128)
    assert rel(plan.TH(dev(y, prec), prec).cpu().numpy(), op.adjoint(y)) < tol_for(prec, 128)


@pytest.mark.parametrize("prec", [gs.GS_FP64, gs.GS_FP32])
def test_single_sample_2d(prec):
    g = synth.rng(52)
    xi = np.array([[3.2, -7.9]])
    op = Operator2D(Basis1D(4, 5), xi)
    plan = gs.Plan.plan_2d(xi, 4, 5, direct=0)
    x, y = rand_c(g, 4**5), rand_c(g, 1)
    assert rel(plan.T(dev(x, prec), prec).cpu().numpy(), op.apply(x)) < tol_for(prec, 64)
    assert rel(plan.TH(dev(y, prec), prec).cpu().numpy(), op.adjoint(y)) < tol_for(prec, 64)


@pytest.mark.parametrize("prec", [gs.GS_FP64, gs.GS_FP32])
def test_largest_2d_grid(prec):
    g = synth.rng(53)
    J, M = 9, 30000
    xi = g.uniform(-768, 768, size=(M, 2))  # |xi / 2^J| up to 1.5: wraps
    plan = gs.Plan.plan_2d(xi, 4, J, direct=0)
    x = rand_c(g, 4**J)
    idx = np.sort(g.choice(M, size=128, replace=False))
    rows = Operator2D(Basis1D(4, J), xi[idx]).apply(x)
    y = plan.T(dev(x, prec), prec).cpu().numpy()
    assert rel(y[idx], rows) < tol_for(prec, 2 * 2**J)
    assert adjoint_gap(plan, prec, g) < (1e-12 if prec == gs.GS_FP64 else 1e-5)


@pytest.mark.parametrize("prec", [gs.GS_FP64, gs.GS_FP32])
def test_largest_1d_grid(prec):
    g = synth.rng(54)
    J, M = 19, 100000
    N = 2**J
    xi = g.uniform(-N, N, size=M)  # |xi / 2^J| up to 1: wraps
    plan = gs.Plan.plan_1d(xi, 4, J, direct=0)
    x = rand_c(g, N)
    idx = np.sort(g.choice(M, size=16, replace=False))
    B = Basis1D(4, J)
    rows = B.factors(xi[idx]) @ x
    y = plan.T(dev(x, prec), prec).cpu().numpy()
    assert rel(y[idx], rows) < tol_for(prec, 2 * N)
    assert adjoint_gap(plan, prec, g) < (1e-12 if prec == gs.GS_FP64 else 1e-5)
    # T^H element by element on the boundary coefficients and 56 sampled interior ones
    u = rand_c(g, M)
    cols = np.r_[0:4, N - 4:N, np.sort(g.choice(np.arange(4, N - 4), 56, replace=False))]
    zref = np.zeros(cols.size, dtype=complex)
    for s in range(0, M, 20000):
        zref += B.factors(xi[s:s + 20000], cols).conj().T @ u[s:s + 20000]
    z = plan.TH(dev(u, prec), prec).cpu().numpy()
    assert rel(z[cols], zref) < tol_for(prec, 2 * N)
