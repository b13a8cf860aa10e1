"""GPU gs_solve against the oracle's least-squares solution.

FP64 mode: the CGLS solution matches the oracle's (Householder QR or textbook
CGLS) to 1e-10 relative once both are run to a normal-equation residual of
1e-12 or below.  Mixed mode (float32 passes, float64 refinement) must reach the
same tolerance on the FP64 residual and the same solution within 1e-8.
"""
import numpy as np
import pytest

from oracle.operator import Basis1D, Operator1D, Operator2D
from oracle.solvers import cgls, qr_lstsq
from oracle.weights import voronoi_1d
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1607_04091_gb300 as gs  # noqa: E402


def dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.complex128, device="cuda")


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def test_haar_integer_grid_solve():
    xi, xt = synth.haar_integers()
    op = Operator1D(Basis1D(1, 6), xi)
    y = op.apply(xt)
    plan = gs.Plan.plan_1d(xi, 1, 6)
    x, info = plan.solve(dev(y), tol=1e-12, mode=gs.GS_SOLVE_FP64)
    assert info["status"] == gs.GS_OK and info["rel_normres"] <= 1e-12
    assert rel(x.cpu().numpy(), xt) < 1e-10  # exact recovery of the real coefficients
    assert rel(x.cpu().numpy(), qr_lstsq(op.T, y)) < 1e-10


@pytest.mark.parametrize("mode", [gs.GS_SOLVE_FP64, gs.GS_SOLVE_MIXED])
def test_1d_db4_jitter_solve(mode):
    g = synth.rng(1002)
    J = 8
    N = 2**J
    xi = synth.jitter_1d(2 * N, g)
    mu = voronoi_1d(xi, 2.0 * N)
    op = Operator1D(Basis1D(4, J), xi, mu)
    xt = synth.piecewise_smooth(N, g) + 0j
    y = op.apply(xt) + 1e-3 * synth.complex_gaussian(xi.size, g) * np.sqrt(mu)
    xq = qr_lstsq(op.T, y)
    plan = gs.Plan.plan_1d(xi, 4, J, bandwidth=2.0 * N, direct=0)
    x, info = plan.solve(dev(y), tol=1e-12, mode=mode, maxit=2000)
    assert info["status"] == gs.GS_OK, info
    assert info["rel_normres"] <= 1e-12
    assert rel(x.cpu().numpy(), xq) < (1e-10 if mode == gs.GS_SOLVE_FP64 else 1e-8)


@pytest.mark.parametrize("mode", [gs.GS_SOLVE_FP64, gs.GS_SOLVE_MIXED])
def test_2d_db4_solve_matches_oracle_cgls(mode):
    g = synth.rng(1003)
    J = 4
    N = 2**J
    xi2 = synth.jitter_2d(2 * N // 2 * 2, g)  # (2N)^2 = 4 N^2 samples over [-N, N)^2
    op = Operator2D(Basis1D(4, J), xi2)
    xt = synth.ellipse_phantom(N, g) + 0j
    y = op.apply(xt)
    xo, it, _ = cgls(op.apply, op.adjoint, y, tol=1e-13, maxit=3000)
    plan = gs.Plan.plan_2d(xi2, 4, J, direct=0)
    x, info = plan.solve(dev(y), tol=1e-11, mode=mode, maxit=3000)
    assert info["status"] == gs.GS_OK, info
    assert rel(x.cpu().numpy(), xo) < (1e-9 if mode == gs.GS_SOLVE_FP64 else 1e-8)
    assert rel(x.cpu().numpy(), xt) < 1e-8  # consistent data: exact recovery


@pytest.mark.parametrize("p", [1, 2])
def test_2d_mixed_solve_other_boundary_widths(p):
    """Mixed solves of 2D Haar (no boundary columns) and db2 (2b = 4): the fused
    CG step, which updates the boundary columns of the direction in the forward
    pass and the interior ones in the adjoint's last pass, reaches the oracle's
    CGLS solution."""
    g = synth.rng(1004 + p)
    J = 4
    N = 2**J
    xi2 = synth.jitter_2d(2 * N, g)
    op = Operator2D(Basis1D(p, J), xi2)
    xt = synth.ellipse_phantom(N, g) + 0j
    y = op.apply(xt)
    xo, it, _ = cgls(op.apply, op.adjoint, y, tol=1e-13, maxit=3000)
    plan = gs.Plan.plan_2d(xi2, p, J, direct=0)
    x, info = plan.solve(dev(y), tol=1e-11, mode=gs.GS_SOLVE_MIXED, maxit=3000)
    assert info["status"] == gs.GS_OK, info
    assert rel(x.cpu().numpy(), xo) < 1e-8
