"""Iteration caps of gs_solve (GPU).

A solve stopped by its iteration cap ends after exactly maxit CGLS iterations,
for odd and even caps, on every path that runs the CG loop as a captured graph.
The captured loops hold two iterations per execution of their while body, so an
odd cap ends in the middle of a body and the iteration after the cap must
change nothing.  Paths covered:
  - float64 mode (one graph per CGLS pass, the plain CGLS step);
  - mixed mode at tol 1e-6 (the whole solve as one graph with nested loops);
  - mixed mode at tol 1e-12 (passes launched from the host, each pass a graph).
In float64 mode the capped iterate is also compared with the oracle's textbook
CGLS iterate after the same number of steps (Sec. 2, the CGLS recurrences): the
cap must stop the same sequence of iterates, not just count to the same number.
"""
import numpy as np
import pytest

from oracle.operator import Basis1D, Operator1D, Operator2D
from oracle.solvers import cgls
from oracle.weights import voronoi_1d
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1607_04091_gb300 as gs  # noqa: E402

CAPS = [1, 6, 7]
# A few CG steps of two float64 solvers whose applies differ by the NFFT error
# (window half-width 8, ~1e-12 relative per apply): a mildly amplified 1e-12.
ITERATE_TOL = 1e-8


def _dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.complex128, device="cuda")


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def _problem(dims):
    if dims == 2:
        g = synth.rng(1011)
        J = 4
        N = 2**J
        xi2 = synth.jitter_2d(2 * N, g)
        op = Operator2D(Basis1D(4, J), xi2)
        y = op.apply(synth.ellipse_phantom(N, g) + 0j) + 1e-2 * synth.complex_gaussian(xi2.shape[0], g)
        return op, gs.Plan.plan_2d(xi2, 4, J, direct=0), y
    g = synth.rng(1012)
    J = 8
    N = 2**J
    xi = synth.jitter_1d(2 * N, g)
    mu = voronoi_1d(xi, 2.0 * N)
    op = Operator1D(Basis1D(4, J), xi, mu)
    y = op.apply(synth.piecewise_smooth(N, g) + 0j) + 1e-2 * synth.complex_gaussian(xi.size, g) * np.sqrt(mu)
    return op, gs.Plan.plan_1d(xi, 4, J, bandwidth=2.0 * N, direct=0), y


@pytest.mark.parametrize("dims", [1, 2])
def test_fp64_cap_stops_at_the_oracle_iterate(dims):
    op, plan, y = _problem(dims)
    for k in CAPS:
        xo, it, _ = cgls(op.apply, op.adjoint, y, tol=0.0, maxit=k)
        assert it == k
        x, info = plan.solve(_dev(y), tol=1e-12, mode=gs.GS_SOLVE_FP64, maxit=k)
        assert info["status"] == gs.GS_ENOTCONV and info["iterations"] == k, (k, info)
        err = _rel(x.cpu().numpy(), xo)
        assert err < ITERATE_TOL, (k, err)


@pytest.mark.parametrize("dims", [1, 2])
@pytest.mark.parametrize("tol", [1e-6, 1e-12])
def test_mixed_cap_is_exact(dims, tol):
    op, plan, y = _problem(dims)
    ynorm = np.linalg.norm(y)
    for k in CAPS:
        x, info = plan.solve(_dev(y), tol=tol, mode=gs.GS_SOLVE_MIXED, maxit=k)
        assert info["status"] == gs.GS_ENOTCONV and info["iterations"] == k, (tol, k, info)
        # CGLS lowers the data residual at every step from x = 0
        res = np.linalg.norm(y - op.apply(x.cpu().numpy())) / ynorm
        assert res < 1.0, (tol, k, res)
