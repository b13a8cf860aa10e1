"""GPU parity at the full sizes of the benchmark configurations.

cfg 2 (1D db4, J = 10, 4096 jittered samples in (-2048, 2048), Voronoi weights):
small enough for the whole oracle, so T, T^H and a mixed-precision solve are
compared entry by entry.

cfg 3 (the bench workload: 2D db4, J = 8, 256 x 1024 radial samples, polar-cell
weights, M = 262,144) in the launch configuration bench.py times: the oracle's
factor rows for all samples take minutes, so T x is compared on 1024 sampled
rows that the oracle evaluates one by one; T^H is checked through the adjoint
identity <T x, y> = <x, T^H y> (which holds at any size; its parity with the
oracle is tested at smaller sizes); the solve is checked by its float64
normal-equation residual.
"""
import os
import sys

import numpy as np
import pytest

from oracle.operator import Basis1D, Operator1D, Operator2D
from oracle.weights import voronoi_1d
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1607_04091_gb300 as gs  # noqa: E402

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def dev(a, prec):
    dt = torch.complex128 if prec == gs.GS_FP64 else torch.complex64
    return torch.tensor(np.asarray(a), dtype=dt, device="cuda")


def rel(a, b):
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(np.asarray(b)))


def tol_for(prec, n):
    return 1e-10 if prec == gs.GS_FP64 else 1e-6 * (1 + np.log2(n))


@pytest.mark.parametrize("prec", [gs.GS_FP64, gs.GS_FP32])
def test_cfg2_1d_db4_J10_full_oracle(prec):
    g = synth.rng(1002)
    J, K = 10, 2048
    xi = synth.jitter_1d(K, g)
    mu = voronoi_1d(xi, float(K))
    xstar = synth.piecewise_smooth(2**J, g) + 0j
    op = Operator1D(Basis1D(4, J), xi, mu)
    plan = gs.Plan.plan_1d(xi, 4, J, bandwidth=float(K), direct=0)
    tol = tol_for(prec, 2 * 2**J)
    y_ref = op.apply(xstar)
    assert rel(plan.T(dev(xstar, prec), prec).cpu().numpy(), y_ref) < tol
    u = g.standard_normal(xi.size) + 1j * g.standard_normal(xi.size)
    assert rel(plan.TH(dev(u, prec), prec).cpu().numpy(), op.adjoint(u)) < tol
    if prec == gs.GS_FP32:  # the mixed solve to 1e-6, checked by the oracle's float64 residual
        y = y_ref + 1e-3 * synth.complex_gaussian(xi.size, g) * np.sqrt(mu)
        x, info = plan.solve(torch.tensor(y, device="cuda"), tol=1e-6)
        assert info["status"] == gs.GS_OK
        xn = x.cpu().numpy()
        r = np.linalg.norm(op.adjoint(y - op.apply(xn))) / np.linalg.norm(op.adjoint(y))
        assert r <= 1.1e-6, r


@pytest.fixture(scope="module")
def cfg3():
    xi, mu, xstar, _ = bench.workload()
    plan = gs.Plan.plan_2d(xi, bench.P_VM, bench.J, weights=mu)
    return xi, mu, xstar, plan


@pytest.mark.parametrize("prec", [gs.GS_FP64, gs.GS_FP32])
def test_cfg3_radial_T_on_sampled_rows(cfg3, prec):
    xi, mu, xstar, plan = cfg3
    g = synth.rng(31)
    idx = np.sort(g.choice(xi.shape[0], size=1024, replace=False))
    y = plan.T(dev(xstar, prec), prec).cpu().numpy()
    rows = Operator2D(Basis1D(bench.P_VM, bench.J), xi[idx], mu[idx]).apply(xstar)
    assert rel(y[idx], rows) < tol_for(prec, 2 * 2**bench.J)


@pytest.mark.parametrize("prec,tol", [(gs.GS_FP64, 1e-12), (gs.GS_FP32, 1e-5)])
def test_cfg3_radial_adjoint_identity(cfg3, prec, tol):
    xi, mu, xstar, plan = cfg3
    g = synth.rng(32)
    x = g.standard_normal(plan.ncoef) + 1j * g.standard_normal(plan.ncoef)
    y = g.standard_normal(plan.M) + 1j * g.standard_normal(plan.M)
    Tx = plan.T(dev(x, prec), prec).cpu().numpy().astype(np.complex128)
    Thy = plan.TH(dev(y, prec), prec).cpu().numpy().astype(np.complex128)
    a, b = np.vdot(y, Tx), np.vdot(Thy, x)
    assert abs(a - b) / abs(a) < tol


def test_cfg3_radial_mixed_solve_meets_tolerance(cfg3):
    xi, mu, xstar, plan = cfg3
    y_clean = plan.T(torch.tensor(xstar, device="cuda")).cpu().numpy()
    sig = 0.01 * np.sqrt(np.mean(np.abs(y_clean) ** 2))
    y = y_clean + sig * synth.complex_gaussian(xi.shape[0], synth.rng(33))
    x, info = plan.solve(torch.tensor(y, device="cuda"), tol=1e-6, maxit=5000)
    assert info["status"] == gs.GS_OK
    assert info["rel_normres"] <= 1e-6
    # the float64 residual of the returned x, recomputed through float64 applies
    xd = x.clone()
    r = torch.tensor(y, device="cuda") - plan.T(xd)
    nr = torch.linalg.norm(plan.TH(r)).item() / torch.linalg.norm(plan.TH(torch.tensor(y, device="cuda"))).item()
    assert nr <= 1.1e-6, nr
