"""Element-wise parity at full size against oracle-written golden files.

tests/golden/make_golden.py stores, from the FP64 oracle alone, T^H u on every
coefficient (or a stated subset) and T x on sampled rows for the cases of
tests/golden/cases.py:
  radial_db4_J8  the benchmark workload in the launch configuration bench.py
                 times (2D db4, J = 8, M = 262,144 radial samples, polar-cell
                 weights, 512^2 grid, 16 x 16 tiles, dense radial centre)
  grid_db4_J9    the largest 2D grid (J = 9, n = 1024), frequencies wrapping
Both applies are compared coefficient by coefficient (sample by sample): float64
within 1e-10 relative, float32 within 1e-6 (1 + log2 n) (Sec. 3.2 NFFT; App. C).
"""
import os

import numpy as np
import pytest

from tests.golden.cases import CASES

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1607_04091_gb300 as gs  # noqa: E402

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def rel(a, b):
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(np.asarray(b)))


def tol_for(prec, n):
    return 1e-10 if prec == gs.GS_FP64 else 1e-6 * (1 + np.log2(n))


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    c = CASES[request.param]()
    gold = np.load(os.path.join(HERE, request.param + ".npz"))
    plan = gs.Plan.plan_2d(c["xi"], c["p"], c["J"], weights=c["mu"])
    yield request.param, c, gold, plan
    del plan


@pytest.mark.parametrize("prec", [gs.GS_FP64, gs.GS_FP32])
def test_golden_adjoint_every_coefficient(case, prec):
    name, c, gold, plan = case
    dt = torch.complex128 if prec == gs.GS_FP64 else torch.complex64
    z = plan.TH(torch.tensor(c["u"], dtype=dt, device="cuda"), prec).cpu().numpy()
    if c["coefs"] is not None:
        z = z[c["coefs"]]
    err = rel(z, gold["TH"])
    assert err < tol_for(prec, 2 * 2 ** c["J"]), (name, err)


@pytest.mark.parametrize("prec", [gs.GS_FP64, gs.GS_FP32])
def test_golden_forward_sampled_rows(case, prec):
    name, c, gold, plan = case
    dt = torch.complex128 if prec == gs.GS_FP64 else torch.complex64
    y = plan.T(torch.tensor(c["x"], dtype=dt, device="cuda"), prec).cpu().numpy()
    err = rel(y[c["rows"]], gold["T"])
    assert err < tol_for(prec, 2 * 2 ** c["J"]), (name, err)
