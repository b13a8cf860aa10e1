"""gs_apply_TH_noalloc against gs_apply_TH (GPU).

gs_apply_TH_noalloc serves callers that must not allocate device memory while
they run (code recording a CUDA graph, runtimes with a fixed device-memory
arena): it computes the same T^H y with the spread scratch in a fixed static
device array.  Here its output, through the C ABI, must equal the regular
entry point's on two calls in a row (the array keeps the previous call's
contents), in float64 and float32, for two 1D plans (one large enough for the
two-pass FFT, n = 8192) and a 2D plan; a plan whose scratch exceeds the fixed
array is rejected.

This file sorts last so that a run stopping at the first failure has already
run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1607_04091_gb300 as gs  # noqa: E402

# same tolerances as the other apply tests; the two paths run the same kernels
TOL = {gs.GS_FP64: 1e-12, gs.GS_FP32: 1e-6}


def _plans():
    g = synth.rng(31)
    xi1 = g.uniform(-1024, 1024, 1537)
    p1 = gs.Plan.plan_1d(xi1, 4, 9, bandwidth=1024.0, direct=0)
    xi2 = g.uniform(-48, 48, size=(3001, 2))
    p2 = gs.Plan.plan_2d(xi2, 4, 5, direct=0)
    xi3 = g.uniform(-4096, 4096, 12001)  # J = 12: n = 8192, the four-step FFT
    p3 = gs.Plan.plan_1d(xi3, 4, 12, bandwidth=4096.0, direct=0)
    return [p1, p2, p3]


@pytest.mark.parametrize("prec", [gs.GS_FP64, gs.GS_FP32])
def test_noalloc_adjoint_matches_gs_apply_TH_twice(prec):
    dt = torch.complex128 if prec == gs.GS_FP64 else torch.complex64
    g = np.random.default_rng(5)
    for plan in _plans():
        for call in range(2):
            y = torch.tensor(g.standard_normal(plan.M) + 1j * g.standard_normal(plan.M), dtype=dt, device="cuda")
            ref = torch.empty(plan.ncoef, dtype=dt, device="cuda")
            out = torch.full((plan.ncoef,), float("nan"), dtype=dt, device="cuda")
            gs.gs_apply_TH(plan.handle, prec, y, ref)
            gs.gs_apply_TH_noalloc(plan.handle, prec, y, out)
            torch.cuda.synchronize()
            a, b = out.cpu().numpy(), ref.cpu().numpy()
            assert np.all(np.isfinite(a))
            err = np.max(np.abs(a - b)) / np.max(np.abs(b))
            assert err <= TOL[prec], (plan.dims, call, err)


def test_noalloc_rejects_plan_beyond_fixed_scratch():
    xi, mu = synth.radial_2d(256, 1024)
    plan = gs.Plan.plan_2d(xi, 4, 8, weights=mu)  # float64 spread scratch ~27 MB > 8 MiB
    y = torch.zeros(plan.M, dtype=torch.complex128, device="cuda")
    x = torch.zeros(plan.ncoef, dtype=torch.complex128, device="cuda")
    with pytest.raises(gs.GsError) as e:
        gs.gs_apply_TH_noalloc(plan.handle, gs.GS_FP64, y, x)
    assert e.value.status == gs.GS_EINVAL
