"""GPU parity of T x and T^H y (through the C ABI) against the FP64 oracle.

Tolerances (relative to the largest entry of the oracle result):
  GS_FP64, NFFT with Kaiser-Bessel m = 8, sigma = 2: 1e-10 (the window's
      aliasing error is ~exp(-beta m) ~ 4e-17 times a growth factor; the rest is
      float64 rounding of the FFT and the sums).
  GS_FP32, m = 4: 1e-6 (1 + log2 n): float32 rounding through log2 n FFT stages
      and the 2m-tap sums, plus the m = 4 window error of ~2e-8.
  direct mode: 1e-12 (float64) / 1e-5 (float32).
"""
import numpy as np
import pytest

from oracle.operator import Basis1D, Operator1D, Operator2D
from oracle.weights import voronoi_1d
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1607_04091_gb300 as gs  # noqa: E402


def dev(a, prec):
    dt = torch.complex128 if prec == gs.GS_FP64 else torch.complex64
    return torch.tensor(np.asarray(a), dtype=dt, device="cuda")


def rel(a, b):
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(np.asarray(b)))


def tol_for(prec, n, direct=False):
    if prec == gs.GS_FP64:
        return 1e-12 if direct else 1e-10
    return 1e-5 if direct else 1e-6 * (1 + np.log2(n))


def rand_c(g, n):
    return g.standard_normal(n) + 1j * g.standard_normal(n)


def check_pair(plan, op, ncoef, M, prec, tol, g):
    x = rand_c(g, ncoef)
    y = rand_c(g, M)
    yg = plan.T(dev(x, prec), prec).cpu().numpy()
    zg = plan.TH(dev(y, prec), prec).cpu().numpy()
    ey, ez = rel(yg, op.apply(x)), rel(zg, op.adjoint(y))
    assert ey < tol, f"T x: {ey:.3e} > {tol:.1e}"
    assert ez < tol, f"T^H y: {ez:.3e} > {tol:.1e}"
    return ey, ez


@pytest.mark.parametrize("prec", [gs.GS_FP64, gs.GS_FP32])
def test_haar_integer_grid_direct(prec):
    """Haar, J = 6, xi = -64..63 (the 128 x 64 case), direct evaluation."""
    xi, _ = synth.haar_integers()
    B = Basis1D(1, 6)
    op = Operator1D(B, xi)
    plan = gs.Plan.plan_1d(xi, 1, 6, direct=1)
    check_pair(plan, op, 64, 128, prec, tol_for(prec, 128, True), np.random.default_rng(5))


@pytest.mark.parametrize("p", [1, 2, 4])
@pytest.mark.parametrize("prec", [gs.GS_FP64, gs.GS_FP32])
def test_1d_nfft_jittered_wrapping(p, prec):
    """db-p, J = 9 (n = 1024: 8 spread tiles), ragged M, |xi/2^J| up to 2 (wraps)."""
    g = synth.rng(77 + p)
    J, M = 9, 3 * 512 + 17
    xi = g.uniform(-1024, 1024, M)
    mu = voronoi_1d(xi, 1024.0)
    op = Operator1D(Basis1D(p, J), xi, mu)
    plan = gs.Plan.plan_1d(xi, p, J, bandwidth=1024.0, direct=0)
    check_pair(plan, op, 2**J, M, prec, tol_for(prec, 2 * 2**J), g)


@pytest.mark.parametrize("prec", [gs.GS_FP64, gs.GS_FP32])
def test_1d_nfft_four_step_fft(prec):
    """J = 11: grid n = 4096 goes through the two-pass (four-step) FFT."""
    g = synth.rng(79)
    J, M = 11, 3001
    xi = g.uniform(-3000, 3000, M)
    op = Operator1D(Basis1D(4, J), xi)
    plan = gs.Plan.plan_1d(xi, 4, J, direct=0)
    check_pair(plan, op, 2**J, M, prec, tol_for(prec, 2 * 2**J), g)


def test_1d_direct_matches_nfft_mode():
    g = synth.rng(3)
    J, M = 7, 700
    xi = g.uniform(-300, 300, M)
    x = rand_c(g, 2**J)
    pd = gs.Plan.plan_1d(xi, 4, J, direct=1)
    pn = gs.Plan.plan_1d(xi, 4, J, direct=0)
    a = pd.T(dev(x, gs.GS_FP64)).cpu().numpy()
    b = pn.T(dev(x, gs.GS_FP64)).cpu().numpy()
    assert rel(b, a) < 1e-10


@pytest.mark.parametrize("p", [1, 2, 4])
@pytest.mark.parametrize("prec", [gs.GS_FP64, gs.GS_FP32])
def test_2d_nfft_random_wrapping(p, prec):
    """db-p, J = 5 (n = 64: 4 x 4 tiles), ragged M, frequencies to +-48 (wrap 1.5x)."""
    g = synth.rng(91 + p)
    J, M = 5, 3001
    xi2 = g.uniform(-48, 48, size=(M, 2))
    mu = g.uniform(0.5, 1.5, M)
    op = Operator2D(Basis1D(p, J), xi2, mu)
    plan = gs.Plan.plan_2d(xi2, p, J, weights=mu, direct=0)
    check_pair(plan, op, 4**J, M, prec, tol_for(prec, 2 * 2**J), g)


def test_2d_direct_small():
    g = synth.rng(11)
    J, M = 3, 257
    xi2 = g.uniform(-20, 20, size=(M, 2))
    op = Operator2D(Basis1D(2, J), xi2)
    plan = gs.Plan.plan_2d(xi2, 2, J, direct=1)
    check_pair(plan, op, 4**J, M, gs.GS_FP64, 1e-12, g)


def test_2d_clustered_center_load_balance():
    """Many samples in one tile (radial-like density): chunked work items."""
    g = synth.rng(12)
    J = 5
    xi2 = np.concatenate([g.normal(0, 0.7, size=(6000, 2)), g.uniform(-32, 32, size=(500, 2))])
    op = Operator2D(Basis1D(4, J), xi2)
    plan = gs.Plan.plan_2d(xi2, 4, J, direct=0)
    check_pair(plan, op, 4**J, xi2.shape[0], gs.GS_FP64, 1e-10, g)


@pytest.mark.parametrize("chunk", [1, 37, 128, 4096, -1])
def test_2d_work_item_sizes(chunk):
    """Work items of 1 sample up to whole tiles, and the autotuned size: the same
    operator (float64 to 1e-10, float32 to its tolerance), and the same bits on a
    second evaluation."""
    g = synth.rng(15)
    J = 5
    xi2 = np.concatenate([g.normal(0, 0.7, size=(3000, 2)), g.uniform(-32, 32, size=(700, 2))])
    M = xi2.shape[0]
    op = Operator2D(Basis1D(4, J), xi2)
    plan = gs.Plan.plan_2d(xi2, 4, J, direct=0, chunk=chunk)
    check_pair(plan, op, 4**J, M, gs.GS_FP64, 1e-10, g)
    x = rand_c(g, 4**J)
    y = rand_c(g, M)
    tol = tol_for(gs.GS_FP32, 2 * 2**J)
    a = plan.T(dev(x, gs.GS_FP32), gs.GS_FP32).cpu().numpy()
    b = plan.TH(dev(y, gs.GS_FP32), gs.GS_FP32).cpu().numpy()
    assert rel(a, op.apply(x)) < tol
    assert rel(b, op.adjoint(y)) < tol
    assert np.array_equal(a, plan.T(dev(x, gs.GS_FP32), gs.GS_FP32).cpu().numpy())
    assert np.array_equal(b, plan.TH(dev(y, gs.GS_FP32), gs.GS_FP32).cpu().numpy())


@pytest.mark.parametrize("p, clustered", [(4, False), (4, True), (2, False), (1, False)])
def test_2d_float64_apply_in_double_float(monkeypatch, p, clustered):
    """The float64 forward apply with its interpolation in double-float arithmetic
    (the refinement residual's apply; GS_DF64 routes every float64 apply there):
    within the float64 tolerance of the oracle and within 1e-12 of the float64
    kernel, for db4, db2 and Haar (no boundary columns)."""
    g = synth.rng(16)
    J = 5
    if clustered:
        xi2 = np.concatenate([g.normal(0, 0.7, size=(3000, 2)), g.uniform(-32, 32, size=(700, 2))])
    else:
        xi2 = g.uniform(-40, 40, size=(2500, 2))
    op = Operator2D(Basis1D(p, J), xi2)
    plan = gs.Plan.plan_2d(xi2, p, J, direct=0)
    x = rand_c(g, 4**J)
    monkeypatch.delenv("GS_DF64", raising=False)
    y64 = plan.T(dev(x, gs.GS_FP64), gs.GS_FP64).cpu().numpy()
    monkeypatch.setenv("GS_DF64", "1")
    ydf = plan.T(dev(x, gs.GS_FP64), gs.GS_FP64).cpu().numpy()
    assert rel(ydf, op.apply(x)) < 1e-10
    assert rel(ydf, y64) < 1e-12


def test_adjoint_identity_on_gpu():
    g = synth.rng(13)
    J, M = 6, 5000
    xi2 = g.uniform(-70, 70, size=(M, 2))
    plan = gs.Plan.plan_2d(xi2, 4, J, direct=0)
    for prec, tol in [(gs.GS_FP64, 1e-13), (gs.GS_FP32, 1e-5)]:
        x = rand_c(g, 4**J)
        y = rand_c(g, M)
        Tx = plan.T(dev(x, prec), prec).cpu().numpy().astype(np.complex128)
        Thy = plan.TH(dev(y, prec), prec).cpu().numpy().astype(np.complex128)
        a, b = np.vdot(y, Tx), np.vdot(Thy, x)
        assert abs(a - b) / abs(a) < tol


def test_2d_tensor_core_and_scalar_paths(monkeypatch):
    """db4, float32, 16 x 16 tiles: the tensor-core interpolation and spread
    (3xTF32) and the scalar kernels (GS_NO_TC=1) both meet the float32 tolerance
    against the oracle, on work items from 1 to 512 samples (dense centre,
    sparse rim, ragged last batches)."""
    g = synth.rng(14)
    J = 6
    xi2 = np.concatenate([g.normal(0, 3.0, size=(9000, 2)), g.uniform(-64, 64, size=(1237, 2))])
    M = xi2.shape[0]
    op = Operator2D(Basis1D(4, J), xi2)
    plan = gs.Plan.plan_2d(xi2, 4, J, direct=0)
    x = rand_c(g, 4**J)
    y = rand_c(g, M)
    ref_T, ref_TH = op.apply(x), op.adjoint(y)
    tol = tol_for(gs.GS_FP32, 2 * 2**J)
    out = {}
    for no_tc in (False, True):
        if no_tc:
            monkeypatch.setenv("GS_NO_TC", "1")
        else:
            monkeypatch.delenv("GS_NO_TC", raising=False)
        yg = plan.T(dev(x, gs.GS_FP32), gs.GS_FP32).cpu().numpy()
        zg = plan.TH(dev(y, gs.GS_FP32), gs.GS_FP32).cpu().numpy()
        assert rel(yg, ref_T) < tol, (no_tc, rel(yg, ref_T))
        assert rel(zg, ref_TH) < tol, (no_tc, rel(zg, ref_TH))
        out[no_tc] = (yg, zg)
    # the two float32 evaluations differ only by rounding
    assert rel(out[False][0], out[True][0]) < tol
    assert rel(out[False][1], out[True][1]) < tol


@pytest.mark.parametrize("prec", [gs.GS_FP32, gs.GS_FP64])
def test_adjoint_right_after_forward_on_one_stream(prec):
    """T^H (T x) with both applies queued back to back on one stream equals, bit for
    bit, the same two applies with the stream synchronised and q copied in between.
    The float32 adjoint's first kernel is launched as a programmatic dependent of
    the kernel before it (the forward interpolation here) and reads q only after
    waiting for that grid; an early read would show here."""
    g = synth.rng(77)
    xi2 = g.uniform(-48, 48, size=(6001, 2))
    plan = gs.Plan.plan_2d(xi2, 4, 5, direct=0)
    x = dev(rand_c(g, plan.ncoef), prec)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        zs = []
        for _ in range(3):
            q = plan.T(x, prec)
            zs.append(plan.TH(q, prec))
    st.synchronize()
    q = plan.T(x, prec)
    torch.cuda.synchronize()
    q2 = q.clone()
    torch.cuda.synchronize()
    z = plan.TH(q2, prec)
    torch.cuda.synchronize()
    ref = z.cpu().numpy()
    for zq in zs:
        assert np.array_equal(zq.cpu().numpy(), ref)
