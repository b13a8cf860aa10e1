"""The learned warm start's kernels (GPU) against the float64 oracle CNN.

Gradients of the float32 training path must match the oracle's backpropagation
to 2e-4 relative (float32 accumulation over up to 16 x 16 x 2 pixels and 32
channels); the float32 forward to 1e-5, the bfloat16-weight forward to 2e-2
(8-bit mantissa weights).  Training steps decrease the loss.  The learned
solve meets the tolerance by the oracle's FP64 residual whichever start it
takes.
"""
import numpy as np
import pytest

from oracle.cnn import forward as oforward, loss_and_grads
from oracle.operator import Basis1D, Operator2D
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1607_04091_gb300 as gs  # noqa: E402


def rand_net(H=16, W=32, channels=8, depth=3, B=2, seed=0):
    net = gs.Cnn(H, W, channels=channels, depth=depth, max_batch=B, seed=seed)
    g = np.random.default_rng(seed)
    w = g.standard_normal(net.weights().size).astype(np.float32) * 0.3
    net.set_weights(w)
    u = g.standard_normal((B, 2, H, W)).astype(np.float32)
    t = g.standard_normal((B, 2, H, W)).astype(np.float32)
    return net, w, u, t


def test_gradients_match_oracle():
    net, w, u, t = rand_net()
    loss, gg = net.gradients(torch.tensor(u, device="cuda"), torch.tensor(t, device="cuda"))
    params = [(W.astype(np.float64), b.astype(np.float64)) for W, b in net.unflatten(w)]
    oloss, ograds = loss_and_grads(params, u.astype(np.float64), t.astype(np.float64))
    assert abs(loss - oloss) / oloss < 1e-5
    gl = net.unflatten(gg)
    for (gW, gb), (oW, ob) in zip(gl, ograds):
        assert np.max(np.abs(gW - oW)) <= 2e-4 * np.max(np.abs(oW))
        assert np.max(np.abs(gb - ob)) <= 2e-4 * np.max(np.abs(ob))


@pytest.mark.parametrize("bf16,tol", [(False, 1e-5), (True, 2e-2)])
def test_forward_matches_oracle(bf16, tol):
    net, w, u, t = rand_net(seed=3)
    x0 = net.forward(torch.tensor(u, device="cuda"), bf16=bf16).cpu().numpy()
    params = [(W.astype(np.float64), b.astype(np.float64)) for W, b in net.unflatten(w)]
    ox, _ = oforward(params, u.astype(np.float64))
    assert np.max(np.abs(x0 - ox)) <= tol * np.max(np.abs(ox - u))


def test_untrained_net_is_identity_and_training_reduces_loss():
    net = gs.Cnn(32, 32, channels=8, depth=3, max_batch=4, seed=5)
    g = np.random.default_rng(6)
    u = torch.tensor(g.standard_normal((4, 2, 32, 32)).astype(np.float32), device="cuda")
    assert torch.equal(net.forward(u, bf16=False), u)
    t = 0.5 * u + 0.1
    losses = [net.train_step(u, t, lr=3e-3) for _ in range(60)]
    assert losses[-1] < 0.5 * losses[0]


def test_learned_solve_meets_tolerance():
    J = 5
    N = 2**J
    xi, mu = synth.radial_2d(64, 128, 0.5)
    op = Operator2D(Basis1D(4, J), xi, mu)
    g = synth.rng(21)
    xt = synth.ellipse_phantom(N, g) + 0j
    y = op.apply(xt) + 1e-3 * synth.complex_gaussian(op.M, g) * np.sqrt(mu)
    plan = gs.Plan.plan_2d(xi, 4, J, weights=mu)
    net = gs.Cnn(N, N, channels=8, depth=3, max_batch=1, seed=7)
    x = torch.zeros(plan.ncoef, dtype=torch.complex128, device="cuda")
    info, used = gs.gs_solve_learned(plan.handle, net, torch.tensor(y, device="cuda"), x, tol=1e-6, maxit=3000)
    assert info["status"] == gs.GS_OK
    r = np.linalg.norm(op.adjoint(y - op.apply(x.cpu().numpy()))) / np.linalg.norm(op.adjoint(y))
    assert r <= 1.1e-6
