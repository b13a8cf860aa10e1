"""The learned warm start gains over the plain method (GPU, small geometry).

A residual CNN is trained by the library's kernels on pairs the method itself
produced (T^H y, CGLS solution) for a 32 x 32 db4 radial problem; on held-out
data the learned start must need at least 5% fewer CGLS iterations to the 1e-6
tolerance than both starts without the network -- from zero and from the
density-compensated adjoint u = T^H y (the untrained, identity net) -- and every
solve must meet the tolerance by the oracle's FP64 residual.  The geometry is a
sparse radial pattern (32 spokes x 256 radii), where CGLS needs ~90 iterations;
on denser patterns the solve converges in ~28 and any start saves little.
"""
import numpy as np
import pytest

from oracle.operator import Basis1D, Operator2D
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1607_04091_gb300 as gs  # noqa: E402


def test_learned_start_gain():
    J = 5
    N = 2**J
    xi, mu = synth.radial_2d(32, 256, 0.5)
    plan = gs.Plan.plan_2d(xi, 4, J, weights=mu)
    op = Operator2D(Basis1D(4, J), xi, mu)

    def problem(seed):
        g = synth.rng(700 + seed)
        xs = (synth.ellipse_phantom(N, g) if seed % 2 == 0 else synth.tensor_phantom(N, g)) + 0j
        yc = op.apply(xs)
        return yc + 0.01 * np.sqrt(np.mean(np.abs(yc) ** 2)) * synth.complex_gaussian(yc.size, g)

    ntrain, B = 192, 8
    U = torch.empty((ntrain, 2, N, N), dtype=torch.float32, device="cuda")
    X = torch.empty_like(U)
    for k in range(ntrain):
        y = torch.tensor(problem(k), device="cuda")
        x, _ = plan.solve(y, tol=1e-6, maxit=4000)
        u, xt = gs.gs_cnn_pair(plan.handle, y, x)
        U[k].copy_(u[0])
        X[k].copy_(xt[0])
    net = gs.Cnn(N, N, channels=32, depth=6, max_batch=B, seed=3)
    ident = gs.Cnn(N, N, channels=32, depth=6, max_batch=1, seed=3)
    g = np.random.default_rng(4)
    losses = []
    for ep in range(40):
        order = g.permutation(ntrain)
        for s0 in range(0, ntrain - B + 1, B):
            idx = torch.tensor(order[s0:s0 + B], device="cuda")
            losses.append(net.train_step(U[idx].contiguous(), X[idx].contiguous(), lr=2e-3))
    assert np.mean(losses[-6:]) < 0.5 * losses[0]
    its = {"zero": [], "adjoint": [], "learned": []}
    for k in range(8):
        yn = problem(1000 + k)
        y = torch.tensor(yn, device="cuda")
        for key in its:
            x = torch.zeros(plan.ncoef, dtype=torch.complex128, device="cuda")
            if key == "zero":
                info = gs.gs_solve(plan.handle, y, x, tol=1e-6, maxit=4000)
            else:
                info, _ = gs.gs_solve_learned(plan.handle, ident if key == "adjoint" else net, y, x, tol=1e-6,
                                              maxit=4000)
            assert info["status"] == gs.GS_OK
            r = np.linalg.norm(op.adjoint(yn - op.apply(x.cpu().numpy()))) / np.linalg.norm(op.adjoint(yn))
            assert r <= 1.1e-6
            its[key].append(info["iterations"])
    mean = {k: float(np.mean(v)) for k, v in its.items()}
    print("mean CGLS iterations to 1e-6:", mean)
    msg = f"mean CGLS iterations to 1e-6: {mean}"
    assert mean["learned"] <= 0.95 * mean["adjoint"], msg
    assert mean["learned"] <= 0.95 * mean["zero"], msg
