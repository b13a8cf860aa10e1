"""2D Voronoi density weights and the density delta on the GPU (App. B) against
the oracle's cells written out from the definition: every cell of small sets and
a jittered grid, sampled cells of a large set, the partition of Y_K, and a
solve weighted by them."""
import numpy as np
import pytest

from oracle.operator import Basis1D, Operator2D
from oracle.weights import cell_area, voronoi_2d, voronoi_cell_2d
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1607_04091_gb300 as gs  # noqa: E402


def test_voronoi_random_points_every_cell():
    g = synth.rng(71)
    xi = g.uniform(-6, 6, size=(300, 2))
    mu, delta = gs.gs_voronoi_2d(xi, 6.5)
    mo, do = voronoi_2d(xi, 6.5)
    assert np.max(np.abs(mu - mo)) <= 1e-12 * np.max(mo)
    assert abs(delta - do) <= 1e-12 * do


def test_voronoi_jittered_grid_and_hand_case():
    g = synth.rng(72)
    xi = synth.jitter_grid_2d(20, 1.0, g)
    mu, delta = gs.gs_voronoi_2d(xi, 10.0)
    mo, do = voronoi_2d(xi, 10.0)
    assert np.max(np.abs(mu - mo)) <= 1e-12 * np.max(mo) and abs(delta - do) <= 1e-12 * do
    mu, delta = gs.gs_voronoi_2d(np.array([[0.0, 0.0], [2.0, 0.0]]), 2.0)
    assert np.allclose(mu, [12.0, 4.0], rtol=0, atol=1e-13) and abs(delta - 2.0 * np.sqrt(2.0)) < 1e-13


def test_voronoi_large_set_sampled_cells_and_partition():
    g = synth.rng(73)
    xi = synth.spiral_2d(20000, 0.5)
    K = float(np.ceil(np.abs(xi).max())) + 1.0
    mu, delta = gs.gs_voronoi_2d(xi, K)
    assert abs(mu.sum() - (2 * K) ** 2) <= 1e-9 * (2 * K) ** 2  # the cells partition Y_K
    idx = g.choice(xi.shape[0], size=24, replace=False)
    ref = np.array([cell_area(voronoi_cell_2d(xi, i, K)) for i in idx])
    assert np.max(np.abs(mu[idx] - ref)) <= 1e-12 * np.max(ref)
    assert delta > 0


def test_voronoi_weighted_solve():
    J = 4
    N = 2**J
    xi = synth.jitter_grid_2d(40, 0.75, synth.rng(74))
    K = 15.5
    mu, _ = gs.gs_voronoi_2d(xi, K)
    op = Operator2D(Basis1D(4, J), xi, mu)
    xt = synth.ellipse_phantom(N, synth.rng(75)) + 0j
    y = op.apply(xt)
    plan = gs.Plan.plan_2d(xi, 4, J, weights=mu, direct=0)
    x, info = plan.solve(torch.tensor(y, device="cuda"), tol=1e-10, mode=gs.GS_SOLVE_FP64, maxit=2000)
    assert info["status"] == gs.GS_OK
    assert np.max(np.abs(x.cpu().numpy() - xt)) / np.max(np.abs(xt)) < 1e-8  # consistent data: exact recovery
