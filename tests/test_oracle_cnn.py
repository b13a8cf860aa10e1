"""Pins of the oracle CNN: its backward pass against central finite differences
of its own loss (an independent derivative), and its convolution against a
brute-force pixel loop."""
import numpy as np

from oracle.cnn import conv3, forward, loss_and_grads


def tiny(seed=0, chans=(2, 3, 3, 2), H=5, W=6, B=2):
    g = np.random.default_rng(seed)
    params = [(g.standard_normal((co, ci, 3, 3)) * 0.5, g.standard_normal(co) * 0.1)
              for ci, co in zip(chans[:-1], chans[1:])]
    u = g.standard_normal((B, chans[0], H, W))
    t = g.standard_normal((B, chans[-1], H, W))
    return params, u, t


def test_conv_matches_pixel_loop():
    g = np.random.default_rng(1)
    inp = g.standard_normal((1, 2, 4, 5))
    W = g.standard_normal((3, 2, 3, 3))
    b = g.standard_normal(3)
    out = conv3(inp, W, b)
    for o in range(3):
        for y in range(4):
            for x in range(5):
                s = b[o]
                for c in range(2):
                    for dy in range(3):
                        for dx in range(3):
                            yy, xx = y + dy - 1, x + dx - 1
                            if 0 <= yy < 4 and 0 <= xx < 5:
                                s += W[o, c, dy, dx] * inp[0, c, yy, xx]
                assert abs(out[0, o, y, x] - s) < 1e-12


def test_backward_matches_finite_differences():
    params, u, t = tiny()
    loss, grads = loss_and_grads(params, u, t)
    eps = 1e-6
    g = np.random.default_rng(2)
    for l, (W, b) in enumerate(params):
        for _ in range(6):
            idx = tuple(g.integers(0, s) for s in W.shape)
            Wp = W.copy(); Wp[idx] += eps
            Wm = W.copy(); Wm[idx] -= eps
            pp = list(params); pp[l] = (Wp, b)
            pm = list(params); pm[l] = (Wm, b)
            fd = (loss_and_grads(pp, u, t)[0] - loss_and_grads(pm, u, t)[0]) / (2 * eps)
            assert abs(fd - grads[l][0][idx]) < 1e-6 * max(1.0, abs(fd))
        k = int(g.integers(0, b.size))
        bp = b.copy(); bp[k] += eps
        bm = b.copy(); bm[k] -= eps
        pp = list(params); pp[l] = (W, bp)
        pm = list(params); pm[l] = (W, bm)
        fd = (loss_and_grads(pp, u, t)[0] - loss_and_grads(pm, u, t)[0]) / (2 * eps)
        assert abs(fd - grads[l][1][k]) < 1e-6 * max(1.0, abs(fd))


def test_residual_identity_with_zero_last_layer():
    params, u, t = tiny()
    W, b = params[-1]
    params[-1] = (np.zeros_like(W), np.zeros_like(b))
    x0, _ = forward(params, u)
    assert np.array_equal(x0, u)
