"""Seeded synthetic inputs for generalized-sampling workloads.

This module is shared by the tests, the benchmark and the oracle checks.  It
holds NO arithmetic of the method itself (no phi-hat, no change-of-basis
entries, no weights that the method computes): only sampling patterns,
coefficient vectors and noise, drawn from numpy's PCG64 generator with the
stated seeds.  Data vectors y = T x* are formed by whoever calls this module.

Workloads (M samples, N = 2^J coefficients per dimension):
  haar_integers      Haar, J=6: xi = -64..63, x* ~ N(0,1) real          (seed 1001)
  jitter_1d          xi_k = k + 1/2 + U(-1/2,1/2), k = -K..K-1           (seed 1002)
  piecewise_smooth   x*_n = 2^-J/2 g(t_n), g with 4 random breakpoints and
                     random degree-<=3 pieces, t_n = (n - 1/2)/N - 1/2
  radial_2d          256 spokes theta_s = pi s/256, 1024 radii (j-511.5)/2;
                     polar cell areas |r| dr dtheta                       (seed 1003)
  ellipse_phantom    X* = 2^-J * sum of 10 random ellipses at cell centres
  jitter_2d, spiral_2d, batch_specs   mixed batch of 512 problems       (seed 4004)
  grid_1d, uniform_2d, jitter_grid_1d, jitter_grid_2d   the shapes of Table 1
"""
from dataclasses import dataclass

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ----------------------------------------------------------------- 1D patterns
def haar_integers(seed: int = 1001):
    """Integer frequencies -64..63 and a real N(0,1) coefficient vector, N = 64."""
    g = rng(seed)
    xi = np.arange(-64, 64, dtype=np.float64)
    x = g.standard_normal(64)
    return xi, x


def jitter_1d(K: int, g: np.random.Generator) -> np.ndarray:
    """xi_k = k + 1/2 + u_k, u_k ~ U(-1/2, 1/2), k = -K..K-1 (all inside (-K, K))."""
    k = np.arange(-K, K, dtype=np.float64)
    return k + 0.5 + g.uniform(-0.5, 0.5, size=k.size)


def piecewise_smooth(N: int, g: np.random.Generator, breaks: int = 4, degree: int = 3) -> np.ndarray:
    """Samples 2^-J/2 g(t_n) of a random piecewise polynomial on [-1/2, 1/2]."""
    t = (np.arange(1, N + 1) - 0.5) / N - 0.5
    bp = np.sort(g.uniform(-0.5, 0.5, size=breaks))
    edges = np.concatenate([[-0.5], bp, [0.5]])
    out = np.zeros(N)
    for a, b in zip(edges[:-1], edges[1:]):
        c = g.uniform(-1.0, 1.0, size=degree + 1)
        sel = (t >= a) & (t < b) if b < 0.5 else (t >= a)
        u = t[sel] - 0.5 * (a + b)
        out[sel] = np.polyval(c, 4.0 * u)
    return out / np.sqrt(N)


# ----------------------------------------------------------------- 2D patterns
def radial_2d(spokes: int = 256, points: int = 1024, dr: float = 0.5):
    """Radial pattern and its polar cell areas; xi is (M, 2) with (xi_x, xi_y) rows.

    Sample order: spoke-major (all radii of spoke 0, then spoke 1, ...).
    """
    theta = np.pi * np.arange(spokes) / spokes
    r = (np.arange(points) - (points - 1) / 2.0) * dr
    R, TH = np.meshgrid(r, theta)  # (spokes, points)
    xi = np.stack([(R * np.cos(TH)).ravel(), (R * np.sin(TH)).ravel()], axis=1)
    area = (np.abs(R) * dr * (np.pi / spokes)).ravel()
    return xi, area


def jitter_2d(K: int, g: np.random.Generator) -> np.ndarray:
    """Jittered unit grid over [-K, K)^2: (k + 1/2 + u, l + 1/2 + v)."""
    k = np.arange(-K, K, dtype=np.float64) + 0.5
    X, Y = np.meshgrid(k, k)
    xi = np.stack([X.ravel(), Y.ravel()], axis=1)
    return xi + g.uniform(-0.5, 0.5, size=xi.shape)


def spiral_2d(M: int, spacing: float = 1.0) -> np.ndarray:
    """Archimedean spiral r = spacing * theta / (2 pi), points `spacing` apart along the arc."""
    a = spacing / (2.0 * np.pi)
    pts = np.empty((M, 2))
    th = 0.0
    for i in range(M):
        r = a * th
        pts[i] = (r * np.cos(th), r * np.sin(th))
        # arc element ds = sqrt(r^2 + a^2) dtheta
        th += spacing / np.sqrt(r * r + a * a)
    return pts


def grid_1d(M: int, eps: float) -> np.ndarray:
    """The uniform grid xi_m = eps (m - 1 - M/2), m = 1..M (the paper's grid(M, eps))."""
    return eps * (np.arange(1, M + 1) - 1 - M / 2)


def uniform_2d(P: int, eps: float) -> np.ndarray:
    """Tensor grid of grid_1d(P, eps) with itself, (P^2, 2), x varying fastest."""
    k = grid_1d(P, eps)
    X, Y = np.meshgrid(k, k)
    return np.stack([X.ravel(), Y.ravel()], axis=1)


def jitter_grid_1d(M: int, spacing: float, g: np.random.Generator) -> np.ndarray:
    """M points spacing apart, centred on 0, each moved by U(-spacing/2, spacing/2)."""
    return grid_1d(M, spacing) + spacing * (0.5 + g.uniform(-0.5, 0.5, size=M))


def jitter_grid_2d(P: int, spacing: float, g: np.random.Generator) -> np.ndarray:
    """P x P points spacing apart, centred on 0, each coordinate moved by U(-spacing/4, spacing/4)."""
    xi = uniform_2d(P, spacing) + 0.5 * spacing
    return xi + g.uniform(-0.25 * spacing, 0.25 * spacing, size=xi.shape)


def ellipse_phantom(N: int, g: np.random.Generator, count: int = 10) -> np.ndarray:
    """2^-J * (sum of random ellipses) at cell centres, x-fastest (i + N*j)."""
    t = (np.arange(N) + 0.5) / N - 0.5
    X, Y = np.meshgrid(t, t)  # X varies along axis 1 (= x index i)
    img = np.zeros((N, N))
    for _ in range(count):
        cx, cy = g.uniform(-0.4, 0.4, size=2)
        ax, ay = g.uniform(0.05, 0.35, size=2)
        ang = g.uniform(0.0, np.pi)
        val = g.uniform(-1.0, 1.0)
        c, s = np.cos(ang), np.sin(ang)
        u = (X - cx) * c + (Y - cy) * s
        v = -(X - cx) * s + (Y - cy) * c
        img[(u / ax) ** 2 + (v / ay) ** 2 <= 1.0] += val
    return (img / N).ravel()


def tensor_phantom(N: int, g: np.random.Generator) -> np.ndarray:
    """Outer product of two random piecewise-smooth profiles (scaled like the
    ellipse phantom), x-fastest."""
    a = piecewise_smooth(N, g) * np.sqrt(N)
    b = piecewise_smooth(N, g) * np.sqrt(N)
    return (np.outer(b, a) / N).ravel()


def complex_gaussian(n: int, g: np.random.Generator) -> np.ndarray:
    """Unit-variance circular complex normal values (variance 1/2 in Re and Im)."""
    return (g.standard_normal(n) + 1j * g.standard_normal(n)) / np.sqrt(2.0)


# ----------------------------------------------------------------- the batch
@dataclass
class Problem:
    dim: int
    p: int
    J: int
    xi: np.ndarray  # (M,) or (M, 2)
    bandwidth: float  # > 0: 1D Voronoi weights on [-K, K]; 0: unit weights
    x_true: np.ndarray  # complex coefficients, N or N^2 (x-fastest)


def batch_specs(count: int = 512, seed: int = 4004, J1=(8, 13), J2=(6, 8)) -> list[Problem]:
    """Half 1D (db2 or db4, J in J1, oversampling r in {2,3,4}, jittered, spacing 1,
    K = r N / 2, Voronoi weights); half 2D (db4, J in J2, r in {2,3,4}; half jittered
    grid over [-K, K)^2 with K = round(sqrt(r) 2^(J-1)), half Archimedean spiral with
    r 4^J points; unit weights)."""
    g = rng(seed)
    out = []
    for i in range(count):
        r = int(g.integers(2, 5))
        if i < count // 2:
            p = 2 if g.uniform() < 0.5 else 4
            J = int(g.integers(J1[0], J1[1] + 1))
            N = 2**J
            K = r * N // 2
            xi = jitter_1d(K, g)
            x = piecewise_smooth(N, g) + 0j
            out.append(Problem(1, p, J, xi, float(K), x))
        else:
            J = int(g.integers(J2[0], J2[1] + 1))
            N = 2**J
            if (i - count // 2) % 2 == 0:
                K = int(round(np.sqrt(r) * 2 ** (J - 1)))
                xi = jitter_2d(K, g)
            else:
                xi = spiral_2d(r * 4**J)
            x = ellipse_phantom(N, g) + 0j
            out.append(Problem(2, 4, J, xi, 0.0, x))
    return out
