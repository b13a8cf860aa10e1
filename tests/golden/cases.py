"""Seeded inputs of the golden-file parity cases (no arithmetic of the method).

Each case returns the sampling pattern, density weights, basis parameters and
the seeded vectors that the oracle (tests/golden/make_golden.py) and the CUDA
path (tests/test_gpu_golden.py) both apply.  The stored expected values come
from the oracle only.

radial_db4_J8   the benchmark workload: 2D db4, J = 8, 256 spokes x 1024 radii
                (M = 262,144), polar-cell weights; u and x complex Gaussian
grid_db4_J9     the largest 2D grid the library plans (J = 9, oversampled grid
                n = 1024): 30,000 uniform frequencies in [-768, 768)^2 (they wrap
                1.5 times), unit weights
"""
import numpy as np

import synth


def radial_db4_J8():
    xi, mu = synth.radial_2d(256, 1024, 0.5)
    M, N = xi.shape[0], 256
    u = synth.complex_gaussian(M, synth.rng(3101))
    x = synth.complex_gaussian(N * N, synth.rng(3102))
    rows = np.sort(synth.rng(3103).choice(M, size=4096, replace=False))
    return dict(xi=xi, mu=mu, p=4, J=8, u=u, x=x, rows=rows, coefs=None)


def grid_db4_J9():
    g = synth.rng(3201)
    M, N = 30000, 512
    xi = g.uniform(-768.0, 768.0, size=(M, 2))
    u = synth.complex_gaussian(M, synth.rng(3202))
    x = synth.complex_gaussian(N * N, synth.rng(3203))
    rows = np.sort(synth.rng(3204).choice(M, size=2048, replace=False))
    # every coefficient whose row or column is a boundary index, plus a random set
    b = 4
    edge = np.r_[0:b, N - b:N]
    ii, jj = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    on_edge = np.isin(ii, edge) | np.isin(jj, edge)
    pick = np.zeros(N * N, dtype=bool)
    pick[(ii + N * jj)[on_edge]] = True
    pick[synth.rng(3205).choice(N * N, size=16384, replace=False)] = True
    return dict(xi=xi, mu=None, p=4, J=9, u=u, x=x, rows=rows, coefs=np.flatnonzero(pick))


CASES = {"radial_db4_J8": radial_db4_J8, "grid_db4_J9": grid_db4_J9}
