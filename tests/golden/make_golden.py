"""Write the golden files of tests/test_gpu_golden.py from the FP64 oracle.

Run from the repository root:  python tests/golden/make_golden.py
For each case of tests/golden/cases.py it stores, computed by oracle/ alone
(direct sums over the entries of T, Sec. 4, Sec. 5, App. C):
  TH     T^H u on the case's coefficient set (all coefficients, or `coefs`)
  T      (T x) on the case's sampled rows
in <case>.npz next to this script.  The oracle's factor rows are built block by
block of samples, so memory stays bounded at full size.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, HERE)

from oracle.operator import Basis1D, Operator2D  # noqa: E402
from cases import CASES  # noqa: E402


def adjoint_blocked(basis, xi, mu, u, block=16384):
    N = basis.N
    z = np.zeros(N * N, dtype=np.complex128)
    for s in range(0, xi.shape[0], block):
        e = min(xi.shape[0], s + block)
        op = Operator2D(basis, xi[s:e], None if mu is None else mu[s:e])
        z += op.adjoint(u[s:e])
    return z


def main(names):
    for name in names:
        c = CASES[name]()
        t0 = time.time()
        basis = Basis1D(c["p"], c["J"])
        z = adjoint_blocked(basis, c["xi"], c["mu"], c["u"])
        rows = c["rows"]
        op = Operator2D(basis, c["xi"][rows], None if c["mu"] is None else c["mu"][rows])
        t = op.apply(c["x"])
        coefs = c["coefs"]
        out = dict(TH=z if coefs is None else z[coefs], T=t)
        np.savez(os.path.join(HERE, name + ".npz"), **out)
        print(f"{name}: {time.time() - t0:.1f} s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(CASES))
