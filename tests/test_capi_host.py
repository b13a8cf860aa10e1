"""Host-side checks of the C ABI (no GPU): the library loads, exports every
function include/gs.h declares, validates arguments before touching CUDA, and
its plan-time constants match the oracle's independent construction."""
import os
import re

import numpy as np
import pytest

import paper_1607_04091_gb300 as gs
from oracle.boundary import EdgeSide
from oracle.filters import daubechies_filter

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "gs.h")


def declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:gs_status|void|const char\*)\s+(gs_\w+)\s*\(", txt, re.M)))


def test_library_exports_every_declared_symbol():
    lib = gs.load()
    names = declared()
    assert "gs_apply_T" in names and "gs_solve" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(gs.EXPORTS) | set(names)


def test_strerror_and_codes():
    lib = gs.load()
    assert lib.gs_strerror(gs.GS_OK) == b"success"
    assert lib.gs_strerror(gs.GS_ENOTCONV) == b"not converged"
    assert lib.gs_strerror(99) == b"unknown status"


@pytest.mark.parametrize("kw", [dict(p=0, J=6), dict(p=7, J=6), dict(p=4, J=2), dict(p=2, J=0)])
def test_plan_rejects_bad_sizes_without_gpu(kw):
    xi = np.linspace(-10, 10, 50)
    with pytest.raises(gs.GsError) as e:
        gs.gs_plan_1d(xi, kw["p"], kw["J"], stream=_NoStream())
    assert e.value.status == gs.GS_EINVAL


def test_plan_rejects_nonfinite_xi_and_weights():
    xi = np.linspace(-10, 10, 50)
    xi[3] = np.nan
    with pytest.raises(gs.GsError) as e:
        gs.gs_plan_1d(xi, 2, 5, stream=_NoStream())
    assert e.value.status == gs.GS_EINVAL
    xi = np.linspace(-10, 10, 50)
    w = np.ones(50)
    w[7] = -1
    with pytest.raises(gs.GsError) as e:
        gs.gs_plan_1d(xi, 2, 5, weights=w, stream=_NoStream())
    assert e.value.status == gs.GS_EINVAL
    with pytest.raises(gs.GsError) as e:
        gs.gs_plan_2d(np.zeros((10, 2)), 2, 5, stream=_NoStream(), sigma=3)
    assert e.value.status == gs.GS_EINVAL
    for chunk in (-2, (1 << 20) + 1):  # work-item size: -1 (autotune), 0 (default) or 1..2^20
        with pytest.raises(gs.GsError) as e:
            gs.gs_plan_2d(np.zeros((10, 2)), 2, 5, stream=_NoStream(), chunk=chunk)
        assert e.value.status == gs.GS_EINVAL


class _NoStream:
    cuda_stream = 0


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_host_constants_match_oracle(p):
    c = gs.gs_boundary_constants(p)
    k, h = daubechies_filter(p)
    assert np.max(np.abs(c["h"] - h)) < 1e-15
    if p == 1:
        return
    tol = 1e-12 if p <= 4 else 1e-10  # the edge construction loses digits as p grows
    for side in ["left", "right"]:
        e = EdgeSide(p, side)
        assert np.max(np.abs(c["U_" + side] - e.U)) < tol
        assert np.max(np.abs(c["V_" + side] - e.V)) < tol
        assert np.max(np.abs(c["v0_" + side] - e.v1_0)) < 10 * tol


def test_plan_rejects_empty_sample_sets():
    with pytest.raises(gs.GsError) as e:
        gs.gs_plan_1d(np.zeros(0), 2, 5, stream=_NoStream())
    assert e.value.status == gs.GS_EINVAL
    with pytest.raises(gs.GsError) as e:
        gs.gs_plan_2d(np.zeros((0, 2)), 2, 5, stream=_NoStream())
    assert e.value.status == gs.GS_EINVAL


def test_nfft_path_beyond_the_grid_limits_is_unsupported():
    """1D grids n = 2 * 2^J above 2^20 and 2D grids above 1024 have no NFFT path;
    asking for it explicitly is GS_EUNSUPPORTED (the automatic choice falls back to
    direct evaluation)."""
    xi = np.linspace(-10, 10, 50)
    with pytest.raises(gs.GsError) as e:
        gs.gs_plan_1d(xi, 2, 20, stream=_NoStream(), direct=0)
    assert e.value.status == gs.GS_EUNSUPPORTED
    with pytest.raises(gs.GsError) as e:
        gs.gs_plan_2d(np.zeros((10, 2)), 2, 10, stream=_NoStream(), direct=0)
    assert e.value.status == gs.GS_EUNSUPPORTED


def test_plan_lattice_option_validated_without_gpu():
    # lattice = 2 requires every sigma xi to be an integer (Sec. 3.2 uniform grids);
    # out-of-range values of the option are bad options
    xi = np.linspace(-10, 10, 50) + 0.1
    with pytest.raises(gs.GsError) as e:
        gs.gs_plan_1d(xi, 2, 5, direct=0, lattice=2, stream=_NoStream())
    assert e.value.status == gs.GS_EINVAL
    assert b"lattice" in gs.load().gs_last_error_detail()
    with pytest.raises(gs.GsError) as e:
        gs.gs_plan_1d(np.arange(-16, 16) / 2.0, 2, 5, direct=0, lattice=3, stream=_NoStream())
    assert e.value.status == gs.GS_EINVAL


def test_voronoi_2d_validates_without_gpu():
    # every coordinate must lie in [-K, K]; K > 0
    with pytest.raises(gs.GsError) as e:
        gs.gs_voronoi_2d(np.array([[0.0, 0.0], [3.0, 0.0]]), 2.0, stream=_NoStream())
    assert e.value.status == gs.GS_EINVAL
    with pytest.raises(gs.GsError) as e:
        gs.gs_voronoi_2d(np.array([[0.0, 0.0]]), 0.0, stream=_NoStream())
    assert e.value.status == gs.GS_EINVAL
