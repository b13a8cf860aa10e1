"""Python binding of libgs, the GB300 generalized-sampling library.

Argument marshalling only: every step of the method runs in libgs's CUDA
kernels (see include/gs.h).  The functions keep the C names; torch tensors
carry device memory and the current CUDA stream.  If the compiled library is
missing, importing the binding raises -- there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

from .build import LIB, build

GS_OK, GS_EINVAL, GS_ENOMEM, GS_ECUDA, GS_ENOTCONV, GS_EBREAKDOWN, GS_ETIMEOUT, GS_EUNSUPPORTED = range(8)
GS_FP64, GS_FP32 = 0, 1
GS_SOLVE_FP64, GS_SOLVE_MIXED = 0, 1


class GsOpts(ctypes.Structure):
    _fields_ = [("kb_m_hi", ctypes.c_int), ("kb_m_lo", ctypes.c_int), ("sigma", ctypes.c_int),
                ("direct", ctypes.c_int), ("chunk", ctypes.c_int), ("lattice", ctypes.c_int)]


class GsSolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxit", ctypes.c_int), ("mode", ctypes.c_int),
                ("x0_given", ctypes.c_int), ("max_outer", ctypes.c_int), ("inner_rtol", ctypes.c_double)]


class GsSolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("outer", ctypes.c_int), ("rel_normres", ctypes.c_double),
                ("rel_res", ctypes.c_double), ("status", ctypes.c_int)]


class GsError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status} ({detail})")
        self.status = status


_lib = None
EXPORTS = ["gs_plan_1d", "gs_plan_2d", "gs_plan_destroy", "gs_plan_sizes", "gs_apply_T", "gs_apply_TH",
           "gs_apply_TH_noalloc", "gs_solve_batch", "gs_cnn_create", "gs_cnn_destroy", "gs_cnn_forward",
           "gs_cnn_train_step", "gs_cnn_gradients", "gs_cnn_weights", "gs_cnn_set_weights", "gs_solve_learned", "gs_solve_batch_learned", "gs_cnn_pair",
           "gs_solve", "gs_boundary_constants", "gs_profile", "gs_profile_report", "gs_strerror",
           "gs_last_error_detail", "gs_voronoi_2d"]


def load(path: str = LIB):
    """Load libgs.so (building it first if it is absent).  Raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        build()
    lib = ctypes.CDLL(path)
    vp, i64, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
    lib.gs_plan_1d.argtypes = [ctypes.POINTER(vp), dp, i64, ctypes.c_int, ctypes.c_int, ctypes.c_double, dp,
                               ctypes.POINTER(GsOpts), vp]
    lib.gs_plan_2d.argtypes = [ctypes.POINTER(vp), dp, i64, ctypes.c_int, ctypes.c_int, dp,
                               ctypes.POINTER(GsOpts), vp]
    lib.gs_plan_destroy.argtypes = [vp]
    lib.gs_plan_destroy.restype = None
    lib.gs_plan_sizes.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(i64), ctypes.POINTER(i64),
                                  ctypes.POINTER(i64)]
    lib.gs_apply_T.argtypes = [vp, ctypes.c_int, vp, vp, vp]
    lib.gs_apply_TH.argtypes = [vp, ctypes.c_int, vp, vp, vp]
    lib.gs_apply_TH_noalloc.argtypes = [vp, ctypes.c_int, vp, vp, vp]
    lib.gs_solve.argtypes = [vp, vp, vp, ctypes.POINTER(GsSolveOpts), ctypes.POINTER(GsSolveInfo), vp]
    lib.gs_solve_batch.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                   ctypes.POINTER(GsSolveOpts), ctypes.POINTER(GsSolveInfo), vp]
    lib.gs_solve_batch.restype = ctypes.c_int
    lib.gs_boundary_constants.argtypes = [ctypes.c_int] + [dp] * 7
    lib.gs_boundary_constants.restype = ctypes.c_int
    lib.gs_profile.argtypes = [ctypes.c_int]
    lib.gs_profile.restype = ctypes.c_int
    lib.gs_profile_report.argtypes = [ctypes.c_char_p, ctypes.c_int64]
    lib.gs_profile_report.restype = ctypes.c_int
    fp = ctypes.POINTER(ctypes.c_float)
    lib.gs_cnn_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_uint64, vp]
    lib.gs_cnn_destroy.argtypes = [vp]
    lib.gs_cnn_destroy.restype = None
    lib.gs_cnn_forward.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, vp]
    lib.gs_cnn_train_step.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_float, dp, vp]
    lib.gs_cnn_gradients.argtypes = [vp, vp, vp, ctypes.c_int, fp, dp]
    lib.gs_cnn_weights.argtypes = [vp, fp, ctypes.POINTER(i64)]
    lib.gs_cnn_set_weights.argtypes = [vp, fp, i64]
    lib.gs_solve_learned.argtypes = [vp, vp, vp, vp, ctypes.POINTER(GsSolveOpts), ctypes.POINTER(GsSolveInfo),
                                     ctypes.POINTER(ctypes.c_int), vp]
    lib.gs_solve_batch_learned.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp, ctypes.POINTER(vp),
                                           ctypes.POINTER(vp), ctypes.POINTER(GsSolveOpts),
                                           ctypes.POINTER(GsSolveInfo), vp]
    lib.gs_cnn_pair.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.gs_voronoi_2d.argtypes = [dp, i64, ctypes.c_double, dp, dp, vp]
    lib.gs_voronoi_2d.restype = ctypes.c_int
    for f in ["gs_cnn_create", "gs_cnn_forward", "gs_cnn_train_step", "gs_cnn_gradients", "gs_cnn_weights",
              "gs_cnn_set_weights", "gs_solve_learned", "gs_solve_batch_learned", "gs_cnn_pair"]:
        getattr(lib, f).restype = ctypes.c_int
    lib.gs_strerror.argtypes = [ctypes.c_int]
    lib.gs_strerror.restype = ctypes.c_char_p
    lib.gs_last_error_detail.restype = ctypes.c_char_p
    for f in ["gs_plan_1d", "gs_plan_2d", "gs_plan_sizes", "gs_apply_T", "gs_apply_TH", "gs_apply_TH_noalloc",
              "gs_solve"]:
        getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != GS_OK:
        detail = load().gs_last_error_detail().decode()
        raise GsError(status, where, detail)


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _opts(kb_m_hi=8, kb_m_lo=4, sigma=2, direct=-1, chunk=0, lattice=0):
    return GsOpts(kb_m_hi, kb_m_lo, sigma, direct, chunk, lattice)


def gs_plan_1d(xi, p: int, J: int, bandwidth: float = 0.0, weights=None, stream=None, **opts):
    lib = load()
    xa, xp = _f64(xi)
    wa, wp = _f64(weights) if weights is not None else (None, None)
    h = ctypes.c_void_p()
    o = _opts(**opts)
    _check(lib.gs_plan_1d(ctypes.byref(h), xp, xa.size, p, J, float(bandwidth), wp, ctypes.byref(o),
                          _stream(stream)), "gs_plan_1d")
    return h


def gs_plan_2d(xi, p: int, J: int, weights=None, stream=None, **opts):
    lib = load()
    xa, xp = _f64(xi)
    if xa.ndim != 2 or xa.shape[1] != 2:
        raise ValueError("xi must be (M, 2)")
    wa, wp = _f64(weights) if weights is not None else (None, None)
    h = ctypes.c_void_p()
    o = _opts(**opts)
    _check(lib.gs_plan_2d(ctypes.byref(h), xp, xa.shape[0], p, J, wp, ctypes.byref(o), _stream(stream)),
           "gs_plan_2d")
    return h


def gs_boundary_constants(p: int) -> dict:
    """Host-side plan constants (filter taps, edge matrices U, V, v1(0)) as numpy arrays."""
    lib = load()
    q = max(p, 1)
    h = np.zeros(2 * p)
    arrs = {"U_left": np.zeros((q, q)), "V_left": np.zeros((q, 2 * q - 1)), "v0_left": np.zeros(q),
            "U_right": np.zeros((q, q)), "V_right": np.zeros((q, 2 * q - 1)), "v0_right": np.zeros(q)}
    ptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    _check(lib.gs_boundary_constants(p, ptr(h), ptr(arrs["U_left"]), ptr(arrs["V_left"]), ptr(arrs["v0_left"]),
                                     ptr(arrs["U_right"]), ptr(arrs["V_right"]), ptr(arrs["v0_right"])),
           "gs_boundary_constants")
    arrs["h"] = h
    return arrs


def gs_profile(on: bool):
    _check(load().gs_profile(int(bool(on))), "gs_profile")


def gs_profile_report() -> dict:
    """{kernel: (launches, total_ms)} of the launches recorded since gs_profile(1)."""
    import json
    buf = ctypes.create_string_buffer(1 << 16)
    _check(load().gs_profile_report(buf, len(buf)), "gs_profile_report")
    return {k: (v[0], v[1]) for k, v in json.loads(buf.value.decode()).items()}


def gs_plan_destroy(plan):
    if plan:
        load().gs_plan_destroy(plan)


def gs_plan_sizes(plan):
    d, M, N, nc = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(load().gs_plan_sizes(plan, ctypes.byref(d), ctypes.byref(M), ctypes.byref(N), ctypes.byref(nc)),
           "gs_plan_sizes")
    return d.value, M.value, N.value, nc.value


def _dev(t, dtype, n):
    import torch
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous() and t.numel() == n):
        raise ValueError(f"expected a contiguous CUDA tensor of {n} {dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _ctype(precision):
    import torch
    return torch.complex128 if precision == GS_FP64 else torch.complex64


def gs_apply_T(plan, precision: int, x, y, stream=None):
    _, M, _, nc = gs_plan_sizes(plan)
    dt = _ctype(precision)
    _check(load().gs_apply_T(plan, precision, _dev(x, dt, nc), _dev(y, dt, M), _stream(stream)), "gs_apply_T")
    return y


def gs_apply_TH(plan, precision: int, y, x, stream=None):
    _, M, _, nc = gs_plan_sizes(plan)
    dt = _ctype(precision)
    _check(load().gs_apply_TH(plan, precision, _dev(y, dt, M), _dev(x, dt, nc), _stream(stream)), "gs_apply_TH")
    return x


def gs_apply_TH_noalloc(plan, precision: int, y, x, stream=None):
    """x = T^H y through the entry point that allocates nothing (fixed static scratch)."""
    _, M, _, nc = gs_plan_sizes(plan)
    dt = _ctype(precision)
    _check(load().gs_apply_TH_noalloc(plan, precision, _dev(y, dt, M), _dev(x, dt, nc), _stream(stream)),
           "gs_apply_TH_noalloc")
    return x


def gs_solve(plan, y, x, tol=1e-6, maxit=1000, mode=GS_SOLVE_MIXED, x0_given=False, max_outer=8, inner_rtol=0.0,
             stream=None, raise_on_notconv=False):
    """Returns the info struct as a dict; raises on errors other than GS_ENOTCONV."""
    import torch
    _, M, _, nc = gs_plan_sizes(plan)
    o = GsSolveOpts(tol, maxit, mode, int(bool(x0_given)), max_outer, inner_rtol)
    info = GsSolveInfo()
    st = load().gs_solve(plan, _dev(y, torch.complex128, M), _dev(x, torch.complex128, nc), ctypes.byref(o),
                         ctypes.byref(info), _stream(stream))
    if st != GS_OK and (st != GS_ENOTCONV or raise_on_notconv):
        _check(st, "gs_solve")
    return {"iterations": info.iterations, "outer": info.outer, "rel_normres": info.rel_normres,
            "rel_res": info.rel_res, "status": info.status}


def gs_solve_batch(plans, ys, xs, tol=1e-6, maxit=1000, mode=GS_SOLVE_MIXED, max_outer=8, inner_rtol=0.0,
                   stream=None):
    """Solve B problems (plans[i], ys[i] -> xs[i], complex128 CUDA tensors); list of info dicts."""
    import torch
    B = len(plans)
    hs = (ctypes.c_void_p * B)(*[p.value if isinstance(p, ctypes.c_void_p) else p for p in plans])
    for p, y, x in zip(plans, ys, xs):
        _, M, _, nc = gs_plan_sizes(p)
        _dev(y, torch.complex128, M)
        _dev(x, torch.complex128, nc)
    yp = (ctypes.c_void_p * B)(*[y.data_ptr() for y in ys])
    xp = (ctypes.c_void_p * B)(*[x.data_ptr() for x in xs])
    o = GsSolveOpts(tol, maxit, mode, 0, max_outer, inner_rtol)
    infos = (GsSolveInfo * B)()
    st = load().gs_solve_batch(hs, B, yp, xp, ctypes.byref(o), infos, _stream(stream))
    if st not in (GS_OK, GS_ENOTCONV):
        _check(st, "gs_solve_batch")
    return [{"iterations": i.iterations, "outer": i.outer, "rel_normres": i.rel_normres, "rel_res": i.rel_res,
             "status": i.status} for i in infos]


class Plan:
    """Owning wrapper around a gs_plan handle (destroyed with the object)."""

    def __init__(self, handle):
        self.handle = handle
        self.dims, self.M, self.N, self.ncoef = gs_plan_sizes(handle)

    @classmethod
    def plan_1d(cls, xi, p, J, bandwidth=0.0, weights=None, **opts):
        return cls(gs_plan_1d(xi, p, J, bandwidth, weights, **opts))

    @classmethod
    def plan_2d(cls, xi, p, J, weights=None, **opts):
        return cls(gs_plan_2d(xi, p, J, weights, **opts))

    def T(self, x, precision=GS_FP64):
        import torch
        y = torch.empty(self.M, dtype=_ctype(precision), device=x.device)
        return gs_apply_T(self.handle, precision, x, y)

    def TH(self, y, precision=GS_FP64):
        import torch
        x = torch.empty(self.ncoef, dtype=_ctype(precision), device=y.device)
        return gs_apply_TH(self.handle, precision, y, x)

    def solve(self, y, x=None, **kw):
        import torch
        if x is None:
            x = torch.zeros(self.ncoef, dtype=torch.complex128, device=y.device)
        info = gs_solve(self.handle, y, x, **kw)
        return x, info

    def __del__(self):
        try:
            if self.handle:
                gs_plan_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


class Cnn:
    """Owning wrapper of a gs_cnn (residual CNN warm start); images are
    (B, 2, H, W) float32 CUDA tensors."""

    def __init__(self, H, W, channels=32, depth=6, max_batch=8, seed=1, stream=None):
        self.H, self.W, self.channels, self.depth, self.max_batch = H, W, channels, depth, max_batch
        h = ctypes.c_void_p()
        _check(load().gs_cnn_create(ctypes.byref(h), H, W, channels, depth, max_batch, seed, _stream(stream)),
               "gs_cnn_create")
        self.handle = h
        self.chans = [2] + [channels] * (depth - 1) + [2]

    def _img(self, t, B):
        import torch
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.numel() == B * 2 * self.H * self.W):
            raise ValueError("expected a contiguous float32 CUDA tensor of shape (B, 2, H, W)")
        return ctypes.c_void_p(t.data_ptr())

    def forward(self, u, bf16=True, stream=None):
        import torch
        B = u.shape[0]
        out = torch.empty_like(u)
        _check(load().gs_cnn_forward(self.handle, self._img(u, B), self._img(out, B), B, int(bool(bf16)),
                                     _stream(stream)), "gs_cnn_forward")
        return out

    def train_step(self, u, target, lr=1e-3, stream=None):
        B = u.shape[0]
        loss = ctypes.c_double()
        _check(load().gs_cnn_train_step(self.handle, self._img(u, B), self._img(target, B), B, lr, ctypes.byref(loss),
                                        _stream(stream)), "gs_cnn_train_step")
        return loss.value

    def gradients(self, u, target):
        B = u.shape[0]
        n = ctypes.c_int64()
        load().gs_cnn_weights(self.handle, None, ctypes.byref(n))
        g = np.zeros(n.value, dtype=np.float32)
        loss = ctypes.c_double()
        _check(load().gs_cnn_gradients(self.handle, self._img(u, B), self._img(target, B), B,
                                       g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(loss)),
               "gs_cnn_gradients")
        return loss.value, g

    def weights(self):
        n = ctypes.c_int64()
        load().gs_cnn_weights(self.handle, None, ctypes.byref(n))
        w = np.zeros(n.value, dtype=np.float32)
        _check(load().gs_cnn_weights(self.handle, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(n)),
               "gs_cnn_weights")
        return w

    def set_weights(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        _check(load().gs_cnn_set_weights(self.handle, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), w.size),
               "gs_cnn_set_weights")

    def unflatten(self, flat):
        """Split a flat weights-then-biases vector into [(W (co, ci, 3, 3), b (co,))]."""
        layers, off = [], 0
        shapes = list(zip(self.chans[:-1], self.chans[1:]))
        for ci, co in shapes:
            layers.append(flat[off:off + co * ci * 9].reshape(co, ci, 3, 3))
            off += co * ci * 9
        out = []
        for (ci, co), W in zip(shapes, layers):
            out.append((W, flat[off:off + co]))
            off += co
        return out

    def __del__(self):
        try:
            if self.handle:
                load().gs_cnn_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


def gs_solve_learned(plan, net, y, x, tol=1e-6, maxit=1000, mode=GS_SOLVE_MIXED, max_outer=8, inner_rtol=0.0,
                     stream=None):
    """Returns (info dict, used_warm_start)."""
    import torch
    _, M, _, nc = gs_plan_sizes(plan)
    o = GsSolveOpts(tol, maxit, mode, 0, max_outer, inner_rtol)
    info = GsSolveInfo()
    used = ctypes.c_int()
    st = load().gs_solve_learned(plan, net.handle, _dev(y, torch.complex128, M), _dev(x, torch.complex128, nc),
                                 ctypes.byref(o), ctypes.byref(info), ctypes.byref(used), _stream(stream))
    if st not in (GS_OK, GS_ENOTCONV):
        _check(st, "gs_solve_learned")
    return ({"iterations": info.iterations, "outer": info.outer, "rel_normres": info.rel_normres,
             "rel_res": info.rel_res, "status": info.status}, bool(used.value))


def gs_solve_batch_learned(plans, net, ys, xs, tol=1e-6, maxit=1000, mode=GS_SOLVE_MIXED, max_outer=8,
                           inner_rtol=0.0, stream=None):
    """gs_solve_batch from the learned start of each problem; list of info dicts."""
    import torch
    B = len(plans)
    hs = (ctypes.c_void_p * B)(*[p.value if isinstance(p, ctypes.c_void_p) else p for p in plans])
    for p, y, x in zip(plans, ys, xs):
        _, M, _, nc = gs_plan_sizes(p)
        _dev(y, torch.complex128, M)
        _dev(x, torch.complex128, nc)
    yp = (ctypes.c_void_p * B)(*[y.data_ptr() for y in ys])
    xp = (ctypes.c_void_p * B)(*[x.data_ptr() for x in xs])
    o = GsSolveOpts(tol, maxit, mode, 1, max_outer, inner_rtol)
    infos = (GsSolveInfo * B)()
    st = load().gs_solve_batch_learned(hs, B, net.handle, yp, xp, ctypes.byref(o), infos, _stream(stream))
    if st not in (GS_OK, GS_ENOTCONV):
        _check(st, "gs_solve_batch_learned")
    return [{"iterations": i.iterations, "outer": i.outer, "rel_normres": i.rel_normres, "rel_res": i.rel_res,
             "status": i.status} for i in infos]


def gs_voronoi_2d(xi, K: float, stream=None):
    """(mu, delta): 2D Voronoi cell areas of the samples within [-K, K]^2 and the density."""
    xa, xp = _f64(xi)
    M = xa.shape[0]
    mu = np.empty(M)
    delta = ctypes.c_double()
    _check(load().gs_voronoi_2d(xp, M, float(K), mu.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                ctypes.byref(delta), _stream(stream)), "gs_voronoi_2d")
    return mu, delta.value


def gs_cnn_pair(plan, y, x=None, stream=None):
    """(u_img, x_img) float32 (1, 2, N, N) images: T^H y / rms and x / the same rms."""
    import torch
    _, M, N, nc = gs_plan_sizes(plan)
    u = torch.empty((1, 2, N, N), dtype=torch.float32, device=y.device)
    xi = torch.empty_like(u) if x is not None else None
    _check(load().gs_cnn_pair(plan, _dev(y, torch.complex128, M),
                              _dev(x, torch.complex128, nc) if x is not None else None,
                              ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(xi.data_ptr()) if xi is not None else None,
                              _stream(stream)), "gs_cnn_pair")
    return u, xi
