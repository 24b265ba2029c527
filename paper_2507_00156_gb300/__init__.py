"""Python binding of the GB300 extrapolated-regularization library (C ABI in include/ers.h).

Argument marshalling only: every step of the evaluation runs in the library's CUDA kernels.
PyTorch supplies device memory and streams.  Importing this package does not need a GPU, but
every call that touches the library raises if ``libers.so`` has not been built (there is no
CPU fallback).

    import paper_2507_00156_gb300 as ers
    s = ers.Surface(center=(0, 0, 0), axes=(1, 1, 1), h=1/64)
    s.set_density(f=f_nodes, q=q_nodes)            # (N,3) cuda float64, canonical node order
    x0, n0, b = s.closest_point(y)                   # (M,3) cuda float64 targets
    u, v = s.eval(y, f0, q0, rho=(2, 3, 4))          # f0, q0: densities at x0
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libers.so")

ERS_OK = 0
ERS_W_CUTOFF = 1
ERS_E_INVAL = -1
ERS_E_NOMEM = -2
ERS_E_CUDA = -3
ERS_E_TIMEOUT = -4
ERS_E_UNSUPPORTED = -5
ERS_E_STATE = -6
LAYER_SL = 1
LAYER_DL = 2
PREC_FP64 = 0
PREC_MIXED = 1
OPT_CONCURRENT = 1
OPT_SHARP = 2
OPT_FOUR_DELTA = 4
OPT_TREECODE = 8

# Every symbol the header declares (checked by the tests).
EXPORTS = ["ers_build_surface", "ers_surface_free", "ers_surface_info", "ers_set_density", "ers_closest_point",
           "ers_eval", "ers_eval_SL", "ers_eval_DL", "ers_eval_host", "ers_last_counts", "ers_profile",
           "ers_last_profile", "ers_set_density_multi", "ers_batch_create", "ers_batch_launch", "ers_batch_info",
           "ers_batch_free", "ers_closure_create", "ers_closure_free", "ers_closure_params", "ers_closure_infer",
           "ers_closure_infer_reference", "ers_closure_status", "ers_closure_range", "ers_closure_set_range_check",
           "ers_closure_last_out_of_range", "ers_closure_grad", "ers_closure_train",
           "ers_closure_data", "ers_eval_learned", "ers_closure_last_gate", "ers_eval_noalloc", "ers_treecode_defaults", "ers_tree_stats",
           "ers_node_interp", "ers_vec_axpby", "ers_gmres", "ers_last_error", "ers_version"]
ERS_W_NOT_CONVERGED = 2

# ers_matvec_fn: int (*)(void *ctx, const double *x, double *y, void *stream)
MATVEC_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
NPARAM = 15648
NFEAT = 5  # closure network inputs (the geometry): lambda_0, kappa_1 h, kappa_2 h, rho_0, rho_1
XSTR = 48  # floats per closure sample record: geometry (16 slots) then the density jets (32 slots)
JET_OFF = 16
NJETS = (18, 27)  # jets of the single and double layer
NOALLOC_MAX_M = 524288


class ErsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"ers error {code}: {msg}")
        self.code = code


class _Shape(ctypes.Structure):
    _fields_ = [("center", ctypes.c_double * 3), ("axes", ctypes.c_double * 3)]


class _Problem(ctypes.Structure):
    _fields_ = [("s", ctypes.c_void_p), ("M", ctypes.c_int64), ("y", ctypes.c_void_p), ("x0", ctypes.c_void_p),
                ("n0", ctypes.c_void_p), ("b", ctypes.c_void_p), ("f0", ctypes.c_void_p), ("q0", ctypes.c_void_p),
                ("u", ctypes.c_void_p), ("v", ctypes.c_void_p)]


class _Params(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_double * 3), ("cutoff_t", ctypes.c_double), ("precision", ctypes.c_int),
                ("layers", ctypes.c_int), ("options", ctypes.c_int), ("rho_sharp", ctypes.c_double),
                ("rho4", ctypes.c_double), ("tree_theta", ctypes.c_double), ("tree_n0", ctypes.c_int),
                ("tree_p", ctypes.c_int)]


_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    from . import buildlib
    return buildlib.build(force=force)


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"libers.so is not built ({LIB_PATH}); run paper_2507_00156_gb300.build() first")
            L = ctypes.CDLL(LIB_PATH)
            vp, i64, dbl, cint = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
            P = ctypes.POINTER
            L.ers_build_surface.argtypes = [P(_Shape), dbl, P(vp)]
            L.ers_surface_free.argtypes = [vp]
            L.ers_surface_info.argtypes = [vp, P(i64), P(dbl), P(vp), P(vp), P(vp)]
            L.ers_set_density.argtypes = [vp, vp, vp, vp]
            L.ers_closest_point.argtypes = [vp, vp, i64, vp, vp, vp, vp]
            L.ers_eval.argtypes = [vp, P(_Params), vp, i64, vp, vp, vp, vp, vp, vp, vp, vp]
            L.ers_eval_SL.argtypes = [vp, P(_Params), vp, i64, vp, vp, vp, vp, vp, vp]
            L.ers_eval_DL.argtypes = [vp, P(_Params), vp, i64, vp, vp, vp, vp, vp, vp]
            L.ers_eval_host.argtypes = [vp, P(_Params), vp, i64, vp, vp, vp, vp, vp, vp, vp, vp]
            L.ers_eval_noalloc.argtypes = [vp, P(_Params), vp, i64, vp, vp, vp, vp, vp, vp, vp, vp]
            L.ers_set_density_multi.argtypes = [vp, vp, vp, cint, vp]
            L.ers_batch_create.argtypes = [P(_Problem), cint, P(_Params), cint, P(vp)]
            L.ers_batch_launch.argtypes = [vp, vp]
            L.ers_batch_info.argtypes = [vp, P(cint), P(cint)]
            L.ers_batch_free.argtypes = [vp]
            fp = ctypes.POINTER(ctypes.c_float)
            L.ers_closure_create.argtypes = [ctypes.c_uint64, P(vp)]
            L.ers_closure_free.argtypes = [vp]
            L.ers_closure_params.argtypes = [vp, cint, vp, vp, i64]
            L.ers_closure_infer.argtypes = [vp, cint, vp, i64, vp, vp]
            L.ers_closure_infer_reference.argtypes = [vp, cint, vp, i64, vp, vp]
            L.ers_closure_status.argtypes = [vp, P(cint)]
            L.ers_closure_range.argtypes = [vp, cint, vp, vp, P(cint)]
            L.ers_closure_set_range_check.argtypes = [vp, cint]
            L.ers_closure_last_out_of_range.argtypes = [vp, P(i64)]
            L.ers_closure_grad.argtypes = [vp, cint, vp, vp, i64, vp, P(dbl), vp]
            L.ers_closure_train.argtypes = [vp, cint, vp, vp, i64, cint, cint, ctypes.c_float, P(dbl), vp]
            L.ers_closure_data.argtypes = [vp, P(_Params), vp, i64] + [vp] * 7 + [cint] + [vp] * 6
            L.ers_eval_learned.argtypes = [vp, vp, P(_Params), vp, i64] + [vp] * 5 + [cint, vp, vp, dbl, cint, P(dbl),
                                                                                         P(cint), vp]
            L.ers_closure_last_gate.argtypes = [vp, P(cint), P(dbl), P(dbl)]
            L.ers_last_counts.argtypes = [vp, P(i64), P(i64), P(i64)]
            L.ers_profile.argtypes = [vp, cint]
            L.ers_last_profile.argtypes = [vp, P(dbl), P(dbl), P(dbl)]
            L.ers_treecode_defaults.argtypes = [dbl, P(dbl), P(cint), P(cint)]
            L.ers_node_interp.argtypes = [vp, vp, vp, vp, i64, vp, vp]
            L.ers_vec_axpby.argtypes = [i64, dbl, vp, dbl, vp, vp]
            L.ers_gmres.argtypes = [i64, MATVEC_FN, vp, vp, vp, dbl, cint, P(cint), P(dbl), vp]
            L.ers_tree_stats.argtypes = [vp, P(i64), cint]
            L.ers_last_error.restype = ctypes.c_char_p
            L.ers_version.restype = ctypes.c_char_p
            for name in EXPORTS:
                if name not in ("ers_last_error", "ers_version"):
                    getattr(L, name).restype = cint
            _lib = L
    return _lib


def check(rc: int) -> int:
    if rc < 0:
        raise ErsError(rc, lib().ers_last_error().decode())
    return rc


def _ptr(t):
    if t is None:
        return None
    import torch
    if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a):
    if a is None:
        return None
    import numpy as np
    if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
        raise ValueError("expected a C-contiguous float64 array")
    return ctypes.c_void_p(a.ctypes.data)


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class _DevView:
    """Zero-copy view of library-owned device memory (CUDA array interface)."""

    def __init__(self, ptr: int, shape, owner):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f8", "data": (ptr, False),
                                         "version": 3, "strides": None}
        self.owner = owner


def params(rho=(2.0, 3.0, 4.0), cutoff_t=6.0, precision=PREC_FP64, layers=LAYER_SL | LAYER_DL,
           concurrent: bool = False, sharp: bool = False, rho_sharp: float = 0.0, tree=None) -> _Params:
    """ers_params; four entries in rho select ERS_OPT_FOUR_DELTA with rho4 = rho[3]; tree = None, or
    (theta, n0, p) for ERS_OPT_TREECODE (zeros select ers_treecode_defaults; True for all three)."""
    if len(rho) not in (3, 4):
        raise ValueError("rho needs 3 entries (or 4 for the O(delta^7) variant)")
    p = _Params()
    for k in range(3):
        p.rho[k] = float(rho[k])
    p.cutoff_t = float(cutoff_t)
    p.precision = int(precision)
    p.layers = int(layers)
    p.options = (OPT_CONCURRENT if concurrent else 0) | (OPT_SHARP if sharp else 0)
    p.rho_sharp = float(rho_sharp)
    if len(rho) == 4:
        p.options |= OPT_FOUR_DELTA
        p.rho4 = float(rho[3])
    if tree is not None and tree is not False:
        theta, n0, deg = (0.0, 0, 0) if tree is True else tree
        p.options |= OPT_TREECODE
        p.tree_theta, p.tree_n0, p.tree_p = float(theta), int(n0), int(deg)
    return p


def treecode_defaults(h: float):
    """(theta, N0, p) of Eq. (optimal_params) for spacing h (ers_treecode_defaults)."""
    t, n, q = ctypes.c_double(), ctypes.c_int(), ctypes.c_int()
    check(lib().ers_treecode_defaults(float(h), ctypes.byref(t), ctypes.byref(n), ctypes.byref(q)))
    return t.value, n.value, q.value


class Surface:
    """A quadrature surface on the current CUDA device (ers_build_surface)."""

    def __init__(self, center, axes, h: float):
        L = lib()
        shp = _Shape()
        for i in range(3):
            shp.center[i] = float(center[i])
            shp.axes[i] = float(axes[i])
        handle = ctypes.c_void_p()
        check(L.ers_build_surface(ctypes.byref(shp), float(h), ctypes.byref(handle)))
        self._h = handle
        self.center, self.axes = tuple(map(float, center)), tuple(map(float, axes))
        N, hh = ctypes.c_int64(), ctypes.c_double()
        xp, npp, wp = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        check(L.ers_surface_info(handle, ctypes.byref(N), ctypes.byref(hh), ctypes.byref(xp), ctypes.byref(npp),
                                 ctypes.byref(wp)))
        self.N, self.h = int(N.value), float(hh.value)
        self._xp, self._np, self._wp = xp.value, npp.value, wp.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.ers_surface_free(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def nodes(self):
        """(x, n, w) as zero-copy CUDA tensors in canonical order."""
        import torch
        x = torch.as_tensor(_DevView(self._xp, (self.N, 3), self), device="cuda")
        n = torch.as_tensor(_DevView(self._np, (self.N, 3), self), device="cuda")
        w = torch.as_tensor(_DevView(self._wp, (self.N,), self), device="cuda")
        return x, n, w

    def set_density(self, f=None, q=None, stream=None):
        check(lib().ers_set_density(self._h, _ptr(f), _ptr(q), _stream(stream)))

    def closest_point(self, y, stream=None):
        import torch
        M = y.shape[0]
        x0 = torch.empty((M, 3), dtype=torch.float64, device=y.device)
        n0 = torch.empty((M, 3), dtype=torch.float64, device=y.device)
        b = torch.empty((M,), dtype=torch.float64, device=y.device)
        check(lib().ers_closest_point(self._h, _ptr(y), M, _ptr(x0), _ptr(n0), _ptr(b), _stream(stream)))
        return x0, n0, b

    def eval(self, y, f0=None, q0=None, rho=(2.0, 3.0, 4.0), cutoff_t=6.0, precision=PREC_FP64,
             layers=LAYER_SL | LAYER_DL, x0=None, n0=None, b=None, u=None, v=None, stream=None,
             concurrent: bool = False, sharp: bool = False, rho_sharp: float = 0.0, tree=None):
        """ers_eval: returns (u, v) (None for a layer not selected).  concurrent=True sets
        ERS_OPT_CONCURRENT; sharp=True sets ERS_OPT_SHARP with delta# = rho_sharp h (0: rho[1]);
        four entries in rho set ERS_OPT_FOUR_DELTA (the O(delta^7) variant); tree = (theta, n0, p) or
        True sets ERS_OPT_TREECODE (far sums by the treecode of Sec. 3.4)."""
        import torch
        M = y.shape[0]
        sl, dl = bool(layers & LAYER_SL), bool(layers & LAYER_DL)
        if sl and u is None:
            u = torch.empty((M, 3), dtype=torch.float64, device=y.device)
        if dl and v is None:
            v = torch.empty((M, 3), dtype=torch.float64, device=y.device)
        p = params(rho, cutoff_t, precision, layers, concurrent, sharp, rho_sharp, tree)
        self._last_nd = len(rho)
        self.last_rc = check(lib().ers_eval(self._h, ctypes.byref(p), _ptr(y), M, _ptr(x0), _ptr(n0), _ptr(b),
                                            _ptr(f0) if sl else None, _ptr(q0) if dl else None,
                                            _ptr(u) if sl else None, _ptr(v) if dl else None, _stream(stream)))
        return (u if sl else None), (v if dl else None)

    def set_density_multi(self, f=None, q=None, stream=None):
        """Densities of several right-hand sides, (nrhs, N, 3) each (ers_set_density_multi)."""
        nrhs = (f if f is not None else q).shape[0]
        check(lib().ers_set_density_multi(self._h, _ptr(f), _ptr(q), nrhs, _stream(stream)))
        self.nrhs_multi = nrhs

    def eval_noalloc(self, y, x0, n0, b, f0=None, q0=None, u=None, v=None, rho=(2.0, 3.0, 4.0), cutoff_t=6.0,
                     precision=PREC_FP64, layers=LAYER_SL | LAYER_DL, stream=None, sharp: bool = False):
        """ers_eval_noalloc: the library allocates nothing; the caller passes every array, including
        the closest-point data (from closest_point) and the outputs u, v."""
        sl, dl = bool(layers & LAYER_SL), bool(layers & LAYER_DL)
        p = params(rho, cutoff_t, precision, layers, sharp=sharp)
        self.last_rc = check(lib().ers_eval_noalloc(self._h, ctypes.byref(p), _ptr(y), y.shape[0], _ptr(x0), _ptr(n0),
                                                    _ptr(b), _ptr(f0) if sl else None, _ptr(q0) if dl else None,
                                                    _ptr(u) if sl else None, _ptr(v) if dl else None,
                                                    _stream(stream)))
        return (u if sl else None), (v if dl else None)

    def eval_host(self, y, f0, q0, rho=(2.0, 3.0, 4.0), cutoff_t=6.0, precision=PREC_FP64,
                  layers=LAYER_SL | LAYER_DL, u=None, v=None, stream=None):
        """ers_eval_host with numpy (ideally pinned) host arrays."""
        import numpy as np
        M = y.shape[0]
        sl, dl = bool(layers & LAYER_SL), bool(layers & LAYER_DL)
        if sl and u is None:
            u = np.empty((M, 3))
        if dl and v is None:
            v = np.empty((M, 3))
        p = params(rho, cutoff_t, precision, layers)
        self._last_nd = len(rho)
        check(lib().ers_eval_host(self._h, ctypes.byref(p), _hptr(y), M, None, None, None,
                                  _hptr(f0) if sl else None, _hptr(q0) if dl else None,
                                  _hptr(u) if sl else None, _hptr(v) if dl else None, _stream(stream)))
        return (u if sl else None), (v if dl else None)

    def profile(self, enable: bool = True):
        check(lib().ers_profile(self._h, 1 if enable else 0))

    def last_profile(self):
        """(ms_closest, ms_far, ms_near) of the most recent profiled eval."""
        a, b_, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        check(lib().ers_last_profile(self._h, ctypes.byref(a), ctypes.byref(b_), ctypes.byref(c)))
        return a.value, b_.value, c.value

    def last_counts(self):
        """(near targets, near pairs, far pairs) of the most recent eval."""
        a, b_, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        check(lib().ers_last_counts(self._h, ctypes.byref(a), ctypes.byref(b_), ctypes.byref(c)))
        return int(a.value), int(b_.value), int(c.value)

    def last_class_counts(self):
        """Near pairs of the most recent eval by the number of deltas with r > cutoff_t delta_k
        (0, 1, 2; and 3 after a four-delta eval): the method's count of regularized terms."""
        c = self._class_counts()
        return c[:3] + ([c[8]] if getattr(self, "_last_nd", 3) == 4 else [])

    def last_defect_class_counts(self):
        """Near pairs of the most recent eval by the number of deltas whose defects 1 - s_p are
        evaluated directly instead of from the table (0..3; and 4 after a four-delta eval)."""
        c = self._class_counts()
        return c[3:7] + ([c[9]] if getattr(self, "_last_nd", 3) == 4 else [])

    def last_sharp_pairs(self):
        """Near pairs of on-surface targets evaluated with the s#_p (ERS_OPT_SHARP) in the most
        recent eval."""
        return self._class_counts()[7]

    def tree_stats(self):
        """dict: clusters, leaves, depth of the surface's tree; approximated (target, cluster) pairs
        and far pairs summed directly by the last treecode eval (ers_tree_stats)."""
        out = (ctypes.c_int64 * 5)()
        check(lib().ers_tree_stats(self._h, out, 5))
        return dict(clusters=out[0], leaves=out[1], depth=out[2], approximated=out[3], direct=out[4])

    def _class_counts(self):
        self.last_counts()
        c = (ctypes.c_int64 * 10)()
        L = lib()
        L.ers_debug_class_counts.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.c_int]
        check(L.ers_debug_class_counts(self._h, c, 10))
        return [int(z) for z in c]


class Batch:
    """A batched evaluation plan (ers_batch_create): one persistent launch, replayed as a CUDA graph.

    problems: list of dicts with keys s (Surface), y, x0, n0, b (M,3)/(M,) and f0, q0, u, v
    (nrhs, M, 3), all contiguous float64 CUDA tensors kept alive by the plan."""

    def __init__(self, problems, nrhs, rho=(2.0, 3.0, 4.0), cutoff_t=6.0, layers=LAYER_SL | LAYER_DL):
        L = lib()
        arr = (_Problem * len(problems))()
        self._keep = problems
        for i, pr in enumerate(problems):
            a = arr[i]
            a.s = pr["s"].handle
            a.M = int(pr["y"].shape[0])
            for k in ("y", "x0", "n0", "b", "f0", "q0", "u", "v"):
                setattr(a, k, _ptr(pr.get(k)))
        p = params(rho, cutoff_t, PREC_MIXED, layers)
        h = ctypes.c_void_p()
        self.rc = check(L.ers_batch_create(arr, len(problems), ctypes.byref(p), int(nrhs), ctypes.byref(h)))
        self._h = h

    def launch(self, stream=None):
        check(lib().ers_batch_launch(self._h, _stream(stream)))

    def info(self):
        a, b = ctypes.c_int(), ctypes.c_int()
        check(lib().ers_batch_info(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.ers_batch_free(h)
            self._h = None


def _fptr(t):
    if t is None:
        return None
    import torch
    if not t.is_cuda or t.dtype not in (torch.float32, torch.int32) or not t.is_contiguous():
        raise ValueError("expected a contiguous float32/int32 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


class Closure:
    """The learned near-field closure (ers_closure_*): two networks (0 = single, 1 = double layer)."""

    def __init__(self, seed: int = 0):
        h = ctypes.c_void_p()
        check(lib().ers_closure_create(ctypes.c_uint64(seed), ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.ers_closure_free(h)
            self._h = None

    def params(self, layer: int):
        import numpy as np
        out = np.empty(NPARAM, dtype=np.float32)
        check(lib().ers_closure_params(self._h, layer, ctypes.c_void_p(out.ctypes.data), None, NPARAM))
        return out

    def set_params(self, layer: int, values):
        import numpy as np
        a = np.ascontiguousarray(values, dtype=np.float32)
        check(lib().ers_closure_params(self._h, layer, None, ctypes.c_void_p(a.ctypes.data), NPARAM))

    def infer(self, layer: int, X, reference: bool = False, stream=None):
        import torch
        if X.dim() != 2 or X.shape[1] != XSTR:
            raise ValueError(f"closure sample records must be (n, {XSTR})")
        Y = torch.zeros((X.shape[0], 4), dtype=torch.float32, device=X.device)
        fn = lib().ers_closure_infer_reference if reference else lib().ers_closure_infer
        check(fn(self._h, layer, _fptr(X), X.shape[0], _fptr(Y), _stream(stream)))
        return Y

    def timed_out(self) -> bool:
        v = ctypes.c_int()
        check(lib().ers_closure_status(self._h, ctypes.byref(v)))
        return bool(v.value)

    def feature_range(self, layer: int):
        """(lo, hi) float32 arrays of the training extent of the 5 geometry inputs, or None while unknown."""
        import numpy as np
        out = np.empty(2 * NFEAT, dtype=np.float32)
        have = ctypes.c_int()
        check(lib().ers_closure_range(self._h, layer, ctypes.c_void_p(out.ctypes.data), None, ctypes.byref(have)))
        return (out[:NFEAT], out[NFEAT:]) if have.value else None

    def set_feature_range(self, layer: int, lo, hi):
        import numpy as np
        a = np.ascontiguousarray(np.concatenate([np.asarray(lo, np.float32), np.asarray(hi, np.float32)]))
        if a.shape != (2 * NFEAT,):
            raise ValueError(f"lo and hi need {NFEAT} entries each")
        check(lib().ers_closure_range(self._h, layer, None, ctypes.c_void_p(a.ctypes.data), None))

    def set_range_check(self, enabled: bool):
        check(lib().ers_closure_set_range_check(self._h, 1 if enabled else 0))

    def last_out_of_range(self) -> int:
        n = ctypes.c_int64()
        check(lib().ers_closure_last_out_of_range(self._h, ctypes.byref(n)))
        return n.value

    def grad(self, layer: int, X, T, stream=None):
        import torch
        G = torch.empty(NPARAM, dtype=torch.float32, device=X.device)
        loss = ctypes.c_double()
        check(lib().ers_closure_grad(self._h, layer, _fptr(X), _fptr(T), X.shape[0], _fptr(G), ctypes.byref(loss),
                                     _stream(stream)))
        return G, loss.value

    def last_gate(self):
        """(used (SL, DL), error with the network (SL, DL), error without it (SL, DL)) of the last
        eval_learned validation."""
        used = (ctypes.c_int * 2)()
        ew, eo = (ctypes.c_double * 2)(), (ctypes.c_double * 2)()
        check(lib().ers_closure_last_gate(self._h, used, ew, eo))
        return (bool(used[0]), bool(used[1])), (ew[0], ew[1]), (eo[0], eo[1])

    def train(self, layer: int, X, T, steps: int, batch: int = 4096, lr: float = 2e-3, stream=None) -> float:
        loss = ctypes.c_double()
        check(lib().ers_closure_train(self._h, layer, _fptr(X), _fptr(T), X.shape[0], int(steps), int(batch),
                                      ctypes.c_float(lr), ctypes.byref(loss), _stream(stream)))
        return loss.value


def closure_data(surface, y, x0, n0, b, f0, q0, u3, v3, rho=(2.0, 3.0, 4.0), cutoff_t=6.0,
                 precision=PREC_MIXED, ndelta=1, stream=None):
    """ers_closure_data: (Xs, Xd, Ts, Td, valid) CUDA tensors for training the two networks:
    sample records (M, 48) and targets (M, 4) = (c in the frame, weight)."""
    import torch
    M = y.shape[0]
    dev = y.device
    Xs = torch.empty((M, XSTR), dtype=torch.float32, device=dev)
    Xd = torch.empty_like(Xs)
    Ts = torch.empty((M, 4), dtype=torch.float32, device=dev)
    Td = torch.empty_like(Ts)
    valid = torch.empty((M,), dtype=torch.int32, device=dev)
    p = params(rho, cutoff_t, precision)
    check(lib().ers_closure_data(surface.handle, ctypes.byref(p), _ptr(y), M, _ptr(x0), _ptr(n0), _ptr(b), _ptr(f0),
                                 _ptr(q0), _ptr(u3), _ptr(v3), int(ndelta), _fptr(Xs), _fptr(Xd), _fptr(Ts),
                                 _fptr(Td), _fptr(valid), _stream(stream)))
    return Xs, Xd, Ts, Td, valid


def eval_learned(surface, closure, y, x0, n0, b, f0, q0, rho=(2.0, 3.0, 4.0), cutoff_t=6.0,
                 precision=PREC_MIXED, tol=1e-5, vstride=32, ndelta=1, u=None, v=None, stream=None):
    """ers_eval_learned: returns (u, v, validation errors (SL, DL), fell_back)."""
    import torch
    M = y.shape[0]
    if u is None:
        u = torch.empty((M, 3), dtype=torch.float64, device=y.device)
    if v is None:
        v = torch.empty((M, 3), dtype=torch.float64, device=y.device)
    p = params(rho, cutoff_t, precision)
    ve = (ctypes.c_double * 2)()
    fb = ctypes.c_int()
    check(lib().ers_eval_learned(surface.handle, closure.handle, ctypes.byref(p), _ptr(y), M, _ptr(x0), _ptr(n0),
                                 _ptr(b), _ptr(f0), _ptr(q0), int(ndelta), _ptr(u), _ptr(v), float(tol),
                                 int(vstride), ve, ctypes.byref(fb), _stream(stream)))
    return u, v, (ve[0], ve[1]), bool(fb.value)


def version() -> str:
    return lib().ers_version().decode()


def node_interp(surface, vals, x0, n0, out=None, stream=None):
    """ers_node_interp: values at surface points x0 (normals n0) of node values vals (N,3)."""
    import torch
    M = x0.shape[0]
    if out is None:
        out = torch.empty((M, 3), dtype=torch.float64, device=x0.device)
    check(lib().ers_node_interp(surface.handle, _ptr(vals), _ptr(x0), _ptr(n0), M, _ptr(out), _stream(stream)))
    return out


def vec_axpby(a, x, b, y, stream=None):
    """y = a x + b y (ers_vec_axpby), device float64 vectors of equal size."""
    check(lib().ers_vec_axpby(y.numel(), float(a), _ptr(x), float(b), _ptr(y), _stream(stream)))
    return y


def gmres(matvec, b, x=None, tol=1e-10, maxit=100, stream=None):
    """ers_gmres with a Python operator matvec(v, w) writing A v into w (device float64 vectors of
    length n).  Returns (x, iterations, relative residual, converged)."""
    import torch
    n = b.numel()
    if x is None:
        x = torch.empty_like(b)
    err = []

    def cb(ctx, xp, yp, sp):
        try:
            v = torch.as_tensor(_DevView(xp, (n,), None), device="cuda")
            w = torch.as_tensor(_DevView(yp, (n,), None), device="cuda")
            matvec(v, w)
            return 0
        except Exception as e:  # reported after the solve
            err.append(e)
            return ERS_E_STATE

    fn = MATVEC_FN(cb)
    it, rel = ctypes.c_int(), ctypes.c_double()
    rc = lib().ers_gmres(n, fn, None, _ptr(b), _ptr(x), float(tol), int(maxit), ctypes.byref(it), ctypes.byref(rel),
                         _stream(stream))
    if err:
        raise err[0]
    rc = check(rc)
    return x, it.value, rel.value, rc == ERS_OK
