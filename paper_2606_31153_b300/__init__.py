"""Python binding of the B300 AB-/BA-GKB library (``libgkb_b300.so``).

Argument marshalling only: every operator and every step of a solve runs in
the library's CUDA kernels.  PyTorch provides device memory and streams.  The
library must have been built (``python -m paper_2606_31153_b300.build``); if it
is missing or cannot be loaded, importing the binding raises -- there is no
fallback path.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgkb_b300.so")

# enums of include/gkb.h
PARALLEL, FAN_FLAT, FAN_ARC = 0, 1, 2
F32, F64, BF16, F16 = 0, 1, 2, 3
AB, BA, MATCHED, AB_GMRES, BA_GMRES = 0, 1, 2, 3, 4
STOP_NONE, STOP_DP, STOP_RNS, STOP_LEARNED, STOP_HYBRID = 0, 1, 2, 3, 4
REASONS = {0: "k_max", 1: "dp", 2: "rns", 3: "breakdown", 4: "error", 5: "learned", 6: "hybrid"}
OK, ERR_INVALID_ARG, ERR_CUDA, ERR_OOM, ERR_NONFINITE, ERR_TIMEOUT, ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
ERR_TOO_LARGE = -7
STATUS_BREAKDOWN, STATUS_NOT_CONVERGED = 1, 2

VARIANTS = {"AB": AB, "BA": BA, "matched": MATCHED, "AB-GMRES": AB_GMRES, "BA-GMRES": BA_GMRES}
STOPS = {"none": STOP_NONE, "dp": STOP_DP, "rns": STOP_RNS, "learned": STOP_LEARNED, "hybrid": STOP_HYBRID}


class GeometryDesc(ctypes.Structure):
    _fields_ = [("beam", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("pixel", ctypes.c_double),
                ("n_angles", ctypes.c_int), ("angles_rad", ctypes.POINTER(ctypes.c_double)),
                ("n_det", ctypes.c_int), ("det_width", ctypes.c_double), ("sod", ctypes.c_double),
                ("sdd", ctypes.c_double)]


class SolveParams(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("k_max", ctypes.c_int), ("stop", ctypes.c_int),
                ("noise_norm", ctypes.c_double), ("tau", ctypes.c_double), ("rns_eps", ctypes.c_double),
                ("reorth", ctypes.c_int), ("storage", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("operands", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("k_stop", ctypes.c_int), ("stop_reason", ctypes.c_int), ("status", ctypes.c_int),
                ("alpha", ctypes.POINTER(ctypes.c_double)), ("t", ctypes.POINTER(ctypes.c_double)),
                ("resid", ctypes.POINTER(ctypes.c_double)), ("lam", ctypes.POINTER(ctypes.c_double))]


class LearnedInfo(ctypes.Structure):
    _fields_ = [("k_hat", ctypes.c_int), ("lam", ctypes.c_double), ("k_dp", ctypes.c_int), ("hybrid", ctypes.c_int),
                ("fallback", ctypes.c_int), ("hybrid_resid", ctypes.c_double)]


class GKBError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_string(status)} ({status})")
        self.status = status


_lib = None


def load_library() -> ctypes.CDLL:
    """Load libgkb_b300.so; raises if it is absent (no CPU fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2606_31153_b300.build`")
    lib = ctypes.CDLL(LIB_PATH)
    vp, ip, st = ctypes.c_void_p, ctypes.c_int, ctypes.c_int
    sig = {
        "gkb_geometry_create": ([ctypes.POINTER(GeometryDesc), ctypes.POINTER(vp)], st),
        "gkb_geometry_destroy": ([vp], st),
        "gkb_geometry_sizes": ([vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)], st),
        "gkb_geometry_autotune": ([vp, ip], st),
        "gkb_geometry_get_shapes": ([vp, vp, vp], st),
        "gkb_geometry_set_shapes": ([vp, vp], st),
        "gkb_geometry_use_scatter": ([vp, ip], st),
        "projector_forward": ([vp, vp, vp, ip, vp], st),
        "projector_back": ([vp, vp, vp, ip, vp], st),
        "projector_forward_adjoint": ([vp, vp, vp, ip, vp], st),
        "projector_back_adjoint": ([vp, vp, vp, ip, vp], st),
        "gkb_solve": ([vp, ctypes.POINTER(SolveParams), vp, vp, ctypes.POINTER(SolveInfo), vp], st),
        "gkb_plan_create": ([vp, ctypes.POINTER(SolveParams), ctypes.POINTER(vp)], st),
        "gkb_plan_execute": ([vp, vp, vp, ctypes.POINTER(SolveInfo), vp], st),
        "gkb_plan_kernel_counts": ([vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)], st),
        "gkb_plan_profile": ([vp, vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong), vp], st),
        "gkb_plan_destroy": ([vp], st),
        "gkb_solve_batched": ([ip, ctypes.POINTER(vp), ctypes.POINTER(SolveParams), ctypes.POINTER(vp),
                               ctypes.POINTER(vp), ctypes.POINTER(SolveInfo), vp], st),
        "gkb_solve_noalloc": ([vp, ctypes.POINTER(SolveParams), vp, vp, ctypes.POINTER(SolveInfo), vp], st),
        "gkb_solve_iterates": ([vp, ctypes.POINTER(SolveParams), vp, vp, ctypes.POINTER(SolveInfo), vp], st),
        "gkb_batch_create": ([ip, ctypes.POINTER(vp), ctypes.POINTER(SolveParams), ctypes.POINTER(vp)], st),
        "gkb_batch_execute": ([vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(SolveInfo), vp], st),
        "gkb_batch_destroy": ([vp], st),
        "gkb_batch_execute_learned": ([vp, vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(SolveInfo),
                                       ctypes.POINTER(LearnedInfo), vp], st),
        "gkb_batch_training_data": ([vp, vp, vp, vp, vp], st),
        "gkb_mlp_create": ([ctypes.POINTER(vp)], st),
        "gkb_mlp_destroy": ([vp], st),
        "gkb_mlp_num_params": ([], ctypes.c_int),
        "gkb_mlp_set_params": ([vp, vp, vp], st),
        "gkb_mlp_get_params": ([vp, vp, vp], st),
        "gkb_mlp_forward": ([vp, vp, ip, vp, ip, vp], st),
        "gkb_mlp_gradient": ([vp, vp, vp, ip, vp, vp, vp], st),
        "gkb_mlp_train_step": ([vp, vp, vp, ip, ctypes.c_float, vp, vp], st),
        "gkb_status_string": ([st], ctypes.c_char_p),
        "gkb_version": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def status_string(s: int) -> str:
    return load_library().gkb_status_string(int(s)).decode()


def _check(s: int, what: str) -> int:
    if s < 0:
        raise GKBError(s, what)
    return s


def _stream_ptr(stream) -> ctypes.c_void_p:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def torch_dtype(dt: int):
    import torch
    return {F32: torch.float32, F64: torch.float64, BF16: torch.bfloat16, F16: torch.float16}[dt]


def dtype_code(tdtype) -> int:
    import torch
    return {torch.float32: F32, torch.float64: F64, torch.bfloat16: BF16, torch.float16: F16}[tdtype]


class Geometry:
    """Device-resident scan geometry (``gkb_geometry``).

    ``desc`` is anything with the fields of ``gkb_inputs.Geometry`` (beam,
    nx, ny, pixel, angles, n_det, det_width, sod, sdd).
    """

    def __init__(self, desc):
        lib = load_library()
        self._angles = np.ascontiguousarray(np.asarray(desc.angles, dtype=np.float64))
        beam = {"parallel": PARALLEL, "fan": FAN_FLAT, "fan_arc": FAN_ARC}.get(desc.beam, desc.beam)
        d = GeometryDesc(beam, int(desc.nx), int(desc.ny), float(desc.pixel), len(self._angles),
                         self._angles.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(desc.n_det),
                         float(desc.det_width), float(getattr(desc, "sod", 0.0)), float(getattr(desc, "sdd", 0.0)))
        h = ctypes.c_void_p()
        _check(lib.gkb_geometry_create(ctypes.byref(d), ctypes.byref(h)), "gkb_geometry_create")
        self._h = h
        self.nx, self.ny = int(desc.nx), int(desc.ny)
        self.n_angles, self.n_det = len(self._angles), int(desc.n_det)
        self.n = self.nx * self.ny
        self.m = self.n_angles * self.n_det
        self._lib = lib

    @property
    def handle(self):
        return self._h

    def autotune(self, dtype=F32):
        """Choose the fastest projector kernel shapes for this geometry (cached per shape)."""
        _check(self._lib.gkb_geometry_autotune(self._h, int(dtype)), "gkb_geometry_autotune")

    def shapes(self):
        """(shape indices, shape counts) of the kernels of A, B, A^T, B^T."""
        sh, ct = (ctypes.c_int * 4)(), (ctypes.c_int * 4)()
        _check(self._lib.gkb_geometry_get_shapes(self._h, sh, ct), "gkb_geometry_get_shapes")
        return list(sh), list(ct)

    def use_scatter(self, enable=True):
        """Transposes by the scatter kernels (True, the default) or by the gather kernels (False)."""
        _check(self._lib.gkb_geometry_use_scatter(self._h, 1 if enable else 0), "gkb_geometry_use_scatter")

    def set_shapes(self, shapes):
        """Pin the kernel shapes of A, B, A^T, B^T (indices below the counts of shapes())."""
        sh = (ctypes.c_int * 4)(*[int(v) for v in shapes])
        _check(self._lib.gkb_geometry_set_shapes(self._h, sh), "gkb_geometry_set_shapes")

    def close(self):
        if self._h:
            self._lib.gkb_geometry_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- the four operators -------------------------------------------------
    def _apply(self, fname, v, n_in, n_out, out=None, stream=None):
        import torch
        if not (v.is_cuda and v.is_contiguous() and v.numel() == n_in):
            raise ValueError(f"{fname}: need a contiguous CUDA tensor of {n_in} values")
        if out is None:
            out = torch.empty(n_out, dtype=v.dtype, device=v.device)
        elif not (out.is_cuda and out.is_contiguous() and out.numel() == n_out and out.dtype == v.dtype):
            raise ValueError(f"{fname}: bad output tensor")
        _check(getattr(self._lib, fname)(self._h, ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                         dtype_code(v.dtype), _stream_ptr(stream)), fname)
        return out

    def A(self, x, out=None, stream=None):
        """y = A x (Joseph forward projection)."""
        return self._apply("projector_forward", x, self.n, self.m, out, stream)

    def B(self, y, out=None, stream=None):
        """x = B y (pixel-driven back projection)."""
        return self._apply("projector_back", y, self.m, self.n, out, stream)

    def AT(self, y, out=None, stream=None):
        """x = A^T y."""
        return self._apply("projector_forward_adjoint", y, self.m, self.n, out, stream)

    def BT(self, x, out=None, stream=None):
        """y = B^T x."""
        return self._apply("projector_back_adjoint", x, self.n, self.m, out, stream)


@dataclass
class SolveResult:
    x: object
    k_stop: int
    reason: str
    status: int
    alpha: np.ndarray
    t: np.ndarray
    resid: np.ndarray
    lam: np.ndarray = None   # hybrid regularisation: lambda_1..lambda_k


def make_params(variant="BA", k_max=30, stop="none", noise_norm=0.0, tau=1.0, rns_eps=0.0, reorth=1,
                storage=F32, use_graph=True, operands=F32) -> SolveParams:
    """operands=BF16 or F16 with storage=F32: FP32 Krylov vectors, 16-bit projector operands."""
    v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    s = STOPS[stop] if isinstance(stop, str) else int(stop)
    return SolveParams(v, int(k_max), s, float(noise_norm), float(tau), float(rns_eps), int(reorth),
                       int(storage), 1 if use_graph else 0, int(operands))


def _result(x, info, k_max, st):
    k = info.k_stop
    return SolveResult(x, k, REASONS.get(info.stop_reason, "?"), st,
                       np.ctypeslib.as_array(info.alpha, (k_max + 1,))[:k].copy(),
                       np.ctypeslib.as_array(info.t, (k_max + 1,))[:k + 1].copy(),
                       np.ctypeslib.as_array(info.resid, (k_max + 1,))[:k].copy(),
                       np.ctypeslib.as_array(info.lam, (k_max + 1,))[:k].copy())


def _info(k_max):
    bufs = [np.zeros(k_max + 1) for _ in range(4)]
    dp = ctypes.POINTER(ctypes.c_double)
    info = SolveInfo(0, 0, 0, *(b.ctypes.data_as(dp) for b in bufs))
    return info, bufs


class Plan:
    """Reusable solve plan (``gkb_plan``): workspace and captured graph built once."""

    def __init__(self, geom: Geometry, **kw):
        self.geom = geom
        self.params = make_params(**kw)
        self._lib = load_library()
        h = ctypes.c_void_p()
        _check(self._lib.gkb_plan_create(geom.handle, ctypes.byref(self.params), ctypes.byref(h)),
               "gkb_plan_create")
        self._h = h

    def execute(self, b, x=None, stream=None) -> SolveResult:
        """b, x: CUDA or CPU tensors (FP64 for F64 storage, FP32 otherwise)."""
        import torch
        want = torch.float64 if self.params.storage == F64 else torch.float32
        if b.dtype != want or not b.is_contiguous() or b.numel() != self.geom.m:
            raise ValueError(f"b must be a contiguous {want} tensor of {self.geom.m} values")
        if x is None:
            x = torch.empty(self.geom.n, dtype=want, device=b.device)
        info, bufs = _info(self.params.k_max)
        st = _check(self._lib.gkb_plan_execute(self._h, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                               ctypes.byref(info), _stream_ptr(stream)), "gkb_plan_execute")
        return _result(x, info, self.params.k_max, st)

    def kernel_counts(self):
        """(kernels outside the iteration loop, kernels per iteration) of the captured graph."""
        o, b = ctypes.c_longlong(), ctypes.c_longlong()
        _check(self._lib.gkb_plan_kernel_counts(self._h, ctypes.byref(o), ctypes.byref(b)), "gkb_plan_kernel_counts")
        return int(o.value), int(b.value)

    PROFILE_CLASSES = ("A", "B", "AT", "BT", "reorth_dots", "reorth_update", "other")

    def profile(self, b, stream=None):
        """One solve with CUDA events between kernel groups (``gkb_plan_profile``):
        {class: (milliseconds, groups)} for A, B, AT, BT, reorth_dots,
        reorth_update and other."""
        ms = (ctypes.c_double * 7)()
        groups = (ctypes.c_longlong * 7)()
        _check(self._lib.gkb_plan_profile(self._h, ctypes.c_void_p(b.data_ptr()), ms, groups, _stream_ptr(stream)),
               "gkb_plan_profile")
        return {c: (float(ms[i]), int(groups[i])) for i, c in enumerate(self.PROFILE_CLASSES)}

    def close(self):
        if self._h:
            self._lib.gkb_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve(geom: Geometry, b, x=None, stream=None, **kw) -> SolveResult:
    """One-shot AB-/BA-/matched GKB solve (``gkb_solve``)."""
    import torch
    p = make_params(**kw)
    want = torch.float64 if p.storage == F64 else torch.float32
    if b.dtype != want or not b.is_contiguous() or b.numel() != geom.m:
        raise ValueError(f"b must be a contiguous {want} tensor of {geom.m} values")
    if x is None:
        x = torch.empty(geom.n, dtype=want, device=b.device)
    info, bufs = _info(p.k_max)
    st = _check(load_library().gkb_solve(geom.handle, ctypes.byref(p), ctypes.c_void_p(b.data_ptr()),
                                         ctypes.c_void_p(x.data_ptr()), ctypes.byref(info), _stream_ptr(stream)),
                "gkb_solve")
    return _result(x, info, p.k_max, st)


class Batch:
    """Reusable batched solve (``gkb_batch``): per-slice workspaces and one
    instantiated graph for the whole batch."""

    def __init__(self, geoms: Sequence[Geometry], params: Sequence[dict]):
        self.geoms = list(geoms)
        self.params = [make_params(**p) for p in params]
        n = len(self.geoms)
        self._lib = load_library()
        G = (ctypes.c_void_p * n)(*[g.handle.value for g in self.geoms])
        P = (SolveParams * n)(*self.params)
        h = ctypes.c_void_p()
        _check(self._lib.gkb_batch_create(n, G, P, ctypes.byref(h)), "gkb_batch_create")
        self._h = h

    def execute(self, bs, xs=None, stream=None):
        import torch
        n = len(self.geoms)
        if xs is None:
            xs = [torch.empty(g.n, dtype=torch.float64 if p.storage == F64 else torch.float32, device=b.device)
                  for g, p, b in zip(self.geoms, self.params, bs)]
        Bp = (ctypes.c_void_p * n)(*[b.data_ptr() for b in bs])
        Xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
        infos = (SolveInfo * n)()
        keep = []
        for i in range(n):
            info, bufs = _info(self.params[i].k_max)
            infos[i] = info
            keep.append(bufs)
        st = _check(self._lib.gkb_batch_execute(self._h, Bp, Xp, infos, _stream_ptr(stream)), "gkb_batch_execute")
        return st, [_result(xs[i], infos[i], self.params[i].k_max, infos[i].status) for i in range(n)]

    def execute_learned(self, mlp, bs, xs=None, stream=None):
        """Learned-stopping batch (all slices GKB_STOP_LEARNED): returns
        (status, results, learned infos)."""
        import torch
        n = len(self.geoms)
        if xs is None:
            xs = [torch.empty(g.n, dtype=torch.float32, device=b.device) for g, b in zip(self.geoms, bs)]
        Bp = (ctypes.c_void_p * n)(*[b.data_ptr() for b in bs])
        Xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
        infos = (SolveInfo * n)()
        linfo = (LearnedInfo * n)()
        keep = []
        for i in range(n):
            info, bufs = _info(self.params[i].k_max)
            infos[i] = info
            keep.append(bufs)
        st = _check(self._lib.gkb_batch_execute_learned(self._h, mlp.handle, Bp, Xp, infos, linfo, _stream_ptr(stream)),
                    "gkb_batch_execute_learned")
        res = [_result(xs[i], infos[i], self.params[i].k_max, infos[i].status) for i in range(n)]
        return st, res, [dict(k_hat=l.k_hat, lam=l.lam, k_dp=l.k_dp, hybrid=l.hybrid, fallback=l.fallback,
                              hybrid_resid=l.hybrid_resid) for l in linfo]

    def training_data(self, stream=None):
        """Features (n x 64), labels (n x 2) and validity of the last plain execution."""
        import torch
        n = len(self.geoms)
        dev = torch.device("cuda")
        X = torch.empty((n, 64), dtype=torch.float32, device=dev)
        T = torch.empty((n, 2), dtype=torch.float32, device=dev)
        V = torch.empty(n, dtype=torch.int32, device=dev)
        _check(self._lib.gkb_batch_training_data(self._h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(T.data_ptr()),
                                                 ctypes.c_void_p(V.data_ptr()), _stream_ptr(stream)),
               "gkb_batch_training_data")
        return X, T, V

    def close(self):
        if self._h:
            self._lib.gkb_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_iterates(geom: Geometry, b, stream=None, **kw):
    """Solve and return every iterate: (result, X) with X[k-1] = x_k (``gkb_solve_iterates``)."""
    import torch
    p = make_params(**kw)
    want = torch.float64 if p.storage == F64 else torch.float32
    if b.dtype != want or not b.is_contiguous() or b.numel() != geom.m:
        raise ValueError(f"b must be a contiguous {want} tensor of {geom.m} values")
    X = torch.zeros((p.k_max, geom.n), dtype=want, device=b.device)
    info, bufs = _info(p.k_max)
    st = _check(load_library().gkb_solve_iterates(geom.handle, ctypes.byref(p), ctypes.c_void_p(b.data_ptr()),
                                                  ctypes.c_void_p(X.data_ptr()), ctypes.byref(info), _stream_ptr(stream)),
                "gkb_solve_iterates")
    res = _result(X[max(info.k_stop - 1, 0)], info, p.k_max, st)
    return res, X


def solve_batched(geoms: Sequence[Geometry], bs, xs=None, params: Optional[Sequence[dict]] = None,
                  stream=None, **kw):
    """Solve independent slices in one call (``gkb_solve_batched``)."""
    import torch
    n = len(geoms)
    plist = [make_params(**(params[i] if params is not None else kw)) for i in range(n)]
    if xs is None:
        xs = [torch.empty(g.n, dtype=torch.float64 if p.storage == F64 else torch.float32, device=b.device)
              for g, p, b in zip(geoms, plist, bs)]
    G = (ctypes.c_void_p * n)(*[g.handle.value for g in geoms])
    P = (SolveParams * n)(*plist)
    Bp = (ctypes.c_void_p * n)(*[b.data_ptr() for b in bs])
    Xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
    infos = (SolveInfo * n)()
    keep = []
    for i in range(n):
        info, bufs = _info(plist[i].k_max)
        infos[i] = info
        keep.append(bufs)
    st = _check(load_library().gkb_solve_batched(n, G, P, Bp, Xp, infos, _stream_ptr(stream)), "gkb_solve_batched")
    return st, [_result(xs[i], infos[i], plist[i].k_max, infos[i].status) for i in range(n)]


class MLP:
    """The learned stopping predictor (``gkb_mlp``)."""

    def __init__(self):
        self._lib = load_library()
        h = ctypes.c_void_p()
        _check(self._lib.gkb_mlp_create(ctypes.byref(h)), "gkb_mlp_create")
        self._h = h
        self.n_params = int(self._lib.gkb_mlp_num_params())

    @property
    def handle(self):
        return self._h

    def set_params(self, theta=None, norm=None):
        """theta: flat FP32 parameters (host array or CUDA tensor); norm: 132 normalisation values."""
        def ptr(a):
            if a is None:
                return None
            if hasattr(a, "data_ptr"):
                return ctypes.c_void_p(a.contiguous().data_ptr())
            a = np.ascontiguousarray(a, dtype=np.float32)
            self._keep = a
            return a.ctypes.data_as(ctypes.c_void_p)
        t = None if theta is None else np.ascontiguousarray(theta, dtype=np.float32)
        nrm = None if norm is None else np.ascontiguousarray(norm, dtype=np.float32)
        _check(self._lib.gkb_mlp_set_params(self._h, None if t is None else t.ctypes.data_as(ctypes.c_void_p),
                                            None if nrm is None else nrm.ctypes.data_as(ctypes.c_void_p)),
               "gkb_mlp_set_params")

    def get_params(self):
        t = np.empty(self.n_params, dtype=np.float32)
        nrm = np.empty(132, dtype=np.float32)
        _check(self._lib.gkb_mlp_get_params(self._h, t.ctypes.data_as(ctypes.c_void_p), nrm.ctypes.data_as(ctypes.c_void_p)),
               "gkb_mlp_get_params")
        return t, nrm

    def forward(self, X, bf16=False, stream=None):
        import torch
        Y = torch.empty((X.shape[0], 2), dtype=torch.float32, device=X.device)
        _check(self._lib.gkb_mlp_forward(self._h, ctypes.c_void_p(X.data_ptr()), int(X.shape[0]),
                                         ctypes.c_void_p(Y.data_ptr()), 1 if bf16 else 0, _stream_ptr(stream)),
               "gkb_mlp_forward")
        return Y

    def gradient(self, X, T, stream=None):
        import torch
        g = torch.empty(self.n_params, dtype=torch.float32, device=X.device)
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        _check(self._lib.gkb_mlp_gradient(self._h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(T.data_ptr()),
                                          int(X.shape[0]), ctypes.c_void_p(g.data_ptr()),
                                          ctypes.c_void_p(loss.data_ptr()), _stream_ptr(stream)), "gkb_mlp_gradient")
        return g, loss

    def train_step(self, X, T, lr=1e-3, loss=None, stream=None):
        _check(self._lib.gkb_mlp_train_step(self._h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(T.data_ptr()),
                                            int(X.shape[0]), ctypes.c_float(lr),
                                            None if loss is None else ctypes.c_void_p(loss.data_ptr()),
                                            _stream_ptr(stream)), "gkb_mlp_train_step")

    def close(self):
        if self._h:
            self._lib.gkb_mlp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
