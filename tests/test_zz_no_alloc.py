"""gkb_solve_noalloc: the solve for callers that cannot allocate device memory
when they solve (their own pool owns the device, or allocation is forbidden
after start-up).  Its workspace is a fixed static array inside the library;
the result must equal gkb_solve's, call after call (the array keeps the last
call's contents, so every call has to clear what starts at zero).

This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import gkb_inputs as gi
from oracle.projectors import Projectors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_31153_b300 as gkb
    return gkb


def _call(gkb, fname, G, params, b, k_max, x=None):
    if x is None:
        x = torch.empty(G.n, dtype=b.dtype, device="cuda")
    bufs = [np.zeros(k_max + 1) for _ in range(3)]
    dp = ctypes.POINTER(ctypes.c_double)
    info = gkb.SolveInfo(0, 0, 0, *(v.ctypes.data_as(dp) for v in bufs))
    st = getattr(gkb.load_library(), fname)(G.handle, ctypes.byref(params), ctypes.c_void_p(b.data_ptr()),
                                             ctypes.c_void_p(x.data_ptr()), ctypes.byref(info),
                                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, x, info.k_stop, bufs


def _device_memory():
    """(free device bytes, bytes reserved by the device's default stream-ordered
    pool): what a cudaMalloc or a cudaMallocAsync anywhere in the process
    would change."""
    free, _ = torch.cuda.mem_get_info()
    rt = ctypes.CDLL("libcudart.so")
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), torch.cuda.current_device()) == 0
    reserved = ctypes.c_uint64()
    assert rt.cudaMemPoolGetAttribute(pool, 0x5, ctypes.byref(reserved)) == 0   # cudaMemPoolAttrReservedMemCurrent
    return free, reserved.value


@pytest.mark.parametrize("variant,storage", [("BA", "f32"), ("AB", "f32"), ("BA", "f64"), ("matched", "f32"),
                                             ("BA", "bf16"), ("AB", "f16")])
def test_noalloc_matches_gkb_solve_twice(lib, variant, storage):
    gkb = lib
    g = gi.fan_geometry(64, 91, 91, 128.0, 256.0)
    P = Projectors(g)
    x_true = gi.ellipse_phantom(64, 8, 3)
    b_np, en = gi.add_noise(P.A(x_true), gi.noise_direction(g.m, 4), 0.02)
    dt = torch.float64 if storage == "f64" else torch.float32
    code = {"f64": gkb.F64, "f32": gkb.F32, "bf16": gkb.BF16, "f16": gkb.F16}[storage]
    b = torch.tensor(b_np, dtype=dt, device="cuda")
    G = gkb.Geometry(g)
    params = gkb.make_params(variant=variant, k_max=40, stop="dp", noise_norm=en, storage=code, use_graph=True)
    st_ref, x_ref, k_ref, h_ref = _call(gkb, "gkb_solve", G, params, b, 40)   # also builds FP64 tables
    assert st_ref >= 0
    _call(gkb, "gkb_solve_noalloc", G, params, b, 40)   # the first call on a device looks the array up
    for _ in range(2):
        x = torch.empty(G.n, dtype=b.dtype, device="cuda")
        before = _device_memory()
        st, x, k, h = _call(gkb, "gkb_solve_noalloc", G, params, b, 40, x=x)
        assert _device_memory() == before          # nothing was allocated, not even stream-ordered
        assert st == st_ref and k == k_ref
        err = float(torch.linalg.norm((x - x_ref).double()) / torch.linalg.norm(x_ref.double()))
        assert err <= 1e-6, err
        assert np.allclose(h[0][:k], h_ref[0][:k], rtol=1e-10)
        assert np.allclose(h[2][:k], h_ref[2][:k], rtol=1e-10)


def test_noalloc_needs_the_geometry_device_current(lib):
    """The workspace array is looked up on the current device; a geometry of
    another device is refused (nothing runs).  With one device the check is
    exercised through a geometry whose recorded device differs: skipped."""
    if torch.cuda.device_count() < 2:
        pytest.skip("one device")
    gkb = lib
    g = gi.parallel_geometry(16, 8, 23)
    with torch.cuda.device(1):
        G = gkb.Geometry(g)
    params = gkb.make_params(variant="BA", k_max=5, storage=gkb.F32)
    b = torch.zeros(g.m, device="cuda:0")
    st, _, _, _ = _call(gkb, "gkb_solve_noalloc", G, params, b, 5)
    assert st == gkb.ERR_INVALID_ARG


def test_noalloc_rejects_oversized_workspace(lib):
    gkb = lib
    g = gi.fan_512().geom   # BA at k = 150: a 158 MB Krylov basis alone
    G = gkb.Geometry(g)
    params = gkb.make_params(variant="BA", k_max=150, storage=gkb.F32)
    b = torch.zeros(g.m, device="cuda")
    st, _, _, _ = _call(gkb, "gkb_solve_noalloc", G, params, b, 150)
    assert st == gkb.ERR_TOO_LARGE
    assert "fixed array" in gkb.status_string(st)
