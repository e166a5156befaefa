"""Parity of the four CUDA projectors with the FP64 oracle (through the C ABI)."""
import math

import numpy as np
import pytest

import gkb_inputs as gi
from oracle.projectors import Projectors
from tests.gpu_helpers import rel, small_fan, to_dev, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

gkb = None


@pytest.fixture(scope="module", autouse=True)
def _lib():
    global gkb
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_31153_b300 as m
    gkb = m


GEOMS = {
    "parallel64": lambda: gi.small_parallel_64().geom,
    "parallel_ragged": lambda: gi.Geometry("parallel", 77, 50, 0.8, np.linspace(0, math.pi, 37, endpoint=False),
                                           131, 0.7),
    "parallel_axes": lambda: gi.Geometry("parallel", 33, 33, 1.0,
                                         np.array([0, math.pi / 4, math.pi / 2, 3 * math.pi / 4, math.pi]), 47, 1.0),
    "fan96": lambda: small_fan(96, 120),
    "fan_ragged": lambda: gi.Geometry("fan", 70, 70, 1.1, np.linspace(0, 2 * math.pi, 53, endpoint=False), 111,
                                      1.7, 160.0, 250.0),
    # arc (equiangular) detector: a band-capable size and a ragged one
    "fanarc96": lambda: gi.fan_geometry(96, 120, 136, 192.0, 384.0, detector="arc"),
    "fanarc_ragged": lambda: gi.Geometry("fan_arc", 70, 70, 1.1, np.linspace(0, 2 * math.pi, 53, endpoint=False),
                                         111, 1.7, 160.0, 250.0),
}


def _ops(g, dt):
    G = gkb.Geometry(g)
    P = Projectors(g)
    rng = np.random.default_rng(7)
    x = np.abs(rng.standard_normal(g.n)) + gi.rasterize(gi.ellipse_params(min(g.nx, g.ny), 4, 3), g.nx, g.ny) \
        if g.nx == g.ny else np.abs(rng.standard_normal(g.n))
    y = np.abs(rng.standard_normal(g.m))
    return G, P, x, y


@pytest.mark.parametrize("name", list(GEOMS))
@pytest.mark.parametrize("dt,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_projectors_match_oracle(name, dt, tol):
    g = GEOMS[name]()
    tdt = torch.float64 if dt == "f64" else torch.float32
    G, P, x, y = _ops(g, dt)
    xd, yd = to_dev(x, tdt), to_dev(y, tdt)
    assert rel(to_np(G.A(xd)), P.A(x)) <= tol
    assert rel(to_np(G.B(yd)), P.B(y)) <= tol
    assert rel(to_np(G.AT(yd)), P.AT(y)) <= tol
    assert rel(to_np(G.BT(xd)), P.BT(x)) <= tol


@pytest.mark.parametrize("name", ["parallel64", "fan96"])
@pytest.mark.parametrize("dt", ["bf16", "f16"])
def test_reduced_precision_storage(name, dt):
    """BF16/FP16 storage with FP32 accumulation: within 5e-3 of the FP64 operator."""
    g = GEOMS[name]()
    tdt = torch.bfloat16 if dt == "bf16" else torch.float16
    G, P, x, y = _ops(g, dt)
    xd, yd = to_dev(x, tdt), to_dev(y, tdt)
    for got, ref in ((G.A(xd), P.A(x)), (G.B(yd), P.B(y)), (G.AT(yd), P.AT(y)), (G.BT(xd), P.BT(x))):
        assert rel(to_np(got), ref) <= 5e-3


@pytest.mark.parametrize("name", ["parallel_ragged", "fan_ragged"])
def test_exact_transposes_on_device(name):
    """<A x, y> = <x, A^T y> and <B y, x> = <y, B^T x> to FP64 round-off in FP64
    storage (the transposes use the forward kernels' own weights)."""
    g = GEOMS[name]()
    G = gkb.Geometry(g)
    rng = np.random.default_rng(3)
    x, y = to_dev(rng.standard_normal(g.n), torch.float64), to_dev(rng.standard_normal(g.m), torch.float64)
    lhs, rhs = float(G.A(x) @ y), float(x @ G.AT(y))
    assert abs(lhs - rhs) <= 1e-12 * float(torch.linalg.norm(G.A(x)) * torch.linalg.norm(y))
    lhs, rhs = float(G.B(y) @ x), float(y @ G.BT(x))
    assert abs(lhs - rhs) <= 1e-12 * float(torch.linalg.norm(G.B(y)) * torch.linalg.norm(x))


def test_full_size_fan512_sampled_entries():
    """The 512x512 fan-beam workload (720 angles, 725 bins) in FP32: sampled
    outputs of all four operators against the oracle's single-entry routines,
    and the adjoint identities over the full vectors."""
    w = gi.fan_512()
    g = w.geom
    G = gkb.Geometry(g)
    P = Projectors(g)
    rng = np.random.default_rng(11)
    x = gi.phantom_of(w)
    y = np.abs(rng.standard_normal(g.m))
    xd, yd = to_dev(x, torch.float32), to_dev(y, torch.float32)
    Ax, By, ATy, BTx = (to_np(v) for v in (G.A(xd), G.B(yd), G.AT(yd), G.BT(xd)))
    scale = {k: np.sqrt(np.mean(v * v)) for k, v in (("A", Ax), ("B", By), ("AT", ATy), ("BT", BTx))}
    for _ in range(24):
        a, d = int(rng.integers(g.n_angles)), int(rng.integers(g.n_det))
        i, j = int(rng.integers(g.ny)), int(rng.integers(g.nx))
        assert abs(Ax[a * g.n_det + d] - P.A_ray(x, a, d)) <= 1e-5 * max(abs(P.A_ray(x, a, d)), scale["A"])
        assert abs(BTx[a * g.n_det + d] - P.BT_ray(x, a, d)) <= 1e-5 * max(abs(P.BT_ray(x, a, d)), scale["BT"])
        assert abs(By[i * g.nx + j] - P.B_pixel(y, i, j)) <= 1e-5 * max(abs(P.B_pixel(y, i, j)), scale["B"])
    for _ in range(6):
        i, j = int(rng.integers(g.ny)), int(rng.integers(g.nx))
        ref = P.AT_pixel(y, i, j)
        assert abs(ATy[i * g.nx + j] - ref) <= 1e-5 * max(abs(ref), scale["AT"])
    xd64, yd64 = xd.double(), yd.double()
    lhs = float(torch.from_numpy(Ax).cuda() @ yd64)
    rhs = float(xd64 @ torch.from_numpy(ATy).cuda())
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs)
    lhs = float(torch.from_numpy(By).cuda() @ xd64)
    rhs = float(yd64 @ torch.from_numpy(BTx).cuda())
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs)


def _sampled_rel(got, ref):
    """Norm-relative error of a matrix-vector product estimated from sampled
    entries: sqrt(sum (g - o)^2 / sum o^2) over the samples."""
    got, ref = np.asarray(got, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    return float(np.sqrt(np.sum((got - ref) ** 2) / np.sum(ref * ref)))


@pytest.mark.parametrize("dt,tol", [("f32", 1e-5), ("bf16", 5e-3), ("f16", 5e-3)])
def test_full_size_parallel2048_sampled_entries(dt, tol):
    """The 2048x2048 precision-sweep workload (1800 angles over 180 degrees,
    2897 bins): 64 sampled outputs of each operator against the oracle's
    single-entry routines, the stated per-matvec criterion (1e-5 for FP32,
    5e-3 for 16-bit storage) applied to the sampled norm ratio.  Interpolation
    coordinates reach 1450 pixels here, where an FP32 ulp is 1.2e-4 pixel."""
    w = gi.parallel_2048()
    g = w.geom
    G = gkb.Geometry(g)
    P = Projectors(g)
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[dt]
    rng = np.random.default_rng(2048)
    x = gi.phantom_of(w)
    # the sinogram input of B and A^T: the device's projection of the phantom,
    # stored in the test's type; the oracle applies its operators to exactly
    # those stored values (the image input is compared from its FP64 values,
    # so 16-bit storage errors of x count against the criterion)
    if dt == "f16":
        # FP16's range ends at 65504: a back projection sums 1800 angles of
        # line integrals of up to ~1000, so the operands are scaled to keep
        # every output finite (the operators are linear)
        x = x / 2048.0
    xd = to_dev(x, tdt)
    y32 = G.A(to_dev(x, torch.float32))
    if dt == "f16":
        y32 = y32 / (g.n_angles * float(y32.abs().max()))
    yd = y32.to(tdt)
    yv = to_np(yd)
    Ax, By, ATy, BTx = (to_np(v) for v in (G.A(xd), G.B(yd), G.AT(yd), G.BT(xd)))
    S = 64
    rays = [(int(rng.integers(g.n_angles)), int(rng.integers(g.n_det // 4, 3 * g.n_det // 4))) for _ in range(S)]
    pix = [(int(rng.integers(g.ny // 8, 7 * g.ny // 8)), int(rng.integers(g.nx // 8, 7 * g.nx // 8))) for _ in range(S)]
    err = {
        "A": _sampled_rel([Ax[a * g.n_det + d] for a, d in rays], [P.A_ray(x, a, d) for a, d in rays]),
        "BT": _sampled_rel([BTx[a * g.n_det + d] for a, d in rays], [P.BT_ray(x, a, d) for a, d in rays]),
        "B": _sampled_rel([By[i * g.nx + j] for i, j in pix], [P.B_pixel(yv, i, j) for i, j in pix]),
        "AT": _sampled_rel([ATy[i * g.nx + j] for i, j in pix], [P.AT_pixel(yv, i, j) for i, j in pix]),
    }
    print(f"parallel2048 {dt} sampled relative errors: {err}")
    assert max(err.values()) <= tol, err


def test_degenerate_sizes():
    for g in (gi.Geometry("parallel", 1, 1, 1.0, np.array([0.3]), 1, 1.0),
              gi.Geometry("parallel", 3, 5, 1.0, np.array([1.0, 2.0]), 2, 2.5),
              gi.Geometry("fan", 2, 3, 1.0, np.array([0.1]), 3, 1.0, 10.0, 20.0)):
        G = gkb.Geometry(g)
        P = Projectors(g)
        rng = np.random.default_rng(1)
        x, y = rng.standard_normal(g.n), rng.standard_normal(g.m)
        xd, yd = to_dev(x, torch.float64), to_dev(y, torch.float64)
        for got, ref in ((G.A(xd), P.A(x)), (G.B(yd), P.B(y)), (G.AT(yd), P.AT(y)), (G.BT(xd), P.BT(x))):
            assert np.allclose(to_np(got), ref, rtol=1e-12, atol=1e-12)


def test_invalid_arguments_are_rejected():
    g = gi.parallel_geometry(16, 8, 23)
    G = gkb.Geometry(g)
    lib = gkb.load_library()
    x = torch.zeros(g.n + 1, device="cuda")
    y = torch.zeros(g.m + 1, device="cuda")
    import ctypes
    # misaligned device pointer
    st = lib.projector_forward(G.handle, ctypes.c_void_p(x.data_ptr() + 4), ctypes.c_void_p(y.data_ptr()),
                               gkb.F32, None)
    assert st == gkb.ERR_INVALID_ARG
    st = lib.projector_forward(G.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), 7, None)
    assert st == gkb.ERR_INVALID_ARG
    with pytest.raises(ValueError):
        G.A(torch.zeros(g.n + 1, device="cuda"))


@pytest.mark.parametrize("name", ["fan_ragged", "parallel_ragged", "fan96", "parallel64", "fanarc96"])
@pytest.mark.parametrize("dt", ["f32", "f16"])
def test_every_kernel_shape_gives_identical_outputs(name, dt):
    """The autotuner's shapes split work differently but keep each pixel's and
    each ray's summation order (the scatter A^T gives every pixel's rays to one
    half-warp in angle order whatever the chunk), so within a kernel family
    every shape returns the same bits."""
    g = GEOMS[name]()
    tdt = torch.float32 if dt == "f32" else torch.float16
    G, _, x, y = _ops(g, dt)
    xd, yd = to_dev(x, tdt), to_dev(y, tdt)
    for scatter in (True, False):
        G.use_scatter(scatter)
        _, counts = G.shapes()
        ref = None
        for c in range(max(counts)):
            G.set_shapes([min(c, n - 1) for n in counts])
            outs = [G.A(xd), G.B(yd), G.AT(yd), G.BT(xd)]
            torch.cuda.synchronize()
            if ref is None:
                ref = outs
            for a, b in zip(outs, ref):
                assert torch.equal(a, b)
    with pytest.raises(gkb.GKBError):
        G.set_shapes([counts[0], 0, 0, 0])
    G.autotune(gkb.F32 if dt == "f32" else gkb.F16)
    outs = [G.A(xd), G.B(yd), G.AT(yd), G.BT(xd)]
    for a, b in zip(outs, ref):
        assert torch.equal(a, b)


@pytest.mark.parametrize("name", list(GEOMS))
def test_gather_transposes_match_oracle(name):
    """The gather family of A^T and B^T (pixel-driven A^T, ray-driven B^T)
    against the oracle; the default scatter family is covered above."""
    g = GEOMS[name]()
    G, P, x, y = _ops(g, "f32")
    G.use_scatter(False)
    xd, yd = to_dev(x, torch.float32), to_dev(y, torch.float32)
    assert rel(to_np(G.AT(yd)), P.AT(y)) <= 1e-5
    assert rel(to_np(G.BT(xd)), P.BT(x)) <= 1e-5


@pytest.mark.parametrize("name", ["fan96", "parallel64", "fan_ragged"])
def test_scatter_bt_integer_sums(name):
    """B^T's integer scatter: an all-zero image gives exact zeros, a NaN
    propagates to every bin, values spanning six decades keep FP32-level
    accuracy (the scale follows each tile's largest value), a single pixel
    reproduces the oracle's column of B^T, and repeated calls are bitwise
    identical."""
    g = GEOMS[name]()
    G, P, _, _ = _ops(g, "f32")
    z = torch.zeros(g.n, device="cuda")
    assert torch.count_nonzero(G.BT(z)) == 0
    rng = np.random.default_rng(5)
    x = rng.standard_normal(g.n) * 10.0 ** rng.uniform(-3, 3, g.n)
    xd = to_dev(x, torch.float32)
    out = G.BT(xd)
    ref = P.BT(to_np(xd).astype(np.float64))
    assert rel(to_np(out), ref) <= 1e-5
    assert torch.equal(out, G.BT(xd))
    # one pixel: every bin holds a single term, rounded on the tile's grid of
    # 2^-30 times (pixels per bin bound x weight bound x tile max)
    e = np.zeros(g.n)
    e[(g.ny // 2) * g.nx + g.nx // 3] = 1.0
    assert rel(to_np(G.BT(to_dev(e, torch.float32))), P.BT(e)) <= 1e-5
    xn = xd.clone()
    xn[7] = float("nan")
    assert torch.isnan(G.BT(xn)).all()


STRESS_FANS = {
    # magnification 6, rays 8 per pixel at the centre: the A^T scatter needs
    # lane strides above its limit in some tiles and falls back to the gather
    "fan_mag6_dense": lambda: gi.fan_geometry(96, 90, 400, 75.0, 450.0, det_width=0.75),
    # magnification 3, rays half a pixel apart: strides 2-3
    "fan_mag3": lambda: gi.fan_geometry(96, 73, 200, 80.0, 240.0, det_width=1.5),
    # source 5 pixels outside the image corner: weights vary 200-fold over the image
    "fan_near_source": lambda: gi.fan_geometry(96, 61, 160, 72.0, 300.0),
    # magnification 3 with the source well outside: the fast kernels apply,
    # and the A^T scatter runs with lane strides 2-3
    "fan_mag3_far": lambda: gi.fan_geometry(96, 67, 240, 200.0, 600.0, det_width=2.0),
    "fanarc_mag6_dense": lambda: gi.fan_geometry(96, 90, 400, 75.0, 450.0, det_width=0.75, detector="arc"),
    "fanarc_near_source": lambda: gi.fan_geometry(96, 61, 160, 72.0, 300.0, detector="arc"),
}


@pytest.mark.parametrize("name", list(STRESS_FANS))
@pytest.mark.parametrize("scatter", [True, False])
def test_fan_weights_under_strong_magnification(name, scatter):
    """Fan geometries with strong magnification or the source close to the
    image, both transpose families, against the oracle and the adjoint
    identities.  FP64 pins the candidate windows (a ray missing from a
    window shows at 1e-5, rounding at 1e-15); in FP32 a bin coordinate of a
    few hundred carries an absolute error of about 1e-5 bins, which on
    detectors finer than the pixels moves the weights by up to 1e-4
    relative, so FP32 is held to 5e-5."""
    g = STRESS_FANS[name]()
    G, P, x, y = _ops(g, "f32")
    G.use_scatter(scatter)
    for dt, tol in ((torch.float64, 1e-12), (torch.float32, 5e-5)):
        xd, yd = to_dev(x, dt), to_dev(y, dt)
        xf, yf = to_np(xd).astype(np.float64), to_np(yd).astype(np.float64)
        Ax, By, ATy, BTx = (to_np(v) for v in (G.A(xd), G.B(yd), G.AT(yd), G.BT(xd)))
        assert rel(Ax, P.A(xf)) <= tol
        assert rel(By, P.B(yf)) <= tol
        assert rel(ATy, P.AT(yf)) <= tol
        assert rel(BTx, P.BT(xf)) <= tol
        assert abs(Ax @ yf - xf @ ATy) <= max(tol, 1e-6) * abs(Ax @ yf)
        assert abs(By @ xf - yf @ BTx) <= max(tol, 1e-6) * abs(By @ xf)


def test_scatter_and_gather_transposes_agree_to_rounding():
    """On the moderate magnification-3 fan (rays closer than one pixel near
    the source) the scatter family is a different summation from the gather
    family: the two agree to rounding, not bit for bit, and the scatter
    gives the same bits on every call (fixed-order sums, integer atomics)."""
    g = STRESS_FANS["fan_mag3_far"]()
    G, P, x, y = _ops(g, "f32")
    yd, xd = to_dev(y, torch.float32), to_dev(x, torch.float32)
    a, a2 = G.AT(yd), G.AT(yd)
    c, c2 = G.BT(xd), G.BT(xd)
    assert torch.equal(a, a2) and torch.equal(c, c2)
    G.use_scatter(False)
    b = G.AT(yd)
    assert not torch.equal(a, b)
    assert rel(to_np(a), to_np(b)) <= 1e-6
    assert rel(to_np(c), to_np(G.BT(xd))) <= 1e-5
