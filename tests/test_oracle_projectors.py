"""Pins of the FP64 projector oracle against what geometry and algebra fix.

Each check would fail for a plausible slip in ``oracle/projectors.c``: a wrong
sign of the detector axis, a swapped row/column index, a dropped 1/c path
factor, an off-by-one in the bin or pixel centre offsets, or a transpose that
does not mirror its forward loop.
"""
import math

import numpy as np
import pytest

import gkb_inputs as gi
from oracle import dense
from oracle.projectors import Projectors


def matrix_of(apply, n_in):
    return np.column_stack([apply(np.eye(n_in)[:, k]) for k in range(n_in)])


def tiny_geometries():
    rng = np.random.default_rng(11)
    out = []
    # parallel: exact 0/45/90/135 degrees plus random angles, odd and even bins, non-unit sizes
    ang = np.concatenate([[0.0, math.pi / 4, math.pi / 2, 3 * math.pi / 4], rng.uniform(0, 2 * math.pi, 4)])
    out.append(gi.Geometry("parallel", 7, 7, 1.0, ang, 11, 1.0))
    out.append(gi.Geometry("parallel", 8, 6, 0.7, ang, 12, 0.55))
    out.append(gi.Geometry("parallel", 5, 9, 1.3, rng.uniform(0, math.pi, 5), 9, 1.7))
    # fan, flat detector: moderate and extreme magnification
    out.append(gi.Geometry("fan", 8, 8, 1.0, rng.uniform(0, 2 * math.pi, 6), 15, 2.0, 16.0, 32.0))
    out.append(gi.Geometry("fan", 6, 7, 0.8, rng.uniform(0, 2 * math.pi, 5), 13, 0.9, 7.0, 40.0))
    out.append(gi.Geometry("fan", 7, 7, 1.0, np.array([0.0, math.pi / 4, math.pi / 2, 1.0]), 10, 1.3, 9.0, 12.0))
    # fan, arc detector (equiangular bins): the same two magnifications
    out.append(gi.Geometry("fan_arc", 8, 8, 1.0, rng.uniform(0, 2 * math.pi, 6), 15, 2.0, 16.0, 32.0))
    out.append(gi.Geometry("fan_arc", 6, 7, 0.8, rng.uniform(0, 2 * math.pi, 5), 13, 0.9, 7.0, 40.0))
    return out


@pytest.mark.parametrize("g", tiny_geometries(), ids=lambda g: f"{g.beam}{g.nx}x{g.ny}")
def test_joseph_march_equals_closed_form(g):
    """Row/column marching equals A[r,p] = (pix/c) Lambda(dist/(pix c)) entrywise."""
    P = Projectors(g)
    A_march = matrix_of(P.A, g.n)
    A_closed = dense.dense_A(g)
    assert np.abs(A_march - A_closed).max() <= 1e-12


@pytest.mark.parametrize("g", tiny_geometries(), ids=lambda g: f"{g.beam}{g.nx}x{g.ny}")
def test_pixel_driven_equals_closed_form(g):
    P = Projectors(g)
    B_loop = matrix_of(P.B, g.m)
    B_closed = dense.dense_B(g)
    assert np.abs(B_loop - B_closed).max() <= 1e-12 * max(1.0, np.abs(B_closed).max())


@pytest.mark.parametrize("g", tiny_geometries(), ids=lambda g: f"{g.beam}{g.nx}x{g.ny}")
def test_transposes_are_exact(g):
    P = Projectors(g)
    A = matrix_of(P.A, g.n)
    B = matrix_of(P.B, g.m)
    assert np.abs(matrix_of(P.AT, g.m) - A.T).max() <= 1e-13
    assert np.abs(matrix_of(P.BT, g.n) - B.T).max() <= 1e-12 * max(1.0, np.abs(B).max())


def test_dot_product_identities_medium():
    rng = np.random.default_rng(5)
    for g in (gi.parallel_geometry(48, 37, 71), gi.fan_geometry(40, 53, 61, 80.0, 160.0),
              gi.fan_geometry(40, 53, 61, 80.0, 160.0, detector="arc")):
        P = Projectors(g)
        x, y = rng.standard_normal(g.n), rng.standard_normal(g.m)
        lhs, rhs = P.A(x) @ y, x @ P.AT(y)
        assert abs(lhs - rhs) <= 1e-13 * np.linalg.norm(P.A(x)) * np.linalg.norm(y) * 10
        lhs, rhs = P.B(y) @ x, y @ P.BT(x)
        assert abs(lhs - rhs) <= 1e-13 * np.linalg.norm(P.B(y)) * np.linalg.norm(x) * 10


def test_zero_degree_bins_average_two_columns():
    """theta = 0, N = 8, 11 bins: u_d - x_j = d - j - 1.5, so bin d is the mean of
    column sums d-2 and d-1 (exact for integer images)."""
    g = gi.Geometry("parallel", 8, 8, 1.0, np.array([0.0]), 11, 1.0)
    img = np.random.default_rng(3).integers(0, 9, size=(8, 8)).astype(float)
    col = np.concatenate([[0.0, 0.0], img.sum(axis=0), [0.0, 0.0]])  # col[k+2] = colsum k
    expect = np.array([0.5 * (col[d] + col[d + 1]) for d in range(11)])
    assert np.array_equal(Projectors(g).A(img.reshape(-1)), expect)


def test_ninety_degree_bins_average_two_rows():
    g = gi.Geometry("parallel", 8, 8, 1.0, np.array([math.pi / 2]), 11, 1.0)
    img = np.random.default_rng(4).integers(0, 9, size=(8, 8)).astype(float)
    row = img.sum(axis=1)
    expect = np.zeros(11)
    for d in range(11):
        for i in (8 - d, 9 - d):  # rows whose centres lie half a pixel from u_d
            if 0 <= i < 8:
                expect[d] += 0.5 * row[i]
    assert np.allclose(Projectors(g).A(img.reshape(-1)), expect, atol=1e-12, rtol=0)


def test_constant_image_gives_row_band_chord():
    """A row-stepping ray that stays inside the columns crosses all ny rows:
    A 1 = ny * pix / |cos(theta)| exactly (the length of the ray inside the row band)."""
    for th in (0.1, 0.4, 0.7, math.pi - 0.3):
        g = gi.Geometry("parallel", 40, 24, 0.5, np.array([th]), 9, 0.5)
        y = Projectors(g).A(np.ones(g.n))
        assert np.allclose(y, 24 * 0.5 / abs(math.cos(th)), rtol=1e-13)


def test_disk_chord_length_converges():
    """Line integrals of a disk of radius r: 2 sqrt(r^2 - s^2), error shrinking with N."""
    errs = []
    for N in (32, 64, 128):
        r = 0.3 * N
        g = gi.parallel_geometry(N, 7, N, arc=math.pi)
        y = Projectors(g).A(gi.disk_phantom(N, r)).reshape(7, N)
        s = (np.arange(N) - (N - 1) / 2.0)
        chord = 2.0 * np.sqrt(np.maximum(r * r - s * s, 0.0))
        errs.append(np.linalg.norm(y - chord[None, :]) / np.linalg.norm(np.broadcast_to(chord, y.shape)))
    assert errs[0] < 0.05 and errs[1] < errs[0] * 0.8 and errs[2] < errs[1] * 0.8, errs


def test_back_projection_of_ones_parallel():
    """Linear-interpolation weights sum to one: (B 1)_p = N_a pix^2/du for pixels
    that project inside the detector."""
    g = gi.Geometry("parallel", 16, 16, 1.0, np.linspace(0, math.pi, 13, endpoint=False), 31, 0.8)
    xb = Projectors(g).B(np.ones(g.m))
    assert np.allclose(xb, 13 * 1.0 / 0.8, rtol=1e-13)


def test_fan_weight_matches_ray_density():
    """Fan-beam weight w(a,p) is the inverse perpendicular ray spacing at the
    pixel, so sum_d A[(a,d),p] ~ w(a,p): B is mass-matched to A^T."""
    g = gi.fan_geometry(48, 24, 121, 96.0, 192.0, det_width=1.0)
    P = Projectors(g)
    X, Y = dense.pixel_centres(g)
    inside = X ** 2 + Y ** 2 < (0.4 * 48) ** 2
    ratios = []
    for a in range(0, 24, 5):
        ya = np.zeros(g.m)
        ya[a * g.n_det:(a + 1) * g.n_det] = 1.0
        colsum = P.AT(ya)  # sum_d A[(a,d),p]
        _, w = dense.detector_coordinate(g, a, X, Y)
        ratios.append(colsum[inside] / w[inside])
    r = np.concatenate(ratios)
    assert abs(r.mean() - 1.0) < 0.02 and r.std() < 0.2


def test_arc_weight_matches_ray_density():
    """The arc detector's weight is the inverse ray spacing rho * du / sdd at
    the pixel, so B is mass-matched to A^T there too."""
    g = gi.fan_geometry(48, 24, 121, 96.0, 192.0, det_width=1.0, detector="arc")
    P = Projectors(g)
    X, Y = dense.pixel_centres(g)
    inside = X ** 2 + Y ** 2 < (0.4 * 48) ** 2
    ratios = []
    for a in range(0, 24, 5):
        ya = np.zeros(g.m)
        ya[a * g.n_det:(a + 1) * g.n_det] = 1.0
        _, w = dense.detector_coordinate(g, a, X, Y)
        ratios.append(P.AT(ya)[inside] / w[inside])
    r = np.concatenate(ratios)
    assert abs(r.mean() - 1.0) < 0.02 and r.std() < 0.2


@pytest.mark.parametrize("beam", ["fan", "fan_arc"])
def test_pixel_bin_lies_on_its_ray(beam):
    """The ray through the fractional bin a pixel projects to passes through
    the pixel centre: the back projector's detector mapping and the forward
    projector's rays are the same geometry (a sign or a tan/atan slip breaks
    it)."""
    g = gi.Geometry(beam, 9, 9, 1.0, np.array([0.3, 2.0, 4.1]), 31, 0.8, 14.0, 30.0)
    X, Y = dense.pixel_centres(g)
    for a in range(g.n_angles):
        u, _ = dense.detector_coordinate(g, a, X, Y)
        for k in range(0, g.n, 7):
            t = u[k] / g.det_width + (g.n_det - 1) / 2.0
            p, e = dense.ray(g, a, t)
            assert abs((X[k] - p[0]) * e[1] - (Y[k] - p[1]) * e[0]) < 1e-12


def test_arc_and_flat_share_the_central_ray():
    """Bin (n_det - 1)/2 is the central ray on both detectors: equal rows of
    A; off-centre bins differ (tan versus angle)."""
    ang = np.array([0.4, 1.9])
    flat = gi.Geometry("fan", 11, 11, 1.0, ang, 21, 1.0, 20.0, 40.0)
    arc = gi.Geometry("fan_arc", 11, 11, 1.0, ang, 21, 1.0, 20.0, 40.0)
    Af, Aa = dense.dense_A(flat), dense.dense_A(arc)
    for a in range(2):
        c = a * 21 + 10
        assert np.abs(Af[c] - Aa[c]).max() <= 1e-14
        assert np.abs(Af[a * 21 + 20] - Aa[a * 21 + 20]).max() > 1e-3
        # one bin off the centre the two detectors nearly agree (tan g ~ g), and
        # not with the mirrored bin: the arc turns the same way as the flat axis
        near = np.linalg.norm(Af[c + 1] - Aa[c + 1])
        assert near < 0.05 * np.linalg.norm(Af[c + 1]) < np.linalg.norm(Af[c + 1] - Aa[c - 1])
    Pa = Projectors(arc)
    assert np.abs(matrix_of(Pa.A, arc.n) - Aa).max() <= 1e-12


def test_AT_equals_B_only_on_axis_angles():
    g0 = gi.Geometry("parallel", 9, 9, 1.0, np.array([0.0, math.pi / 2]), 13, 1.0)
    A = dense.dense_A(g0)
    B = dense.dense_B(g0)
    assert np.abs(A.T - B).max() <= 1e-12
    g45 = gi.Geometry("parallel", 9, 9, 1.0, np.array([math.pi / 4]), 13, 1.0)
    assert np.abs(dense.dense_A(g45).T - dense.dense_B(g45)).max() > 0.1


def test_single_entry_routines_match_full_passes():
    rng = np.random.default_rng(9)
    for g in (gi.parallel_geometry(20, 11, 29), gi.fan_geometry(18, 13, 27, 40.0, 80.0),
              gi.fan_geometry(18, 13, 27, 40.0, 80.0, detector="arc")):
        P = Projectors(g)
        x, y = rng.standard_normal(g.n), rng.standard_normal(g.m)
        Ax, By, ATy, BTx = P.A(x), P.B(y), P.AT(y), P.BT(x)
        for _ in range(6):
            a, d = rng.integers(g.n_angles), rng.integers(g.n_det)
            i, j = rng.integers(g.ny), rng.integers(g.nx)
            assert abs(P.A_ray(x, a, d) - Ax[a * g.n_det + d]) <= 1e-12
            assert abs(P.BT_ray(x, a, d) - BTx[a * g.n_det + d]) <= 1e-11
            assert abs(P.B_pixel(y, i, j) - By[i * g.nx + j]) <= 1e-11
            assert abs(P.AT_pixel(y, i, j) - ATy[i * g.nx + j]) <= 1e-12


def test_snr_of_paper_noise_levels():
    """Sec. 5: 4 % <-> SNR ~ 28, 7 % <-> ~ 23, 10 % <-> ~ 20."""
    assert round(gi.snr_db(0.04)) == 28
    assert round(gi.snr_db(0.07)) == 23
    assert round(gi.snr_db(0.10)) == 20


def test_noise_norm_is_exact():
    bt = np.random.default_rng(1).standard_normal(500)
    b, en = gi.add_noise(bt, gi.noise_direction(500, 2), 0.03)
    assert abs(en - 0.03 * np.linalg.norm(bt)) <= 1e-14 * en
    assert abs(np.linalg.norm(b - bt) - en) <= 1e-12 * en


def test_oracle_results_do_not_depend_on_thread_count():
    """The parallel loops split independent outputs and keep each output's
    summation order, so 1 and 4 threads give identical bits (fan and parallel,
    all four operators)."""
    from oracle import projectors as op
    saved = op.threads()
    try:
        for g in (gi.fan_geometry(40, 37, 59, 80.0, 160.0), gi.parallel_geometry(33, 29, 47)):
            P = Projectors(g)
            rng = np.random.default_rng(8)
            x, y = rng.standard_normal(g.n), rng.standard_normal(g.m)
            op.set_threads(1)
            one = [P.A(x), P.B(y), P.AT(y), P.BT(x)]
            op.set_threads(4)
            four = [P.A(x), P.B(y), P.AT(y), P.BT(x)]
            for a, b in zip(one, four):
                assert np.array_equal(a, b)
    finally:
        op.set_threads(saved)
