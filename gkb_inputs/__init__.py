"""Seeded synthetic CT inputs shared by the oracle, the tests and the benchmark.

This module only *describes* problems and draws random numbers: scan
geometries, ellipse phantoms sampled at pixel centres, and white Gaussian
noise directions.  It contains none of the reconstruction method's
arithmetic (no projector, no Krylov step), so both the FP64 CPU oracle and
the CUDA path can consume exactly the same inputs without sharing code.

Conventions (the paper uses ASTRA and states none; these readings are fixed
here and restated in the design notes):

* Image: ``ny`` rows by ``nx`` columns, row-major, pixel width ``pixel``.
  Pixel (i, j) has its centre at x = (j - (nx-1)/2)*pixel,
  y = ((ny-1)/2 - i)*pixel.
* Parallel beam: angle theta, bin d has detector coordinate
  u_d = (d - (n_det-1)/2)*det_width; the ray is the line of points whose
  coordinate x*cos(theta) + y*sin(theta) equals u_d.
* Fan beam with a flat detector: source at sod*(cos, sin); detector line at
  distance sdd from the source through -(sdd-sod)*(cos, sin), axis
  (-sin, cos); bin centres at u_d along that axis.
* Fan beam with an arc detector (equiangular bins): the same source; the
  detector is the circle of radius sdd about the source and bin d sits at
  arc length u_d from the central ray, i.e. ray d leaves the source at the
  angle gamma_d = u_d / sdd from the central ray, turned towards (-sin, cos).
* Noise: e = eta * ||b_true|| * g / ||g|| with g ~ N(0, I), so that
  ||e|| = eta * ||b_true|| exactly (Sec. 5: the noise level is the ratio of
  norms; "4 % noise" is quoted with SNR ~ 28 = 20*log10(1/0.04)).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List

import numpy as np

PARALLEL = "parallel"
FAN = "fan"
FAN_ARC = "fan_arc"


@dataclasses.dataclass
class Geometry:
    beam: str
    nx: int
    ny: int
    pixel: float
    angles: np.ndarray  # radians, float64
    n_det: int
    det_width: float
    sod: float = 0.0
    sdd: float = 0.0

    @property
    def n_angles(self) -> int:
        return int(len(self.angles))

    @property
    def n(self) -> int:
        return self.nx * self.ny

    @property
    def m(self) -> int:
        return self.n_angles * self.n_det


def parallel_geometry(N: int, n_angles: int, n_det: int | None = None,
                      arc: float = math.pi, det_width: float = 1.0,
                      pixel: float = 1.0, ny: int | None = None) -> Geometry:
    """Angles evenly over [0, arc), endpoint excluded; bins default to ceil(sqrt(2) N)."""
    if n_det is None:
        n_det = int(math.ceil(math.sqrt(2.0) * N))
    ang = np.arange(n_angles, dtype=np.float64) * (arc / n_angles)
    return Geometry(PARALLEL, N, N if ny is None else ny, pixel, ang, n_det, det_width)


def fan_geometry(N: int, n_angles: int, n_det: int, sod: float, sdd: float,
                 det_width: float | None = None, arc: float = 2.0 * math.pi,
                 pixel: float = 1.0, detector: str = "flat") -> Geometry:
    """Fan beam with a flat (default) or arc detector.  Default bin width
    sdd/sod makes the bin width at the rotation centre one pixel (on the
    arc detector: the angular bin width pixel/sod)."""
    if det_width is None:
        det_width = sdd / sod * pixel
    ang = np.arange(n_angles, dtype=np.float64) * (arc / n_angles)
    beam = {"flat": FAN, "arc": FAN_ARC}[detector]
    return Geometry(beam, N, N, pixel, ang, n_det, det_width, sod, sdd)


# ---------------------------------------------------------------------------
# phantoms and noise

def ellipse_params(N: int, n_ellipses: int, seed: int, pixel: float = 1.0) -> np.ndarray:
    """Rows (cx, cy, a, b, phi, rho): centre, semi-axes, orientation, intensity.

    Full axes are drawn from U[0.05, 0.4] * FOV (FOV = N * pixel), the
    orientation from U[0, pi), the intensity from U[0.1, 1], and the centre
    uniformly in the disk of radius FOV/2 - semi-major, so every ellipse lies
    inside the inscribed circle of the image.
    """
    rng = np.random.default_rng(seed)
    fov = N * pixel
    out = np.empty((n_ellipses, 6))
    for e in range(n_ellipses):
        ax = rng.uniform(0.05, 0.4, size=2) * fov / 2.0
        phi = rng.uniform(0.0, math.pi)
        rho = rng.uniform(0.1, 1.0)
        rmax = fov / 2.0 - ax.max()
        r = rmax * math.sqrt(rng.uniform())
        psi = rng.uniform(0.0, 2.0 * math.pi)
        out[e] = (r * math.cos(psi), r * math.sin(psi), ax[0], ax[1], phi, rho)
    return out


def rasterize(params: np.ndarray, nx: int, ny: int, pixel: float = 1.0) -> np.ndarray:
    """Point-sample the sum of ellipse indicators at pixel centres (row-major)."""
    xs = (np.arange(nx) - (nx - 1) / 2.0) * pixel
    ys = ((ny - 1) / 2.0 - np.arange(ny)) * pixel
    X, Y = np.meshgrid(xs, ys)
    img = np.zeros((ny, nx))
    for cx, cy, a, b, phi, rho in params:
        c, s = math.cos(phi), math.sin(phi)
        u = (X - cx) * c + (Y - cy) * s
        v = -(X - cx) * s + (Y - cy) * c
        img += rho * ((u / a) ** 2 + (v / b) ** 2 <= 1.0)
    return img.reshape(-1)


def ellipse_phantom(N: int, n_ellipses: int, seed: int, pixel: float = 1.0) -> np.ndarray:
    return rasterize(ellipse_params(N, n_ellipses, seed, pixel), N, N, pixel)


def disk_phantom(N: int, radius: float, pixel: float = 1.0) -> np.ndarray:
    """Unit-density centred disk, point-sampled (used by the chord-length check)."""
    return rasterize(np.array([[0.0, 0.0, radius, radius, 0.0, 1.0]]), N, N, pixel)


def noise_direction(m: int, seed: int) -> np.ndarray:
    """White Gaussian draw g ~ N(0, I) of length m."""
    return np.random.default_rng(seed).standard_normal(m)


def add_noise(b_true: np.ndarray, g: np.ndarray, eta: float):
    """Return (b, ||e||) with e = eta*||b_true||*g/||g||."""
    bt = np.asarray(b_true, dtype=np.float64)
    e = eta * np.linalg.norm(bt) * g / np.linalg.norm(g)
    return bt + e, float(np.linalg.norm(e))


def snr_db(eta: float) -> float:
    """SNR in dB of a noise level eta = ||e|| / ||b_true||."""
    return 20.0 * math.log10(1.0 / eta)


# ---------------------------------------------------------------------------
# the workloads

@dataclasses.dataclass
class Workload:
    name: str
    geom: Geometry
    n_ellipses: int
    phantom_seed: int
    noise_seed: int
    eta: float
    k_max: int


def small_parallel_64() -> Workload:
    """64x64, parallel beam, 90 angles over [0, 180), 91 bins, 10 ellipses, 1 % noise, k = 30."""
    return Workload("parallel64_a90_d91", parallel_geometry(64, 90, 91), 10, 1, 101, 0.01, 30)


def fan_512() -> Workload:
    """512x512 flat fan beam, 720 angles over [0, 360), 725 bins, SOD 1024,
    SDD 2048 (bin width 2 px: 1 px at the rotation centre), 30 ellipses,
    2 % noise, k = 150."""
    return Workload("fan512_a720_d725", fan_geometry(512, 720, 725, 1024.0, 2048.0), 30, 2, 102, 0.02, 150)


def parallel_2048() -> Workload:
    """2048x2048 parallel beam, 1800 angles over [0, 180), 2897 bins, 50 ellipses, 1 % noise, k = 200."""
    return Workload("parallel2048_a1800_d2897", parallel_geometry(2048, 1800, 2897), 50, 4, 104, 0.01, 200)


def fan_256_training() -> Workload:
    """The 512 fan geometry scaled to 256x256: SOD 512, SDD 1024, 363 bins, 720 angles over 360."""
    return Workload("fan256_a720_d363", fan_geometry(256, 720, 363, 512.0, 1024.0), 20, 5, 105, 0.02, 150)


def batch_slices(n_slices: int = 256, seed: int = 3, k_max: int = 150) -> List[Workload]:
    """Uneven multi-slice batch: N uniform in {256,384,512,768,1024}, angles
    uniform in {180,360,720} over [0,180), bins ceil(sqrt(2) N), 10-30
    ellipses, noise U[0.5 %, 5 %]; slice i uses phantom seed 1000+i and noise
    seed 2000+i."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_slices):
        N = int(rng.choice([256, 384, 512, 768, 1024]))
        na = int(rng.choice([180, 360, 720]))
        ne = int(rng.integers(10, 31))
        eta = float(rng.uniform(0.005, 0.05))
        out.append(Workload(f"slice{i}", parallel_geometry(N, na), ne, 1000 + i, 2000 + i, eta, k_max))
    return out


def scaled_batch_slices(n_slices: int, sizes, angles, seed: int = 7, k_max: int = 30) -> List[Workload]:
    """A smaller batch with the same recipe, for tests the oracle can finish."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_slices):
        N = int(rng.choice(sizes))
        na = int(rng.choice(angles))
        ne = int(rng.integers(3, 9))
        eta = float(rng.uniform(0.005, 0.05))
        out.append(Workload(f"small_slice{i}", parallel_geometry(N, na), ne, 3000 + i, 4000 + i, eta, k_max))
    return out


def phantom_of(w: Workload) -> np.ndarray:
    return ellipse_phantom(w.geom.nx, w.n_ellipses, w.phantom_seed, w.geom.pixel)
