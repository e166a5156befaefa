"""Explicit matrices of the projectors from their closed forms (tiny grids only).

This is a second, independent route to the same operators as
``projectors.c``: instead of marching along rows, every entry is written
down directly.

* Joseph (forward) entry.  On a row crossed at abscissa x*, the pixel at
  x_j gets weight Lambda((x* - x_j)/pix) with Lambda(t) = max(0, 1 - |t|).
  The horizontal offset x* - x_j equals dist/|e_y|, dist being the
  perpendicular distance of the pixel centre from the ray, so
  A[r, p] = (pix/c) * Lambda(dist / (pix*c)) with c = max(|e_x|, |e_y|) for
  either stepping axis.
* Pixel-driven (back) entry.  B[p, (a, d)] = w(a, p) * Lambda((u_p - u_d)/du)
  with u_p the detector coordinate of the pixel centre at angle a.
"""
from __future__ import annotations

import numpy as np


def _tri(t):
    return np.maximum(0.0, 1.0 - np.abs(t))


def pixel_centres(geom):
    xs = (np.arange(geom.nx) - (geom.nx - 1) / 2.0) * geom.pixel
    ys = ((geom.ny - 1) / 2.0 - np.arange(geom.ny)) * geom.pixel
    X, Y = np.meshgrid(xs, ys)
    return X.reshape(-1), Y.reshape(-1)


def bin_coordinate(geom, d):
    return (d - (geom.n_det - 1) / 2.0) * geom.det_width


def ray(geom, a, d):
    """A point on ray (a, d) and its unit direction."""
    th = geom.angles[a]
    c, s = np.cos(th), np.sin(th)
    u = bin_coordinate(geom, d)
    if geom.beam == "parallel":
        return np.array([u * c, u * s]), np.array([-s, c])
    src = geom.sod * np.array([c, s])
    if geom.beam == "fan_arc":
        g = u / geom.sdd
        return src, np.cos(g) * np.array([-c, -s]) + np.sin(g) * np.array([-s, c])
    binc = -(geom.sdd - geom.sod) * np.array([c, s]) + u * np.array([-s, c])
    e = binc - src
    return src, e / np.linalg.norm(e)


def detector_coordinate(geom, a, X, Y):
    """(u_p, w) of every pixel centre at angle a."""
    th = geom.angles[a]
    c, s = np.cos(th), np.sin(th)
    pix2 = geom.pixel ** 2
    if geom.beam == "parallel":
        return X * c + Y * s, np.full(X.shape, pix2 / geom.det_width)
    U = geom.sod - (X * c + Y * s)
    L = -X * s + Y * c
    if geom.beam == "fan_arc":
        return geom.sdd * np.arctan2(L, U), pix2 * geom.sdd / (geom.det_width * np.hypot(U, L))
    u = geom.sdd * L / U
    w = pix2 * geom.sdd * np.sqrt(U * U + L * L) / (geom.det_width * U * U)
    return u, w


def dense_A(geom) -> np.ndarray:
    X, Y = pixel_centres(geom)
    A = np.zeros((geom.m, geom.n))
    for a in range(geom.n_angles):
        for d in range(geom.n_det):
            p, e = ray(geom, a, d)
            dist = np.abs((X - p[0]) * e[1] - (Y - p[1]) * e[0])
            c = max(abs(e[0]), abs(e[1]))
            A[a * geom.n_det + d] = geom.pixel / c * _tri(dist / (geom.pixel * c))
    return A


def dense_B(geom) -> np.ndarray:
    X, Y = pixel_centres(geom)
    B = np.zeros((geom.n, geom.m))
    for a in range(geom.n_angles):
        u, w = detector_coordinate(geom, a, X, Y)
        for d in range(geom.n_det):
            B[:, a * geom.n_det + d] = w * _tri((u - bin_coordinate(geom, d)) / geom.det_width)
    return B
