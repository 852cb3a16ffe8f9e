"""Oracle: one-point quadrature on a triangle soup -- TEST INFRASTRUCTURE ONLY.

Sec. III (electrostatic implementation): one quadrature point per triangle at its
centroid; the weight is the element's area, taken as the exact spherical-triangle
area when the body is a sphere and as the flat triangle area otherwise; the value
of the constant-monomial unknown lives at that same point.

Readings where the paper is silent (listed in the design notes):
* the point is the flat-triangle centroid, not its projection onto the sphere;
* on a sphere the normal is radial at the centroid, (c - C)/|c - C|; on a flat
  facet it is the unit facet normal from the vertex winding.

The spherical area is R^2 times the spherical excess E of the triangle whose
corners are the unit vectors a, b, c from the centre, with
tan(E/2) = |a.(b x c)| / (1 + a.b + b.c + c.a)   (Van Oosterom & Strackee, 1983).
"""
from __future__ import annotations

import numpy as np


def quadrature_points(tri: np.ndarray, sph: np.ndarray):
    """Return (xyz (3,T), w (T,), nrm (3,T)) in float64, structure-of-arrays."""
    tri = np.asarray(tri, dtype=np.float64)
    sph = np.asarray(sph, dtype=np.float64)
    A, B, C = tri[:, 0], tri[:, 1], tri[:, 2]
    cen = (A + B + C) / 3.0
    cr = np.cross(B - A, C - A)
    flat_area = 0.5 * np.linalg.norm(cr, axis=1)
    flat_n = cr / np.linalg.norm(cr, axis=1, keepdims=True)

    R = sph[:, 3]
    on_sphere = R > 0
    w = flat_area.copy()
    nrm = flat_n.copy()
    if np.any(on_sphere):
        ctr = sph[on_sphere, :3]
        Rs = R[on_sphere]
        a = A[on_sphere] - ctr
        b = B[on_sphere] - ctr
        c = C[on_sphere] - ctr
        a /= np.linalg.norm(a, axis=1, keepdims=True)
        b /= np.linalg.norm(b, axis=1, keepdims=True)
        c /= np.linalg.norm(c, axis=1, keepdims=True)
        trip = np.abs(np.einsum("ij,ij->i", a, np.cross(b, c)))
        den = 1.0 + np.einsum("ij,ij->i", a, b) + np.einsum("ij,ij->i", b, c) \
            + np.einsum("ij,ij->i", c, a)
        excess = 2.0 * np.arctan2(trip, den)
        w[on_sphere] = Rs * Rs * excess
        d = cen[on_sphere] - ctr
        nrm[on_sphere] = d / np.linalg.norm(d, axis=1, keepdims=True)
    return np.ascontiguousarray(cen.T), w, np.ascontiguousarray(nrm.T)
