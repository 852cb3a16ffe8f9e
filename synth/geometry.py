"""Triangle-soup meshes of the paper's synthetic geometries (spheres, cubes, sphere packs).

The paper meshes dielectric spheres and magnetic cubes/spheres with an external
mesher (Sec. III) and places one quadrature point per triangle.  Here the
meshes are generated directly:

* ``geodesic_sphere(f)``: every face of an icosahedron is cut into f*f
  triangles on a barycentric grid and all vertices are pushed onto the sphere;
  20*f*f triangles (f = 32 gives 20,480 = the level-5 icosphere count).
* ``cube_surface(n)``: each face of a cube is an n x n grid of squares, two
  triangles per square, wound counter-clockwise seen from outside; 12*n*n
  triangles.
* ``sphere_pack``: non-overlapping spheres with radii and centres drawn from a
  seeded generator, accepted only with a gap between surfaces.

A mesh is a triangle soup: ``tri`` (T, 3, 3) vertex coordinates, ``sph``
(T, 4) the centre and radius of the sphere a triangle lies on (radius 0 for a
flat facet), ``body`` (T,) the index of the body it belongs to.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Mesh:
    tri: np.ndarray   # (T, 3, 3) float64 vertex coordinates
    sph: np.ndarray   # (T, 4) float64 sphere centre + radius, radius 0 => flat facet
    body: np.ndarray  # (T,) int32 body index

    @property
    def n(self) -> int:
        return int(self.tri.shape[0])

    def concat(self, other: "Mesh") -> "Mesh":
        off = int(self.body.max()) + 1 if self.n else 0
        return Mesh(np.concatenate([self.tri, other.tri]),
                    np.concatenate([self.sph, other.sph]),
                    np.concatenate([self.body, other.body + off]).astype(np.int32))


def _icosahedron():
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
                  [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    return v, f


def geodesic_sphere(freq: int, center=(0.0, 0.0, 0.0), radius: float = 1.0) -> Mesh:
    """Frequency-``freq`` geodesic sphere: 20*freq^2 triangles on the sphere."""
    if freq < 1:
        raise ValueError("freq must be >= 1")
    v, f = _icosahedron()
    # barycentric grid cells (i, j), i + j < freq: an "up" triangle per cell and a
    # "down" triangle where i + j < freq - 1
    ii, jj = np.meshgrid(np.arange(freq), np.arange(freq), indexing="ij")
    up = (ii + jj) < freq
    dn = (ii + jj) < freq - 1
    iu, ju = ii[up], jj[up]
    idn, jdn = ii[dn], jj[dn]
    cells = [((iu, ju), (iu + 1, ju), (iu, ju + 1)),
             ((idn + 1, jdn), (idn + 1, jdn + 1), (idn, jdn + 1))]
    out = []
    for a, b, c in f:
        A, B, C = v[a], v[b], v[c]
        face = []
        for corners in cells:
            pts = []
            for (i, j) in corners:
                k = freq - i - j
                pts.append((k[:, None] * A + i[:, None] * B + j[:, None] * C) / freq)
            face.append(np.stack(pts, axis=1))
        out.append(np.concatenate(face))
    tri = np.concatenate(out).astype(np.float64)
    tri /= np.linalg.norm(tri, axis=2, keepdims=True)
    tri = tri * radius + np.asarray(center, dtype=np.float64)
    sph = np.empty((tri.shape[0], 4))
    sph[:, :3] = center
    sph[:, 3] = radius
    return Mesh(tri, sph, np.zeros(tri.shape[0], dtype=np.int32))


def cube_surface(n: int, side: float = 1.0, center=(0.0, 0.0, 0.0)) -> Mesh:
    """Axis-aligned cube of edge ``side``: 12*n^2 triangles, outward winding."""
    if n < 1:
        raise ValueError("n must be >= 1")
    h = side / 2.0
    g = np.linspace(-h, h, n + 1)
    uu, vv = np.meshgrid(g[:-1], g[:-1], indexing="ij")
    du = side / n
    u0, v0 = uu.ravel(), vv.ravel()
    out = []
    for a in range(3):
        for sgn in (1.0, -1.0):
            b, c = (a + 1) % 3, (a + 2) % 3
            if sgn < 0:
                b, c = c, b          # keep e_b x e_c = sgn * e_a

            def pt(u, v):
                p = np.zeros((u.size, 3))
                p[:, a] = sgn * h
                p[:, b] = u
                p[:, c] = v
                return p

            p00, p10 = pt(u0, v0), pt(u0 + du, v0)
            p11, p01 = pt(u0 + du, v0 + du), pt(u0, v0 + du)
            out.append(np.stack([p00, p10, p11], axis=1))
            out.append(np.stack([p00, p11, p01], axis=1))
    tri = np.concatenate(out) + np.asarray(center, dtype=np.float64)
    return Mesh(tri, np.zeros((tri.shape[0], 4)), np.zeros(tri.shape[0], dtype=np.int32))


def sphere_pack(n_spheres: int, rmin: float, rmax: float, box: float, gap: float,
                seed: int, max_tries: int = 100000):
    """Rejection-sampled non-overlapping spheres in [0, box]^3.

    Radii ~ U[rmin, rmax]; a candidate centre ~ U[r, box - r]^3 is accepted when
    its surface keeps at least ``gap`` from every accepted sphere.  Returns
    (centres (n,3), radii (n,)).
    """
    rng = np.random.default_rng(seed)
    radii = rng.uniform(rmin, rmax, size=n_spheres)
    centres = np.zeros((n_spheres, 3))
    for i, r in enumerate(radii):
        for _ in range(max_tries):
            c = rng.uniform(r, box - r, size=3)
            if i == 0 or np.all(np.linalg.norm(centres[:i] - c, axis=1) >= radii[:i] + r + gap):
                centres[i] = c
                break
        else:
            raise RuntimeError("sphere_pack: could not place sphere %d" % i)
    return centres, radii


def pack_mesh(centres, radii, freq: int) -> Mesh:
    """One geodesic sphere of frequency ``freq`` per (centre, radius)."""
    unit = geodesic_sphere(freq)
    T = unit.n
    tri = np.empty((len(radii) * T, 3, 3))
    sph = np.empty((len(radii) * T, 4))
    body = np.empty(len(radii) * T, dtype=np.int32)
    for i, (c, r) in enumerate(zip(centres, radii)):
        tri[i * T:(i + 1) * T] = unit.tri * r + c
        sph[i * T:(i + 1) * T, :3] = c
        sph[i * T:(i + 1) * T, 3] = r
        body[i * T:(i + 1) * T] = i
    return Mesh(tri, sph, body)


def cube_n_for_triangles(t: int) -> int:
    """Smallest n with 12 n^2 >= t."""
    return int(math.ceil(math.sqrt(t / 12.0)))


def geodesic_freq_for_triangles(t: int) -> int:
    """Smallest f with 20 f^2 >= t."""
    return int(math.ceil(math.sqrt(t / 20.0)))
