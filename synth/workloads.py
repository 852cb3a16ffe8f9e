"""Named synthetic workloads shaped like the paper's test problems.

Each entry fixes the geometry, the seed of its random draws and the FMM knobs.
Sizes follow the configurations the library is benchmarked and tested on:

* ``sl_sphere_20k``   unit geodesic sphere f=32 (20,480 triangles), single-layer,
                      densities U[-1,1], p=6, at most 64 points per leaf.
* ``demag_cube_1m``   unit cube, n=296 per face (1,051,392 triangles), double
                      layer with density n.M, M = z-hat, p=10 (p=8 misses 1e-6),
                      both pseudo-inverses truncated at 1e-8 (enough on flat faces),
                      at most 192 points per leaf (``demag_cube_270k``: n=150, the
                      same knobs but the truncations, for profiling).
* ``demag_sphere_1m`` unit geodesic sphere f=229 (1,048,820 triangles), same
                      (default truncations), at most 128 points per leaf.
* ``polar_64``        64 spheres, radii U[0.5,1.5], centres in a 20^3 box with a
                      0.05 surface gap, f=23 (10,580 triangles each, 677,120
                      unknowns), contrast eps_in/eps_out U[2,20], E0 = z-hat; adjoint
                      double layer at p=11 (p=10 reaches only about 1e-6), at most 96
                      points per leaf.
* ``batch_256``       256 independent instances of 1-64 spheres (radii U[0.5,1.5],
                      packed at the density of polar_64), each of a total size
                      log-uniform in 1k-200k triangles (about 10M in all),
                      single-layer densities U[-1,1]; one forest.
* ``batch_32``        the same recipe with 32 instances of 1k-50k (a quick case).

``serve_requests`` draws a serving stream: Poisson arrivals at a given rate, sizes
log-uniform in 2k-500k triangles, half polarization solves on sphere packs (1-64
spheres, contrast U[2,20]) and half demag evaluations on a cube or a sphere.
"""
from __future__ import annotations

import numpy as np

from .geometry import Mesh, cube_surface, geodesic_sphere, pack_mesh, sphere_pack


def uniform_density(n: int, seed: int) -> np.ndarray:
    """Seeded densities uniform in [-1, 1]."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=n)


def _sl_sphere_20k():
    m = geodesic_sphere(32)
    return dict(mesh=m, kernel="sl", p=6, max_leaf=64, density=uniform_density(m.n, 1000))


def _demag_cube_1m():
    m = cube_surface(296)
    return dict(mesh=m, kernel="dl", p=10, max_leaf=192, magnetization=(0.0, 0.0, 1.0), pinv_cutoff=1e-8)


def _demag_cube_270k():
    m = cube_surface(150)
    return dict(mesh=m, kernel="dl", p=10, max_leaf=192, magnetization=(0.0, 0.0, 1.0))


def _demag_sphere_1m():
    m = geodesic_sphere(229)
    return dict(mesh=m, kernel="dl", p=10, max_leaf=128, magnetization=(0.0, 0.0, 1.0))


def _polar_64():
    c, r = sphere_pack(64, 0.5, 1.5, 20.0, 0.05, seed=3000)
    m = pack_mesh(c, r, 23)
    contrast = np.random.default_rng(3001).uniform(2.0, 20.0, size=64)
    return dict(mesh=m, kernel="adl", p=11, max_leaf=96, centres=c, radii=r,
                contrast=contrast, eps_out=1.0, e0=(0.0, 0.0, 1.0))


def batch_instances(n_inst: int, lo: int, hi: int, seed: int):
    """Meshes of ``n_inst`` sphere packs: sizes log-uniform in [lo, hi] triangles, 1-64
    spheres each (f chosen so 20 f^2 per sphere meets the size), centres packed in a
    box scaled to keep the sphere density of a 64-sphere 20^3 pack."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_inst))
    nsph = rng.integers(1, 65, size=n_inst)
    meshes = []
    for i in range(n_inst):
        f = max(1, int(round(np.sqrt(sizes[i] / (20.0 * nsph[i])))))
        box = max(4.0, 20.0 * (nsph[i] / 64.0) ** (1.0 / 3.0))
        c, r = sphere_pack(int(nsph[i]), 0.5, 1.5, box, 0.05, seed=seed + 1 + i)
        meshes.append(pack_mesh(c, r, f))
    return meshes


def _batch(n_inst: int, lo: int, hi: int, seed: int):
    ms = batch_instances(n_inst, lo, hi, seed)
    off = np.concatenate([[0], np.cumsum([m.n for m in ms])]).astype(np.int64)
    m = Mesh(np.concatenate([x.tri for x in ms]), np.concatenate([x.sph for x in ms]),
             np.concatenate([x.body + 64 * i for i, x in enumerate(ms)]).astype(np.int32))
    return dict(mesh=m, kernel="sl", p=8, max_leaf=64, instances=off,
                density=uniform_density(m.n, seed + 999))


def _batch_256():
    return _batch(256, 1000, 200000, 4000)


def _batch_32():
    return _batch(32, 1000, 50000, 4100)


def serve_requests(n_req: int, rate: float, seed: int, lo: int = 2000, hi: int = 500000,
                   polar_frac: float = 0.5):
    """Geometry and arrival time of each request of a serving stream (dicts; the
    serving loop wraps them).  Arrivals: exponential gaps of mean 1/rate seconds."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n_req))
    sizes = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_req))
    out = []
    for i in range(n_req):
        if rng.uniform() < polar_frac:
            ns = int(rng.integers(1, 65))
            f = max(1, int(round(np.sqrt(sizes[i] / (20.0 * ns)))))
            box = max(4.0, 20.0 * (ns / 64.0) ** (1.0 / 3.0))
            c, r = sphere_pack(ns, 0.5, 1.5, box, 0.05, seed=seed + 1 + i)
            m = pack_mesh(c, r, f)
            contrast = rng.uniform(2.0, 20.0, size=ns)
            out.append(dict(arrival=float(t[i]), kind="polar", tri=m.tri, sph=m.sph,
                            eps_in=contrast[m.body] * 1.0, curv=1.0 / m.sph[:, 3], eps_out=1.0))
        else:
            if rng.uniform() < 0.5:
                m = cube_surface(max(1, int(round(np.sqrt(sizes[i] / 12.0)))))
            else:
                m = geodesic_sphere(max(1, int(round(np.sqrt(sizes[i] / 20.0)))))
            out.append(dict(arrival=float(t[i]), kind="demag", tri=m.tri, sph=m.sph))
    return out


WORKLOADS = {
    "sl_sphere_20k": _sl_sphere_20k,
    "demag_cube_1m": _demag_cube_1m,
    "demag_cube_270k": _demag_cube_270k,
    "demag_sphere_1m": _demag_sphere_1m,
    "polar_64": _polar_64,
    "batch_256": _batch_256,
    "batch_32": _batch_32,
}


def workload(name: str) -> dict:
    return WORKLOADS[name]()


__all__ = ["Mesh", "WORKLOADS", "workload", "uniform_density", "batch_instances", "serve_requests"]
