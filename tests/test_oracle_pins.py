"""Pins of the oracle against facts fixed by the paper and by potential theory.

None of these re-types the oracle's formula: each checks it against a closed
form, an identity or a convergence rate that a dropped term, a wrong sign, a
wrong power of r or a swapped source/target normal would break.

Closed forms on a sphere of radius 1 with density Y_l (l = 0: 1, l = 1: z):
  single layer   inside  4pi/(2l+1) r^l Y_l           surface  4pi/(2l+1) Y_l
  double layer   inside  -4pi(l+1)/(2l+1) r^l Y_l     surface  -2pi/(2l+1) Y_l
                 outside 4pi l/(2l+1) r^-(l+1) Y_l
  adjoint DL     surface 2pi/(2l+1) Y_l
(Gauss's identity is the l = 0 double layer.)  Interior/exterior values of the
one-point rule converge as h^2; surface values, with the self term dropped, as h.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import bie
from oracle.gmres import gmres
from oracle.quadrature import quadrature_points

PI4 = 4.0 * math.pi


def sphere(f, center=(0.0, 0.0, 0.0), radius=1.0):
    m = synth.geodesic_sphere(f, center=center, radius=radius)
    return quadrature_points(m.tri, m.sph)


@pytest.fixture(scope="module")
def spheres():
    return {f: sphere(f) for f in (8, 16, 32)}


INTERIOR = np.array([[0.0, 0.0, 0.0], [0.3, -0.2, 0.1], [0.0, 0.0, 0.5]]).T
EXTERIOR = np.array([[0.0, 0.0, 2.0], [1.5, 1.0, -0.5]]).T


# ---------------------------------------------------------------- quadrature (Sec. III)
def test_spherical_weights_sum_to_sphere_area():
    for f, R, c in ((5, 1.0, (0, 0, 0)), (7, 1.7, (3.0, -2.0, 0.5))):
        xyz, w, n = sphere(f, c, R)
        assert abs(w.sum() - PI4 * R * R) < 1e-12 * PI4 * R * R
        assert np.allclose(np.linalg.norm(n, axis=0), 1.0, atol=1e-14)
        radial = (xyz - np.asarray(c)[:, None]) / np.linalg.norm(xyz - np.asarray(c)[:, None], axis=0)
        assert np.allclose(n, radial, atol=1e-14)


def test_cube_weights_and_outward_normals():
    m = synth.cube_surface(7, side=2.0, center=(1.0, 0.0, -1.0))
    xyz, w, n = quadrature_points(m.tri, m.sph)
    assert m.n == 12 * 49
    assert abs(w.sum() - 6 * 4.0) < 1e-12
    assert np.allclose(w, 4.0 / (2 * 49))
    rel = xyz - np.array([1.0, 0.0, -1.0])[:, None]
    # outward: the normal is the axis of the face the centroid lies on
    ax = np.argmax(np.abs(rel), axis=0)
    expect = np.zeros_like(n)
    expect[ax, np.arange(m.n)] = np.sign(rel[ax, np.arange(m.n)])
    assert np.array_equal(n, expect)
    # a closed flat surface: sum of n w vanishes
    assert np.abs((n * w).sum(axis=1)).max() < 1e-12


# ---------------------------------------------------------------- single layer
def test_single_layer_interior_exterior(spheres):
    errs = []
    for f in (16, 32):
        xyz, w, n = spheres[f]
        e1 = np.abs(oracle.direct("sl", INTERIOR, xyz, w) - PI4).max()
        e2 = np.abs(oracle.direct("sl", INTERIOR, xyz, w * xyz[2]) - PI4 / 3 * INTERIOR[2]).max()
        r = np.linalg.norm(EXTERIOR, axis=0)
        e3 = np.abs(oracle.direct("sl", EXTERIOR, xyz, w) - PI4 / r).max()
        e4 = np.abs(oracle.direct("sl", EXTERIOR, xyz, w * xyz[2]) - PI4 / 3 * EXTERIOR[2] / r**3).max()
        errs.append(max(e1, e2, e3, e4))
    assert errs[1] < 4e-3
    assert errs[1] < 0.3 * errs[0]          # O(h^2)


def test_single_layer_surface(spheres):
    errs = []
    for f in (16, 32):
        xyz, w, n = spheres[f]
        errs.append(np.abs(oracle.direct("sl", xyz, xyz, w) - PI4).max())
    assert errs[1] < 0.12
    assert errs[1] < 0.6 * errs[0]          # O(h)


# ---------------------------------------------------------------- double layer (Eq. kernel)
def test_double_layer_gauss_identity(spheres):
    errs = []
    for f in (16, 32):
        xyz, w, n = spheres[f]
        e1 = np.abs(oracle.direct("dl", INTERIOR, xyz, w, src_nrm=n) + PI4).max()
        e2 = np.abs(oracle.direct("dl", EXTERIOR, xyz, w, src_nrm=n)).max()
        errs.append(max(e1, e2))
    assert errs[1] < 8e-3
    assert errs[1] < 0.3 * errs[0]


def test_double_layer_first_harmonic(spheres):
    errs = []
    for f in (16, 32):
        xyz, w, n = spheres[f]
        q = w * xyz[2]
        e1 = np.abs(oracle.direct("dl", INTERIOR, xyz, q, src_nrm=n) + 8 * math.pi / 3 * INTERIOR[2]).max()
        r = np.linalg.norm(EXTERIOR, axis=0)
        e2 = np.abs(oracle.direct("dl", EXTERIOR, xyz, q, src_nrm=n) - PI4 / 3 * EXTERIOR[2] / r**3).max()
        errs.append(max(e1, e2))
    assert errs[1] < 3e-3
    assert errs[1] < 0.3 * errs[0]


def test_double_layer_surface_principal_value(spheres):
    errs = []
    for f in (16, 32):
        xyz, w, n = spheres[f]
        e1 = np.abs(oracle.direct("dl", xyz, xyz, w, src_nrm=n) + 2 * math.pi).max()
        e2 = np.abs(oracle.direct("dl", xyz, xyz, w * xyz[2], src_nrm=n) + 2 * math.pi / 3 * xyz[2]).max()
        errs.append(max(e1, e2))
    assert errs[1] < 0.06
    assert errs[1] < 0.6 * errs[0]


# ---------------------------------------------------------------- adjoint double layer (Eq. kernel_pol)
def test_adjoint_double_layer_surface(spheres):
    errs = []
    for f in (16, 32):
        xyz, w, n = spheres[f]
        e1 = np.abs(oracle.direct("adl", xyz, xyz, w, trg_nrm=n) - 2 * math.pi).max()
        e2 = np.abs(oracle.direct("adl", xyz, xyz, w * xyz[2], trg_nrm=n) - 2 * math.pi / 3 * xyz[2]).max()
        errs.append(max(e1, e2))
    assert errs[1] < 0.06
    assert errs[1] < 0.6 * errs[0]


def test_demag_uniform_sphere_interior_field(spheres):
    """H = -M/3 inside a uniformly magnetized sphere (Sec. IV.A: 4pi/3 in Gaussian units)."""
    errs = []
    for f in (16, 32):
        xyz, w, n = spheres[f]
        zhat = np.zeros_like(INTERIOR)
        zhat[2] = 1.0
        hz = oracle.direct("adl", INTERIOR, xyz, w * n[2], trg_nrm=zhat) / PI4
        errs.append(np.abs(hz + 1.0 / 3.0).max())
    assert errs[1] < 3e-4
    assert errs[1] < 0.3 * errs[0]


def test_fredkin_koehler_sphere_potential(spheres):
    """phi_1 = 4pi M.r, phi = phi_1 + phi_2 = (4pi/3) z on the sphere (Eq. fk_integral)."""
    errs = []
    for f in (16, 32):
        xyz, w, n = spheres[f]
        phi1 = PI4 * xyz[2]
        phi2 = bie.demag_phi2(xyz, n, w, phi1, np.full(xyz.shape[1], 2 * math.pi))
        errs.append(np.abs(phi1 + phi2 - PI4 / 3 * xyz[2]).max())
    assert errs[1] < 0.06
    assert errs[1] < 0.6 * errs[0]


# ---------------------------------------------------------------- identities on random points
def _random_cloud(n, seed):
    rng = np.random.default_rng(seed)
    p = rng.uniform(-1, 1, size=(3, n))
    nv = rng.normal(size=(3, n))
    nv /= np.linalg.norm(nv, axis=0)
    return p, nv, rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)


def test_adjoint_and_symmetry_identities():
    """<a, ADL b> = -<DL a, b>  and  <a, SL b> = <SL a, b>: catches swapped normals/indices."""
    p, nv, a, b = _random_cloud(600, 7)
    lhs = np.dot(a, oracle.direct("adl", p, p, b, trg_nrm=nv))
    rhs = -np.dot(b, oracle.direct("dl", p, p, a, src_nrm=nv))
    assert abs(lhs - rhs) < 1e-11 * (abs(lhs) + 1.0)
    s1 = np.dot(a, oracle.direct("sl", p, p, b))
    s2 = np.dot(b, oracle.direct("sl", p, p, a))
    assert abs(s1 - s2) < 1e-11 * abs(s1)


def test_scaling_exponents():
    """Scaling every coordinate by L divides SL by L and DL/ADL by L^2."""
    p, nv, a, _ = _random_cloud(300, 8)
    L = 3.7
    for k, power in (("sl", 1), ("dl", 2), ("adl", 2)):
        kw = {"src_nrm": nv} if k == "dl" else ({"trg_nrm": nv} if k == "adl" else {})
        f1 = oracle.direct(k, p, p, a, **kw)
        f2 = oracle.direct(k, L * p, L * p, a, **kw)
        assert np.allclose(f2 * L**power, f1, rtol=1e-12, atol=1e-12 * np.abs(f1).max())


def test_flat_plate_double_layer():
    """A flat plate's double layer, dipoles along its normal: exactly zero at the plate's
    own points (n.(x - y) = 0 for every pair), and the solid angle of the square on its
    axis (4 atan(a^2 / (z sqrt(2 a^2 + z^2))) for a square of side 2a at height z),
    approached as h^2 by the midpoint rule."""
    a, z = 1.0, 0.3
    omega = 4.0 * math.atan(a * a / (z * math.sqrt(2 * a * a + z * z)))
    errs = []
    for n in (32, 64):
        h = 2 * a / n
        c = -a + h * (np.arange(n) + 0.5)
        gx, gy = np.meshgrid(c, c, indexing="ij")
        src = np.stack([gx.ravel(), gy.ravel(), np.zeros(n * n)])
        nrm = np.zeros_like(src)
        nrm[2] = 1.0
        w = np.full(n * n, h * h)
        own = oracle.direct("dl", src, src, w, src_nrm=nrm)
        assert np.all(own == 0.0)
        above = oracle.direct("dl", np.array([[0.0], [0.0], [z]]), src, w, src_nrm=nrm)[0]
        below = oracle.direct("dl", np.array([[0.0], [0.0], [-z]]), src, w, src_nrm=nrm)[0]
        assert below == pytest.approx(-above, rel=1e-14)
        errs.append(abs(above - omega) / omega)
    assert errs[1] < 1e-3
    assert 0.15 < errs[1] / errs[0] < 0.35


def test_tolerance_radius_exclusion():
    """Pairs closer than 1e-5 contribute nothing (Sec. III.A.1); farther pairs do."""
    d = oracle.DELTA
    trg = np.zeros((3, 2))
    trg[0, 1] = 5.0
    src = np.array([[0.1 * d, 10 * d], [0.0, 0.0], [0.0, 0.0]])
    q = np.array([1.0, 1.0])
    out = oracle.direct("sl", trg, src, q)
    assert out[0] == pytest.approx(1.0 / (10 * d), rel=1e-14)
    nrm = np.array([[1.0, 1.0], [0.0, 0.0], [0.0, 0.0]])
    out = oracle.direct("dl", trg, src, q, src_nrm=nrm)
    assert out[0] == pytest.approx(-1.0 / (10 * d) ** 2, rel=1e-12)


def test_rounding_against_extended_precision():
    """The FP64 plain sum stays within 1e-13 of an extended-precision sum (fixed order)."""
    p, nv, a, _ = _random_cloud(200, 9)
    f = oracle.direct("dl", p, p, a, src_nrm=nv)
    P = p.astype(np.longdouble)
    N = nv.astype(np.longdouble)
    A = a.astype(np.longdouble)
    d = P[:, :, None] - P[:, None, :]
    r2 = (d * d).sum(axis=0)
    np.fill_diagonal(r2, 1.0)
    nd = (N[:, None, :] * d).sum(axis=0)
    K = nd / (r2 * np.sqrt(r2))
    np.fill_diagonal(K, 0.0)
    ref = (K * A[None, :]).sum(axis=1)
    assert np.abs(f - ref.astype(np.float64)).max() < 1e-13 * np.abs(K * A[None, :]).sum(axis=1).max()


def test_sampled_targets_match_full():
    p, nv, a, _ = _random_cloud(400, 10)
    full = oracle.direct("adl", p, p, a, trg_nrm=nv)
    idx = np.array([5, 0, 399, 17])
    assert np.array_equal(oracle.direct("adl", p, p, a, trg_nrm=nv, idx=idx), full[idx])


# ---------------------------------------------------------------- GMRES
def test_gmres_matches_dense_solve():
    rng = np.random.default_rng(11)
    n = 60
    A = np.eye(n) * 4.0 + rng.normal(size=(n, n)) / math.sqrt(n)
    b = rng.normal(size=n)
    ref = np.linalg.solve(A, b)
    for restart in (60, 7):                        # with and without restarts
        x, it, rel, ok = gmres(lambda v: A @ v, b, tol=1e-12, restart=restart, max_iter=2000)
        assert ok
        assert np.linalg.norm(A @ x - b) <= 1.01e-12 * np.linalg.norm(b) * 10
        assert np.linalg.norm(x - ref) < 1e-10 * np.linalg.norm(ref)


def test_gmres_zero_rhs():
    x, it, rel, ok = gmres(lambda v: 2 * v, np.zeros(5))
    assert ok and it == 0 and not x.any()


# ---------------------------------------------------------------- polarization closed form (Sec. II.C)
def test_dielectric_sphere_in_uniform_field():
    """sigma_b = 3(eps_i - eps_m)/(eps_i + 2 eps_m) E0 cos(theta); converges with refinement.

    Also selects the reading of the self term: the disc reading converges, the
    printed constant and no self term stay an order of magnitude off.
    """
    ei, em, R = 10.0, 1.0, 1.3
    s_exact = 3 * (ei - em) / (ei + 2 * em)
    err = {}
    for f in (8, 16):
        xyz, w, n = sphere(f, (1.0, 2.0, 3.0), R)
        H = np.full(xyz.shape[1], 1.0 / R)
        for ss in ("disc", "literal"):
            x, it, rel, ok = bie.polarization_solve(xyz, n, w, np.full(xyz.shape[1], ei), em, H,
                                                    (0.0, 0.0, 1.0), tol=1e-10, self_scale=ss)
            assert ok
            ex = s_exact * n[2]
            err[(f, ss)] = np.linalg.norm(x - ex) / np.linalg.norm(ex)
    assert err[(16, "disc")] < 1e-3
    assert err[(16, "disc")] < 0.5 * err[(8, "disc")]
    assert err[(16, "literal")] > 5 * err[(16, "disc")]


# ---------------------------------------------------------------- field and force (Sec. II.C)
def test_field_of_a_charged_sphere():
    """Field sum of a uniformly charged unit sphere: zero inside, Q/(4 pi r^2) r-hat
    outside with Q = 4 pi sigma (the 1/4pi of Eq. Eb applied), converging as h^2.  Each
    component is checked, so a swapped axis or sign fails."""
    errs = []
    for f in (16, 32):
        xyz, w, n = sphere(f)
        Ein = bie.field(INTERIOR, xyz, w) / PI4
        Eout = bie.field(EXTERIOR, xyz, w) / PI4
        r = np.linalg.norm(EXTERIOR, axis=0)
        errs.append(max(np.abs(Ein).max(), np.abs(Eout - EXTERIOR / r**3).max()))
    assert errs[1] < 1e-3
    assert errs[1] < 0.3 * errs[0]


def test_surface_field_is_the_average_of_both_sides():
    """At the elements of a charged sphere (sigma = 1) the normal component of the
    discrete field with its self-patch term tends to the mean of the outer (sigma) and
    inner (0) normal fields, E^j . n_j -> 1/2 (the principal value), at O(h).  (The
    one-point rule does not resolve the tangential part at an element: neighbours at
    distance h each contribute O(1) there.  Summed over a body, those pair terms cancel
    two by two, which the force tests below rely on.)"""
    errs = []
    for f in (16, 32):
        xyz, w, n = sphere(f)
        E = bie.polarization_field(xyz, n, w, np.ones(w.size), np.ones(w.size))
        errs.append(np.abs((E * n).sum(axis=0) - 0.5).max())
    assert errs[1] < 0.01
    assert errs[1] < 0.6 * errs[0]


def _solve_pack(centres, radii, eps_in_body, f, e0=(0.0, 0.0, 0.0), charges=None, eps_out=1.0):
    m = synth.pack_mesh(np.asarray(centres, float), np.asarray(radii, float), f)
    xyz, w, n = quadrature_points(m.tri, m.sph)
    eps = np.asarray(eps_in_body, float)[m.body]
    curv = 1.0 / m.sph[:, 3]
    sf = np.zeros(m.n)
    if charges is not None:
        sf = np.asarray(charges, float)[m.body] / (PI4 * np.asarray(radii, float)[m.body] ** 2)
    A = bie.polarization_operator(xyz, n, w, eps, eps_out, curv)
    b = bie.polarization_rhs(xyz, n, w, eps, eps_out, curv, e0, sf)
    sb, _, _, ok = gmres(A, b, tol=1e-12, restart=60)
    assert ok
    F = bie.polarization_force(xyz, n, w, sf + sb, curv, m.body, eps_out, e0)
    return m, sf, sb, F


def test_uncharged_sphere_feels_no_force_in_a_uniform_field():
    """A neutral dielectric sphere in a uniform field: its bound charge is odd under
    inversion and the field even, so sigma E is odd and the net force vanishes (the
    geodesic mesh is centrally symmetric)."""
    m, sf, sb, F = _solve_pack([[0.0, 0.0, 0.0]], [1.0], [10.0], 8, e0=(0.3, -0.2, 1.0))
    scale = np.abs(sb).max() ** 2 * PI4
    assert np.abs(F).max() < 1e-10 * scale
    assert abs((sb * quadrature_points(m.tri, m.sph)[1]).sum()) < 1e-10 * scale   # no net bound charge


@pytest.mark.parametrize("eps_in", [2.0, 10.0])
def test_charged_spheres_coulomb_limit(eps_in):
    """Two charged spheres of radius 1 at distance 20 in a medium eps_m = 2.
    - eps_in = eps_m: the solve gives sigma_b = -sigma_f / 2 exactly (Eq. Ax and Eq.
      rhs with deps = 0), so each body carries Q_i / eps_m in all;
    - eps_in = 10: the same total charge up to the one-point rule's O(h) error in the
      surface field (f = 8 vs f = 16 checked to converge);
    and F = eps_m q1 q2 / (4 pi d^2) along the axis with q_i those totals (the shell
    theorem: the force on a uniform shell is that on its centre), equal and opposite.
    With eps_in = eps_m the charge is uniform and that holds to the solve's tolerance.
    With eps_in = 10 it holds up to the induced-dipole terms, (R/d)^3 ~ 1e-4 relative,
    and the self-patch term c_j sigma_j n_j: on the now uneven charge it leaves an O(h)
    net self-force, which halves from f = 8 to f = 16."""
    d, Q1, Q2, em = 20.0, 3.0, 2.0, 2.0
    errs, ferr = [], []
    for f in (8, 16):
        m, sf, sb, F = _solve_pack([[0.0, 0.0, 0.0], [d, 0.0, 0.0]], [1.0, 1.0], [eps_in, eps_in], f,
                                   charges=[Q1, Q2], eps_out=em)
        w = quadrature_points(m.tri, m.sph)[1]
        tot = [((sf + sb) * w)[m.body == b].sum() for b in (0, 1)]
        errs.append(max(abs(tot[0] - Q1 / em) / Q1, abs(tot[1] - Q2 / em) / Q2))
        coul = em * tot[0] * tot[1] / (PI4 * d * d)
        ferr.append(max(abs(F[1, 0] - coul), abs(F[0, 0] + coul)) / coul)
        assert np.abs(F[:, 1:]).max() < 1e-6 * coul
    if eps_in == em:
        assert max(errs) < 1e-9 and max(ferr) < 3e-4
    else:
        assert errs[1] < 0.6 * errs[0] and errs[1] < 5e-3
        assert ferr[1] < 0.6 * ferr[0] and ferr[1] < 0.01
