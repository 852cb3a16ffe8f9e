"""Field vectors and body forces on the GPU (KIFMM_KERNEL_FIELD, kifmm_polarization_field,
kifmm_polarization_force, kifmm_polarization_rhs_free) against the oracle.

The field kernel is the gradient kernel of Eq. kernel_pol with all three components (Eq.
Eb); the force on a body integrates the surface force density eps_m sigma E over it
(Sec. II.C).  The mixed form is held to rel-L2 <= 1e-6 at p = 11, the order the
adjoint double layer (one component of the same gradient) needs; FP64 at p = 12.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import bie as obie
from oracle.gmres import gmres
from oracle.quadrature import quadrature_points

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
P_FIELD = 11


def gpu_points(m):
    from paper_1605_01715_gb300 import kifmm_quadrature_points
    tri = torch.from_numpy(np.ascontiguousarray(m.tri.reshape(-1, 9))).to(DEV)
    sph = torch.from_numpy(np.ascontiguousarray(m.sph)).to(DEV)
    return kifmm_quadrature_points(tri, sph)


def t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


MESHES = {
    "sphere": lambda: synth.geodesic_sphere(16),
    "pack": lambda: synth.pack_mesh(*synth.sphere_pack(4, 0.5, 1.5, 8.0, 0.05, 1), 10),
    "cube": lambda: synth.cube_surface(37),
}


@pytest.mark.parametrize("geom", ["sphere", "pack", "cube"])
@pytest.mark.parametrize("prec,p,tol", [("mixed", P_FIELD, 1e-6), ("fp64", 12, 1e-7)])
def test_field_matches_oracle(geom, prec, p, tol):
    from paper_1605_01715_gb300 import Plan, Tree
    m = MESHES[geom]()
    hx, hw, hn = quadrature_points(m.tri, m.sph)
    xyz, w, nrm = gpu_points(m)
    sig = synth.uniform_density(m.n, 21)
    ref = obie.field(hx, hx, sig * hw)
    plan = Plan(Tree(xyz, max_leaf=40), kernel="field", p=p, precision=prec)
    out = plan.matvec(t(sig) * w).cpu().numpy().reshape(3, m.n)
    plan.check()
    err = rel(out, ref)
    print("%s field %s p=%d rel-L2 %.3e" % (geom, prec, p, err))
    assert err < tol


def test_field_at_volume_targets_and_host_buffers():
    """Targets off the surface (the target-source model), and the host-buffer matvec,
    whose output holds the three components as three blocks of n_trg."""
    from paper_1605_01715_gb300 import Plan, Tree
    m = synth.cube_surface(37)
    hx, hw, hn = quadrature_points(m.tri, m.sph)
    xyz, w, nrm = gpu_points(m)
    sig = synth.uniform_density(m.n, 21)
    rng = np.random.default_rng(4)
    trg = rng.uniform(-0.7, 0.7, size=(3, 3001))
    ref = obie.field(trg, hx, sig * hw)
    plan = Plan(Tree(xyz, t(trg), max_leaf=48), kernel="field", p=P_FIELD, precision="mixed")
    q = t(sig) * w
    out = plan.matvec(q)
    err = rel(out.cpu().numpy().reshape(3, -1), ref)
    print("volume targets field rel-L2 %.3e" % err)
    assert err < 1e-6
    oh = torch.empty(3 * 3001, dtype=torch.float64).pin_memory()
    plan.matvec_host(q.cpu().pin_memory(), oh, graph=True)
    torch.cuda.synchronize()
    assert float((oh - out.cpu()).abs().max()) <= 1e-6 * float(out.abs().max())


def _two_charged_spheres(f=8):
    """The paper's two-sphere problem (Sec. IV.B, Fig. fig_color_dielectric (a)): radius
    1, eps_1 = eps_2 = 15 in eps_m = 1, charges 10 q and q, centres 2.5 apart."""
    c = np.array([[0.0, 0.0, 0.0], [2.5, 0.0, 0.0]])
    r = np.array([1.0, 1.0])
    m = synth.pack_mesh(c, r, f)
    hx, hw, hn = quadrature_points(m.tri, m.sph)
    eps = np.full(m.n, 15.0)
    curv = 1.0 / m.sph[:, 3]
    Q = np.array([10.0, 1.0])
    sf = Q[m.body] / (4 * np.pi * r[m.body] ** 2)
    return m, (hx, hw, hn), eps, curv, sf


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_force_between_charged_dielectric_spheres(prec):
    """Free-charge right-hand side, GMRES solve, surface field and the force on each
    body, each against the oracle.
    - rhs: rel-L2 1e-6 (mixed) / 1e-7 (FP64 at p = 12);
    - field evaluated on the oracle's own charge: rel-L2 1e-6 / 1e-7;
    - forces on that charge: the same bound on the error of each force component,
      relative to the size of its summands, sum_j |eps_m sigma_j a_j| |E^j| (a body's
      force is a small remainder of them: that is the error norm the field's rel-L2 fixes);
    - the GPU solve: residual under the oracle's operator below 1e-6 / 1e-7, and the
      GPU forces on that solution against the oracle's forces on it, as above.  (How far
      the solve's residual moves the force is a property of the system, printed.)"""
    from paper_1605_01715_gb300 import Plan, Tree
    m, (hx, hw, hn), eps, curv, sf = _two_charged_spheres()
    xyz, w, nrm = gpu_points(m)
    p = P_FIELD if prec == "mixed" else 12
    tol = 1e-6 if prec == "mixed" else 1e-7
    e0 = (0.0, 0.0, 0.0)
    # oracle chain
    A = obie.polarization_operator(hx, hn, hw, eps, 1.0, curv)
    b_ref = obie.polarization_rhs(hx, hn, hw, eps, 1.0, curv, e0, sf)
    sb_ref, _, _, ok = gmres(A, b_ref, tol=1e-12, restart=60)
    assert ok
    sig_ref = sf + sb_ref
    E_ref = obie.polarization_field(hx, hn, hw, sig_ref, curv, e0)
    F_ref = obie.polarization_force(hx, hn, hw, sig_ref, curv, m.body, 1.0, e0)
    # GPU chain
    tree = Tree(xyz, max_leaf=32)
    adl = Plan(tree, kernel="adl", p=p, precision=prec, trg_nrm=nrm)
    fld = Plan(tree, kernel="field", p=p, precision=prec)
    b = adl.polarization_rhs_free(w, t(eps), 1.0, t(curv), nrm, t(sf), e0)
    err_b = rel(b.cpu().numpy(), b_ref)
    E = fld.polarization_field(w, t(curv), nrm, t(sig_ref), e0)
    err_E = rel(E.cpu().numpy(), E_ref)
    body = t(m.body.astype(np.int32))
    F = fld.polarization_force(w, t(curv), nrm, t(sig_ref), 1.0, body, 2, e0).cpu().numpy()
    fscale = np.bincount(m.body, weights=np.abs(sig_ref * hw) * np.linalg.norm(E_ref, axis=0))
    err_F = (np.abs(F - F_ref).max(axis=1) / fscale).max()
    x, it, rr, rc = adl.bie_solve(w, t(eps), 1.0, t(curv), b, tol=1e-10 if prec == "fp64" else 1e-8, restart=50)
    assert rc == 0
    F2 = fld.polarization_force(w, t(curv), nrm, t(sf) + x, 1.0, body, 2, e0).cpu().numpy()
    xh = x.cpu().numpy()
    res_or = np.linalg.norm(b_ref - A(xh)) / np.linalg.norm(b_ref)
    F2_or = obie.polarization_force(hx, hn, hw, sf + xh, curv, m.body, 1.0, e0)
    err_F2 = (np.abs(F2 - F2_or).max(axis=1) / fscale).max()
    moved = np.abs(F2_or - F_ref).max() / np.abs(F_ref).max()
    print("%s: rhs %.2e field %.2e force %.2e; solve %d its, oracle residual %.2e, force on it %.2e "
          "(the residual moves the force by %.2e); F = %s" % (prec, err_b, err_E, err_F, it, res_or, err_F2, moved,
                                                              F_ref.tolist()))
    assert err_b < tol and err_E < tol and err_F < tol
    assert abs(F_ref[0, 0] + F_ref[1, 0]) < 0.05 * abs(F_ref[0, 0])      # nearly equal and opposite
    assert res_or < (1e-7 if prec == "fp64" else 1e-6)
    assert err_F2 < tol


def test_demag_field_inside_a_uniformly_magnetized_sphere():
    """H = -M/3 inside a uniformly magnetized sphere (Sec. IV.A, 4 pi / 3 in Gaussian
    units), through the library: with M = z the field's z component at an interior
    point is (1/4pi) sum_j (n_j . M) w_j z.(r - r_j)/|r - r_j|^3, the adjoint double
    layer of the charge n_j . M with target normal z, in the target-source model.
    - against the oracle at every target: rel-L2 <= 1e-6 (mixed, p = 11);
    - against -1/3: within 2e-4 at every target of radius <= 0.6, the discretization
      error of the 32,000-point sphere (the oracle on the same points: 1.1e-4)."""
    from paper_1605_01715_gb300 import Plan, Tree
    m = synth.geodesic_sphere(40)
    hx, hw, hn = quadrature_points(m.tri, m.sph)
    xyz, w, nrm = gpu_points(m)
    rng = np.random.default_rng(11)
    n = 2000
    v = rng.normal(size=(3, n))
    trg = v / np.linalg.norm(v, axis=0) * 0.6 * rng.uniform(0, 1, n) ** (1 / 3)
    zhat = np.zeros((3, n))
    zhat[2] = 1.0
    ref = oracle.direct("adl", trg, hx, hn[2] * hw, trg_nrm=zhat) / (4 * np.pi)
    plan = Plan(Tree(xyz, t(trg), max_leaf=64), kernel="adl", p=P_FIELD, precision="mixed", trg_nrm=t(zhat))
    Hz = plan.matvec(nrm[2] * w).cpu().numpy() / (4 * np.pi)
    plan.check()
    err = rel(Hz, ref)
    dev = np.abs(Hz + 1.0 / 3.0).max()
    print("interior H_z: rel-L2 vs oracle %.3e, max |H_z + 1/3| %.3e (oracle %.3e)"
          % (err, dev, np.abs(ref + 1.0 / 3.0).max()))
    assert err < 1e-6
    assert dev < 2e-4
