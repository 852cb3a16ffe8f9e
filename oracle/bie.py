"""Oracle: the boundary-integral operators built on the direct sums -- TEST INFRASTRUCTURE ONLY.

Polarization (Sec. II.C and III.A.2), with eps_0 = 1 (it cancels between Eq. Ax and
Eq. Eb):

    (A sigma)_j = ebar_j sigma_j + deps_j (E_b^j . n_j)                         (Eq. Ax)
    E_b^j . n_j = (1/4pi) [ sum_{k != j} n_j.(r_j - r_k)/|r_j - r_k|^3 sigma_k a_k
                            + c_j sigma_j ]                                     (Eq. pol_discret)
    ebar_j = (eps_j + eps_m)/2,  deps_j = eps_m - eps_j
    b_j = (1 - ebar_j) sigma_f,j - deps_j E_f . n_j                             (Eq. rhs)

Reading of the self-correction term (the paper's term lacks sigma and its constant
is ambiguous): c_j sigma_j with c_j = H_j sqrt(pi a_j) -- the principal-value normal
field at the centre of a disc of area a_j on a surface of mean curvature H_j
carrying unit density (pi rho H with rho = sqrt(a_j/pi)).  ``self_scale='literal'``
uses the printed sqrt(a_j/pi) H_j instead.  H_j = 1/R on a sphere, 0 when flat.

Field and force (Sec. II.C, Eqs. Eb and pol_discret, the force on a body and its
surface force density), for total surface charge sigma = sigma_f + sigma_b:

    E^j   = E0 + (1/4pi) [ sum_{k != j} (r_j - r_k)/|r_j - r_k|^3 sigma_k a_k + c_j sigma_j n_j ]
    F_b   = sum_{j in body b} eps_m sigma_j E^j a_j                             (f = eps_m sigma E)

with E0 the applied uniform field (the free-volume-charge term of Eq. Ef is absent).

Demagnetization (Sec. II.B and III.A.1):

    phi_2(r_i) = (1/4pi) sum_j n_j.(r_i - r_j)/|r_i - r_j|^3 phi_1(r_j) w_j
                 + (Omega_i/4pi - 1) phi_1(r_i)                                (Eq. fk_integral_discrete)
"""
from __future__ import annotations

import math

import numpy as np

from . import direct
from .gmres import gmres

FOUR_PI = 4.0 * math.pi


def self_coefficient(area, curvature, self_scale: str = "disc"):
    area = np.asarray(area, dtype=np.float64)
    curvature = np.asarray(curvature, dtype=np.float64)
    if self_scale == "disc":
        return curvature * np.sqrt(math.pi * area)
    if self_scale == "literal":
        return curvature * np.sqrt(area / math.pi)
    if self_scale == "none":
        return np.zeros_like(area)
    raise ValueError(self_scale)


def polarization_operator(xyz, nrm, area, eps_in, eps_out, curvature, self_scale="disc"):
    """Return matvec(sigma) for the polarization system A sigma = b."""
    eps_in = np.asarray(eps_in, dtype=np.float64)
    ebar = 0.5 * (eps_in + eps_out)
    deps = eps_out - eps_in
    c = self_coefficient(area, curvature, self_scale)

    def matvec(sigma):
        sigma = np.asarray(sigma, dtype=np.float64)
        adl = direct("adl", xyz, xyz, sigma * area, trg_nrm=nrm)
        return ebar * sigma + deps * (adl + c * sigma) / FOUR_PI

    return matvec


def field(trg, src, q):
    """The raw field sum f_i = sum_j (r_i - r_j)/|r_i - r_j|^3 q_j, (3, n_trg): component
    k is the adjoint-double-layer sum with the constant target normal e_k (Eq. kernel_pol
    is the gradient kernel; dotted with e_k it is that component)."""
    trg = np.asarray(trg, dtype=np.float64)
    out = np.empty((3, trg.shape[1]))
    for k in range(3):
        e = np.zeros_like(trg)
        e[k] = 1.0
        out[k] = direct("adl", trg, src, q, trg_nrm=e)
    return out


def polarization_field(xyz, nrm, area, sigma, curvature, e0=(0.0, 0.0, 0.0), self_scale="disc"):
    """E^j at the elements (3, n) for total surface charge sigma (Eq. pol_discret with
    the self-patch term c_j sigma_j n_j) plus the applied field E0."""
    sigma = np.asarray(sigma, dtype=np.float64)
    c = self_coefficient(area, curvature, self_scale)
    E = (field(xyz, xyz, sigma * area) + c * sigma * np.asarray(nrm)) / FOUR_PI
    return E + np.asarray(e0, dtype=np.float64)[:, None]


def polarization_force(xyz, nrm, area, sigma, curvature, body, eps_out, e0=(0.0, 0.0, 0.0), self_scale="disc"):
    """Force on each body, (n_body, 3): F_b = sum_{j in b} eps_m sigma_j E^j a_j."""
    E = polarization_field(xyz, nrm, area, sigma, curvature, e0, self_scale)
    f = eps_out * sigma * area * E
    body = np.asarray(body)
    nb = int(body.max()) + 1
    return np.stack([np.bincount(body, weights=f[k], minlength=nb) for k in range(3)], axis=1)


def polarization_rhs(xyz, nrm, area, eps_in, eps_out, curvature, e0=(0.0, 0.0, 0.0), sigma_f=None,
                     self_scale="disc"):
    """b = (1 - ebar) sigma_f - deps (E_f . n)  (Eq. rhs): E_f the applied field plus the
    field of the free surface charge sigma_f (Eq. Ef without its volume term), at the
    elements as in Eq. pol_discret."""
    eps_in = np.asarray(eps_in, dtype=np.float64)
    ebar = 0.5 * (eps_in + eps_out)
    deps = eps_out - eps_in
    nrm = np.asarray(nrm, dtype=np.float64)
    sf = np.zeros(nrm.shape[1]) if sigma_f is None else np.asarray(sigma_f, dtype=np.float64)
    Ef = polarization_field(xyz, nrm, area, sf, curvature, e0, self_scale)
    return (1.0 - ebar) * sf - deps * (Ef * nrm).sum(axis=0)


def polarization_rhs_uniform_field(nrm, eps_in, eps_out, e0):
    """b = -deps (E0 . n): no free charge, the free-charge field replaced by E0."""
    deps = eps_out - np.asarray(eps_in, dtype=np.float64)
    e0 = np.asarray(e0, dtype=np.float64)
    return -deps * (e0[0] * nrm[0] + e0[1] * nrm[1] + e0[2] * nrm[2])


def polarization_solve(xyz, nrm, area, eps_in, eps_out, curvature, e0, tol=1e-6,
                       restart=50, max_iter=1000, self_scale="disc"):
    A = polarization_operator(xyz, nrm, area, eps_in, eps_out, curvature, self_scale)
    b = polarization_rhs_uniform_field(nrm, eps_in, eps_out, e0)
    return gmres(A, b, tol=tol, restart=restart, max_iter=max_iter)


def demag_phi2(xyz, nrm, w, phi1, omega):
    """phi_2 on the boundary from phi_1 (Eq. fk_integral_discrete)."""
    phi1 = np.asarray(phi1, dtype=np.float64)
    dl = direct("dl", xyz, xyz, phi1 * w, src_nrm=nrm)
    return dl / FOUR_PI + (np.asarray(omega) / FOUR_PI - 1.0) * phi1
