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
