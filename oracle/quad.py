"""Triangle quadrature rules and closed-form potential integrals over a flat triangle.

Test infrastructure (oracle). The paper delegates the integration of the Galerkin entries to
the literature (Sec. II-A: "entries ... computed through numeric integration"; Sec. II-B:
"specialized integration routines are needed when conductivity is high"). The project's
reading, used identically by the oracle and the CUDA setup (written twice, independently):

* outer (testing) integrals: the 7-point degree-5 rule of Radon;
* inner (source) integrals of well-separated triangle pairs: the same 7-point rule;
* inner integrals of near pairs (centroid distance below NEAR_FACTOR times the larger
  triangle diameter): the static 1/R parts of G and grad G in closed form, plus the 7-point
  rule on each of the four midpoint sub-triangles for the bounded remainder.

The closed forms are the classical potential integrals of a uniform and a linear density
over a flat triangle (Wilton et al. 1984; Graglia 1993), restated here from their derivation
through the surface divergence theorem.
"""
from __future__ import annotations

import math

import numpy as np

NEAR_FACTOR = 2.1


def radon7():
    """Radon's symmetric 7-point rule, exact for polynomials of total degree 5.

    Returns barycentric points [7, 3] and weights [7] that sum to one (multiply by the area).
    """
    s = math.sqrt(15.0)
    a1 = (6.0 - s) / 21.0
    a2 = (6.0 + s) / 21.0
    w1 = (155.0 - s) / 1200.0
    w2 = (155.0 + s) / 1200.0
    pts = [(1 / 3, 1 / 3, 1 / 3),
           (a1, a1, 1 - 2 * a1), (a1, 1 - 2 * a1, a1), (1 - 2 * a1, a1, a1),
           (a2, a2, 1 - 2 * a2), (a2, 1 - 2 * a2, a2), (1 - 2 * a2, a2, a2)]
    w = [9.0 / 40.0, w1, w1, w1, w2, w2, w2]
    return np.array(pts, dtype=np.float64), np.array(w, dtype=np.float64)


def gauss_tri(nu, nv=None):
    """Collapsed Gauss-Legendre product rule (Duffy map) with nu x nv points.

    Exact for total degree min(2*nu - 2, 2*nv - 1). Barycentric points and unit-sum weights.
    """
    nv = nu if nv is None else nv
    xu, wu = np.polynomial.legendre.leggauss(nu)
    xv, wv = np.polynomial.legendre.leggauss(nv)
    u = 0.5 * (xu + 1.0)
    v = 0.5 * (xv + 1.0)
    wu = 0.5 * wu
    wv = 0.5 * wv
    U, Vv = np.meshgrid(u, v, indexing="ij")
    WU, WV = np.meshgrid(wu, wv, indexing="ij")
    l1 = U.ravel()
    l2 = (Vv * (1.0 - U)).ravel()
    w = (2.0 * WU * WV * (1.0 - U)).ravel()
    return np.stack([l1, l2, 1.0 - l1 - l2], axis=1), w


def subdivide4(rule):
    """Apply a rule on each of the four midpoint sub-triangles (weights scaled by 1/4)."""
    pts, w = rule
    c = np.eye(3)
    m01, m12, m20 = (c[0] + c[1]) / 2, (c[1] + c[2]) / 2, (c[2] + c[0]) / 2
    subs = [(c[0], m01, m20), (m01, c[1], m12), (m20, m12, c[2]), (m01, m12, m20)]
    P, W = [], []
    for (A, B, C) in subs:
        P.append(pts[:, :1] * A + pts[:, 1:2] * B + pts[:, 2:3] * C)
        W.append(w / 4.0)
    return np.concatenate(P), np.concatenate(W)


def rule_points(tri_xyz, bary):
    """Physical points of a rule on triangles: tri_xyz [..., 3, 3] -> [..., nq, 3]."""
    return np.einsum("qk,...kd->...qd", bary, tri_xyz)


def monomial_integral(area, a, b, c):
    """Exact integral of l1^a l2^b l3^c over a triangle of the given area (barycentric l)."""
    return 2.0 * area * math.factorial(a) * math.factorial(b) * math.factorial(c) / \
        math.factorial(a + b + c + 2)


def static_potentials(r, tri, nrm, area_scale=None):
    """Closed-form integrals over flat triangles, observation points r.

    r    [M, 3] observation points
    tri  [M, 3, 3] vertices (counter-clockwise about nrm)
    nrm  [M, 3] unit normals
    Returns, per point,
      I0    = int_T 1/R dS'
      Irho  = int_T (rho' - rho)/R dS'   (rho = projection of r on the plane; in-plane vector)
      gI    = grad_r int_T 1/R dS' = -int_T (r - r')/R^3 dS'
    The solid-angle (normal) part of gI is dropped when |d| <= 1e-10 * diameter: that is the
    principal value on the triangle's own plane.
    """
    r = np.asarray(r, dtype=np.float64)
    p0 = tri[:, 0, :]
    d = np.einsum("md,md->m", r - p0, nrm)
    rho = r - d[:, None] * nrm
    ad = np.abs(d)
    diam = np.max(np.stack([np.linalg.norm(tri[:, 1] - tri[:, 0], axis=1),
                            np.linalg.norm(tri[:, 2] - tri[:, 1], axis=1),
                            np.linalg.norm(tri[:, 0] - tri[:, 2], axis=1)]), axis=0)
    sgn = np.where(ad <= 1e-10 * diam, 0.0, np.sign(d))
    ad = np.where(ad <= 1e-10 * diam, 0.0, ad)
    I0 = np.zeros(r.shape[0])
    Irho = np.zeros_like(r)
    gI = np.zeros_like(r)
    omega = np.zeros(r.shape[0])
    for i in range(3):
        pa = tri[:, i, :]
        pb = tri[:, (i + 1) % 3, :]
        lv = pb - pa
        lhat = lv / np.linalg.norm(lv, axis=1)[:, None]
        uhat = np.cross(lhat, nrm)
        lp = np.einsum("md,md->m", pb - rho, lhat)
        lm = np.einsum("md,md->m", pa - rho, lhat)
        P0 = np.einsum("md,md->m", pa - rho, uhat)
        R0sq = P0 * P0 + ad * ad
        Rp = np.sqrt(lp * lp + R0sq)
        Rm = np.sqrt(lm * lm + R0sq)
        pos = (lp + lm) >= 0.0
        with np.errstate(divide="ignore", invalid="ignore"):
            f = np.where(pos, np.log((Rp + lp) / (Rm + lm)), np.log((Rm - lm) / (Rp - lp)))
            dp = R0sq + ad * Rp
            dm = R0sq + ad * Rm
            bp = np.where(dp > 0, np.arctan(P0 * lp / np.where(dp > 0, dp, 1.0)), 0.0)
            bm = np.where(dm > 0, np.arctan(P0 * lm / np.where(dm > 0, dm, 1.0)), 0.0)
        f = np.where(np.abs(P0) == 0.0, np.where(np.isfinite(f), f, 0.0), f)
        I0 += P0 * f
        omega += bp - bm
        Irho += 0.5 * uhat * (R0sq * f + lp * Rp - lm * Rm)[:, None]
        gI -= uhat * f[:, None]
    I0 -= ad * omega
    gI -= (sgn * omega)[:, None] * nrm
    return I0, Irho, gI
