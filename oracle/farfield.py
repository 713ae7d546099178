"""Radiated far field, monostatic RCS and the Mie series. Test infrastructure (oracle), FP64.

In the SLIM equivalent problem only J_Delta radiates into the background (Sec. II), so
  E_far(rhat) = -j k0 eta0 exp(-j k0 r)/(4 pi r) (I - rhat rhat) . int J_Delta exp(j k0 rhat.r') dS'
and the RCS is sigma = 4 pi r^2 |E_far|^2 / |E_0|^2. The paper validates with a copper sphere
against the Mie series (Sec. IV-A); the series is written here from Bohren and Huffman (1983),
with the logarithmic derivative D_n(mx) by downward recurrence (Wiscombe 1980).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

from .quad import radon7, rule_points
from .rwg import RWG


def radiation_vector(rw: RWG, j, k0, rhat):
    """N(rhat) = int J exp(j k0 rhat . r') dS' for J = sum_n j_n f_n (7-point rule)."""
    b, w = radon7()
    X = rw.verts[rw.tris]
    rq = rule_points(X, b)                                  # [nt, 7, 3]
    Jq = np.zeros(rq.shape, dtype=np.complex128)
    for i in range(3):
        n = rw.t_edges[:, i]
        v = rw.verts[rw.t_evert[:, i]]
        cf = rw.t_esign[:, i] * rw.elen[n] / (2 * rw.area) * j[n]
        Jq += cf[:, None, None] * (rq - v[:, None, :])
    out = []
    for rh in np.atleast_2d(rhat):
        ph = np.exp(1j * k0 * (rq @ rh))
        out.append(np.einsum("t,q,tq,tqd->d", rw.area, w, ph, Jq))
    return np.array(out)


def rcs(rw: RWG, j, k0, rhat):
    """sigma / ell^2 for a unit incident field, J scaled so that the RHS was <f, E_inc>
    (i.e. j = eta0 * J_Delta)."""
    N = radiation_vector(rw, j, k0, rhat)
    rh = np.atleast_2d(rhat)
    Nt = N - np.einsum("id,id->i", rh, N)[:, None] * rh
    return k0 ** 2 / (4 * math.pi) * np.sum(np.abs(Nt) ** 2, axis=1)


def mie_backscatter(x, m):
    """Backscattering cross-section / (pi a^2) of a sphere (size parameter x = k a, relative
    index m, Bohren-Huffman convention Im m >= 0)."""
    nmax = int(round(x + 4.0 * x ** (1.0 / 3.0) + 2.0))
    nstart = int(max(nmax, abs(m * x)) + 16)
    mx = m * x
    D = np.zeros(nstart + 1, dtype=np.complex128)
    for n in range(nstart, 0, -1):
        D[n - 1] = n / mx - 1.0 / (D[n] + n / mx)
    n = np.arange(0, nmax + 1)
    psi = x * special.spherical_jn(n, x)
    chi = -x * special.spherical_yn(n, x)
    xi = psi - 1j * chi
    s = 0.0 + 0.0j
    for k in range(1, nmax + 1):
        da = D[k] / m + k / x
        db = m * D[k] + k / x
        a = (da * psi[k] - psi[k - 1]) / (da * xi[k] - xi[k - 1])
        bq = (db * psi[k] - psi[k - 1]) / (db * xi[k] - xi[k - 1])
        s += (2 * k + 1) * (-1) ** k * (a - bq)
    return abs(s) ** 2 / x ** 2
