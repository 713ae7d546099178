"""Lumped (delta-gap) ports. Test infrastructure (oracle).

The paper excites structures through lumped ports (Sec. II, citing Wang 2004) without giving the
model. Reading: a port is a closed ring of mesh edges around a conductor's cross-section at
axial position z_p; a gap voltage V drives E_inc = V delta(z - z_p) zhat, so
  <f_m, E_inc> = s_m V l_m   for the ring edges (s_m = +1 if f_m crosses the edge along +z),
and the port current is the circulation of H around the ring (Ampere),
  I = sum_m s_m l_m h_m.
Units: with lengths in micrometres the first block row of the system is the SI row divided by
ell^2 (ell = 1e-6 m), so port_rhs(V = 1) is the excitation of a gap voltage eta0 * ell volts
(the RHS carries the 1/eta0 of the E_inc/eta0 row), port_current is the current in amperes
divided by ell, and the input impedance is Z = eta0 / port_current(V = 1) ohms.
"""
from __future__ import annotations

import numpy as np

from .rwg import RWG


def ring_edges(rw: RWG, obj, z, axis=2, tol=1e-9):
    """Edges of object `obj` lying in the plane x_axis = z, with crossing signs s_m."""
    va = rw.verts[rw.ev[:, 0], axis]
    vb = rw.verts[rw.ev[:, 1], axis]
    sel = np.nonzero((rw.obj_e == obj) & (np.abs(va - z) < tol) & (np.abs(vb - z) < tol))[0]
    # f_m points from T+ into T-: the sign is that of (centroid(T-) - centroid(T+)) along axis
    d = rw.centroid[rw.et[sel, 1], axis] - rw.centroid[rw.et[sel, 0], axis]
    return sel, np.sign(d)


def port_rhs(rw: RWG, edges, signs, V=1.0):
    b = np.zeros(rw.ne, dtype=np.complex128)
    b[edges] = signs * V * rw.elen[edges]
    return b


def port_current(rw: RWG, edges, signs, h):
    return np.sum(signs * rw.elen[edges] * h[edges])
