"""Pins of the oracle's near-pair integrals at large |k| (oracle/highk.py; Sec. II-B: the
specialised integration needed for highly conducting objects).

* The edge-integral form of the inner integrals against plain subdivision with the static part
  in closed form (points off the source plane, where that converges) and against direct polar
  integration about the observation point (points on the plane, inside the triangle): two
  computations that share none of the edge-integral algebra.
* The outer rule is a partition of T (its weights add up to T's area) and reduces to Radon's
  7-point rule where no subdivision is asked for.
* At the switch |k| diam = 0.5 the edge-integral scheme and the small-|k| singularity-subtraction
  scheme (two independent formulations) give the same pair moments to the accuracy of their
  outer rules.
* Convergence: the change of the pair moments under one more subdivision level and two more
  Gauss-Legendre points per interval, at |k| diam = 1.5, 5 and 36.
* P4, the Leontovich limit: inside a gold box at 1 THz (skin depth 79 nm, elements 0.5 um) the
  internal operator reproduces the surface-impedance relation n x E = Z_s n x (n x H),
  Z_s = (1 + j)/(sigma delta), on the rows away from the box's edges.
"""
import math

import numpy as np
import pytest

from oracle import highk, operators as op, quad
from oracle.rwg import from_mesh
from paper_2108_03991_gb300 import synth

TRI = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0], [0.3, 1.7, 0.0]])
NRM = np.array([0.0, 0.0, 1.0])
DIAM = max(np.linalg.norm(TRI[i] - TRI[(i + 1) % 3]) for i in range(3))


def _k(kd):
    """A good conductor's wavenumber (1 - j)|k|/sqrt(2) with |k| diam = kd."""
    return kd / DIAM * (1 - 1j) / math.sqrt(2)


def _subdivided(r, k, lev=8):
    """S0, S1, V at r by the static part in closed form plus the bounded remainder on 4^lev
    sub-triangles (7 points each)."""
    P, W = quad.radon7()
    for _ in range(lev):
        P, W = quad.subdivide4((P, W))
    area = 0.5 * np.linalg.norm(np.cross(TRI[1] - TRI[0], TRI[2] - TRI[0]))
    X = P @ TRI
    Rv = r - X
    R = np.linalg.norm(Rv, axis=1)
    I0, Irho, gI = quad.static_potentials(r[None], TRI[None], NRM[None])
    e = np.exp(-1j * k * R)
    g = (e - 1) / (4 * np.pi * R)
    d = np.dot(r - TRI[0], NRM)
    rho = r - d * NRM
    S0 = I0[0] / (4 * np.pi) + area * np.sum(W * g)
    S1 = (Irho[0] + rho * I0[0]) / (4 * np.pi) + area * np.einsum("q,qd,q->d", W, X, g)
    gd = (1 - (1 + 1j * k * R) * e) / (4 * np.pi * R ** 3)
    V = gI[0] / (4 * np.pi) + area * np.einsum("q,qd,q->d", W, Rv, gd)
    return S0, S1, V


@pytest.mark.parametrize("kd", [0.6, 1.5, 5.0, 36.0])
def test_inner_off_plane_matches_subdivision(kd):
    k = _k(kd)
    pts = np.array([[0.7, 0.5, 0.05], [0.7, 0.5, -0.3], [2.2, 0.3, 0.1], [1.0, 0.0, 0.02],
                    [-0.5, -0.5, 0.4], [0.15, 0.85, 0.01], [1.2, 0.9, -0.08]])
    S0, S1, V = highk.inner(pts, TRI, NRM, DIAM, k)
    for i, r in enumerate(pts):
        b0, b1, bv = _subdivided(r, k)
        # the edge rule is accurate to a few 1e-9 of the largest values; far from S at large
        # |k| the values are exponentially small and the rule's cut-off (exp(-18) of the peak)
        # and the O(0.1) static parts' rounding set an absolute floor
        assert abs(S0[i] - b0) <= 1e-8 * abs(b0) + 1e-10
        assert np.linalg.norm(S1[i] - b1) <= 1e-8 * np.linalg.norm(b1) + 1e-10
        # V's remainder keeps an R^-3 part where |k| R >> 1 (the static subtraction no longer
        # cancels it), so the subdivision is the less accurate side there
        assert np.linalg.norm(V[i] - bv) <= 3e-8 * np.linalg.norm(bv) + 1e-10


def _polar(rho, k, nseg=64, ng=16):
    """S0 and S1 at an in-plane point inside TRI by integrating over the polar angle about it,
    the radial integrals in closed form: int_0^R exp(-jku) du and int_0^R u exp(-jku) du."""
    x, w = np.polynomial.legendre.leggauss(ng)
    ang = []
    for v in TRI:
        dv = v - rho
        ang.append(math.atan2(dv[1], dv[0]))
    ang = np.sort(np.mod(ang, 2 * np.pi))
    ang = np.append(ang, ang[0] + 2 * np.pi)
    S0 = 0j
    S1 = np.zeros(3, complex)
    for a0, a1 in zip(ang[:-1], ang[1:]):
        edges = np.linspace(a0, a1, nseg + 1)
        for p0, p1 in zip(edges[:-1], edges[1:]):
            phi = 0.5 * (p0 + p1) + 0.5 * (p1 - p0) * x
            wt = 0.5 * (p1 - p0) * w
            for f, wf in zip(phi, wt):
                u = np.array([math.cos(f), math.sin(f), 0.0])
                # distance to the boundary along u
                R = np.inf
                for i in range(3):
                    pa, pb = TRI[i], TRI[(i + 1) % 3]
                    e = pb - pa
                    den = u[0] * e[1] - u[1] * e[0]
                    if abs(den) < 1e-300:
                        continue
                    s = ((pa - rho)[0] * e[1] - (pa - rho)[1] * e[0]) / den
                    t = ((pa - rho)[0] * u[1] - (pa - rho)[1] * u[0]) / den
                    if s > 0 and -1e-12 <= t <= 1 + 1e-12:
                        R = min(R, s)
                E = np.exp(-1j * k * R)
                S0 += wf * (1 - E) / (1j * k)
                S1 += wf * u * (E * (1 + 1j * k * R) - 1) / (k * k)
    return S0 / (4 * np.pi), rho * S0 / (4 * np.pi) + S1 / (4 * np.pi)


@pytest.mark.parametrize("kd", [1.5, 5.0, 36.0])
def test_inner_in_plane_matches_polar(kd):
    k = _k(kd)
    pts = np.array([[0.7, 0.5, 0.0], [1.0, 0.01, 0.0], [0.2, 0.85, 0.0], [1.6, 0.3, 0.0]])
    S0, S1, _ = highk.inner(pts, TRI, NRM, DIAM, k)
    for i, r in enumerate(pts):
        b0, b1 = _polar(r, k)
        assert abs(S0[i] - b0) <= 1e-8 * abs(b0)
        assert np.linalg.norm(S1[i] - b1) <= 1e-8 * np.linalg.norm(b1)


def test_outer_rule_partitions_the_triangle():
    T = np.array([[2.0, 0, 0], [2.0, 2.0, 0], [0, 2.0, 0]])
    area = 2.0
    for kd in (0.8, 5.0, 36.0):
        p, w = highk.leaves(T, TRI, NRM, DIAM, _k(kd))
        assert abs(w.sum() - area) <= 1e-14 * area
    p, w = highk.leaves(T, TRI, NRM, DIAM, _k(0.8))  # |k| diam_T < 1: depth 0
    b, wr = quad.radon7()
    assert np.allclose(p, b @ T, rtol=0, atol=1e-15) and np.allclose(w, wr * area)


PAIRS = {"self": np.array([[0.0, 0, 0], [2.0, 0, 0], [0.0, 2.0, 0]]),
         "edge_coplanar": np.array([[2.0, 0, 0], [2.0, 2.0, 0], [0, 2.0, 0]]),
         "edge_90": np.array([[0.0, 0, 0], [0, 0, -2.0], [2.0, 0, 0]]),
         "edge_7deg": np.array([[2.0, 0, 0], [0, 0, 0], [1.0, -2 * math.cos(0.1257), -2 * math.sin(0.1257)]]),
         "vertex": np.array([[2.0, 0, 0], [4.0, 0, 0], [2.0, -2.0, 0]])}
SRC = PAIRS["self"]
SDIAM = 2 * math.sqrt(2)


def _moments(T, kd, depth=0, ngl=highk.NGL):
    highk.set_refinement(depth, ngl)
    try:
        return highk.pair_moments(T, SRC, NRM, SDIAM, kd / SDIAM * (1 - 1j) / math.sqrt(2))
    finally:
        highk.set_refinement(0, highk.NGL)


def _change(m, mr, kabs):
    """(L-type change relative to the largest L-type moment, K-type change relative to |k| |M0|)."""
    sL = max(np.abs(mr[q]).max() for q in ("M0", "M1", "M1p", "M2"))
    eL = max(np.abs(m[q] - mr[q]).max() for q in ("M0", "M1", "M1p", "M2")) / sL
    eK = max(np.abs(m[q] - mr[q]).max() for q in ("Vs", "U")) / (kabs * abs(mr["M0"]))
    return eL, eK


def test_schemes_agree_at_the_switch():
    """|k| diam just above 0.5, where neither rule subdivides T (Radon's 7 points on T for both):
    the edge-integral inner integrals against the small-|k| ones (static part in closed form,
    4 x 7-point remainder) give the same pair moments, for every pair kind, to the accuracy of
    the small-|k| remainder rule."""
    from oracle import operators as o
    kd = 0.55
    k = kd / SDIAM * (1 - 1j) / math.sqrt(2)
    for name, T in PAIRS.items():
        c = T.mean(axis=0)  # tri_pair_moments measures positions from the testing centroid
        mh = highk.pair_moments(T - c, SRC - c, NRM, SDIAM, k)
        verts = np.concatenate([T, SRC])
        tris = np.array([[0, 1, 2], [3, 4, 5]], dtype=np.int32)
        # a two-triangle "mesh" holding just the pair, for the small-|k| rule of operators.py
        rw = _pair_rwg(verts, tris)
        highk_before = highk.HIGHK
        highk.HIGHK = 1e9  # force the small-|k| rule
        try:
            ml = o.tri_pair_moments(rw, k, [0], [1])
        finally:
            highk.HIGHK = highk_before
        ml = {q: v[0] for q, v in ml.items()}
        eL, eK = _change(ml, mh, kd / SDIAM)
        assert eL < 3e-5 and eK < 5e-4, (name, eL, eK)


def _pair_rwg(verts, tris):
    """Only the fields tri_pair_moments reads, for two triangles."""
    class R:
        pass
    r = R()
    r.verts = verts
    r.tris = tris
    X = verts[tris]
    n = np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0])
    r.area = 0.5 * np.linalg.norm(n, axis=1)
    r.normal = n / np.linalg.norm(n, axis=1)[:, None]
    r.centroid = X.mean(axis=1)
    r.diam = np.max(np.stack([np.linalg.norm(X[:, 1] - X[:, 0], axis=1),
                              np.linalg.norm(X[:, 2] - X[:, 1], axis=1),
                              np.linalg.norm(X[:, 0] - X[:, 2], axis=1)]), axis=0)
    return r


# measured change of the pair moments under one more level and two more GL points (L-type,
# K-type); the assertion guards against a regression of the rule's convergence
REFINE_BOUND = {1.5: (5e-3, 1.5e-1), 5.0: (5e-3, 8e-2), 36.0: (2e-2, 2e-1)}


@pytest.mark.parametrize("kd", [1.5, 5.0, 36.0])
def test_refinement_change(kd):
    out = {}
    for name, T in PAIRS.items():
        m = _moments(T, kd)
        mr = _moments(T, kd, depth=1, ngl=highk.NGL + 2)
        out[name] = _change(m, mr, kd / SDIAM)
    print(f"|k| diam = {kd}: " + ", ".join(f"{n} L {a:.1e} K {b:.1e}" for n, (a, b) in out.items()))
    bL, bK = REFINE_BOUND[kd]
    for name, (eL, eK) in out.items():
        assert eL < bL and eK < bK, (name, eL, eK)


def test_leontovich_limit():
    """P4: gold box 2 x 2 x 2 um at 1 THz (|k_i| times the element diameter = 12.7). For the
    tangential field of a uniform H, Galerkin-tested n x E from the internal operator,
    G Zhat h, equals the surface-impedance value -(Z_s/eta0) I_x h on every row whose two
    triangles keep a full element away from the box's edges, within 2%; on all rows the corners
    (where the surface-impedance relation does not hold) make it about 10%."""
    f = 1e12
    rw = from_mesh(synth.bar_mesh(2.0, 2.0, 2.0, 0.5, sigma=synth.SIGMA_AU))
    k0 = op.k0_of(f)
    epsc = op.eps_rc(synth.SIGMA_AU, f)
    k = op.k_medium(k0, epsc)
    ix = op.ix_matrix(rw).toarray()
    G = op.gram_matrix(rw).toarray()
    Zhat = -np.linalg.solve(op.dense_rwg(rw, k, "L"), op.dense_rwg(rw, k, "K") + 0.5 * ix) \
        / (1j * k0 * epsc)
    zs = 1.0 / np.sqrt(epsc)  # Z_s / eta0 = sqrt(mu0 / eps_c) / eta0
    assert abs(zs - (1 + 1j) / (synth.SIGMA_AU * math.sqrt(2 / (2 * math.pi * f * op.MU0 *
                                                                   synth.SIGMA_AU)) * op.ETA0)) \
        < 1e-3 * abs(zs)
    V = rw.verts
    lo, hi = V.min(0), V.max(0)
    on_edge = (np.isclose(V, lo) | np.isclose(V, hi)).sum(1) >= 2
    rows = np.nonzero(~on_edge[rw.tris].any(1)[rw.et].any(1))[0]
    assert rows.size == 48
    b, _ = quad.radon7()
    nr = np.repeat(rw.normal[:, None, :], 7, axis=1).reshape(-1, 3)
    for H in (np.array([0, 1.0, 0]), np.array([1.0, 0, 0]), np.array([0.6, 0, 0.8])):
        h = np.linalg.solve(G, op.project_tangential(rw, lambda r: np.cross(nr, np.broadcast_to(H, r.shape))))
        lhs = G @ (Zhat @ h)
        rhs = -zs * (ix @ h)
        assert np.linalg.norm((lhs - rhs)[rows]) < 0.02 * np.linalg.norm(rhs[rows])
        assert np.linalg.norm(lhs - rhs) < 0.2 * np.linalg.norm(rhs)
