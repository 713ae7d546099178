"""Near-pair integrals of G(k) for a large |k| (lossy conductors). Test infrastructure (oracle).

Sec. II-B notes that specialised integration routines are needed when the conductivity is high,
without naming them. Inside a good conductor G(k_i, R) = exp(-j k_i R)/(4 pi R) decays over a
skin depth, far below the element size, so the static-part subtraction used for near pairs at
small |k| (oracle/quad.py) no longer works: G is negligible where 1/R is not. The reading
taken here (used alike by the oracle and the CUDA set-up, written independently):

Inner (source) integrals at an observation point r over a flat triangle S (normal n, vertices
CCW about n). With d = (r - v0).n, a = |d| and rho = r - d n, the fan of S about rho splits
every surface integral into three edge terms; along edge e (unit direction l_e, outward in-plane
normal u_e = l_e x n, signed distance P_e = (v_a - rho).u_e, foot parameters l- and l+,
R_e(t) = sqrt(P_e^2 + t^2 + a^2)) the radial integral of every kernel below has a closed form,
and what remains are one-dimensional edge integrals:
    int_S G dS'             = [Omega exp(-j k a) - sum_e J1_e] / (4 pi j k)
    int_S (r' - rho) G dS'  = -sum_e u_e J2_e / (4 pi j k)              (gradient theorem)
    int_S grad_r G dS'      = -[sum_e u_e J3_e + n (sgn(d) Omega exp(-j k a) - d sum_e J4_e)] / (4 pi)
with J1 = int P exp(-jkR)/(P^2+t^2) dt, J2 = int exp(-jkR) dt, J3 = int exp(-jkR)/R dt,
J4 = int P exp(-jkR)/((P^2+t^2) R) dt over [l-, l+], and Omega = sum_e [atan(l+/P) - atan(l-/P)]
the plane angle that S subtends at rho (2 pi inside, 0 outside). On S's own plane the normal
term is the principal value (dropped, as in the small-|k| rule). An edge whose line passes
through rho (|P| <= 1e-12 diam) has J1 = J4 = 0 and no angle: the limits from both sides agree.

The edge integrals use a graded Gauss-Legendre rule (6 points per interval) in |t|, the
integrands being even in t: breakpoints at h0 2^j up to the first one above 2 dmax, then steps
of dmax, with h0 = min(|P| (w if P = 0), 1/|k|)/2, dmax = 6/|k| and w = sqrt(P^2 + a^2); the
rule stops where |Im k| (R - w) exceeds 18 (exp(-18) ~ 2e-8 of the peak) and skips an edge
whose |Im k| (w - a) exceeds 18. The edge integrals are then accurate to a few 1e-9, far below
the outer rule's own error (about 1e-3 at |k| diam = 36, see the refinement study).

Outer (testing) integrals: T is split into four midpoint sub-triangles, recursively, wherever
a sub-triangle lies close to where the inner integrals vary fast, down to depth
D = min(3, ceil(log2(|k| diam_T))); every leaf takes Radon's 7-point rule. "Where they vary
fast" is the boundary of S when T lies in S's plane, and S itself otherwise. The split test,
with c the sub-triangle's centroid, rad its circumradius about c and dm its diameter: the
distance from c to that set is below rad + dm/4, and (for a lossy medium) the sub-triangle's
nearest point lies within 12/|Im k| of it (farther on, the integrand is below exp(-12) of its
peak and the leaf's 7 points take it as it is).

Pairs use this scheme when they are near (the small-|k| criterion: centroid distance below
2.1 times the larger diameter) and |k| max(diam_t, diam_s) > 0.5; a near pair whose testing
triangle lies wholly farther than 18/|Im k| from the source (T's centroid distance to S minus
T's circumradius) takes the regular 7 x 7 rule, its values being below exp(-18) of the
touching pairs'.
"""
from __future__ import annotations

import math

import numpy as np

from .quad import radon7

HIGHK = 0.5
DECAY = 18.0
NGL = 6
DEPTH_MAX = 3
P_ZERO = 1e-12
# refinement controls for the convergence study (0 = the rule above): extra subdivision levels
# and extra Gauss-Legendre points per interval
REFINE_DEPTH = 0
SPLIT_MARGIN = 0.25
SPLIT_DECAY = 12.0
DMAX_FACTOR = 6.0


def _gl01(n=NGL):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


_GX, _GW = _gl01()


def _breakpoints(s_a, s_e, h0, dmax):
    """Breakpoints [M, K] of the graded rule on [s_a, s_e] (rows padded with s_e)."""
    M = s_a.size
    # doubling points h0 2^j while h0 2^j <= 2 dmax
    jmax = int(np.max(np.floor(np.log2(2.0 * dmax / h0)))) + 2
    D = h0[:, None] * (2.0 ** np.arange(jmax))[None, :]
    ok = D <= 2.0 * dmax
    D = np.where(ok, D, np.inf)
    last = np.max(np.where(ok, D, 0.0), axis=1)
    nlin = int(np.max(np.ceil(np.maximum(s_e - last, 0.0) / dmax))) + 1
    Lin = last[:, None] + dmax * np.arange(1, nlin + 1)[None, :]
    G = np.concatenate([D, Lin], axis=1)
    G = np.where(G <= s_a[:, None], s_a[:, None], G)
    G = np.where(G >= s_e[:, None], s_e[:, None], G)
    B = np.concatenate([s_a[:, None], G, s_e[:, None]], axis=1)
    B = np.sort(B, axis=1)
    # drop columns that are zero-length in every row
    keep = np.concatenate([[True], np.any(np.diff(B, axis=1) > 0, axis=0)])
    return B[:, keep] if M else B


def _edge_integrals(P, a, pieces, k, h0, dmax, cut):
    """J1..J4 for one edge at M points; pieces: list of (s_a, s_b) arrays (|t| ranges)."""
    M = P.size
    w2 = P * P + a * a
    J = [np.zeros(M, complex) for _ in range(4)]
    for s_a, s_b in pieces:
        s_e = np.minimum(s_b, cut)
        act = s_e > s_a
        if not np.any(act):
            continue
        idx = np.nonzero(act)[0]
        B = _breakpoints(s_a[idx], s_e[idx], h0[idx], dmax)
        lo, hi = B[:, :-1], B[:, 1:]
        L = hi - lo
        t = lo[:, :, None] + L[:, :, None] * _GX[None, None, :]
        wt = L[:, :, None] * _GW[None, None, :]
        R = np.sqrt(w2[idx][:, None, None] + t * t)
        E = np.exp(-1j * k * R)
        Pi = P[idx][:, None, None]
        lor = Pi / (Pi * Pi + t * t)
        J[0][idx] += np.sum(wt * lor * E, axis=(1, 2))
        J[1][idx] += np.sum(wt * E, axis=(1, 2))
        J[2][idx] += np.sum(wt * E / R, axis=(1, 2))
        J[3][idx] += np.sum(wt * lor * E / R, axis=(1, 2))
    return J


def inner(r, tri, nrm, diam, k):
    """Inner integrals at observation points r [M, 3] over source triangles tri ([3, 3], or
    [M, 3, 3] with nrm [M, 3] and diam [M], one per point): S0 = int G, S1 = int r' G
    (vector), V = int grad_r G (vector)."""
    r = np.atleast_2d(np.asarray(r, dtype=np.float64))
    M = r.shape[0]
    tri = np.broadcast_to(np.asarray(tri, dtype=np.float64), (M, 3, 3))
    nrm = np.broadcast_to(np.asarray(nrm, dtype=np.float64), (M, 3))
    diam = np.broadcast_to(np.asarray(diam, dtype=np.float64), (M,))
    k = complex(k)
    kabs = abs(k)
    kim = abs(k.imag)
    x = 1.0 / kabs
    dmax = DMAX_FACTOR * x
    d = np.einsum("md,md->m", r - tri[:, 0], nrm)
    a = np.abs(d)
    coplanar = a <= 1e-10 * diam
    a = np.where(coplanar, 0.0, a)
    sg = np.where(coplanar, 0.0, np.sign(d))
    rho = r - d[:, None] * nrm
    Om = np.zeros(M)
    SJ1 = np.zeros(M, complex)
    SJ4 = np.zeros(M, complex)
    SJ2 = np.zeros((M, 3), complex)
    SJ3 = np.zeros((M, 3), complex)
    for i in range(3):
        pa, pb = tri[:, i], tri[:, (i + 1) % 3]
        le = pb - pa
        lh = le / np.linalg.norm(le, axis=1)[:, None]
        uh = np.cross(lh, nrm)
        P = np.einsum("md,md->m", pa - rho, uh)
        lm = np.einsum("md,md->m", pa - rho, lh)
        lp = np.einsum("md,md->m", pb - rho, lh)
        pz = np.abs(P) <= P_ZERO * diam
        P = np.where(pz, 0.0, P)
        w = np.maximum(np.sqrt(P * P + a * a), P_ZERO * diam)
        with np.errstate(divide="ignore", invalid="ignore"):
            th = np.where(pz, 0.0, np.arctan(lp / P) - np.arctan(lm / P))
        Om += th
        skip = kim * (w - a) > DECAY if kim > 0 else np.zeros(M, bool)
        if np.all(skip):
            continue
        h0 = 0.5 * np.minimum(np.where(pz, w, np.abs(P)), x)
        cut = np.sqrt(DECAY / kim * (2.0 * w + DECAY / kim)) if kim > 0 else np.full(M, np.inf)
        # |t| pieces of [lm, lp] (the integrands are even in t)
        both = (lm < 0) & (lp > 0)
        s1a = np.where(both, 0.0, np.minimum(np.abs(lm), np.abs(lp)))
        s1b = np.where(both, -lm, np.maximum(np.abs(lm), np.abs(lp)))
        s2a = np.zeros(M)
        s2b = np.where(both, lp, 0.0)
        pieces = [(s1a, s1b), (s2a, s2b)]
        act = ~skip
        J = _edge_integrals(P[act], a[act], [(p[act], q[act]) for p, q in pieces], k, h0[act],
                            dmax, cut[act])
        SJ1[act] += J[0]
        SJ2[act] += J[1][:, None] * uh[act]
        SJ3[act] += J[2][:, None] * uh[act]
        SJ4[act] += J[3]
    ea = np.exp(-1j * k * a)
    f4 = 4.0 * math.pi
    S0 = (Om * ea - SJ1) / (f4 * 1j * k)
    S1 = rho * S0[:, None] - SJ2 / (f4 * 1j * k)
    V = -(SJ3 + nrm * (sg * Om * ea - d * SJ4)[:, None]) / f4
    return S0, S1, V


def _sub3(a, b):
    return (a[0] - b[0], a[1] - b[1], a[2] - b[2])


def _dot3(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def _cross3(a, b):
    return (a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0])


def _seg_dist(c, p, q):
    v = _sub3(q, p)
    t = min(max(_dot3(_sub3(c, p), v) / _dot3(v, v), 0.0), 1.0)
    e = (c[0] - (p[0] + t * v[0]), c[1] - (p[1] + t * v[1]), c[2] - (p[2] + t * v[2]))
    return math.sqrt(_dot3(e, e))


def _tri_dist(c, tri, nrm):
    """Distance from the point c to the filled triangle tri (unit normal nrm)."""
    c = tuple(float(v) for v in c)
    tri = [tuple(float(v) for v in row) for row in tri]
    nrm = tuple(float(v) for v in nrm)
    d = _dot3(_sub3(c, tri[0]), nrm)
    rho = (c[0] - d * nrm[0], c[1] - d * nrm[1], c[2] - d * nrm[2])
    inside = True
    for i in range(3):
        pa, pb = tri[i], tri[(i + 1) % 3]
        if _dot3(_cross3(_sub3(pb, pa), _sub3(rho, pa)), nrm) < 0:
            inside = False
    if inside:
        return abs(d)
    return min(_seg_dist(c, tri[i], tri[(i + 1) % 3]) for i in range(3))


def _mid(a, b):
    return (0.5 * (a[0] + b[0]), 0.5 * (a[1] + b[1]), 0.5 * (a[2] + b[2]))


def _sub4(t):
    v0, v1, v2 = t
    m01, m12, m20 = _mid(v0, v1), _mid(v1, v2), _mid(v2, v0)
    return [(v0, m01, m20), (m01, v1, m12), (m20, m12, v2), (m01, m12, m20)]


def coplanar(T, S, nS, diamS):
    nT = np.cross(T[1] - T[0], T[2] - T[0])
    nT = nT / np.linalg.norm(nT)
    cT = T.mean(axis=0)
    return abs(np.dot(nT, nS)) >= 1.0 - 1e-12 and abs(np.dot(cT - S[0], nS)) <= 1e-10 * diamS


def depth_of(k, diamT):
    q = abs(k) * diamT
    return int(min(DEPTH_MAX, max(0, math.ceil(math.log2(q))))) + REFINE_DEPTH if q > 1.0 \
        else REFINE_DEPTH


def set_refinement(depth=0, ngl=NGL):
    """Refined variants of the rule for the convergence study (depth levels and GL points)."""
    global REFINE_DEPTH, _GX, _GW
    REFINE_DEPTH = depth
    _GX, _GW = _gl01(ngl)


def leaves(T, S, nS, diamS, k):
    """Outer rule on T for the source S: points [M, 3] and weights [M] (area included)."""
    diamT = max(np.linalg.norm(T[1] - T[0]), np.linalg.norm(T[2] - T[1]), np.linalg.norm(T[0] - T[2]))
    D = depth_of(k, diamT)
    cop = coplanar(T, S, nS, diamS)
    bary, wr = radon7()
    Sl = [tuple(float(v) for v in row) for row in S]
    nSl = tuple(float(v) for v in nS)
    kim = abs(complex(k).imag)
    out = []

    def dist(c):
        if cop:
            return min(_seg_dist(c, Sl[i], Sl[(i + 1) % 3]) for i in range(3))
        return _tri_dist(c, Sl, nSl)

    def rec(t, lev):
        c = ((t[0][0] + t[1][0] + t[2][0]) / 3.0, (t[0][1] + t[1][1] + t[2][1]) / 3.0,
             (t[0][2] + t[1][2] + t[2][2]) / 3.0)
        if lev < D:
            rad = max(math.sqrt(_dot3(_sub3(t[j], c), _sub3(t[j], c))) for j in range(3))
            dm = max(math.sqrt(_dot3(_sub3(t[1], t[0]), _sub3(t[1], t[0]))),
                     math.sqrt(_dot3(_sub3(t[2], t[1]), _sub3(t[2], t[1]))),
                     math.sqrt(_dot3(_sub3(t[0], t[2]), _sub3(t[0], t[2]))))
            dc = dist(c)
            if dc < rad + SPLIT_MARGIN * dm and (kim == 0.0 or kim * (dc - rad) < SPLIT_DECAY):
                for ch in _sub4(t):
                    rec(ch, lev + 1)
                return
        out.append(t)

    rec(tuple(tuple(float(v) for v in row) for row in T), 0)
    L = np.array(out, dtype=np.float64)                       # [nleaf, 3, 3]
    area = 0.5 * np.linalg.norm(np.cross(L[:, 1] - L[:, 0], L[:, 2] - L[:, 0]), axis=1)
    pts = np.einsum("qk,lkd->lqd", bary, L).reshape(-1, 3)
    wts = (wr[None, :] * area[:, None]).ravel()
    return pts, wts


def pair_moments(T, S, nS, diamS, k, want_K=True):
    """Moments of G(k) over the pair (T testing, S source) with the rules above:
    M0 = int int G, M1 = int int r G, M1p = int int r' G, M2 = int int r.r' G,
    Vs = int_T V, U = int_T V x r with V(r) = int_S grad_r G."""
    rp, wp = leaves(T, S, nS, diamS, k)
    S0, S1, V = inner(rp, S, nS, diamS, k)
    out = {"M0": np.sum(wp * S0), "M1": np.einsum("p,pd,p->d", wp, rp, S0),
           "M1p": np.einsum("p,pd->d", wp, S1), "M2": np.einsum("p,pd,pd->", wp, rp, S1)}
    if want_K:
        out["Vs"] = np.einsum("p,pd->d", wp, V)
        out["U"] = np.einsum("p,pd->d", wp, np.cross(V, rp))
    return out


def pair_moments_batch(Ts, Ss, nSs, diamSs, k, want_K=True, chunk=20000):
    """pair_moments for many pairs at once (Ts, Ss [npair, 3, 3], nSs [npair, 3], diamSs
    [npair]); returns a dict of arrays like operators.tri_pair_moments."""
    npair = len(Ts)
    pts, wts, own = [], [], []
    for i in range(npair):
        p, w = leaves(Ts[i], Ss[i], nSs[i], diamSs[i], k)
        pts.append(p)
        wts.append(w)
        own.append(np.full(w.size, i))
    rp = np.concatenate(pts)
    wp = np.concatenate(wts)
    own = np.concatenate(own)
    out = {"M0": np.zeros(npair, complex), "M2": np.zeros(npair, complex)}
    for key in ("M1", "M1p", "Vs", "U"):
        out[key] = np.zeros((npair, 3), complex)
    for c0 in range(0, rp.shape[0], chunk):
        sl = slice(c0, c0 + chunk)
        o = own[sl]
        S0, S1, V = inner(rp[sl], Ss[o], nSs[o], diamSs[o], k)
        w = wp[sl]
        r = rp[sl]
        np.add.at(out["M0"], o, w * S0)
        np.add.at(out["M1"], o, (w * S0)[:, None] * r)
        np.add.at(out["M1p"], o, w[:, None] * S1)
        np.add.at(out["M2"], o, w * np.einsum("pd,pd->p", r, S1))
        if want_K:
            np.add.at(out["Vs"], o, w[:, None] * V)
            np.add.at(out["U"], o, w[:, None] * np.cross(V, r))
    return out


def separated(T, S, nS, k):
    """True when the pair is beyond the decay range (regular rule): every point of T lies farther
    than DECAY / |Im k| from S (distance of T's centroid to S minus T's circumradius)."""
    kim = abs(complex(k).imag)
    if kim == 0.0:
        return False
    c = T.mean(axis=0)
    rad = max(np.linalg.norm(T[j] - c) for j in range(3))
    return kim * (_tri_dist(c, S, nS) - rad) > DECAY
