"""Pins of the ground-plane (PEC half-space) Green's function and operators of the oracle
(oracle/ground.py), the first piece of the layered background of the paper's Table I: the
boundary condition on the plane, the Lorenz gauge between the vector and scalar potentials of
horizontal and vertical current elements (which fixes every image sign), reciprocity of the
Galerkin operators, the free-space limit, the grid form of the image term, and image theory
at the level of a port solve of the whole system."""
import numpy as np
import pytest

from oracle import ground, operators as op, ports
from oracle.rwg import from_mesh
from paper_2108_03991_gb300 import synth

K0 = op.k0_of(30e12)  # 0.63 / um: phase over the test distances
ZG = -0.7


def test_boundary_condition_on_the_plane():
    """On the plane the tangential vector potential and the scalar potential vanish (so does the
    tangential E = -j w A - grad Phi), the normal vector potential doubles."""
    rng = np.random.default_rng(1)
    rp = rng.uniform(-1, 1, (50, 3))
    rp[:, 2] = ZG + rng.uniform(0.2, 2.0, 50)
    r = rng.uniform(-3, 3, (50, 3))
    r[:, 2] = ZG
    GA, GP = ground.kernels(K0, r, rp, ZG)
    g = ground.green(K0, np.linalg.norm(r - rp, axis=1))
    assert np.max(np.abs(GA[:, :2])) < 1e-13 * np.max(np.abs(g))
    assert np.max(np.abs(GP)) < 1e-13 * np.max(np.abs(g))
    assert np.allclose(GA[:, 2], 2 * g, rtol=1e-13)


def test_lorenz_gauge_fixes_the_image_signs():
    """For a current element l at r' (charges +-I/(j w) at its ends) the potentials obey
    div A + j w mu eps Phi = 0, i.e. div_r (G^A l) = -(l . grad_r') G^Phi, for horizontal and
    vertical elements (central differences); with the opposite image sign for the vertical
    vector potential, or for the scalar one, it fails."""
    rng = np.random.default_rng(2)
    d = 1e-4
    for _ in range(20):
        rp = np.array([rng.uniform(-1, 1), rng.uniform(-1, 1), ZG + rng.uniform(0.3, 1.5)])
        r = np.array([rng.uniform(-2, 2), rng.uniform(-2, 2), ZG + rng.uniform(0.3, 2.0)])
        for c in range(3):
            l = np.eye(3)[c]
            div = 0.0
            for a in range(3):
                e = np.eye(3)[a] * d
                GAp, _ = ground.kernels(K0, r + e, rp, ZG)
                GAm, _ = ground.kernels(K0, r - e, rp, ZG)
                div += (GAp[a] * l[a] - GAm[a] * l[a]) / (2 * d)
            _, Pp = ground.kernels(K0, r, rp + l * d, ZG)
            _, Pm = ground.kernels(K0, r, rp - l * d, ZG)
            dphi = (Pp - Pm) / (2 * d)
            assert abs(div + dphi) < 1e-6 * abs(div), (c, div, dphi)
            if c == 2:  # the wrong image sign for the vertical vector potential breaks it
                R = np.linalg.norm(r - rp)
                rp_i = ground.image(rp, ZG)
                gi = lambda x: ground.green(K0, np.linalg.norm(x - rp_i))
                g = lambda x: ground.green(K0, np.linalg.norm(x - rp))
                e = np.array([0, 0, d])
                wrong = ((g(r + e) - gi(r + e)) - (g(r - e) - gi(r - e))) / (2 * d)
                assert abs(wrong + dphi) > 1e-3 * abs(div)


def test_ground_operators_reciprocal_and_far_limit():
    """The image parts of L^A and L^Phi are symmetric (Galerkin with a symmetric kernel and the
    same rule on both sides; the free-space near-pair rule is symmetric only to its accuracy),
    sizeable for a box near the plane, and vanish as the plane recedes."""
    mesh = synth.box((0.0, 0.0, 0.0), (1.0, 1.0, 1.0), (2, 2, 2))
    rw = from_mesh(synth.merge([mesh], [synth.SIGMA_CU]))
    LA0, LP0 = op.dense_rwg(rw, K0, "A"), op.dense_lphi(rw, K0)
    LA, LP = ground.dense_ground_operators(rw, K0, -0.3)
    for M in (LA - LA0, LP - LP0):
        assert np.linalg.norm(M - M.T) < 1e-12 * np.linalg.norm(M)
    assert np.linalg.norm(LP - LP0) > 0.1 * np.linalg.norm(LP0)
    assert np.linalg.norm(LA - LA0) > 0.05 * np.linalg.norm(LA0)
    LAf, LPf = ground.dense_ground_operators(rw, K0, -1e4)
    assert 0 < np.linalg.norm(LPf - LP0) < 1e-3 * np.linalg.norm(LP0)
    assert 0 < np.linalg.norm(LAf - LA0) < 1e-3 * np.linalg.norm(LA0)


def test_grid_image_term_as_a_convolution():
    """The image part of the grid convolution (a correlation in z) equals the ordinary
    zero-padded FFT convolution of the z-reflected sources on the grid extended below the
    plane: the form a GPU convolution can take."""
    h = np.array([0.5, 0.4, 0.3])
    n = (6, 5, 4)
    zg = -1.0
    origin = np.array([0.1, -0.2, zg + 2 * h[2]])
    s = synth.rand_cvec(n[0] * n[1] * n[2], 3)
    for sign in (1.0, -1.0):
        a = ground.grid_image_direct(K0, h, n, origin, zg, s, sign)
        b = ground.grid_image_fft(K0, h, n, origin, zg, s, sign)
        assert np.linalg.norm(a - b) < 1e-12 * np.linalg.norm(a)


def test_image_parts_use_the_pinned_kernels():
    """Entries of the operators' image parts recomputed from ground.kernels (whose signs the
    gauge test fixes) minus the free-space kernel, with the same 7-point rule on both
    triangles (pairs that share no triangle, where the free-space kernel is finite at every
    pair of rule points)."""
    from oracle.quad import radon7, rule_points
    mesh = synth.box((0.0, 0.0, 0.0), (1.0, 1.0, 1.0), (2, 2, 2))
    rw = from_mesh(synth.merge([mesh], [synth.SIGMA_CU]))
    zg = -0.3
    LA, LP = ground.dense_ground_operators(rw, K0, zg)
    LA0, LP0 = op.dense_rwg(rw, K0, "A"), op.dense_lphi(rw, K0)
    b, w = radon7()
    rq = rule_points(rw.verts[rw.tris], b)

    def half(m, t):  # RWG m on triangle t at the rule points: [7, 3]
        a = [i for i in range(3) if rw.t_edges[t, i] == m][0]
        c = rw.t_esign[t, a] * rw.elen[m] / (2 * rw.area[t])
        return c * (rq[t] - rw.verts[rw.t_evert[t, a]])

    rng = np.random.default_rng(6)
    pairs = [(m, n) for m, n in rng.integers(0, rw.ne, (40, 2))
             if not set(rw.et[m]) & set(rw.et[n])][:6]
    assert len(pairs) == 6
    for m, n in pairs:
        v = 0.0
        for t in rw.et[m]:
            for s in rw.et[n]:
                r, rp = rq[t][:, None, :], rq[s][None, :, :]
                GA, _ = ground.kernels(K0, r, rp, zg)
                g = ground.green(K0, np.linalg.norm(r - rp, axis=-1))
                img = GA - g[..., None]
                fm, fn = half(m, t), half(n, s)
                v += rw.area[t] * rw.area[s] * np.einsum(
                    "q,p,qd,qpd,pd->", w, w, fm, img, fn)
        assert abs(v - (LA - LA0)[m, n]) < 1e-12 * abs(LA - LA0).max()
    for t, s in [(t, s) for t, s in rng.integers(0, rw.nt, (20, 2)) if t != s][:6]:
        r, rp = rq[t][:, None, :], rq[s][None, :, :]
        _, GP = ground.kernels(K0, r, rp, zg)
        g = ground.green(K0, np.linalg.norm(r - rp, axis=-1))
        v = rw.area[t] * rw.area[s] * np.einsum("q,p,qp->", w, w, GP - g)
        assert abs(v - (LP - LP0)[t, s]) < 1e-12 * abs(LP - LP0).max()


def test_mirror_geometry_identity():
    """Image theory restated with the free-space oracle: the ground-plane operator between two
    RWG functions equals the free-space one between f_m and f_n minus the free-space one between
    f_m and the mirrored function D f_n(M r) (M: the reflection in the plane), the mirror box
    meshed as a second object (its triangles reversed to stay outward). Two independent codes:
    the free-space oracle's rules against the image parts' 7-point rule, 1e-10 with the plane
    far enough for both to use the regular rule."""
    V, F = synth.box((0.0, 0.0, 0.0), (1.0, 1.0, 1.0), (2, 2, 2))
    zg = -2.0
    Vm = ground.image(V, zg)
    Fm = F[:, ::-1]  # the reflection reverses orientation: reverse to keep the normals outward
    mesh2 = synth.merge([(V, F), (Vm, Fm)], [synth.SIGMA_CU] * 2)
    rw1 = from_mesh(synth.merge([(V, F)], [synth.SIGMA_CU]))
    rw2 = from_mesh(mesh2)
    LA, LP = ground.dense_ground_operators(rw1, K0, zg)
    LA2, LP2 = op.dense_rwg(rw2, K0, "A"), op.dense_lphi(rw2, K0)
    ne, nt, nv = rw1.ne, rw1.nt, V.shape[0]
    # the mirrored function of edge n: edge (a + nv, b + nv) of the second object, with the sign
    # that makes f'_n'(r) = D f_n(M r) (compared at the centroid of the mirrored T+)
    key = {tuple(e): i for i, e in enumerate(rw2.ev)}
    mir, sgn = np.zeros(ne, int), np.zeros(ne)
    for n in range(ne):
        a, b = rw1.ev[n]
        n2 = key[(a + nv, b + nv)]
        t = rw1.et[n, 0]
        c = rw1.centroid[t]
        f = rw1.elen[n] / (2 * rw1.area[t]) * (c - rw1.verts[rw1.eopp[n, 0]])
        cm = ground.image(c, zg)
        k = 0 if np.allclose(rw2.centroid[rw2.et[n2, 0]], cm) else 1
        tm = rw2.et[n2, k]
        s2 = 1.0 if k == 0 else -1.0
        f2 = s2 * rw2.elen[n2] / (2 * rw2.area[tm]) * (cm - rw2.verts[rw2.eopp[n2, k]])
        mir[n] = n2
        sgn[n] = 1.0 if np.allclose(f2, ground.D_IMG * f) else -1.0
        assert np.allclose(sgn[n] * f2, ground.D_IMG * f)
    ref = LA2[:ne, :ne] - LA2[:ne, mir] * sgn[None, :]
    assert np.linalg.norm(LA - ref) < 1e-10 * np.linalg.norm(ref)
    # pulses: the mirrored triangle of t is t + nt (same order), the image charge opposite
    refP = LP2[:nt, :nt] - LP2[:nt, nt:]
    assert np.linalg.norm(LP - refP) < 1e-10 * np.linalg.norm(refP)


@pytest.fixture(scope="module")
def ground_aim():
    """Two boxes 0.3 um above the plane, grid spacing 0.25 um, the plane the node plane two
    below the grid."""
    parts = [synth.box((0.0, 0.0, 0.0), (1.0, 1.0, 0.5), (2, 2, 1)),
             synth.box((2.0, 0.0, 0.0), (1.0, 1.0, 0.5), (2, 2, 1))]
    rw = from_mesh(synth.merge(parts, [synth.SIGMA_CU] * 2))
    h = np.array([0.25, 0.25, 0.25])
    origin = np.array([-0.5, -0.5, -0.5]) + h / 12.0
    origin[2] = -0.5
    zg = origin[2] - 2 * h[2]
    n = (17, 9, 9)
    LA, LP = ground.dense_ground_operators(rw, K0, zg)
    G = ground.GroundAim(rw, origin, h, n, K0, zg).build_near(LA, LP)
    return rw, G, LA, LP


def test_ground_aim_matches_dense(ground_aim):
    """O-AIM with images against the dense ground-plane operators: within the AIM far-field
    error (8e-4 for L^A and 1.4e-3 for L^Phi measured, 5e-3 allowed as for P7 in free space),
    the image part being a fifth of the product."""
    rw, G, LA, LP = ground_aim
    j = synth.rand_cvec(rw.ne, 7)
    q = synth.rand_cvec(rw.nt, 8)
    assert np.linalg.norm(G.LA(j) - LA @ j) < 5e-3 * np.linalg.norm(LA @ j)
    assert np.linalg.norm(G.LPhi(q) - LP @ q) < 5e-3 * np.linalg.norm(LP @ q)
    LA0, LP0 = op.dense_rwg(rw, K0, "A"), op.dense_lphi(rw, K0)
    assert np.linalg.norm((LP - LP0) @ q) > 0.1 * np.linalg.norm(LP @ q)


def test_ground_aim_restores_exact_near_entries(ground_aim):
    """The precorrection (free-space and image grid terms) restores the exact ground-plane
    entries on the near pairs (1e-12)."""
    rw, G, LA, LP = ground_aim
    M, N = G.A.near_e
    cols = np.unique(N)[:12]
    for c in cols:
        e = np.zeros(rw.ne)
        e[c] = 1.0
        col = G.LA(e)
        rows = M[N == c]
        assert np.max(np.abs(col[rows] - LA[rows, c])) < 1e-12 * np.abs(LA).max()
    T, S = G.A.near_t
    for c in np.unique(S)[:12]:
        e = np.zeros(rw.nt)
        e[c] = 1.0
        col = G.LPhi(e)
        rows = T[S == c]
        assert np.max(np.abs(col[rows] - LP[rows, c])) < 1e-12 * np.abs(LP).max()


def test_port_current_over_ground_is_image_theory():
    """The whole SLIM system above the ground plane (Eq. AEFIEoutJ with the ground-plane L^A and
    L^Phi; the internal problems unchanged) against image theory at the level of a solve: a
    copper bar 1 um above the plane, along x, driven by a delta-gap port at its middle (10 GHz),
    carries the port current that the same bar carries in free space beside its mirror image
    driven in antiphase (the image of an x-directed gap field is reversed), both systems solved
    densely (1e-10; 2e-16 measured). The plane changes the current by 1.7%, an in-phase image
    by 3.2%."""
    freq = 10e9
    k0 = op.k0_of(freq)
    V, F = synth.box((0.0, 0.0, 2.0), (2.0, 1.0, 1.0), (4, 2, 2))
    zg = 1.0
    m1 = synth.merge([(V, F)], [synth.SIGMA_CU])
    rw1 = from_mesh(m1)
    Zs, Ys = op.internal_blocks(rw1, freq, m1.sigma)
    LA, LP = ground.dense_ground_operators(rw1, k0, zg)
    S1 = op.SlimSystem(rw1, freq, Zs, Ys, lambda v: LA @ v, lambda v: LP @ v)
    e1, s1 = ports.ring_edges(rw1, 0, 1.0, axis=0)
    x = np.linalg.solve(S1.dense(), np.concatenate([ports.port_rhs(rw1, e1, s1), np.zeros(rw1.nt)]))
    Ig = ports.port_current(rw1, e1, s1, x[:rw1.ne])
    m2 = synth.merge([(V, F), (ground.image(V, zg), F[:, ::-1])], [synth.SIGMA_CU] * 2)
    rw2 = from_mesh(m2)
    S2, _, _ = op.dense_system(rw2, freq, m2.sigma)
    A2 = S2.dense()
    ea, sa = ports.ring_edges(rw2, 0, 1.0, axis=0)
    eb, sb = ports.ring_edges(rw2, 1, 1.0, axis=0)
    cur = {}
    for sgn in (-1.0, 1.0):
        b = np.concatenate([ports.port_rhs(rw2, ea, sa) + sgn * ports.port_rhs(rw2, eb, sb),
                            np.zeros(rw2.nt)])
        x2 = np.linalg.solve(A2, b)
        cur[sgn] = ports.port_current(rw2, ea, sa, x2[:rw2.ne])
    assert abs(cur[-1.0] - Ig) < 1e-10 * abs(Ig)
    assert abs(cur[1.0] - Ig) > 1e-2 * abs(Ig)
    S0, _, _ = op.dense_system(rw1, freq, m1.sigma)
    x0 = np.linalg.solve(S0.dense(), np.concatenate([ports.port_rhs(rw1, e1, s1), np.zeros(rw1.nt)]))
    assert abs(ports.port_current(rw1, e1, s1, x0[:rw1.ne]) - Ig) > 1e-2 * abs(Ig)
