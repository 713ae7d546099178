"""Pins of the whole solve: Mie series (Sec. IV-A validation), GMRES and ports."""
import numpy as np
import pytest

from oracle import farfield, gmres, operators as op, ports
from oracle.rwg import from_mesh
from paper_2108_03991_gb300 import synth


def test_mie_rayleigh_limit():
    x, m = 0.05, 1.5 + 0.01j
    ref = 4 * x ** 4 * abs((m * m - 1) / (m * m + 2)) ** 2
    assert abs(farfield.mie_backscatter(x, m) / ref - 1) < 3e-3


def test_mie_conductor_geometric_limit():
    # a large, highly conducting sphere backscatters about its geometric cross-section
    assert abs(farfield.mie_backscatter(60.0, 300 + 300j) - 1.0) < 0.1


@pytest.mark.parametrize("ka,tol", [(0.5, 0.09), (1.0, 0.03)])
def test_sphere_rcs_vs_mie(ka, tol):
    """P1: monostatic RCS of a lossy sphere (eps_rc = 1 - 30j) from the dense SLIM solve agrees
    with the Mie series (480 edges; the error falls to 1.7% / 0.4% at 1920 edges)."""
    rw = from_mesh(synth.sphere_mesh(1.0, 2, sigma=0.0))
    freq = ka / (2 * np.pi) * op.C0 / op.ELL
    k0 = op.k0_of(freq)
    sigma = 30 * 2 * np.pi * freq * op.EPS0
    S, _, _ = op.dense_system(rw, freq, [sigma])
    b = np.concatenate([op.plane_wave_rhs(rw, k0), np.zeros(rw.nt)])
    x, it, hist = gmres.gmres(S.matvec, b, tol=1e-8, restart=300, max_iter=3000)
    assert np.linalg.norm(S.matvec(x) - b) / np.linalg.norm(b) < 1e-7
    _, _, _, _, j = S.parts(x)
    s = farfield.rcs(rw, j, k0, np.array([[0, 0, -1.0]]))[0]
    ref = np.pi * farfield.mie_backscatter(ka, np.conj(np.sqrt(1 - 30j)))
    assert abs(s / ref - 1) < tol


def test_gmres_matches_direct_solve():
    rng = np.random.default_rng(0)
    n = 120
    A = 3 * np.eye(n) + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = synth.rand_cvec(n, 1)
    x, it, hist = gmres.gmres(lambda v: A @ v, b, tol=1e-12, restart=25)
    assert np.linalg.norm(x - np.linalg.solve(A, b)) < 1e-10 * np.linalg.norm(x)
    assert all(h2 <= h1 * (1 + 1e-12) for h1, h2 in zip(hist[1:25], hist[2:26]))


def test_two_port_admittance_symmetric():
    """P6 (ports): the 2x2 port admittance of a bar is symmetric (reciprocity), to the
    quadrature's symmetry level."""
    m = synth.bar_mesh(1.0, 1.0, 4.0, 0.5)
    rw = from_mesh(m)
    freq = 10e9
    S, _, _ = op.dense_system(rw, freq, [5.8e7])
    A = S.dense()
    rings = [ports.ring_edges(rw, 0, z) for z in (0.5, 3.5)]
    Ymat = np.zeros((2, 2), complex)
    for q, (eq, sq) in enumerate(rings):
        b = np.concatenate([ports.port_rhs(rw, eq, sq), np.zeros(rw.nt)])
        x = np.linalg.solve(A, b)
        for p, (ep, spp) in enumerate(rings):
            Ymat[p, q] = ports.port_current(rw, ep, spp, x[:rw.ne])
    assert len(rings[0][0]) == 8
    assert abs(Ymat[0, 1] - Ymat[1, 0]) <= 2e-3 * abs(Ymat[0, 1])


def test_square_loop_dc_resistance_and_inductance():
    """P5 (ports + internal problem): input impedance of a closed square copper loop (outer side
    10 um, cross-section 2 x 2 um, centreline side 8 um) driven by one delta-gap port at 100 MHz,
    where the skin depth (6.6 um) exceeds the cross-section. Re Z is the DC resistance: against
    the centreline estimate l_c / (sigma w t) it is low by the corner crowding (12%); counting
    each square corner of the strip as 0.559 squares (the conformal-mapping value for a
    right-angle bend) it agrees to 5%. Im Z / omega is the loop inductance: against the
    round-wire square-loop formula L = (2 mu0 s / pi)(ln(s / r) - 0.774) (Grover) with the
    equivalent radius r = 0.2235 (w + t) of a rectangular section, within 10%. The current is
    the same through every cross-section of the loop."""
    w = t = 2.0
    side, f = 10.0, 1e8
    sig = synth.SIGMA_CU
    mesh = synth.square_loop(side, w, t, 1.0, sigma=sig)
    rw = from_mesh(mesh)
    S, _, _ = op.dense_system(rw, f, mesh.sigma)
    A = S.dense()

    def ring(axis, lo_side):
        e, s = ports.ring_edges(rw, 0, side / 2, axis=axis)
        mid = 0.5 * (rw.verts[rw.ev[e, 0]] + rw.verts[rw.ev[e, 1]])
        k = (mid[:, 1 - axis] < side / 2) == lo_side
        return e[k], s[k]
    ep, sp = ring(0, True)
    b = np.concatenate([ports.port_rhs(rw, ep, sp), np.zeros(rw.nt)])
    x = np.linalg.solve(A, b)
    I = ports.port_current(rw, ep, sp, x[:rw.ne])
    Z = op.ETA0 / I
    # the same current through the other three cross-sections
    for axis, lo in ((0, False), (1, True), (1, False)):
        e2, s2 = ring(axis, lo)
        assert abs(abs(ports.port_current(rw, e2, s2, x[:rw.ne])) - abs(I)) < 1e-8 * abs(I)
    sq = side - w                                   # centreline side, um
    r_centre = 4 * sq * 1e-6 / (sig * w * t * 1e-12)
    squares = 4 * (side - 2 * w) / w + 4 * 0.559
    r_corner = squares / (sig * t * 1e-6)
    assert 0.80 < Z.real / r_centre < 0.95
    assert abs(Z.real / r_corner - 1) < 0.05
    L = Z.imag / (2 * np.pi * f)
    L_grover = 2 * op.MU0 * sq * 1e-6 / np.pi * (np.log(sq / (0.2235 * (w + t))) - 0.774)
    assert abs(L / L_grover - 1) < 0.10
