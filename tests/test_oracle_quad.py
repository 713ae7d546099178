"""Pins of the oracle's quadrature rules and closed-form potential integrals."""
import itertools

import numpy as np
import pytest

from oracle import quad


def _monos(deg):
    for a, b, c in itertools.product(range(deg + 1), repeat=3):
        if a + b + c <= deg:
            yield a, b, c


@pytest.mark.parametrize("rule,deg", [(quad.radon7(), 5), (quad.gauss_tri(5), 8),
                                      (quad.subdivide4(quad.radon7()), 5)])
def test_rules_exact_on_polynomials(rule, deg):
    p, w = rule
    assert abs(w.sum() - 1.0) < 1e-14
    for a, b, c in _monos(deg):
        got = np.sum(w * p[:, 0] ** a * p[:, 1] ** b * p[:, 2] ** c)
        # exact: 2 A a! b! c! / (a+b+c+2)! with A = 1/2, rule weights normalised by A
        assert abs(got - quad.monomial_integral(0.5, a, b, c) / 0.5) < 1e-15


def test_radon7_is_not_degree6():
    p, w = quad.radon7()
    err = np.sum(w * p[:, 0] ** 6) - quad.monomial_integral(0.5, 6, 0, 0) / 0.5
    assert abs(err) > 1e-5


def _brute(r, tri, nrm, lev=6):
    P, W = quad.radon7()
    for _ in range(lev):
        P, W = quad.subdivide4((P, W))
    area = 0.5 * np.linalg.norm(np.cross(tri[1] - tri[0], tri[2] - tri[0]))
    X = P @ tri
    Rv = r - X
    R = np.linalg.norm(Rv, axis=1)
    d = (r - tri[0]) @ nrm
    rho = r - d * nrm
    return (area * np.sum(W / R), area * np.sum(W[:, None] * (X - rho) / R[:, None], axis=0),
            -area * np.sum(W[:, None] * Rv / R[:, None] ** 3, axis=0))


@pytest.mark.parametrize("r", [(0.4, 0.3, 0.5), (2.0, 1.0, 0.3), (-0.5, 0.4, -0.2),
                               (0.4, 0.3, 0.05), (1.5, 1.5, 0.0), (0.2, -0.3, -0.1)])
def test_static_potentials_vs_brute_force(r):
    tri = np.array([[0, 0, 0], [1.0, 0.2, 0], [0.3, 0.9, 0.0]])
    nrm = np.cross(tri[1] - tri[0], tri[2] - tri[0])
    nrm /= np.linalg.norm(nrm)
    r = np.array(r)
    got = quad.static_potentials(r[None], tri[None], nrm[None])
    ref = _brute(r, tri, nrm)
    for g, e in zip(got, ref):
        g = np.asarray(g).ravel()
        e = np.asarray(e).ravel()
        assert np.max(np.abs(g - e)) < 1e-10 * max(1.0, np.max(np.abs(e)))


def test_static_potentials_rotation_invariant():
    rng = np.random.default_rng(3)
    tri = np.array([[0, 0, 0], [1.0, 0.2, 0], [0.3, 0.9, 0.0]])
    nrm = np.array([0, 0, 1.0])
    r = np.array([0.3, 0.7, 0.4])
    A = np.linalg.qr(rng.standard_normal((3, 3)))[0]
    if np.linalg.det(A) < 0:
        A[:, 0] *= -1
    I0a, Ira, gIa = quad.static_potentials(r[None], tri[None], nrm[None])
    I0b, Irb, gIb = quad.static_potentials((A @ r)[None], (tri @ A.T)[None], (A @ nrm)[None])
    assert abs(I0a[0] - I0b[0]) < 1e-13
    assert np.allclose(A @ Ira[0], Irb[0], atol=1e-13)
    assert np.allclose(A @ gIa[0], gIb[0], atol=1e-13)


def test_solid_angle_inside_limit():
    # just above the triangle interior the normal part of grad int 1/R tends to -2 pi
    tri = np.array([[0, 0, 0], [1.0, 0, 0], [0, 1.0, 0.0]])
    nrm = np.array([0, 0, 1.0])
    _, _, gI = quad.static_potentials(np.array([[0.2, 0.2, 1e-7]]), tri[None], nrm[None])
    assert abs(gI[0, 2] + 2 * np.pi) < 1e-5
