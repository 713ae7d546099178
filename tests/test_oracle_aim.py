"""Pins of the AIM oracle (Sec. III-A item 1, Eq. AIM_L)."""
import itertools

import numpy as np
import pytest

from oracle import aim, operators as op, quad
from oracle.rwg import from_mesh
from paper_2108_03991_gb300 import synth


@pytest.fixture(scope="module")
def setup():
    m = synth.bar_mesh(1.0, 1.0, 3.0, 0.25)
    rw = from_mesh(m)
    k0 = op.k0_of(10e9)
    LA = op.dense_rwg(rw, k0, "A")
    LP = op.dense_lphi(rw, k0)
    return m, rw, k0, LA, LP


def test_fft_convolution_equals_direct_sum(setup):
    """P8: the zero-padded FFT convolution equals the direct sum."""
    m, rw, k0, _, _ = setup
    g = synth.grid_box(m, 0.25)
    A = aim.Aim(rw, g.origin, g.h, g.n, k0)
    s = synth.rand_cvec(A.ng, 1)
    ref = A.conv_direct(s)
    assert np.max(np.abs(A.conv(s) - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_weights_reproduce_quadratics(setup):
    """Lagrange projection matches every moment of degree <= 2 per axis (an independent,
    higher-order rule computes the moments)."""
    m, rw, k0, _, _ = setup
    g = synth.grid_box(m, 0.3)
    A = aim.Aim(rw, g.origin, g.h, g.n, k0)
    b, w = quad.gauss_tri(7)
    X = rw.verts[rw.tris]
    ctr = 0.5 * (rw.centroid[rw.et[:, 0]] + rw.centroid[rw.et[:, 1]])
    nodes = A.origin + (A.anc_e[:, None, :] + aim.OFFS[None]) * A.h        # [ne, 27, 3]
    for ex in itertools.product(range(3), repeat=3):
        pn = np.prod((nodes - ctr[:, None, :]) ** np.array(ex), axis=-1)     # [ne, 27]
        lhs = np.einsum("mck,mk->mc", A.WA, pn)
        rhs = np.zeros((rw.ne, 3))
        for side, sgn in ((0, 1.0), (1, -1.0)):
            t = rw.et[:, side]
            pts = quad.rule_points(X[t], b)
            f = sgn * (rw.elen / (2 * rw.area[t]))[:, None, None] * (pts - rw.verts[rw.eopp[:, side]][:, None])
            p = np.prod((pts - ctr[:, None, :]) ** np.array(ex), axis=-1)
            rhs += np.einsum("q,m,mqc,mq->mc", w, rw.area[t], f, p)
        assert np.max(np.abs(lhs - rhs)) < 1e-13


def test_near_pairs_complete(setup):
    m, rw, k0, _, _ = setup
    g = synth.grid_box(m, 0.25)
    A = aim.Aim(rw, g.origin, g.h, g.n, k0)
    M, N = A.near_e
    d = np.max(np.abs(A.anc_e[:, None] - A.anc_e[None]), axis=-1)
    ref = np.argwhere(d <= 2)
    got = np.stack([M, N], axis=1)
    assert np.array_equal(ref, got)


def test_precorrection_restores_exact_near_entries(setup):
    """For near pairs the AIM operator's entries equal the exact Galerkin entries."""
    m, rw, k0, LA, LP = setup
    g = synth.grid_box(m, 0.25)
    A = aim.Aim(rw, g.origin, g.h, g.n, k0).build_near(LA, LP)
    M, N = A.near_e
    sel = np.random.default_rng(0).choice(M.size, 40, replace=False)
    for i in sel:
        e = np.zeros(rw.ne, complex)
        e[N[i]] = 1.0
        assert abs(A.LA(e)[M[i]] - LA[M[i], N[i]]) <= 1e-12 * abs(LA).max()


def test_aim_vs_dense(setup):
    """P7: the AIM operator approximates the dense one; the error shrinks with the grid."""
    m, rw, k0, LA, LP = setup
    j = synth.rand_cvec(rw.ne, 2)
    q = synth.rand_cvec(rw.nt, 3)
    errs = []
    for hg in (0.25, 0.15):
        g = synth.grid_box(m, hg)
        A = aim.Aim(rw, g.origin, g.h, g.n, k0).build_near(LA, LP)
        ea = np.linalg.norm(A.LA(j) - LA @ j) / np.linalg.norm(LA @ j)
        ep = np.linalg.norm(A.LPhi(q) - LP @ q) / np.linalg.norm(LP @ q)
        errs.append(max(ea, ep))
    assert errs[0] < 5e-3 and errs[1] < errs[0]


def test_far_part_bilinear_symmetric(setup):
    m, rw, k0, _, _ = setup
    g = synth.grid_box(m, 0.25)
    A = aim.Aim(rw, g.origin, g.h, g.n, k0)
    x = synth.rand_cvec(rw.ne, 5)
    y = synth.rand_cvec(rw.ne, 6)
    a, b = x @ A.far_A(y), y @ A.far_A(x)
    assert abs(a - b) <= 1e-13 * abs(a)


def test_stencil_outside_grid_rejected(setup):
    m, rw, k0, _, _ = setup
    g = synth.grid_box(m, 0.25)
    with pytest.raises(aim.GridError):
        aim.Aim(rw, g.origin + 0.5, g.h, g.n, k0)
