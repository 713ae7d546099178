"""Pins of the oracle's sparse internal operators (Sec. III-A, third item: at high frequency
L_{k_i} and K_{k_i} are treated as sparse, distant interactions dropped)."""
import numpy as np
import pytest

from oracle import operators as op
from oracle import sparse_internal as si
from oracle.rwg import from_mesh
from paper_2108_03991_gb300 import synth


def _points_on(rw, t, k, rng):
    """k uniform random points on triangle t."""
    u = rng.random((k, 2))
    flip = u.sum(1) > 1
    u[flip] = 1 - u[flip]
    A, B, C = rw.verts[rw.tris[t]]
    return A + u[:, :1] * (B - A) + u[:, 1:] * (C - A)


def test_support_distance_is_a_lower_bound():
    """d_mn never exceeds the distance between sampled points of the two supports (a formula
    that dropped the radii would exceed it for near supports), and supports that share a
    vertex have d_mn = 0 (to rounding); the kept pattern is symmetric."""
    rw = from_mesh(synth.bar_mesh(1.0, 1.0, 3.0, 0.5))
    D = si.support_distance(rw, 0, rw.ne)
    assert np.allclose(D, D.T)
    rng = np.random.default_rng(3)
    P = [np.concatenate([_points_on(rw, t, 40, rng) for t in rw.et[m]]) for m in range(rw.ne)]
    for m in rng.choice(rw.ne, 24, replace=False):
        for n in range(rw.ne):
            dmin = np.min(np.linalg.norm(P[m][:, None, :] - P[n][None, :, :], axis=2))
            assert D[m, n] <= dmin + 1e-12
            shared = set(rw.tris[rw.et[m]].ravel()) & set(rw.tris[rw.et[n]].ravel())
            if shared:
                assert D[m, n] <= 1e-12
    M = si.pattern(rw, 0, rw.ne, 0.05)
    assert np.array_equal(M, M.T) and M.diagonal().all()


def test_full_pattern_at_low_frequency():
    """Copper at 10 GHz (delta = 0.66 um): R_cut = 15 um covers the 3 um bar, every pair is kept
    and Z_s is the dense Z of Eq. MFIEinZin."""
    mesh = synth.bar_mesh(1.0, 1.0, 3.0, 0.5)
    rw = from_mesh(mesh)
    S = si.SparseZ(rw, 10e9, mesh.sigma[0], 0, rw.ne)
    assert S.density == 1.0
    Z, _ = op.internal_blocks(rw, 10e9, mesh.sigma)
    h = synth.rand_cvec(rw.ne, 1)
    assert np.linalg.norm(S(h) - Z[0] @ h) <= 1e-12 * np.linalg.norm(Z[0] @ h)


@pytest.fixture(scope="module")
def gold_bar():
    """A 1 x 1 x 4 um gold bar at 1 THz (delta = 79 nm, R_cut = 1.8 um): 216 edges."""
    mesh = synth.bar_mesh(1.0, 1.0, 4.0, 0.5, sigma=synth.SIGMA_AU)
    rw = from_mesh(mesh)
    k0 = op.k0_of(1e12)
    epsc = op.eps_rc(mesh.sigma[0], 1e12)
    L, K = op.dense_rwg(rw, op.k_medium(k0, epsc), ("L", "K"))
    return rw, mesh, L, K, epsc, k0


def test_dropped_entries_are_negligible(gold_bar):
    """Every dropped entry of L_{k_i} and K_{k_i} is below 1e-9 of the largest (the kernel
    factor e^{-R/delta} is 1e-10 at R_cut), while pairs are dropped even on this 4 um bar."""
    rw, mesh, L, K, epsc, k0 = gold_bar
    S = si.SparseZ(rw, 1e12, mesh.sigma[0], 0, rw.ne, LK=(L, K))
    assert S.density < 0.9
    drop = ~S.mask
    assert np.abs(L[drop]).max() < 1e-9 * np.abs(L).max()
    assert np.abs(K[drop]).max() < 1e-9 * np.abs(K).max()


def test_sparse_product_matches_dense(gold_bar):
    """Z_s h (sparse LU of L_s) agrees with the dense Z h of Eq. MFIEinZin to 1e-9."""
    rw, mesh, L, K, epsc, k0 = gold_bar
    S = si.SparseZ(rw, 1e12, mesh.sigma[0], 0, rw.ne, LK=(L, K))
    ix = op.ix_matrix(rw).toarray()
    Z = -np.linalg.solve(L, K + 0.5 * ix) / (1j * k0 * epsc)
    for seed in (1, 2):
        h = synth.rand_cvec(rw.ne, seed)
        assert np.linalg.norm(S(h) - Z @ h) <= 1e-9 * np.linalg.norm(Z @ h)
