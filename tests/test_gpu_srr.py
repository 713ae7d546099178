"""GPU parity on the split-ring array family (the large metasurface workload) in a size the
oracle can follow: 4 x 4 gold rings (seed 2) at 1 THz, 14,592 RWG + 9,728 pulse unknowns, AIM
grid 64 x 64 x 8 with the array's anisotropic spacing. The skin depth (79 nm) is a 25th of the
element size, so every touching pair of the internal operator takes the large-|k| rule. The
oracle forms the internal matrices of one ring and the near-region rows it needs, and checks:
the set-up matrices L_{k_i}, K_{k_i} + I_x/2 before the LU (same rule on both sides), Z and
Y_eq, the internal products on that ring's rows, and sampled rows of both block rows of the
system matvec for x = [h; q] with h on that ring only (or q = 0); a plane-wave solve with the
block-diagonal preconditioner reaches a true FP64 residual of 1e-6."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import aim as oaim, operators as op  # noqa: E402
from oracle.rwg import from_mesh  # noqa: E402
from paper_2108_03991_gb300 import api, synth  # noqa: E402
from syscheck import check_system, max_rel, rel  # noqa: E402

RING = 5  # the ring whose internal matrices the oracle forms


@pytest.fixture(scope="module")
def srr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_03991_gb300 import build
    build.build()
    mesh, grid, freq = synth.srr_array_config(2, 4)
    ctx = api.Context(mesh, grid, freq)
    rw = from_mesh(mesh)
    k0 = op.k0_of(freq)
    a, b = rw.obj_edge_ranges()[RING]
    rng = np.random.default_rng(5)
    rows_e = np.sort(np.concatenate([rng.choice(rw.ne, 32, replace=False),
                                     rng.choice(np.arange(a, b), 32, replace=False)]))
    rows_t = np.sort(rng.choice(rw.nt, 48, replace=False))
    A = oaim.Aim(rw, grid.origin, grid.h, grid.n, k0)
    A.build_near(rows_e=rows_e, rows_t=np.unique(np.concatenate([rows_t, rw.et[rows_e].ravel()])))
    ix = op.ix_matrix(rw)
    ixr = ix[a:b, a:b].toarray()
    epsc = op.eps_rc(mesh.sigma[RING], freq)
    ki = op.k_medium(k0, epsc)
    Lk, Kk = op.dense_rwg(rw, ki, ("L", "K"), a, b)
    Kk = Kk + 0.5 * ixr
    Z = -np.linalg.solve(Lk, Kk) / (1j * k0 * epsc)  # Eq. MFIEinZin, as operators.internal_blocks
    Ll, Kl = op.dense_rwg(rw, k0, ("L", "K"), a, b)
    Y = np.linalg.solve(Ll, Kl + 0.5 * ixr) / (1j * k0)
    return dict(ctx=ctx, rw=rw, k0=k0, ki=ki, A=A, rows_e=rows_e, rows_t=rows_t, rng=(a, b),
                Lk=Lk, Kk=Kk, Z=Z, Y=Y, ix=ix, fd=op.fd_matrix(rw))


def test_srr_sparse_internal_built(srr):
    """At 1 THz (skin depth 79 nm, a 25th of the element size) every ring qualifies for the
    sparse internal operator: it is built, checked against the dense Z at set-up and in use,
    at under half of the dense Z's bytes; the oracle's sparse product (Sec. III-A, third item)
    agrees with the dense Z h of the ring to 1e-10."""
    from oracle import sparse_internal as si
    ctx = srr["ctx"]
    sp = ctx.internal_sparse(True)
    assert sp["objects"] == ctx.nobj and sp["on"] and 0 < sp["band"] <= 256
    assert sp["check"] is not None and sp["check"] < 1e-8 and not sp["wait_timed_out"]
    assert sp["bytes_c32"] < 0.5 * ctx.zy_bytes_c32 / 2
    a, b = srr["rng"]
    ixr = srr["ix"][a:b, a:b].toarray()
    S = si.SparseZ(srr["rw"], 1e12, synth.SIGMA_AU, a, b, ix=srr["ix"],
                   LK=(srr["Lk"], srr["Kk"] - 0.5 * ixr))
    assert S.density < 0.2
    h = synth.rand_cvec(b - a, 31)
    assert rel(S(h), srr["Z"] @ h) < 1e-10
    srr["S"] = S


def test_srr_setup_matrices(srr):
    """L_{k_i} and K_{k_i} + I_x/2 of one ring before the LU (1e-12 of the largest entry), and
    the formed Z and Y_eq (Z well conditioned at this |k_i|: 1e-10; Y_eq 1e-6, the LU of the
    ill-conditioned L_{k0})."""
    ctx = srr["ctx"]
    assert abs(srr["ki"]) * srr["rw"].diam.max() > 30
    Lg, Kg = ctx.LK(RING)
    assert max_rel(Lg, srr["Lk"]) < 1e-12
    assert max_rel(Kg, srr["Kk"]) < 1e-12
    assert rel(ctx.Z(RING), srr["Z"]) < 1e-10
    assert rel(ctx.Y(RING), srr["Y"]) < 1e-6


@pytest.mark.parametrize("sparse", [True, False])
@pytest.mark.parametrize("prec,tol_z,tol_y", [(api.BEM_C32, 1e-5, 1e-5), (api.BEM_C64, 1e-10, 1e-6)])
def test_srr_internal_rows(srr, prec, tol_z, tol_y, sparse):
    """e = Z h (sparse Z_s or dense Z) and h_eq = Y_eq e on the oracle ring's rows."""
    ctx = srr["ctx"]
    ctx.internal_sparse(sparse)
    a, b = srr["rng"]
    h = synth.rand_cvec(ctx.ne, 23)
    npdt = np.complex64 if prec == api.BEM_C32 else np.complex128
    e, heq = ctx.internal(torch.from_numpy(h.astype(npdt)).cuda(), prec=prec)
    eo = srr["Z"] @ h[a:b]
    ho = srr["Y"] @ eo
    e, heq = e.cpu().numpy()[a:b], heq.cpu().numpy()[a:b]
    assert rel(e, eo) < tol_z and max_rel(e, eo) < 3 * tol_z
    assert rel(heq, ho) < tol_y and max_rel(heq, ho) < 3 * tol_y
    if sparse and "S" in srr:  # against the oracle's own sparse product as well
        es = srr["S"](h[a:b])
        assert rel(e, es) < tol_z and max_rel(e, es) < 3 * tol_z
    ctx.internal_sparse(True)


@pytest.mark.parametrize("sparse", [True, False])
@pytest.mark.parametrize("case", ["both", "q0"])
@pytest.mark.parametrize("prec,tol", [(api.BEM_C32, 1e-5), (api.BEM_C64, 1e-7)])
def test_srr_system_rows(srr, prec, tol, case, sparse):
    ctx, A, rw, k0 = srr["ctx"], srr["A"], srr["rw"], srr["k0"]
    ctx.internal_sparse(sparse)
    re, rt = srr["rows_e"], srr["rows_t"]
    a, b = srr["rng"]
    h = np.zeros(ctx.ne, complex)
    h[a:b] = synth.rand_cvec(b - a, 24)
    q = synth.rand_cvec(ctx.nt, 25) if case == "both" else np.zeros(ctx.nt, complex)
    x = np.concatenate([h, q])
    npdt = np.complex64 if prec == api.BEM_C32 else np.complex128
    y = ctx.matvec(torch.from_numpy(x.astype(npdt)).cuda(), prec=prec).cpu().numpy()
    e = np.zeros(ctx.ne, complex)
    e[a:b] = srr["Z"] @ h[a:b]
    j = h.copy()
    j[a:b] -= srr["Y"] @ e[a:b]
    lphi_q = A.far_P(q) + A.LNR_P @ q
    y1 = 1j * k0 * (A.far_A(j) + A.LNR_A @ j) + srr["ix"] @ e - srr["fd"].T @ lphi_q
    y2 = srr["fd"] @ j + 1j * k0 * q
    check_system(np.concatenate([y[re], y[ctx.ne + rt]]), np.concatenate([y1[re], y2[rt]]),
                 ctx.ne, tol, rows=(re, rt))
    ctx.internal_sparse(True)


@pytest.mark.parametrize("prec,tol", [(api.BEM_C32, 1e-6), (api.BEM_C64, 1e-12)])
def test_srr_sparse_matches_dense_everywhere(srr, prec, tol):
    """The whole system product and a 3-vector batch with the sparse Z_s against the dense Z on
    the same device (every ring, not only the oracle's)."""
    ctx = srr["ctx"]
    npdt = np.complex64 if prec == api.BEM_C32 else np.complex128
    x = torch.from_numpy(synth.rand_cvec(ctx.n, 26).astype(npdt)).cuda()
    xb = torch.from_numpy(np.stack([synth.rand_cvec(ctx.n, 27 + r) for r in range(3)]).astype(npdt)).cuda()
    out = {}
    for sparse in (False, True):
        ctx.internal_sparse(sparse)
        out[sparse] = (ctx.matvec(x, prec=prec).cpu().numpy(),
                       ctx.matvec_batch(xb, prec=prec).cpu().numpy())
    for a, b in zip(out[True], out[False]):
        for ar, br in zip(a.reshape(-1, ctx.n), b.reshape(-1, ctx.n)):
            check_system(ar, br, ctx.ne, tol)


def test_srr_chosen_solve(srr):
    """FP32-bulk FGMRES with the block-diagonal preconditioner on the 4 x 4 array: a true FP64
    residual of 1e-6 for a normally incident plane wave."""
    ctx = srr["ctx"]
    b = ctx.rhs_plane_wave((1.0, 0.0, 0.0), (0.0, 0.0, -1.0), prec=api.BEM_C64)
    x, info = ctx.solve(b, tol=1e-6, restart=100, max_iter=500, prec_mode=api.BEM_C32, precond=1)
    assert info["status"] == api.BEM_OK and info["resid_true"] <= 1e-6
    assert info["iters"] < 100
    pb = ctx.precond_build  # built in FP32 with every block passing its check
    assert pb["prec"] == api.BEM_C32 and pb["fp64_blocks"] == 0 and pb["check"] < 1e-3
