"""GPU parity at the benchmark's full size, in the launch configuration bench.py times: the 4x4
Cu bar array (seed 0), 17,832 RWG + 11,888 pulse unknowns, 10 GHz, AIM grid 35 x 35 x 78, set up
exactly as bench.py does (the set-up autotuner picks the GEMV launch). The oracle cannot form
every near pair and every internal block at this size in a test's time, so it computes sampled
outputs one by one: 64 seeded rows of L^A and of L^Phi (far part by the full FFT convolution,
near part from the exact entries of those rows), the rows of the smallest and of the largest
object for the internal products (the largest block, 1,824 rows, is where the task list's row
panels and partial tasks fall), and sampled rows of the whole system matvec for an x whose h is
non-zero on one of those objects only (so j needs only that object's Z and Y_eq); each block row
of the system product is compared against its own norm and element by element."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import aim as oaim, operators as op  # noqa: E402
from oracle.rwg import from_mesh  # noqa: E402
from paper_2108_03991_gb300 import api, synth  # noqa: E402
from syscheck import check_system, max_rel, rel  # noqa: E402


@pytest.fixture(scope="module")
def full():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_03991_gb300 import build
    build.build()
    mesh, grid, freq = synth.bar_array_config(0, 10e9)
    ctx = api.Context(mesh, grid, freq)
    rw = from_mesh(mesh)
    k0 = op.k0_of(freq)
    rng = np.random.default_rng(12)
    rows_e = np.sort(rng.choice(rw.ne, 64, replace=False))
    rows_t = np.sort(rng.choice(rw.nt, 64, replace=False))
    A = oaim.Aim(rw, grid.origin, grid.h, grid.n, k0)
    # L^Phi rows: the sampled triangles and the two triangles of every sampled edge
    tri = np.unique(np.concatenate([rows_t, rw.et[rows_e].ravel()]))
    A.build_near(rows_e=rows_e, rows_t=tri)
    ranges = rw.obj_edge_ranges()
    sizes = [b - a for a, b in ranges]
    objs = {"smallest": int(np.argmin(sizes)), "largest": int(np.argmax(sizes))}
    ix = op.ix_matrix(rw)
    Zs, Ys = op.internal_blocks(rw, freq, mesh.sigma, ix=ix, objects=list(objs.values()))
    return dict(ctx=ctx, rw=rw, k0=k0, A=A, rows_e=rows_e, rows_t=rows_t, objs=objs,
                ranges=ranges, Z=Zs, Y=Ys, ix=ix, fd=op.fd_matrix(rw))


@pytest.mark.parametrize("prec,tol", [(api.BEM_C32, 1e-5), (api.BEM_C64, 1e-11)])
def test_fullsize_LA_LPhi_rows(full, prec, tol):
    ctx, A, re, rt = full["ctx"], full["A"], full["rows_e"], full["rows_t"]
    j = synth.rand_cvec(ctx.ne, 21)
    q = synth.rand_cvec(ctx.nt, 22)
    npdt = np.complex64 if prec == api.BEM_C32 else np.complex128
    ya = ctx.matvec(torch.from_numpy(j.astype(npdt)).cuda(), which=api.AIM_OP_LA, prec=prec)
    yp = ctx.matvec(torch.from_numpy(q.astype(npdt)).cuda(), which=api.AIM_OP_LPHI, prec=prec)
    ref_a = (A.far_A(j) + A.LNR_A @ j)[re]
    ref_p = (A.far_P(q) + A.LNR_P @ q)[rt]
    assert rel(ya.cpu().numpy()[re], ref_a) < tol
    assert rel(yp.cpu().numpy()[rt], ref_p) < tol


@pytest.mark.parametrize("which", ["smallest", "largest"])
@pytest.mark.parametrize("prec,tol_z,tol_y", [(api.BEM_C32, 1e-5, 1e-5), (api.BEM_C64, 1e-9, 1e-6)])
def test_fullsize_internal_rows(full, prec, tol_z, tol_y, which):
    """e = Z h and h_eq = Y_eq e on every row of the smallest and of the largest object, with the
    launch the autotuner chose for all 16 objects (the other objects' rows are computed in the
    same launch), in the 2-norm of the object's rows and element by element. FP64 bounds as in
    the small-problem tests (two independent LU solves)."""
    ctx = full["ctx"]
    obj = full["objs"][which]
    a, b = full["ranges"][obj]
    h = synth.rand_cvec(ctx.ne, 23)
    npdt = np.complex64 if prec == api.BEM_C32 else np.complex128
    e, heq = ctx.internal(torch.from_numpy(h.astype(npdt)).cuda(), prec=prec)
    eo = full["Z"][obj] @ h[a:b]
    ho = full["Y"][obj] @ eo
    e, heq = e.cpu().numpy()[a:b], heq.cpu().numpy()[a:b]
    assert rel(e, eo) < tol_z and max_rel(e, eo) < 3 * tol_z
    assert rel(heq, ho) < tol_y and max_rel(heq, ho) < 3 * tol_y


@pytest.mark.parametrize("case", ["both", "q0"])
@pytest.mark.parametrize("which", ["smallest", "largest"])
@pytest.mark.parametrize("prec,tol", [(api.BEM_C32, 1e-5), (api.BEM_C64, 1e-7)])
def test_fullsize_system_rows(full, prec, tol, which, case):
    """Sampled rows of the system matvec of Eq. AEFIEoutJ (both block rows, each against its own
    norm) for x = [h; q] with h non-zero on one object only and q everywhere (or q = 0, where
    row 1 is j k0 L^A j + I_x e alone)."""
    ctx, A, rw, k0 = full["ctx"], full["A"], full["rw"], full["k0"]
    re, rt = full["rows_e"], full["rows_t"]
    obj = full["objs"][which]
    a, b = full["ranges"][obj]
    h = np.zeros(ctx.ne, complex)
    h[a:b] = synth.rand_cvec(b - a, 24)
    q = synth.rand_cvec(ctx.nt, 25) if case == "both" else np.zeros(ctx.nt, complex)
    if case == "q0":
        # sample the rows of row 1 where j's near and far fields are large: the object's own rows
        re = np.unique(np.concatenate([re, np.arange(a, b, max(1, (b - a) // 64))]))
    x = np.concatenate([h, q])
    npdt = np.complex64 if prec == api.BEM_C32 else np.complex128
    y = ctx.matvec(torch.from_numpy(x.astype(npdt)).cuda(), prec=prec).cpu().numpy()
    e = np.zeros(ctx.ne, complex)
    e[a:b] = full["Z"][obj] @ h[a:b]
    j = h.copy()
    j[a:b] -= full["Y"][obj] @ e[a:b]
    A.build_near(rows_e=re, rows_t=np.unique(np.concatenate([rt, rw.et[re].ravel()])))
    lphi_q = A.far_P(q) + A.LNR_P @ q  # exact on the triangles of the sampled edges
    y1 = 1j * k0 * (A.far_A(j) + A.LNR_A @ j) + full["ix"] @ e - full["fd"].T @ lphi_q
    y2 = full["fd"] @ j + 1j * k0 * q
    got = np.concatenate([y[re], y[ctx.ne + rt]])
    ref = np.concatenate([y1[re], y2[rt]])
    check_system(got, ref, ctx.ne, tol, rows=(re, rt))


@pytest.mark.parametrize("prec,tol", [(api.BEM_C32, 1e-6), (api.BEM_C64, 1e-12)])
def test_fullsize_batch_matches_single(full, prec, tol):
    """The batched system matvec of 4 right-hand sides at full size against the one-vector
    matvec (itself checked against the oracle above) for each right-hand side."""
    ctx = full["ctx"]
    npdt = np.complex64 if prec == api.BEM_C32 else np.complex128
    xs = np.stack([synth.rand_cvec(ctx.n, 300 + r) for r in range(4)]).astype(npdt)
    y = ctx.matvec_batch(torch.from_numpy(xs.ravel()).cuda(), prec=prec).cpu().numpy().reshape(4, -1)
    for r in range(4):
        y1 = ctx.matvec(torch.from_numpy(xs[r]).cuda(), prec=prec).cpu().numpy()
        assert rel(y[r], y1) < tol
