"""GPU parity at the benchmark's full size, in the launch configuration bench.py times: the
32 x 32 gold split-ring array at 1 THz (seed 2), 933,888 RWG + 622,592 pulse unknowns, AIM grid
512 x 512 x 8 (padded 1024 x 1024 x 15), set up exactly as bench.py sets it up (autotuned
launches, the sparse internal operator in use). The oracle cannot form a million-unknown
problem, so it computes sampled outputs one by one: 64 seeded rows of L^A and of L^Phi (far part
by its own FFT convolution on the padded grid, near part from the exact entries of those rows),
the internal products on every row of one ring, and sampled rows of both block rows of the
system matvec for an x whose h is non-zero on that ring only (so j needs only that ring's Z and
Y_eq). The oracle's share (RWG tables, projection matrices, the ring's internal matrices: a few
minutes of host time) runs in a thread while the device sets up."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import aim as oaim, operators as op  # noqa: E402
from oracle.rwg import from_mesh  # noqa: E402
from paper_2108_03991_gb300 import api, synth  # noqa: E402
from syscheck import check_system, max_rel, rel  # noqa: E402

RING = 517  # an interior ring of the array (row 16, column 5)


def _oracle_side(mesh, grid, freq):
    rw = from_mesh(mesh)
    k0 = op.k0_of(freq)
    rng = np.random.default_rng(12)
    a, b = rw.obj_edge_ranges()[RING]
    rows_e = np.sort(np.concatenate([rng.choice(rw.ne, 64, replace=False),
                                     a + rng.choice(b - a, 32, replace=False)]))
    rows_t = np.sort(rng.choice(rw.nt, 64, replace=False))
    A = oaim.Aim(rw, grid.origin, grid.h, grid.n, k0)
    A.build_near(rows_e=rows_e, rows_t=np.unique(np.concatenate([rows_t, rw.et[rows_e].ravel()])))
    ix = op.ix_matrix(rw)
    Zs, Ys = op.internal_blocks(rw, freq, mesh.sigma, ix=ix, objects=[RING])
    return dict(rw=rw, k0=k0, A=A, rows_e=rows_e, rows_t=rows_t, rng=(a, b), Z=Zs[RING],
                Y=Ys[RING], ix=ix, fd=op.fd_matrix(rw))


@pytest.fixture(scope="module")
def full():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_03991_gb300 import build
    build.build()
    mesh, grid, freq = synth.srr_array_config(2, 32)
    with ThreadPoolExecutor(1) as ex:
        fut = ex.submit(_oracle_side, mesh, grid, freq)
        ctx = api.Context(mesh, grid, freq)
        out = fut.result()
    out["ctx"] = ctx
    return out


def test_full_setup_state(full):
    """The sparse internal operator is built for all 1024 rings and in use, as in the bench."""
    ctx = full["ctx"]
    assert ctx.nobj == 1024 and ctx.ne == 933888 and ctx.nt == 622592
    sp = ctx.sparse_internal
    assert sp["objects"] == 1024 and sp["on"] and sp["check"] < 1e-8


@pytest.mark.parametrize("prec,tol", [(api.BEM_C32, 1e-5), (api.BEM_C64, 1e-11)])
def test_full_LA_LPhi_rows(full, prec, tol):
    ctx, A, re, rt = full["ctx"], full["A"], full["rows_e"], full["rows_t"]
    j = synth.rand_cvec(ctx.ne, 21)
    q = synth.rand_cvec(ctx.nt, 22)
    npdt = np.complex64 if prec == api.BEM_C32 else np.complex128
    ya = ctx.matvec(torch.from_numpy(j.astype(npdt)).cuda(), which=api.AIM_OP_LA, prec=prec)
    yp = ctx.matvec(torch.from_numpy(q.astype(npdt)).cuda(), which=api.AIM_OP_LPHI, prec=prec)
    ref_a = (A.far_A(j) + A.LNR_A @ j)[re]
    ref_p = (A.far_P(q) + A.LNR_P @ q)[rt]
    ya, yp = ya.cpu().numpy()[re], yp.cpu().numpy()[rt]
    assert rel(ya, ref_a) < tol and max_rel(ya, ref_a) < 3 * tol
    assert rel(yp, ref_p) < tol and max_rel(yp, ref_p) < 3 * tol


@pytest.mark.parametrize("prec,tol_z,tol_y", [(api.BEM_C32, 1e-5, 1e-5), (api.BEM_C64, 1e-10, 1e-6)])
def test_full_internal_rows(full, prec, tol_z, tol_y):
    """e = Z_s h (the sparse operator, all 1024 rings in one launch) and h_eq = Y_eq e on every
    row of the ring, against the oracle's dense Z and Y_eq of that ring."""
    ctx = full["ctx"]
    a, b = full["rng"]
    h = synth.rand_cvec(ctx.ne, 23)
    npdt = np.complex64 if prec == api.BEM_C32 else np.complex128
    e, heq = ctx.internal(torch.from_numpy(h.astype(npdt)).cuda(), prec=prec)
    eo = full["Z"] @ h[a:b]
    ho = full["Y"] @ eo
    e, heq = e.cpu().numpy()[a:b], heq.cpu().numpy()[a:b]
    assert rel(e, eo) < tol_z and max_rel(e, eo) < 3 * tol_z
    assert rel(heq, ho) < tol_y and max_rel(heq, ho) < 3 * tol_y


@pytest.mark.parametrize("case", ["both", "q0"])
@pytest.mark.parametrize("prec,tol", [(api.BEM_C32, 1e-5), (api.BEM_C64, 1e-7)])
def test_full_system_rows(full, prec, tol, case):
    """Sampled rows of both block rows of the system matvec of Eq. AEFIEoutJ for x = [h; q], h on
    the ring only, q everywhere (or q = 0: row 1 is then j k0 L^A j + I_x e alone, and the ring's
    own rows are among the sampled ones)."""
    ctx, A, rw, k0 = full["ctx"], full["A"], full["rw"], full["k0"]
    re, rt = full["rows_e"], full["rows_t"]
    a, b = full["rng"]
    h = np.zeros(ctx.ne, complex)
    h[a:b] = synth.rand_cvec(b - a, 24)
    q = synth.rand_cvec(ctx.nt, 25) if case == "both" else np.zeros(ctx.nt, complex)
    x = np.concatenate([h, q])
    npdt = np.complex64 if prec == api.BEM_C32 else np.complex128
    y = ctx.matvec(torch.from_numpy(x.astype(npdt)).cuda(), prec=prec).cpu().numpy()
    e = np.zeros(ctx.ne, complex)
    e[a:b] = full["Z"] @ h[a:b]
    j = h.copy()
    j[a:b] -= full["Y"] @ e[a:b]
    lphi_q = A.far_P(q) + A.LNR_P @ q  # exact on the triangles of the sampled edges
    y1 = 1j * k0 * (A.far_A(j) + A.LNR_A @ j) + full["ix"] @ e - full["fd"].T @ lphi_q
    y2 = full["fd"] @ j + 1j * k0 * q
    check_system(np.concatenate([y[re], y[ctx.ne + rt]]), np.concatenate([y1[re], y2[rt]]),
                 ctx.ne, tol, rows=(re, rt))
