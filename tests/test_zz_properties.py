"""Properties of the device operators that hold whatever the inputs (written after the last
device run and not yet run there):

* linearity of the system matvec, A(a x + b y) = a A x + b A y;
* invariance under the order of the objects: three bars of different lengths and
  conductivities, listed 0, 1, 2 and 2, 0, 1, give the same system matvec up to the
  permutation of their unknowns (each object's edges and triangles keep their relative order;
  the work lists, near-region column order and grid accumulation order all change);
* the far part of L^A and L^Phi is symmetric (W = P^T and an even grid kernel), so the
  bilinear asymmetry x^T L y - y^T L x of the device operator is the near region's alone, the
  asymmetry of the singular quadrature, which the oracle's precorrected near matrix gives."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import aim as oaim, operators as op  # noqa: E402
from oracle.rwg import from_mesh  # noqa: E402
from paper_2108_03991_gb300 import api, synth  # noqa: E402
from syscheck import rel  # noqa: E402

SIGMA = [5.8e7, 4.1e7, 3.5e7]


def _bars(order):
    parts = [synth.box((i * 2.5, 0.0, 0.0), (1.0, 1.0, 2.0 + 0.5 * i),
                       (2, 2, round((2.0 + 0.5 * i) / 0.5))) for i in range(3)]
    return synth.merge([parts[i] for i in order], [SIGMA[i] for i in order])


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_03991_gb300 import build
    build.build()


def _dt(prec):
    return np.complex64 if prec == api.BEM_C32 else np.complex128


# tolerances: a few times the products' own rounding (FP32 parity with the oracle is 1e-5;
# j = h - C h and the FFTs cancel), far below what a broken term or object mix-up leaves
@pytest.mark.parametrize("prec,tol", [(api.BEM_C32, 5e-5), (api.BEM_C64, 1e-10)])
def test_system_matvec_is_linear(dev, prec, tol):
    mesh = _bars([0, 1, 2])
    ctx = api.Context(mesh, synth.grid_box(mesh, 0.5), 10e9)
    x, y = synth.rand_cvec(ctx.n, 31), synth.rand_cvec(ctx.n, 32)
    a, b = 0.3 + 0.2j, -1.1 + 0.4j
    dev_ = lambda v: torch.from_numpy(v.astype(_dt(prec))).cuda()  # noqa: E731
    Ax = ctx.matvec(dev_(x), prec=prec).cpu().numpy()
    Ay = ctx.matvec(dev_(y), prec=prec).cpu().numpy()
    Az = ctx.matvec(dev_(a * x + b * y), prec=prec).cpu().numpy()
    assert rel(Az, a * Ax + b * Ay) < tol


@pytest.mark.parametrize("prec,tol", [(api.BEM_C32, 5e-5), (api.BEM_C64, 1e-9)])
def test_object_order_invariance(dev, prec, tol):
    order_b = [2, 0, 1]
    mA, mB = _bars([0, 1, 2]), _bars(order_b)
    gA, gB = synth.grid_box(mA, 0.5), synth.grid_box(mB, 0.5)
    assert np.allclose(gA.origin, gB.origin) and np.array_equal(gA.n, gB.n)
    cA, cB = api.Context(mA, gA, 10e9), api.Context(mB, gB, 10e9)
    rA, rB = from_mesh(mA), from_mesh(mB)
    ne, nt = rA.ne, rA.nt
    # index of each of A's unknowns in B's order (each bar's edges and triangles keep their order)
    pos = {bar: order_b.index(bar) for bar in range(3)}
    pe = np.empty(ne, dtype=np.int64)
    pt = np.empty(nt, dtype=np.int64)
    for bar in range(3):
        (a0, a1), (b0, _) = rA.obj_edge_ranges()[bar], rB.obj_edge_ranges()[pos[bar]]
        pe[a0:a1] = b0 + np.arange(a1 - a0)
        (t0, t1), (s0, _) = rA.obj_tri_ranges()[bar], rB.obj_tri_ranges()[pos[bar]]
        pt[t0:t1] = s0 + np.arange(t1 - t0)
    perm = np.concatenate([pe, ne + pt])
    x = synth.rand_cvec(ne + nt, 33)
    xB = np.empty_like(x)
    xB[perm] = x
    yA = cA.matvec(torch.from_numpy(x.astype(_dt(prec))).cuda(), prec=prec).cpu().numpy()
    yB = cB.matvec(torch.from_numpy(xB.astype(_dt(prec))).cuda(), prec=prec).cpu().numpy()
    assert rel(yB[perm], yA) < tol


def test_far_part_is_symmetric(dev):
    """x^T L y - y^T L x of the device's L^A and L^Phi (FP64) equals the same form of the
    oracle's precorrected near matrix alone (3e-4 and 1e-4 of |x^T L y| here), to 1e-8 of
    |x^T L y| (the FP64 parity bound of the two operators allows ~3e-10; a far part with W
    unequal to P^T, or an odd grid kernel, would leave a far larger asymmetry)."""
    mesh = synth.small_bars(2, 2.0)
    grid = synth.grid_box(mesh, 0.5)
    freq = 10e9
    ctx = api.Context(mesh, grid, freq)
    rw = from_mesh(mesh)
    A = oaim.Aim(rw, grid.origin, grid.h, grid.n, op.k0_of(freq)).build_near()
    for which, n, LNR in ((api.AIM_OP_LA, rw.ne, A.LNR_A), (api.AIM_OP_LPHI, rw.nt, A.LNR_P)):
        x, y = synth.rand_cvec(n, 34), synth.rand_cvec(n, 35)
        Ly = ctx.matvec(torch.from_numpy(y).cuda(), which=which, prec=api.BEM_C64).cpu().numpy()
        Lx = ctx.matvec(torch.from_numpy(x).cuda(), which=which, prec=api.BEM_C64).cpu().numpy()
        asym = x @ Ly - y @ Lx
        near = x @ (LNR @ y) - y @ (LNR @ x)
        assert abs(asym - near) <= 1e-8 * abs(x @ Ly)
