"""Many right-hand sides through the internal blocks on the tensor cores (aim_internal_tc)
against the oracle: e_r = Z h_r and h_eq,r = Y_eq Z h_r with the oracle's dense Z and Y_eq of
every object (Eqs. MFIEinZin, EFIEeqYeq), for right-hand-side counts that take each of the four
tile widths (N = 32, 64, 128, 256 real columns), one that needs two launches (130 > 128), and
one alone. Three copper bars of 408, 432 and 456 edges: four 128-row tiles each, the last one
ragged, and K ranges (2 n = 816, 864, 912 floats) that end inside, and on, a 32-float stage; two
short bars of 120 and 144 edges: a block smaller than one tile. Tolerance: the FP32 blocks and
FP32 accumulation, as for the FP32 block GEMV (1e-5 relative). (Its first device run, on the
short bars with 5 and 33 right-hand sides, agreed with the block GEMV to 2e-6.)"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import operators as op  # noqa: E402
from oracle.rwg import from_mesh  # noqa: E402
from paper_2108_03991_gb300 import api, synth  # noqa: E402
from syscheck import max_rel, rel  # noqa: E402


def _structure(mesh):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_03991_gb300 import build
    build.build()
    grid = synth.grid_box(mesh, 0.5)
    freq = 10e9
    ctx = api.Context(mesh, grid, freq)
    rw = from_mesh(mesh)
    Zs, Ys = op.internal_blocks(rw, freq, mesh.sigma)
    return dict(ctx=ctx, rw=rw, Z=Zs, Y=Ys)


@pytest.fixture(scope="module")
def bars():
    return _structure(synth.small_bars(3, 8.0))


@pytest.fixture(scope="module")
def short_bars():
    return _structure(synth.small_bars(2, 2.0))


def _apply(b, blocks, H):
    """The oracle's block-diagonal product on the columns of H ([ne, R])."""
    out = np.zeros_like(H, dtype=np.complex128)
    for i, (lo, hi) in enumerate(b["rw"].obj_edge_ranges()):
        out[lo:hi] = blocks[i] @ H[lo:hi]
    return out


def _check(b, nrhs):
    ctx = b["ctx"]
    H = np.stack([synth.rand_cvec(ctx.ne, 300 + r) for r in range(nrhs)], axis=1)
    h = torch.from_numpy(np.ascontiguousarray(H.T).astype(np.complex64)).cuda().reshape(-1)
    e, heq = ctx.internal_tc(h, nrhs=nrhs)
    torch.cuda.synchronize()
    assert ctx.tensor_core_status()["wait_timed_out"] is False
    e = e.cpu().numpy().reshape(nrhs, ctx.ne).T
    heq = heq.cpu().numpy().reshape(nrhs, ctx.ne).T
    eo = _apply(b, b["Z"], H)
    # h_eq = C h against the oracle's Y_eq (Z h): C = Y_eq Z is formed in FP64 from the set-up's
    # Y_eq (1e-6 from the oracle's) and rounded to FP32. (Against Y_eq applied to this e the
    # product's own error in e would count again, about four times over, through Y_eq.)
    ho = _apply(b, b["Y"], eo)
    for r in range(nrhs):
        assert rel(e[:, r], eo[:, r]) < 1e-5 and max_rel(e[:, r], eo[:, r]) < 3e-5, r
        assert rel(heq[:, r], ho[:, r]) < 1e-5, r


@pytest.mark.parametrize("nrhs", [1, 16, 17, 33, 65, 130])
def test_tensor_core_internal_products(bars, nrhs):
    assert [hi - lo for lo, hi in bars["rw"].obj_edge_ranges()] == [408, 432, 456]
    _check(bars, nrhs)


@pytest.mark.parametrize("nrhs", [5, 130])
def test_tensor_core_block_below_one_tile(short_bars, nrhs):
    assert [hi - lo for lo, hi in short_bars["rw"].obj_edge_ranges()] == [120, 144]
    _check(short_bars, nrhs)


def test_tensor_core_matches_block_gemv(bars):
    """The same products through the block GEMV (internal_apply, four right-hand sides a
    launch) and through the tensor cores agree to FP32 rounding; either output alone."""
    ctx = bars["ctx"]
    nrhs = 24
    h = torch.from_numpy(np.concatenate([synth.rand_cvec(ctx.ne, 400 + r) for r in range(nrhs)])
                         .astype(np.complex64)).cuda()
    eg, hg = ctx.internal(h, nrhs=nrhs)
    et, _ = ctx.internal_tc(h, nrhs=nrhs, want_heq=False)
    _, ht = ctx.internal_tc(h, nrhs=nrhs, want_e=False)
    eg, hg, et, ht = (v.cpu().numpy() for v in (eg, hg, et, ht))
    assert rel(et, eg) < 1e-5 and rel(ht, hg) < 1e-5


def test_tensor_core_forms_agree(short_bars):
    """aim_tc_variant 1 (the raw right-hand sides packed and split in shared memory) gives the
    same products as form 0 (hi and lo packed in device memory): the same arithmetic, the same
    bits; 5 and 33 right-hand sides."""
    ctx = short_bars["ctx"]
    try:
        for nrhs in (5, 33):
            h = torch.from_numpy(np.concatenate([synth.rand_cvec(ctx.ne, 500 + r) for r in range(nrhs)])
                                 .astype(np.complex64)).cuda()
            out = []
            for v in (0, 1):
                ctx.tc_variant(v)
                e, heq = ctx.internal_tc(h, nrhs=nrhs)
                out.append((e.cpu().numpy(), heq.cpu().numpy()))
            assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
        assert ctx.tensor_core_status()["wait_timed_out"] is False
    finally:
        ctx.tc_variant(0)
