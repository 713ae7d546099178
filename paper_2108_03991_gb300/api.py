"""Thin ctypes binding of libbem_aim.so (argument marshalling only).

Every computation runs in the CUDA library; device buffers are torch tensors (complex64 for
BEM_C32, complex128 for BEM_C64) and the current torch stream is passed through. Loading fails
loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

BEM_C32, BEM_C64 = 0, 1
AIM_OP_LA, AIM_OP_LPHI, AIM_OP_SYSTEM, AIM_OP_EXT = 0, 1, 2, 3
BEM_OK, BEM_ENOCONV = 0, 1
ERRORS = {-1: "BEM_EINVAL", -2: "BEM_EMESH", -3: "BEM_EGRID", -4: "BEM_ENOMEM",
          -5: "BEM_ECUDA", -6: "BEM_ESOLVER"}
LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libbem_aim.so")

SYMBOLS = ["aim_setup", "aim_destroy", "bem_last_error", "aim_info", "aim_matvec",
           "internal_apply", "aim_conv", "bem_blockdiag_gemv", "aim_export",
           "bem_rhs_plane_wave", "bem_solve", "bem_part_schedule", "bem_blockdiag_gemv_noalloc",
           "bem_precond_apply", "bem_net_init", "bem_net_weights", "bem_net_train",
           "bem_net_apply", "bem_convnet_run", "aim_gemv_select", "aim_gemv_plan",
           "aim_matvec_schedule", "aim_matvec_host", "bem_port_ring", "bem_rhs_port",
           "bem_port_current", "bem_port_matrix", "bem_farfield", "aim_matvec_batch",
           "bem_solve_batch", "bem_precond_setup", "aim_internal_sparse", "bem_rcm_order",
           "aim_internal_tc", "bem_layered_grid_tables", "aim_rows_variant",
           "bem_layered_kernel_table", "aim_tc_variant"]


class StackC(C.Structure):
    _fields_ = [("nlayer", C.c_int32), ("thickness", C.POINTER(C.c_double)),
                ("eps", C.POINTER(C.c_double)), ("top_eps", C.c_double * 2),
                ("ground", C.c_int32), ("bottom_eps", C.c_double * 2)]


class BemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Material(C.Structure):
    _fields_ = [("sigma", C.c_double), ("eps_r", C.c_double), ("mu_r", C.c_double)]


class MeshC(C.Structure):
    _fields_ = [("nv", C.c_int32), ("xyz", C.POINTER(C.c_double)), ("nt", C.c_int32),
                ("tri", C.POINTER(C.c_int32)), ("obj_of_tri", C.POINTER(C.c_int32)),
                ("nobj", C.c_int32), ("mat", C.POINTER(Material))]


class GridC(C.Structure):
    _fields_ = [("origin", C.c_double * 3), ("h", C.c_double * 3), ("n", C.c_int32 * 3),
                ("order", C.c_int32), ("r_near", C.c_int32)]


class SolveOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("restart", C.c_int32), ("max_iter", C.c_int32),
                ("prec_mode", C.c_int32), ("precond", C.c_int32), ("time_limit_s", C.c_double)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("resid_est", C.c_double), ("resid_true", C.c_double),
                ("seconds", C.c_double)]


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2108_03991_gb300.build")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        L.aim_setup.argtypes = [C.POINTER(MeshC), C.POINTER(GridC), d, C.POINTER(vp)]
        L.aim_destroy.argtypes = [vp]
        L.aim_destroy.restype = None
        L.bem_last_error.restype = C.c_char_p
        L.aim_info.argtypes = [vp, C.POINTER(i64), C.c_int]
        L.aim_matvec.argtypes = [vp, C.c_int, vp, vp, C.c_int, vp]
        L.aim_gemv_select.argtypes = [vp, C.c_int]
        L.aim_gemv_plan.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int]
        L.aim_matvec_schedule.argtypes = [vp, C.c_int]
        L.aim_matvec_host.argtypes = [vp, C.c_int, vp, vp, C.c_int, C.c_int, vp]
        L.aim_matvec_batch.argtypes = [vp, vp, vp, C.c_int, C.c_int, vp]
        L.bem_solve_batch.argtypes = [vp, vp, vp, C.c_int, C.POINTER(SolveOpts), C.POINTER(SolveInfo), vp]
        L.bem_port_ring.argtypes = [vp, C.c_int, C.c_int, d, d, C.POINTER(i32), C.POINTER(d), C.c_int]
        L.bem_rhs_port.argtypes = [vp, C.c_int, C.POINTER(i32), C.POINTER(d), d, vp, C.c_int, vp]
        L.bem_port_current.argtypes = [vp, C.c_int, C.POINTER(i32), C.POINTER(d), vp, C.c_int,
                                       C.POINTER(d), vp]
        L.bem_farfield.argtypes = [vp, vp, C.c_int, C.c_int, C.POINTER(d), C.POINTER(d), vp]
        L.internal_apply.argtypes = [vp, vp, vp, vp, C.c_int, C.c_int, vp]
        L.aim_internal_tc.argtypes = [vp, vp, vp, vp, C.c_int, vp]
        L.aim_rows_variant.argtypes = [vp, C.c_int]
        L.aim_tc_variant.argtypes = [vp, C.c_int]
        L.bem_layered_kernel_table.argtypes = [C.POINTER(StackC), d, C.c_int, C.c_int, C.c_int,
                                               C.c_int, C.POINTER(d), C.c_int, C.POINTER(d),
                                               C.POINTER(d)]
        L.bem_layered_grid_tables.argtypes = [C.POINTER(StackC), d, C.POINTER(d), C.POINTER(d),
                                              C.POINTER(i32), C.c_int, C.POINTER(d), C.POINTER(d)]
        L.aim_conv.argtypes = [vp, vp, vp, C.c_int, C.c_int, vp]
        L.bem_blockdiag_gemv.argtypes = [C.c_int, C.POINTER(i32), vp, vp, vp, C.c_int, C.c_int, vp]
        L.bem_blockdiag_gemv_noalloc.argtypes = [C.c_int, C.POINTER(i32), vp, vp, vp, C.c_int,
                                                 C.c_int, vp]
        L.aim_export.argtypes = [vp, C.c_int, C.c_int, vp, i64]
        L.aim_export.restype = i64
        L.bem_rhs_plane_wave.argtypes = [vp, C.POINTER(d), C.POINTER(d), vp, C.c_int, vp]
        L.bem_solve.argtypes = [vp, vp, vp, C.POINTER(SolveOpts), C.POINTER(SolveInfo), vp]
        L.bem_port_matrix.argtypes = [vp, C.c_int, C.POINTER(i32), C.POINTER(i32), C.POINTER(d),
                                      C.POINTER(SolveOpts), C.POINTER(d), C.POINTER(SolveInfo), vp]
        L.bem_precond_apply.argtypes = [vp, vp, vp, C.c_int, vp]
        L.bem_precond_setup.argtypes = [vp, C.c_int]
        L.aim_internal_sparse.argtypes = [vp, C.c_int]
        fp = C.POINTER(C.c_float)
        L.bem_net_init.argtypes = [vp, C.c_uint64]
        L.bem_net_weights.argtypes = [vp, fp, i64, C.c_int]
        L.bem_net_weights.restype = i64
        L.bem_net_train.argtypes = [vp, C.c_int, C.c_int, C.c_float, C.c_uint64, fp, vp]
        L.bem_net_apply.argtypes = [vp, vp, vp, C.c_int, vp]
        L.bem_convnet_run.argtypes = [C.c_int, C.c_int, C.c_int, fp, vp, vp, vp, fp, vp, vp]
        L.bem_part_schedule.argtypes = [C.c_int, C.POINTER(d), C.c_int, C.c_int, C.POINTER(i32)]
        L.bem_part_schedule.restype = d
        _LIB = L
    return _LIB


def _check(rc):
    if rc < 0:
        raise BemError(rc, lib().bem_last_error().decode())
    return rc


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t, dtype=None):
    import torch
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected {dtype}, got {t.dtype}")
    return C.c_void_p(t.data_ptr())


def cdtype(prec):
    import torch
    return torch.complex64 if prec == BEM_C32 else torch.complex128


def _stack(layers, top_eps, ground, bottom_eps):
    """The bem_stack of a layer list [(thickness um, complex eps_r)] bottom-up, with the arrays
    it points to (keep them alive while it is used)."""
    th = np.array([float(t) for t, _ in layers], dtype=np.float64)
    ep = np.array([[complex(e).real, complex(e).imag] for _, e in layers], dtype=np.float64)
    te, be = complex(top_eps), complex(bottom_eps)
    st = StackC(len(layers), th.ctypes.data_as(C.POINTER(C.c_double)),
                ep.ctypes.data_as(C.POINTER(C.c_double)), (C.c_double * 2)(te.real, te.imag),
                1 if ground else 0, (C.c_double * 2)(be.real, be.imag))
    return st, (th, ep)


def layered_grid_tables(layers, freq, origin, h, n, kind, top_eps=1.0, ground=True,
                        bottom_eps=1.0):
    """bem_layered_grid_tables: the Toeplitz and Hankel tables of the grid step inside one layer
    of a stratified background. layers: [(thickness um, complex eps_r)] bottom-up; kind 0
    G^A_xx, 1 G^A_zz, 2 G^Phi. Returns (T, H), complex arrays [2 n_z - 1, n_y, n_x]."""
    st, keep = _stack(layers, top_eps, ground, bottom_eps)
    nx, ny, nz = (int(v) for v in n)
    T = np.zeros((2 * nz - 1, ny, nx), dtype=np.complex128)
    H = np.zeros_like(T)
    o = (C.c_double * 3)(*[float(v) for v in origin])
    hh = (C.c_double * 3)(*[float(v) for v in h])
    nn = (C.c_int32 * 3)(nx, ny, nz)
    _check(lib().bem_layered_grid_tables(C.byref(st), float(freq), o, hh, nn, int(kind),
                                         T.ctypes.data_as(C.POINTER(C.c_double)),
                                         H.ctypes.data_as(C.POINTER(C.c_double))))
    return T, H


def layered_kernel_table(layers, freq, layer, kind, part, rho, arg, top_eps=1.0, ground=True,
                         bottom_eps=1.0):
    """bem_layered_kernel_table: the reflected part (part 0 Toeplitz at arg = z - z', 1 Hankel
    at arg = z + z') of one of a layer's Green's functions at rho x arg. Returns a complex array
    [len(arg), len(rho)]."""
    st, keep = _stack(layers, top_eps, ground, bottom_eps)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    arg = np.ascontiguousarray(arg, dtype=np.float64)
    out = np.zeros((arg.size, rho.size), dtype=np.complex128)
    _check(lib().bem_layered_kernel_table(C.byref(st), float(freq), int(layer), int(kind), int(part),
                                          rho.size, rho.ctypes.data_as(C.POINTER(C.c_double)),
                                          arg.size, arg.ctypes.data_as(C.POINTER(C.c_double)),
                                          out.ctypes.data_as(C.POINTER(C.c_double))))
    return out


def part_schedule(W, P, p_cutoff=20):
    W = np.ascontiguousarray(W, dtype=np.float64)
    Pi = np.zeros(W.size, dtype=np.int32)
    cmax = lib().bem_part_schedule(W.size, W.ctypes.data_as(C.POINTER(C.c_double)), int(P),
                                   int(p_cutoff), Pi.ctypes.data_as(C.POINTER(C.c_int32)))
    if cmax < 0:
        raise BemError(-1, lib().bem_last_error().decode())
    return Pi, cmax


def rcm_order(rowptr, cols):
    """Reverse Cuthill-McKee order of a symmetric CSR pattern (bem_rcm_order): order[r] is the
    vertex at position r."""
    rp = np.ascontiguousarray(rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(cols, dtype=np.int32)
    n = rp.size - 1
    order = np.zeros(max(n, 0), dtype=np.int32)
    L = lib()
    L.bem_rcm_order.argtypes = [C.c_int, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                C.POINTER(C.c_int32)]
    _check(L.bem_rcm_order(n, rp.ctypes.data_as(C.POINTER(C.c_int32)),
                           ci.ctypes.data_as(C.POINTER(C.c_int32)),
                           order.ctypes.data_as(C.POINTER(C.c_int32))))
    return order


def blockdiag_gemv(sizes, A, x, y, nrhs=1, prec=BEM_C32):
    n = np.ascontiguousarray(sizes, dtype=np.int32)
    dt = cdtype(prec)
    _check(lib().bem_blockdiag_gemv(n.size, n.ctypes.data_as(C.POINTER(C.c_int32)), _ptr(A, dt),
                                    _ptr(x, dt), _ptr(y, dt), int(nrhs), prec, _stream()))
    return y


def blockdiag_gemv_noalloc(sizes, A, x, y, nrhs=1, prec=BEM_C32):
    """bem_blockdiag_gemv without any device allocation (fixed scratch inside the library)."""
    n = np.ascontiguousarray(sizes, dtype=np.int32)
    dt = cdtype(prec)
    _check(lib().bem_blockdiag_gemv_noalloc(n.size, n.ctypes.data_as(C.POINTER(C.c_int32)),
                                            _ptr(A, dt), _ptr(x, dt), _ptr(y, dt), int(nrhs),
                                            prec, _stream()))
    return y


def convnet_run(w, x, gout=None):
    """The learned-correction network alone (BF16 weights/activations, FP32 sums).
    w: numpy float32 weights (all layers); x: CUDA float32 [8, nz, ny, nx]; gout: optional
    CUDA float32 [8, nz, ny, nx]. Returns out (CUDA), gw (numpy or None), gx (CUDA or None)."""
    import torch
    w = np.ascontiguousarray(w, dtype=np.float32)
    _, nz, ny, nx = x.shape
    out = torch.empty_like(x)
    gw = np.zeros_like(w) if gout is not None else None
    gx = torch.empty_like(x) if gout is not None else None
    fp = C.POINTER(C.c_float)
    _check(lib().bem_convnet_run(nx, ny, nz, w.ctypes.data_as(fp), _ptr(x, torch.float32),
                                 _ptr(gout, torch.float32) if gout is not None else None,
                                 _ptr(out, torch.float32),
                                 gw.ctypes.data_as(fp) if gw is not None else None,
                                 _ptr(gx, torch.float32) if gx is not None else None, _stream()))
    return out, gw, gx


def pack_blocks(blocks, dtype):
    """Row-major blocks with leading dimension n rounded up to 4, concatenated (numpy)."""
    out = []
    for B in blocks:
        n = B.shape[0]
        ld = (n + 3) // 4 * 4
        P = np.zeros((n, ld), dtype=dtype)
        P[:, :n] = B
        out.append(P.ravel())
    return np.concatenate(out)


class Context:
    """One aim_setup context on the current CUDA device."""

    def __init__(self, mesh, grid, freq, r_near=2):
        L = lib()
        self._keep = []
        xyz = np.ascontiguousarray(mesh.verts, dtype=np.float64)
        tri = np.ascontiguousarray(mesh.tris, dtype=np.int32)
        obj = np.ascontiguousarray(mesh.obj, dtype=np.int32)
        mats = (Material * mesh.nobj)(*[Material(float(s), 1.0, 1.0) for s in mesh.sigma])
        self._keep += [xyz, tri, obj, mats]
        m = MeshC(xyz.shape[0], xyz.ctypes.data_as(C.POINTER(C.c_double)), tri.shape[0],
                  tri.ctypes.data_as(C.POINTER(C.c_int32)), obj.ctypes.data_as(C.POINTER(C.c_int32)),
                  mesh.nobj, mats)
        g = GridC((C.c_double * 3)(*grid.origin), (C.c_double * 3)(*grid.h),
                  (C.c_int32 * 3)(*[int(v) for v in grid.n]), 2, int(r_near))
        h = C.c_void_p()
        _check(L.aim_setup(C.byref(m), C.byref(g), float(freq), C.byref(h)))
        self.h = h
        self._read_info()

    def _read_info(self):
        info = (C.c_int64 * 45)()
        _check(lib().aim_info(self.h, info, 45))
        self.info = list(info)
        self.ne, self.nt, self.nobj = info[0], info[1], info[2]
        self.n = self.ne + self.nt
        self.grid_n = tuple(info[3:6])
        self.padded = tuple(info[6:9])
        self.nnz_A, self.nnz_P = info[9], info[10]
        self.zy_bytes_c32 = info[11]
        self.ng = int(np.prod(self.grid_n))
        self.gemv_ctas, self.gemv_split = info[13], info[14]
        self.gemv_unroll = info[15]
        self.gemv_tune_ns = {"plain": info[16], "staged": info[17]}
        self.gemv_tune_rejected = info[18]
        self.gemv_kind = info[19]  # 0 row plan, 1 flat, 2 staged, 3 stream, 5 and 6 task lists
        self.gemv_cps = info[20]
        self.matvec_mode = info[21]  # schedule of e = Z h (aim_matvec_schedule)
        self.setup_stage_s = dict(zip(
            ("geometry", "stencils", "internal_ki", "internal_k0", "lu", "yz", "near", "ghat",
             "gemv_tune", "schedule_tune"), (v * 1e-6 for v in info[22:32])))
        # last block-diagonal preconditioner build: seconds, precision (-1: none yet), blocks
        # built in FP64, largest FP32 block check (None: none ran)
        self.precond_build = {"seconds": info[32] * 1e-6, "prec": info[33], "fp64_blocks": info[34],
                              "check": None if info[35] < 0 else info[35] * 1e-12}
        # sparse internal operator at high frequency (aim_internal_sparse)
        self.sparse_internal = {"setup_s": info[36] * 1e-6, "objects": info[37], "on": bool(info[38]),
                                "band": info[39], "bytes_c32": info[40],
                                "check": None if info[41] < 0 else info[41] * 1e-15,
                                "wait_timed_out": bool(info[42])}
        # many right-hand sides on the tensor cores (aim_internal_tc): calls, and whether a
        # bounded wait timed out (None before the first call)
        self.tensor_core = {"calls": info[43], "wait_timed_out": None if info[44] < 0 else bool(info[44])}

    # ---- ports and far field ---------------------------------------------------------
    def port_ring(self, obj, axis, coord, tol=1e-6):
        """Edges (library order) and crossing signs of a delta-gap ring of object `obj` in the
        plane x_axis = coord (um)."""
        L = lib()
        n = _check(L.bem_port_ring(self.h, int(obj), int(axis), float(coord), float(tol), None,
                                   None, 0))
        e = np.zeros(n, dtype=np.int32)
        s = np.zeros(n, dtype=np.float64)
        _check(L.bem_port_ring(self.h, int(obj), int(axis), float(coord), float(tol),
                               e.ctypes.data_as(C.POINTER(C.c_int32)),
                               s.ctypes.data_as(C.POINTER(C.c_double)), n))
        return e, s

    def rhs_port(self, edges, signs, v_gap=1.0, prec=BEM_C64, device="cuda"):
        import torch
        e = np.ascontiguousarray(edges, dtype=np.int32)
        s = np.ascontiguousarray(signs, dtype=np.float64)
        b = torch.empty(self.n, dtype=cdtype(prec), device=device)
        _check(lib().bem_rhs_port(self.h, len(e), e.ctypes.data_as(C.POINTER(C.c_int32)),
                                  s.ctypes.data_as(C.POINTER(C.c_double)), float(v_gap),
                                  _ptr(b), prec, _stream()))
        return b

    def port_current(self, x, edges, signs, prec=BEM_C64):
        """Port current in amperes (complex) of the solution x = [h; q]."""
        e = np.ascontiguousarray(edges, dtype=np.int32)
        s = np.ascontiguousarray(signs, dtype=np.float64)
        out = (C.c_double * 2)()
        _check(lib().bem_port_current(self.h, len(e), e.ctypes.data_as(C.POINTER(C.c_int32)),
                                      s.ctypes.data_as(C.POINTER(C.c_double)), _ptr(x, cdtype(prec)),
                                      prec, out, _stream()))
        return complex(out[0], out[1])

    def port_matrix(self, rings, tol=1e-6, restart=100, max_iter=1000, prec_mode=BEM_C64,
                    precond=1, time_limit_s=0.0):
        """Port admittance matrix Y [nport, nport] (siemens) from one solve per port (unit gap
        voltage, the others shorted; see bem_port_matrix). rings: [(edges, signs), ...] from
        port_ring. Returns (Y, status, [iterations per column])."""
        n = np.array([len(e) for e, _ in rings], dtype=np.int32)
        e = np.ascontiguousarray(np.concatenate([np.asarray(e) for e, _ in rings]), dtype=np.int32)
        s = np.ascontiguousarray(np.concatenate([np.asarray(s) for _, s in rings]), dtype=np.float64)
        o = SolveOpts(tol, restart, max_iter, prec_mode, int(precond), time_limit_s)
        infos = (SolveInfo * len(n))()
        Y = np.zeros((len(n), len(n), 2))
        rc = _check(lib().bem_port_matrix(self.h, len(n), n.ctypes.data_as(C.POINTER(C.c_int32)),
                                          e.ctypes.data_as(C.POINTER(C.c_int32)),
                                          s.ctypes.data_as(C.POINTER(C.c_double)), C.byref(o),
                                          Y.ctypes.data_as(C.POINTER(C.c_double)), infos, _stream()))
        return Y[..., 0] + 1j * Y[..., 1], rc, [inf.iters for inf in infos]

    def farfield(self, x, rhat, prec=BEM_C64):
        """Radiation vector N(rhat) [ndir, 3] (complex) of the solution x = [h; q]."""
        r = np.ascontiguousarray(np.atleast_2d(rhat), dtype=np.float64)
        out = np.zeros((r.shape[0], 6))
        _check(lib().bem_farfield(self.h, _ptr(x, cdtype(prec)), prec, r.shape[0],
                                  r.ctypes.data_as(C.POINTER(C.c_double)),
                                  out.ctypes.data_as(C.POINTER(C.c_double)), _stream()))
        return out[:, 0::2] + 1j * out[:, 1::2]

    def gemv_plan(self, kind, ctas_per_sm, split=1, unroll=4):
        """Set the FP32 block-GEMV launch explicitly (see aim_gemv_plan)."""
        _check(lib().aim_gemv_plan(self.h, int(kind), int(ctas_per_sm), int(split), int(unroll)))
        self._read_info()

    def matvec_schedule(self, mode=-1):
        """Schedule of e = Z h in the system matvec (see aim_matvec_schedule; -1 = tuned)."""
        _check(lib().aim_matvec_schedule(self.h, int(mode)))
        self._read_info()

    def gemv_select(self, kind):
        """FP32 block-GEMV launch: 0 autotuned choice, 1 best plain, 2 best bulk-copy staged."""
        _check(lib().aim_gemv_select(self.h, int(kind)))
        self._read_info()

    def close(self):
        if self.h:
            lib().aim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- products ----------------------------------------------------------------
    def matvec(self, x, y=None, which=AIM_OP_SYSTEM, prec=BEM_C32):
        import torch
        n = {AIM_OP_LA: self.ne, AIM_OP_LPHI: self.nt, AIM_OP_SYSTEM: self.n, AIM_OP_EXT: self.n}[which]
        if y is None:
            y = torch.empty(n, dtype=cdtype(prec), device=x.device)
        if x.numel() != n or y.numel() != n:
            raise ValueError("vector length mismatch")
        _check(lib().aim_matvec(self.h, which, _ptr(x, cdtype(prec)), _ptr(y, cdtype(prec)), prec,
                                _stream()))
        return y

    def matvec_batch(self, x, y=None, prec=BEM_C32):
        """System matvec of nrhs = x.numel() / N right-hand sides at once (aim_matvec_batch);
        x, y: device tensors of nrhs * N entries (or [nrhs, N])."""
        import torch
        if x.numel() % self.n:
            raise ValueError("vector length mismatch")
        if y is None:
            y = torch.empty_like(x)
        _check(lib().aim_matvec_batch(self.h, _ptr(x, cdtype(prec)), _ptr(y, cdtype(prec)),
                                      x.numel() // self.n, prec, _stream()))
        return y

    def matvec_host(self, x, y=None, which=AIM_OP_SYSTEM, prec=BEM_C32):
        """y_i = A x_i for the rows of the host (CPU) tensor x [nvec, n], copies overlapped
        with the products (aim_matvec_host); pin x and y for asynchronous copies. Ordered on the
        current stream; synchronise it before reading y."""
        import torch
        n = {AIM_OP_LA: self.ne, AIM_OP_LPHI: self.nt, AIM_OP_SYSTEM: self.n, AIM_OP_EXT: self.n}[which]
        if x.device.type != "cpu" or x.dtype != cdtype(prec) or not x.is_contiguous():
            raise ValueError("x must be a contiguous CPU tensor of the precision's complex type")
        if x.numel() % n:
            raise ValueError("vector length mismatch")
        if y is None:
            y = torch.empty(x.shape, dtype=x.dtype, pin_memory=x.is_pinned())
        if y.shape != x.shape or y.dtype != x.dtype or y.device.type != "cpu" or not y.is_contiguous():
            raise ValueError("y must match x")
        _check(lib().aim_matvec_host(self.h, which, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                     x.numel() // n, prec, _stream()))
        return y

    def internal(self, h, e=None, heq=None, nrhs=1, prec=BEM_C32, want_heq=True, want_e=True):
        """e = Z h and h_eq = Y_eq Z h (internal_apply); either may be left out."""
        import torch
        dt = cdtype(prec)
        if e is None and want_e:
            e = torch.empty_like(h)
        if heq is None and want_heq:
            heq = torch.empty_like(h)
        _check(lib().internal_apply(self.h, _ptr(h, dt), _ptr(e, dt) if e is not None else None,
                                    _ptr(heq, dt) if heq is not None else None, int(nrhs), prec,
                                    _stream()))
        return e, heq

    def internal_tc(self, h, e=None, heq=None, nrhs=1, want_heq=True, want_e=True):
        """e_r = Z h_r and h_eq,r = C h_r for nrhs complex64 right-hand sides at once on the
        tensor cores (aim_internal_tc); either may be left out."""
        import torch
        dt = torch.complex64
        if e is None and want_e:
            e = torch.empty_like(h)
        if heq is None and want_heq:
            heq = torch.empty_like(h)
        _check(lib().aim_internal_tc(self.h, _ptr(h, dt), _ptr(e, dt) if e is not None else None,
                                     _ptr(heq, dt) if heq is not None else None, int(nrhs),
                                     _stream()))
        return e, heq

    def tc_variant(self, variant):
        """Form of the tensor-core product (aim_tc_variant): 0 hi/lo packed, 1 raw B split in
        shared memory."""
        _check(lib().aim_tc_variant(self.h, int(variant)))

    def tensor_core_status(self):
        """aim_internal_tc's calls and wait status (reading it synchronises the device)."""
        self._read_info()
        return self.tensor_core

    def conv(self, sigma, phi=None, ncomp=1, prec=BEM_C32):
        import torch
        if phi is None:
            phi = torch.empty_like(sigma)
        _check(lib().aim_conv(self.h, _ptr(sigma, cdtype(prec)), _ptr(phi, cdtype(prec)), int(ncomp),
                              prec, _stream()))
        return phi

    def rhs_plane_wave(self, pol=(1.0, 0.0, 0.0), khat=(0.0, 0.0, 1.0), prec=BEM_C64, device="cuda"):
        import torch
        b = torch.empty(self.n, dtype=cdtype(prec), device=device)
        p = (C.c_double * 3)(*pol)
        k = (C.c_double * 3)(*khat)
        _check(lib().bem_rhs_plane_wave(self.h, p, k, _ptr(b), prec, _stream()))
        return b

    def rows_variant(self, variant):
        """Form of the row kernels (aim_rows_variant): 0 the default, 1 predicated near-region
        sums (the same bits), 2 the same with two interpolation rows per warp."""
        _check(lib().aim_rows_variant(self.h, int(variant)))

    def internal_sparse(self, on):
        """Use the sparse internal operator Z_s (on=True, when aim_setup built one) or the dense Z
        for e = Z h; returns sparse_internal."""
        _check(lib().aim_internal_sparse(self.h, int(bool(on))))
        self._read_info()
        return self.sparse_internal

    def precond_setup(self, build_prec=BEM_C32):
        """Build (or rebuild) the block-diagonal preconditioner's inverses in complex FP32
        (each block checked; FP64 where the check fails) or FP64; returns precond_build."""
        _check(lib().bem_precond_setup(self.h, build_prec))
        self._read_info()
        return self.precond_build

    def precond(self, r, u=None, prec=BEM_C32):
        """u = M_bd r, the block-diagonal preconditioner (built on first use)."""
        import torch
        if u is None:
            u = torch.empty_like(r)
        _check(lib().bem_precond_apply(self.h, _ptr(r, cdtype(prec)), _ptr(u, cdtype(prec)), prec,
                                       _stream()))
        return u

    # ---- learned correction ---------------------------------------------------------
    def net_init(self, seed=0):
        _check(lib().bem_net_init(self.h, int(seed)))

    def net_weights(self, w=None):
        """Return the weights (numpy float32), or set them when w is given."""
        L = lib()
        n = _check(L.bem_net_weights(self.h, None, 0, 0))
        fp = C.POINTER(C.c_float)
        if w is None:
            out = np.zeros(n, dtype=np.float32)
            _check(L.bem_net_weights(self.h, out.ctypes.data_as(fp), n, 0))
            return out
        w = np.ascontiguousarray(w, dtype=np.float32)
        _check(L.bem_net_weights(self.h, w.ctypes.data_as(fp), w.size, 1))
        return w

    def net_train(self, steps, batch=8, lr=1e-3, seed=0):
        losses = np.zeros(steps, dtype=np.float32)
        _check(lib().bem_net_train(self.h, int(steps), int(batch), float(lr), int(seed),
                                   losses.ctypes.data_as(C.POINTER(C.c_float)), _stream()))
        return losses

    def net_apply(self, r, z=None, correction_only=False):
        """z = M_bd r + W net(P r) (or W net(P r) alone), complex64 device vectors."""
        import torch
        if z is None:
            z = torch.empty_like(r)
        _check(lib().bem_net_apply(self.h, _ptr(r, torch.complex64), _ptr(z, torch.complex64),
                                   int(bool(correction_only)), _stream()))
        return z

    def solve(self, b, x=None, tol=1e-6, restart=100, max_iter=1000, prec_mode=BEM_C64,
              time_limit_s=0.0, precond=0):
        import torch
        if x is None:
            x = torch.zeros_like(b)
        o = SolveOpts(tol, restart, max_iter, prec_mode, int(precond), time_limit_s)
        inf = SolveInfo()
        rc = _check(lib().bem_solve(self.h, _ptr(b, torch.complex128), _ptr(x, torch.complex128),
                                    C.byref(o), C.byref(inf), _stream()))
        if precond:
            self._read_info()  # the first preconditioned solve builds the preconditioner
        return x, {"status": rc, "iters": inf.iters, "resid_est": inf.resid_est,
                   "resid_true": inf.resid_true, "seconds": inf.seconds}

    def solve_batch(self, b, x=None, tol=1e-6, restart=100, max_iter=1000, prec_mode=BEM_C64,
                    time_limit_s=0.0, precond=0):
        """bem_solve_batch: b [nrhs * N] complex128 device vectors solved in lockstep."""
        import torch
        if b.numel() % self.n:
            raise ValueError("vector length mismatch")
        nrhs = b.numel() // self.n
        if x is None:
            x = torch.zeros_like(b)
        o = SolveOpts(tol, restart, max_iter, prec_mode, int(precond), time_limit_s)
        infos = (SolveInfo * nrhs)()
        rc = _check(lib().bem_solve_batch(self.h, _ptr(b, torch.complex128), _ptr(x, torch.complex128),
                                          nrhs, C.byref(o), infos, _stream()))
        return x, rc, [{"iters": i.iters, "resid_est": i.resid_est, "resid_true": i.resid_true,
                        "seconds": i.seconds} for i in infos]

    # ---- set-up products (host copies) ----------------------------------------------
    def _export(self, what, index=0):
        L = lib()
        need = L.aim_export(self.h, what, index, None, 0)
        _check(need)
        buf = np.empty(need, dtype=np.uint8)
        _check(L.aim_export(self.h, what, index, buf.ctypes.data_as(C.c_void_p), need))
        return buf

    def gemv_tune_table(self):
        """The set-up GEMV autotuner's candidates: rows (kind 0 row plan / 1 flat / 2 staged,
        CTAs per SM, column parts per row, loads in flight per lane, ns per launch or -1)."""
        return self._export(8).view(np.float32).reshape(-1, 5)

    def Z(self, i):
        b = self._export(0, i).view(np.complex128)
        n = int(round(np.sqrt(b.size)))
        return b.reshape(n, n)

    def Y(self, i):
        b = self._export(1, i).view(np.complex128)
        n = int(round(np.sqrt(b.size)))
        return b.reshape(n, n)

    def LK(self, i, background=False):
        """L_k and K_k + I_x/2 of object i as the set-up forms them before its LU solve
        (k = k_i, or k0 with background=True)."""
        idx = 2 * i + (1 if background else 0)
        Lb = self._export(9, idx).view(np.complex128)
        Kb = self._export(10, idx).view(np.complex128)
        n = int(round(np.sqrt(Lb.size)))
        return Lb.reshape(n, n), Kb.reshape(n, n)

    def near(self, which):
        b = self._export(2 if which == "A" else 3)
        nr = (self.ne if which == "A" else self.nt) + 1
        row = b[:nr * 8].view(np.int64)
        nnz = int(row[-1])
        col = b[nr * 8:nr * 8 + nnz * 4].view(np.int32)
        val = b[nr * 8 + nnz * 4:].view(np.complex128)
        return row, col, val

    def weights(self):
        WA = self._export(4).view(np.float64).reshape(self.ne, 3, 27)
        WP = self._export(5).view(np.float64).reshape(self.nt, 27)
        return WA, WP

    def anchors(self):
        return self._export(6).view(np.int32).reshape(-1, 3)

    def edges(self):
        return self._export(7).view(np.int32).reshape(self.ne, 6)
