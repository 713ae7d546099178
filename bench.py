"""Benchmark: SLIM system matvecs per second on one GB300 (and N independent replicas).

Workload (the largest configuration): a 32 x 32 array of gold split-ring resonators at 1 THz
(seed 2; outer radius 20 um, width 4 um, gap 4 um with +-5% seeded size jitter, thickness 1 um,
pitch 50 um; 608 triangles per ring: 622,592 triangles, 933,888 RWG edges, 1,024 objects), AIM
grid 512 x 512 x 8 (3.137 x 3.137 x 0.5 um), order-2 stencils, near radius 2 cells. A step is
one system matrix-vector product of Eq. (AEFIEoutJ) in complex FP32 (internal blocks Z and
C = Y_eq Z, AIM projection, FFT convolution, interpolation, near region, sparse terms). Inputs
(Z and C alone are 13.6 GB) exceed the 129 MB L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--bar-array]

`--impl reference` times the FP64 CPU oracle on the host cores (a bounded sample of the same
workload, scaled to the full workload's matvec cost). `--bar-array` adds the 4 x 4 copper bar
array's numbers (solves with the learned correction, batched solves, the copper bar).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "matvecs/s (HBM roofline %) and time to 1e-6 residual, chosen vs plain, 1 GB300"
UNIT = "matvecs/s"
WORKLOAD = ("32x32 Au split-ring array (seed 2), 933888 RWG + 622592 pulse unknowns, 1 THz, "
            "AIM grid 512x512x8")
BAR_WORKLOAD = "4x4 Cu bar array (seed 0), 17832 RWG + 11888 pulse unknowns, 10 GHz, AIM 0.5 um grid"
SUB = 8  # the oracle's sample: the 8 x 8 sub-array (64 of the 1,024 rings)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.rows = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([s.strip() for s in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
                for k, nme in enumerate(names):
                    if r[3 + k].lower().startswith("active"):
                        reasons.add(nme)
            except (ValueError, IndexError):
                pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(values, device="cpu"):
    """The element-wise maximum over all ranks of a few per-rank timings (the job is as slow
    as its slowest replica); the values themselves on a single process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def replicas_value(ms_per_step, world):
    """Whole-job matvecs/s of `world` independent replicas, each step taking ms_per_step (the
    maximum over ranks)."""
    return world * 1e3 / ms_per_step


class OracleMatvec:
    """The FP64 oracle's O-AIM system matvec (Eq. AEFIEoutJ as a sequence, NumPy/SciPy) on a
    bounded sample of the workload: the SUB x SUB sub-array of the split-ring array (same ring
    geometry, grid spacing and near-region rule), its matvec time scaled to the full array by
    the number of rings (every part of the product grows with it). The dense internal blocks
    and the near-region values are seeded random numbers of the true sizes and sparsity: the
    matvec's cost does not depend on the values, and forming the true ones takes the oracle
    tens of minutes."""

    def __init__(self, sub=SUB, nfull=32):
        import numpy as np
        import scipy.sparse as sp

        from oracle import aim as oaim, operators as op
        from oracle.rwg import from_mesh
        from paper_2108_03991_gb300 import synth

        mesh, grid, freq = synth.srr_array_config(2, sub)
        rw = from_mesh(mesh)
        A = oaim.Aim(rw, grid.origin, grid.h, grid.n, op.k0_of(freq))
        rng = np.random.default_rng(7)
        M, N = A.near_e
        A.LNR_A = sp.csr_matrix((rng.standard_normal(M.size) + 0j, (M, N)), shape=(rw.ne, rw.ne))
        T, S_ = A.near_t
        A.LNR_P = sp.csr_matrix((rng.standard_normal(T.size) + 0j, (T, S_)), shape=(rw.nt, rw.nt))
        sizes = [b - a for a, b in rw.obj_edge_ranges()]
        blocks = synth.rand_blocks(sizes, 8)
        self.S = op.SlimSystem(rw, freq, blocks, blocks, A.LA, A.LPhi)
        self.x = synth.rand_cvec(self.S.n, 1)
        self.scale = (nfull * nfull) / (sub * sub)
        self.desc = (f"the {sub}x{sub} sub-array ({rw.ne} RWG + {rw.nt} pulse unknowns, {mesh.nobj} "
                     f"rings, grid {'x'.join(str(int(v)) for v in grid.n)}), time scaled by the "
                     f"ring count ({self.scale:g}x) to the {nfull}x{nfull} array; internal blocks "
                     "and near-region values seeded random of the true sizes")

    def run(self, seconds=0.0):
        """Sample matvecs for at least `seconds` (at least one); returns seconds per matvec of
        the full workload (the sample's time times the scale)."""
        n, t0 = 0, time.perf_counter()
        while True:
            self.S.matvec(self.x)
            n += 1
            if time.perf_counter() - t0 >= seconds:
                return self.scale * (time.perf_counter() - t0) / n


def oracle_baseline(seconds=15.0):
    """The oracle timed on the host cores on a bounded sample of the workload (about
    `seconds` of work)."""
    om = OracleMatvec()
    om.run()
    dt = om.run(seconds)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": 1.0 / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{om.desc}: {dt / om.scale:.3f} s per sample matvec over {seconds:g} s"}


def run_reference(args, rank, world):
    """The oracle as the reference arm: W untimed matvecs, then K timed steps of the same
    workload within about a minute in all (one sample matvec per step at least)."""
    if rank != 0:
        return
    om = OracleMatvec()
    for _ in range(max(0, args.warmup)):
        om.run()
    per_step = 60.0 / max(1, args.steps)
    t0 = time.perf_counter()
    dts = [om.run(per_step) for _ in range(max(1, args.steps))]
    v = 1.0 / (sum(dts) / len(dts))
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    cb = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
          "sample": f"{om.desc}; {len(dts)} steps in {time.perf_counter() - t0:.1f} s"}
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / v,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic", "config": {"workload": WORKLOAD, "parallelism": "replicas"},
        "cpu_baseline": cb, "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                                    "d2h_bytes_per_step": 0}}))


# DRAM bytes (read + write) per launch of the GEMV shapes captured with ncu on the split-ring
# array, keyed by (rings per side, "pair" for the paired launch of C and Z, kind, CTAs per SM,
# split, loads in flight) as aim_info reports them; a launch of another shape reports none.
# The C GEMV of the 32 x 32 array: captured on the 8 x 8 array in the same launch shape
# (426,572,032 + 9,975,552 B per launch, profiles/gemv_C_srr_array.md) and scaled by the 16
# times as many rings (every ring has the same 912 x 912 block)
PROFILED_GEMV: dict = {(32, "one", 5, 16, 2, 4): 16 * (426572032 + 9975552)}


def gemv_traffic(ctx, rings, paired=False):
    key = (rings, "pair" if paired else "one", ctx.gemv_kind, ctx.gemv_cps, ctx.gemv_split,
           ctx.gemv_unroll)
    b = PROFILED_GEMV.get(key)
    return int(b) if b else None


def ncu_case(args):
    """Small cases for profiler captures.
    gemv: the block-diagonal GEMV alone on random blocks with the workload's block sizes (one of
          Z or Y_eq: ~200 MB in FP32, larger than L2);
    aim:  the grid convolution (4 components) on the workload's AIM grid, set up on two small
          boxes at opposite corners of the array's bounding box (same grid, tiny set-up);
    internal: the split-ring array's internal products (e = Z h, h_eq = Y e; --rings per side,
          8 for a capture that fits the profiler) with the launch the set-up autotuner chose,
          inside the profiler range "internal_steps".
    batch: the workload's batched system matvec of 4 right-hand sides, inside the profiler
          range "batch_steps"."""
    import numpy as np
    import torch

    from paper_2108_03991_gb300 import api, build, synth
    build.build()
    if args.ncu_case == "aim":
        full = synth.bar_array(0)
        hi = full.verts.max(axis=0)
        parts = [synth.box((0.0, 0.0, 0.0), (1.0, 1.0, 1.0), (2, 2, 2)),
                 synth.box(tuple(hi - 1.0), (1.0, 1.0, 1.0), (2, 2, 2))]
        mesh = synth.merge(parts, [synth.SIGMA_CU] * 2)
        ctx = api.Context(mesh, synth.grid_box(full, 0.5), 10e9)
        s = torch.from_numpy(np.concatenate([synth.rand_cvec(ctx.ng, c) for c in range(4)])
                             .astype(np.complex64)).cuda()
        phi = torch.empty_like(s)
        for _ in range(args.steps):
            ctx.conv(s, phi, ncomp=4, prec=api.BEM_C32)
        torch.cuda.synchronize()
        print(json.dumps({"ncu_case": "aim", "grid": list(ctx.grid_n), "fft": list(ctx.padded)}))
        return
    if args.ncu_case == "aim_srr":
        # the grid convolution (4 components) on the split-ring array's grid (--rings per side;
        # 32: 512 x 512 x 8, padded 1024 x 1024 x 15), set up on two small gold boxes at opposite
        # corners of the array (same grid, tiny set-up)
        g = synth.srr_grid(args.rings)
        top = 50.0 * args.rings
        parts = [synth.box((1.0, 1.0, 0.0), (1.0, 1.0, 1.0), (2, 2, 2)),
                 synth.box((top - 2.0, top - 2.0, 0.0), (1.0, 1.0, 1.0), (2, 2, 2))]
        mesh = synth.merge(parts, [synth.SIGMA_AU] * 2)
        ctx = api.Context(mesh, g, 1e12)
        s = torch.from_numpy(np.concatenate([synth.rand_cvec(ctx.ng, c) for c in range(4)])
                             .astype(np.complex64)).cuda()
        phi = torch.empty_like(s)
        for _ in range(args.steps):
            ctx.conv(s, phi, ncomp=4, prec=api.BEM_C32)
        torch.cuda.synchronize()
        print(json.dumps({"ncu_case": "aim_srr", "grid": list(ctx.grid_n), "fft": list(ctx.padded)}))
        return
    if args.ncu_case == "srr":
        mesh, grid, freq = synth.srr_array_config(2, args.rings)
        ctx = api.Context(mesh, grid, freq)
        x = torch.from_numpy(synth.rand_cvec(ctx.n, 1).astype(np.complex64)).cuda()
        y = torch.empty_like(x)
        for _ in range(3):
            ctx.matvec(x, y)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("srr_steps")
        for _ in range(args.steps):
            ctx.matvec(x, y)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        print(json.dumps({"ncu_case": "srr", "rings": args.rings, "sparse_internal": ctx.sparse_internal,
                          "nnz_near": [ctx.nnz_A, ctx.nnz_P]}))
        return
    if args.ncu_case == "batch":
        mesh, grid, freq = synth.bar_array_config(0, 10e9)
        ctx = api.Context(mesh, grid, freq)
        xb = torch.from_numpy(np.concatenate([synth.rand_cvec(ctx.n, 500 + r) for r in range(4)])
                              .astype(np.complex64)).cuda()
        yb = torch.empty_like(xb)
        ctx.matvec_batch(xb, yb)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("batch_steps")
        for _ in range(args.steps):
            ctx.matvec_batch(xb, yb)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        print(json.dumps({"ncu_case": "batch", "nrhs": 4}))
        return
    if args.ncu_case == "internal":
        mesh, grid, freq = synth.srr_array_config(2, args.rings)
        ctx = api.Context(mesh, grid, freq)
        if args.gemv_shape:  # the launch the timed run chose (the autotuner's timing under a
            ctx.gemv_plan(*[int(v) for v in args.gemv_shape.split(",")])  # profiler differs)
        if args.schedule is not None:  # 3: both products in the paired launch
            ctx.matvec_schedule(args.schedule)
        h = torch.from_numpy(synth.rand_cvec(ctx.ne, 4).astype(np.complex64)).cuda()
        e, heq = torch.empty_like(h), torch.empty_like(h)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("internal_steps")
        for _ in range(args.steps):
            ctx.internal(h, e, heq, prec=api.BEM_C32)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        print(json.dumps({"ncu_case": "internal", "kind": ctx.gemv_kind, "ctas": ctx.gemv_ctas,
                          "split": ctx.gemv_split,
                          "loads_in_flight": ctx.gemv_unroll, "tune_ns": ctx.gemv_tune_ns}))
        return
    mesh = synth.bar_array(0)
    sizes = [int(np.sum(mesh.obj == i)) * 3 // 2 for i in range(mesh.nobj)]
    N = sum(sizes)
    A = torch.from_numpy(api.pack_blocks(synth.rand_blocks(sizes, 3), np.complex64)).cuda()
    x = torch.from_numpy(synth.rand_cvec(N, 4).astype(np.complex64)).cuda()
    y = torch.empty_like(x)
    for _ in range(args.steps):
        api.blockdiag_gemv(sizes, A, x, y, 1, api.BEM_C32)
    torch.cuda.synchronize()
    print(json.dumps({"ncu_case": "gemv", "blocks": len(sizes), "rows": N,
                      "bytes": int(A.numel() * 8)}))


def copper_bar_numbers(api, synth, torch):
    """The single 2x2x20 um copper bar at 10 GHz (2016 RWG + 1344 pulse unknowns): microseconds
    per graph-replayed system matvec in FP64 and FP32, and the time to a true FP64 residual of
    1e-6 for the plane wave, plain FP64 GMRES against the chosen FP32-bulk FGMRES with the
    block-diagonal preconditioner (after an untimed warm-up solve of each)."""
    mesh, grid, freq = synth.copper_bar()
    ctx = api.Context(mesh, grid, freq)
    out = {"structure": "Cu bar 2x2x20 um, 10 GHz", "ne": ctx.ne, "nt": ctx.nt}
    for prec, name in ((api.BEM_C64, "matvec_us_fp64"), (api.BEM_C32, "matvec_us_fp32")):
        x = torch.from_numpy(synth.rand_cvec(ctx.n, 2)).to(api.cdtype(prec)).cuda()
        y = torch.empty_like(x)
        for _ in range(10):
            ctx.matvec(x, y, prec=prec)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(100):
            ctx.matvec(x, y, prec=prec)
        e1.record()
        torch.cuda.synchronize()
        out[name] = e0.elapsed_time(e1) * 10.0  # 100 launches, ms -> us each
    b = ctx.rhs_plane_wave(prec=api.BEM_C64)
    for name, mode, pc in (("plain_fp64", api.BEM_C64, 0), ("chosen_fp32_block", api.BEM_C32, 1)):
        ctx.solve(b, tol=1e-6, restart=200, max_iter=2, prec_mode=mode, precond=pc)  # warm-up
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        _, info = ctx.solve(b, tol=1e-6, restart=200, max_iter=3000, prec_mode=mode,
                            time_limit_s=60.0, precond=pc)
        torch.cuda.synchronize()
        out[name] = {"seconds": time.perf_counter() - t1, "iters": info["iters"],
                     "resid_true": info["resid_true"], "status": info["status"]}
    ctx.close()
    return out


def precision_study(args):
    """FP32-bulk against FP64 on the 4x4 bar array over 1-100 GHz: for each frequency the
    relative error of the complex-FP32 system matvec, and of every solve output of the chosen
    FP32-bulk FGMRES (block-diagonal preconditioner, 1e-6) against an FP64 FGMRES solve to 1e-10
    of the same system: h, j = h - Y Z h, q, the radiation vector in three directions, and the
    2x2 admittance of two delta-gap ports on bar 0 (1 um from its ends)."""
    import numpy as np
    import torch

    from paper_2108_03991_gb300 import api, build, synth
    build.build()
    out = []
    rh = np.array([[0.0, 0.0, -1.0], [1.0, 0.0, 0.0], [0.0, 0.6, 0.8]])

    def rel(a, b):
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

    for f_ghz in (1, 10, 30, 60, 100):
        mesh, grid, freq = synth.bar_array_config(0, f_ghz * 1e9)
        t0 = time.perf_counter()
        ctx = api.Context(mesh, grid, freq)
        zs = mesh.verts[np.unique(mesh.tris[mesh.obj == 0])][:, 2]
        rings = [ctx.port_ring(0, 2, z) for z in (zs.min() + 1.0, zs.max() - 1.0)]
        xr = synth.rand_cvec(ctx.n, 9)
        y32 = ctx.matvec(torch.from_numpy(xr.astype(np.complex64)).cuda(), prec=api.BEM_C32)
        y64 = ctx.matvec(torch.from_numpy(xr).cuda(), prec=api.BEM_C64)
        row = {"GHz": f_ghz, "matvec_fp32": rel(y32.cpu().numpy(), y64.cpu().numpy())}
        rhs = [("plane_wave", ctx.rhs_plane_wave(prec=api.BEM_C64))]
        rhs += [(f"port{q}", ctx.rhs_port(e, sgn, v_gap=1.0)) for q, (e, sgn) in enumerate(rings)]
        sol = {}
        for mode, tol in ((api.BEM_C64, 1e-10), (api.BEM_C32, 1e-6)):
            for name, b in rhs:
                x, info = ctx.solve(b, tol=tol, restart=200, max_iter=2000, prec_mode=mode,
                                    time_limit_s=60.0, precond=1)
                sol[(mode, name)] = (x, info)
        x64, i64 = sol[(api.BEM_C64, "plane_wave")]
        x32, i32 = sol[(api.BEM_C32, "plane_wave")]

        def parts(x):
            h = x[:ctx.ne].contiguous()
            _, heq = ctx.internal(h, prec=api.BEM_C64)
            return (h.cpu().numpy(), (h - heq).cpu().numpy(), x[ctx.ne:].cpu().numpy(),
                    ctx.farfield(x, rh, prec=api.BEM_C64))
        h64, j64, q64, n64 = parts(x64)
        h32, j32, q32, n32 = parts(x32)
        Y = {}
        for mode in (api.BEM_C64, api.BEM_C32):
            M = np.zeros((2, 2), complex)
            for qi in range(2):
                xq = sol[(mode, f"port{qi}")][0]
                for p, (e, sgn) in enumerate(rings):
                    M[p, qi] = ctx.port_current(xq, e, sgn, prec=api.BEM_C64)
            Y[mode] = M
        row.update({"h": rel(h32, h64), "j": rel(j32, j64), "q": rel(q32, q64),
                    "far_field": rel(n32, n64),
                    "port_Y": float(np.max(np.abs(Y[api.BEM_C32] - Y[api.BEM_C64]))
                                    / np.max(np.abs(Y[api.BEM_C64]))),
                    "Y11_S": [Y[api.BEM_C64][0, 0].real, Y[api.BEM_C64][0, 0].imag],
                    "iters_fp64_1e-10": i64["iters"], "iters_fp32_1e-6": i32["iters"],
                    "resid_true_fp32": i32["resid_true"],
                    "seconds_with_setup": time.perf_counter() - t0})
        out.append(row)
        ctx.close()
        print(json.dumps(row), file=sys.stderr)
    print(json.dumps({"precision_study": out, "workload": WORKLOAD.replace("10 GHz", "1-100 GHz")}))


def bar_array_section(args, api, synth, torch, np, dev):
    """The 4 x 4 copper bar array (10 GHz): the time to a true FP64 relative residual of 1e-6
    for the plane wave, plain FP64 GMRES (no preconditioner) against FP64 FGMRES and the chosen
    FP32-bulk FGMRES (FP64 Arnoldi) with the block-diagonal preconditioner, with and without
    the learned correction; four plane waves one by one and batched; the copper bar."""
    mesh, grid, freq = synth.bar_array_config(0, 10e9)
    t0 = time.perf_counter()
    ctx = api.Context(mesh, grid, freq)
    torch.cuda.synchronize()
    out = {"workload": BAR_WORKLOAD, "setup_s": time.perf_counter() - t0}
    solve = {}
    b = ctx.rhs_plane_wave(prec=api.BEM_C64)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    solve["precond_build"] = ctx.precond_setup(api.BEM_C32)
    torch.cuda.synchronize()
    solve["precond_setup_s"] = time.perf_counter() - t1
    # learned correction: trained on another seed of the same family (the benchmark
    # structure is unseen), weights carried over
    t1 = time.perf_counter()
    tmesh, tgrid, _ = synth.bar_array_config(100, 10e9)
    tctx = api.Context(tmesh, tgrid, 10e9)
    tctx.net_init(1)
    losses = tctx.net_train(steps=args.train_steps, batch=4, lr=2e-3, seed=2)
    w = tctx.net_weights()
    tctx.close()
    ctx.net_weights(w)
    torch.cuda.synchronize()
    solve["learned_training"] = {
        "structure": "4x4 Cu bar array, seed 100", "steps": args.train_steps, "batch": 4,
        "loss_first10": float(np.mean(losses[:10])), "loss_last10": float(np.mean(losses[-10:])),
        "seconds_incl_setup": time.perf_counter() - t1}
    # untimed warm-up: allocates the context's Krylov workspace and captures the FP64 and
    # FP32 matvec graphs, as a long-lived solver context has them before its next solve
    for mode in (api.BEM_C64, api.BEM_C32):
        ctx.solve(b, tol=1e-6, restart=200, max_iter=2, prec_mode=mode, precond=1)
    solve["warm"] = "workspace and matvec graphs from an untimed 2-iteration solve"
    for name, mode, pc in (("plain_fp64", api.BEM_C64, 0), ("block_fp64", api.BEM_C64, 1),
                           ("chosen_fp32_block", api.BEM_C32, 1),
                           ("chosen_fp32_block_learned", api.BEM_C32, 2)):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        torch.cuda.nvtx.range_push("solve_" + name)  # profiler range of this solve
        xs, info = ctx.solve(b, tol=1e-6, restart=200, max_iter=3000, prec_mode=mode,
                             time_limit_s=120.0, precond=pc)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    solve[name] = {"seconds": time.perf_counter() - t1, "iters": info["iters"],
                       "resid_true": info["resid_true"], "status": info["status"]}
    # four plane waves (polarisation x, y along +z; z, y along +x): solved one after
    # another with the chosen form, and together with the batched FGMRES
    waves = [((1.0, 0.0, 0.0), (0.0, 0.0, 1.0)), ((0.0, 1.0, 0.0), (0.0, 0.0, 1.0)),
             ((0.0, 0.0, 1.0), (1.0, 0.0, 0.0)), ((0.0, 1.0, 0.0), (1.0, 0.0, 0.0))]
    bw = torch.cat([ctx.rhs_plane_wave(pol, kh, prec=api.BEM_C64) for pol, kh in waves])
    ctx.solve_batch(bw, tol=1e-6, restart=200, max_iter=2, prec_mode=api.BEM_C32, precond=1)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    its = []
    for r in range(4):
        _, info = ctx.solve(bw[r * ctx.n:(r + 1) * ctx.n].contiguous(), tol=1e-6, restart=200,
                            max_iter=3000, prec_mode=api.BEM_C32, precond=1)
        its.append(info["iters"])
    torch.cuda.synchronize()
    solve["chosen_4_waves_one_by_one"] = {"seconds": time.perf_counter() - t1, "iters": its}
    t1 = time.perf_counter()
    torch.cuda.nvtx.range_push("solve_batch4")
    _, rc, infos = ctx.solve_batch(bw, tol=1e-6, restart=200, max_iter=3000,
                                   prec_mode=api.BEM_C32, precond=1, time_limit_s=120.0)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    solve["chosen_4_waves_batched"] = {
        "seconds": time.perf_counter() - t1, "iters": infos[0]["iters"], "status": rc,
        "resid_true": [i["resid_true"] for i in infos]}
    # time to solution with the preconditioner's one-off set-up counted: for one right-hand
    # side, and the number of right-hand sides after which the chosen form (set-up once,
    # then one chosen solve each) beats plain FP64 GMRES (one plain solve each)
    su, pl, ch = (solve["precond_setup_s"], solve["plain_fp64"]["seconds"],
              solve["chosen_fp32_block"]["seconds"])
    solve["chosen_incl_precond_setup"] = {
        "seconds_one_rhs": su + ch, "plain_fp64_seconds_one_rhs": pl,
        "break_even_rhs": (math.ceil(su / (pl - ch)) if pl > ch else None),
        "note": "set-up of the block-diagonal preconditioner once per structure, then per "
                "right-hand side one chosen solve against one plain FP64 solve"}

    out["solve"] = solve
    ctx.close()
    out["copper_bar"] = copper_bar_numbers(api, synth, torch)
    return out


def tensor_core_section(ctx, api, synth, torch, np, dev, hbm, reps=10):
    """h_eq = C h for R right-hand sides at once (C = Y_eq Z, complex FP32): the tensor-core
    product (one pass over C per 128 right-hand sides, TF32 with the hi/lo split) against the
    block GEMV (one pass per 4), both through the library; the two agree to FP32 rounding. Per
    R: ms per product, C's bytes over that time, and the complex flops 8 sum n_i^2 R over it."""
    ZY = ctx.zy_bytes_c32 // 2
    n2 = ZY / 8  # sum of n_i ld_i complex entries of C
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s = torch.cuda.current_stream()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        ev0.record(s)
        for _ in range(reps):
            fn()
        ev1.record(s)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / reps

    rows = []
    for R in (4, 8, 16, 32, 64, 128):
        h = torch.from_numpy(np.concatenate([synth.rand_cvec(ctx.ne, 700 + r) for r in range(R)])
                             .astype(np.complex64)).to(dev)
        y_tc = torch.empty_like(h)
        y_mv = torch.empty_like(h)
        t_tc = timed(lambda: ctx.internal_tc(h, None, y_tc, nrhs=R, want_e=False))
        t_mv = timed(lambda: ctx.internal(h, None, y_mv, nrhs=R, prec=api.BEM_C32, want_e=False))
        d = float(torch.linalg.vector_norm(y_tc - y_mv) / torch.linalg.vector_norm(y_mv))
        ctx.tc_variant(1)  # the raw right-hand sides split in shared memory (half the packed bytes)
        t_raw = timed(lambda: ctx.internal_tc(h, None, y_tc, nrhs=R, want_e=False))
        ctx.tc_variant(0)
        d_raw = float(torch.linalg.vector_norm(y_tc - y_mv) / torch.linalg.vector_norm(y_mv))
        rows.append({"nrhs": R, "ms_tensor_core": t_tc, "ms_tensor_core_raw_b": t_raw,
                     "ms_block_gemv": t_mv,
                     "speedup": t_mv / t_tc, "rel_diff": d, "rel_diff_raw_b": d_raw,
                     "tensor_core_GBps": ZY / (t_tc * 1e-3) / 1e9,
                     "tensor_core_frac_hbm": ZY / (t_tc * 1e-3) / 1e9 / hbm,
                     "tensor_core_TFLOPs": 8 * n2 * R / (t_tc * 1e-3) / 1e12})
        del h, y_tc, y_mv
    st = ctx.tensor_core_status()
    cross = next((r["nrhs"] for r in rows if r["speedup"] > 1), None)
    return {"product": "h_eq = C h, R right-hand sides (aim_internal_tc vs internal_apply)",
            "rows": rows, "crossover_nrhs": cross, "wait_timed_out": st["wait_timed_out"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--bar-array", action="store_true",
                    help="add the 4x4 copper bar array's solves (learned correction, batches)")
    ap.add_argument("--ncu-case", default=None, choices=["gemv", "aim", "aim_srr", "internal", "batch", "srr"])
    ap.add_argument("--train-steps", type=int, default=300)
    ap.add_argument("--precision-study", action="store_true")
    ap.add_argument("--schedule", type=int, default=None,
                    help="matvec schedule (aim_matvec_schedule) in --ncu-case internal")
    ap.add_argument("--gemv-shape", default=None,
                    help="kind,ctas_per_sm,split,unroll of the GEMV launch in --ncu-case internal")
    ap.add_argument("--rings", type=int, default=32,
                    help="rings per side of the split-ring array (32: the full workload)")
    ap.add_argument("--rows-variant", type=int, default=None, choices=[0, 1, 2],
                    help="form of the row kernels (aim_rows_variant) for the timed matvecs")
    ap.add_argument("--no-tensor-core", action="store_true",
                    help="leave out h_eq = C h for 4..128 right-hand sides at once (the "
                         "tensor-core product against the block GEMV)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.ncu_case:
        return ncu_case(args)
    if args.precision_study:
        return precision_study(args)
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2108_03991_gb300 import api, build, synth
    build.build()
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")

    mesh, grid, freq = synth.srr_array_config(2, args.rings)
    t0 = time.perf_counter()
    ctx = api.Context(mesh, grid, freq)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    if args.rows_variant is not None:
        ctx.rows_variant(args.rows_variant)
    s = torch.cuda.current_stream()
    x = torch.from_numpy(synth.rand_cvec(ctx.n, 1 + rank)).to(torch.complex64).to(dev)
    y = torch.empty_like(x)
    for _ in range(args.warmup):
        ctx.matvec(x, y, prec=api.BEM_C32)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ev0.record(s)
        for _ in range(reps):
            fn()
        ev1.record(s)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / reps

    with ClockSampler(local) as clk:
        # the same matvecs for about a second before the timed steps, so that the 200 ms clock
        # samples see the GPU under this load
        t_load = time.perf_counter()
        while time.perf_counter() - t_load < 1.0:
            for _ in range(20):
                ctx.matvec(x, y, prec=api.BEM_C32)
            torch.cuda.synchronize()
        ev0.record(s)
        torch.cuda.nvtx.range_push("matvec_steps")  # profiler range of the timed steps
        for _ in range(args.steps):
            ctx.matvec(x, y, prec=api.BEM_C32)
        torch.cuda.nvtx.range_pop()
        ev1.record(s)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / args.steps
        # dominant kernel: the block-diagonal GEMV, as the matvec launches it: one paired launch
        # of C and Z per internal_apply under the paired schedule, else two launches
        e = torch.empty(ctx.ne, dtype=torch.complex64, device=dev)
        heq = torch.empty_like(e)
        h = x[:ctx.ne].contiguous()
        sparse = ctx.sparse_internal["on"]
        paired = ctx.matvec_mode == 3 and not sparse
        zsp_ms = None
        if sparse:
            # the matvec's internal part with the sparse internal operator: j = h - C h, the one
            # dense block GEMV (the dominant kernel), and e = Z_s h beside it
            gemv_ms = timed(lambda: ctx.internal(h, None, heq, prec=api.BEM_C32, want_e=False),
                            args.steps)
            zsp_ms = timed(lambda: ctx.internal(h, e, None, prec=api.BEM_C32, want_heq=False),
                           args.steps)
        else:
            gemv_ms = timed(lambda: ctx.internal(h, e, heq, prec=api.BEM_C32), args.steps) / \
                (1 if paired else 2)
        # the AIM external part alone (Sec. III-A: projection, FFT convolution, interpolation,
        # precorrected near region) for the RWG vector components (L^A) and the charges (L^Phi)
        ja = x[:ctx.ne].contiguous()
        qa = x[ctx.ne:].contiguous()
        ya = torch.empty_like(ja)
        yp = torch.empty_like(qa)
        aim_la_ms = timed(lambda: ctx.matvec(ja, ya, which=api.AIM_OP_LA, prec=api.BEM_C32), args.steps)
        aim_lp_ms = timed(lambda: ctx.matvec(qa, yp, which=api.AIM_OP_LPHI, prec=api.BEM_C32), args.steps)
        # both at once, the two branches concurrent as in the system matvec (AIM_OP_EXT)
        yx = torch.empty_like(x)
        aim_ms = timed(lambda: ctx.matvec(x, yx, which=api.AIM_OP_EXT, prec=api.BEM_C32), args.steps)
        # the batched system matvec: 4 right-hand sides per graph launch
        xb = torch.from_numpy(np.concatenate([synth.rand_cvec(ctx.n, 500 + r) for r in range(4)])
                              .astype(np.complex64)).to(dev)
        yb = torch.empty_like(xb)
        batch_ms = timed(lambda: ctx.matvec_batch(xb, yb, prec=api.BEM_C32), args.steps)
        del xb, yb
        # end to end through the host-buffer call: K distinct pinned host inputs, each copied
        # to the device, multiplied and copied back (the copies of neighbouring steps overlap
        # the products)
        xh = torch.from_numpy(np.stack([synth.rand_cvec(ctx.n, 1000 + i).astype(np.complex64)
                                        for i in range(args.steps)])).pin_memory()
        yh = torch.empty(xh.shape, dtype=xh.dtype, pin_memory=True)
        ctx.matvec_host(xh[:3].contiguous(), prec=api.BEM_C32)
        torch.cuda.synchronize()
        ev0.record(s)
        ctx.matvec_host(xh, yh, prec=api.BEM_C32)
        ev1.record(s)
        torch.cuda.synchronize()
        e2e_ms = ev0.elapsed_time(ev1) / args.steps
        # the same call one vector per product (the product `value` times, copies included)
        for i in range(3):
            ctx.matvec_host(xh[i:i + 1], yh[i:i + 1], prec=api.BEM_C32)
        torch.cuda.synchronize()
        ev0.record(s)
        for i in range(args.steps):
            ctx.matvec_host(xh[i:i + 1], yh[i:i + 1], prec=api.BEM_C32)
        ev1.record(s)
        torch.cuda.synchronize()
        e2e1_ms = ev0.elapsed_time(ev1) / args.steps
        del xh, yh
    ms, e2e_ms, batch_ms, e2e1_ms = max_over_ranks([ms, e2e_ms, batch_ms, e2e1_ms], dev)

    solve = None
    if not args.no_solve and rank == 0:
        # time to a true FP64 relative residual of 1e-6 for a plane wave at normal incidence
        # (E along x, the gap's axis; propagation along -z): plain = FP64 GMRES without a
        # preconditioner; chosen = FP32-bulk FGMRES (FP64 Arnoldi and true residual) with the
        # block-diagonal preconditioner (inverses built in complex FP32, each block checked), its
        # one-off set-up timed separately and counted
        solve = {"excitation": "plane wave, E along x, k along -z"}
        b = ctx.rhs_plane_wave((1.0, 0.0, 0.0), (0.0, 0.0, -1.0), prec=api.BEM_C64)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        solve["precond_build"] = ctx.precond_setup(api.BEM_C32)
        torch.cuda.synchronize()
        solve["precond_setup_s"] = time.perf_counter() - t1
        for mode, pc in ((api.BEM_C64, 0), (api.BEM_C32, 1)):  # workspace and graphs
            ctx.solve(b, tol=1e-6, restart=100, max_iter=2, prec_mode=mode, precond=pc)
        solve["warm"] = "workspace and matvec graphs from an untimed 2-iteration solve"
        for name, mode, pc, lim in (("chosen_fp32_block", api.BEM_C32, 1, 120.0),
                                    ("plain_fp64", api.BEM_C64, 0, 90.0)):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            torch.cuda.nvtx.range_push("solve_" + name)
            _, info = ctx.solve(b, tol=1e-6, restart=100, max_iter=100000, prec_mode=mode,
                                time_limit_s=lim, precond=pc)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
            solve[name] = {"seconds": time.perf_counter() - t1, "iters": info["iters"],
                           "resid_true": info["resid_true"], "status": info["status"],
                           "time_limit_s": lim}
        su, pl, ch = (solve["precond_setup_s"], solve["plain_fp64"], solve["chosen_fp32_block"])
        solve["chosen_incl_precond_setup"] = {
            "seconds": su + ch["seconds"], "reached_1e-6": ch["resid_true"] <= 1e-6,
            "plain_fp64_seconds": pl["seconds"], "plain_reached_1e-6": pl["resid_true"] <= 1e-6,
            "note": "plain FP64 GMRES stops at its time limit when it has not reached 1e-6; "
                    "status 1 marks that, resid_true is where it stood"}

    if rank == 0:
        hbm, src = peaks()
        ZY = ctx.zy_bytes_c32 // 2  # bytes of Z (or C) in FP32
        # algorithmic bytes of one launch: the matrix (both under the paired schedule), x read,
        # the output(s) written
        gemv_bytes = 2 * ZY + 3 * 8 * ctx.ne if paired else ZY + 2 * 8 * ctx.ne
        achieved = gemv_bytes / (gemv_ms * 1e-3) / 1e9
        # the AIM external part's algorithmic bytes (complex FP32 s = 8, FP32 weights r = 4):
        # vectors in and out, stencils read by the projection and again by the interpolation,
        # per grid component 20 N_g values (scatter, FFT read, padded spectra write and read,
        # inverse output, gather), the octant of the grid kernel, the near-region CSR values and
        # columns
        ne, nt, ng = ctx.ne, ctx.nt, ctx.ng
        gx, gy, gz = ctx.grid_n
        b_aim = (2 * 8 * (ne + nt) + 2 * (4 * (81 * ne + 27 * nt) + 4 * (ne + nt))
                 + 4 * 8 * 20 * ng + 8 * (gx + 1) * (gy + 1) * (gz + 1)
                 + (ctx.nnz_A + ctx.nnz_P) * (8 + 4))
        aim_ach = b_aim / (aim_ms * 1e-3) / 1e9
        cpu = None
        if not args.no_cpu:
            cpu = oracle_baseline(seconds=15.0)
        value = replicas_value(ms, world)
        stream_init = 1 if ctx.gemv_kind == 3 else 0
        if sparse:  # C's GEMV, the two kernels of e = Z_s h
            launches_per_step = 11 + 1 + stream_init + 2
        else:
            launches_per_step = 11 + (1 if ctx.matvec_mode == 3 else
                                      2 + stream_init * (2 if ctx.matvec_mode == 2 else 1))
        zsp = None
        if sparse:
            sp = ctx.sparse_internal
            # the operator's FP32 bytes (L and U column tables, inverse diagonal, CSR values and
            # columns of K_s + I_x/2), h gathered, the permuted rows written and read, e written
            zb = sp["bytes_c32"] + 4 * 8 * ctx.ne
            zsp = {"kernels": "k_zsp_rows (rows of K_s + I_x/2) + k_zsp_solve (banded L_s^-1, "
                              "one warp per ring)",
                   "bytes": zb, "ms": zsp_ms, "achieved": zb / (zsp_ms * 1e-3) / 1e9,
                   "unit": "GB/s", "frac": zb / (zsp_ms * 1e-3) / 1e9 / hbm,
                   "half_bandwidth": sp["band"], "setup_check": sp["check"],
                   "dense_Z_bytes": ZY}
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": WORKLOAD if args.rings == 32 else
                       WORKLOAD.replace("32x32", f"{args.rings}x{args.rings}"),
                       "unknowns": ctx.n, "ne": ctx.ne, "nt": ctx.nt,
                       "objects": ctx.nobj, "grid": list(ctx.grid_n), "fft": list(ctx.padded),
                       "nnz_near": [ctx.nnz_A, ctx.nnz_P], "parallelism": f"replicas{world}",
                       "l2": "inputs larger than L2 (C %.1f GB, %s)" % (
                           ZY / 1e9, "sparse Z_s %.1f GB" % (ctx.sparse_internal["bytes_c32"] / 1e9)
                           if sparse else "Z %.1f GB" % (ZY / 1e9)),
                       "internal": "sparse Z_s (Sec. III-A, high frequency)" if sparse else "dense Z",
                       "rows_variant": args.rows_variant or 0,
                       "setup_s": setup_s, "setup_stage_s": ctx.setup_stage_s,
                       "reference_arm": "FP64 oracle on the host cores on the 8x8 sub-array, "
                                        "scaled by the ring count; its internal blocks and "
                                        "near-region values are seeded random numbers of the "
                                        "true sizes and sparsity"},
            "roofline": {"kernel": ("k_gemv_pair (C = Y_eq Z and Z in one launch)" if paired
                                    else "block GEMV of C = Y_eq Z" if sparse
                                    else "k_gemv (block-diagonal Z / C)"), "bound": "hbm",
                         "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "peak_source": src,
                         "traffic": gemv_traffic(ctx, args.rings, paired),
                         "traffic_unit": "DRAM bytes per launch (ncu, profiles/)",
                         "bytes_per_launch": gemv_bytes, "ms_per_launch": gemv_ms,
                         "launch": {"kind": {0: "row plan", 1: "flat", 2: "staged", 3: "stream",
                                             5: "Part_Schedule task list",
                                             6: "Part_Schedule tasks, persistent CTAs"}[ctx.gemv_kind],
                                    "shape": [ctx.gemv_kind, ctx.gemv_cps,
                                              max(ctx.gemv_split, 1), ctx.gemv_unroll],
                                    "ctas": ctx.gemv_ctas,
                                    "autotune_ns_per_launch": ctx.gemv_tune_ns,
                                    "matvec_schedule": ctx.matvec_mode}},
            "roofline_aim": {"part": "AIM external operators L^A (3 components) and L^Phi "
                                     "(aim_matvec AIM_OP_EXT, the two branches concurrent as in "
                                     "the system matvec): projection, FFT convolution, "
                                     "interpolation, near region",
                             "bound": "hbm", "achieved": aim_ach, "peak": hbm, "unit": "GB/s",
                             "frac": aim_ach / hbm, "peak_source": src,
                             "bytes_per_matvec": b_aim, "ms": aim_ms,
                             "ms_LA": aim_la_ms, "ms_LPhi": aim_lp_ms},
            "sparse_internal": zsp,
            "e2e": {"value": replicas_value(e2e_ms, world), "unit": UNIT,
                    "h2d_bytes_per_step": 8 * ctx.n, "d2h_bytes_per_step": 8 * ctx.n,
                    "call": f"aim_matvec_host: {args.steps} distinct pinned host vectors in one "
                            "call, taken 4 at a time by the batched product, copies overlapped "
                            "with the products",
                    "one_vector_per_call": {
                        "value": replicas_value(e2e1_ms, world), "unit": UNIT,
                        "call": f"aim_matvec_host once per vector ({args.steps} calls): the "
                                "one-vector product that `value` times, with its copies"}},
            "batched": {"nrhs": 4, "value": replicas_value(batch_ms / 4, world), "unit": UNIT,
                        "ms_per_launch": batch_ms,
                        "note": "aim_matvec_batch: 4 right-hand sides per graph, matvecs/s counted per right-hand side"},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": dict(clk.summary(), window="the timed steps plus about 1 s of the "
                                                 "same matvecs just before them"),
            "solve": solve,
            "cpu_baseline": cpu,
        }
    if rank == 0 and not args.no_tensor_core:
        # last, after every number of the line is taken: a failure here is reported in the line
        try:
            out["tensor_core"] = tensor_core_section(ctx, api, synth, torch, np, dev, peaks()[0])
        except Exception as exc:  # noqa: BLE001 - recorded, the line still prints
            out["tensor_core"] = {"error": str(exc)[:300]}
    ctx.close()
    if rank == 0 and args.bar_array and not args.no_solve:
        out["bar_array"] = bar_array_section(args, api, synth, torch, np, dev)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()

if __name__ == "__main__":
    main()
