/*
 * bem_aim.h - C ABI of the GB300 SLIM boundary-element library (libbem_aim.so).
 *
 * The library applies the system matrix of the SLIM formulation (Marek, Sharma, Triverio,
 * "A Parallel Boundary Element Method for the Electromagnetic Analysis of Large Structures
 * With Lossy Conductors", Sec. II-C, Eq. AEFIEoutJ) and solves it with GMRES (Sec. III-E).
 * The external operators L^A and L^Phi are applied with the adaptive integral method
 * (Sec. III-A item 1, Eq. AIM_L); the internal problem uses dense per-object matrices
 * Z_i (Eq. MFIEinZin) and Y_i,eq (Eq. EFIEeqYeq), block-diagonal over objects (Sec. II-C).
 *
 * Conventions shared by every call
 *  - Lengths are in micrometres; frequency in Hz; time convention exp(j w t).
 *  - Complex vectors are interleaved (re, im): float pairs for BEM_C32, double pairs for BEM_C64.
 *  - Unknown ordering: edges (RWG functions) sorted by object, then by the vertex pair (a<b);
 *    triangles (pulse functions) in input order. Objects must be contiguous in the triangle
 *    list, so each object's edges form one contiguous range.
 *  - The system vector is x = [h; q] of length N = N_E + N_T: h the n x H coefficients,
 *    q = c0 * rho_Delta. The internal vector e = E/eta0 has length N_E.
 *  - Pointers named x, y, h, e, heq, b, sigma, phi are DEVICE pointers owned by the caller
 *    (for example torch tensors); the library never frees them. Calls taking a `stream`
 *    (a cudaStream_t passed as void*, NULL = legacy default stream) are asynchronous on it.
 *  - Return value: BEM_OK (0), a positive status (BEM_ENOCONV) or a negative error code. The
 *    message of the last error on the calling thread is returned by bem_last_error().
 */
#ifndef BEM_AIM_H
#define BEM_AIM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BEM_OK 0
#define BEM_ENOCONV 1     /* GMRES stopped at max_iter / time limit; x holds the best iterate */
#define BEM_EINVAL (-1)   /* null pointer, NaN, bad size or option */
#define BEM_EMESH (-2)    /* open / non-manifold / inconsistently oriented surface */
#define BEM_EGRID (-3)    /* an AIM stencil falls outside the grid, or grid too large */
#define BEM_ENOMEM (-4)   /* device allocation failed */
#define BEM_ECUDA (-5)    /* a CUDA runtime or library call failed */
#define BEM_ESOLVER (-6)  /* singular internal matrix in the LU factorisation */

enum { BEM_C32 = 0, BEM_C64 = 1 };
enum { AIM_OP_LA = 0, AIM_OP_LPHI = 1, AIM_OP_SYSTEM = 2, AIM_OP_EXT = 3 };

typedef struct aim_ctx aim_ctx;

/* Material of one conductor (Sec. II: permittivity, permeability, conductivity). */
typedef struct {
  double sigma; /* S/m */
  double eps_r;
  double mu_r;
} bem_material;

/* Surface mesh of all conductors (Sec. II: S meshed with triangles; multiple objects
 * S = union S_i, Sec. II-C). Triangles are counter-clockwise seen from outside. The
 * background is vacuum. All arrays are HOST arrays, copied by aim_setup. */
typedef struct {
  int32_t nv;
  const double* xyz;         /* [nv][3] */
  int32_t nt;
  const int32_t* tri;        /* [nt][3] */
  const int32_t* obj_of_tri; /* [nt], non-decreasing, values 0..nobj-1 */
  int32_t nobj;
  const bem_material* mat;   /* [nobj] */
} bem_mesh;

/* Uniform auxiliary AIM grid (Sec. III-A item 1). Node (i,j,k) sits at origin + (i,j,k)*h.
 * order must be 2 (3x3x3 stencils) and r_near the near-region radius in cells (max-norm of
 * anchor differences). */
typedef struct {
  double origin[3];
  double h[3];
  int32_t n[3];
  int32_t order;
  int32_t r_near;
} aim_grid;

/* Build every setup product on the current CUDA device: RWG data, projection stencils,
 * FFT of the grid Green's function, precorrected near-region matrices L^A_NR and L^Phi_NR
 * (Sec. III-A item 1, Phillips 1997), the dense internal matrices Z_i and Y_i,eq of every
 * object (Eqs. MFIEinZin, EFIEeqYeq; FP64 integrals, LU by cuSOLVER), in FP64 and FP32 copies.
 * On success *out owns all device memory; release it with aim_destroy.
 * Errors: BEM_EINVAL, BEM_EMESH, BEM_EGRID, BEM_ENOMEM, BEM_ECUDA, BEM_ESOLVER. */
int aim_setup(const bem_mesh* mesh, const aim_grid* grid, double freq_hz, aim_ctx** out);

/* Free every device and host resource of ctx (NULL is allowed). */
void aim_destroy(aim_ctx* ctx);

/* Message of the last failing call on this thread ("" if none). */
const char* bem_last_error(void);

/* Sizes: info[0]=N_E, [1]=N_T, [2]=nobj, [3..5]=grid n, [6..8]=padded FFT lengths,
 * [9]=nnz(L^A_NR), [10]=nnz(L^Phi_NR), [11]=bytes of Z and Y (C32), [12]=max n_i,
 * [13]=CTAs of the block GEMV launch, [14]=column parts per row of the row-plan kernel, rows
 * per task / 8 of the task list, 0 for the flat and stream kernels, or minus the number of
 * shared-memory stages when the bulk-copy-staged kernel was chosen, [15]=16-byte loads in flight
 * per lane (0 for the staged kernel) (all chosen by the set-up autotuner), [16]=ns per launch of
 * the best plain candidate, [17]=ns per launch of the best staged candidate (-1 if none ran
 * correctly), [18]=autotuner candidates rejected (product differed from the first candidate's
 * beyond FP32 rounding, or a bounded wait timed out; set-up products include the preconditioner
 * blocks once they are built), [19]=kind of the chosen FP32 launch (0 row plan, 1 flat, 2
 * bulk-copy staged, 3 stream, 5 the modified Part_Schedule's task list, 6 the same tasks taken
 * in turn by persistent CTAs), [20]=CTAs per SM of that launch's shape (for the task list:
 * 4, 8 or 16, the variant), [21]=schedule of the internal products in the system matvec
 * (aim_matvec_schedule modes 0-3), [22..31]=wall time in microseconds of the set-up stages:
 * host geometry, projection stencils, internal integrals at k_i (all objects), internal
 * integrals at k0, LU solves, C = Y Z, near region, FFT of the grid kernel, GEMV autotuner,
 * matvec schedule tuner, [32]=wall time in microseconds of the last preconditioner build (0
 * before one), [33]=its precision (BEM_C32 or BEM_C64), [34]=blocks it built in FP64,
 * [35]=its largest FP32 block check (the forward-error estimate of bem_precond_setup) in units
 * of 1e-12 (-1 if none ran), [36]=wall time in microseconds of the sparse internal operator's
 * set-up (aim_internal_sparse), [37]=objects on that operator (0: none built), [38]=1 while it
 * is in use, [39]=its largest half-bandwidth, [40]=its bytes per product in complex FP32,
 * [41]=its set-up check |Z_s h - Z h| / |Z h| (largest over the objects) in units of 1e-15
 * (-1: none), [42]=1 if one of its products had a bounded wait time out (that product's e is
 * invalid; reading it synchronises the device), [43]=calls of aim_internal_tc, [44]=1 if one
 * of its products had a bounded wait time out, 0 if none did, -1 before its first call (reading
 * it synchronises the device). Writes min(n, 45) entries. */
int aim_info(const aim_ctx* ctx, int64_t* info, int n);

/* Sparse internal operator at high frequency (Sec. III-A, third item of the internal problem:
 * at small skin depth L_{k_i} and K_{k_i} are treated as sparse, physically distant
 * interactions dropped, and L^{-1} applied by a sparse direct solve). aim_setup builds it when
 * every object qualifies: a pair of RWG functions is kept when their supports come within
 * 23 skin depths delta_i = -1/Im k_i (centroid distance less the triangles' centroid-to-vertex
 * radii, nearest of the 2 x 2 triangle pairs); the kept pattern is ordered by reverse
 * Cuthill-McKee and L_s factorised as a band without pivoting (FP64, then rounded for the FP32
 * path); the band and the kept rows must be below half the dense Z's bytes, the half-bandwidth
 * at most 256, and Z_s h must match the dense Z h to 1e-8 at set-up (FP64, one probe vector).
 * Then e = Z_s h = -(1/(j k0 eps_rc)) L_s^{-1}(K_s + I_x/2) h replaces e = Z h in aim_matvec,
 * internal_apply and bem_solve (C = Y_eq Z stays dense), and is on after aim_setup. on = 0
 * selects the dense Z again, on = 1 the sparse form (BEM_EINVAL when none was built).
 * Synchronises the device; captured matvec graphs are rebuilt on next use. */
int aim_internal_sparse(aim_ctx* ctx, int on);

/* Form of the row kernels of aim_matvec, aim_matvec_batch and bem_solve (the precorrected
 * near-region rows of L^A_NR and L^Phi_NR and the interpolation W, Sec. III-A item 1): 0 (after
 * aim_setup) takes each warp lane's near-region entries four at a time while four remain and
 * the rest one at a time, one row per warp; 1 predicates the lane's last group so that its
 * loads are issued together; 2 does the same and interpolates two RWG rows per warp. All add
 * the same terms in the same order: 1 gives the same bits as 0 (up to the sign of zero), 2 the
 * same up to rounding. Drops the cached matvec graphs; synchronises the device. Errors:
 * BEM_EINVAL. */
int aim_rows_variant(aim_ctx* ctx, int variant);

/* Select the FP32 block-GEMV launch used by aim_matvec, internal_apply and bem_solve (the
 * GPU counterpart of the paper's choice of schedule for the internal products, Sec. III-C):
 * kind 0 = the set-up autotuner's choice (default), 1 = the fastest persistent register-path
 * candidate, 2 = the fastest bulk-copy-staged candidate. Waits for the device to be idle and
 * drops the captured matvec graphs. BEM_EINVAL if kind is out of range or no candidate of that
 * kind ran correctly at set-up (aim_info entries 16-17). FP64 products always use kind 1. */
int aim_gemv_select(aim_ctx* ctx, int kind);

/* Set the FP32 block-GEMV launch explicitly (reproducible timing or profiling; the autotuner's
 * choice otherwise): kind 0 row plan (ctas_per_sm 4 or 6, split 1, 2 or 4 column parts per
 * row, unroll 4, or 8 with 4 CTAs/SM), 1 flat or 3 stream ((6, unroll 4) or (4, unroll 8);
 * split ignored), 2 bulk-copy staged (ctas_per_sm 1 or 2; split, unroll ignored), 5 the task
 * list of the modified Part_Schedule (Alg. 2) over 4 CTA slots per SM, one CTA per task of at
 * most 8 * split rows (split 1, 2 or 4; unroll 4 or 8; ctas_per_sm ignored), 6 the same tasks
 * taken in turn from a counter by ctas_per_sm (1-8) persistent CTAs per SM. The launch's
 * product of a fixed vector is checked against the reference launch before it is used. Waits
 * for the device to be idle and drops the captured matvec graphs. Errors: BEM_EINVAL for an
 * unsupported shape, BEM_ECUDA if the check fails. aim_gemv_select(ctx, 0) restores the
 * autotuner's choice. */
int aim_gemv_plan(aim_ctx* ctx, int kind, int ctas_per_sm, int split, int unroll);

/* Schedule of the two internal products in the system matvec (e = Z h and j = h - C h, C =
 * Y_eq Z; the GPU counterpart of the paper's placement of the internal workload beside the
 * external one, Sec. III-C): mode 0 = e beside j's GEMV with the tuned few-CTA launch, 1 = e
 * beside the AIM chain of j once j is out, 2 = e on the main stream right after j's GEMV with
 * j's launch, 3 = both in one paired task-list launch (in j's launch shape when that is a
 * task list, else 8-row tasks on 8 warps), -1 = the set-up schedule tuner's choice. Drops the
 * captured matvec graphs; BEM_EINVAL for a mode out of range (or 3 when the set-up built no
 * paired plan). aim_info entry 21 reports it; aim_export item 8 holds the tuner's timings. */
int aim_matvec_schedule(aim_ctx* ctx, int mode);

/* y = A x for which = AIM_OP_LA (A = L^A by AIM, vectors of N_E), AIM_OP_LPHI (L^Phi, N_T)
 * or AIM_OP_SYSTEM (the SLIM system of Eq. AEFIEoutJ, vectors of N_E + N_T):
 *   e = Z h, h_eq = Y e, j = h - h_eq,
 *   y1 = j k0 L^A j + I_x e - (F D)^T L^Phi q,  y2 = F D j + j k0 q;
 * or AIM_OP_EXT (both external operators by AIM at once, vectors of N_E + N_T:
 * y = [L^A j; L^Phi q] for x = [j; q], the two run concurrently as in the system matvec).
 * x and y must not alias. prec selects the arithmetic (BEM_C32 or BEM_C64). BEM_EINVAL for an
 * unknown operator. */
int aim_matvec(aim_ctx* ctx, int which, const void* x, void* y, int prec, void* stream);

/* The system matvec of aim_matvec (AIM_OP_SYSTEM) for nrhs (1..4) right-hand sides at once:
 * x, y: device vectors of nrhs (N_E + N_T) entries, one right-hand side after another. Each
 * internal block matrix is read once for all of them and the grid convolution transforms all
 * their grids per launch, so a batch costs much less than nrhs separate products (the
 * many-right-hand-side use of the internal blocks, Sec. III-C). x and y must not alias.
 * The first call per precision allocates the batch buffers (about 130 MB in FP32 at the
 * 4x4 bar array); later calls allocate nothing. BEM_EINVAL for nrhs out of range. */
int aim_matvec_batch(aim_ctx* ctx, const void* x, void* y, int nrhs, int prec, void* stream);

/* y_i = A x_i for nvec vectors in HOST memory (x, y: nvec vectors of the operator's length,
 * one after another; page-locked memory lets the copies run asynchronously): the products of
 * aim_matvec (the system operator takes the vectors four at a time through aim_matvec_batch),
 * with the host-to-device copy of the next vectors and the device-to-host copy of the previous
 * ones overlapping the current product (two device buffer pairs kept by the context, two copy
 * streams). Ordered after the work already on `stream`; the work on `stream` after the call
 * waits for the last copy to the host, so synchronising `stream` makes y readable. x and y must
 * not alias. Errors: BEM_EINVAL (bad pointers, nvec < 1, unknown operator), BEM_ENOMEM. */
int aim_matvec_host(aim_ctx* ctx, int which, const void* x, void* y, int nvec, int prec,
                    void* stream);

/* The internal problem (Sec. II-B, Eqs. MFIEinZin, EFIEeqYeq): e = Z h, h_eq = Y e, for
 * nrhs right-hand sides stored one after another (each N_E long). Either output may be NULL
 * (not both): h_eq alone is the one block GEMV of C = Y_eq Z. With one right-hand side, both
 * outputs, the dense Z and the paired matvec schedule (aim_matvec_schedule mode 3), the two
 * products are one launch, as in the system matvec; with the sparse internal operator
 * (aim_internal_sparse) e = Z_s h. */
int internal_apply(aim_ctx* ctx, const void* h, void* e, void* heq, int nrhs, int prec,
                   void* stream);

/* The internal products of many right-hand sides at once on the tensor cores: e_r = Z h_r and
 * h_eq,r = C h_r (C = Y_eq Z; Eqs. MFIEinZin, EFIEeqYZ, block diagonal over the objects as in
 * Sec. II-C) for r < nrhs, complex FP32 (interleaved re, im), the right-hand sides stored one
 * after another, each N_E long, in the conductor-contiguous order of aim_matvec. Every block is
 * streamed from device memory once per 128 right-hand sides: each complex block product is one
 * real GEMM (TF32 tensor cores, hi/lo split of both operands for FP32 accuracy). Always the
 * dense Z, also while the sparse internal operator is on. Either output may be NULL (not both);
 * h, e and h_eq must not alias. Asynchronous on `stream`; the first call builds the per-object
 * operand descriptors and the packed right-hand-side workspace (2 x 2 x NP x sum ld_i FP32
 * values, NP = 2 nrhs rounded up to 32, 64, 128 or 256; it grows and synchronises `stream` when
 * a later call needs more). A bounded wait that times out leaves that product invalid and
 * shows in aim_info[44]. Errors: BEM_EINVAL (bad pointers, nrhs < 1, no FP32 blocks),
 * BEM_ENOMEM, BEM_ECUDA (the driver has no tensor-map encoder, or a launch failed). */
int aim_internal_tc(aim_ctx* ctx, const void* h, void* e, void* heq, int nrhs, void* stream);

/* Form of aim_internal_tc's product: 0 (after aim_setup) packs B's TF32 hi and lo parts in
 * device memory and loads both per stage; 1 packs the raw FP32 values (half the bytes) and
 * splits them in shared memory as it does the matrix. The same arithmetic: the results agree
 * to rounding. Takes effect at the next call. Errors: BEM_EINVAL. */
int aim_tc_variant(aim_ctx* ctx, int variant);

/* The grid step H of Eq. AIM_L alone: phi_c = sum_b G_grid(a - b) sigma_c(b) (linear
 * convolution) for ncomp (1..4) grids of n[0]*n[1]*n[2] points (x fastest) stored one after
 * another. sigma and phi may alias. */
int aim_conv(aim_ctx* ctx, const void* sigma, void* phi, int ncomp, int prec, void* stream);

/* y_i = A_i x_i for nblk square blocks (Sec. II-C block-diagonal Z, Y_eq). n: HOST array of
 * block sizes. A: DEVICE array, block i row-major with leading dimension ld_i = n_i rounded up
 * to a multiple of 4, blocks one after another (offsets sum of n_j*ld_j). x, y: nrhs vectors of
 * sum n_i each. */
int bem_blockdiag_gemv(int nblk, const int32_t* n, const void* A, const void* x, void* y,
                       int nrhs, int prec, void* stream);

/* The same product as bem_blockdiag_gemv for callers that cannot allocate device memory (the
 * paper has no counterpart). bem_blockdiag_gemv allocates its row-panel work list on every
 * call; this variant allocates nothing and keeps the list in a fixed 1 MiB device array built
 * into the library, which every GPU that loads the library holds until exit. It takes the
 * same arguments and gives the same result. Limit: at most 32768 panels of 16 rows, i.e. the
 * sum over blocks of ceil(n_i / 16) <= 32768 (up to 524,288 rows); larger inputs return
 * BEM_EINVAL with a message. Every call looks up the array's device address on the current
 * device (cudaGetSymbolAddress) and copies its work list there from a static host array. The
 * call cannot be captured into a CUDA graph (a replay would re-read that host array after other
 * calls rewrote it): while `stream` is capturing it returns BEM_EINVAL and does nothing. All
 * calls share the one array: calls whose GPU work overlaps (other streams, other threads) race
 * on it. */
int bem_blockdiag_gemv_noalloc(int nblk, const int32_t* n, const void* A, const void* x, void* y,
                               int nrhs, int prec, void* stream);

/* Copy a setup product to HOST memory `out` (capacity cap bytes, at least the size needed):
 *   what 0: Z_i (complex double, row-major n_i x n_i), index = object
 *   what 1: Y_i (same)
 *   what 2: near-region L^A_NR as CSR: int64 rowptr[N_E+1], int32 col[nnz], complex double
 *           val[nnz], packed one after another
 *   what 3: near-region L^Phi_NR (same layout, N_T rows)
 *   what 4: RWG projection weights, double [N_E][3][27]
 *   what 5: pulse projection weights, double [N_T][27]
 *   what 6: stencil anchors, int32 [N_E + N_T][3]
 *   what 7: edge table, int32 [N_E][6] = (a, b, T+, T-, v+, v-)
 *   what 8: the set-up autotuners' table, float [candidates][5] = (kind: 0 row plan,
 *           1 flat, 2 bulk-copy staged, 3 stream, 5 Part_Schedule task list (one CTA per
 *           task), 6 the same tasks taken in turn by persistent CTAs; CTAs per SM; column parts
 *           per row, or rows per task / 8 for kinds 5 and 6; loads in flight per lane; ns per
 *           launch, or -1 when the candidate was rejected or not applicable), then the
 *           system-matvec schedules (4; CTAs per SM of the e = Z h launch that runs beside the
 *           AIM chain, 0 when it runs on the main stream; 0 = it starts with j's GEMV, 1 = after
 *           it beside the chain, 2 = after it on the main stream with j's launch shape, 3 = both
 *           in one paired launch; kind of that launch; ns per matvec), then the
 *           multi-right-hand-side GEMV shapes of the batched matvec (7; 16; rows per warp; 4;
 *           ns per launch of 4 right-hand sides)
 *   what 9: the dense L_k of object index / 2 (Sec. II-B: the EFIE operator of the object's
 *           interior, k = k_i, when index is even; of the background, k = k0, when odd), as the
 *           set-up forms it before the LU solve of Eqs. MFIEinZin / EFIEeqYeq: complex double,
 *           row-major n_i x n_i. Recomputed on the device for the call (FP64 integrals).
 *   what 10: K_k + I_x/2 of the same object and wavenumber (same layout)
 * Returns the number of bytes needed when out is NULL. */
int64_t aim_export(const aim_ctx* ctx, int what, int index, void* out, int64_t cap);

/* b = [<f_m, E_inc>/eta0 ; 0] for E_inc = pol exp(-j k0 khat . r) (unit amplitude, V/m),
 * Sec. II-A right-hand side. pol and khat are host arrays of 3 doubles. */
int bem_rhs_plane_wave(aim_ctx* ctx, const double* pol, const double* khat, void* b, int prec,
                       void* stream);

/* Lumped ports. The paper excites structures through lumped ports (Sec. II, after Wang 2004)
 * without giving the model; reading: a delta gap on a closed ring of mesh edges around a
 * conductor's cross-section. bem_port_ring lists the edges of object obj whose two vertices lie
 * within tol of the plane x_axis = coord (micrometres), with s_m = +1 when the RWG function
 * f_m crosses the plane towards +axis, -1 otherwise. edges and signs are HOST arrays receiving
 * the first min(count, cap) entries (NULL: count only). Returns the count or BEM_EINVAL. */
int bem_port_ring(aim_ctx* ctx, int obj, int axis, double coord, double tol, int32_t* edges,
                  double* signs, int cap);

/* b = [s_m l_m V / (eta0 ell) on the ring edges (l_m in micrometres, ell = 1e-6 m), 0 on the
 * other edges; 0 on the triangles]: the delta-gap excitation <f_m, E_inc> / eta0 of a gap
 * voltage V (volts) in the micrometre scaling of bem_rhs_plane_wave (the first block row is the
 * SI row divided by ell^2), so that the solution's h is H in A/m. edges, signs: HOST arrays of n
 * entries (from bem_port_ring). b: device vector of N_E + N_T in prec. Synchronises the stream.
 * Errors: BEM_EINVAL for an empty port or an edge out of range. */
int bem_rhs_port(aim_ctx* ctx, int n, const int32_t* edges, const double* signs, double v_gap,
                 void* b, int prec, void* stream);

/* Port current I = sum_m s_m l_m h_m of the solution x = [h; q] (device, prec): the
 * circulation of H around the ring (Ampere's law), in amperes (h in A/m, lengths converted to
 * metres). The port admittance is Y_pq = I_p / V_q. current: HOST, 2 doubles (re, im).
 * Synchronises the stream. */
int bem_port_current(aim_ctx* ctx, int n, const int32_t* edges, const double* signs,
                     const void* x, int prec, double* current, void* stream);

/* Radiation vector N(rhat) = int J_Delta(r') exp(j k0 rhat . r') dS' of the solution x = [h; q]
 * (device, prec), with J_Delta = sum_n j_n f_n and j = h - Y_eq Z h: in the equivalent problem
 * only J_Delta radiates into the background (Sec. II). The far field is
 * E(r) = -j k0 eta0 exp(-j k0 r) / (4 pi r) (I - rhat rhat) N, so the monostatic RCS of a unit
 * plane wave is sigma = k0^2 eta0^2 |(I - rhat rhat) N|^2 / (4 pi) (um^2, k0 in 1/um).
 * The integral uses the 7-point rule per triangle, accumulated in FP64. rhat: HOST [ndir][3]
 * unit vectors; nvec: HOST [ndir][3] complex doubles (re, im interleaved), in (A/m) um^2. Uses
 * the context's internal work vectors (as aim_matvec does); synchronises the stream. */
int bem_farfield(aim_ctx* ctx, const void* x, int prec, int ndir, const double* rhat,
                 double* nvec, void* stream);

/* Options of bem_solve. prec_mode: BEM_C64 (plain: FP64 everywhere) or BEM_C32 (system
 * matvec in complex FP32, Arnoldi and Givens in FP64). */
typedef struct {
  double tol;          /* relative residual target, e.g. 1e-6 */
  int32_t restart;     /* Krylov subspace size before restart, 1..512 */
  int32_t max_iter;
  int32_t prec_mode;
  int32_t precond;     /* 0 = none, 1 = block-diagonal (bem_precond_apply), 2 = block-diagonal
                          plus the learned correction (bem_net_apply); on the right */
  double time_limit_s; /* <= 0: none */
} bem_solve_opts;

/* u = M r with the block-diagonal preconditioner M = blockdiag(A_ii^{-1}): A_ii is the system
 * of Eq. AEFIEoutJ restricted to object i's unknowns [h_i; q_i] with the object's exact dense
 * L^A and L^Phi (the paper's own constraint preconditioner, from Qian 2009, is not given in the
 * paper; this is the fallback). The first call (or the first bem_solve with precond = 1) builds
 * the inverses as bem_precond_setup(ctx, BEM_C32) does; they are stored in FP64 and FP32.
 * r, u: device vectors of N_E + N_T in the precision prec; they must not alias. */
int bem_precond_apply(aim_ctx* ctx, const void* r, void* u, int prec, void* stream);

/* Build (or rebuild) the inverses of bem_precond_apply in the precision build_prec. BEM_C32
 * (what the first bem_precond_apply or preconditioned bem_solve uses): each A_ii is formed,
 * LU-factorised and inverted in complex FP32, then checked with four pseudo-random columns V:
 * the first iterative-refinement correction relative to X V, ||X (A_ii X V - V)||_F /
 * ||X V||_F, estimates the inverse's forward error; a block above 1e-2 is rebuilt in FP64. BEM_C64: every block in FP64. L^A_ii and L^Phi_ii are FP64 integrals in both cases.
 * aim_info entries 32-35 report the build. Synchronises the device. */
int bem_precond_setup(aim_ctx* ctx, int build_prec);

typedef struct {
  int32_t iters;
  double resid_est;   /* Arnoldi estimate at exit */
  double resid_true;  /* ||b - A x|| / ||b|| with the FP64 system matvec */
  double seconds;
} bem_solve_info;

/* Solve A x = b (Eq. AEFIEoutJ) with restarted GMRES on the device (Sec. III-E). b and x
 * are complex double device vectors of N_E + N_T; x holds the initial guess on entry (all
 * zeros: none, and the first residual needs no matvec) and the solution on exit. The Krylov
 * workspace ((m+1) + m vectors of N_E + N_T complex doubles with a preconditioner, m + 1
 * without; m = restart) is allocated by the first solve that needs it and kept by the context
 * for later solves (freed by aim_destroy). Returns BEM_OK when the true residual reaches tol,
 * BEM_ENOCONV (positive) when max_iter or the time limit stops it first. */
int bem_solve(aim_ctx* ctx, const void* b, void* x, const bem_solve_opts* opts,
              bem_solve_info* info, void* stream);

/* bem_solve for nrhs (1..4) right-hand sides at once: b and x hold nrhs complex double device
 * vectors of N_E + N_T, one after another (x: initial guesses in, solutions out). The systems
 * run in lockstep, each with its own Krylov basis: every iteration applies the preconditioner
 * and the system matrix to all of them together (aim_matvec_batch; the block matrices are read
 * once per iteration for all right-hand sides), and a cycle ends when every residual estimate is
 * below tol. opts as for bem_solve with precond 0 or 1 (the learned correction is not batched).
 * infos: HOST [nrhs] (or NULL), iterations and residuals per right-hand side. The batched
 * workspace ((2m + 4) nrhs vectors) is kept by the context. Returns BEM_OK when every true
 * residual reaches tol, BEM_ENOCONV otherwise. */
int bem_solve_batch(aim_ctx* ctx, const void* b, void* x, int nrhs, const bem_solve_opts* opts,
                    bem_solve_info* infos, void* stream);

/* Port admittance matrix: for each port q, the solve (bem_solve with opts) of a unit gap
 * voltage on q with the other ports shorted, then the currents of every port p:
 * Y[p][q] = I_p / V_q in siemens (the paper's port excitation, Sec. II; its S-parameter and
 * impedance outputs follow from Y). Ports are given as rings (bem_port_ring): ring_n[p] edges
 * each, edges and signs HOST arrays holding the rings one after another. Y: HOST
 * [nport][nport] complex doubles (re, im interleaved); infos: HOST [nport] (or NULL), the
 * solve information of each column. With precond 0 or 1 the ports are solved up to four at a
 * time (bem_solve_batch). Allocates device vectors for the group's right-hand sides and
 * solutions for the call; synchronises the stream. Returns BEM_OK, BEM_ENOCONV when a solve stopped
 * before tol (Y is still filled), or a negative error (BEM_EINVAL for an empty port or an edge
 * out of range). */
int bem_port_matrix(aim_ctx* ctx, int nport, const int32_t* ring_n, const int32_t* edges,
                    const double* signs, const bem_solve_opts* opts, double* Y,
                    bem_solve_info* infos, void* stream);

/* Learned correction of the preconditioner (an extension; not in the paper). A 4-layer 3-D
 * convolutional net on the AIM grid (3x3x3 kernels, zero padding, no biases, ReLU between
 * layers, channels 8-16-16-16-8; BF16 weights and activations, FP32 sums) maps the projected
 * residual P r (Re/Im of the four grid components, scaled by their RMS) to a grid correction:
 *   M(r) = M_bd r + W net(P r),  W = P^T (Sec. III-A item 1 operators).
 * Weight layout: layer after layer, each [C_out][C_in][3][3][3] (dz, dy, dx), FP32; 20736 in all.
 * bem_net_init: He-normal weights from a splitmix64 counter hash of seed.
 * bem_net_weights: copy weights from (set = 1) or to (set = 0) the HOST array w of n floats;
 *   with w = NULL returns the number of weights.
 * bem_net_train: `steps` Adam steps of lr on batches of `batch` pairs r = A x (x complex normal
 *   from the hash of seed, half of them smoothed on the grid), minimising the grid-projected
 *   error |P (W net(P r) - t)|^2 / |P t|^2 with t = x - M_bd r; losses
 *   (HOST, may be NULL) receives the mean loss of each step. Builds M_bd in FP64
 *   (bem_precond_setup(ctx, BEM_C64)) unless it is so built already: t carries M_bd's own error.
 * bem_net_apply: z = M_bd r + W net(P r) for complex FP32 device vectors of N_E + N_T
 *   (z = W net(P r) alone when correction_only is non-zero).
 * bem_convnet_run: the network alone on an nx x ny x nz grid, for verification: x [8][ng] FP32
 *   device input (rounded to BF16), w_host FP32 weights (rounded to BF16), out [8][ng] FP32
 *   device output; when gout [8][ng] is given, the backward pass writes gw_host (FP32 host,
 *   may be NULL) and gx [8][ng] (device, may be NULL). Synchronous on stream. */
int bem_net_init(aim_ctx* ctx, uint64_t seed);
int64_t bem_net_weights(aim_ctx* ctx, float* w, int64_t n, int set);
int bem_net_train(aim_ctx* ctx, int steps, int batch, float lr, uint64_t seed, float* losses,
                  void* stream);
int bem_net_apply(aim_ctx* ctx, const void* r, void* z, int correction_only, void* stream);
int bem_convnet_run(int nx, int ny, int nz, const float* w_host, const float* x, const float* gout,
                    float* out, float* gw_host, float* gx, void* stream);

/* Work lists for uneven block-diagonal products (Sec. III-C): LPT (Alg. 1) and the modified
 * Part_Schedule (Alg. 2). W: HOST task weights sorted in decreasing order (W_i = n_i^2);
 * P processors; p_cutoff <= 0 selects the original Part_Schedule. Outputs: Pi[ntask]
 * processors per task; returns the schedule length C_max (negative on error). */
double bem_part_schedule(int ntask, const double* W, int P, int p_cutoff, int32_t* Pi);

/* The ordering behind the sparse internal operator's band (aim_internal_sparse), host only:
 * reverse Cuthill-McKee (Cuthill and McKee 1969, reversed) of a symmetric pattern of n
 * vertices given as HOST CSR (rowptr[n + 1], cols[rowptr[n]]; self loops ignored): from each
 * component's vertex of least degree (lowest index on ties), breadth first with the unvisited
 * neighbours in increasing degree (ties in the order of the row's columns), the whole sequence
 * reversed. order[r] (HOST, n) receives the
 * vertex at position r. Errors: BEM_EINVAL (bad pointers, decreasing row pointers, a column
 * outside [0, n)). The pattern's symmetry is the caller's to ensure. */
int bem_rcm_order(int n, const int32_t* rowptr, const int32_t* cols, int32_t* order);

/* A planar stratified background (the layered media of Table I): nlayer layers bottom-up,
 * each a thickness in um and a complex relative permittivity (re, im; exp(j w t), so im <= 0
 * in a lossy layer: eps_r - j sigma / (w eps0)); a half-space of top_eps above; under layer 0
 * a perfectly conducting plane at z = 0 (ground = 1) or a half-space of bottom_eps
 * (ground = 0). Non-magnetic. The caller owns the arrays. */
typedef struct {
  int32_t nlayer;
  const double* thickness;   /* [nlayer] um */
  const double* eps;         /* [nlayer][2] */
  double top_eps[2];
  int32_t ground;
  double bottom_eps[2];
} bem_stack;

/* Set-up of the AIM grid step inside one layer of a stratified background (Table I): the
 * tables of phi(a) = sum_b [G_T(rho_ab, z_a - z_b) + G_H(rho_ab, z_a + z_b)] sigma(b) for the
 * grid of nodes origin + (i, j, k) h, i < n[0], j < n[1], k < n[2], whose node planes must lie
 * strictly inside one layer. kind 0: G^A_xx (= G^A_yy, the x and y current components), 1:
 * G^A_zz, 2: G^Phi (times the layer's relative permittivity); each equals G(k_n, R) =
 * e^{-j k_n R} / (4 pi R) in a homogeneous medium of the layer's wavenumber k_n. Green's
 * functions of the transmission-line form of the stratified medium for sources and observers
 * in the same layer (no x-z coupling of horizontal currents); Sommerfeld integrals of the
 * reflected terms. Outputs (HOST, caller-owned, complex double as (re, im) pairs):
 * T[dz + n[2] - 1][dy][dx] for dz = -(n[2]-1) .. n[2]-1 (the direct term included, 0 at
 * R = 0) and H[s][dy][dx] for s = k_a + k_b = 0 .. 2 n[2] - 2, dx < n[0], dy < n[1]: each
 * (2 n[2] - 1) n[1] n[0] complex values. Host computation only; its cost grows with
 * n[0] n[1] (at most 65536) times the integration path's length. Errors: BEM_EINVAL (bad
 * arguments or layers), BEM_EGRID (bad grid, or node planes not inside one layer). */
int bem_layered_grid_tables(const bem_stack* stack, double freq_hz, const double* origin,
                            const double* h, const int32_t* n, int kind, double* T, double* H);

/* The reflected part of one of a layer's Green's functions (kind as above) on a tensor grid,
 * for interpolation where sources and observers are not grid nodes (the near-region entries
 * of objects inside the layer): part 0, the doubly reflected (Toeplitz) terms at arg = z - z'
 * (|arg| below the layer's thickness); part 1, the singly reflected (Hankel) terms at
 * arg = z + z' (strictly between twice the layer's bottom and top). out[j][i] (HOST,
 * caller-owned, complex double as (re, im) pairs) at rho[i] >= 0 and arg[j], nrho narg at most
 * 2^26. The direct term is not included. Host computation only. Errors: BEM_EINVAL. */
int bem_layered_kernel_table(const bem_stack* stack, double freq_hz, int layer, int kind,
                             int part, int nrho, const double* rho, int narg, const double* arg,
                             double* out);

#ifdef __cplusplus
}
#endif
#endif /* BEM_AIM_H */
