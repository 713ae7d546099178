// Shared definitions of the GB300 SLIM library: error handling, complex helpers, context.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "../../include/bem_aim.h"

namespace bem {

void set_error(const char* fmt, ...);

#define BEM_CUDA(call)                                                              \
  do {                                                                             \
    cudaError_t _e = (call);                                                       \
    if (_e != cudaSuccess) {                                                       \
      ::bem::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(_e)); \
      return BEM_ECUDA;                                                            \
    }                                                                              \
  } while (0)

#define BEM_TRY(call)            \
  do {                           \
    int _r = (call);             \
    if (_r < 0) return _r;       \
  } while (0)

// ---------------------------------------------------------------------------------------
// complex arithmetic on float2 / double2 (interleaved re, im)
// ---------------------------------------------------------------------------------------
template <typename R> struct C2;
template <> struct C2<float> { typedef float2 T; };
template <> struct C2<double> { typedef double2 T; };

__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
template <typename V> __host__ __device__ __forceinline__ V cadd(V a, V b) { return mk(a.x + b.x, a.y + b.y); }
template <typename V> __host__ __device__ __forceinline__ V csub(V a, V b) { return mk(a.x - b.x, a.y - b.y); }
template <typename V> __host__ __device__ __forceinline__ V cmul(V a, V b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename V> __host__ __device__ __forceinline__ V cconj(V a) { return mk(a.x, -a.y); }
template <typename V> __host__ __device__ __forceinline__ V czero();
template <> __host__ __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }
template <> __host__ __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }
template <typename V, typename R> __host__ __device__ __forceinline__ V cscale(V a, R s) {
  return mk(a.x * s, a.y * s);
}
// a += b * c
template <typename V> __host__ __device__ __forceinline__ void cfma(V& a, V b, V c) {
  a.x = fma(b.x, c.x, fma(-b.y, c.y, a.x));
  a.y = fma(b.x, c.y, fma(b.y, c.x, a.y));
}
__device__ __forceinline__ void cfma(float2& a, float2 b, float2 c) {
  a.x = fmaf(b.x, c.x, fmaf(-b.y, c.y, a.x));
  a.y = fmaf(b.x, c.y, fmaf(b.y, c.x, a.y));
}

template <typename V> __device__ __forceinline__ V warp_sum(V v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

static inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// ---------------------------------------------------------------------------------------
// one FFT length: radix plan and twiddle table e^{-2 pi i k / P}
// ---------------------------------------------------------------------------------------
constexpr int kMaxStages = 16;
struct FftPlan {
  int P = 0;
  int nst = 0;
  int rad[kMaxStages] = {0};
  // exact division by multiply-high: q = umulhi(n, mag) for n < 2^16 and divisors < 2^11
  uint32_t mag_m[kMaxStages] = {0};   // divisor m_s = P / R_s
  uint32_t mag_ns[kMaxStages] = {0};  // divisor Ns_s = R_0 ... R_{s-1} (0 when Ns_s = 1)
};
static inline uint32_t div_magic(uint32_t d) {
  return d <= 1 ? 0u : (uint32_t)(((1ull << 32) + d - 1) / d);
}
bool make_fft_plan(int P, FftPlan* plan);
int smooth_length(int need);  // smallest length >= need whose factors are 2, 3, 5, 7

// ---------------------------------------------------------------------------------------
// precision-specific device buffers
// ---------------------------------------------------------------------------------------
template <typename R> struct PrecBuf {
  typedef typename C2<R>::T V;
  V* Z = nullptr;      // packed row-major blocks (ld_i = round_up(n_i, 4))
  V* Y = nullptr;      // Y_eq blocks, FP64 only (export and preconditioner set-up)
  V* C = nullptr;      // C_i = Y_i Z_i (Eq. EFIEeqYZ: h_eq = Y_eq Z h), same layout as Z
  R* WA = nullptr;     // [ne][3][27] projection weights of RWG functions
  R* WP = nullptr;     // [nt][27] projection weights of pulses
  R* WAT = nullptr;    // [nnzPe][3] the same weights in grid-node-major (CSR) order
  R* WPT = nullptr;    // [nnzPt]
  V* LA = nullptr;     // near-region values (CSR, shared structure with the host arrays)
  V* LP = nullptr;
  V* Ghat = nullptr;   // octant of the scaled FFT of the circulant grid kernel
  V* Gz = nullptr;     // FP32: Ghat per z line [Py][Px][M][L] in the register z pass's lane order
  V* Gs = nullptr;     // FP32, slab passes: Ghat octant as [fx][fz][fy]
  V* tw[3] = {nullptr, nullptr, nullptr};  // twiddle tables of the three axes
  R* ix = nullptr;     // [ne][4] I_x values
  R* fdE = nullptr;    // [ne][2] (l/A+, l/A-) : (F D)^T rows
  R* fdT = nullptr;    // [nt][3] signed l/A for the triangle's edges : F D rows
  // workspaces
  V* sigma = nullptr;  // [4][ng]
  V* ws = nullptr;     // [4][Pz][Py][Px]
  V* e = nullptr;      // [ne]
  V* heq = nullptr;    // [ne]
  V* j = nullptr;      // [ne]
  V* p = nullptr;      // [nt]
  V* anear = nullptr;  // [ne] near-region part L^A_NR j of the system matvec
  // batched system matvec (up to kMaxBatch right-hand sides; made on first use): j and e with
  // the input's stride N_E + N_T, L^A_NR j [r][ne], p [r][nt], grids [r][3][ng] and [r][ng],
  // FFT workspaces [3 r][P3] and [r][P3]
  V *bj = nullptr, *be = nullptr, *ban = nullptr, *bp = nullptr, *bsE = nullptr, *bsT = nullptr,
    *bwsE = nullptr, *bwsT = nullptr;
  V* xin = nullptr;    // [ne + nt] conversion buffer for mixed precision
  V* yout = nullptr;
};

struct GemvTask {  // a run of rows of one block
  int64_t aoff;    // element offset of the block
  int32_t xoff;    // first unknown of the block
  int32_t n;       // block size
  int32_t ld;
  int32_t row0;
  int32_t nrows;
  int32_t sel;     // paired launch: 0 = first matrix (y0, minus from hsub), 1 = second (y1)
};

struct RowInfo {   // one row of the block-diagonal matrix (global row = output index)
  int64_t aoff;    // element offset of the row's first entry
  int32_t n;       // row length (block size)
  int32_t xoff;    // first unknown of the block
};

struct TmaStage {  // whole rows [r0, r1) streamed as one bulk copy of nel complex elements
  int32_t r0, r1;
  int64_t e0;      // element offset of the first row
  int32_t nel;
  int32_t pad;
};
// Row table of one stage, bulk-copied into shared memory beside the stage's matrix bytes so
// the consumers never wait on global memory for it.
constexpr int kTmaMaxRows = 64;  // rows per stage
struct TmaDesc {
  int32_t r0, nr, nel, pad;        // first global row, rows, complex elements in the stage
  int32_t soff[kTmaMaxRows + 4];   // element offset of row k inside the stage; soff[nr] = nel
  int32_t n[kTmaMaxRows];          // row length (block size)
  int32_t xoff[kTmaMaxRows];       // offset of the block's slice of x
};
static_assert(sizeof(TmaDesc) % 16 == 0, "bulk copies move multiples of 16 bytes");

// Persistent launch of a block-diagonal product: CTA p streams the rows of its segments
// [seg[cta_seg[p]], ..., seg[cta_seg[p+1]-1]], each a range [r0, r1) of global rows. With
// tma set, the rows are fed through shared-memory stages by bulk copies (gemv_tma.cu); with
// flat set, a CTA's rows are read as chunks of whole rows described like the stages.
struct GemvPlan {
  RowInfo* rows = nullptr;   // device [nrows]
  int2* segs = nullptr;      // device [nseg]
  int32_t* cta_seg = nullptr;// device [ncta + 1]
  int ncta = 0;
  int nrows = 0;
  int cps = 0;                 // the shape's CTAs per SM (as asked of make_gemv_plan)
  int split = 2;               // column parts per row (1, 2 or 4), picked by the autotuner
  int unroll = 4;              // 16-byte loads in flight per lane (4 or 8), likewise
  int flat = 0;                // flat form: rows in chunks (stages, descs, cta_stage as chunks)
  int stream = 0;              // stream form: equal vector shares per warp, atomic row sums
  GemvTask* tasks = nullptr;   // task-list form: the modified Part_Schedule's row panels
  int ntasks = 0;              //   (one CTA per task of <= 8 * split rows), when non-zero
  int task_form = 0;           // task list, one right-hand side: 0 = 8 warps per CTA, 1 = 8
                               //   warps and 8 resident CTAs per SM (32 registers), 2 = 4 warps,
                               //   16 resident CTAs per SM, tasks of <= 4 * split rows
  int* ctr = nullptr;          // dynamic task list: device [2] = next task, CTAs finished; the
                               //   ncta persistent CTAs take tasks in turn (zero between launches)
  int32_t* wrow = nullptr;     // device [warps]: row holding each warp's first vector
  int64_t nquad = 0;           // whole block storage in units of 4 complex elements
  double cmax_over_ideal = 0;  // schedule length / (total work / ncta)
  // bulk-copy staging
  int tma = 0;
  TmaStage* stages = nullptr;  // device
  int32_t* cta_stage = nullptr;// device [ncta + 1]
  TmaDesc* descs = nullptr;    // device [stages] row tables
  int nstage = 4;              // buffers in the ring
  int stage_bytes = 0;
  int* err = nullptr;          // device: non-zero after a bounded wait timed out
};
bool build_tma_stages(const std::vector<RowInfo>& rows, const std::vector<int2>& segs,
                      const std::vector<int32_t>& cta_seg, int64_t stage_elems,
                      std::vector<TmaStage>* stages, std::vector<int32_t>* cta_stage,
                      std::vector<TmaDesc>* descs);
int tma_init_attrs();
template <typename R>
int run_gemv_tma(const GemvPlan& p, const typename C2<R>::T* A, const typename C2<R>::T* x,
                 typename C2<R>::T* y, int nrhs, int64_t vstride, const typename C2<R>::T* hsub,
                 cudaStream_t s);
void build_gemv_plan(const std::vector<int32_t>& n, const std::vector<int64_t>& off,
                     const std::vector<int32_t>& ld, int ncta, std::vector<RowInfo>* rows,
                     std::vector<int2>* segs, std::vector<int32_t>* cta_seg, double* ratio);
// physical constants (SI) and the length unit of the library (micrometre)
constexpr double kC0 = 299792458.0;
constexpr double kMu0 = 4e-7 * 3.14159265358979323846;
constexpr double kEps0 = 1.0 / (kMu0 * kC0 * kC0);
constexpr double kEta0 = kMu0 * kC0;
constexpr double kEll = 1e-6;
// Radon's 7-point degree-5 rule on the triangle: (l1, l2, l3, w) x 7, weights summing to one
void radon7_host(double* out);
constexpr int kGemvThreads = 256;
constexpr int kGemvCtasPerSm = 6;

}  // namespace bem

struct aim_ctx {
  int device = 0;
  int ne = 0, nt = 0, nobj = 0, nv = 0;
  int gn[3] = {0, 0, 0};
  int gp[3] = {0, 0, 0};  // padded FFT lengths
  double go[3], gh[3];
  int64_t ng = 0;
  int r_near = 2;
  double freq = 0, k0 = 0;
  // host copies
  std::vector<double> verts;          // [nv*3]
  std::vector<int32_t> tris;          // [nt*3]
  std::vector<int32_t> obj_t;
  std::vector<bem_material> mat;
  std::vector<int32_t> ev, et, eopp;  // [ne*2]
  std::vector<int32_t> obj_e;
  std::vector<double> elen, area, normal, centroid, diam;
  std::vector<int32_t> t_edges, t_esign, t_evert;  // [nt*3]
  std::vector<int32_t> e0, e1, t0, t1;             // object ranges
  std::vector<int32_t> anc;                        // [(ne+nt)*3]
  std::vector<int64_t> rowA, rowP;                 // near CSR row pointers
  std::vector<int32_t> colA, colP;
  // the same columns as one list per anchor node (cl) and each row's offset into it (lst)
  std::vector<int64_t> lstA, lstP;
  std::vector<int32_t> clA, clP;
  std::vector<int64_t> zoff;                       // element offset of block i
  std::vector<int32_t> zld;
  int64_t zelems = 0;
  bem::GemvPlan gplan;    // FP32 products (autotuned; may use bulk-copy staging)
  bem::GemvPlan gplan64;  // FP64 products
  bem::GemvPlan gbg32, gbg64;  // e = Z h beside the AIM chain in the system matvec (few CTAs)
  bem::GemvPlan gpair;         // j = h - C h and e = Z h as one task list (both precisions)
  bem::GemvPlan gmr;           // several right-hand sides: task list of 16-row tasks (k_gemv_mr)
  bem::GemvPlan gplan_auto;    // the autotuner's FP32 choice
  bem::GemvPlan gplan_alt[2];  // best plain and best staged FP32 plans (ncta = 0: none)
  // wall time of the set-up stages in ms (aim_info entries 22-31): host geometry, stencils,
  // internal integrals at k_i, internal integrals at k0, LU solves, C = Y Z, near region,
  // FFT of the grid kernel, GEMV autotuner, matvec schedule tuner
  double setup_ms[11] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};  // [10]: sparse internal operator
  float tune_ms[2] = {0, 0};  // autotuner: best plain, best staged candidate (5 launches, ms)
  int tune_rejected = 0;      // autotuner candidates rejected (wrong product or timed out)
  std::vector<float> tune_table;  // autotuner: (kind, cps, split, unroll, ns) per candidate
  bem::FftPlan plan[3];
  // device: integer tables
  int32_t* d_nodeE = nullptr;  // [ne] linear index of the anchor node
  int32_t* d_nodeT = nullptr;  // [nt]
  // projection P as grid-node-major CSR (row = grid node, entries = sources touching it)
  int32_t* d_prowE = nullptr;  // [ng + 1]
  int32_t* d_pcolE = nullptr;  // [27 ne] source (RWG) index
  int32_t* d_prowT = nullptr;  // [ng + 1]
  int32_t* d_pcolT = nullptr;  // [27 nt] source (triangle) index
  // grid nodes with at least one entry in P (work list of the projection) and the others
  // (zero-filled by the same launch); [0, nwE) then [nwE, ng) for RWG, likewise for pulses
  int32_t* d_pnodeE = nullptr;  // [ng]
  int32_t* d_pnodeT = nullptr;  // [ng]
  int32_t nwE = 0, nwT = 0;
  int64_t* d_rowA = nullptr;
  int32_t* d_colA = nullptr;  // per entry (set-up kernels)
  int64_t* d_lstA = nullptr;  // per row: offset of its anchor's list in d_clA
  int32_t* d_clA = nullptr;
  int64_t* d_lstP = nullptr;
  int32_t* d_clP = nullptr;
  int64_t* d_rowP = nullptr;
  int32_t* d_colP = nullptr;
  int32_t* d_ixcol = nullptr;  // [ne][4]
  int32_t* d_et = nullptr;     // [ne][2]
  int32_t* d_tedge = nullptr;  // [nt][3]
  bem::PrecBuf<float> f32;
  bem::PrecBuf<double> f64;
  std::vector<void*> allocs;   // every device allocation, freed by aim_destroy
  void* geo_store = nullptr;   // device geometry descriptor (set-up kernels, right-hand sides)
  // streams of the system matvec (main, charge side, e = Z h side) and its CUDA-graph capture
  cudaStream_t cap = nullptr, side = nullptr, zside = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_z = nullptr, ev_c = nullptr;
  // host-buffer matvecs: two device buffer pairs, copy streams and their events (lazily made)
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_comp[2] = {nullptr, nullptr},
              ev_out[2] = {nullptr, nullptr};
  void* hbuf[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [buffer][x, y]
  size_t hbuf_bytes = 0;
  int z_after = 0;  // e = Z h: 0 beside j's GEMV, 1 beside the AIM chain once j = h - C h is
                    // out, 2 on the main stream after j's GEMV with the whole GPU, 3 in one
                    // launch with j's GEMV (gpair)
  int z_tuned = 0;  // the schedule tuner's choice of z_after
  struct GKey {
    int which, prec;
    const void* x;
    void* y;
    bool operator<(const GKey& o) const {
      if (which != o.which) return which < o.which;
      if (prec != o.prec) return prec < o.prec;
      if (x != o.x) return x < o.x;
      return y < o.y;
    }
  };
  std::map<GKey, cudaGraphExec_t> graphs;  // captured matvecs, keyed by operator and buffers
  bool use_graphs = true;
  // block-diagonal preconditioner: explicit inverses of the per-object blocks A_ii, packed
  // row-major in object-major unknown order ([h_i; q_i] per object), built on first use
  bool pc_ready = false;
  bool pc_planned = false;  // the GEMV plans over the blocks exist (made by the first build)
  int pc_prec = 0;          // precision of the last build (BEM_C32 or BEM_C64)
  int pc_nfp64 = 0;         // blocks built in FP64 by that build
  double pc_resid = 0;      // largest FP32 block check ||X (A X V - V)||_F / ||X V||_F
  double pc_ms = 0;         // wall time of that build
  bem::GemvPlan pcplan;
  bem::GemvPlan pcplan64;
  float2* pc32 = nullptr;
  double2* pc64 = nullptr;
  int32_t* d_pcperm = nullptr;  // object-major position -> system index
  float2* pcw32[2] = {nullptr, nullptr};
  double2* pcw64[2] = {nullptr, nullptr};
  bem::GemvPlan pcmr;                        // several right-hand sides (k_gemv_mr)
  float2* pcb32[2] = {nullptr, nullptr};     // [kMaxBatch][N] work vectors of the batched apply
  // batched FGMRES: workspace kept between solves, batched FP32 / FP64 vectors [kMaxBatch][N]
  void* gmb_ws = nullptr;
  size_t gmb_bytes = 0;
  // GMRES workspace kept between solves (gmres.cu)
  void* gm_ws = nullptr;
  size_t gm_bytes = 0;
  // far-field geometry (post.cu), built on first use
  void* far_geo = nullptr;
  // learned correction network on the AIM grid (learned.cu)
  void* net = nullptr;
  // sparse internal operator at high frequency (zsparse.cu): built at set-up when every object
  // qualifies (zsp_ready), used for e = Z h while zsp_on
  void* zsp = nullptr;
  bool zsp_ready = false, zsp_on = false;
  // many right-hand sides through Z and C on the tensor cores (zgemm_tc.cu), made on first use
  void* tc = nullptr;
  // form of that product (aim_tc_variant): 0 B's hi and lo packed in device memory, 1 the raw B
  // packed and split in shared memory
  int tc_variant = 0;
  // form of the row kernels (aim_rows_variant): 0 near sums four-deep with a one-entry tail,
  // 1 four-deep predicated, 2 predicated and two interpolation rows per warp (k_rows_e2)
  int rows_variant = 0;
};

namespace bem {
int dalloc(aim_ctx* c, void** p, size_t bytes);
template <typename T> int dalloc_t(aim_ctx* c, T** p, size_t count) {
  return dalloc(c, reinterpret_cast<void**>(p), count * sizeof(T));
}
template <typename T> int upload(aim_ctx* c, T** p, const T* host, size_t count) {
  BEM_TRY(dalloc_t(c, p, count));
  if (count) BEM_CUDA(cudaMemcpy(*p, host, count * sizeof(T), cudaMemcpyHostToDevice));
  return BEM_OK;
}

// geometry (host, geom.cpp)
int build_geometry(aim_ctx* c, const bem_mesh* m, const aim_grid* g);
// scheduling (host, sched.cpp)
void build_gemv_tasks(const std::vector<int32_t>& n, const std::vector<int64_t>& off,
                      const std::vector<int32_t>& xoff, const std::vector<int32_t>& ld,
                      int nsm, int rows_per_task, std::vector<GemvTask>* tasks);
// setup (setup.cu)
int setup_device(aim_ctx* c);
// hot path (hot.cu)
template <typename R>
int run_gemv(const GemvTask* d_tasks, int ntasks, const typename C2<R>::T* A,
             const typename C2<R>::T* x, typename C2<R>::T* y, int nrhs, int64_t vstride,
             const typename C2<R>::T* hsub, cudaStream_t s);
template <typename R>
int run_gemv_mr(const GemvPlan& p, const typename C2<R>::T* A, const typename C2<R>::T* x,
                typename C2<R>::T* y, int nrhs, int64_t vstride, const typename C2<R>::T* hsub,
                cudaStream_t s);
template <typename R>
int run_gemv_pair(const GemvPlan& p, const typename C2<R>::T* A0, const typename C2<R>::T* A1,
                  const typename C2<R>::T* x, typename C2<R>::T* y0, typename C2<R>::T* y1,
                  const typename C2<R>::T* hsub, cudaStream_t s);
template <typename R>
int run_gemv_plan(const GemvPlan& p, const typename C2<R>::T* A, const typename C2<R>::T* x,
                  typename C2<R>::T* y, int nrhs, int64_t vstride, const typename C2<R>::T* hsub,
                  cudaStream_t s);
template <typename R> int matvec(aim_ctx* c, int which, const void* x, void* y, cudaStream_t s);
// the system matvec of nrhs right-hand sides in one graph: which = kBatchOp + nrhs
constexpr int kBatchOp = 16, kMaxBatch = 4;
template <typename R> int batch_buffers(aim_ctx* c);
// matvec through a cached CUDA graph (captured on first use for these buffers)
template <typename R> int matvec_graph(aim_ctx* c, int which, const void* x, void* y,
                                       cudaStream_t s);
int init_streams(aim_ctx* c);
void release_streams(aim_ctx* c);
int fft_init_attrs();
template <typename R> int internal(aim_ctx* c, const void* h, void* e, void* heq, int nrhs,
                                   cudaStream_t s);
template <typename R> int conv(aim_ctx* c, const void* sigma, void* phi, int ncomp,
                               cudaStream_t s);
// fft (fft.cu)
template <typename R>
int fft_conv(aim_ctx* c, PrecBuf<R>& b, const typename C2<R>::T* sigma, typename C2<R>::T* phi,
             int ncomp, typename C2<R>::T* ws, cudaStream_t s);
template <typename R> int make_twiddles(aim_ctx* c, PrecBuf<R>& b);
int make_ghat(aim_ctx* c);
int rhs_plane_wave(aim_ctx* c, const double* pol, const double* kh, void* b, int prec,
                   cudaStream_t st);
// builds (or rebuilds in another precision) the block-diagonal preconditioner; prec: BEM_C32
// (FP32 blocks, each checked, FP64 where the check fails), BEM_C64, or -1: as it stands if
// built, else BEM_C32
int setup_precond(aim_ctx* c, int prec = -1);
template <typename R> inline PrecBuf<R>& buf(aim_ctx* c);
template <> inline PrecBuf<float>& buf<float>(aim_ctx* c) { return c->f32; }
template <> inline PrecBuf<double>& buf<double>(aim_ctx* c) { return c->f64; }
template <typename R>
int project_all(aim_ctx* c, const typename C2<R>::T* r, typename C2<R>::T* sigma, cudaStream_t s);
template <typename R>
int interp_all(aim_ctx* c, const typename C2<R>::T* phi, typename C2<R>::T* u, cudaStream_t s);
// learned correction (learned.cu): z = M_bd r + W net(P r) in FP32
int net_apply(aim_ctx* c, const float2* r, float2* z, cudaStream_t s);
void free_net(aim_ctx* c);
template <typename R> int precond_apply(aim_ctx* c, const void* r, void* u, cudaStream_t s);
int precond_apply_mixed(aim_ctx* c, const double2* r, float2* u32, double2* u64, cudaStream_t s);
int precond_apply_batch(aim_ctx* c, const double2* r, int nrhs, float2* u32, double2* u64,
                        cudaStream_t s);
void free_geo_store(aim_ctx* c);
double wall_ms();  // host wall clock in milliseconds
// the dense L_k and K_k + I_x/2 of one object as the set-up forms them before its LU solve
// (pass 0: k = k_i, pass 1: k = k0), row-major n_i x n_i complex doubles on the host
int export_LK(aim_ctx* c, int obj, int pass, double2* L_out, double2* K_out);
void free_far_geo(aim_ctx* c);
// sparse internal operator at high frequency (zsparse.cu)
int zsp_prepare(aim_ctx* c, const double* d_verts, const int32_t* d_tris, const double* d_cen);
int zsp_gather(aim_ctx* c, int obj, const double2* L, const double2* B);
int zsp_factor(aim_ctx* c);
int zsp_check(aim_ctx* c);
void free_zsp(aim_ctx* c);
// objects, in use, max band, FP32 bytes, check (1e-15), a product's wait timed out (1)
void zsp_stats(const aim_ctx* c, int64_t* out);
template <typename R>
int zsp_apply(aim_ctx* c, const typename C2<R>::T* h, typename C2<R>::T* e, int nrhs, int64_t hs,
              int64_t es, cudaStream_t s);
// many right-hand sides through the FP32 Z and C on the tensor cores (zgemm_tc.cu)
int internal_tc(aim_ctx* c, const float2* h, float2* e, float2* heq, int nrhs, cudaStream_t s);
void free_tc(aim_ctx* c);
// products made, a wait timed out (1) or not (0), -1 when never used
void tc_stats(const aim_ctx* c, int64_t* out);
int set_gemv_shape(aim_ctx* c, int kind, int cps, int split, int unroll);
int tune_matvec_schedule(aim_ctx* c);
double k0_of(double f);
// solver (gmres.cu)
int gmres_solve_batch(aim_ctx* c, const void* b, void* x, int nrhs, const bem_solve_opts* o,
                      bem_solve_info* infos, cudaStream_t s);
int gmres_solve(aim_ctx* c, const void* b, void* x, const bem_solve_opts* o, bem_solve_info* info,
                cudaStream_t s);
}  // namespace bem
