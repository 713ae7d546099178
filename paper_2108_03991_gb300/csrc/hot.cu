// Hot path: the system matrix-vector product of Eq. (AEFIEoutJ), applied as a sequence
// (never assembled), in complex FP32 or FP64:
//   e = Z h                     block-diagonal GEMV over objects        (Eq. MFIEinZin)
//   j = h - Y e                 block-diagonal GEMV, fused subtraction  (Eqs. EFIEeqYeq, Jdeltadis)
//   sigma = P [j; q]            27-node stencil scatter (3 RWG components + pulses)
//   phi = H sigma               zero-padded FFT convolution (fft.cu)
//   p = W_Phi phi + L^Phi_NR q  ;  y2 = F D j + j k0 q          (one warp per triangle)
//   a = W phi + L^A_NR j        ;  y1 = j k0 a + I_x e - (F D)^T p  (one warp per edge)
// Sec. III-A item 1 (Eq. AIM_L) gives L = L_NR + W H P; Sec. II-C (Eq. Cdef) gives the
// combination C = (-j k0 L^A Y + I_x/eta0) Z.
#include "common.cuh"

namespace bem {

// ---------------------------------------------------------------------------------------
// block-diagonal GEMV: one warp per row, 16-byte vector loads, x read through the L1 cache
// ---------------------------------------------------------------------------------------
// complex atomic add: one 8-byte vector atomic in FP32, two scalar atomics in FP64
__device__ __forceinline__ void catomic_add(float2* o, float2 v) { atomicAdd(o, v); }
__device__ __forceinline__ void catomic_add(double2* o, double2 v) {
  atomicAdd(&o->x, v.x);
  atomicAdd(&o->y, v.y);
}

template <typename R> struct Vec16;
template <> struct Vec16<float> { typedef float4 T; static constexpr int kCplx = 2; };
template <> struct Vec16<double> { typedef double2 T; static constexpr int kCplx = 1; };

// acc[r] += sum over the 16-byte vectors [v0, v1) of one row of A (lane-strided) times x_r.
// U vectors per lane are loaded before any is used, so each lane keeps U loads in flight.
template <typename R, int NRHS, int U>
__device__ __forceinline__ void dot_range(const typename Vec16<R>::T* __restrict__ arow,
                                          const typename C2<R>::T* __restrict__ xb, int n, int v0,
                                          int v1, int64_t vstride, int lane,
                                          typename C2<R>::T* acc) {
  typedef typename Vec16<R>::T L16;
  constexpr int CP = Vec16<R>::kCplx;
  // x_r read as one 16-byte load per vector when its slice is 16-byte aligned (col is even)
  bool x16[NRHS];
#pragma unroll
  for (int r = 0; r < NRHS; ++r)
    x16[r] = CP == 2 && ((reinterpret_cast<uintptr_t>(xb + r * vstride) & 15) == 0);
  auto use = [&](const L16& a, int col) {
    if constexpr (CP == 2) {
      const auto a0 = mk(a.x, a.y), a1 = mk(a.z, a.w);
#pragma unroll
      for (int r = 0; r < NRHS; ++r) {
        if (x16[r] && col + 1 < n) {
          const float4 q = __ldg(reinterpret_cast<const float4*>(xb + r * vstride + col));
          cfma(acc[r], a0, mk(q.x, q.y));
          cfma(acc[r], a1, mk(q.z, q.w));
        } else {
          cfma(acc[r], a0, __ldg(xb + r * vstride + col));
          if (col + 1 < n) cfma(acc[r], a1, __ldg(xb + r * vstride + col + 1));
        }
      }
    } else {
#pragma unroll
      for (int r = 0; r < NRHS; ++r) cfma(acc[r], mk(a.x, a.y), __ldg(xb + r * vstride + col));
    }
  };
  // every batch, the last one included, has its U loads issued before any is used (a plain
  // remainder loop would wait for one load at a time at the end of every row)
  for (int v = v0 + lane; v < v1; v += U * 32) {
    L16 a[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (v + 32 * u < v1) a[u] = __ldcs(arow + v + 32 * u);
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (v + 32 * u < v1) use(a[u], (v + 32 * u) * CP);
  }
}

// One row of the product, one warp: acc[r] = sum_k A[row, k] x_r[k]. Rows are streamed with
// 16-byte loads (two complex FP32 or one complex FP64 per load), evict-first so the streamed
// matrix does not displace the vectors in L2; x is read through the read-only path (L1).
template <typename R, int NRHS, int U = 4>
__device__ __forceinline__ void row_dot(const typename C2<R>::T* __restrict__ arow,
                                        const typename C2<R>::T* __restrict__ xb, int n,
                                        int64_t vstride, int lane, typename C2<R>::T* acc) {
  constexpr int CP = Vec16<R>::kCplx;
#pragma unroll
  for (int r = 0; r < NRHS; ++r) acc[r] = czero<typename C2<R>::T>();
  dot_range<R, NRHS, U>(reinterpret_cast<const typename Vec16<R>::T*>(arow), xb, n, 0,
                        (n + CP - 1) / CP, vstride, lane, acc);
#pragma unroll
  for (int r = 0; r < NRHS; ++r) acc[r] = warp_sum(acc[r]);
}

// Task-list form: one CTA per task (a run of rows of one block), NW warps taking the rows in
// turn; U = 16-byte loads in flight per lane; MINB resident CTAs per SM asked of the compiler
// (0: no request).
template <typename R, int NRHS, int U = 4, int NW = 8, int MINB = 0>
__global__ void __launch_bounds__(NW * 32, MINB) k_gemv(const GemvTask* __restrict__ tasks,
                                              const typename C2<R>::T* __restrict__ A,
                                              const typename C2<R>::T* __restrict__ x,
                                              typename C2<R>::T* __restrict__ y, int64_t vstride,
                                              const typename C2<R>::T* __restrict__ hsub) {
  typedef typename C2<R>::T V;
  const GemvTask t = tasks[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const V* xb = x + t.xoff;
  for (int rr = warp; rr < t.nrows; rr += NW) {
    const int row = t.row0 + rr;
    V acc[NRHS];
    row_dot<R, NRHS, U>(A + t.aoff + (int64_t)row * t.ld, xb, t.n, vstride, lane, acc);
#pragma unroll
    for (int r = 0; r < NRHS; ++r) {
      if (lane == 0) {
        int64_t o = r * vstride + t.xoff + row;
        y[o] = hsub ? csub(hsub[o], acc[r]) : acc[r];
      }
    }
  }
}

// Several right-hand sides at once: each warp takes RB (2 or 4) rows of its task and NR right-hand
// sides, so every 16-byte load of the matrix (two complex entries of one row) meets NR vectors
// and every load of x serves RB rows (a register tile of RB x NR accumulators). One CTA of NW
// warps per task of at most RB NW rows; y_r = A x_r, or hsub_r - A x_r. x is read as 8-byte
// complex pairs (its slices need not be 16-byte aligned); an odd row length masks the last
// pair's second entry.
template <typename R, int NR, int NW, int RB>
__global__ void __launch_bounds__(NW * 32) k_gemv_mr(const GemvTask* __restrict__ tasks,
                                                     const typename C2<R>::T* __restrict__ A,
                                                     const typename C2<R>::T* __restrict__ x,
                                                     typename C2<R>::T* __restrict__ y, int64_t vstride,
                                                     const typename C2<R>::T* __restrict__ hsub) {
  typedef typename C2<R>::T V;
  typedef typename Vec16<R>::T L16;  // 16 bytes: two complex FP32 or one complex FP64
  constexpr int CP = Vec16<R>::kCplx;
  const GemvTask t = tasks[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = t.row0 + warp * RB;
  const int nr = min(RB, t.row0 + t.nrows - r0);
  if (nr <= 0) return;
  const V* xb = x + t.xoff;
  const L16* arow[RB];
#pragma unroll
  for (int k = 0; k < RB; ++k)
    arow[k] = reinterpret_cast<const L16*>(A + t.aoff + (int64_t)(r0 + min(k, nr - 1)) * t.ld);
  V acc[RB][NR];
#pragma unroll
  for (int k = 0; k < RB; ++k)
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[k][r] = czero<V>();
  constexpr int U = 2;                 // 16-byte loads in flight per row and lane
  const int nv = (t.n + CP - 1) / CP;  // 16-byte vectors per row
  for (int v = lane; v < nv; v += 32 * U) {
    L16 a[U][RB];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int k = 0; k < RB; ++k)
        if (v + 32 * u < nv) a[u][k] = __ldcs(arow[k] + v + 32 * u);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (v + 32 * u >= nv) break;
#pragma unroll
      for (int q = 0; q < CP; ++q) {
        const int col = (v + 32 * u) * CP + q;
        if (col >= t.n) break;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          const V xv = __ldg(xb + r * vstride + col);
#pragma unroll
          for (int k = 0; k < RB; ++k) {
            V av;
            if constexpr (CP == 2) av = q == 0 ? mk(a[u][k].x, a[u][k].y) : mk(a[u][k].z, a[u][k].w);
            else av = mk(a[u][k].x, a[u][k].y);
            cfma(acc[k][r], av, xv);
          }
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < RB; ++k)
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[k][r] = warp_sum(acc[k][r]);
  if (lane < RB * NR) {
    const int k = lane / NR, r = lane % NR;
    V out = czero<V>();
#pragma unroll
    for (int kk = 0; kk < RB; ++kk)
#pragma unroll
      for (int rr = 0; rr < NR; ++rr)
        if (kk == k && rr == r) out = acc[kk][rr];
    if (k < nr) {
      const int64_t o = r * vstride + t.xoff + r0 + k;
      y[o] = hsub ? csub(hsub[o], out) : out;
    }
  }
}

template <typename R>
int run_gemv_mr(const GemvPlan& p, const typename C2<R>::T* A, const typename C2<R>::T* x,
                typename C2<R>::T* y, int nrhs, int64_t vstride, const typename C2<R>::T* hsub,
                cudaStream_t s) {
  if (p.ntasks == 0) return BEM_OK;
  for (int r0 = 0; r0 < nrhs; r0 += 4) {
    const int nr = std::min(4, nrhs - r0);
    const int64_t o = r0 * vstride;
    const typename C2<R>::T* hs = hsub ? hsub + o : nullptr;
    // RB = rows per warp = the plan's rows per task / 4 warps (its split)
#define BEM_MR(NRV, RBV) k_gemv_mr<R, NRV, 4, RBV><<<p.ntasks, 128, 0, s>>>(p.tasks, A, x + o, y + o, vstride, hs)
    if (p.split == 2) {
      switch (nr) {
        case 1: BEM_MR(1, 2); break;
        case 2: BEM_MR(2, 2); break;
        case 3: BEM_MR(3, 2); break;
        default: BEM_MR(4, 2); break;
      }
    } else {
      switch (nr) {
        case 1: BEM_MR(1, 4); break;
        case 2: BEM_MR(2, 4); break;
        case 3: BEM_MR(3, 4); break;
        default: BEM_MR(4, 4); break;
      }
    }
#undef BEM_MR
  }
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}
template int run_gemv_mr<float>(const GemvPlan&, const float2*, const float2*, float2*, int, int64_t,
                                const float2*, cudaStream_t);
template int run_gemv_mr<double>(const GemvPlan&, const double2*, const double2*, double2*, int,
                                 int64_t, const double2*, cudaStream_t);

// Paired task list: two block-diagonal matrices of the same layout applied to one x in one
// launch; a task with sel = 0 computes y0 = hsub - A0 x (or A0 x) on its rows, sel = 1
// computes y1 = A1 x. One right-hand side.
template <typename R, int U, int NW, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB) k_gemv_pair(const GemvTask* __restrict__ tasks,
                                                           const typename C2<R>::T* __restrict__ A0,
                                                           const typename C2<R>::T* __restrict__ A1,
                                                           const typename C2<R>::T* __restrict__ x,
                                                           typename C2<R>::T* __restrict__ y0,
                                                           typename C2<R>::T* __restrict__ y1,
                                                           const typename C2<R>::T* __restrict__ hsub) {
  typedef typename C2<R>::T V;
  const GemvTask t = tasks[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const V* A = t.sel ? A1 : A0;
  V* y = t.sel ? y1 : y0;
  const V* hs = t.sel ? nullptr : hsub;
  const V* xb = x + t.xoff;
  for (int rr = warp; rr < t.nrows; rr += NW) {
    const int row = t.row0 + rr;
    V acc[1];
    row_dot<R, 1, U>(A + t.aoff + (int64_t)row * t.ld, xb, t.n, 0, lane, acc);
    if (lane == 0) {
      const int64_t o = t.xoff + row;
      y[o] = hs ? csub(hs[o], acc[0]) : acc[0];
    }
  }
}

template <typename R>
int run_gemv_pair(const GemvPlan& p, const typename C2<R>::T* A0, const typename C2<R>::T* A1,
                  const typename C2<R>::T* x, typename C2<R>::T* y0, typename C2<R>::T* y1,
                  const typename C2<R>::T* hsub, cudaStream_t s) {
  if (p.ntasks == 0) return BEM_OK;
  if (p.unroll == 8) {
    k_gemv_pair<R, 8, 8, 0><<<p.ntasks, 256, 0, s>>>(p.tasks, A0, A1, x, y0, y1, hsub);
  } else if constexpr (sizeof(R) == 8) {  // FP64 needs more than 32 registers
    if (p.task_form == 2)
      k_gemv_pair<R, 4, 4, 0><<<p.ntasks, 128, 0, s>>>(p.tasks, A0, A1, x, y0, y1, hsub);
    else
      k_gemv_pair<R, 4, 8, 0><<<p.ntasks, 256, 0, s>>>(p.tasks, A0, A1, x, y0, y1, hsub);
  } else {
    if (p.task_form == 0)
      k_gemv_pair<R, 4, 8, 0><<<p.ntasks, 256, 0, s>>>(p.tasks, A0, A1, x, y0, y1, hsub);
    else if (p.task_form == 1)
      k_gemv_pair<R, 4, 8, 8><<<p.ntasks, 256, 0, s>>>(p.tasks, A0, A1, x, y0, y1, hsub);
    else
      k_gemv_pair<R, 4, 4, 16><<<p.ntasks, 128, 0, s>>>(p.tasks, A0, A1, x, y0, y1, hsub);
  }
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}
template int run_gemv_pair<float>(const GemvPlan&, const float2*, const float2*, const float2*,
                                  float2*, float2*, const float2*, cudaStream_t);
template int run_gemv_pair<double>(const GemvPlan&, const double2*, const double2*, const double2*,
                                   double2*, double2*, const double2*, cudaStream_t);

// Dynamic task list: ncta persistent CTAs take the tasks in list order from a counter (the
// largest blocks first, as in LPT), so a launch of few CTAs per SM still balances like the
// one-CTA-per-task form. The CTA that finishes last sets the counters back to zero for the
// next launch of the plan (a plan never runs concurrently with itself). Every CTA leaves the
// loop after at most ntasks + gridDim.x fetches in all; nothing waits.
template <typename R, int U>
__global__ void __launch_bounds__(256) k_gemv_dyn(const GemvTask* __restrict__ tasks, int ntasks,
                                                  int* __restrict__ ctr,
                                                  const typename C2<R>::T* __restrict__ A,
                                                  const typename C2<R>::T* __restrict__ x,
                                                  typename C2<R>::T* __restrict__ y,
                                                  const typename C2<R>::T* __restrict__ hsub) {
  typedef typename C2<R>::T V;
  __shared__ int s_task;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (;;) {
    if (threadIdx.x == 0) s_task = atomicAdd(&ctr[0], 1);
    __syncthreads();
    const int ti = s_task;
    __syncthreads();  // all have read s_task before the next fetch overwrites it
    if (ti >= ntasks) break;
    const GemvTask t = tasks[ti];
    const V* xb = x + t.xoff;
    for (int rr = warp; rr < t.nrows; rr += 8) {
      const int row = t.row0 + rr;
      V acc[1];
      row_dot<R, 1, U>(A + t.aoff + (int64_t)row * t.ld, xb, t.n, 0, lane, acc);
      if (lane == 0) {
        const int64_t o = t.xoff + row;
        y[o] = hsub ? csub(hsub[o], acc[0]) : acc[0];
      }
    }
  }
  if (threadIdx.x == 0 && atomicAdd(&ctr[1], 1) == (int)gridDim.x - 1) {
    atomicExch(&ctr[0], 0);
    atomicExch(&ctr[1], 0);
  }
}

// Persistent form: CTA p streams the rows of its byte-balanced range (GemvPlan). Each row is
// cut into S equal column parts; the S * rows work items of a chunk are dealt to the 8 warps
// in turn (one warp reduction per part), partial sums meet in shared memory and the CTA adds
// the S parts of each row at the end of the chunk. S = 1 is one warp per row; S = 2 or 4
// evens out the work of the warps when a CTA holds only a few rows per warp. U = loads in
// flight per lane (U = 8 needs more registers: 4 CTAs per SM instead of 6).
constexpr int kGemvChunk = 64;

template <typename R, int NRHS, int S, int U>
__global__ void __launch_bounds__(kGemvThreads, U >= 8 ? 4 : kGemvCtasPerSm)
    k_gemv_plan(const RowInfo* __restrict__ rows, const int2* __restrict__ segs,
                const int32_t* __restrict__ cta_seg, const typename C2<R>::T* __restrict__ A,
                const typename C2<R>::T* __restrict__ x, typename C2<R>::T* __restrict__ y,
                int64_t vstride, const typename C2<R>::T* __restrict__ hsub) {
  typedef typename C2<R>::T V;
  typedef typename Vec16<R>::T L16;
  constexpr int CP = Vec16<R>::kCplx;
  constexpr int nw = kGemvThreads / 32;
  __shared__ V part[kGemvChunk][S][NRHS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s1 = cta_seg[blockIdx.x + 1];
  for (int s = cta_seg[blockIdx.x]; s < s1; ++s) {
    const int2 sg = segs[s];
    for (int c0 = sg.x; c0 < sg.y; c0 += kGemvChunk) {
      const int c1 = min(sg.y, c0 + kGemvChunk);
      for (int it = warp; it < (c1 - c0) * S; it += nw) {
        const int rl = it / S, pp = it - rl * S;
        const RowInfo ri = rows[c0 + rl];
        const int nvec = (ri.n + CP - 1) / CP;
        const int per = (nvec + S - 1) / S;
        const int v0 = pp * per, v1 = min(nvec, v0 + per);
        V acc[NRHS];
#pragma unroll
        for (int r = 0; r < NRHS; ++r) acc[r] = czero<V>();
        dot_range<R, NRHS, U>(reinterpret_cast<const L16*>(A + ri.aoff), x + ri.xoff, ri.n, v0, v1,
                              vstride, lane, acc);
#pragma unroll
        for (int r = 0; r < NRHS; ++r) {
          const V t = warp_sum(acc[r]);
          if (lane == 0) part[rl][pp][r] = t;
        }
      }
      __syncthreads();
      for (int i = threadIdx.x; i < (c1 - c0) * NRHS; i += blockDim.x) {
        const int rr = i / NRHS, r = i - rr * NRHS;
        V t = part[rr][0][r];
#pragma unroll
        for (int q = 1; q < S; ++q) t = cadd(t, part[rr][q][r]);
        const int64_t o = r * vstride + c0 + rr;
        y[o] = hsub ? csub(hsub[o], t) : t;
      }
      __syncthreads();
    }
  }
}

template <typename R, int S, int U>
static void launch_gemv_plan(const GemvPlan& p, const typename C2<R>::T* A,
                             const typename C2<R>::T* x, typename C2<R>::T* y, int nr,
                             int64_t vstride, const typename C2<R>::T* hs, cudaStream_t s) {
  switch (nr) {
    case 1: k_gemv_plan<R, 1, S, U><<<p.ncta, kGemvThreads, 0, s>>>(p.rows, p.segs, p.cta_seg, A, x, y, vstride, hs); break;
    case 2: k_gemv_plan<R, 2, S, U><<<p.ncta, kGemvThreads, 0, s>>>(p.rows, p.segs, p.cta_seg, A, x, y, vstride, hs); break;
    case 3: k_gemv_plan<R, 3, S, U><<<p.ncta, kGemvThreads, 0, s>>>(p.rows, p.segs, p.cta_seg, A, x, y, vstride, hs); break;
    default: k_gemv_plan<R, 4, S, U><<<p.ncta, kGemvThreads, 0, s>>>(p.rows, p.segs, p.cta_seg, A, x, y, vstride, hs); break;
  }
}

template <typename R, int U>
static void launch_gemv_plan_u(const GemvPlan& p, const typename C2<R>::T* A,
                               const typename C2<R>::T* x, typename C2<R>::T* y, int nr,
                               int64_t vstride, const typename C2<R>::T* hs, cudaStream_t s) {
  switch (p.split) {
    case 1: launch_gemv_plan<R, 1, U>(p, A, x, y, nr, vstride, hs, s); break;
    case 4: launch_gemv_plan<R, 4, U>(p, A, x, y, nr, vstride, hs, s); break;
    default: launch_gemv_plan<R, 2, U>(p, A, x, y, nr, vstride, hs, s); break;
  }
}

// Flat form: a CTA's rows are adjacent in memory, so its range is one contiguous run of matrix
// bytes. It is taken in chunks of at most kTmaMaxRows whole rows (the row tables of the staged
// form); the 8 warps split a chunk's 16-byte vectors evenly whatever the row lengths, walk the
// rows their share touches (lanes strided within a row, U loads in flight per lane) and add each
// row's warp sum into a per-row partial in shared memory. No warp waits on another's rows, and
// every warp of every CTA streams the same number of bytes (to one vector).
template <typename R, int NRHS, int U>
__global__ void __launch_bounds__(kGemvThreads, U >= 8 ? 4 : kGemvCtasPerSm)
    k_gemv_flat(const TmaStage* __restrict__ chunks, const TmaDesc* __restrict__ descs,
                const int32_t* __restrict__ cta_chunk, const typename C2<R>::T* __restrict__ A,
                const typename C2<R>::T* __restrict__ x, typename C2<R>::T* __restrict__ y,
                int64_t vstride, const typename C2<R>::T* __restrict__ hsub) {
  typedef typename C2<R>::T V;
  typedef typename Vec16<R>::T L16;
  constexpr int CP = Vec16<R>::kCplx;
  constexpr int nw = kGemvThreads / 32;
  __shared__ __align__(16) TmaDesc d;
  __shared__ V part[kTmaMaxRows * NRHS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ch1 = cta_chunk[blockIdx.x + 1];
  for (int ch = cta_chunk[blockIdx.x]; ch < ch1; ++ch) {
    {
      const int4* src = reinterpret_cast<const int4*>(descs + ch);
      int4* dst = reinterpret_cast<int4*>(&d);
      for (int i = threadIdx.x; i < (int)(sizeof(TmaDesc) / 16); i += blockDim.x) dst[i] = src[i];
      for (int i = threadIdx.x; i < kTmaMaxRows * NRHS; i += blockDim.x) part[i] = czero<V>();
    }
    const L16* a16 = reinterpret_cast<const L16*>(A + chunks[ch].e0);
    __syncthreads();
    const int nr = d.nr;
    const int nvec = d.nel / CP;
    const int per = (nvec + nw - 1) / nw;
    const int v0 = min(nvec, warp * per), v1 = min(nvec, v0 + per);
    int k = 0;
    while (k + 1 < nr && d.soff[k + 1] <= v0 * CP) ++k;
    for (int vs = v0; vs < v1; ++k) {
      const int ve = min(v1, d.soff[k + 1] / CP);
      const int c0 = d.soff[k];
      V acc[NRHS];
#pragma unroll
      for (int r = 0; r < NRHS; ++r) acc[r] = czero<V>();
      // element e of the chunk is column e - c0 of row k: shift the row's x slice by c0 and
      // let dot_range count columns from the chunk start (its bound n becomes c0 + n)
      dot_range<R, NRHS, U>(a16, x + d.xoff[k] - c0, c0 + d.n[k], vs, ve, vstride, lane, acc);
#pragma unroll
      for (int r = 0; r < NRHS; ++r) {
        const V t = warp_sum(acc[r]);
        if (lane == 0) {
          atomicAdd(&part[k * NRHS + r].x, t.x);
          atomicAdd(&part[k * NRHS + r].y, t.y);
        }
      }
      vs = ve;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nr * NRHS; t += blockDim.x) {
      const int rr = t / NRHS, r = t - rr * NRHS;
      const int64_t o = r * vstride + d.r0 + rr;
      y[o] = hsub ? csub(hsub[o], part[t]) : part[t];
    }
    __syncthreads();
  }
}

template <typename R, int U>
static void launch_gemv_flat(const GemvPlan& p, const typename C2<R>::T* A,
                             const typename C2<R>::T* x, typename C2<R>::T* y, int nr,
                             int64_t vstride, const typename C2<R>::T* hs, cudaStream_t s) {
  switch (nr) {
    case 1: k_gemv_flat<R, 1, U><<<p.ncta, kGemvThreads, 0, s>>>(p.stages, p.descs, p.cta_stage, A, x, y, vstride, hs); break;
    case 2: k_gemv_flat<R, 2, U><<<p.ncta, kGemvThreads, 0, s>>>(p.stages, p.descs, p.cta_stage, A, x, y, vstride, hs); break;
    case 3: k_gemv_flat<R, 3, U><<<p.ncta, kGemvThreads, 0, s>>>(p.stages, p.descs, p.cta_stage, A, x, y, vstride, hs); break;
    default: k_gemv_flat<R, 4, U><<<p.ncta, kGemvThreads, 0, s>>>(p.stages, p.descs, p.cta_stage, A, x, y, vstride, hs); break;
  }
}

// Stream form: the blocks' storage (rows back to back, no gaps) is one run of 16-byte vectors,
// cut into equal shares, one per warp of the grid (to 32 bytes), so every warp streams the
// same bytes and starts at once. A warp walks the rows its share touches (the next row's
// descriptor is fetched while the current row streams) and adds each row's warp sum atomically
// into y, which k_gemv_init first set to 0, or to hsub with the sums subtracted.
template <typename R, int NRHS, int U>
__global__ void __launch_bounds__(kGemvThreads, U >= 8 ? 4 : kGemvCtasPerSm)
    k_gemv_stream(const int32_t* __restrict__ wrow, const RowInfo* __restrict__ rows,
                  int64_t nquad, const typename C2<R>::T* __restrict__ A,
                  const typename C2<R>::T* __restrict__ x, typename C2<R>::T* __restrict__ y,
                  int64_t vstride, R sign) {
  typedef typename C2<R>::T V;
  typedef typename Vec16<R>::T L16;
  constexpr int CP = Vec16<R>::kCplx;
  constexpr int nw = kGemvThreads / 32;
  const int lane = threadIdx.x & 31;
  const int64_t W = (int64_t)gridDim.x * nw;
  const int64_t w = (int64_t)blockIdx.x * nw + (threadIdx.x >> 5);
  // shares in units of 4 complex elements (one row of ld is a whole number of them), so the
  // per-warp first rows are the same for FP32 and FP64
  const int64_t v0 = 4 * (nquad * w / W) / CP;
  const int len = (int)(4 * (nquad * (w + 1) / W) / CP - v0);
  if (len <= 0) return;
  const L16* a16 = reinterpret_cast<const L16*>(A) + v0;  // the warp's share
  int k = wrow[w];
  RowInfo ri = rows[k];
  for (int pos = 0; pos < len; ++k) {
    const int rs = (int)(ri.aoff / CP - v0);  // row start relative to the share (may be < 0)
    const int ve = min(len, rs + ((ri.n + 3) & ~3) / CP);
    RowInfo nxt = ri;
    if (ve < len) nxt = rows[k + 1];
    V acc[NRHS];
#pragma unroll
    for (int r = 0; r < NRHS; ++r) acc[r] = czero<V>();
    dot_range<R, NRHS, U>(a16 + rs, x + ri.xoff, ri.n, pos - rs, ve - rs, vstride, lane, acc);
#pragma unroll
    for (int r = 0; r < NRHS; ++r) {
      const V t = warp_sum(acc[r]);
      if (lane == 0) catomic_add(y + r * vstride + k, mk(sign * t.x, sign * t.y));
    }
    ri = nxt;
    pos = ve;
  }
}

// y_r = 0, or y_r = hsub_r, for the rows [0, nrows) of nrhs vectors
template <typename V>
__global__ void k_gemv_init(V* __restrict__ y, const V* __restrict__ hsub, int64_t nrows, int nrhs,
                            int64_t vstride) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nrows * nrhs) return;
  const int64_t r = i / nrows, m = i - r * nrows;
  y[r * vstride + m] = hsub ? hsub[r * vstride + m] : czero<V>();
}

template <typename R, int U>
static void launch_gemv_stream(const GemvPlan& p, const typename C2<R>::T* A,
                               const typename C2<R>::T* x, typename C2<R>::T* y, int nr,
                               int64_t vstride, R sign, cudaStream_t s) {
  switch (nr) {
    case 1: k_gemv_stream<R, 1, U><<<p.ncta, kGemvThreads, 0, s>>>(p.wrow, p.rows, p.nquad, A, x, y, vstride, sign); break;
    case 2: k_gemv_stream<R, 2, U><<<p.ncta, kGemvThreads, 0, s>>>(p.wrow, p.rows, p.nquad, A, x, y, vstride, sign); break;
    case 3: k_gemv_stream<R, 3, U><<<p.ncta, kGemvThreads, 0, s>>>(p.wrow, p.rows, p.nquad, A, x, y, vstride, sign); break;
    default: k_gemv_stream<R, 4, U><<<p.ncta, kGemvThreads, 0, s>>>(p.wrow, p.rows, p.nquad, A, x, y, vstride, sign); break;
  }
}

template <typename R>
int run_gemv_plan(const GemvPlan& p, const typename C2<R>::T* A, const typename C2<R>::T* x,
                  typename C2<R>::T* y, int nrhs, int64_t vstride, const typename C2<R>::T* hsub,
                  cudaStream_t s) {
  if (p.ncta == 0 || p.nrows == 0) return BEM_OK;
  if (p.tma) return run_gemv_tma<R>(p, A, x, y, nrhs, vstride, hsub, s);
  if (p.ntasks > 0) {
    if (p.ctr && nrhs == 1) {
      if (p.unroll >= 8)
        k_gemv_dyn<R, 8><<<p.ncta, 256, 0, s>>>(p.tasks, p.ntasks, p.ctr, A, x, y, hsub);
      else
        k_gemv_dyn<R, 4><<<p.ncta, 256, 0, s>>>(p.tasks, p.ntasks, p.ctr, A, x, y, hsub);
      BEM_CUDA(cudaGetLastError());
      return BEM_OK;
    }
    if (nrhs == 1 && (p.unroll == 8 || p.task_form != 0)) {
      if (p.unroll == 8)
        k_gemv<R, 1, 8><<<p.ntasks, 256, 0, s>>>(p.tasks, A, x, y, vstride, hsub);
      else if constexpr (sizeof(R) == 8)  // FP64 needs more than 32 registers: no occupancy request
        if (p.task_form == 1)
          k_gemv<R, 1, 4, 8, 0><<<p.ntasks, 256, 0, s>>>(p.tasks, A, x, y, vstride, hsub);
        else
          k_gemv<R, 1, 4, 4, 0><<<p.ntasks, 128, 0, s>>>(p.tasks, A, x, y, vstride, hsub);
      else if (p.task_form == 1)
        k_gemv<R, 1, 4, 8, 8><<<p.ntasks, 256, 0, s>>>(p.tasks, A, x, y, vstride, hsub);
      else
        k_gemv<R, 1, 4, 4, 16><<<p.ntasks, 128, 0, s>>>(p.tasks, A, x, y, vstride, hsub);
      BEM_CUDA(cudaGetLastError());
      return BEM_OK;
    }
    return run_gemv<R>(p.tasks, p.ntasks, A, x, y, nrhs, vstride, hsub, s);
  }
  if (p.stream) {
    k_gemv_init<<<(unsigned)((p.nrows * (int64_t)nrhs + 255) / 256), 256, 0, s>>>(y, hsub, (int64_t)p.nrows,
                                                                               nrhs, vstride);
    const R sign = hsub ? R(-1) : R(1);
    for (int r0 = 0; r0 < nrhs; r0 += 4) {
      const int nr = std::min(4, nrhs - r0);
      const int64_t o = r0 * vstride;
      if (p.unroll >= 8) launch_gemv_stream<R, 8>(p, A, x + o, y + o, nr, vstride, sign, s);
      else launch_gemv_stream<R, 4>(p, A, x + o, y + o, nr, vstride, sign, s);
    }
    BEM_CUDA(cudaGetLastError());
    return BEM_OK;
  }
  for (int r0 = 0; r0 < nrhs; r0 += 4) {
    const int nr = std::min(4, nrhs - r0);
    const int64_t o = r0 * vstride;
    const typename C2<R>::T* hs = hsub ? hsub + o : nullptr;
    if (p.flat) {
      if (p.unroll >= 8) launch_gemv_flat<R, 8>(p, A, x + o, y + o, nr, vstride, hs, s);
      else launch_gemv_flat<R, 4>(p, A, x + o, y + o, nr, vstride, hs, s);
    } else if (p.unroll >= 8) {
      launch_gemv_plan_u<R, 8>(p, A, x + o, y + o, nr, vstride, hs, s);
    } else {
      launch_gemv_plan_u<R, 4>(p, A, x + o, y + o, nr, vstride, hs, s);
    }
  }
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}
template int run_gemv_plan<float>(const GemvPlan&, const float2*, const float2*, float2*, int,
                                  int64_t, const float2*, cudaStream_t);
template int run_gemv_plan<double>(const GemvPlan&, const double2*, const double2*, double2*, int,
                                   int64_t, const double2*, cudaStream_t);

template <typename R>
int run_gemv(const GemvTask* d_tasks, int ntasks, const typename C2<R>::T* A,
             const typename C2<R>::T* x, typename C2<R>::T* y, int nrhs, int64_t vstride,
             const typename C2<R>::T* hsub, cudaStream_t s) {
  if (ntasks == 0) return BEM_OK;
  for (int r0 = 0; r0 < nrhs; r0 += 4) {
    const int nr = std::min(4, nrhs - r0);
    const int64_t o = r0 * vstride;
    const typename C2<R>::T* hs = hsub ? hsub + o : nullptr;
    switch (nr) {
      case 1: k_gemv<R, 1><<<ntasks, 256, 0, s>>>(d_tasks, A, x + o, y + o, vstride, hs); break;
      case 2: k_gemv<R, 2><<<ntasks, 256, 0, s>>>(d_tasks, A, x + o, y + o, vstride, hs); break;
      case 3: k_gemv<R, 3><<<ntasks, 256, 0, s>>>(d_tasks, A, x + o, y + o, vstride, hs); break;
      default: k_gemv<R, 4><<<ntasks, 256, 0, s>>>(d_tasks, A, x + o, y + o, vstride, hs); break;
    }
  }
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}
template int run_gemv<float>(const GemvTask*, int, const float2*, const float2*, float2*, int,
                             int64_t, const float2*, cudaStream_t);
template int run_gemv<double>(const GemvTask*, int, const double2*, const double2*, double2*, int,
                              int64_t, const double2*, cudaStream_t);

// ---------------------------------------------------------------------------------------
// projection P (Sec. III-A item 1): gather form, no atomics, deterministic
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int node_offset(int k, int nx, int ny) {
  return ((k / 9 - 1) * ny + ((k / 3) % 3 - 1)) * nx + (k % 3 - 1);
}

// sigma_c(node) = sum over the CSR entries e of the node of WT[e][c] * src[col[e]], for the NC
// components of one source kind. A group of G lanes shares one node of the work list (the nodes
// some stencil touches): the lanes take every G-th entry, so a node's entries are fetched in
// parallel, and meet in a shuffle reduction. Blocks past nb_work write the zeros of the nodes
// no stencil touches (the rest of the work list), so every node is written each time.
constexpr int kProjG = 8;

template <typename R, int NC>
__global__ void __launch_bounds__(256) k_project(const int32_t* __restrict__ work, int nwork,
                                                 int64_t ng, int nb_work,
                                                 const int32_t* __restrict__ prow,
                                                 const int32_t* __restrict__ pcol,
                                                 const R* __restrict__ WT,
                                                 const typename C2<R>::T* __restrict__ src,
                                                 typename C2<R>::T* __restrict__ sigma,
                                                 int64_t src_rs, int64_t sig_rs) {
  typedef typename C2<R>::T V;
  src += blockIdx.y * src_rs;  // right-hand side blockIdx.y of a batch
  sigma += blockIdx.y * sig_rs;
  if ((int)blockIdx.x >= nb_work) {
    const int64_t i = nwork + (int64_t)(blockIdx.x - nb_work) * blockDim.x + threadIdx.x;
    if (i < ng) {
      const int nd = work[i];
#pragma unroll
      for (int c = 0; c < NC; ++c) sigma[c * ng + nd] = czero<V>();
    }
    return;
  }
  const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kProjG;
  const int l = threadIdx.x & (kProjG - 1);
  V acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = czero<V>();
  int nd = 0;
  if (g < nwork) {
    nd = work[g];
    const int e1 = prow[nd + 1];
#pragma unroll 4
    for (int e = prow[nd] + l; e < e1; e += kProjG) {
      const V v = src[pcol[e]];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const R w = WT[(int64_t)NC * e + c];
        acc[c].x += w * v.x;
        acc[c].y += w * v.y;
      }
    }
  }
#pragma unroll
  for (int o = kProjG / 2; o > 0; o >>= 1)
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      acc[c].x += __shfl_xor_sync(0xffffffffu, acc[c].x, o);
      acc[c].y += __shfl_xor_sync(0xffffffffu, acc[c].y, o);
    }
  if (l == 0 && g < nwork) {
#pragma unroll
    for (int c = 0; c < NC; ++c) sigma[c * ng + nd] = acc[c];
  }
}

static inline unsigned nb(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// sigma_{x,y,z} = P_c j (RWG sources, 3 components)
template <typename R>
static void project_e(const aim_ctx* c, const R* WT, const typename C2<R>::T* j,
                      typename C2<R>::T* sigma, cudaStream_t s, int nrhs = 1, int64_t j_rs = 0) {
  const int nbw = (int)nb((int64_t)c->nwE * kProjG, 256);
  const int nbz = (int)nb(c->ng - c->nwE, 256);
  k_project<R, 3><<<dim3(nbw + nbz, nrhs), 256, 0, s>>>(c->d_pnodeE, c->nwE, c->ng, nbw, c->d_prowE,
                                                        c->d_pcolE, WT, j, sigma, j_rs, 3 * c->ng);
}
// sigma_q = P_Phi q (pulse sources, 1 component)
template <typename R>
static void project_t(const aim_ctx* c, const R* WT, const typename C2<R>::T* q,
                      typename C2<R>::T* sigma, cudaStream_t s, int nrhs = 1, int64_t q_rs = 0) {
  const int nbw = (int)nb((int64_t)c->nwT * kProjG, 256);
  const int nbz = (int)nb(c->ng - c->nwT, 256);
  k_project<R, 1><<<dim3(nbw + nbz, nrhs), 256, 0, s>>>(c->d_pnodeT, c->nwT, c->ng, nbw, c->d_prowT,
                                                        c->d_pcolT, WT, q, sigma, q_rs, c->ng);
}

// ---------------------------------------------------------------------------------------
// interpolation W + near region + combination, one warp per output row
// ---------------------------------------------------------------------------------------
template <typename V, typename R>
__device__ __forceinline__ V jk0(V a, R k0) { return mk(-k0 * a.y, k0 * a.x); }

// acc += sum over the CSR row [i0, i1) of val[i] * x[col[i]], one warp (the callers pass the
// row's values and its anchor node's column list, shared by every row anchored there); four
// independent entries per lane are in flight at a time (the column load and the gather it feeds
// are a dependent pair, so a plain loop would wait on both for every entry). Eight per lane,
// predicated, so that a whole row of up to 256 entries is one round, ran 30% slower (more
// registers, fewer resident warps).
template <typename V>
__device__ __forceinline__ void near_row(const V* __restrict__ val, const int32_t* __restrict__ col,
                                         const V* __restrict__ x, int64_t i0, int64_t i1, int lane,
                                         V& acc) {
  int64_t i = i0 + lane;
  for (; i + 96 < i1; i += 128) {
    const int c0 = col[i], c1 = col[i + 32], c2 = col[i + 64], c3 = col[i + 96];
    const V a0 = val[i], a1 = val[i + 32], a2 = val[i + 64], a3 = val[i + 96];
    const V x0 = x[c0], x1 = x[c1], x2 = x[c2], x3 = x[c3];
    cfma(acc, a0, x0);
    cfma(acc, a1, x1);
    cfma(acc, a2, x2);
    cfma(acc, a3, x3);
  }
  for (; i < i1; i += 32) cfma(acc, val[i], x[col[i]]);
}

// The same sum with the lane's last group predicated instead of taken one entry at a time: a lane
// with 1-3 entries left issues their loads together (a missing entry repeats the group's first
// column, with value 0), so every lane's share of a row of up to 256 entries takes at most two
// rounds of dependent loads. The entries, their lanes and each lane's order of accumulation are
// those of near_row, and the missing entries add exact zeros: the sums are the same bits.
template <typename V>
__device__ __forceinline__ void near_row_p(const V* __restrict__ val, const int32_t* __restrict__ col,
                                           const V* __restrict__ x, int64_t i0, int64_t i1, int lane,
                                           V& acc) {
  for (int64_t i = i0 + lane; i < i1; i += 128) {
    const bool p1 = i + 32 < i1, p2 = i + 64 < i1, p3 = i + 96 < i1;
    const int c0 = col[i];
    const int c1 = p1 ? col[i + 32] : c0, c2 = p2 ? col[i + 64] : c0, c3 = p3 ? col[i + 96] : c0;
    const V a0 = val[i];
    const V a1 = p1 ? val[i + 32] : czero<V>(), a2 = p2 ? val[i + 64] : czero<V>();
    const V a3 = p3 ? val[i + 96] : czero<V>();
    const V x0 = x[c0], x1 = x[c1], x2 = x[c2], x3 = x[c3];
    cfma(acc, a0, x0);
    cfma(acc, a1, x1);
    cfma(acc, a2, x2);
    cfma(acc, a3, x3);
  }
}
template <int PV, typename V>
__device__ __forceinline__ void near_row_v(const V* __restrict__ val, const int32_t* __restrict__ col,
                                           const V* __restrict__ x, int64_t i0, int64_t i1, int lane,
                                           V& acc) {
  if constexpr (PV == 1) near_row_p(val, col, x, i0, i1, lane, acc);
  else near_row(val, col, x, i0, i1, lane, acc);
}

// p_t = (W_Phi phi)_t + (L^Phi_NR q)_t, written to out[t] (y for L^Phi alone, p in the system);
// PV selects the near-row form (0: near_row, 1: near_row_p)
template <typename R, int PV = 0>
__global__ void __launch_bounds__(256) k_rows_t(
    const R* __restrict__ WP, const int32_t* __restrict__ node,
    const typename C2<R>::T* __restrict__ phi, const int64_t* __restrict__ rowP,
    const int64_t* __restrict__ lstP, const int32_t* __restrict__ colP,
    const typename C2<R>::T* __restrict__ LP,
    const typename C2<R>::T* __restrict__ q, int nt, int nx, int ny,
    typename C2<R>::T* __restrict__ out, int64_t phi_rs = 0, int64_t q_rs = 0, int64_t out_rs = 0) {
  typedef typename C2<R>::T V;
  phi += blockIdx.y * phi_rs;  // right-hand side blockIdx.y of a batch
  q += blockIdx.y * q_rs;
  out += blockIdx.y * out_rs;
  const int t = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (t >= nt) return;
  V acc = czero<V>();
  if (lane < 27) {
    const R w = WP[(int64_t)t * 27 + lane];
    const V f = phi[node[t] + node_offset(lane, nx, ny)];
    acc = mk(w * f.x, w * f.y);
  }
  near_row_v<PV>(LP + rowP[t], colP + lstP[t], q, 0, rowP[t + 1] - rowP[t], lane, acc);
  acc = warp_sum(acc);
  if (lane == 0) out[t] = acc;
}

// offsets of right-hand side blockIdx.y in a batch (0: one right-hand side)
struct RowsStride {
  int64_t phi = 0, j = 0, e = 0, p = 0, q = 0, an = 0, y = 0;
};

// mode 0: y[m] = a_m (L^A alone).
// mode 1 (system), rows m < ne:  y1_m = j k0 a_m + (I_x e)_m - ((F D)^T p)_m
//                  rows ne + t:  y2_t = (F D j)_t + j k0 q_t
template <typename R>
__global__ void __launch_bounds__(256) k_rows_e(
    const R* __restrict__ WA, const int32_t* __restrict__ node,
    const typename C2<R>::T* __restrict__ phi, int64_t ng, const int64_t* __restrict__ rowA,
    const int64_t* __restrict__ lstA, const int32_t* __restrict__ colA,
    const typename C2<R>::T* __restrict__ LA,
    const typename C2<R>::T* __restrict__ j, const R* __restrict__ ix,
    const int32_t* __restrict__ ixcol, const typename C2<R>::T* __restrict__ e,
    const R* __restrict__ fdE, const int32_t* __restrict__ et,
    const typename C2<R>::T* __restrict__ p, int ne, int nx, int ny, R k0, int mode,
    typename C2<R>::T* __restrict__ y, int nt, const R* __restrict__ fdT,
    const int32_t* __restrict__ tedge, const typename C2<R>::T* __restrict__ q,
    const typename C2<R>::T* __restrict__ anear, RowsStride rs = RowsStride()) {
  typedef typename C2<R>::T V;
  {
    const int64_t r = blockIdx.y;
    phi += r * rs.phi;
    j += r * rs.j;
    if (e) e += r * rs.e;
    if (p) p += r * rs.p;
    if (q) q += r * rs.q;
    if (anear) anear += r * rs.an;
    y += r * rs.y;
  }
  const int nbE = (ne + 7) >> 3;  // blocks of the RWG rows (one warp per row); then the pulse
  if ((int)blockIdx.x >= nbE) {   // rows of mode 1, one thread per row
    const int t = (blockIdx.x - nbE) * blockDim.x + threadIdx.x;
    if (mode == 1 && t < nt) {
      V s = jk0(q[t], k0);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const V jj = j[tedge[3 * t + i]];
        const R c = fdT[3 * t + i];
        s.x += c * jj.x;
        s.y += c * jj.y;
      }
      y[ne + t] = s;
    }
    return;
  }
  const int m = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (m >= ne) return;
  // mode 1: the lanes the stencil leaves free take the sparse terms of row 1, each its own
  // dependent pair of loads, at the same time as the stencil's (lanes 27-30: (I_x e)_m, lane 31:
  // -((F D)^T p)_m); the row's sum is then one reduction of j k0 (a part) + (these terms)
  V b = czero<V>();
  if (mode == 1 && lane >= 27) {
    if (lane < 31) {
      const int i = lane - 27;
      const V ev = e[ixcol[4 * m + i]];
      const R c = ix[4 * m + i];
      b.x = c * ev.x;
      b.y = c * ev.y;
    } else {
      const V pp = p[et[2 * m]], pm = p[et[2 * m + 1]];
      const R cp = fdE[2 * m], cm = fdE[2 * m + 1];
      b.x = -cp * pp.x + cm * pm.x;
      b.y = -cp * pp.y + cm * pm.y;
    }
  }
  V acc = czero<V>();
  if (lane < 27) {
    const int64_t nd = node[m] + node_offset(lane, nx, ny);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const R w = WA[(int64_t)m * 81 + c * 27 + lane];
      const V f = phi[c * ng + nd];
      acc.x += w * f.x;
      acc.y += w * f.y;
    }
  }
  if (!anear) near_row(LA + rowA[m], colA + lstA[m], j, 0, rowA[m + 1] - rowA[m], lane, acc);
  if (anear && lane == 0) {
    const V an = anear[m];
    acc.x += an.x;
    acc.y += an.y;
  }
  if (mode == 0) {
    acc = warp_sum(acc);
    if (lane == 0) y[m] = acc;
  } else {
    V t = jk0(acc, k0);
    t.x += b.x;
    t.y += b.y;
    t = warp_sum(t);
    if (lane == 0) y[m] = t;
  }
}

// The same rows, two per warp: each lane issues the loads of both rows' stencil node (and its
// near-region entries, predicated) before it sums either, so twice the loads are in flight per
// warp. Every row's terms, their lanes and their order are those of k_rows_e (near_row_p's sums
// are near_row's bits), so the outputs are the same bits. 16 rows per block of 8 warps; the
// pulse rows of mode 1 follow as in k_rows_e.
template <typename R>
__global__ void __launch_bounds__(256) k_rows_e2(
    const R* __restrict__ WA, const int32_t* __restrict__ node,
    const typename C2<R>::T* __restrict__ phi, int64_t ng, const int64_t* __restrict__ rowA,
    const int64_t* __restrict__ lstA, const int32_t* __restrict__ colA,
    const typename C2<R>::T* __restrict__ LA,
    const typename C2<R>::T* __restrict__ j, const R* __restrict__ ix,
    const int32_t* __restrict__ ixcol, const typename C2<R>::T* __restrict__ e,
    const R* __restrict__ fdE, const int32_t* __restrict__ et,
    const typename C2<R>::T* __restrict__ p, int ne, int nx, int ny, R k0, int mode,
    typename C2<R>::T* __restrict__ y, int nt, const R* __restrict__ fdT,
    const int32_t* __restrict__ tedge, const typename C2<R>::T* __restrict__ q,
    const typename C2<R>::T* __restrict__ anear, RowsStride rs = RowsStride()) {
  typedef typename C2<R>::T V;
  {
    const int64_t r = blockIdx.y;
    phi += r * rs.phi;
    j += r * rs.j;
    if (e) e += r * rs.e;
    if (p) p += r * rs.p;
    if (q) q += r * rs.q;
    if (anear) anear += r * rs.an;
    y += r * rs.y;
  }
  const int nbE = (ne + 15) >> 4;  // blocks of the RWG rows (two per warp); then the pulse rows
  if ((int)blockIdx.x >= nbE) {
    const int t = (blockIdx.x - nbE) * blockDim.x + threadIdx.x;
    if (mode == 1 && t < nt) {
      V s = jk0(q[t], k0);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const V jj = j[tedge[3 * t + i]];
        const R c = fdT[3 * t + i];
        s.x += c * jj.x;
        s.y += c * jj.y;
      }
      y[ne + t] = s;
    }
    return;
  }
  const int lane = threadIdx.x & 31;
  const int m0 = (blockIdx.x * 8 + (threadIdx.x >> 5)) * 2;
  if (m0 >= ne) return;
  const bool two = m0 + 1 < ne;
  const int m1 = two ? m0 + 1 : m0;
  // mode 1: lanes 27-31 take the sparse terms of row 1 for both rows
  V b0 = czero<V>(), b1 = czero<V>();
  if (mode == 1 && lane >= 27) {
    if (lane < 31) {
      const int i = lane - 27;
      const V e0 = e[ixcol[4 * m0 + i]], e1 = e[ixcol[4 * m1 + i]];
      const R c0 = ix[4 * m0 + i], c1 = ix[4 * m1 + i];
      b0.x = c0 * e0.x;
      b0.y = c0 * e0.y;
      b1.x = c1 * e1.x;
      b1.y = c1 * e1.y;
    } else {
      const V pp0 = p[et[2 * m0]], pm0 = p[et[2 * m0 + 1]];
      const V pp1 = p[et[2 * m1]], pm1 = p[et[2 * m1 + 1]];
      const R cp0 = fdE[2 * m0], cm0 = fdE[2 * m0 + 1], cp1 = fdE[2 * m1], cm1 = fdE[2 * m1 + 1];
      b0.x = -cp0 * pp0.x + cm0 * pm0.x;
      b0.y = -cp0 * pp0.y + cm0 * pm0.y;
      b1.x = -cp1 * pp1.x + cm1 * pm1.x;
      b1.y = -cp1 * pp1.y + cm1 * pm1.y;
    }
  }
  V acc0 = czero<V>(), acc1 = czero<V>();
  if (lane < 27) {
    const int64_t off = node_offset(lane, nx, ny);
    const int64_t nd0 = node[m0] + off, nd1 = node[m1] + off;
    R w0[3], w1[3];
    V f0[3], f1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      w0[c] = WA[(int64_t)m0 * 81 + c * 27 + lane];
      w1[c] = WA[(int64_t)m1 * 81 + c * 27 + lane];
      f0[c] = phi[c * ng + nd0];
      f1[c] = phi[c * ng + nd1];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      acc0.x += w0[c] * f0[c].x;
      acc0.y += w0[c] * f0[c].y;
      acc1.x += w1[c] * f1[c].x;
      acc1.y += w1[c] * f1[c].y;
    }
  }
  if (!anear) {
    near_row_p(LA + rowA[m0], colA + lstA[m0], j, 0, rowA[m0 + 1] - rowA[m0], lane, acc0);
    near_row_p(LA + rowA[m1], colA + lstA[m1], j, 0, rowA[m1 + 1] - rowA[m1], lane, acc1);
  }
  if (anear && lane == 0) {
    const V an0 = anear[m0], an1 = anear[m1];
    acc0.x += an0.x;
    acc0.y += an0.y;
    acc1.x += an1.x;
    acc1.y += an1.y;
  }
  if (mode == 0) {
    acc0 = warp_sum(acc0);
    acc1 = warp_sum(acc1);
  } else {
    V t0 = jk0(acc0, k0), t1 = jk0(acc1, k0);
    t0.x += b0.x;
    t0.y += b0.y;
    t1.x += b1.x;
    t1.y += b1.y;
    acc0 = warp_sum(t0);
    acc1 = warp_sum(t1);
  }
  if (lane == 0) {
    y[m0] = acc0;
    if (two) y[m1] = acc1;
  }
}

// a = L^A_NR j (the near region of the RWG rows), one warp per row: the part of the system
// matvec's first row that needs only j, run beside the convolution
template <typename R, int PV = 0>
__global__ void __launch_bounds__(256) k_near_e(const int64_t* __restrict__ rowA,
                                                const int64_t* __restrict__ lstA,
                                                const int32_t* __restrict__ colA,
                                                const typename C2<R>::T* __restrict__ LA,
                                                const typename C2<R>::T* __restrict__ j, int ne,
                                                typename C2<R>::T* __restrict__ a, int64_t j_rs = 0,
                                                int64_t a_rs = 0) {
  typedef typename C2<R>::T V;
  j += blockIdx.y * j_rs;  // right-hand side blockIdx.y of a batch
  a += blockIdx.y * a_rs;
  const int m = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (m >= ne) return;
  V acc = czero<V>();
  near_row_v<PV>(LA + rowA[m], colA + lstA[m], j, 0, rowA[m + 1] - rowA[m], lane, acc);
  acc = warp_sum(acc);
  if (lane == 0) a[m] = acc;
}


// the row kernels' form the context selects (aim_rows_variant)
template <typename R> static decltype(&k_rows_t<R, 0>) rows_t_kernel(const aim_ctx* c) {
  return c->rows_variant >= 1 ? &k_rows_t<R, 1> : &k_rows_t<R, 0>;
}
template <typename R> static decltype(&k_near_e<R, 0>) near_e_kernel(const aim_ctx* c) {
  return c->rows_variant >= 1 ? &k_near_e<R, 1> : &k_near_e<R, 0>;
}
// (k_rows_e keeps near_row in form 1: its near sums run only for L^A alone, and near_row_p
// there would cost the system matvec's interpolation rows registers for nothing)
template <typename R> static decltype(&k_rows_e<R>) rows_e_kernel(const aim_ctx* c) {
  return c->rows_variant == 2 ? &k_rows_e2<R> : &k_rows_e<R>;
}
static inline int rows_e_per_block(const aim_ctx* c) { return c->rows_variant == 2 ? 16 : 8; }

// The system matvec of Eq. AEFIEoutJ for nrhs right-hand sides x_r = [h_r; q_r] (stride
// N_E + N_T) at once: each block matrix is read once for all of them (the GEMV takes the
// right-hand sides together), the convolution transforms 3 nrhs and nrhs grids per launch, and
// the projection, near-region and row kernels take the right-hand side from blockIdx.y. The
// internal products run on the main stream one after the other, the charge branch and the near
// region of j on the side stream (the serial schedule of the one-vector matvec).
template <typename R>
int matvec_batch(aim_ctx* c, const void* xv, void* yv, int nrhs, cudaStream_t s) {
  typedef typename C2<R>::T V;
  PrecBuf<R>& b = buf<R>(c);
  if (!b.bwsT) {
    set_error("batched matvec: buffers not made");
    return BEM_EINVAL;
  }
  const V* x = static_cast<const V*>(xv);
  V* y = static_cast<V*>(yv);
  const int ne = c->ne, nt = c->nt, nx = c->gn[0], ny = c->gn[1];
  const int64_t ng = c->ng, N = (int64_t)ne + nt;
  const R k0 = (R)c->k0;
  const GemvPlan& gp = sizeof(R) == 4 ? c->gplan : c->gplan64;
  BEM_CUDA(cudaEventRecord(c->ev_fork, s));
  BEM_CUDA(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
  project_t<R>(c, b.WPT, x + ne, b.bsT, c->side, nrhs, N);
  BEM_TRY(fft_conv<R>(c, b, b.bsT, b.bsT, nrhs, b.bwsT, c->side));
  rows_t_kernel<R>(c)<<<dim3(nb(nt, 8), nrhs), 256, 0, c->side>>>(b.WP, c->d_nodeT, b.bsT, c->d_rowP, c->d_lstP, c->d_clP,
                                                           b.LP, x + ne, nt, nx, ny, b.bp, ng, N, nt);
  auto gemv = [&](const V* A, V* out, const V* hs) -> int {
    return c->gmr.ntasks > 0 ? run_gemv_mr<R>(c->gmr, A, x, out, nrhs, N, hs, s)
                             : run_gemv_plan<R>(gp, A, x, out, nrhs, N, hs, s);
  };
  BEM_TRY(gemv(b.C, b.bj, x));  // j_r = h_r - C h_r
  BEM_CUDA(cudaEventRecord(c->ev_c, s));
  BEM_CUDA(cudaStreamWaitEvent(c->side, c->ev_c, 0));
  near_e_kernel<R>(c)<<<dim3(nb(ne, 8), nrhs), 256, 0, c->side>>>(c->d_rowA, c->d_lstA, c->d_clA, b.LA, b.bj, ne, b.ban,
                                                           N, ne);
  BEM_CUDA(cudaEventRecord(c->ev_join, c->side));
  if (c->zsp_on)  // e_r = Z_s h_r, the sparse internal operator
    BEM_TRY(zsp_apply<R>(c, x, b.be, nrhs, N, N, s));
  else
    BEM_TRY(gemv(b.Z, b.be, nullptr));  // e_r = Z h_r
  project_e<R>(c, b.WAT, b.bj, b.bsE, s, nrhs, N);
  BEM_TRY(fft_conv<R>(c, b, b.bsE, b.bsE, 3 * nrhs, b.bwsE, s));
  BEM_CUDA(cudaStreamWaitEvent(s, c->ev_join, 0));
  RowsStride rs;
  rs.phi = 3 * ng;
  rs.j = N;
  rs.e = N;
  rs.p = nt;
  rs.q = N;
  rs.an = ne;
  rs.y = N;
  rows_e_kernel<R>(c)<<<dim3(nb(ne, rows_e_per_block(c)) + nb(nt, 256), nrhs), 256, 0, s>>>(
      b.WA, c->d_nodeE, b.bsE, ng, c->d_rowA, c->d_lstA, c->d_clA, b.LA, b.bj, b.ix, c->d_ixcol, b.be, b.fdE,
      c->d_et, b.bp, ne, nx, ny, k0, 1, y, nt, b.fdT, c->d_tedge, x + ne, b.ban, rs);
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

template <typename R>
int batch_buffers(aim_ctx* c) {
  PrecBuf<R>& b = buf<R>(c);
  if (b.bwsT) return BEM_OK;
  const int64_t N = (int64_t)c->ne + c->nt, P3 = (int64_t)c->gp[0] * c->gp[1] * c->gp[2];
  BEM_TRY(dalloc_t(c, &b.bj, kMaxBatch * N));
  BEM_TRY(dalloc_t(c, &b.be, kMaxBatch * N));
  BEM_TRY(dalloc_t(c, &b.ban, kMaxBatch * (int64_t)c->ne));
  BEM_TRY(dalloc_t(c, &b.bp, kMaxBatch * (int64_t)c->nt));
  BEM_TRY(dalloc_t(c, &b.bsE, 3 * kMaxBatch * c->ng));
  BEM_TRY(dalloc_t(c, &b.bsT, kMaxBatch * c->ng));
  BEM_TRY(dalloc_t(c, &b.bwsE, 3 * kMaxBatch * P3));
  BEM_TRY(dalloc_t(c, &b.bwsT, kMaxBatch * P3));
  return BEM_OK;
}
template int batch_buffers<float>(aim_ctx*);
template int batch_buffers<double>(aim_ctx*);

template <typename R>
int matvec(aim_ctx* c, int which, const void* xv, void* yv, cudaStream_t s) {
  typedef typename C2<R>::T V;
  if (which > kBatchOp) return matvec_batch<R>(c, xv, yv, which - kBatchOp, s);
  PrecBuf<R>& b = buf<R>(c);
  const V* x = static_cast<const V*>(xv);
  V* y = static_cast<V*>(yv);
  const int ne = c->ne, nt = c->nt, nx = c->gn[0], ny = c->gn[1];
  const int64_t ng = c->ng;
  const R k0 = (R)c->k0;
  const int64_t P3 = (int64_t)c->gp[0] * c->gp[1] * c->gp[2];
  if (which == AIM_OP_LA) {
    project_e<R>(c, b.WAT, x, b.sigma, s);
    BEM_TRY(fft_conv<R>(c, b, b.sigma, b.sigma, 3, b.ws, s));
    rows_e_kernel<R>(c)<<<nb(ne, rows_e_per_block(c)), 256, 0, s>>>(
        b.WA, c->d_nodeE, b.sigma, ng, c->d_rowA, c->d_lstA, c->d_clA, b.LA, x, b.ix, c->d_ixcol,
        nullptr, b.fdE, c->d_et, nullptr, ne, nx, ny, k0, 0, y, nt, b.fdT, c->d_tedge, nullptr,
        nullptr, RowsStride());
  } else if (which == AIM_OP_LPHI) {
    V* sq = b.sigma + 3 * ng;
    project_t<R>(c, b.WPT, x, sq, s);
    BEM_TRY(fft_conv<R>(c, b, sq, sq, 1, b.ws + 3 * P3, s));
    rows_t_kernel<R>(c)<<<nb(nt, 8), 256, 0, s>>>(b.WP, c->d_nodeT, sq, c->d_rowP, c->d_lstP, c->d_clP, b.LP, x, nt,
                                          nx, ny, y, 0, 0, 0);
  } else if (which == AIM_OP_EXT) {
    // both external operators of Eq. AEFIEoutJ, as the system matvec runs them: L^A j on the
    // main stream, L^Phi q on the side stream, joined at the end
    const V* q = x + ne;
    V* sq = b.sigma + 3 * ng;
    BEM_CUDA(cudaEventRecord(c->ev_fork, s));
    BEM_CUDA(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    project_t<R>(c, b.WPT, q, sq, c->side);
    BEM_TRY(fft_conv<R>(c, b, sq, sq, 1, b.ws + 3 * P3, c->side));
    rows_t_kernel<R>(c)<<<nb(nt, 8), 256, 0, c->side>>>(b.WP, c->d_nodeT, sq, c->d_rowP, c->d_lstP, c->d_clP, b.LP, q,
                                                nt, nx, ny, y + ne, 0, 0, 0);
    BEM_CUDA(cudaEventRecord(c->ev_join, c->side));
    project_e<R>(c, b.WAT, x, b.sigma, s);
    BEM_TRY(fft_conv<R>(c, b, b.sigma, b.sigma, 3, b.ws, s));
    rows_e_kernel<R>(c)<<<nb(ne, rows_e_per_block(c)), 256, 0, s>>>(
        b.WA, c->d_nodeE, b.sigma, ng, c->d_rowA, c->d_lstA, c->d_clA, b.LA, x, b.ix, c->d_ixcol,
        nullptr, b.fdE, c->d_et, nullptr, ne, nx, ny, k0, 0, y, nt, b.fdT, c->d_tedge, nullptr,
        nullptr, RowsStride());
    BEM_CUDA(cudaStreamWaitEvent(s, c->ev_join, 0));
  } else if (which == AIM_OP_SYSTEM) {
    // With C = Y_eq Z formed at set-up (Eq. EFIEeqYZ), j = h - C h and e = Z h are
    // independent. The main stream runs j and its AIM chain (projection, convolution, rows);
    // e = Z h (needed only by the last kernel, for I_x e) runs, as the set-up schedule tuner
    // chose, beside j's GEMV or beside the chain with few CTAs (z_after 0 or 1), after j's
    // GEMV on the main stream (2), or in one launch with j's GEMV (3). The charge branch
    // p = L^Phi q runs on the side stream, followed there by the near region L^A_NR j once j is
    // out, so that only the interpolation and the combination follow the convolution.
    // With the sparse internal operator, e = Z_s h runs on its own stream from the start.
    const V* h = x;
    const V* q = x + ne;
    V* sq = b.sigma + 3 * ng;
    const int za = c->zsp_on ? 0 : c->z_after;
    BEM_CUDA(cudaEventRecord(c->ev_fork, s));
    BEM_CUDA(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    if (za < 2) BEM_CUDA(cudaStreamWaitEvent(c->zside, c->ev_fork, 0));
    project_t<R>(c, b.WPT, q, sq, c->side);
    BEM_TRY(fft_conv<R>(c, b, sq, sq, 1, b.ws + 3 * P3, c->side));
    rows_t_kernel<R>(c)<<<nb(nt, 8), 256, 0, c->side>>>(b.WP, c->d_nodeT, sq, c->d_rowP, c->d_lstP, c->d_clP, b.LP, q,
                                                nt, nx, ny, b.p, 0, 0, 0);
    const GemvPlan& gp = sizeof(R) == 4 ? c->gplan : c->gplan64;
    const GemvPlan& gb = sizeof(R) == 4 ? c->gbg32 : c->gbg64;
    if (c->zsp_on) BEM_TRY(zsp_apply<R>(c, h, b.e, 1, ne, ne, c->zside));
    if (za == 3)  // j = h - C h and e = Z h in one launch
      BEM_TRY(run_gemv_pair<R>(c->gpair, b.C, b.Z, h, b.j, b.e, h, s));
    else
      BEM_TRY(run_gemv_plan<R>(gp, b.C, h, b.j, 1, ne, h, s));
    BEM_CUDA(cudaEventRecord(c->ev_c, s));
    BEM_CUDA(cudaStreamWaitEvent(c->side, c->ev_c, 0));
    near_e_kernel<R>(c)<<<nb(ne, 8), 256, 0, c->side>>>(c->d_rowA, c->d_lstA, c->d_clA, b.LA, b.j, ne, b.anear,
                                                      0, 0);
    BEM_CUDA(cudaEventRecord(c->ev_join, c->side));
    if (za == 2) {  // e = Z h right after j's GEMV on the main stream, whole GPU
      BEM_TRY(run_gemv_plan<R>(gp, b.Z, h, b.e, 1, ne, nullptr, s));
    } else if (za != 3 && !c->zsp_on) {
      if (za)  // e = Z h once j is out, beside the AIM chain only
        BEM_CUDA(cudaStreamWaitEvent(c->zside, c->ev_c, 0));
      BEM_TRY(run_gemv_plan<R>(gb, b.Z, h, b.e, 1, ne, nullptr, c->zside));
    }
    BEM_CUDA(cudaEventRecord(c->ev_z, za >= 2 ? s : c->zside));
    project_e<R>(c, b.WAT, b.j, b.sigma, s);
    BEM_TRY(fft_conv<R>(c, b, b.sigma, b.sigma, 3, b.ws, s));
    BEM_CUDA(cudaStreamWaitEvent(s, c->ev_join, 0));
    BEM_CUDA(cudaStreamWaitEvent(s, c->ev_z, 0));
    rows_e_kernel<R>(c)<<<nb(ne, rows_e_per_block(c)) + nb(nt, 256), 256, 0, s>>>(
        b.WA, c->d_nodeE, b.sigma, ng, c->d_rowA, c->d_lstA, c->d_clA, b.LA, b.j, b.ix, c->d_ixcol,
        b.e, b.fdE, c->d_et, b.p, ne, nx, ny, k0, 1, y, nt, b.fdT, c->d_tedge, q, b.anear,
        RowsStride());
  } else {
    set_error("aim_matvec: unknown operator %d", which);
    return BEM_EINVAL;
  }
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}
template int matvec<float>(aim_ctx*, int, const void*, void*, cudaStream_t);
template int matvec<double>(aim_ctx*, int, const void*, void*, cudaStream_t);

int init_streams(aim_ctx* c) {
  BEM_CUDA(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
  BEM_CUDA(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
  BEM_CUDA(cudaStreamCreateWithFlags(&c->zside, cudaStreamNonBlocking));
  BEM_CUDA(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
  BEM_CUDA(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
  BEM_CUDA(cudaEventCreateWithFlags(&c->ev_z, cudaEventDisableTiming));
  BEM_CUDA(cudaEventCreateWithFlags(&c->ev_c, cudaEventDisableTiming));
  return BEM_OK;
}

void release_streams(aim_ctx* c) {
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
  c->graphs.clear();
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->ev_z) cudaEventDestroy(c->ev_z);
  if (c->ev_c) cudaEventDestroy(c->ev_c);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->zside) cudaStreamDestroy(c->zside);
  if (c->cap) cudaStreamDestroy(c->cap);
  c->ev_fork = c->ev_join = nullptr;
  c->side = c->cap = nullptr;
  for (int b = 0; b < 2; ++b) {
    for (cudaEvent_t* e : {&c->ev_in[b], &c->ev_comp[b], &c->ev_out[b]})
      if (*e) cudaEventDestroy(*e), *e = nullptr;
    for (void*& p : c->hbuf[b])
      if (p) cudaFree(p), p = nullptr;
  }
  if (c->h2d) cudaStreamDestroy(c->h2d);
  if (c->d2h) cudaStreamDestroy(c->d2h);
  c->h2d = c->d2h = nullptr;
}

// The matvec is ~12 kernels; replaying it as one CUDA graph removes the per-launch host cost.
// Graphs are captured on the context's private stream (the caller's stream may be the legacy
// default stream, which cannot be captured) and keyed by operator, precision and buffers.
template <typename R>
int matvec_graph(aim_ctx* c, int which, const void* x, void* y, cudaStream_t s) {
  if (!c->use_graphs) return matvec<R>(c, which, x, y, s);
  aim_ctx::GKey key{which, (int)sizeof(R), x, y};
  auto it = c->graphs.find(key);
  if (it == c->graphs.end()) {
    if (c->graphs.size() >= 64) {
      for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
      c->graphs.clear();
    }
    BEM_CUDA(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    int rc = matvec<R>(c, which, x, y, c->cap);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap, &g);
    if (rc != BEM_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      if (rc == BEM_OK) set_error("matvec capture: %s", cudaGetErrorString(e));
      return rc != BEM_OK ? rc : BEM_ECUDA;
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      set_error("matvec graph instantiate: %s", cudaGetErrorString(e));
      return BEM_ECUDA;
    }
    it = c->graphs.emplace(key, ex).first;
  }
  BEM_CUDA(cudaGraphLaunch(it->second, s));
  return BEM_OK;
}
template int matvec_graph<float>(aim_ctx*, int, const void*, void*, cudaStream_t);
template int matvec_graph<double>(aim_ctx*, int, const void*, void*, cudaStream_t);

// pure interpolation W (= P^T): u_m = sum_c sum_k WA[m][c][k] phi_c(node), u_{ne+t} likewise
template <typename R>
__global__ void __launch_bounds__(256) k_interp(const R* __restrict__ WA, const R* __restrict__ WP,
                                                const int32_t* __restrict__ nodeE,
                                                const int32_t* __restrict__ nodeT,
                                                const typename C2<R>::T* __restrict__ phi, int64_t ng,
                                                int ne, int nt, int nx, int ny,
                                                typename C2<R>::T* __restrict__ u) {
  typedef typename C2<R>::T V;
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= ne + nt) return;
  V acc = czero<V>();
  if (lane < 27) {
    if (row < ne) {
      const int64_t nd = nodeE[row] + node_offset(lane, nx, ny);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const R w = WA[(int64_t)row * 81 + c * 27 + lane];
        const V f = phi[c * ng + nd];
        acc.x += w * f.x;
        acc.y += w * f.y;
      }
    } else {
      const int t = row - ne;
      const R w = WP[(int64_t)t * 27 + lane];
      const V f = phi[3 * ng + nodeT[t] + node_offset(lane, nx, ny)];
      acc = mk(w * f.x, w * f.y);
    }
  }
  acc = warp_sum(acc);
  if (lane == 0) u[row] = acc;
}

// sigma = P r for a system vector r = [r_E; r_T]: comps 0..2 from r_E, comp 3 from r_T
template <typename R>
int project_all(aim_ctx* c, const typename C2<R>::T* r, typename C2<R>::T* sigma, cudaStream_t s) {
  PrecBuf<R>& b = buf<R>(c);
  const int64_t ng = c->ng;
  project_e<R>(c, b.WAT, r, sigma, s);
  project_t<R>(c, b.WPT, r + c->ne, sigma + 3 * ng, s);
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}
template int project_all<float>(aim_ctx*, const float2*, float2*, cudaStream_t);
template int project_all<double>(aim_ctx*, const double2*, double2*, cudaStream_t);

template <typename R>
int interp_all(aim_ctx* c, const typename C2<R>::T* phi, typename C2<R>::T* u, cudaStream_t s) {
  PrecBuf<R>& b = buf<R>(c);
  k_interp<R><<<nb(c->ne + c->nt, 8), 256, 0, s>>>(b.WA, b.WP, c->d_nodeE, c->d_nodeT, phi, c->ng,
                                                   c->ne, c->nt, c->gn[0], c->gn[1], u);
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}
template int interp_all<float>(aim_ctx*, const float2*, float2*, cudaStream_t);
template int interp_all<double>(aim_ctx*, const double2*, double2*, cudaStream_t);

template <typename R>
int internal(aim_ctx* c, const void* hv, void* ev, void* heqv, int nrhs, cudaStream_t s) {
  typedef typename C2<R>::T V;
  PrecBuf<R>& b = buf<R>(c);
  const GemvPlan& gp = sizeof(R) == 4 ? c->gplan : c->gplan64;
  if (!ev) {
  } else if (c->zsp_on) {  // e = Z_s h, the sparse internal operator
    BEM_TRY(zsp_apply<R>(c, (const V*)hv, (V*)ev, nrhs, c->ne, c->ne, s));
  } else if (nrhs == 1 && heqv && c->z_after == 3 && c->gpair.ntasks > 0) {  // the matvec's pair
    return run_gemv_pair<R>(c->gpair, b.C, b.Z, (const V*)hv, (V*)heqv, (V*)ev, nullptr, s);
  } else {
    BEM_TRY(run_gemv_plan<R>(gp, b.Z, (const V*)hv, (V*)ev, nrhs, c->ne, nullptr, s));
  }
  if (heqv) BEM_TRY(run_gemv_plan<R>(gp, b.C, (const V*)hv, (V*)heqv, nrhs, c->ne, nullptr, s));
  return BEM_OK;
}
template int internal<float>(aim_ctx*, const void*, void*, void*, int, cudaStream_t);
template int internal<double>(aim_ctx*, const void*, void*, void*, int, cudaStream_t);

template <typename R>
int conv(aim_ctx* c, const void* sigma, void* phi, int ncomp, cudaStream_t s) {
  typedef typename C2<R>::T V;
  PrecBuf<R>& b = buf<R>(c);
  return fft_conv<R>(c, b, (const V*)sigma, (V*)phi, ncomp, b.ws, s);
}
template int conv<float>(aim_ctx*, const void*, void*, int, cudaStream_t);
template int conv<double>(aim_ctx*, const void*, void*, int, cudaStream_t);

}  // namespace bem
