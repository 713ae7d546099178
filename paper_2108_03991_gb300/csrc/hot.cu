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
template <typename R> struct Vec16;
template <> struct Vec16<float> { typedef float4 T; static constexpr int kCplx = 2; };
template <> struct Vec16<double> { typedef double2 T; static constexpr int kCplx = 1; };

// One row of the product, one warp: acc[r] = sum_k A[row, k] x_r[k]. Rows are streamed with
// 16-byte loads (two complex FP32 or one complex FP64 per load), evict-first so the streamed
// matrix does not displace the vectors in L2; x is read through the read-only path (L1).
template <typename R, int NRHS>
__device__ __forceinline__ void row_dot(const typename C2<R>::T* __restrict__ arow_,
                                        const typename C2<R>::T* __restrict__ xb, int n,
                                        int64_t vstride, int lane, typename C2<R>::T* acc) {
  typedef typename C2<R>::T V;
  typedef typename Vec16<R>::T L16;
  constexpr int CP = Vec16<R>::kCplx;
  const L16* arow = reinterpret_cast<const L16*>(arow_);
#pragma unroll
  for (int r = 0; r < NRHS; ++r) acc[r] = czero<V>();
  const int nvec = (n + CP - 1) / CP;
#pragma unroll 4
  for (int v = lane; v < nvec; v += 32) {
    L16 a = __ldcs(arow + v);
    const int col = v * CP;
    if constexpr (CP == 2) {
      V a0 = mk(a.x, a.y), a1 = mk(a.z, a.w);
#pragma unroll
      for (int r = 0; r < NRHS; ++r) {
        V x0 = __ldg(xb + r * vstride + col);
        cfma(acc[r], a0, x0);
        if (col + 1 < n) {
          V x1 = __ldg(xb + r * vstride + col + 1);
          cfma(acc[r], a1, x1);
        }
      }
    } else {
      V a0 = mk(a.x, a.y);
#pragma unroll
      for (int r = 0; r < NRHS; ++r) cfma(acc[r], a0, __ldg(xb + r * vstride + col));
    }
  }
#pragma unroll
  for (int r = 0; r < NRHS; ++r) acc[r] = warp_sum(acc[r]);
}

// Task-list form (one CTA per task of at most 16 rows).
template <typename R, int NRHS>
__global__ void __launch_bounds__(256) k_gemv(const GemvTask* __restrict__ tasks,
                                              const typename C2<R>::T* __restrict__ A,
                                              const typename C2<R>::T* __restrict__ x,
                                              typename C2<R>::T* __restrict__ y, int64_t vstride,
                                              const typename C2<R>::T* __restrict__ hsub) {
  typedef typename C2<R>::T V;
  const GemvTask t = tasks[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const V* xb = x + t.xoff;
  for (int rr = warp; rr < t.nrows; rr += 8) {
    const int row = t.row0 + rr;
    V acc[NRHS];
    row_dot<R, NRHS>(A + t.aoff + (int64_t)row * t.ld, xb, t.n, vstride, lane, acc);
#pragma unroll
    for (int r = 0; r < NRHS; ++r) {
      if (lane == 0) {
        int64_t o = r * vstride + t.xoff + row;
        y[o] = hsub ? csub(hsub[o], acc[r]) : acc[r];
      }
    }
  }
}

// Persistent form: CTA p streams the rows of its byte-balanced range (GemvPlan). Each row is
// cut into S equal column parts; the S * rows work items of a chunk are dealt to the 8 warps
// in turn (one warp reduction per part), partial sums meet in shared memory and the CTA adds
// the S parts of each row at the end of the chunk. S = 1 is one warp per row; S = 2 or 4
// evens out the work of the warps when a CTA holds only a few rows per warp.
constexpr int kGemvChunk = 64;

template <typename R, int NRHS, int S>
__global__ void __launch_bounds__(kGemvThreads, kGemvCtasPerSm)
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
        const L16* arow = reinterpret_cast<const L16*>(A + ri.aoff);
        const V* xb = x + ri.xoff;
        V acc[NRHS];
#pragma unroll
        for (int r = 0; r < NRHS; ++r) acc[r] = czero<V>();
#pragma unroll 4
        for (int v = v0 + lane; v < v1; v += 32) {
          const L16 a = __ldcs(arow + v);
          const int col = v * CP;
          if constexpr (CP == 2) {
            const V a0 = mk(a.x, a.y), a1 = mk(a.z, a.w);
#pragma unroll
            for (int r = 0; r < NRHS; ++r) {
              cfma(acc[r], a0, __ldg(xb + r * vstride + col));
              if (col + 1 < ri.n) cfma(acc[r], a1, __ldg(xb + r * vstride + col + 1));
            }
          } else {
#pragma unroll
            for (int r = 0; r < NRHS; ++r) cfma(acc[r], mk(a.x, a.y), __ldg(xb + r * vstride + col));
          }
        }
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

template <typename R, int S>
static void launch_gemv_plan(const GemvPlan& p, const typename C2<R>::T* A,
                             const typename C2<R>::T* x, typename C2<R>::T* y, int nr,
                             int64_t vstride, const typename C2<R>::T* hs, cudaStream_t s) {
  switch (nr) {
    case 1: k_gemv_plan<R, 1, S><<<p.ncta, kGemvThreads, 0, s>>>(p.rows, p.segs, p.cta_seg, A, x, y, vstride, hs); break;
    case 2: k_gemv_plan<R, 2, S><<<p.ncta, kGemvThreads, 0, s>>>(p.rows, p.segs, p.cta_seg, A, x, y, vstride, hs); break;
    case 3: k_gemv_plan<R, 3, S><<<p.ncta, kGemvThreads, 0, s>>>(p.rows, p.segs, p.cta_seg, A, x, y, vstride, hs); break;
    default: k_gemv_plan<R, 4, S><<<p.ncta, kGemvThreads, 0, s>>>(p.rows, p.segs, p.cta_seg, A, x, y, vstride, hs); break;
  }
}

template <typename R>
int run_gemv_plan(const GemvPlan& p, const typename C2<R>::T* A, const typename C2<R>::T* x,
                  typename C2<R>::T* y, int nrhs, int64_t vstride, const typename C2<R>::T* hsub,
                  cudaStream_t s) {
  if (p.ncta == 0 || p.nrows == 0) return BEM_OK;
  if (p.tma) return run_gemv_tma<R>(p, A, x, y, nrhs, vstride, hsub, s);
  for (int r0 = 0; r0 < nrhs; r0 += 4) {
    const int nr = std::min(4, nrhs - r0);
    const int64_t o = r0 * vstride;
    const typename C2<R>::T* hs = hsub ? hsub + o : nullptr;
    switch (p.split) {
      case 1: launch_gemv_plan<R, 1>(p, A, x + o, y + o, nr, vstride, hs, s); break;
      case 4: launch_gemv_plan<R, 4>(p, A, x + o, y + o, nr, vstride, hs, s); break;
      default: launch_gemv_plan<R, 2>(p, A, x + o, y + o, nr, vstride, hs, s); break;
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
// projection P: scatter with atomics, one thread per (source, stencil node)
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int node_offset(int k, int nx, int ny) {
  return ((k / 9 - 1) * ny + ((k / 3) % 3 - 1)) * nx + (k % 3 - 1);
}

// complex atomic add: one 8-byte vector atomic in FP32, two scalar atomics in FP64
__device__ __forceinline__ void catomic_add(float2* o, float2 v) { atomicAdd(o, v); }
__device__ __forceinline__ void catomic_add(double2* o, double2 v) {
  atomicAdd(&o->x, v.x);
  atomicAdd(&o->y, v.y);
}

template <typename R>
__global__ void k_scatter_e(const R* __restrict__ WA, const int32_t* __restrict__ node,
                            const typename C2<R>::T* __restrict__ j, typename C2<R>::T* sigma,
                            int ne, int nx, int ny, int64_t ng) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)ne * 27) return;
  const int m = (int)(idx / 27), k = (int)(idx - (int64_t)m * 27);
  const typename C2<R>::T v = j[m];
  const int64_t nd = node[m] + node_offset(k, nx, ny);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const R w = WA[(int64_t)m * 81 + c * 27 + k];
    catomic_add(sigma + c * ng + nd, mk(w * v.x, w * v.y));
  }
}

template <typename R>
__global__ void k_scatter_t(const R* __restrict__ WP, const int32_t* __restrict__ node,
                            const typename C2<R>::T* __restrict__ q, typename C2<R>::T* sigma,
                            int nt, int nx, int ny) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)nt * 27) return;
  const int t = (int)(idx / 27), k = (int)(idx - (int64_t)t * 27);
  const typename C2<R>::T v = q[t];
  const R w = WP[(int64_t)t * 27 + k];
  catomic_add(sigma + node[t] + node_offset(k, nx, ny), mk(w * v.x, w * v.y));
}

// Gather form of the projection (no atomics, deterministic): one thread per grid node sums the
// sources whose stencils touch it, from the node-major CSR of P^T. Every node is written, so
// the grids need no clearing.
template <typename R>
__global__ void __launch_bounds__(256) k_project_e(const int32_t* __restrict__ prow,
                                                   const int32_t* __restrict__ pcol,
                                                   const R* __restrict__ WT,
                                                   const typename C2<R>::T* __restrict__ j,
                                                   typename C2<R>::T* __restrict__ sigma, int64_t ng) {
  typedef typename C2<R>::T V;
  const int64_t nd = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (nd >= ng) return;
  V a0 = czero<V>(), a1 = czero<V>(), a2 = czero<V>();
  const int e1 = prow[nd + 1];
  for (int e = prow[nd]; e < e1; ++e) {
    const V v = j[pcol[e]];
    const R w0 = WT[3 * (int64_t)e], w1 = WT[3 * (int64_t)e + 1], w2 = WT[3 * (int64_t)e + 2];
    a0.x += w0 * v.x; a0.y += w0 * v.y;
    a1.x += w1 * v.x; a1.y += w1 * v.y;
    a2.x += w2 * v.x; a2.y += w2 * v.y;
  }
  sigma[nd] = a0;
  sigma[ng + nd] = a1;
  sigma[2 * ng + nd] = a2;
}

template <typename R>
__global__ void __launch_bounds__(256) k_project_t(const int32_t* __restrict__ prow,
                                                   const int32_t* __restrict__ pcol,
                                                   const R* __restrict__ WT,
                                                   const typename C2<R>::T* __restrict__ q,
                                                   typename C2<R>::T* __restrict__ sigma, int64_t ng) {
  typedef typename C2<R>::T V;
  const int64_t nd = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (nd >= ng) return;
  V a = czero<V>();
  const int e1 = prow[nd + 1];
  for (int e = prow[nd]; e < e1; ++e) {
    const V v = q[pcol[e]];
    const R w = WT[e];
    a.x += w * v.x;
    a.y += w * v.y;
  }
  sigma[nd] = a;
}

// ---------------------------------------------------------------------------------------
// interpolation W + near region + combination, one warp per output row
// ---------------------------------------------------------------------------------------
template <typename V, typename R>
__device__ __forceinline__ V jk0(V a, R k0) { return mk(-k0 * a.y, k0 * a.x); }

// p_t = (W_Phi phi)_t + (L^Phi_NR q)_t, written to out[t] (y for L^Phi alone, p in the system)
template <typename R>
__global__ void __launch_bounds__(256) k_rows_t(
    const R* __restrict__ WP, const int32_t* __restrict__ node,
    const typename C2<R>::T* __restrict__ phi, const int64_t* __restrict__ rowP,
    const int32_t* __restrict__ colP, const typename C2<R>::T* __restrict__ LP,
    const typename C2<R>::T* __restrict__ q, int nt, int nx, int ny,
    typename C2<R>::T* __restrict__ out) {
  typedef typename C2<R>::T V;
  const int t = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (t >= nt) return;
  V acc = czero<V>();
  if (lane < 27) {
    const R w = WP[(int64_t)t * 27 + lane];
    const V f = phi[node[t] + node_offset(lane, nx, ny)];
    acc = mk(w * f.x, w * f.y);
  }
  for (int64_t i = rowP[t] + lane; i < rowP[t + 1]; i += 32) cfma(acc, LP[i], q[colP[i]]);
  acc = warp_sum(acc);
  if (lane == 0) out[t] = acc;
}

// mode 0: y[m] = a_m (L^A alone).
// mode 1 (system), rows m < ne:  y1_m = j k0 a_m + (I_x e)_m - ((F D)^T p)_m
//                  rows ne + t:  y2_t = (F D j)_t + j k0 q_t
template <typename R>
__global__ void __launch_bounds__(256) k_rows_e(
    const R* __restrict__ WA, const int32_t* __restrict__ node,
    const typename C2<R>::T* __restrict__ phi, int64_t ng, const int64_t* __restrict__ rowA,
    const int32_t* __restrict__ colA, const typename C2<R>::T* __restrict__ LA,
    const typename C2<R>::T* __restrict__ j, const R* __restrict__ ix,
    const int32_t* __restrict__ ixcol, const typename C2<R>::T* __restrict__ e,
    const R* __restrict__ fdE, const int32_t* __restrict__ et,
    const typename C2<R>::T* __restrict__ p, int ne, int nx, int ny, R k0, int mode,
    typename C2<R>::T* __restrict__ y, int nt, const R* __restrict__ fdT,
    const int32_t* __restrict__ tedge, const typename C2<R>::T* __restrict__ q) {
  typedef typename C2<R>::T V;
  const int m = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (mode == 1 && m >= ne && m < ne + nt) {
    if (lane == 0) {
      const int t = m - ne;
      V s = jk0(q[t], k0);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const V jj = j[tedge[3 * t + i]];
        const R c = fdT[3 * t + i];
        s.x += c * jj.x;
        s.y += c * jj.y;
      }
      y[m] = s;
    }
    return;
  }
  if (m >= ne) return;
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
  for (int64_t i = rowA[m] + lane; i < rowA[m + 1]; i += 32) cfma(acc, LA[i], j[colA[i]]);
  acc = warp_sum(acc);
  if (lane == 0) {
    if (mode == 0) {
      y[m] = acc;
    } else {
      V s = jk0(acc, k0);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const V ev = e[ixcol[4 * m + i]];
        const R c = ix[4 * m + i];
        s.x += c * ev.x;
        s.y += c * ev.y;
      }
      const V pp = p[et[2 * m]], pm = p[et[2 * m + 1]];
      const R cp = fdE[2 * m], cm = fdE[2 * m + 1];
      s.x += -cp * pp.x + cm * pm.x;
      s.y += -cp * pp.y + cm * pm.y;
      y[m] = s;
    }
  }
}

static inline unsigned nb(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

template <typename R> PrecBuf<R>& buf(aim_ctx* c);
template <> PrecBuf<float>& buf<float>(aim_ctx* c) { return c->f32; }
template <> PrecBuf<double>& buf<double>(aim_ctx* c) { return c->f64; }

template <typename R>
int matvec(aim_ctx* c, int which, const void* xv, void* yv, cudaStream_t s) {
  typedef typename C2<R>::T V;
  PrecBuf<R>& b = buf<R>(c);
  const V* x = static_cast<const V*>(xv);
  V* y = static_cast<V*>(yv);
  const int ne = c->ne, nt = c->nt, nx = c->gn[0], ny = c->gn[1];
  const int64_t ng = c->ng;
  const R k0 = (R)c->k0;
  const int64_t P3 = (int64_t)c->gp[0] * c->gp[1] * c->gp[2];
  if (which == AIM_OP_LA) {
    k_project_e<R><<<nb(ng, 256), 256, 0, s>>>(c->d_prowE, c->d_pcolE, b.WAT, x, b.sigma, ng);
    BEM_TRY(fft_conv<R>(c, b, b.sigma, b.sigma, 3, b.ws, s));
    k_rows_e<R><<<nb(ne, 8), 256, 0, s>>>(b.WA, c->d_nodeE, b.sigma, ng, c->d_rowA, c->d_colA, b.LA,
                                          x, b.ix, c->d_ixcol, nullptr, b.fdE, c->d_et, nullptr, ne,
                                          nx, ny, k0, 0, y, nt, b.fdT, c->d_tedge, nullptr);
  } else if (which == AIM_OP_LPHI) {
    V* sq = b.sigma + 3 * ng;
    k_project_t<R><<<nb(ng, 256), 256, 0, s>>>(c->d_prowT, c->d_pcolT, b.WPT, x, sq, ng);
    BEM_TRY(fft_conv<R>(c, b, sq, sq, 1, b.ws + 3 * P3, s));
    k_rows_t<R><<<nb(nt, 8), 256, 0, s>>>(b.WP, c->d_nodeT, sq, c->d_rowP, c->d_colP, b.LP, x, nt,
                                          nx, ny, y);
  } else if (which == AIM_OP_SYSTEM) {
    // Two branches: the charge branch p = L^Phi q does not depend on the internal problem and
    // runs on the side stream while the GEMVs stream Z and Y_eq.
    const V* h = x;
    const V* q = x + ne;
    V* sq = b.sigma + 3 * ng;
    BEM_CUDA(cudaEventRecord(c->ev_fork, s));
    BEM_CUDA(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    k_project_t<R><<<nb(ng, 256), 256, 0, c->side>>>(c->d_prowT, c->d_pcolT, b.WPT, q, sq, ng);
    BEM_TRY(fft_conv<R>(c, b, sq, sq, 1, b.ws + 3 * P3, c->side));
    k_rows_t<R><<<nb(nt, 8), 256, 0, c->side>>>(b.WP, c->d_nodeT, sq, c->d_rowP, c->d_colP, b.LP, q,
                                                nt, nx, ny, b.p);
    BEM_CUDA(cudaEventRecord(c->ev_join, c->side));
    const GemvPlan& gp = sizeof(R) == 4 ? c->gplan : c->gplan64;
    BEM_TRY(run_gemv_plan<R>(gp, b.Z, h, b.e, 1, ne, nullptr, s));
    BEM_TRY(run_gemv_plan<R>(gp, b.Y, b.e, b.j, 1, ne, h, s));
    k_project_e<R><<<nb(ng, 256), 256, 0, s>>>(c->d_prowE, c->d_pcolE, b.WAT, b.j, b.sigma, ng);
    BEM_TRY(fft_conv<R>(c, b, b.sigma, b.sigma, 3, b.ws, s));
    BEM_CUDA(cudaStreamWaitEvent(s, c->ev_join, 0));
    k_rows_e<R><<<nb(ne + nt, 8), 256, 0, s>>>(b.WA, c->d_nodeE, b.sigma, ng, c->d_rowA, c->d_colA,
                                               b.LA, b.j, b.ix, c->d_ixcol, b.e, b.fdE, c->d_et, b.p,
                                               ne, nx, ny, k0, 1, y, nt, b.fdT, c->d_tedge, q);
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
  BEM_CUDA(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
  BEM_CUDA(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
  return BEM_OK;
}

void release_streams(aim_ctx* c) {
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
  c->graphs.clear();
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->cap) cudaStreamDestroy(c->cap);
  c->ev_fork = c->ev_join = nullptr;
  c->side = c->cap = nullptr;
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
  k_project_e<R><<<nb(ng, 256), 256, 0, s>>>(c->d_prowE, c->d_pcolE, b.WAT, r, sigma, ng);
  k_project_t<R><<<nb(ng, 256), 256, 0, s>>>(c->d_prowT, c->d_pcolT, b.WPT, r + c->ne, sigma + 3 * ng, ng);
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
  BEM_TRY(run_gemv_plan<R>(gp, b.Z, (const V*)hv, (V*)ev, nrhs, c->ne, nullptr, s));
  if (heqv) BEM_TRY(run_gemv_plan<R>(gp, b.Y, (const V*)ev, (V*)heqv, nrhs, c->ne, nullptr, s));
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
