// Block-diagonal GEMV with bulk-copy (TMA) staging: the internal-problem products e = Z h and
// h_eq = Y e (Eqs. MFIEinZin, EFIEeqYeq; block diagonal over objects, Sec. II-C).
//
// Each persistent CTA owns a byte-balanced, contiguous range of matrix rows (rows of consecutive
// blocks are adjacent in memory), cut on the host into stages of whole rows. A producer warp
// streams the stages into a ring of shared-memory buffers with cp.async.bulk; an mbarrier's
// transaction count signals arrival. Eight consumer warps treat a stage as one flat array of
// 16-byte vectors split evenly between them whatever the row lengths; every lane accumulates the
// dot product of its current row and adds it into a per-row partial in shared memory when its row
// changes. The partials are written out (optionally as hsub - A x) when the stage is done and the
// buffer goes back to the producer. Every wait is bounded: on a timeout the kernel records an
// error code in *err and all warps leave together (the result is then invalid, the context
// stays usable).
#include "common.cuh"

namespace bem {

constexpr int kTmaConsumerWarps = 8;
constexpr int kTmaThreads = (kTmaConsumerWarps + 1) * 32;
constexpr int kTmaMaxRows = 64;          // rows per stage
constexpr uint32_t kTmaSpin = 1u << 24;  // bounded mbarrier polls

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity) {
  for (uint32_t it = 0; it < kTmaSpin; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// barrier of the consumer warps only (named barrier 1); returns true when any thread passed fail
__device__ __forceinline__ bool consumers_any(bool fail) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred p, 1, %2, q;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)fail), "n"(kTmaConsumerWarps * 32)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void consumers_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kTmaConsumerWarps * 32) : "memory");
}

__device__ __forceinline__ void sadd(float2* p, float2 v) {
  atomicAdd(&p->x, v.x);
  atomicAdd(&p->y, v.y);
}
__device__ __forceinline__ void sadd(double2* p, double2 v) {
  atomicAdd(&p->x, v.x);
  atomicAdd(&p->y, v.y);
}

template <typename R> struct Vec16T;
template <> struct Vec16T<float> { typedef float4 T; static constexpr int kCplx = 2; };
template <> struct Vec16T<double> { typedef double2 T; static constexpr int kCplx = 1; };

template <typename R, int NRHS, int NST>
__global__ void __launch_bounds__(kTmaThreads, 1)
    k_gemv_tma(const RowInfo* __restrict__ rows, const int32_t* __restrict__ soff,
               const TmaStage* __restrict__ stages, const int32_t* __restrict__ cta_stage,
               const typename C2<R>::T* __restrict__ A, const typename C2<R>::T* __restrict__ x,
               typename C2<R>::T* __restrict__ y, int64_t vstride,
               const typename C2<R>::T* __restrict__ hsub, int stage_bytes, int* err) {
  typedef typename C2<R>::T V;
  typedef typename Vec16T<R>::T L16;
  constexpr int CP = Vec16T<R>::kCplx;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* bufs = smem;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)NST * stage_bytes);
  uint64_t* empty = full + NST;
  V* part = reinterpret_cast<V*>(empty + NST);  // [kTmaMaxRows][NRHS]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int st0 = cta_stage[blockIdx.x], nst = cta_stage[blockIdx.x + 1] - st0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kTmaConsumerWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = threadIdx.x; i < kTmaMaxRows * NRHS; i += blockDim.x) part[i] = czero<V>();
  __syncthreads();
  if (warp == kTmaConsumerWarps) {
    // ---------------- producer ----------------
    if (lane == 0) {
      for (int i = 0; i < nst; ++i) {
        const int s = i % NST;
        if (!mbar_wait(&empty[s], ((i / NST) & 1) ^ 1)) {
          atomicExch(err, 1);
          break;
        }
        const TmaStage st = stages[st0 + i];
        const uint32_t bytes = (uint32_t)st.nel * (uint32_t)sizeof(V);
        mbar_arrive_tx(&full[s], bytes);
        bulk_g2s(bufs + (size_t)s * stage_bytes, A + st.e0, bytes, &full[s]);
      }
    }
    return;
  }
  // ---------------- consumers ----------------
  for (int i = 0; i < nst; ++i) {
    const int s = i % NST;
    const bool ok = mbar_wait(&full[s], (i / NST) & 1);
    if (consumers_any(!ok)) {
      if (threadIdx.x == 0) atomicExch(err, 2);
      break;
    }
    const TmaStage st = stages[st0 + i];
    const int nr = st.r1 - st.r0;
    const L16* sb = reinterpret_cast<const L16*>(bufs + (size_t)s * stage_bytes);
    const int nvec = st.nel / CP;
    const int per = (nvec + kTmaConsumerWarps - 1) / kTmaConsumerWarps;
    const int v0 = warp * per, v1 = min(nvec, v0 + per);
    if (v0 + lane < v1) {
      int k = 0;
      int e = (v0 + lane) * CP;
      while (k < nr - 1 && e >= soff[st.r0 + k + 1]) ++k;
      int rend = (k < nr - 1) ? soff[st.r0 + k + 1] : st.nel;
      RowInfo ri = rows[st.r0 + k];
      int rbeg = soff[st.r0 + k];
      V acc[NRHS];
#pragma unroll
      for (int r = 0; r < NRHS; ++r) acc[r] = czero<V>();
      for (int v = v0 + lane; v < v1; v += 32) {
        e = v * CP;
        if (e >= rend) {
#pragma unroll
          for (int r = 0; r < NRHS; ++r) { sadd(&part[k * NRHS + r], acc[r]); acc[r] = czero<V>(); }
          while (k < nr - 1 && e >= soff[st.r0 + k + 1]) ++k;
          rend = (k < nr - 1) ? soff[st.r0 + k + 1] : st.nel;
          rbeg = soff[st.r0 + k];
          ri = rows[st.r0 + k];
        }
        const int col = e - rbeg;
        const L16 a = sb[v];
        const V* xb = x + ri.xoff + col;
        if constexpr (CP == 2) {
          if (col < ri.n) {
#pragma unroll
            for (int r = 0; r < NRHS; ++r) cfma(acc[r], mk(a.x, a.y), __ldg(xb + r * vstride));
          }
          if (col + 1 < ri.n) {
#pragma unroll
            for (int r = 0; r < NRHS; ++r) cfma(acc[r], mk(a.z, a.w), __ldg(xb + r * vstride + 1));
          }
        } else {
          if (col < ri.n) {
#pragma unroll
            for (int r = 0; r < NRHS; ++r) cfma(acc[r], mk(a.x, a.y), __ldg(xb + r * vstride));
          }
        }
      }
#pragma unroll
      for (int r = 0; r < NRHS; ++r) sadd(&part[k * NRHS + r], acc[r]);
    }
    consumers_sync();
    for (int t = threadIdx.x; t < nr * NRHS; t += kTmaConsumerWarps * 32) {
      const int rr = t / NRHS, r = t - rr * NRHS;
      const int64_t o = r * vstride + st.r0 + rr;
      const V val = part[t];
      y[o] = hsub ? csub(hsub[o], val) : val;
      part[t] = czero<V>();
    }
    consumers_sync();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
}

template <typename R, int NST>
static void launch_tma(const GemvPlan& p, const typename C2<R>::T* A, const typename C2<R>::T* x,
                       typename C2<R>::T* y, int nr, int64_t vstride, const typename C2<R>::T* hs,
                       cudaStream_t s) {
  typedef typename C2<R>::T V;
  const size_t sm = (size_t)NST * p.stage_bytes + 2 * NST * 8 + (size_t)kTmaMaxRows * 4 * sizeof(V);
#define BEM_TMA(NR)                                                                               \
  do {                                                                                           \
    k_gemv_tma<R, NR, NST><<<p.ncta, kTmaThreads, sm, s>>>(p.rows, p.soff, p.stages, p.cta_stage, \
                                                           A, x, y, vstride, hs, p.stage_bytes,   \
                                                           p.err);                                \
  } while (0)
  switch (nr) {
    case 1: BEM_TMA(1); break;
    case 2: BEM_TMA(2); break;
    case 3: BEM_TMA(3); break;
    default: BEM_TMA(4); break;
  }
#undef BEM_TMA
}

template <typename R>
int run_gemv_tma(const GemvPlan& p, const typename C2<R>::T* A, const typename C2<R>::T* x,
                 typename C2<R>::T* y, int nrhs, int64_t vstride, const typename C2<R>::T* hsub,
                 cudaStream_t s) {
  for (int r0 = 0; r0 < nrhs; r0 += 4) {
    const int nr = std::min(4, nrhs - r0);
    const int64_t o = r0 * vstride;
    const typename C2<R>::T* hs = hsub ? hsub + o : nullptr;
    if (p.nstage == 3) launch_tma<R, 3>(p, A, x + o, y + o, nr, vstride, hs, s);
    else launch_tma<R, 4>(p, A, x + o, y + o, nr, vstride, hs, s);
  }
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}
template int run_gemv_tma<float>(const GemvPlan&, const float2*, const float2*, float2*, int,
                                 int64_t, const float2*, cudaStream_t);
template int run_gemv_tma<double>(const GemvPlan&, const double2*, const double2*, double2*, int,
                                  int64_t, const double2*, cudaStream_t);

// Allow the ring of stages (up to 4 x 48 KB) in dynamic shared memory; called at set-up.
int tma_init_attrs() {
  const int lim = 200 * 1024;
#define BEM_ATTR(RR, NR, NST) \
  BEM_CUDA(cudaFuncSetAttribute(k_gemv_tma<RR, NR, NST>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))
  BEM_ATTR(float, 1, 3); BEM_ATTR(float, 2, 3); BEM_ATTR(float, 3, 3); BEM_ATTR(float, 4, 3);
  BEM_ATTR(float, 1, 4); BEM_ATTR(float, 2, 4); BEM_ATTR(float, 3, 4); BEM_ATTR(float, 4, 4);
  BEM_ATTR(double, 1, 3); BEM_ATTR(double, 2, 3); BEM_ATTR(double, 3, 3); BEM_ATTR(double, 4, 3);
  BEM_ATTR(double, 1, 4); BEM_ATTR(double, 2, 4); BEM_ATTR(double, 3, 4); BEM_ATTR(double, 4, 4);
#undef BEM_ATTR
  return BEM_OK;
}

// Cut the rows of each CTA's byte-balanced range into stages of whole rows: at most stage_elems
// complex elements (row storage ld = n rounded up to 4) and kTmaMaxRows rows. soff[row] is the
// row's element offset inside its stage. False when one row does not fit a stage.
bool build_tma_stages(const std::vector<RowInfo>& rows, const std::vector<int2>& segs,
                      const std::vector<int32_t>& cta_seg, int64_t stage_elems,
                      std::vector<TmaStage>* stages, std::vector<int32_t>* cta_stage,
                      std::vector<int32_t>* soff) {
  const int ncta = (int)cta_seg.size() - 1;
  stages->clear();
  cta_stage->assign(ncta + 1, 0);
  soff->assign(rows.size(), 0);
  for (int c = 0; c < ncta; ++c) {
    for (int q = cta_seg[c]; q < cta_seg[c + 1]; ++q) {
      int cur = segs[q].x;
      const int end = segs[q].y;
      while (cur < end) {
        const int start = cur;
        int64_t el = 0;
        while (cur < end && cur - start < kTmaMaxRows) {
          const int64_t ld = (rows[cur].n + 3) & ~3;
          if (el + ld > stage_elems) break;
          (*soff)[cur] = (int32_t)el;
          el += ld;
          ++cur;
        }
        if (cur == start) return false;
        TmaStage st;
        st.r0 = start;
        st.r1 = cur;
        st.e0 = rows[start].aoff;
        st.nel = (int32_t)el;
        st.pad = 0;
        stages->push_back(st);
      }
    }
    (*cta_stage)[c + 1] = (int32_t)stages->size();
  }
  return true;
}

}  // namespace bem
