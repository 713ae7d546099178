// Block-diagonal GEMV with bulk-copy (TMA) staging: the internal-problem products e = Z h and
// h_eq = Y e (Eqs. MFIEinZin, EFIEeqYeq; block diagonal over objects, Sec. II-C).
//
// Each persistent CTA owns a byte-balanced, contiguous range of matrix rows (rows of consecutive
// blocks are adjacent in memory), cut on the host into stages of whole rows. A producer warp
// streams the stages into a ring of shared-memory slots with cp.async.bulk: the stage's matrix
// bytes and its row table (TmaDesc) land in the slot and an mbarrier's transaction count
// signals arrival. Sixteen consumer warps split a stage's 16-byte vectors evenly between them
// whatever the row lengths; a warp walks the rows its share touches, lanes strided within a
// row with 4 vectors in flight each (2 when two CTAs share an SM), and adds each row's warp sum
// into a per-row partial in shared memory. The consumer warps do not meet at a barrier: a
// per-slot counter elects the last warp done with a stage, which writes the stage's rows out
// (optionally as hsub - A x) and clears the partials; every warp then releases the slot to the
// producer.
// Every wait is bounded: on a timeout the kernel records an error code in *err and the warps
// leave (the result is then invalid, the context stays usable).
#include "bulk.cuh"
#include "common.cuh"

namespace bem {

constexpr int kTmaConsumerWarps = 16;
constexpr int kTmaThreads = (kTmaConsumerWarps + 1) * 32;

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

// shared-memory layout of one CTA (byte offsets), shared by the kernel and its launcher
struct TmaSmem {
  size_t desc, full, empty, done, part, total;
  __host__ __device__ TmaSmem(int nst, int stage_bytes, int part_bytes) {
    desc = (size_t)nst * stage_bytes;
    full = desc + (size_t)nst * sizeof(TmaDesc);
    empty = full + 8 * (size_t)nst;
    done = empty + 8 * (size_t)nst;
    part = (done + 4 * (size_t)nst + 15) & ~(size_t)15;
    total = part + (size_t)nst * part_bytes;
  }
};

template <typename R, int NRHS, int NST>
__global__ void __launch_bounds__(kTmaThreads, NST == 3 ? 2 : 1)
    k_gemv_tma(const TmaStage* __restrict__ stages, const TmaDesc* __restrict__ descs,
               const int32_t* __restrict__ cta_stage, const typename C2<R>::T* __restrict__ A,
               const typename C2<R>::T* __restrict__ x, typename C2<R>::T* __restrict__ y,
               int64_t vstride, const typename C2<R>::T* __restrict__ hsub, int stage_bytes,
               int* err) {
  typedef typename C2<R>::T V;
  typedef typename Vec16T<R>::T L16;
  constexpr int CP = Vec16T<R>::kCplx;
  constexpr int CW = kTmaConsumerWarps;
  constexpr int kPart = kTmaMaxRows * NRHS;  // partials per slot
  constexpr int kTmaU = NST == 3 ? 2 : 4;    // 16-byte vectors in flight per consumer lane
  extern __shared__ __align__(128) unsigned char smem[];
  const TmaSmem L(NST, stage_bytes, kPart * (int)sizeof(V));
  TmaDesc* desc = reinterpret_cast<TmaDesc*>(smem + L.desc);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.full);
  uint64_t* empty = reinterpret_cast<uint64_t*>(smem + L.empty);
  int* done = reinterpret_cast<int*>(smem + L.done);
  V* part = reinterpret_cast<V*>(smem + L.part);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int st0 = cta_stage[blockIdx.x], nst = cta_stage[blockIdx.x + 1] - st0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], CW);
      done[s] = 0;
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = threadIdx.x; i < NST * kPart; i += blockDim.x) part[i] = czero<V>();
  __syncthreads();
  if (warp == CW) {
    // ---------------- producer ----------------
    if (lane == 0) {
      int issued = 0;
      for (int i = 0; i < nst; ++i) {
        const int s = i % NST;
        if (!mbar_wait(&empty[s], ((i / NST) & 1) ^ 1)) {
          atomicExch(err, 1);
          break;
        }
        const TmaStage st = stages[st0 + i];
        const uint32_t bytes = (uint32_t)st.nel * (uint32_t)sizeof(V);
        mbar_arrive_tx(&full[s], bytes + (uint32_t)sizeof(TmaDesc));
        bulk_g2s(smem + (size_t)s * stage_bytes, A + st.e0, bytes, &full[s]);
        bulk_g2s(&desc[s], descs + st0 + i, (uint32_t)sizeof(TmaDesc), &full[s]);
        issued = i + 1;
      }
      // no copy may still be landing in shared memory when the CTA ends: wait (bounded) for
      // the last copy into each slot (later waits on the same phase return at once)
      for (int i = max(0, issued - NST); i < issued; ++i)
        if (!mbar_wait(&full[i % NST], (i / NST) & 1)) atomicExch(err, 3);
    }
    return;
  }
  // ---------------- consumers ----------------
  for (int i = 0; i < nst; ++i) {
    const int s = i % NST;
    const bool ok = mbar_wait(&full[s], (i / NST) & 1);
    if (__any_sync(0xffffffffu, !ok)) {
      if (lane == 0) atomicExch(err, 2);
      break;
    }
    const TmaDesc& d = desc[s];
    const int nr = d.nr;
    const L16* sb = reinterpret_cast<const L16*>(smem + (size_t)s * stage_bytes);
    V* ps = part + s * kPart;
    // the warp's piece of the stage: an equal share of the 16-byte vectors, walked row by row
    // (warp-uniform), lanes strided within a row; one warp reduction and one shared-memory
    // add per (warp, row) pair
    const int nvec = d.nel / CP;
    const int per = (nvec + CW - 1) / CW;
    const int v0 = min(nvec, warp * per), v1 = min(nvec, v0 + per);
    int k = 0;
    while (k + 1 < nr && d.soff[k + 1] <= v0 * CP) ++k;
    for (int vs = v0; vs < v1; ++k) {
      const int ve = min(v1, d.soff[k + 1] / CP);
      const int nn = d.n[k], c0 = d.soff[k];
      const V* xb = x + d.xoff[k] - c0;  // element e of the stage is column e - c0 of row k
      V acc[NRHS];
#pragma unroll
      for (int r = 0; r < NRHS; ++r) acc[r] = czero<V>();
      auto use = [&](const L16& a, int e) {
        const int col = e - c0;
        if constexpr (CP == 2) {
#pragma unroll
          for (int r = 0; r < NRHS; ++r) {
            if (col < nn) cfma(acc[r], mk(a.x, a.y), __ldg(xb + r * vstride + e));
            if (col + 1 < nn) cfma(acc[r], mk(a.z, a.w), __ldg(xb + r * vstride + e + 1));
          }
        } else {
#pragma unroll
          for (int r = 0; r < NRHS; ++r)
            if (col < nn) cfma(acc[r], mk(a.x, a.y), __ldg(xb + r * vstride + e));
        }
      };
      int v = vs + lane;
      for (; v + (kTmaU - 1) * 32 < ve; v += 32 * kTmaU) {
        L16 a[kTmaU];
#pragma unroll
        for (int u = 0; u < kTmaU; ++u) a[u] = sb[v + 32 * u];
#pragma unroll
        for (int u = 0; u < kTmaU; ++u) use(a[u], (v + 32 * u) * CP);
      }
      for (; v < ve; v += 32) use(sb[v], v * CP);
#pragma unroll
      for (int r = 0; r < NRHS; ++r) {
        const V t = warp_sum(acc[r]);
        if (lane == 0) sadd(&ps[k * NRHS + r], t);
      }
      vs = ve;
    }
    // the last consumer warp done with this stage writes its rows and clears the partials
    __syncwarp();
    __threadfence_block();
    int last = 0;
    if (lane == 0) last = atomicAdd(&done[s], 1) == CW - 1;
    last = __shfl_sync(0xffffffffu, last, 0);
    if (last) {
      __threadfence_block();
      for (int t = lane; t < nr * NRHS; t += 32) {
        const int rr = t / NRHS, r = t - rr * NRHS;
        const int64_t o = r * vstride + d.r0 + rr;
        const V val = ps[t];
        y[o] = hsub ? csub(hsub[o], val) : val;
        ps[t] = czero<V>();
      }
      if (lane == 0) done[s] = 0;
      __syncwarp();
      __threadfence_block();
    }
    if (lane == 0) mbar_arrive(&empty[s]);
  }
}

template <typename R, int NST>
static void launch_tma(const GemvPlan& p, const typename C2<R>::T* A, const typename C2<R>::T* x,
                       typename C2<R>::T* y, int nr, int64_t vstride, const typename C2<R>::T* hs,
                       cudaStream_t s) {
  typedef typename C2<R>::T V;
#define BEM_TMA(NR)                                                                                \
  do {                                                                                            \
    const TmaSmem L(NST, p.stage_bytes, kTmaMaxRows * NR * (int)sizeof(V));                       \
    k_gemv_tma<R, NR, NST><<<p.ncta, kTmaThreads, L.total, s>>>(p.stages, p.descs, p.cta_stage, A, \
                                                                x, y, vstride, hs, p.stage_bytes,  \
                                                                p.err);                            \
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

// Allow the ring of slots (4 x 40 KB or 3 x 24 KB plus row tables and partials) in dynamic
// shared memory; called at set-up.
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
// complex elements (row storage ld = n rounded up to 4) and kTmaMaxRows rows, each with its row
// table. False when one row does not fit a stage.
bool build_tma_stages(const std::vector<RowInfo>& rows, const std::vector<int2>& segs,
                      const std::vector<int32_t>& cta_seg, int64_t stage_elems,
                      std::vector<TmaStage>* stages, std::vector<int32_t>* cta_stage,
                      std::vector<TmaDesc>* descs) {
  const int ncta = (int)cta_seg.size() - 1;
  stages->clear();
  descs->clear();
  cta_stage->assign(ncta + 1, 0);
  for (int c = 0; c < ncta; ++c) {
    for (int q = cta_seg[c]; q < cta_seg[c + 1]; ++q) {
      int cur = segs[q].x;
      const int end = segs[q].y;
      while (cur < end) {
        const int start = cur;
        TmaDesc d{};
        int64_t el = 0;
        while (cur < end && cur - start < kTmaMaxRows) {
          const int64_t ld = (rows[cur].n + 3) & ~3;
          // rows of one stage must be adjacent in memory (one bulk copy)
          if (el + ld > stage_elems || (cur > start && rows[cur].aoff != rows[start].aoff + el)) break;
          d.soff[cur - start] = (int32_t)el;
          d.n[cur - start] = rows[cur].n;
          d.xoff[cur - start] = rows[cur].xoff;
          el += ld;
          ++cur;
        }
        if (cur == start) return false;
        d.r0 = start;
        d.nr = cur - start;
        d.nel = (int32_t)el;
        d.soff[d.nr] = (int32_t)el;
        TmaStage st;
        st.r0 = start;
        st.r1 = cur;
        st.e0 = rows[start].aoff;
        st.nel = (int32_t)el;
        st.pad = 0;
        stages->push_back(st);
        descs->push_back(d);
      }
    }
    (*cta_stage)[c + 1] = (int32_t)stages->size();
  }
  return true;
}

}  // namespace bem
