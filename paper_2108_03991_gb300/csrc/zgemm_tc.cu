// Many right-hand sides through the internal blocks on the 5th-generation tensor cores: the
// products e_r = Z h_r and h_eq,r = C h_r (C = Y_eq Z, Eqs. MFIEinZin, EFIEeqYZ; block diagonal
// over the objects, Sec. II-C) for r = 1..R in one pass over each block, as the dense complex
// GEMM the internal problem becomes when many port excitations (Sec. IV) share the matrices.
//
// A complex product is one real GEMM. Row m of a block, stored as interleaved (re, im) FP32,
// is a real row of length 2n; right-hand side r contributes two real columns of B,
//   column 2r     = (Re x_0, -Im x_0, Re x_1, -Im x_1, ...)   (gives Re y_r),
//   column 2r + 1 = ( Im x_0,  Re x_0,  Im x_1,  Re x_1, ...)   (gives Im y_r),
// so D = A_real B (M = n, K = 2n, N = 2R) holds y_r as the (re, im) pair of columns 2r, 2r + 1.
//
// FP32 accuracy from TF32 tensor cores by the three-product split: a = a_hi + a_lo with a_hi the
// value with its 13 low mantissa bits cleared (exact in TF32) and a_lo = a - a_hi (exact in
// FP32, 11 significant bits kept by TF32), D = A_hi B_hi + A_hi B_lo + A_lo B_hi; the dropped
// A_lo B_lo and the truncation of the lo parts leave about 2^-20 relative error per product.
//
// Layout. B (both halves) is packed once per call from x into [N][K_tot] with every object's
// K range starting at 2 sum_{j<i} ld_j (a multiple of 8 floats, so every TMA start is 16-byte
// aligned) and zeros in the padding slots. A is read in place through one 2-D tensor map per
// object (inner extent 2n, rows n, row pitch 8 ld bytes): TMA fills the K tail and the rows
// past n with zeros, so a tile that reads past its object's K range in B meets zeros in A.
// Shared-memory tiles are K-major with the 128-byte swizzle, 32 floats of K per row.
//
// One CTA of four warps per 128-row tile of one block (tiles in decreasing block size). Thread
// 0 issues the TMA loads into a ring of stages and the MMAs (M = 128, N = 2R padded to NP, K = 8
// per instruction) into one TMEM accumulator of NP columns; all threads split the stage's A
// tile into hi and lo parts in shared memory while the previous stage's MMAs run. The epilogue
// reads TMEM lane by lane (warp w owns rows 32w..32w+31) and writes y_r coalesced along rows.
// Every wait is bounded: on a timeout the CTA records an error (err[0], kept across products)
// and raises the launch's abort flag (err[1], cleared before each launch), waits (with a short
// limit) for its own MMAs and copies in flight, frees its TMEM and leaves; the other CTAs see
// the flag in their waits, or before they start, and leave too. The results are then invalid.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "bulk.cuh"
#include "common.cuh"

namespace bem {

constexpr int kTcM = 128;       // rows per tile (MMA M, TMEM lanes)
constexpr int kTcK = 32;        // floats of K per stage: one 128-byte swizzle row
constexpr int kTcThreads = 128;
constexpr int kTcMaxRhs = 128;  // N = 2R <= 256 per launch
constexpr uint32_t kTcAtile = kTcM * kTcK * 4;  // 16 KB

struct TcTile {  // one 128-row tile of one block
  int32_t obj, row0;
};
struct TcObj {   // per object: size, first unknown, first K column in the packed B
  int32_t n, xoff;
  int64_t koff;
};

// K-major operand in shared memory with the 128-byte swizzle: rows of 128 bytes, 8-row groups
// 1024 bytes apart (stride byte offset), leading byte offset unused (1), descriptor version 1,
// layout type 2 (128-byte swizzle). The tile base is 1024-byte aligned; the K steps inside the
// 128-byte row advance the start address by 32 bytes.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// instruction descriptor of kind::tf32: D in FP32 (bits 4-5 = 1), A and B TF32 (bits 7-9 and
// 10-12 = 2), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t tf32_idesc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
static_assert(tf32_idesc(128, 256) == 0x08400910u, "instruction descriptor fields");

__device__ __forceinline__ void tma_load_2d(void* dst, const void* tmap, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tc_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
// arrives on the mbarrier once every MMA this thread issued before it has completed
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
// 16 consecutive FP32 columns of this thread's TMEM lane (32x32b shape: lane = thread of the
// warp, from the warp's 32-lane quarter), waited for inside the same statement
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ float tf32_hi(float a) { return __uint_as_float(__float_as_uint(a) & 0xFFFFE000u); }

// Bounded wait on an mbarrier phase that also gives up as soon as any CTA of the launch has
// recorded a failure in *err (polled every 256 tries), so that one stuck CTA does not make
// every later CTA wait out its own limit.
constexpr uint32_t kTcSpin = 1u << 22;
constexpr uint32_t kTcSpinCleanup = 1u << 16;
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity, const int* err, uint32_t spins) {
  for (uint32_t it = 0; it < spins; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 255) == 255 && *(const volatile int*)err) return false;
  }
  return false;
}

// B from x, hi and lo parts (or, with bl null, the raw FP32 values into bh): rows 2r and 2r + 1
// for right-hand side r < R (zero rows up to NP), columns 2u and 2u + 1 for padded slot u
// (slot[u] = its unknown, -1 in a block's padding). Grid: x over the slots, y over the NP / 2
// row pairs.
__global__ void k_tc_pack(const float2* __restrict__ x, int64_t vstride, int R,
                          const int32_t* __restrict__ slot, int64_t nslot, float* __restrict__ bh,
                          float* __restrict__ bl) {
  const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (u >= nslot) return;
  const int j = slot[u];
  float2 v = make_float2(0.f, 0.f);
  if (r < R && j >= 0) v = x[r * vstride + j];
  const int64_t ktot = 2 * nslot;
  const float2 re = make_float2(v.x, -v.y), im = make_float2(v.y, v.x);
  const float2 reh = make_float2(tf32_hi(re.x), tf32_hi(re.y)), imh = make_float2(tf32_hi(im.x), tf32_hi(im.y));
  const int64_t o0 = (2 * r) * ktot + 2 * u, o1 = o0 + ktot;
  if (!bl) {  // the raw values: the product splits them in shared memory
    *reinterpret_cast<float2*>(bh + o0) = re;
    *reinterpret_cast<float2*>(bh + o1) = im;
    return;
  }
  *reinterpret_cast<float2*>(bh + o0) = reh;
  *reinterpret_cast<float2*>(bh + o1) = imh;
  *reinterpret_cast<float2*>(bl + o0) = make_float2(re.x - reh.x, re.y - reh.y);
  *reinterpret_cast<float2*>(bl + o1) = make_float2(im.x - imh.x, im.y - imh.y);
}

// shared memory of one CTA: S stages of [A (hi after the split) | A lo | B hi | B lo], each tile
// 1024-byte aligned, then the full/empty barriers of the stages, the done barrier, the TMEM slot
template <int NP, int S> struct TcSmem {
  static constexpr uint32_t kBtile = NP * kTcK * 4;
  static constexpr uint32_t kStage = 2 * kTcAtile + 2 * kBtile;
  static constexpr uint32_t kBars = S * kStage;
  static constexpr uint32_t kBytes = kBars + 8 * (2 * S + 1) + 8 + 1024;  // + alignment slack
};

// BS = 0: B's hi and lo parts arrive packed (two TMA loads a stage); BS = 1: the raw B arrives
// (one load) and is split in shared memory like A
template <int NP, int S, int BS = 0>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_zgemm_tc(const __grid_constant__ CUtensorMap mbh, const __grid_constant__ CUtensorMap mbl,
               const CUtensorMap* __restrict__ ma, const TcTile* __restrict__ tiles,
               const TcObj* __restrict__ objs, float2* __restrict__ y, int64_t vstride, int R,
               int* err) {
  typedef TcSmem<NP, S> L;
  constexpr uint32_t kTx = kTcAtile + (BS ? 1 : 2) * L::kBtile;  // bytes landing per stage
  constexpr uint32_t kIdesc = tf32_idesc(kTcM, NP);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + L::kBars);
  uint64_t* empty = full + S;
  uint64_t* done = empty + S;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const TcTile t = tiles[blockIdx.x];
  const TcObj o = objs[t.obj];
  const CUtensorMap* mA = ma + t.obj;
  const int nk = (2 * o.n + kTcK - 1) / kTcK;
  int* const abort_flag = err + 1;  // set by any CTA of this launch that gave up

  // a CTA that starts after another one gave up leaves at once (one decision for the block)
  __shared__ int s_skip;
  if (tid == 0) s_skip = *(const volatile int*)abort_flag;
  __syncthreads();
  if (s_skip) return;

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tc_alloc(tslot, NP);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  // thread 0's bookkeeping: chunks 0..issued-1 have their loads issued; no load after a failed wait
  int issued = 0;
  bool stalled = false;
  auto load = [&](int kc) {
    const int s = kc % S;
    uint8_t* st = base + s * L::kStage;
    const int kx = (int)(o.koff + (int64_t)kc * kTcK);
    mbar_arrive_tx(&full[s], kTx);
    tma_load_2d(st, mA, kc * kTcK, t.row0, &full[s]);
    tma_load_2d(st + 2 * kTcAtile, &mbh, kx, 0, &full[s]);
    if constexpr (BS == 0) tma_load_2d(st + 2 * kTcAtile + L::kBtile, &mbl, kx, 0, &full[s]);
    issued = kc + 1;
  };
  if (tid == 0) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(mA)) : "memory");
    for (int kc = 0; kc < nk && kc < S; ++kc) load(kc);
  }

  int kc_fail = -1;  // block-uniform: the chunk whose wait timed out for some thread
  for (int kc = 0; kc < nk; ++kc) {
    const int s = kc % S;
    const bool ok = tc_wait(&full[s], (kc / S) & 1, abort_flag, kTcSpin);
    if (ok) {  // split the A tile: hi in place, lo beside it (same offsets, same swizzle)
      float4* a = reinterpret_cast<float4*>(base + s * L::kStage);
      float4* al = reinterpret_cast<float4*>(base + s * L::kStage + kTcAtile);
#pragma unroll 4
      for (int i = tid; i < (int)(kTcAtile / 16); i += kTcThreads) {
        const float4 v = a[i];
        const float4 h = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
        a[i] = h;
        al[i] = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
      }
      if constexpr (BS == 1) {  // the same split of the raw B tile
        float4* b = reinterpret_cast<float4*>(base + s * L::kStage + 2 * kTcAtile);
        float4* bl = reinterpret_cast<float4*>(base + s * L::kStage + 2 * kTcAtile + L::kBtile);
#pragma unroll 4
        for (int i = tid; i < (int)(L::kBtile / 16); i += kTcThreads) {
          const float4 v = b[i];
          const float4 h = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
          b[i] = h;
          bl[i] = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (__syncthreads_or(!ok)) {
      kc_fail = kc;
      break;
    }
    if (tid == 0) {
      tc_fence_after();
      const uint32_t sa = smem_u32(base + s * L::kStage);
      const uint32_t sb = sa + 2 * kTcAtile;
#pragma unroll
      for (int k = 0; k < kTcK / 8; ++k) {  // 8 TF32 = 32 bytes of K per instruction
        const uint64_t ah = sw128_desc(sa + 32 * k), alo = sw128_desc(sa + kTcAtile + 32 * k);
        const uint64_t bh = sw128_desc(sb + 32 * k), blo = sw128_desc(sb + L::kBtile + 32 * k);
        tc_mma_tf32(tmem, alo, bh, kIdesc, (kc > 0 || k > 0) ? 1u : 0u);
        tc_mma_tf32(tmem, ah, blo, kIdesc, 1u);
        tc_mma_tf32(tmem, ah, bh, kIdesc, 1u);
      }
      tc_commit(&empty[s]);
      // the previous chunk's stage takes chunk kc - 1 + S once that chunk's MMAs are done
      const int nxt = kc - 1 + S;
      if (kc >= 1 && nxt < nk && !stalled) {
        if (tc_wait(&empty[(kc - 1) % S], ((kc - 1) / S) & 1, abort_flag, kTcSpin)) load(nxt);
        else stalled = true;  // the loop's next wait on chunk nxt times out for every thread
      }
    }
  }

  bool ok = kc_fail < 0;
  if (ok) {
    if (tid == 0) tc_commit(done);
    ok = !__syncthreads_or(!tc_wait(done, 0, abort_flag, kTcSpin));
    if (!ok) kc_fail = nk;
  }
  if (!ok) {  // leave cleanly: error code, MMAs and copies in flight waited for (bounded)
    if (tid == 0) {
      atomicExch(err, 1);
      atomicExch(abort_flag, 1);
      if (kc_fail < nk) tc_commit(done);
      const int none = 0;  // the cleanup waits run their own short limit to the end
      tc_wait(done, 0, &none, kTcSpinCleanup);
      for (int c = max(kc_fail, 0); c < issued; ++c) tc_wait(&full[c % S], (c / S) & 1, &none, kTcSpinCleanup);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tc_dealloc(tmem, NP);
    return;
  }

  tc_fence_after();
  const int row = t.row0 + warp * 32 + lane;
  const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
  for (int c0 = 0; c0 < 2 * R && c0 < NP; c0 += 16) {
    float v[16];
    tc_ld16(tl + c0, v);
    if (row < o.n) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int r = c0 / 2 + q;
        if (r < R) y[r * vstride + o.xoff + row] = make_float2(v[2 * q], v[2 * q + 1]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tc_dealloc(tmem, NP);
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
typedef PFN_cuTensorMapEncodeTiled_v12000 TcEncode;

struct TcState {
  CUtensorMap* mz = nullptr;  // per object, over the FP32 Z and C blocks (device)
  CUtensorMap* mc = nullptr;
  TcTile* tiles = nullptr;
  int ntiles = 0;
  TcObj* objs = nullptr;
  int32_t* slot = nullptr;    // [nslot] unknown of each padded slot, -1 in padding
  int64_t nslot = 0;          // sum of ld_i
  float *bh = nullptr, *bl = nullptr;  // packed B, [np_cap][2 nslot] each
  int np_cap = 0;
  int* err = nullptr;         // [2]: a wait timed out in some product (sticky); this launch gave up
  int64_t calls = 0;
  ~TcState() {
    for (void* p : {(void*)mz, (void*)mc, (void*)tiles, (void*)objs, (void*)slot, (void*)bh,
                    (void*)bl, (void*)err})
      if (p) cudaFree(p);
  }
};

static TcEncode tc_encoder() {
  static TcEncode fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<TcEncode>(p);
  }
  return fn;
}

// 2-D FP32 tensor map, inner extent `inner` floats, `rows` rows `pitch` bytes apart, box of
// 32 floats x box_rows, 128-byte swizzle, zero fill outside
static int tc_map(TcEncode enc, CUtensorMap* m, const void* base, int64_t inner, int64_t rows,
                  int64_t pitch, int box_rows) {
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)pitch};
  const cuuint32_t box[2] = {(cuuint32_t)kTcK, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  if ((reinterpret_cast<uintptr_t>(base) & 15) || (pitch & 15)) {
    set_error("tensor-core product: operand not 16-byte aligned");
    return BEM_EINVAL;
  }
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides,
                         box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("tensor-core product: cuTensorMapEncodeTiled failed (%d)", (int)r);
    return BEM_ECUDA;
  }
  return BEM_OK;
}

// tiles, object table, slot table and the per-object tensor maps of Z and C (first use)
static int tc_prepare(aim_ctx* c, TcState** out) {
  if (c->tc) {
    *out = static_cast<TcState*>(c->tc);
    return BEM_OK;
  }
  TcEncode enc = tc_encoder();
  if (!enc) {
    set_error("tensor-core product: cuTensorMapEncodeTiled is not available from the driver");
    return BEM_ECUDA;
  }
  if (!c->f32.Z || !c->f32.C) {
    set_error("tensor-core product: no FP32 internal blocks");
    return BEM_EINVAL;
  }
  TcState* t = new TcState();
  std::vector<TcObj> objs(c->nobj);
  std::vector<TcTile> tiles;
  std::vector<int32_t> slot;
  std::vector<CUtensorMap> mz(c->nobj), mc(c->nobj);
  int rc = BEM_OK;
  for (int i = 0, xo = 0; i < c->nobj && rc == BEM_OK; ++i) {
    const int n = c->e1[i] - c->e0[i], ld = c->zld[i];
    objs[i] = TcObj{n, xo, 2 * (int64_t)slot.size()};
    for (int l = 0; l < ld; ++l) slot.push_back(l < n ? xo + l : -1);
    for (int r0 = 0; r0 < n; r0 += kTcM) tiles.push_back(TcTile{i, r0});
    rc = tc_map(enc, &mz[i], c->f32.Z + c->zoff[i], 2 * (int64_t)n, n, 8 * (int64_t)ld, kTcM);
    if (rc == BEM_OK) rc = tc_map(enc, &mc[i], c->f32.C + c->zoff[i], 2 * (int64_t)n, n, 8 * (int64_t)ld, kTcM);
    xo += n;
  }
  if (rc == BEM_OK && 2 * (int64_t)slot.size() > INT32_MAX) {
    set_error("tensor-core product: more than 2^30 unknowns");
    rc = BEM_EINVAL;
  }
  // largest blocks first: their tiles carry the longest K loops
  std::stable_sort(tiles.begin(), tiles.end(), [&](const TcTile& a, const TcTile& b) {
    return objs[a.obj].n > objs[b.obj].n;
  });
  t->ntiles = (int)tiles.size();
  t->nslot = (int64_t)slot.size();
  auto up = [&](void** p, const void* h, size_t bytes) {
    if (rc != BEM_OK) return;
    if (cudaMalloc(p, bytes) != cudaSuccess || cudaMemcpy(*p, h, bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
      set_error("tensor-core product: device allocation failed");
      rc = BEM_ENOMEM;
    }
  };
  up((void**)&t->mz, mz.data(), mz.size() * sizeof(CUtensorMap));
  up((void**)&t->mc, mc.data(), mc.size() * sizeof(CUtensorMap));
  up((void**)&t->tiles, tiles.data(), tiles.size() * sizeof(TcTile));
  up((void**)&t->objs, objs.data(), objs.size() * sizeof(TcObj));
  up((void**)&t->slot, slot.data(), slot.size() * sizeof(int32_t));
  const int zero[2] = {0, 0};  // [0]: a wait timed out in some product; [1]: this launch gave up
  up((void**)&t->err, zero, sizeof(zero));
  if (rc != BEM_OK) {
    delete t;
    return rc;
  }
  c->tc = t;
  *out = t;
  return BEM_OK;
}

template <int NP, int S, int BS>
static int tc_launch(TcState* t, const CUtensorMap& mbh, const CUtensorMap& mbl, const CUtensorMap* ma,
                     float2* y, int64_t vstride, int R, cudaStream_t s) {
  constexpr uint32_t kSmem = TcSmem<NP, S>::kBytes;
  static_assert(kSmem <= 227 * 1024, "shared memory per CTA");
  // per call: the attribute belongs to the current device (cheap next to the product)
  BEM_CUDA(cudaFuncSetAttribute(k_zgemm_tc<NP, S, BS>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem));
  BEM_CUDA(cudaMemsetAsync(t->err + 1, 0, sizeof(int), s));
  k_zgemm_tc<NP, S, BS><<<t->ntiles, kTcThreads, kSmem, s>>>(mbh, mbl, ma, t->tiles, t->objs, y, vstride,
                                                            R, t->err);
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

// e_r = Z h_r and h_eq,r = C h_r for r < nrhs (FP32, vectors ne apart); either output may be null
int internal_tc(aim_ctx* c, const float2* h, float2* e, float2* heq, int nrhs, cudaStream_t s) {
  TcState* t = nullptr;
  BEM_TRY(tc_prepare(c, &t));
  if (t->ntiles == 0) return BEM_OK;
  TcEncode enc = tc_encoder();
  const int64_t ne = c->ne;
  for (int r0 = 0; r0 < nrhs; r0 += kTcMaxRhs) {
    const int R = std::min(kTcMaxRhs, nrhs - r0);
    const int NP = R <= 16 ? 32 : R <= 32 ? 64 : R <= 64 ? 128 : 256;
    if (NP > t->np_cap) {
      BEM_CUDA(cudaStreamSynchronize(s));  // the old workspace may be in use on s
      if (t->bh) cudaFree(t->bh);
      if (t->bl) cudaFree(t->bl);
      t->bh = t->bl = nullptr;
      t->np_cap = 0;
      const size_t bytes = (size_t)NP * 2 * t->nslot * sizeof(float);
      if (cudaMalloc((void**)&t->bh, bytes) != cudaSuccess || cudaMalloc((void**)&t->bl, bytes) != cudaSuccess) {
        set_error("tensor-core product: no device memory for the packed right-hand sides");
        return BEM_ENOMEM;
      }
      t->np_cap = NP;
    }
    // form 1 packs the raw values only (B split in shared memory); the second map is then unused
    const bool raw = c->tc_variant == 1;
    CUtensorMap mbh, mbl;
    BEM_TRY(tc_map(enc, &mbh, t->bh, 2 * t->nslot, NP, 2 * t->nslot * (int64_t)sizeof(float), NP));
    BEM_TRY(tc_map(enc, &mbl, t->bl, 2 * t->nslot, NP, 2 * t->nslot * (int64_t)sizeof(float), NP));
    const dim3 pg((unsigned)((t->nslot + 255) / 256), NP / 2);
    k_tc_pack<<<pg, 256, 0, s>>>(h + r0 * ne, ne, R, t->slot, t->nslot, t->bh, raw ? nullptr : t->bl);
    BEM_CUDA(cudaGetLastError());
    for (int w = 0; w < 2; ++w) {
      float2* y = w == 0 ? e : heq;
      if (!y) continue;
      const CUtensorMap* ma = w == 0 ? t->mz : t->mc;
      y += r0 * ne;
#define BEM_TC(NPV, SV)                                                               \
  BEM_TRY(raw ? (tc_launch<NPV, SV, 1>(t, mbh, mbl, ma, y, ne, R, s))                 \
              : (tc_launch<NPV, SV, 0>(t, mbh, mbl, ma, y, ne, R, s)))
      switch (NP) {
        case 32: BEM_TC(32, 5); break;
        case 64: BEM_TC(64, 4); break;
        case 128: BEM_TC(128, 3); break;
        default: BEM_TC(256, 2); break;
      }
#undef BEM_TC
    }
  }
  ++t->calls;
  return BEM_OK;
}

void free_tc(aim_ctx* c) {
  delete static_cast<TcState*>(c->tc);
  c->tc = nullptr;
}

// products made, a wait timed out (1) or not (0); -1 when the product was never used
void tc_stats(const aim_ctx* c, int64_t* out) {
  const TcState* t = static_cast<const TcState*>(c->tc);
  out[0] = t ? t->calls : 0;
  out[1] = -1;
  int v = 0;
  if (t && cudaMemcpy(&v, t->err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess) out[1] = v;
}

}  // namespace bem
