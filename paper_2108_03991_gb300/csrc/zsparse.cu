// Sparse internal operators at high frequency (Sec. III-A, third item of the internal problem).
// When the skin depth delta_i = -1/Im k_i is small against an object, L_{k_i} and K_{k_i}
// couple each basis function only to its near neighbours: they are treated as sparse, the pairs
// whose RWG supports lie farther apart than R_cut = 23 delta_i dropped (e^{-23} ~ 1e-10; the
// support distance is bounded from below by the centroid distance less the two triangles'
// centroid-to-vertex radii, nearest of the 2 x 2 triangle pairs), and
//   e = Z_s h = -(1 / (j k0 eps_rc)) L_s^{-1} (K_s + I_x/2) h
// replaces the dense e = Z h of Eq. MFIEinZin. The paper applies L_s^{-1} with a sparse direct
// solver; here the kept pattern of each object is reordered by reverse Cuthill-McKee (host), so
// that L_s becomes a band of half-width b, factorised without pivoting in FP64 (one CTA per
// object), and each product is the sparse rows of K_s + I_x/2 (all objects in one launch) and
// then one warp per object for a forward and a back substitution, blocked by kZspBW columns
// (each column of L and of U stored contiguously, a block's columns streamed into shared memory
// by one bulk copy while the warp works on the previous block). C = Y_eq Z stays dense, so j = h - C h is unchanged and e = Z_s h, needed only by the
// I_x e term of the system matvec, runs beside it. The sparse form is used when every object
// qualifies (band and rows below half the dense bytes, b <= 256) and a set-up check of Z_s h
// against the dense Z h (FP64, one probe vector) stays below 1e-8.
#include <algorithm>
#include <cmath>
#include <complex>
#include <memory>
#include <vector>

#include "bulk.cuh"
#include "common.cuh"

namespace bem {

constexpr double kZspCut = 23.0;     // R_cut / delta
constexpr int kZspBandMax = 192;     // largest half-bandwidth of the product kernel
constexpr size_t kZspSmemMax = 220 * 1024;  // its shared memory (FP64: vector and two slabs)
constexpr int kZspRows = (kZspBandMax + 31) / 32;  // rows per lane in a block's update
// columns per block of the substitutions (slab: kZspBW b entries). 8: a warp's shared memory
// (the vector and two slabs) is 22 KB at b = 114, so all the objects' warps are resident at once;
// 16 and 32 took 30% and 70% longer per product on the 32 x 32 ring array
constexpr int kZspBW = 8;
constexpr double kZspCheck = 1e-8;   // set-up check of Z_s h against Z h
constexpr double kTwoPi = 6.283185307179586476925;

struct ZspObj {
  int e0, n, b, pad;
  int64_t loff;   // offset of the object's n x b column tables of L and U
  int64_t woff;   // offset of its FP64 band (set-up only), n x (2b + 1)
  double ar, ai;  // alpha = -1 / (j k0 eps_rc)
};

struct Zsp {
  std::vector<ZspObj> obj;
  ZspObj* d_obj = nullptr;
  int32_t *d_perm = nullptr, *d_pos = nullptr;  // row e0 + r <-> edge e0 + perm[r], both global
  int32_t *d_row = nullptr, *d_col = nullptr;   // K_s + I_x/2 in permuted row order (CSR)
  int64_t nnz = 0, nband = 0, nwork = 0;
  int bmax = 0, nmax = 0;
  double2* W = nullptr;                          // FP64 bands during set-up
  double2 *kv64 = nullptr, *L64 = nullptr, *U64 = nullptr, *D64 = nullptr;
  float2 *kv32 = nullptr, *L32 = nullptr, *U32 = nullptr, *D32 = nullptr;
  int* d_fail = nullptr;
  int* d_err = nullptr;    // set by a product whose bounded wait timed out
  float2* v32 = nullptr;   // [kMaxBatch][ne] rows of K_s + I_x/2 h, permuted (product scratch)
  double2* v64 = nullptr;
  double check = -1;  // max over objects of |Z_s h - Z h| / |Z h| at set-up
  ~Zsp() {
    if (W) cudaFree(W);
  }
};

// ---------------------------------------------------------------------------------------
// set-up kernels
// ---------------------------------------------------------------------------------------
__global__ void k_tri_radius(const double* verts, const int32_t* tris, const double* cen, int nt,
                             double* rad) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  double r = 0;
  for (int a = 0; a < 3; ++a) {
    const double* v = &verts[3 * tris[3 * t + a]];
    const double dx = v[0] - cen[3 * t], dy = v[1] - cen[3 * t + 1], dz = v[2] - cen[3 * t + 2];
    r = fmax(r, sqrt(dx * dx + dy * dy + dz * dz));
  }
  rad[t] = r;
}

// mask[m n + k] = 1 iff the supports of edges e0 + m and e0 + k come within rcut
__global__ void k_zsp_mask(const double* cen, const double* rad, const int32_t* et, int e0, int n,
                           double rcut, uint8_t* mask) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  const int m = e0 + (int)(idx / n), k = e0 + (int)(idx % n);
  double d = 1e300;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      const int t = et[2 * m + a], s = et[2 * k + b];
      const double dx = cen[3 * t] - cen[3 * s], dy = cen[3 * t + 1] - cen[3 * s + 1],
                   dz = cen[3 * t + 2] - cen[3 * s + 2];
      d = fmin(d, fmax(0.0, sqrt(dx * dx + dy * dy + dz * dz) - rad[t] - rad[s]));
    }
  mask[idx] = d <= rcut ? 1 : 0;
}

// the kept entries of L (band of the permuted matrix) and of B = K + I_x/2 (CSR values), from
// the object's dense column-major n x n matrices; one thread per permuted row
__global__ void k_zsp_gather(ZspObj o, const double2* L, const double2* B, const int32_t* perm,
                             const int32_t* pos, const int32_t* row, const int32_t* col,
                             double2* W, double2* kv) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= o.n) return;
  const int w = 2 * o.b + 1;
  const int node = perm[o.e0 + r] - o.e0;
  for (int k = row[o.e0 + r]; k < row[o.e0 + r + 1]; ++k) {
    const int cl = col[k] - o.e0;
    const int64_t src = node + (int64_t)cl * o.n;
    kv[k] = B[src];
    const int j = pos[col[k]] - o.e0;
    W[o.woff + (int64_t)r * w + (j - r + o.b)] = L[src];
  }
}

// LU without pivoting of each object's band (one CTA per object, in place, FP64): W[i][j - i + b]
// holds A_ij; afterwards the strict lower band holds L (unit diagonal) and the rest U.
__global__ void __launch_bounds__(256) k_zsp_lu(const ZspObj* objs, double2* Wall, int* fail) {
  const ZspObj o = objs[blockIdx.x];
  const int n = o.n, b = o.b, w = 2 * b + 1;
  double2* W = Wall + o.woff;
  __shared__ double2 lcol[kZspBandMax], urow[kZspBandMax];
  __shared__ double red[256];
  // scale: the largest diagonal magnitude
  double mx = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double2 d = W[(int64_t)i * w + b];
    mx = fmax(mx, sqrt(d.x * d.x + d.y * d.y));
  }
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  const double tiny = 1e-13 * red[0];
  for (int k = 0; k < n; ++k) {
    const int m = min(b, n - 1 - k);  // rows (and columns) below (right of) the pivot in the band
    double2 p = W[(int64_t)k * w + b];
    const double pm = p.x * p.x + p.y * p.y;
    if (!(sqrt(pm) > tiny)) {
      if (threadIdx.x == 0) atomicExch(&fail[blockIdx.x], 1);
      p = make_double2(red[0], 0.0);
    }
    const double den = p.x * p.x + p.y * p.y;
    const double2 ip = make_double2(p.x / den, -p.y / den);
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
      double2* a = &W[(int64_t)(k + 1 + t) * w + (b - 1 - t)];  // A[k+1+t][k]
      const double2 l = cmul(*a, ip);
      *a = l;
      lcol[t] = l;
      urow[t] = W[(int64_t)k * w + (b + 1 + t)];  // A[k][k+1+t]
    }
    __syncthreads();
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
      const int i = t / m, j = t % m;  // row k+1+i, column k+1+j
      double2* a = &W[(int64_t)(k + 1 + i) * w + (j - i + b)];
      const double2 u = cmul(lcol[i], urow[j]);
      a->x -= u.x;
      a->y -= u.y;
    }
    __syncthreads();
  }
}

// column tables for the substitutions: Lc[c][k] = L[c+1+k][c], Uc[c][k] = U[c-1-k][c] (zero
// outside the matrix), D[c] = 1 / U[c][c]; FP64 and FP32 copies
__global__ void k_zsp_extract(const ZspObj* objs, const double2* Wall, double2* L64, double2* U64,
                              double2* D64, float2* L32, float2* U32, float2* D32) {
  const ZspObj o = objs[blockIdx.y];
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int n = o.n, b = o.b, w = 2 * b + 1;
  if (idx >= (int64_t)n * b) return;
  const int c = (int)(idx / b), k = (int)(idx % b);
  const double2* W = Wall + o.woff;
  double2 l = make_double2(0, 0), u = make_double2(0, 0);
  if (c + 1 + k < n) l = W[(int64_t)(c + 1 + k) * w + (b - 1 - k)];
  if (c - 1 - k >= 0) u = W[(int64_t)(c - 1 - k) * w + (b + 1 + k)];
  L64[o.loff + idx] = l;
  U64[o.loff + idx] = u;
  L32[o.loff + idx] = make_float2((float)l.x, (float)l.y);
  U32[o.loff + idx] = make_float2((float)u.x, (float)u.y);
  if (k == 0) {
    const double2 d = W[(int64_t)c * w + b];
    const double den = d.x * d.x + d.y * d.y;
    const double2 id = make_double2(d.x / den, -d.y / den);
    D64[o.e0 + c] = id;
    D32[o.e0 + c] = make_float2((float)id.x, (float)id.y);
  }
}

__global__ void k_round_kv(const double2* a, float2* b, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

// ---------------------------------------------------------------------------------------
// the product e = Z_s h in two launches: the rows of K_s + I_x/2 (all objects' rows in one
// launch, eight lanes per row), then the substitutions (one warp per object and right-hand
// side), blocked by kZspBW columns: the warp solves a block's triangle in registers (shuffles,
// the triangle's entries read up front) and then applies the block's solved values to the b
// rows below (above, going back) it as a small dense product, every lane on several rows at
// once, instead of walking the band one column at a time.
// ---------------------------------------------------------------------------------------
template <typename V> __device__ __forceinline__ V vzero() { V v; v.x = 0; v.y = 0; return v; }
template <typename V> __device__ __forceinline__ V vmul(V a, V b) {
  V r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename V> __device__ __forceinline__ void vfma(V a, V b, V& acc) {
  acc.x += a.x * b.x - a.y * b.y;
  acc.y += a.x * b.y + a.y * b.x;
}
template <typename V> __device__ __forceinline__ V vshfl(V a, int src) {
  V r;
  r.x = __shfl_sync(0xffffffffu, a.x, src);
  r.y = __shfl_sync(0xffffffffu, a.y, src);
  return r;
}

// v[r] (permuted row r of every object, stride vs per right-hand side) = ((K_s + I_x/2) h)[perm r]
template <typename R>
__global__ void __launch_bounds__(256) k_zsp_rows(const int32_t* __restrict__ row,
                                                  const int32_t* __restrict__ col,
                                                  const typename C2<R>::T* __restrict__ kv,
                                                  const typename C2<R>::T* __restrict__ x, int64_t xs,
                                                  typename C2<R>::T* __restrict__ v, int64_t vs,
                                                  int ne) {
  typedef typename C2<R>::T V;
  const int r = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 3);
  const int sub = threadIdx.x & 7;
  const V* h = x + blockIdx.y * xs;
  V acc = vzero<V>();
  if (r < ne)
    for (int k = row[r] + sub; k < row[r + 1]; k += 8) vfma(kv[k], h[col[k]], acc);
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  if (r < ne && sub == 0) v[blockIdx.y * vs + r] = acc;
}

// one warp per (object, right-hand side): the band's slabs of kZspBW columns (of L forward, of U
// going back) are streamed into two shared-memory slots by bulk copies, the next slab in flight
// while the warp works on the current one; every wait is bounded and a timeout sets *err
template <typename R>
__global__ void __launch_bounds__(32) k_zsp_solve(const ZspObj* __restrict__ objs,
                                                  const int32_t* __restrict__ perm,
                                                  const typename C2<R>::T* __restrict__ Lc,
                                                  const typename C2<R>::T* __restrict__ Uc,
                                                  const typename C2<R>::T* __restrict__ D,
                                                  const typename C2<R>::T* __restrict__ vin,
                                                  int64_t vs, typename C2<R>::T* __restrict__ y,
                                                  int64_t ys, int vbytes, int slab_bytes, int* err) {
  typedef typename C2<R>::T V;
  extern __shared__ __align__(16) unsigned char zsp_smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(zsp_smem);
  V* v = reinterpret_cast<V*>(zsp_smem + 16);
  unsigned char* slabs = zsp_smem + 16 + vbytes;  // two slots of slab_bytes
  const ZspObj o = objs[blockIdx.x];
  const int l = threadIdx.x;
  const int n = o.n, b = o.b, e0 = o.e0;
  const V* Lo = Lc + o.loff;
  const V* Uo = Uc + o.loff;
  const int nblk = (n + kZspBW - 1) / kZspBW, nslab = 2 * nblk;
  // slab s: L's columns of block s (forward), then U's of block 2 nblk - 1 - s (going back)
  auto issue = [&](int s) {
    if (l == 0 && s < nslab) {
      const int kb = s < nblk ? s : nslab - 1 - s;
      const int c0 = kZspBW * kb, nb = min(kZspBW, n - c0);
      const uint32_t bytes = (uint32_t)(((size_t)nb * b * sizeof(V) + 15) & ~(size_t)15);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier reads of the slot
      mbar_arrive_tx(&bar[s & 1], bytes);
      bulk_g2s(slabs + (s & 1) * slab_bytes, (s < nblk ? Lo : Uo) + (int64_t)c0 * b, bytes, &bar[s & 1]);
    }
  };
  if (l == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  issue(0);
  const V* vi = vin + blockIdx.y * vs + e0;
  V* e = y + blockIdx.y * ys;
  for (int r = l; r < n; r += 32) v[r] = vi[r];
  __syncwarp();
  V al;
  al.x = (R)o.ar;
  al.y = (R)o.ai;
  for (int s = 0; s < nslab; ++s) {
    issue(s + 1);
    if (!mbar_wait(&bar[s & 1], (s >> 1) & 1)) {
      if (l == 0) atomicExch(err, 1);
      if (s + 1 < nslab) mbar_wait(&bar[(s + 1) & 1], ((s + 1) >> 1) & 1);  // the copy in flight
      return;
    }
    const V* S = reinterpret_cast<const V*>(slabs + (s & 1) * slab_bytes);  // S[t b + k]: column c0 + t, entry k
    if (s < nblk) {
      // forward substitution with the unit lower band, block s
      const int c0 = kZspBW * s, nb = min(kZspBW, n - c0);
      V tri[kZspBW - 1];
#pragma unroll
      for (int t = 0; t < kZspBW - 1; ++t) {  // L[c0+l][c0+t] for t < l
        const int k = l - t - 1;
        tri[t] = (k >= 0 && k < b && l < nb) ? S[t * b + k] : vzero<V>();
      }
      V yl = l < nb ? v[c0 + l] : vzero<V>();
#pragma unroll
      for (int t = 0; t < kZspBW - 1; ++t) {
        if (t < nb) {
          const V u = vmul(tri[t], vshfl(yl, t));
          yl.x -= u.x;
          yl.y -= u.y;
        }
      }
      if (l < nb) v[c0 + l] = yl;
      // the block's solved values on the b rows below it: lane l takes rows c0 + nb + l + 32 r,
      // all of them at once (independent sums, each x_t broadcast once)
      const int rend = min(n, c0 + nb + b);
      V acc[kZspRows];
#pragma unroll
      for (int r = 0; r < kZspRows; ++r) acc[r] = vzero<V>();
      for (int t = 0; t < nb; ++t) {
        const V xt = vshfl(yl, t);
#pragma unroll
        for (int r = 0; r < kZspRows; ++r) {
          const int i = c0 + nb + l + 32 * r, k = nb + l + 32 * r - t - 1;
          if (i < rend && k < b) vfma(S[t * b + k], xt, acc[r]);
        }
      }
#pragma unroll
      for (int r = 0; r < kZspRows; ++r) {
        const int i = c0 + nb + l + 32 * r;
        if (i < rend) {
          v[i].x -= acc[r].x;
          v[i].y -= acc[r].y;
        }
      }
    } else {
      // back substitution with U, block 2 nblk - 1 - s; x goes out as e = alpha x (unpermuted)
      const int c0 = kZspBW * (nslab - 1 - s), nb = min(kZspBW, n - c0);
      V tri[kZspBW];
#pragma unroll
      for (int t = 0; t < kZspBW; ++t) {  // U[c0+l][c0+t] for t > l
        const int k = t - l - 1;
        tri[t] = (k >= 0 && k < b && t < nb) ? S[t * b + k] : vzero<V>();
      }
      const V dl = l < nb ? D[e0 + c0 + l] : vzero<V>();
      V yl = l < nb ? v[c0 + l] : vzero<V>();
#pragma unroll
      for (int t = kZspBW - 1; t >= 0; --t) {
        if (t < nb) {
          const V w = vmul(tri[t], vshfl(vmul(yl, dl), t));  // x_t = y_t / U_tt, final here
          yl.x -= w.x;
          yl.y -= w.y;
        }
      }
      const V xl = vmul(yl, dl);
      if (l < nb) {
        v[c0 + l] = xl;
        e[perm[e0 + c0 + l]] = vmul(al, xl);
      }
      // on the b rows above the block: lane l takes rows c0 - 1 - l - 32 r
      const int rlo = max(0, c0 - b);
      V acc[kZspRows];
#pragma unroll
      for (int r = 0; r < kZspRows; ++r) acc[r] = vzero<V>();
      for (int t = 0; t < nb; ++t) {
        const V xt = vshfl(xl, t);
#pragma unroll
        for (int r = 0; r < kZspRows; ++r) {
          const int i = c0 - 1 - l - 32 * r, k = t + l + 32 * r;
          if (i >= rlo && k < b) vfma(S[t * b + k], xt, acc[r]);
        }
      }
#pragma unroll
      for (int r = 0; r < kZspRows; ++r) {
        const int i = c0 - 1 - l - 32 * r;
        if (i >= rlo) {
          v[i].x -= acc[r].x;
          v[i].y -= acc[r].y;
        }
      }
    }
    __syncwarp();
  }
}

template <typename R>
int zsp_apply(aim_ctx* c, const typename C2<R>::T* h, typename C2<R>::T* e, int nrhs, int64_t hs,
              int64_t es, cudaStream_t s) {
  typedef typename C2<R>::T V;
  Zsp* z = static_cast<Zsp*>(c->zsp);
  if (!z || !c->zsp_ready) {
    set_error("sparse internal operator not built");
    return BEM_EINVAL;
  }
  if (nrhs < 1 || nrhs > kMaxBatch) {
    set_error("sparse internal operator: 1 <= nrhs <= %d", kMaxBatch);
    return BEM_EINVAL;
  }
  const bool f = sizeof(R) == 4;
  V* v = f ? (V*)z->v32 : (V*)z->v64;
  const int ne = c->ne;
  k_zsp_rows<R><<<dim3((unsigned)(((int64_t)ne * 8 + 255) / 256), nrhs), 256, 0, s>>>(
      z->d_row, z->d_col, f ? (const V*)z->kv32 : (const V*)z->kv64, h, hs, v, ne, ne);
  const int vbytes = (int)(((size_t)z->nmax * sizeof(V) + 15) & ~(size_t)15);
  const int slab_bytes = kZspBW * z->bmax * (int)sizeof(V);
  const size_t sm = 16 + (size_t)vbytes + 2 * (size_t)slab_bytes;
  static size_t attr = 48 * 1024;  // dynamic shared memory allowed so far
  if (sm > attr) {
    BEM_CUDA(cudaFuncSetAttribute(k_zsp_solve<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    attr = sm;
  }
  k_zsp_solve<R><<<dim3((unsigned)z->obj.size(), nrhs), 32, sm, s>>>(
      z->d_obj, z->d_perm, f ? (const V*)z->L32 : (const V*)z->L64,
      f ? (const V*)z->U32 : (const V*)z->U64, f ? (const V*)z->D32 : (const V*)z->D64, v, ne, e,
      es, vbytes, slab_bytes, z->d_err);
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

template int zsp_apply<float>(aim_ctx*, const float2*, float2*, int, int64_t, int64_t, cudaStream_t);
template int zsp_apply<double>(aim_ctx*, const double2*, double2*, int, int64_t, int64_t,
                               cudaStream_t);

// ---------------------------------------------------------------------------------------
// set-up
// ---------------------------------------------------------------------------------------
// reverse Cuthill-McKee order of a symmetric pattern (adjacency lists, self loops ignored):
// breadth-first from a minimum-degree vertex of each component, neighbours taken in increasing
// degree, the whole order reversed (Cuthill and McKee 1969; George's reversal)
static std::vector<int> rcm_order(int n, const std::vector<int>& rp, const std::vector<int>& ci) {
  std::vector<int> deg(n), order;
  order.reserve(n);
  for (int i = 0; i < n; ++i) deg[i] = rp[i + 1] - rp[i];
  std::vector<char> seen(n, 0);
  std::vector<int> byd(n);
  for (int i = 0; i < n; ++i) byd[i] = i;
  std::stable_sort(byd.begin(), byd.end(), [&](int a, int b) { return deg[a] < deg[b]; });
  std::vector<int> nb;
  for (int start : byd) {
    if (seen[start]) continue;
    size_t head = order.size();
    order.push_back(start);
    seen[start] = 1;
    while (head < order.size()) {
      const int v = order[head++];
      nb.clear();
      for (int k = rp[v]; k < rp[v + 1]; ++k)
        if (!seen[ci[k]]) {
          seen[ci[k]] = 1;
          nb.push_back(ci[k]);
        }
      std::stable_sort(nb.begin(), nb.end(), [&](int a, int b) { return deg[a] < deg[b]; });
      order.insert(order.end(), nb.begin(), nb.end());
    }
  }
  std::reverse(order.begin(), order.end());
  return order;
}

void free_zsp(aim_ctx* c) {
  delete static_cast<Zsp*>(c->zsp);
  c->zsp = nullptr;
  c->zsp_ready = false;
  c->zsp_on = false;
}

int zsp_prepare(aim_ctx* c, const double* d_verts, const int32_t* d_tris, const double* d_cen) {
  const int nobj = c->nobj;
  const double w = kTwoPi * c->freq;
  std::vector<double> rcut(nobj);
  int64_t dense = 0, nmax = 0;
  for (int i = 0; i < nobj; ++i) {
    const bem_material& mt = c->mat[i];
    std::complex<double> epsc(mt.eps_r, -mt.sigma / (w * kEps0));
    std::complex<double> ki = c->k0 * std::sqrt(epsc * mt.mu_r);
    if (ki.imag() > 0) ki = -ki;
    if (!(ki.imag() < 0)) return BEM_OK;  // lossless: no skin depth
    rcut[i] = kZspCut / -ki.imag();
    // extent of the object: no sparsity to find when R_cut spans it
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int t = c->t0[i]; t < c->t1[i]; ++t)
      for (int a = 0; a < 3; ++a)
        for (int q = 0; q < 3; ++q) {
          const double v = c->verts[3 * (size_t)c->tris[3 * (size_t)t + a] + q];
          lo[q] = std::min(lo[q], v);
          hi[q] = std::max(hi[q], v);
        }
    const double ext = std::sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                                 (hi[2] - lo[2]) * (hi[2] - lo[2]));
    if (rcut[i] >= 0.5 * ext) return BEM_OK;
    const int64_t n = c->e1[i] - c->e0[i];
    dense += n * n;
    nmax = std::max(nmax, n);
  }
  if (nmax * (int64_t)sizeof(double2) > 200 * 1024) return BEM_OK;  // vector beyond shared memory
  double* rad = nullptr;
  uint8_t* dmask = nullptr;
  BEM_CUDA(cudaMalloc(&rad, c->nt * sizeof(double)));
  std::unique_ptr<void, decltype(&cudaFree)> hold_rad(rad, &cudaFree);
  BEM_CUDA(cudaMalloc(&dmask, nmax * nmax));
  std::unique_ptr<void, decltype(&cudaFree)> hold_mask(dmask, &cudaFree);
  k_tri_radius<<<(c->nt + 255) / 256, 256>>>(d_verts, d_tris, d_cen, c->nt, rad);
  BEM_CUDA(cudaGetLastError());
  Zsp* z = new Zsp();
  std::unique_ptr<Zsp> hold(z);
  std::vector<int32_t> perm(c->ne), pos(c->ne), row(c->ne + 1, 0), col;
  std::vector<uint8_t> mask(nmax * nmax);
  std::vector<int> rp, ci;
  int64_t nband = 0, nwork = 0;
  for (int i = 0; i < nobj; ++i) {
    const int e0 = c->e0[i], n = c->e1[i] - e0;
    k_zsp_mask<<<(unsigned)(((int64_t)n * n + 255) / 256), 256>>>(d_cen, rad, c->d_et, e0, n,
                                                                   rcut[i], dmask);
    BEM_CUDA(cudaGetLastError());
    BEM_CUDA(cudaMemcpy(mask.data(), dmask, (size_t)n * n, cudaMemcpyDeviceToHost));
    rp.assign(n + 1, 0);
    ci.clear();
    for (int m = 0; m < n; ++m) {
      for (int k = 0; k < n; ++k)
        if (mask[(size_t)m * n + k] && k != m) ci.push_back(k);
      rp[m + 1] = (int)ci.size();
    }
    const std::vector<int> ord = rcm_order(n, rp, ci);
    std::vector<int> p(n);
    for (int r = 0; r < n; ++r) p[ord[r]] = r;
    int b = 0;
    for (int m = 0; m < n; ++m)
      for (int k = rp[m]; k < rp[m + 1]; ++k) b = std::max(b, std::abs(p[m] - p[ci[k]]));
    if (b > kZspBandMax) return BEM_OK;
    b = std::max(b, 1);
    ZspObj o;
    o.e0 = e0;
    o.n = n;
    o.b = b;
    o.pad = 0;
    o.loff = nband;
    o.woff = nwork;
    std::complex<double> epsc(c->mat[i].eps_r, -c->mat[i].sigma / (w * kEps0));
    const std::complex<double> al = -1.0 / (std::complex<double>(0.0, c->k0) * epsc);
    o.ar = al.real();
    o.ai = al.imag();
    z->obj.push_back(o);
    nband += ((int64_t)n * b + 1) & ~(int64_t)1;  // even: 16-byte aligned FP32 slabs
    nwork += (int64_t)n * (2 * b + 1);
    z->bmax = std::max(z->bmax, b);
    for (int r = 0; r < n; ++r) {
      perm[e0 + r] = e0 + ord[r];
      pos[e0 + ord[r]] = e0 + r;
      const int m = ord[r];
      col.push_back(e0 + m);  // the diagonal, then the other kept columns
      for (int k = rp[m]; k < rp[m + 1]; ++k) col.push_back(e0 + ci[k]);
      row[e0 + r + 1] = (int32_t)col.size();
    }
  }
  // the product kernel's shared memory in FP64: the vector and two slabs
  if (16 + ((nmax * 16 + 15) & ~(int64_t)15) + 2 * kZspBW * (int64_t)z->bmax * 16 > (int64_t)kZspSmemMax)
    return BEM_OK;
  // worth it only below half the dense bytes (FP32: band tables, diagonal, rows and columns)
  const int64_t sparse_b = 2 * nband * 8 + (int64_t)c->ne * 8 + (int64_t)col.size() * 12;
  if (sparse_b > 4 * dense) return BEM_OK;
  z->nnz = (int64_t)col.size();
  z->nband = nband;
  z->nwork = nwork;
  z->nmax = (int)nmax;
  BEM_TRY(upload(c, &z->d_obj, z->obj.data(), z->obj.size()));
  BEM_TRY(upload(c, &z->d_perm, perm.data(), perm.size()));
  BEM_TRY(upload(c, &z->d_pos, pos.data(), pos.size()));
  BEM_TRY(upload(c, &z->d_row, row.data(), row.size()));
  BEM_TRY(upload(c, &z->d_col, col.data(), col.size()));
  BEM_TRY(dalloc_t(c, &z->kv64, z->nnz));
  BEM_TRY(dalloc_t(c, &z->kv32, z->nnz));
  // two spare entries: a slab's copy is rounded up to 16 bytes
  BEM_TRY(dalloc_t(c, &z->L64, nband + 2));
  BEM_TRY(dalloc_t(c, &z->U64, nband + 2));
  BEM_TRY(dalloc_t(c, &z->D64, c->ne));
  BEM_TRY(dalloc_t(c, &z->L32, nband + 2));
  BEM_TRY(dalloc_t(c, &z->U32, nband + 2));
  BEM_TRY(dalloc_t(c, &z->D32, c->ne));
  BEM_TRY(dalloc_t(c, &z->d_fail, z->obj.size()));
  BEM_TRY(dalloc_t(c, &z->d_err, 1));
  BEM_CUDA(cudaMemset(z->d_err, 0, sizeof(int)));
  BEM_TRY(dalloc_t(c, &z->v32, (size_t)kMaxBatch * c->ne));
  BEM_TRY(dalloc_t(c, &z->v64, (size_t)kMaxBatch * c->ne));
  BEM_CUDA(cudaMemset(z->d_fail, 0, z->obj.size() * sizeof(int)));
  BEM_CUDA(cudaMalloc(&z->W, nwork * sizeof(double2)));
  BEM_CUDA(cudaMemset(z->W, 0, nwork * sizeof(double2)));
  c->zsp = hold.release();
  return BEM_OK;
}

int zsp_gather(aim_ctx* c, int obj, const double2* L, const double2* B) {
  Zsp* z = static_cast<Zsp*>(c->zsp);
  if (!z || !z->W) return BEM_OK;
  const ZspObj& o = z->obj[obj];
  k_zsp_gather<<<(o.n + 127) / 128, 128>>>(o, L, B, z->d_perm, z->d_pos, z->d_row, z->d_col, z->W,
                                           z->kv64);
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

int zsp_factor(aim_ctx* c) {
  Zsp* z = static_cast<Zsp*>(c->zsp);
  if (!z || !z->W) return BEM_OK;
  const int nobj = (int)z->obj.size();
  k_zsp_lu<<<nobj, 256>>>(z->d_obj, z->W, z->d_fail);
  BEM_CUDA(cudaGetLastError());
  int64_t mx = 0;
  for (const ZspObj& o : z->obj) mx = std::max(mx, (int64_t)o.n * o.b);
  k_zsp_extract<<<dim3((unsigned)((mx + 255) / 256), nobj), 256>>>(z->d_obj, z->W, z->L64, z->U64,
                                                                   z->D64, z->L32, z->U32, z->D32);
  k_round_kv<<<(unsigned)((z->nnz + 255) / 256), 256>>>(z->kv64, z->kv32, z->nnz);
  BEM_CUDA(cudaGetLastError());
  std::vector<int> fail(nobj);
  BEM_CUDA(cudaMemcpy(fail.data(), z->d_fail, nobj * sizeof(int), cudaMemcpyDeviceToHost));
  cudaFree(z->W);
  z->W = nullptr;
  for (int f : fail)
    if (f) {  // a vanishing pivot: the dense form stays
      free_zsp(c);
      return BEM_OK;
    }
  return BEM_OK;
}

__global__ void k_zsp_probe(double2* h, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t v = (uint64_t)i * 0x9E3779B97F4A7C15ull + 0xD1B54A32D192ED03ull;
  v ^= v >> 31;
  v *= 0xBF58476D1CE4E5B9ull;
  v ^= v >> 29;
  h[i] = make_double2((double)(v >> 40) / 8388608.0 - 1.0, (double)((v >> 8) & 0xFFFFFF) / 8388608.0 - 1.0);
}

// Z_s h against the dense Z h (FP64) for one probe vector; the sparse form is kept when every
// object agrees to kZspCheck
int zsp_check(aim_ctx* c) {
  Zsp* z = static_cast<Zsp*>(c->zsp);
  if (!z) return BEM_OK;
  const int ne = c->ne;
  double2 *h = nullptr, *e1 = nullptr, *e2 = nullptr;
  BEM_CUDA(cudaMalloc(&h, 3 * (size_t)ne * sizeof(double2)));
  std::unique_ptr<void, decltype(&cudaFree)> hold(h, &cudaFree);
  e1 = h + ne;
  e2 = h + 2 * (size_t)ne;
  k_zsp_probe<<<(ne + 255) / 256, 256>>>(h, ne);
  c->zsp_ready = true;
  int rc = zsp_apply<double>(c, h, e1, 1, ne, ne, 0);
  if (rc == BEM_OK) rc = run_gemv_plan<double>(c->gplan64, c->f64.Z, h, e2, 1, ne, nullptr, 0);
  if (rc != BEM_OK) {
    free_zsp(c);
    return rc;
  }
  std::vector<double2> a(ne), d(ne);
  int err = 0;
  BEM_CUDA(cudaMemcpy(&err, z->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {  // a bounded wait of the product timed out: keep the dense form
    free_zsp(c);
    return BEM_OK;
  }
  BEM_CUDA(cudaMemcpy(a.data(), e1, ne * sizeof(double2), cudaMemcpyDeviceToHost));
  BEM_CUDA(cudaMemcpy(d.data(), e2, ne * sizeof(double2), cudaMemcpyDeviceToHost));
  double worst = 0;
  for (const ZspObj& o : z->obj) {
    double num = 0, den = 0;
    for (int r = o.e0; r < o.e0 + o.n; ++r) {
      const double dx = a[r].x - d[r].x, dy = a[r].y - d[r].y;
      num += dx * dx + dy * dy;
      den += d[r].x * d[r].x + d[r].y * d[r].y;
    }
    worst = std::max(worst, den > 0 ? std::sqrt(num / den) : (num > 0 ? 1.0 : 0.0));
  }
  z->check = worst;
  if (!(worst <= kZspCheck)) {
    free_zsp(c);
    return BEM_OK;
  }
  c->zsp_on = true;
  return BEM_OK;
}

void zsp_stats(const aim_ctx* c, int64_t* out) {
  const Zsp* z = static_cast<const Zsp*>(c->zsp);
  if (!z || !c->zsp_ready) {
    out[0] = 0;
    out[1] = 0;
    out[2] = 0;
    out[3] = 0;
    out[4] = -1;
    out[5] = 0;
    return;
  }
  out[0] = (int64_t)z->obj.size();
  out[1] = c->zsp_on ? 1 : 0;
  out[2] = z->bmax;
  out[3] = 2 * z->nband * 8 + (int64_t)c->ne * 8 + z->nnz * 12;
  out[4] = (int64_t)(z->check * 1e15);
  int err = 0;  // set by a product whose bounded wait timed out
  if (cudaMemcpy(&err, z->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) err = -1;
  out[5] = err;
}

}  // namespace bem

extern "C" int bem_rcm_order(int n, const int32_t* rowptr, const int32_t* cols, int32_t* order) {
  if (n < 0 || (n > 0 && (!rowptr || !order || (rowptr[n] > 0 && !cols)))) {
    bem::set_error("bem_rcm_order: bad arguments");
    return BEM_EINVAL;
  }
  std::vector<int> rp(n + 1, 0), ci;  // the pattern without self loops
  for (int i = 0; i < n; ++i) {
    if (rowptr[i + 1] < rowptr[i]) {
      bem::set_error("bem_rcm_order: row pointers decrease at row %d", i);
      return BEM_EINVAL;
    }
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      if (cols[k] < 0 || cols[k] >= n) {
        bem::set_error("bem_rcm_order: column %d out of range at row %d", cols[k], i);
        return BEM_EINVAL;
      }
      if (cols[k] != i) ci.push_back(cols[k]);
    }
    rp[i + 1] = (int)ci.size();
  }
  const std::vector<int> ord = bem::rcm_order(n, rp, ci);
  for (int i = 0; i < n; ++i) order[i] = ord[i];
  return BEM_OK;
}
