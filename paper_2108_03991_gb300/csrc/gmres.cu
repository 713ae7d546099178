// Restarted GMRES on the device (Sec. III-E: the solver only needs products with the system
// matrix of Eq. AEFIEoutJ). Arnoldi with classical Gram-Schmidt applied twice (CGS2) in FP64,
// Givens rotations and the small triangular solve in FP64 on the device. The system matvec
// runs in complex FP64 (prec_mode BEM_C64, the plain method) or complex FP32 (BEM_C32); in the
// FP32 mode every restart recomputes the residual with the FP64 matvec, so the outer loop is an
// iterative refinement and the reported true residual is an FP64 one.
#include <chrono>

#include "common.cuh"

namespace bem {

static constexpr int kChunks = 304;  // 2 x 152 SMs

// Dot products h[j] = V_j^H w of nv basis vectors with w: per-block partial sums (k_dots),
// then one block per vector adds them (k_reduce); for a long basis.
__global__ void k_dots(const double2* __restrict__ V, int64_t ldv, int nv,
                       const double2* __restrict__ w, int64_t n, double2* __restrict__ partial) {
  __shared__ double2 red[8];
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = blockIdx.x * per, i1 = min(n, i0 + per);
  for (int j = 0; j < nv; ++j) {
    double2 acc = make_double2(0, 0);
    const double2* v = V + j * ldv;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      double2 a = v[i], b = w[i];
      acc.x += a.x * b.x + a.y * b.y;  // conj(a) b
      acc.y += a.x * b.y - a.y * b.x;
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double2 s = make_double2(0, 0);
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { s.x += red[k].x; s.y += red[k].y; }
      partial[(int64_t)j * gridDim.x + blockIdx.x] = s;
    }
    __syncthreads();
  }
}

// h[j] = sum of partials; if acc != nullptr: acc[j] += h[j]
__global__ void k_reduce(const double2* __restrict__ partial, int nchunks, int nv, double2* h,
                         double2* acc) {
  const int j = blockIdx.x;
  if (j >= nv) return;
  double2 s = make_double2(0, 0);
  for (int i = threadIdx.x; i < nchunks; i += blockDim.x) {
    s.x += partial[(int64_t)j * nchunks + i].x;
    s.y += partial[(int64_t)j * nchunks + i].y;
  }
  s = warp_sum(s);
  __shared__ double2 red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 t = make_double2(0, 0);
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { t.x += red[k].x; t.y += red[k].y; }
    h[j] = t;
    if (acc) { acc[j].x += t.x; acc[j].y += t.y; }
  }
}

// Offsets of right-hand side blockIdx.y when a kernel serves a batch of systems (batched
// FGMRES); all zero for one system.
struct KOff {
  int64_t V = 0, w = 0, h = 0, acc = 0, part = 0, out = 0, H = 0, cs = 0, g = 0, res = 0;
};

// The same and their reduction in one launch, for a short basis: every block writes its
// partial sums, and the block that finishes last (a counter it sets back to zero) adds the partials:
// h[j] = sum of partials; if acc != nullptr: acc[j] += h[j]. No block waits for another.
__global__ void __launch_bounds__(256) k_dots_red(const double2* __restrict__ V, int64_t ldv, int nv,
                                                  const double2* __restrict__ w, int64_t n,
                                                  double2* __restrict__ partial, unsigned* ctr,
                                                  double2* __restrict__ h, double2* acc,
                                                  KOff o = KOff()) {
  __shared__ double2 red[8];
  __shared__ bool last;
  {
    const int64_t y = blockIdx.y;  // the counter of system y is ctr[y]
    V += y * o.V;
    w += y * o.w;
    partial += y * o.part;
    ctr += y;
    h += y * o.h;
    if (acc) acc += y * o.acc;
  }
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = blockIdx.x * per, i1 = min(n, i0 + per);
  for (int j = 0; j < nv; ++j) {
    double2 a2 = make_double2(0, 0);
    const double2* v = V + j * ldv;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      double2 a = v[i], b = w[i];
      a2.x += a.x * b.x + a.y * b.y;  // conj(a) b
      a2.y += a.x * b.y - a.y * b.x;
    }
    a2 = warp_sum(a2);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a2;
    __syncthreads();
    if (threadIdx.x == 0) {
      double2 t = make_double2(0, 0);
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { t.x += red[k].x; t.y += red[k].y; }
      partial[(int64_t)j * gridDim.x + blockIdx.x] = t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    __threadfence();  // this block's partials are visible before it is counted
    last = atomicAdd(ctr, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = warp; j < nv; j += (int)(blockDim.x >> 5)) {
    double2 t = make_double2(0, 0);
    for (int i = lane; i < (int)gridDim.x; i += 32) {
      const double2 q = __ldcg(&partial[(int64_t)j * gridDim.x + i]);
      t.x += q.x;
      t.y += q.y;
    }
    t = warp_sum(t);
    if (lane == 0) {
      h[j] = t;
      if (acc) { acc[j].x += t.x; acc[j].y += t.y; }
    }
  }
  if (threadIdx.x == 0) *ctr = 0u;
}

// w += sign * sum_j h[j] V[j]
__global__ void k_axpy_basis(const double2* __restrict__ V, int64_t ldv, int nv,
                             const double2* __restrict__ h, double sign, double2* w, int64_t n,
                             KOff o = KOff()) {
  extern __shared__ double2 hs[];
  V += blockIdx.y * o.V;
  h += blockIdx.y * o.h;
  w += blockIdx.y * o.w;
  for (int j = threadIdx.x; j < nv; j += blockDim.x) hs[j] = h[j];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double2 acc = w[i];
    for (int j = 0; j < nv; ++j) {
      double2 v = V[j * ldv + i], c = hs[j];
      acc.x += sign * (c.x * v.x - c.y * v.y);
      acc.y += sign * (c.x * v.y + c.y * v.x);
    }
    w[i] = acc;
  }
}

// out = in * (1 / |norm2|)  where nrm2 holds |w|^2 (as the real part of a dot product)
__global__ void k_normalize(const double2* __restrict__ in, const double2* nrm2, double2* out,
                            double* hsub, int64_t n) {
  const double nr = sqrt(fmax(nrm2->x, 0.0));
  if (blockIdx.x == 0 && threadIdx.x == 0 && hsub) *hsub = nr;
  const double s = nr > 0 ? 1.0 / nr : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = make_double2(in[i].x * s, in[i].y * s);
}

__global__ void k_sub(const double2* a, const double2* b, double2* o, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    o[i] = make_double2(a[i].x - b[i].x, a[i].y - b[i].y);
}

__global__ void k_to32(const double2* a, float2* o, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    o[i] = make_float2((float)a[i].x, (float)a[i].y);
}
__global__ void k_to64(const float2* a, double2* o, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    o[i] = make_double2(a[i].x, a[i].y);
}

// Givens step for column k of H (leading dimension ldh = m + 1), one thread.
// Rotation (c, s) acts as (x, y) -> (conj(c) x + conj(s) y, -s x + c y).
__device__ void givens_step(double2* H, int ldh, int k, double hsub, double2* cs, double2* sn,
                            double2* g, double* resid) {
  double2* col = H + (int64_t)k * ldh;
  col[k + 1] = make_double2(hsub, 0.0);
  for (int i = 0; i < k; ++i) {
    double2 a = col[i], b = col[i + 1], c = cs[i], s = sn[i];
    double2 t = cadd(cmul(cconj(c), a), cmul(cconj(s), b));
    col[i + 1] = csub(cmul(c, b), cmul(s, a));
    col[i] = t;
  }
  double2 a = col[k], b = col[k + 1];
  double den = sqrt(a.x * a.x + a.y * a.y + b.x * b.x + b.y * b.y);
  double2 c = den > 0 ? make_double2(a.x / den, a.y / den) : make_double2(1, 0);
  double2 s = den > 0 ? make_double2(b.x / den, b.y / den) : make_double2(0, 0);
  cs[k] = c;
  sn[k] = s;
  col[k] = make_double2(den, 0.0);
  col[k + 1] = make_double2(0, 0);
  double2 gk = g[k];
  g[k + 1] = mk(-(s.x * gk.x - s.y * gk.y), -(s.x * gk.y + s.y * gk.x));
  g[k] = cmul(cconj(c), gk);
  *resid = sqrt(g[k + 1].x * g[k + 1].x + g[k + 1].y * g[k + 1].y);
}

// v_{k+1} = w / |w| and, in block 0's first thread, the Givens step of column k with the
// subdiagonal |w| (the Arnoldi step's last two operations in one launch)
__global__ void k_normalize_givens(const double2* __restrict__ in, const double2* nrm2, double2* out,
                                   int64_t n, double2* H, int ldh, int k, double2* cs, double2* sn,
                                   double2* g, double* resid, KOff o = KOff()) {
  {
    const int64_t y = blockIdx.y;
    in += y * o.w;
    nrm2 += y * o.h;
    out += y * o.out;
    H += y * o.H;
    cs += y * o.cs;
    sn += y * o.cs;
    g += y * o.g;
    resid += y * o.res;
  }
  const double nr = sqrt(fmax(nrm2->x, 0.0));
  const double s = nr > 0 ? 1.0 / nr : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = make_double2(in[i].x * s, in[i].y * s);
  if (blockIdx.x == 0 && threadIdx.x == 0) givens_step(H, ldh, k, nr, cs, sn, g, resid);
}

// y = R^{-1} g for the leading k x k upper-triangular block, one thread
__global__ void k_backsolve(const double2* H, int ldh, int k, const double2* g, double2* y) {
  for (int i = k - 1; i >= 0; --i) {
    double2 s = g[i];
    for (int j = i + 1; j < k; ++j) s = csub(s, cmul(H[(int64_t)j * ldh + i], y[j]));
    double2 d = H[(int64_t)i * ldh + i];
    double dd = d.x * d.x + d.y * d.y;
    y[i] = dd > 0 ? cmul(s, make_double2(d.x / dd, -d.y / dd)) : make_double2(0, 0);
  }
}

__global__ void k_set_g0(double2* g, int m1, const double* beta) {
  for (int i = threadIdx.x; i < m1; i += blockDim.x) g[i] = make_double2(i == 0 ? *beta : 0.0, 0.0);
}

// Krylov workspace, carved from one device buffer that the context keeps between solves
struct GmWork {
  double2 *V = nullptr, *w = nullptr, *r = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr,
          *g = nullptr, *h = nullptr, *hacc = nullptr, *partial = nullptr, *y = nullptr, *Zb = nullptr;
  double* dsc = nullptr;  // [0] = subdiagonal, [1] = residual estimate, [2] = beta,
                          // [4] = block counter of k_dots_red (zero between launches)
};

static int gm_workspace(aim_ctx* c, int64_t n, int m, bool flexible, GmWork* W) {
  const int ldh = m + 1;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t z = sizeof(double2);
  const size_t sizes[13] = {al((size_t)(m + 1) * n * z), al(n * z), al(n * z), al((size_t)ldh * m * z),
                            al(m * z), al(m * z), al((m + 1) * z), al((m + 1) * z), al((m + 1) * z),
                            al((size_t)(m + 1) * kChunks * z), al((m + 1) * z),
                            flexible ? al((size_t)m * n * z) : 0, al(8 * sizeof(double))};
  size_t total = 0;
  for (size_t v : sizes) total += v;
  if (c->gm_bytes < total) {
    if (c->gm_ws) cudaFree(c->gm_ws);
    c->gm_ws = nullptr;
    c->gm_bytes = 0;
    cudaError_t e = cudaMalloc(&c->gm_ws, total);
    if (e != cudaSuccess) {
      set_error("gmres workspace (%zu bytes): %s", total, cudaGetErrorString(e));
      c->gm_ws = nullptr;
      return BEM_ENOMEM;
    }
    c->gm_bytes = total;
  }
  char* p = static_cast<char*>(c->gm_ws);
  double2** dst[12] = {&W->V, &W->w, &W->r, &W->H, &W->cs, &W->sn, &W->g, &W->h, &W->hacc,
                       &W->partial, &W->y, &W->Zb};
  for (int i = 0; i < 12; ++i) {
    *dst[i] = sizes[i] ? reinterpret_cast<double2*>(p) : nullptr;
    p += sizes[i];
  }
  W->dsc = reinterpret_cast<double*>(p);
  return BEM_OK;
}

static int dot_into(const double2* V, int64_t ldv, int nv, const double2* w, int64_t n, GmWork& W,
                    double2* h, double2* acc, cudaStream_t s) {
  if (nv <= 16) {  // one launch; the last block's reduction is short
    k_dots_red<<<kChunks, 256, 0, s>>>(V, ldv, nv, w, n, W.partial,
                                       reinterpret_cast<unsigned*>(W.dsc + 4), h, acc);
  } else {
    k_dots<<<kChunks, 256, 0, s>>>(V, ldv, nv, w, n, W.partial);
    k_reduce<<<nv, 256, 0, s>>>(W.partial, kChunks, nv, h, acc);
  }
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

// y = A x in FP64 (plain) or through the FP32 matvec
// (both go through the context's fixed buffers so one captured graph serves every iteration)
static int sys_apply(aim_ctx* c, int prec, const double2* x, double2* y, cudaStream_t s) {
  const int64_t n = (int64_t)c->ne + c->nt;
  if (prec == BEM_C64) {
    BEM_CUDA(cudaMemcpyAsync(c->f64.xin, x, n * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    BEM_TRY(matvec_graph<double>(c, AIM_OP_SYSTEM, c->f64.xin, c->f64.yout, s));
    BEM_CUDA(cudaMemcpyAsync(y, c->f64.yout, n * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    return BEM_OK;
  }
  k_to32<<<kChunks, 256, 0, s>>>(x, c->f32.xin, n);
  BEM_TRY(matvec_graph<float>(c, AIM_OP_SYSTEM, c->f32.xin, c->f32.yout, s));
  k_to64<<<kChunks, 256, 0, s>>>(c->f32.yout, y, n);
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

int gmres_solve(aim_ctx* c, const void* bv, void* xv, const bem_solve_opts* o, bem_solve_info* info,
                cudaStream_t s) {
  using clk = std::chrono::steady_clock;
  const auto t0 = clk::now();
  const double2* b = (const double2*)bv;
  double2* x = (double2*)xv;
  const int64_t n = (int64_t)c->ne + c->nt;
  const int m = o->restart;
  const int ldh = m + 1;
  // right preconditioning (flexible form: the preconditioned directions Zb are kept)
  const bool flexible = o->precond == 1 || o->precond == 2;
  if (flexible) BEM_TRY(setup_precond(c));
  GmWork W;
  BEM_TRY(gm_workspace(c, n, m, flexible, &W));
  BEM_CUDA(cudaMemsetAsync(W.dsc + 4, 0, sizeof(double), s));
  double2* Zb = W.Zb;
  BEM_CUDA(cudaMemsetAsync(W.H, 0, sizeof(double2) * ldh * m, s));
  // ||b|| and ||x0|| (a zero initial guess needs no first matvec: r = b)
  BEM_TRY(dot_into(b, n, 1, b, n, W, W.h, nullptr, s));
  BEM_TRY(dot_into(x, n, 1, x, n, W, W.h + 1, nullptr, s));
  double2 bb[2];
  BEM_CUDA(cudaMemcpyAsync(bb, W.h, 2 * sizeof(double2), cudaMemcpyDeviceToHost, s));
  BEM_CUDA(cudaStreamSynchronize(s));
  const double bnorm = std::sqrt(std::max(bb[0].x, 0.0));
  bool x_zero = bb[1].x == 0.0;
  int iters = 0;
  double est = 1.0, truer = 1.0;
  int status = BEM_ENOCONV;
  if (bnorm == 0) {
    BEM_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double2), s));
    status = BEM_OK;
    est = truer = 0;
  }
  bool fresh = bnorm == 0;
  while (status != BEM_OK && iters < o->max_iter) {
    // r = b - A x (FP64 matvec), beta = ||r||
    const double2* r = b;
    if (!x_zero) {
      BEM_TRY(sys_apply(c, BEM_C64, x, W.w, s));
      k_sub<<<kChunks, 256, 0, s>>>(b, W.w, W.r, n);
      r = W.r;
    }
    x_zero = false;
    BEM_TRY(dot_into(r, n, 1, r, n, W, W.h, nullptr, s));
    k_normalize<<<kChunks, 256, 0, s>>>(r, W.h, W.V, W.dsc + 2, n);
    double beta;
    BEM_CUDA(cudaMemcpyAsync(&beta, W.dsc + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaStreamSynchronize(s));
    truer = beta / bnorm;
    est = truer;
    fresh = true;  // truer is the true FP64 residual of the current x
    if (truer <= o->tol) { status = BEM_OK; break; }
    if (o->time_limit_s > 0 && std::chrono::duration<double>(clk::now() - t0).count() > o->time_limit_s) break;
    k_set_g0<<<1, 256, 0, s>>>(W.g, m + 1, W.dsc + 2);
    int k = 0;
    for (; k < m && iters < o->max_iter; ++k) {
      const double2* vk = W.V + (int64_t)k * n;
      if (Zb) {
        double2* zk = Zb + (int64_t)k * n;
        if (o->precond == 2) {  // block-diagonal + learned correction (FP32)
          k_to32<<<kChunks, 256, 0, s>>>(vk, c->f32.xin, n);
          BEM_TRY(net_apply(c, c->f32.xin, c->f32.yout, s));
          k_to64<<<kChunks, 256, 0, s>>>(c->f32.yout, zk, n);
        } else if (o->prec_mode == BEM_C64) {
          BEM_TRY(precond_apply<double>(c, vk, zk, s));
        } else {
          // the preconditioned vector lands in the FP32 matvec's input buffer (and in zk), so
          // the FP32 product below starts from it without converting zk back
          BEM_TRY(precond_apply_mixed(c, vk, c->f32.xin, zk, s));
        }
        vk = zk;
      }
      if (Zb && o->precond == 1 && o->prec_mode == BEM_C32) {
        BEM_TRY(matvec_graph<float>(c, AIM_OP_SYSTEM, c->f32.xin, c->f32.yout, s));
        k_to64<<<kChunks, 256, 0, s>>>(c->f32.yout, W.w, n);
      } else {
        BEM_TRY(sys_apply(c, o->prec_mode, vk, W.w, s));
      }
      // CGS2: h = V^H w, w -= V h, twice; accumulate into column k of H
      double2* Hk = W.H + (int64_t)k * ldh;
      BEM_CUDA(cudaMemsetAsync(Hk, 0, sizeof(double2) * (k + 1), s));
      for (int pass = 0; pass < 2; ++pass) {
        BEM_TRY(dot_into(W.V, n, k + 1, W.w, n, W, W.h, Hk, s));
        k_axpy_basis<<<kChunks, 256, (k + 1) * sizeof(double2), s>>>(W.V, n, k + 1, W.h, -1.0, W.w, n);
      }
      BEM_TRY(dot_into(W.w, n, 1, W.w, n, W, W.h, nullptr, s));
      k_normalize_givens<<<kChunks, 256, 0, s>>>(W.w, W.h, W.V + (int64_t)(k + 1) * n, n, W.H, ldh, k,
                                                 W.cs, W.sn, W.g, W.dsc + 1);
      BEM_CUDA(cudaGetLastError());
      double res;
      BEM_CUDA(cudaMemcpyAsync(&res, W.dsc + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
      BEM_CUDA(cudaStreamSynchronize(s));
      ++iters;
      est = res / bnorm;
      if (est <= o->tol) { ++k; break; }
      if (o->time_limit_s > 0 && std::chrono::duration<double>(clk::now() - t0).count() > o->time_limit_s) { ++k; break; }
    }
    // x += V[:k] y, y = R^{-1} g
    k_backsolve<<<1, 1, 0, s>>>(W.H, ldh, k, W.g, W.y);
    k_axpy_basis<<<kChunks, 256, (k + 1) * sizeof(double2), s>>>(Zb ? Zb : W.V, n, k, W.y, 1.0, x, n);
    fresh = false;
    BEM_CUDA(cudaGetLastError());
    if (o->time_limit_s > 0 && std::chrono::duration<double>(clk::now() - t0).count() > o->time_limit_s) break;
  }
  // true residual with the FP64 matvec, unless the loop just took it for this x (the FP64
  // matvec is the most expensive step of an FP32-bulk solve on this hardware)
  if (!fresh) {
    BEM_TRY(sys_apply(c, BEM_C64, x, W.w, s));
    k_sub<<<kChunks, 256, 0, s>>>(b, W.w, W.r, n);
    BEM_TRY(dot_into(W.r, n, 1, W.r, n, W, W.h, nullptr, s));
    double2 rr;
    BEM_CUDA(cudaMemcpyAsync(&rr, W.h, sizeof(double2), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaStreamSynchronize(s));
    truer = bnorm > 0 ? std::sqrt(std::max(rr.x, 0.0)) / bnorm : 0.0;
  }
  status = truer <= o->tol ? BEM_OK : BEM_ENOCONV;
  if (info) {
    info->iters = iters;
    info->resid_est = est;
    info->resid_true = truer;
    info->seconds = std::chrono::duration<double>(clk::now() - t0).count();
  }
  return status;
}

// ---------------------------------------------------------------------------------------
// Batched FGMRES: nrhs (<= kMaxBatch) systems A x_r = b_r solved in lockstep. Each right-hand
// side has its own Krylov basis, Hessenberg matrix and rotations; every iteration applies the
// preconditioner and the system matrix to all of them at once (aim_matvec_batch and the
// batched preconditioner read each block matrix once for all), the Gram-Schmidt and Givens
// steps run per right-hand side. Basis vectors of one step are stored side by side
// (V[k][r][N]) so the batched products read them as one block. A cycle ends when every
// right-hand side's residual estimate is below tol (or after m steps); the true FP64 residuals
// are then taken with one batched FP64 product.
// ---------------------------------------------------------------------------------------
struct GmBatch {
  double2 *V = nullptr, *Zb = nullptr, *w = nullptr, *rr = nullptr, *ax = nullptr;
  float2 *x32 = nullptr, *y32 = nullptr;
  double2 *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr, *h = nullptr,
          *partial = nullptr;
  double* dsc = nullptr;  // [r][8]: [1] residual estimate, [2] beta; [kMaxBatch * 8] counter
};

static int gm_batch_workspace(aim_ctx* c, int64_t n, int m, int B, bool flexible, GmBatch* W) {
  const int ldh = m + 1;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t z = sizeof(double2), f = sizeof(float2);
  const size_t sizes[14] = {al((size_t)(m + 1) * B * n * z), flexible ? al((size_t)m * B * n * z) : 0,
                            al(B * n * z), al(B * n * z), al(B * n * z), al(B * n * f), al(B * n * f),
                            al((size_t)B * ldh * m * z), al((size_t)B * m * z), al((size_t)B * m * z),
                            al((size_t)B * (m + 1) * z), al((size_t)B * (m + 1) * z),
                            al((size_t)B * (m + 1) * z), al((size_t)B * (m + 1) * kChunks * z)};
  size_t total = al((size_t)(kMaxBatch * 8 + 8) * sizeof(double));
  for (size_t v : sizes) total += v;
  if (c->gmb_bytes < total) {
    if (c->gmb_ws) cudaFree(c->gmb_ws);
    c->gmb_ws = nullptr;
    c->gmb_bytes = 0;
    if (cudaMalloc(&c->gmb_ws, total) != cudaSuccess) {
      set_error("batched gmres workspace (%zu bytes): out of device memory", total);
      return BEM_ENOMEM;
    }
    c->gmb_bytes = total;
  }
  char* p = static_cast<char*>(c->gmb_ws);
  void** dst[14] = {(void**)&W->V, (void**)&W->Zb, (void**)&W->w, (void**)&W->rr, (void**)&W->ax,
                    (void**)&W->x32, (void**)&W->y32, (void**)&W->H, (void**)&W->cs, (void**)&W->sn,
                    (void**)&W->g, (void**)&W->y, (void**)&W->h, (void**)&W->partial};
  for (int i = 0; i < 14; ++i) {
    *dst[i] = sizes[i] ? static_cast<void*>(p) : nullptr;
    p += sizes[i];
  }
  W->dsc = reinterpret_cast<double*>(p);
  return BEM_OK;
}

static int dots_b(const double2* V, int64_t ldv, int nv, const double2* w, int64_t n, GmBatch& W,
                  double2* h, double2* acc, cudaStream_t s) {
  if (nv <= 16) {
    k_dots_red<<<kChunks, 256, 0, s>>>(V, ldv, nv, w, n, W.partial,
                                       reinterpret_cast<unsigned*>(W.dsc + kMaxBatch * 8), h, acc);
  } else {
    k_dots<<<kChunks, 256, 0, s>>>(V, ldv, nv, w, n, W.partial);
    k_reduce<<<nv, 256, 0, s>>>(W.partial, kChunks, nv, h, acc);
  }
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

// y (FP64, B vectors of N) = A x for the batch: FP64 batched product, or FP32 from x32
static int batch_apply64(aim_ctx* c, const double2* x, double2* y, int B, cudaStream_t s) {
  BEM_TRY(batch_buffers<double>(c));
  return matvec_graph<double>(c, kBatchOp + B, x, y, s);
}

int gmres_solve_batch(aim_ctx* c, const void* bv, void* xv, int B, const bem_solve_opts* o,
                      bem_solve_info* infos, cudaStream_t s) {
  using clk = std::chrono::steady_clock;
  const auto t0 = clk::now();
  const double2* b = (const double2*)bv;
  double2* x = (double2*)xv;
  const int64_t n = (int64_t)c->ne + c->nt, Bn = B * n;
  const int m = o->restart, ldh = m + 1, m1 = m + 1;
  const bool flexible = o->precond == 1;
  const bool fp32 = o->prec_mode == BEM_C32;
  if (flexible) BEM_TRY(setup_precond(c));
  if (fp32) BEM_TRY(batch_buffers<float>(c));
  BEM_TRY(batch_buffers<double>(c));
  GmBatch W;
  BEM_TRY(gm_batch_workspace(c, n, m, B, flexible, &W));
  BEM_CUDA(cudaMemsetAsync(W.dsc + kMaxBatch * 8, 0, 8 * sizeof(double), s));  // counters
  BEM_CUDA(cudaMemsetAsync(W.H, 0, sizeof(double2) * B * ldh * m, s));
  std::vector<double2> hh((size_t)B * m1);
  std::vector<double> dh((size_t)B * 8);
  for (int r = 0; r < B; ++r) {
    BEM_TRY(dots_b(b + r * n, n, 1, b + r * n, n, W, W.h + r * m1, nullptr, s));
    BEM_TRY(dots_b(x + r * n, n, 1, x + r * n, n, W, W.h + r * m1 + 1, nullptr, s));
  }
  BEM_CUDA(cudaMemcpyAsync(hh.data(), W.h, hh.size() * sizeof(double2), cudaMemcpyDeviceToHost, s));
  BEM_CUDA(cudaStreamSynchronize(s));
  std::vector<double> bnorm(B), est(B, 1.0), truer(B, 1.0);
  bool x_zero = true;
  for (int r = 0; r < B; ++r) {
    bnorm[r] = std::sqrt(std::max(hh[(size_t)r * m1].x, 0.0));
    if (bnorm[r] == 0) {  // a zero right-hand side has the zero solution
      BEM_CUDA(cudaMemsetAsync(x + r * n, 0, n * sizeof(double2), s));
    } else if (hh[(size_t)r * m1 + 1].x != 0.0) {
      x_zero = false;
    }
  }
  auto rel = [&](double v, int r) { return bnorm[r] > 0 ? v / bnorm[r] : 0.0; };
  auto all_below = [&](const std::vector<double>& v) {
    for (int r = 0; r < B; ++r)
      if (!(v[r] <= o->tol)) return false;
    return true;
  };
  auto out_of_time = [&]() {
    return o->time_limit_s > 0 && std::chrono::duration<double>(clk::now() - t0).count() > o->time_limit_s;
  };
  int iters = 0;
  bool fresh = false, converged = false;
  while (iters < o->max_iter) {
    // r = b - A x with the batched FP64 product (none for a zero initial guess)
    if (!x_zero) {
      BEM_TRY(batch_apply64(c, x, W.ax, B, s));
      k_sub<<<kChunks, 256, 0, s>>>(b, W.ax, W.rr, Bn);
    } else {
      BEM_CUDA(cudaMemcpyAsync(W.rr, b, Bn * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    }
    x_zero = false;
    for (int r = 0; r < B; ++r) {
      BEM_TRY(dots_b(W.rr + r * n, n, 1, W.rr + r * n, n, W, W.h + r * m1, nullptr, s));
      k_normalize<<<kChunks, 256, 0, s>>>(W.rr + r * n, W.h + r * m1, W.V + r * n, W.dsc + r * 8 + 2, n);
    }
    BEM_CUDA(cudaMemcpyAsync(dh.data(), W.dsc, dh.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaStreamSynchronize(s));
    for (int r = 0; r < B; ++r) est[r] = truer[r] = rel(dh[(size_t)r * 8 + 2], r);
    fresh = true;
    if (all_below(truer)) { converged = true; break; }
    if (out_of_time()) break;
    for (int r = 0; r < B; ++r) k_set_g0<<<1, 256, 0, s>>>(W.g + r * m1, m1, W.dsc + r * 8 + 2);
    int k = 0;
    for (; k < m && iters < o->max_iter; ++k) {
      const double2* Vk = W.V + (int64_t)k * Bn;
      const double2* in64 = Vk;
      if (flexible) {
        double2* Zk = W.Zb + (int64_t)k * Bn;
        if (fp32) {
          BEM_TRY(precond_apply_batch(c, Vk, B, W.x32, Zk, s));  // FP32 copy lands in x32
        } else {
          for (int r = 0; r < B; ++r) BEM_TRY(precond_apply<double>(c, Vk + r * n, Zk + r * n, s));
        }
        in64 = Zk;
      }
      if (fp32) {
        if (!flexible) k_to32<<<kChunks, 256, 0, s>>>(in64, W.x32, Bn);
        BEM_TRY(matvec_graph<float>(c, kBatchOp + B, W.x32, W.y32, s));
        k_to64<<<kChunks, 256, 0, s>>>(W.y32, W.w, Bn);
      } else {
        // through a fixed input buffer, so that one captured graph serves every step
        BEM_CUDA(cudaMemcpyAsync(W.rr, in64, Bn * sizeof(double2), cudaMemcpyDeviceToDevice, s));
        BEM_TRY(batch_apply64(c, W.rr, W.w, B, s));
      }
      if (k + 1 <= 16) {  // every system's Gram-Schmidt and Givens steps in the same launches
        for (int r = 0; r < B; ++r)
          BEM_CUDA(cudaMemsetAsync(W.H + (int64_t)r * ldh * m + (int64_t)k * ldh, 0,
                                   sizeof(double2) * (k + 1), s));
        unsigned* ctr = reinterpret_cast<unsigned*>(W.dsc + kMaxBatch * 8);
        KOff o;
        o.V = n;
        o.w = n;
        o.h = m1;
        o.acc = (int64_t)ldh * m;
        o.part = (int64_t)m1 * kChunks;
        const dim3 gb(kChunks, B);
        for (int pass = 0; pass < 2; ++pass) {
          k_dots_red<<<gb, 256, 0, s>>>(W.V, Bn, k + 1, W.w, n, W.partial, ctr, W.h,
                                        W.H + (int64_t)k * ldh, o);
          k_axpy_basis<<<gb, 256, (k + 1) * sizeof(double2), s>>>(W.V, Bn, k + 1, W.h, -1.0, W.w, n, o);
        }
        KOff on;
        on.V = n;
        on.w = n;
        on.h = m1;
        on.part = (int64_t)m1 * kChunks;
        k_dots_red<<<gb, 256, 0, s>>>(W.w, n, 1, W.w, n, W.partial, ctr, W.h, nullptr, on);
        KOff og;
        og.w = n;
        og.h = m1;
        og.out = n;
        og.H = (int64_t)ldh * m;
        og.cs = m;
        og.g = m1;
        og.res = 8;
        k_normalize_givens<<<gb, 256, 0, s>>>(W.w, W.h, W.V + (int64_t)(k + 1) * Bn, n, W.H, ldh, k,
                                              W.cs, W.sn, W.g, W.dsc + 1, og);
      }
      for (int r = 0; r < B && k + 1 > 16; ++r) {
        const double2* Vr = W.V + r * n;
        double2* wr = W.w + r * n;
        double2* hr = W.h + r * m1;
        double2* Hr = W.H + (int64_t)r * ldh * m;
        double2* Hk = Hr + (int64_t)k * ldh;
        BEM_CUDA(cudaMemsetAsync(Hk, 0, sizeof(double2) * (k + 1), s));
        for (int pass = 0; pass < 2; ++pass) {
          BEM_TRY(dots_b(Vr, Bn, k + 1, wr, n, W, hr, Hk, s));
          k_axpy_basis<<<kChunks, 256, (k + 1) * sizeof(double2), s>>>(Vr, Bn, k + 1, hr, -1.0, wr, n);
        }
        BEM_TRY(dots_b(wr, n, 1, wr, n, W, hr, nullptr, s));
        k_normalize_givens<<<kChunks, 256, 0, s>>>(wr, hr, W.V + (int64_t)(k + 1) * Bn + r * n, n, Hr, ldh,
                                                   k, W.cs + r * m, W.sn + r * m, W.g + r * m1,
                                                   W.dsc + r * 8 + 1);
      }
      BEM_CUDA(cudaGetLastError());
      BEM_CUDA(cudaMemcpyAsync(dh.data(), W.dsc, dh.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
      BEM_CUDA(cudaStreamSynchronize(s));
      ++iters;
      for (int r = 0; r < B; ++r) est[r] = rel(dh[(size_t)r * 8 + 1], r);
      if (all_below(est)) { ++k; break; }
      if (out_of_time()) { ++k; break; }
    }
    // x_r += Z_r y_r (or V_r y_r), y_r = R_r^{-1} g_r
    for (int r = 0; r < B; ++r) {
      k_backsolve<<<1, 1, 0, s>>>(W.H + (int64_t)r * ldh * m, ldh, k, W.g + r * m1, W.y + r * m1);
      k_axpy_basis<<<kChunks, 256, (k + 1) * sizeof(double2), s>>>((flexible ? W.Zb : W.V) + r * n, Bn, k,
                                                                 W.y + r * m1, 1.0, x + r * n, n);
    }
    fresh = false;
    BEM_CUDA(cudaGetLastError());
    if (out_of_time()) break;
  }
  if (!fresh && !converged) {  // the true residuals of the last update
    BEM_TRY(batch_apply64(c, x, W.ax, B, s));
    k_sub<<<kChunks, 256, 0, s>>>(b, W.ax, W.rr, Bn);
    for (int r = 0; r < B; ++r)
      BEM_TRY(dots_b(W.rr + r * n, n, 1, W.rr + r * n, n, W, W.h + r * m1, nullptr, s));
    BEM_CUDA(cudaMemcpyAsync(hh.data(), W.h, hh.size() * sizeof(double2), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaStreamSynchronize(s));
    for (int r = 0; r < B; ++r) truer[r] = rel(std::sqrt(std::max(hh[(size_t)r * m1].x, 0.0)), r);
  }
  const double secs = std::chrono::duration<double>(clk::now() - t0).count();
  if (infos)
    for (int r = 0; r < B; ++r) {
      infos[r].iters = iters;
      infos[r].resid_est = est[r];
      infos[r].resid_true = truer[r];
      infos[r].seconds = secs;
    }
  return all_below(truer) ? BEM_OK : BEM_ENOCONV;
}

}  // namespace bem
