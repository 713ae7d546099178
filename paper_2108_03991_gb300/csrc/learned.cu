// Learned correction for the preconditioned solve (an extension; the paper's own preconditioner
// is the constraint preconditioner of Qian 2009, Sec. II-C). A 4-layer 3-D convolutional net
// on the AIM grid (3x3x3 kernels, zero padding, no biases, ReLU between layers, channels
// 8 -> 16 -> 16 -> 16 -> 8) maps the projected residual P r (Re/Im of the four grid components,
// scaled by their RMS) to a grid correction that W = P^T interpolates back:
//   M(r) = M_bd r + W net(P r),
// used on the right in flexible GMRES. Weights and activations are BF16, every sum is FP32;
// gradients are FP32. Training minimises |P (W net(P r) - t)|^2 / |P t|^2, t = x - M_bd r, over
// pairs r = A x with x drawn on the device (splitmix64 counter hash, Box-Muller; half of them
// smoothed as grid potentials of random grid sources), with Adam. The error is measured on the
// grid: the block-diagonal part leaves mesh-scale error modes that no grid field represents, and
// the network is meant as a coarse (grid-level) correction beside it.
#include <cuda_bf16.h>

#include <cmath>
#include <vector>

#include "common.cuh"

namespace bem {

constexpr int kLayers = 4;
constexpr int kCh[kLayers + 1] = {8, 16, 16, 16, 8};
constexpr int kTX = 8, kTY = 8, kTZ = 4;  // output tile: 256 points, one per thread
constexpr int kHX = kTX + 2, kHY = kTY + 2, kHZ = kTZ + 2;
constexpr int kHalo = kHX * kHY * kHZ;

static int wcount(int l) { return kCh[l] * kCh[l + 1] * 27; }
static int woffset(int l) {
  int o = 0;
  for (int i = 0; i < l; ++i) o += wcount(i);
  return o;
}
static int wtotal() { return woffset(kLayers); }

// ---------------------------------------------------------------------------------------
// splitmix64 (Steele, Lea, Flood 2014) as a counter-based hash; Box-Muller normals
// ---------------------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
__host__ __device__ __forceinline__ double u01(uint64_t h) {  // (0, 1)
  return ((h >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}
__global__ void k_randn_c(uint64_t seed, int n, float2* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double u1 = u01(splitmix64(seed ^ (2ull * i))), u2 = u01(splitmix64(seed ^ (2ull * i + 1)));
  double r = sqrt(-2.0 * log(u1)), th = 2.0 * 3.14159265358979323846 * u2;
  out[i] = make_float2((float)(r * cos(th)), (float)(r * sin(th)));
}

// ---------------------------------------------------------------------------------------
// convolution kernels
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ void from_f(float v, float* o) { *o = v; }
__device__ __forceinline__ void from_f(float v, __nv_bfloat16* o) { *o = __float2bfloat16(v); }

struct Dims {
  int nx, ny, nz;
  int64_t ng;
  int tx, ty;  // tiles per axis (x, y)
};

// load the (kTZ+2)(kTY+2)(kTX+2) halo of channel block [C] into shared memory (zero padding)
template <int C, typename T>
__device__ __forceinline__ void load_halo(const T* in, const Dims& d, int x0, int y0, int z0,
                                          float* s) {
  for (int i = threadIdx.x; i < C * kHalo; i += blockDim.x) {
    const int c = i / kHalo, h = i - c * kHalo;
    const int hz = h / (kHY * kHX), hy = (h / kHX) % kHY, hx = h % kHX;
    const int x = x0 + hx - 1, y = y0 + hy - 1, z = z0 + hz - 1;
    float v = 0.f;
    if (x >= 0 && y >= 0 && z >= 0 && x < d.nx && y < d.ny && z < d.nz)
      v = to_f(in[c * d.ng + ((int64_t)z * d.ny + y) * d.nx + x]);
    s[i] = v;
  }
}

// out[co][p] = act( sum_ci sum_taps w[co][ci][tap] in[ci][p + tap - 1] ) (* mask[co][p] > 0)
// w is read as BF16-rounded values (the network's weights are BF16)
template <int CI, int CO, typename TI, typename TO, bool RELU>
__global__ void __launch_bounds__(256) k_conv(const TI* __restrict__ in, const float* __restrict__ w,
                                              TO* __restrict__ out,
                                              const __nv_bfloat16* __restrict__ mask, Dims d,
                                              int round_w) {
  extern __shared__ float sm[];
  float* sw = sm;                 // [CO][CI][27]
  float* sin_ = sm + CO * CI * 27;  // [CI][halo]
  const int tile = blockIdx.x;
  const int x0 = (tile % d.tx) * kTX, y0 = (tile / d.tx) * kTY, z0 = blockIdx.y * kTZ;
  for (int i = threadIdx.x; i < CO * CI * 27; i += blockDim.x)
    sw[i] = round_w ? __bfloat162float(__float2bfloat16(w[i])) : w[i];
  load_halo<CI>(in, d, x0, y0, z0, sin_);
  __syncthreads();
  const int tx = threadIdx.x % kTX, ty = (threadIdx.x / kTX) % kTY, tz = threadIdx.x / (kTX * kTY);
  float acc[CO];
#pragma unroll
  for (int co = 0; co < CO; ++co) acc[co] = 0.f;
  for (int ci = 0; ci < CI; ++ci) {
    const float* sc = sin_ + ci * kHalo;
#pragma unroll
    for (int t = 0; t < 27; ++t) {
      const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
      const float v = sc[((tz + dz) * kHY + (ty + dy)) * kHX + (tx + dx)];
#pragma unroll
      for (int co = 0; co < CO; ++co) acc[co] = fmaf(sw[(co * CI + ci) * 27 + t], v, acc[co]);
    }
  }
  const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
  if (x >= d.nx || y >= d.ny || z >= d.nz) return;
  const int64_t p = ((int64_t)z * d.ny + y) * d.nx + x;
#pragma unroll
  for (int co = 0; co < CO; ++co) {
    float v = acc[co];
    if (RELU) v = fmaxf(v, 0.f);
    if (mask && !(__bfloat162float(mask[co * d.ng + p]) > 0.f)) v = 0.f;
    from_f(v, &out[co * d.ng + p]);
  }
}

// gw[co][ci][tap] += sum_p g[co][p] in[ci][p + tap - 1]
template <int CI, int CO, typename TI>
__global__ void __launch_bounds__(256) k_conv_gw(const TI* __restrict__ in, const float* __restrict__ g,
                                                 float* __restrict__ gw, Dims d) {
  extern __shared__ float sm[];
  float* sg = sm;                 // [CO][256]
  float* sin_ = sm + CO * 256;    // [CI][halo]
  const int tile = blockIdx.x;
  const int x0 = (tile % d.tx) * kTX, y0 = (tile / d.tx) * kTY, z0 = blockIdx.y * kTZ;
  load_halo<CI>(in, d, x0, y0, z0, sin_);
  for (int i = threadIdx.x; i < CO * 256; i += blockDim.x) {
    const int co = i / 256, q = i % 256;
    const int tx = q % kTX, ty = (q / kTX) % kTY, tz = q / (kTX * kTY);
    const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
    float v = 0.f;
    if (x < d.nx && y < d.ny && z < d.nz) v = g[co * d.ng + ((int64_t)z * d.ny + y) * d.nx + x];
    sg[i] = v;
  }
  __syncthreads();
  for (int tr = threadIdx.x; tr < CO * CI * 27; tr += blockDim.x) {
    const int t = tr % 27, ci = (tr / 27) % CI, co = tr / (27 * CI);
    const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
    const float* sc = sin_ + ci * kHalo;
    const float* gg = sg + co * 256;
    float acc = 0.f;
    for (int q = 0; q < 256; ++q) {
      const int tx = q % kTX, ty = (q / kTX) % kTY, tz = q / (kTX * kTY);
      acc = fmaf(gg[q], sc[((tz + dz) * kHY + (ty + dy)) * kHX + (tx + dx)], acc);
    }
    atomicAdd(&gw[tr], acc);
  }
}

// wt[ci][co][26 - t] = w[co][ci][t] (transposed, flipped kernel of the backward-data pass)
__global__ void k_flip(const float* w, int CI, int CO, float* wt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= CI * CO * 27) return;
  int t = i % 27, ci = (i / 27) % CI, co = i / (27 * CI);
  wt[(ci * CO + co) * 27 + (26 - t)] = __bfloat162float(__float2bfloat16(w[i]));
}

__global__ void k_adam(float* w, float* m, float* v, const float* g, int n, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gi = g[i];
  float mi = b1 * m[i] + (1.f - b1) * gi, vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ---------------------------------------------------------------------------------------
// grid <-> channels
// ---------------------------------------------------------------------------------------
__global__ void k_sumsq(const float2* s, int64_t n, float* out) {
  float acc = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += s[i].x * s[i].x + s[i].y * s[i].y;
  acc = warp_sum(make_float2(acc, 0.f)).x;
  if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}
// x[2c][p] = Re sigma_c(p) / rms, x[2c+1][p] = Im sigma_c(p) / rms (rms over all 8 channels)
__global__ void k_pack(const float2* sig, const float* sumsq, int64_t ng, __nv_bfloat16* x) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= 4 * ng) return;
  const float rms = sqrtf(fmaxf(*sumsq, 1e-30f) / (8.f * ng));
  const int64_t c = i / ng, p = i - c * ng;
  x[2 * c * ng + p] = __float2bfloat16(sig[i].x / rms);
  x[(2 * c + 1) * ng + p] = __float2bfloat16(sig[i].y / rms);
}
// phi_c(p) = rms (out[2c][p] + i out[2c+1][p])
__global__ void k_unpack(const float* out, const float* sumsq, int64_t ng, float2* phi) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= 4 * ng) return;
  const float rms = sqrtf(fmaxf(*sumsq, 1e-30f) / (8.f * ng));
  const int64_t c = i / ng, p = i - c * ng;
  phi[i] = make_float2(rms * out[2 * c * ng + p], rms * out[(2 * c + 1) * ng + p]);
}
// g_out[2c][p] = rms Re gphi_c(p) * scale, g_out[2c+1][p] = rms Im gphi_c(p) * scale
__global__ void k_pack_grad(const float2* gphi, const float* sumsq, const float* tnorm2, int64_t ng,
                            float* g) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= 4 * ng) return;
  const float rms = sqrtf(fmaxf(*sumsq, 1e-30f) / (8.f * ng));
  const float sc = 2.f * rms / fmaxf(*tnorm2, 1e-30f);
  const int64_t c = i / ng, p = i - c * ng;
  g[2 * c * ng + p] = sc * gphi[i].x;
  g[(2 * c + 1) * ng + p] = sc * gphi[i].y;
}
__global__ void k_axpy_c(const float2* a, const float2* b, float sb, int n, float2* o) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) o[i] = make_float2(a[i].x + sb * b[i].x, a[i].y + sb * b[i].y);
}

// ---------------------------------------------------------------------------------------
// network state
// ---------------------------------------------------------------------------------------
struct Net {
  int nw = 0;
  float *w = nullptr, *m = nullptr, *v = nullptr, *g = nullptr, *wt = nullptr;
  __nv_bfloat16* act[kLayers] = {nullptr, nullptr, nullptr, nullptr};  // x, h1, h2, h3
  float* out = nullptr;      // [8][ng]
  float* gbuf[2] = {nullptr, nullptr};  // [16][ng] gradients
  float* scal = nullptr;     // [0] sumsq of the input grid, [1..2] |e|^2, |t|^2
  float2 *sig = nullptr, *phi = nullptr, *g2 = nullptr;  // [4][ng]
  float2 *x = nullptr, *r = nullptr, *t = nullptr, *u = nullptr, *e = nullptr;  // [N]
  int adam_t = 0;
  std::vector<void*> mem;
  ~Net() { for (void* p : mem) cudaFree(p); }
  template <typename T> int alloc(T** p, size_t n) {
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T) + 16);
    if (e != cudaSuccess) { set_error("net allocation: %s", cudaGetErrorString(e)); return BEM_ENOMEM; }
    mem.push_back(*p);
    return BEM_OK;
  }
};

static Dims dims_of(int nx, int ny, int nz) {
  Dims d;
  d.nx = nx; d.ny = ny; d.nz = nz;
  d.ng = (int64_t)nx * ny * nz;
  d.tx = (nx + kTX - 1) / kTX;
  d.ty = (ny + kTY - 1) / kTY;
  return d;
}

static size_t conv_smem(int CI, int CO) { return ((size_t)CO * CI * 27 + (size_t)CI * kHalo) * 4; }
static size_t gw_smem(int CI, int CO) { return ((size_t)CO * 256 + (size_t)CI * kHalo) * 4; }

template <int CI, int CO, typename TI, typename TO, bool RELU>
static int launch_conv(const TI* in, const float* w, TO* out, const __nv_bfloat16* mask, const Dims& d,
                       int round_w, cudaStream_t s) {
  static bool attr = false;
  const size_t sm = conv_smem(CI, CO);
  if (!attr) {
    BEM_CUDA(cudaFuncSetAttribute(k_conv<CI, CO, TI, TO, RELU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    attr = true;
  }
  dim3 grid(d.tx * d.ty, (d.nz + kTZ - 1) / kTZ);
  k_conv<CI, CO, TI, TO, RELU><<<grid, 256, sm, s>>>(in, w, out, mask, d, round_w);
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

template <int CI, int CO, typename TI>
static int launch_gw(const TI* in, const float* g, float* gw, const Dims& d, cudaStream_t s) {
  static bool attr = false;
  const size_t sm = gw_smem(CI, CO);
  if (!attr) {
    BEM_CUDA(cudaFuncSetAttribute(k_conv_gw<CI, CO, TI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    attr = true;
  }
  dim3 grid(d.tx * d.ty, (d.nz + kTZ - 1) / kTZ);
  k_conv_gw<CI, CO, TI><<<grid, 256, sm, s>>>(in, g, gw, d);
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

// forward: act[0] = x (BF16) given; act[1..3] = ReLU layers (BF16); out (FP32)
static int net_forward(Net& n, const Dims& d, cudaStream_t s) {
  const float* w = n.w;
  BEM_TRY((launch_conv<8, 16, __nv_bfloat16, __nv_bfloat16, true>(n.act[0], w + woffset(0), n.act[1], nullptr, d, 1, s)));
  BEM_TRY((launch_conv<16, 16, __nv_bfloat16, __nv_bfloat16, true>(n.act[1], w + woffset(1), n.act[2], nullptr, d, 1, s)));
  BEM_TRY((launch_conv<16, 16, __nv_bfloat16, __nv_bfloat16, true>(n.act[2], w + woffset(2), n.act[3], nullptr, d, 1, s)));
  BEM_TRY((launch_conv<16, 8, __nv_bfloat16, float, false>(n.act[3], w + woffset(3), n.out, nullptr, d, 1, s)));
  return BEM_OK;
}

// backward from gout = dL/d(out) (FP32 [8][ng]) in n.gbuf[0]; accumulates n.g; returns dL/dx in
// gx (FP32 [8][ng]) when gx != nullptr
static int net_backward(Net& n, const Dims& d, float* gx, cudaStream_t s) {
  float* g0 = n.gbuf[0];
  float* g1 = n.gbuf[1];
  // layer 3: 16 -> 8
  BEM_TRY((launch_gw<16, 8, __nv_bfloat16>(n.act[3], g0, n.g + woffset(3), d, s)));
  k_flip<<<(wcount(3) + 255) / 256, 256, 0, s>>>(n.w + woffset(3), 16, 8, n.wt);
  BEM_TRY((launch_conv<8, 16, float, float, false>(g0, n.wt, g1, n.act[3], d, 0, s)));
  // layer 2: 16 -> 16
  BEM_TRY((launch_gw<16, 16, __nv_bfloat16>(n.act[2], g1, n.g + woffset(2), d, s)));
  k_flip<<<(wcount(2) + 255) / 256, 256, 0, s>>>(n.w + woffset(2), 16, 16, n.wt);
  BEM_TRY((launch_conv<16, 16, float, float, false>(g1, n.wt, g0, n.act[2], d, 0, s)));
  // layer 1: 16 -> 16
  BEM_TRY((launch_gw<16, 16, __nv_bfloat16>(n.act[1], g0, n.g + woffset(1), d, s)));
  k_flip<<<(wcount(1) + 255) / 256, 256, 0, s>>>(n.w + woffset(1), 16, 16, n.wt);
  BEM_TRY((launch_conv<16, 16, float, float, false>(g0, n.wt, g1, n.act[1], d, 0, s)));
  // layer 0: 8 -> 16
  BEM_TRY((launch_gw<8, 16, __nv_bfloat16>(n.act[0], g1, n.g + woffset(0), d, s)));
  if (gx) {
    k_flip<<<(wcount(0) + 255) / 256, 256, 0, s>>>(n.w + woffset(0), 8, 16, n.wt);
    BEM_TRY((launch_conv<16, 8, float, float, false>(g1, n.wt, gx, nullptr, d, 0, s)));
  }
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

static int net_alloc_grid(Net& n, int64_t ng) {
  BEM_TRY(n.alloc(&n.act[0], 8 * (size_t)ng));
  for (int l = 1; l < kLayers; ++l) BEM_TRY(n.alloc(&n.act[l], 16 * (size_t)ng));
  BEM_TRY(n.alloc(&n.out, 8 * (size_t)ng));
  BEM_TRY(n.alloc(&n.gbuf[0], 16 * (size_t)ng));
  BEM_TRY(n.alloc(&n.gbuf[1], 16 * (size_t)ng));
  BEM_TRY(n.alloc(&n.wt, (size_t)16 * 16 * 27));
  return BEM_OK;
}

static int net_alloc_weights(Net& n) {
  n.nw = wtotal();
  BEM_TRY(n.alloc(&n.w, n.nw));
  BEM_TRY(n.alloc(&n.m, n.nw));
  BEM_TRY(n.alloc(&n.v, n.nw));
  BEM_TRY(n.alloc(&n.g, n.nw));
  BEM_CUDA(cudaMemset(n.m, 0, n.nw * sizeof(float)));
  BEM_CUDA(cudaMemset(n.v, 0, n.nw * sizeof(float)));
  return BEM_OK;
}

static Net* get_net(aim_ctx* c, int* rc) {
  *rc = BEM_OK;
  if (c->net) return static_cast<Net*>(c->net);
  Net* n = new Net();
  *rc = net_alloc_weights(*n);
  if (*rc == BEM_OK) *rc = net_alloc_grid(*n, c->ng);
  const size_t N = (size_t)c->ne + c->nt;
  if (*rc == BEM_OK) *rc = n->alloc(&n->scal, 8);
  if (*rc == BEM_OK) *rc = n->alloc(&n->sig, 4 * (size_t)c->ng);
  if (*rc == BEM_OK) *rc = n->alloc(&n->phi, 4 * (size_t)c->ng);
  if (*rc == BEM_OK) *rc = n->alloc(&n->g2, 4 * (size_t)c->ng);
  for (float2** p : {&n->x, &n->r, &n->t, &n->u, &n->e})
    if (*rc == BEM_OK) *rc = n->alloc(p, N);
  if (*rc != BEM_OK) {
    delete n;
    return nullptr;
  }
  c->net = n;
  return n;
}

void free_net(aim_ctx* c) {
  delete static_cast<Net*>(c->net);
  c->net = nullptr;
}

// u = W net(P r) (FP32), using the context's grid; scal[0] holds the input grid's sum of squares
static int net_correction(aim_ctx* c, Net& n, const float2* r, float2* u, cudaStream_t s) {
  const Dims d = dims_of(c->gn[0], c->gn[1], c->gn[2]);
  BEM_TRY(project_all<float>(c, r, n.sig, s));
  BEM_CUDA(cudaMemsetAsync(n.scal, 0, sizeof(float), s));
  k_sumsq<<<304, 256, 0, s>>>(n.sig, 4 * c->ng, n.scal);
  k_pack<<<(unsigned)((4 * c->ng + 255) / 256), 256, 0, s>>>(n.sig, n.scal, c->ng, n.act[0]);
  BEM_TRY(net_forward(n, d, s));
  k_unpack<<<(unsigned)((4 * c->ng + 255) / 256), 256, 0, s>>>(n.out, n.scal, c->ng, n.phi);
  BEM_TRY(interp_all<float>(c, n.phi, u, s));
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

int net_apply(aim_ctx* c, const float2* r, float2* z, cudaStream_t s) {
  int rc = BEM_OK;
  Net* n = get_net(c, &rc);
  if (!n) return rc;
  const int N = c->ne + c->nt;
  BEM_TRY(setup_precond(c));
  BEM_TRY(precond_apply<float>(c, r, z, s));
  BEM_TRY(net_correction(c, *n, r, n->u, s));
  k_axpy_c<<<(N + 255) / 256, 256, 0, s>>>(z, n->u, 1.f, N, z);
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

// one training step over `batch` fresh pairs; returns the mean relative loss
static int net_train_step(aim_ctx* c, Net& n, int batch, float lr, uint64_t seed, float* loss,
                          cudaStream_t s) {
  const Dims d = dims_of(c->gn[0], c->gn[1], c->gn[2]);
  const int N = c->ne + c->nt;
  BEM_CUDA(cudaMemsetAsync(n.g, 0, n.nw * sizeof(float), s));
  double lsum = 0;
  for (int b = 0; b < batch; ++b) {
    if (b % 2 == 0) {
      // white x
      k_randn_c<<<(N + 255) / 256, 256, 0, s>>>(splitmix64(seed * 7919ull + b), N, n.x);
    } else {
      // smooth x: grid potentials of random grid sources, interpolated to the unknowns
      const int64_t n4 = 4 * c->ng;
      k_randn_c<<<(unsigned)((n4 + 255) / 256), 256, 0, s>>>(splitmix64(seed * 7919ull + b), (int)n4,
                                                             n.sig);
      BEM_TRY(fft_conv<float>(c, c->f32, n.sig, n.phi, 4, c->f32.ws, s));
      BEM_TRY(interp_all<float>(c, n.phi, n.x, s));
    }
    BEM_TRY(matvec_graph<float>(c, AIM_OP_SYSTEM, n.x, n.r, s));          // r = A x
    BEM_TRY(precond_apply<float>(c, n.r, n.t, s));                        // t = M_bd r
    k_axpy_c<<<(N + 255) / 256, 256, 0, s>>>(n.x, n.t, -1.f, N, n.t);     // t = x - M_bd r
    BEM_TRY(net_correction(c, n, n.r, n.u, s));                           // u = W net(P r)
    // loss |P e|^2 / |P t|^2 with e = u - t: the error measured on the grid, where the
    // correction lives; gradient w.r.t. the output grid = 2 P W P e / |P t|^2
    BEM_CUDA(cudaMemsetAsync(n.scal + 1, 0, 2 * sizeof(float), s));
    k_axpy_c<<<(N + 255) / 256, 256, 0, s>>>(n.u, n.t, -1.f, N, n.e);     // e = u - t
    BEM_TRY(project_all<float>(c, n.e, n.phi, s));                         // P e
    BEM_TRY(project_all<float>(c, n.t, n.g2, s));                          // P t
    k_sumsq<<<304, 256, 0, s>>>(n.phi, 4 * c->ng, n.scal + 1);
    k_sumsq<<<304, 256, 0, s>>>(n.g2, 4 * c->ng, n.scal + 2);
    BEM_TRY(interp_all<float>(c, n.phi, n.e, s));                          // W P e
    BEM_TRY(project_all<float>(c, n.e, n.phi, s));                         // P W P e
    k_pack_grad<<<(unsigned)((4 * c->ng + 255) / 256), 256, 0, s>>>(n.phi, n.scal, n.scal + 2,
                                                                        c->ng, n.gbuf[0]);
    BEM_TRY(net_backward(n, d, nullptr, s));
    float h[2];
    BEM_CUDA(cudaMemcpyAsync(h, n.scal + 1, 2 * sizeof(float), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaStreamSynchronize(s));
    lsum += h[0] / std::max(h[1], 1e-30f);
  }
  // Adam on the batch-summed gradient: the step m/sqrt(v) does not change when the gradient is
  // scaled, so summing instead of averaging only rescales eps (passed as eps * batch)
  ++n.adam_t;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)n.adam_t), c2 = 1.f - std::pow(b2, (float)n.adam_t);
  k_adam<<<(n.nw + 255) / 256, 256, 0, s>>>(n.w, n.m, n.v, n.g, n.nw, lr, b1, b2, 1e-8f * batch,
                                            c1, c2);
  BEM_CUDA(cudaGetLastError());
  *loss = (float)(lsum / batch);
  return BEM_OK;
}

}  // namespace bem

using namespace bem;

extern "C" {

int bem_net_init(aim_ctx* c, uint64_t seed) {
  if (!c) { set_error("bem_net_init: null context"); return BEM_EINVAL; }
  int rc = BEM_OK;
  Net* n = get_net(c, &rc);
  if (!n) return rc;
  std::vector<float> w(n->nw);
  int o = 0;
  for (int l = 0; l < kLayers; ++l) {
    const double sd = std::sqrt(2.0 / (27.0 * kCh[l]));
    for (int i = 0; i < wcount(l); ++i, ++o) {
      double u1 = u01(splitmix64(seed ^ (2ull * o))), u2 = u01(splitmix64(seed ^ (2ull * o + 1)));
      w[o] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2));
    }
  }
  BEM_CUDA(cudaMemcpy(n->w, w.data(), n->nw * sizeof(float), cudaMemcpyHostToDevice));
  BEM_CUDA(cudaMemset(n->m, 0, n->nw * sizeof(float)));
  BEM_CUDA(cudaMemset(n->v, 0, n->nw * sizeof(float)));
  n->adam_t = 0;
  return BEM_OK;
}

int64_t bem_net_weights(aim_ctx* c, float* w, int64_t n, int set) {
  if (!c) { set_error("bem_net_weights: null context"); return BEM_EINVAL; }
  int rc = BEM_OK;
  Net* net = get_net(c, &rc);
  if (!net) return rc;
  if (!w) return net->nw;
  if (n != net->nw) { set_error("bem_net_weights: expected %d weights", net->nw); return BEM_EINVAL; }
  if (set) {
    BEM_CUDA(cudaMemcpy(net->w, w, n * sizeof(float), cudaMemcpyHostToDevice));
    BEM_CUDA(cudaMemset(net->m, 0, n * sizeof(float)));
    BEM_CUDA(cudaMemset(net->v, 0, n * sizeof(float)));
    net->adam_t = 0;
  } else {
    BEM_CUDA(cudaMemcpy(w, net->w, n * sizeof(float), cudaMemcpyDeviceToHost));
  }
  return n;
}

int bem_net_train(aim_ctx* c, int steps, int batch, float lr, uint64_t seed, float* losses,
                  void* stream) {
  if (!c || steps < 1 || batch < 1 || !(lr > 0)) {
    set_error("bem_net_train: bad arguments");
    return BEM_EINVAL;
  }
  int rc = BEM_OK;
  Net* n = get_net(c, &rc);
  if (!n) return rc;
  // the targets x - M_bd A x hold M_bd's own error A_ii^{-1} - X_ii: with inverses built in FP32
  // that is the FP32 LU's error (left residual ~ cond * eps), mesh-scale noise no grid
  // correction can learn, so training builds them in FP64
  BEM_TRY(setup_precond(c, BEM_C64));
  cudaStream_t s = (cudaStream_t)stream;
  for (int k = 0; k < steps; ++k) {
    float l = 0;
    BEM_TRY(net_train_step(c, *n, batch, lr, splitmix64(seed + 1000003ull * k), &l, s));
    if (losses) losses[k] = l;
  }
  return BEM_OK;
}

int bem_net_apply(aim_ctx* c, const void* r, void* z, int correction_only, void* stream) {
  if (!c || !r || !z || r == z) {
    set_error("bem_net_apply: bad arguments");
    return BEM_EINVAL;
  }
  if (!correction_only) return net_apply(c, (const float2*)r, (float2*)z, (cudaStream_t)stream);
  int rc = BEM_OK;
  Net* n = get_net(c, &rc);
  if (!n) return rc;
  return net_correction(c, *n, (const float2*)r, (float2*)z, (cudaStream_t)stream);
}

// Standalone network pass for verification: x [8][ng] FP32 (rounded to BF16 on entry), weights
// FP32 host (rounded to BF16 in the kernels), out [8][ng] FP32; with gout [8][ng] the backward
// pass writes gw (host, FP32, layers one after another) and gx [8][ng] (device).
int bem_convnet_run(int nx, int ny, int nz, const float* w_host, const float* x, const float* gout,
                    float* out, float* gw_host, float* gx, void* stream) {
  if (nx < 1 || ny < 1 || nz < 1 || !w_host || !x || !out) {
    set_error("bem_convnet_run: bad arguments");
    return BEM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  Net n;
  const Dims d = dims_of(nx, ny, nz);
  BEM_TRY(net_alloc_weights(n));
  BEM_TRY(net_alloc_grid(n, d.ng));
  BEM_CUDA(cudaMemcpyAsync(n.w, w_host, n.nw * sizeof(float), cudaMemcpyHostToDevice, s));
  {
    std::vector<float> hx(8 * (size_t)d.ng);
    std::vector<__nv_bfloat16> hb(hx.size());
    BEM_CUDA(cudaMemcpyAsync(hx.data(), x, hx.size() * 4, cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaStreamSynchronize(s));
    for (size_t i = 0; i < hx.size(); ++i) hb[i] = __float2bfloat16(hx[i]);
    BEM_CUDA(cudaMemcpyAsync(n.act[0], hb.data(), hb.size() * 2, cudaMemcpyHostToDevice, s));
    BEM_CUDA(cudaStreamSynchronize(s));
  }
  BEM_TRY(net_forward(n, d, s));
  BEM_CUDA(cudaMemcpyAsync(out, n.out, 8 * d.ng * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (gout) {
    BEM_CUDA(cudaMemsetAsync(n.g, 0, n.nw * sizeof(float), s));
    BEM_CUDA(cudaMemcpyAsync(n.gbuf[0], gout, 8 * d.ng * sizeof(float), cudaMemcpyDeviceToDevice, s));
    BEM_TRY(net_backward(n, d, gx, s));
    if (gw_host) BEM_CUDA(cudaMemcpyAsync(gw_host, n.g, n.nw * sizeof(float), cudaMemcpyDeviceToHost, s));
  }
  BEM_CUDA(cudaStreamSynchronize(s));
  return BEM_OK;
}

}  // extern "C"
