// The grid step H of the adaptive integral method (Sec. III-A item 1, Eq. AIM_L): linear
// convolution of the grid sources with the grid Green's function by zero-padded FFTs.
//
// Layout: grid data [comp][nz][ny][nx] (x fastest); padded workspace [comp][Pz][Py][Px] with
// P >= 2n - 1 per axis (factors 2, 3, 5, 7). The convolution runs as five batched 1-D passes
// that skip the zero padding:
//   X forward  : ny*nz lines of nx inputs  -> Px outputs
//   Y forward  : Px*nz lines of ny inputs  -> Py outputs
//   Z fused    : Px*Py lines: forward FFT of nz inputs, times Ghat, inverse FFT, nz outputs
//   Y inverse  : Px*nz lines of Py inputs  -> ny outputs
//   X inverse  : ny*nz lines of Px inputs  -> nx outputs
// Ghat is stored as one octant (the circulant kernel is even along every axis) with the
// 1/(Px Py Pz) normalisation folded in. Each pass stages TL lines in shared memory and runs a
// Stockham autosort FFT (mixed radix 4, 2, 3, 5, 7; twiddles from a per-axis table).
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace bem {

bool make_fft_plan(int P, FftPlan* plan) {
  plan->P = P;
  plan->nst = 0;
  int n = P;
  const int rads[5] = {4, 2, 3, 5, 7};
  for (int r : rads)
    while (n % r == 0) {
      if (plan->nst >= kMaxStages) return false;
      plan->rad[plan->nst++] = r;
      n /= r;
    }
  return n == 1 && P >= 1;
}

int smooth_length(int need) {
  for (int m = std::max(need, 1);; ++m) {
    int n = m;
    for (int r : {2, 3, 5, 7})
      while (n % r == 0) n /= r;
    if (n == 1) return m;
  }
}

struct LinePass {
  int P, nin, nout;
  int64_t ies, oes;
  int n0, n1;
  int64_t is0, is1, is2;
  int64_t os0, os1, os2;
  int fused;        // 1: forward, multiply by Ghat, inverse
  int inverse;      // plain pass direction
  int TL;           // lines per CTA
  int gx, gy;       // octant dims (Px/2+1, Py/2+1) for the fused pass
  int Px, Py;
  FftPlan plan;
};

template <typename V>
__device__ __forceinline__ V tw_get(const V* tw, int idx, bool inv) {
  V w = tw[idx];
  if (inv) w.y = -w.y;
  return w;
}

// one Stockham stage on TL lines: src -> dst
template <typename V>
__device__ __forceinline__ void stage(const V* src, V* dst, const V* tw, int P, int TL, int R,
                                      int Ns, bool inv) {
  const int m = P / R;
  const int stride_tw = P / (Ns * R);
  for (int idx = threadIdx.x; idx < TL * m; idx += blockDim.x) {
    const int l = idx / m, j = idx - l * m;
    const V* s = src + (int64_t)l * P;
    V* d = dst + (int64_t)l * P;
    const int k = j % Ns;
    V v[7];
    for (int r = 0; r < R; ++r) {
      V x = s[j + r * m];
      if (Ns > 1 && r > 0) x = cmul(x, tw_get(tw, r * k * stride_tw, inv));
      v[r] = x;
    }
    const int base = (j / Ns) * Ns * R + k;
    if (R == 2) {
      d[base] = cadd(v[0], v[1]);
      d[base + Ns] = csub(v[0], v[1]);
    } else if (R == 4) {
      V y0 = cadd(v[0], v[2]), y1 = csub(v[0], v[2]), y2 = cadd(v[1], v[3]), y3 = csub(v[1], v[3]);
      // forward: y3 * (-i); inverse: y3 * (+i)
      y3 = inv ? mk(-y3.y, y3.x) : mk(y3.y, -y3.x);
      d[base] = cadd(y0, y2);
      d[base + Ns] = cadd(y1, y3);
      d[base + 2 * Ns] = csub(y0, y2);
      d[base + 3 * Ns] = csub(y1, y3);
    } else {
      const int step = P / R;  // e^{-2 pi i q / R} = tw[q * P / R]
      for (int q = 0; q < R; ++q) {
        V acc = v[0];
        for (int r = 1; r < R; ++r) acc = cadd(acc, cmul(v[r], tw_get(tw, ((r * q) % R) * step, inv)));
        d[base + q * Ns] = acc;
      }
    }
  }
}

template <typename V>
__device__ __forceinline__ V* run_stages(V* a, V* b, const V* tw, const LinePass& p, bool inv) {
  int Ns = 1;
  for (int st = 0; st < p.plan.nst; ++st) {
    const int R = p.plan.rad[st];
    stage(a, b, tw, p.P, p.TL, R, Ns, inv);
    __syncthreads();
    V* t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
}

template <typename V>
__global__ void __launch_bounds__(256) k_fft_lines(const V* in, V* out,
                                                   const V* __restrict__ twg, const V* __restrict__ ghat,
                                                   LinePass p) {
  extern __shared__ unsigned char smem_raw[];
  V* tw = reinterpret_cast<V*>(smem_raw);
  V* A = tw + p.P;
  V* B = A + (int64_t)p.TL * p.P;
  const int i0base = blockIdx.x * p.TL;
  const int i1 = blockIdx.y, i2 = blockIdx.z;
  const int nl = min(p.TL, p.n0 - i0base);
  for (int i = threadIdx.x; i < p.P; i += blockDim.x) tw[i] = twg[i];
  // load (zero padding beyond nin)
  const int64_t ib = i1 * p.is1 + i2 * p.is2;
  if (p.ies == 1) {
    for (int idx = threadIdx.x; idx < p.TL * p.P; idx += blockDim.x) {
      const int l = idx / p.P, e = idx - l * p.P;
      V v = czero<V>();
      if (l < nl && e < p.nin) v = in[ib + (int64_t)(i0base + l) * p.is0 + e];
      A[idx] = v;
    }
  } else {
    for (int idx = threadIdx.x; idx < p.TL * p.P; idx += blockDim.x) {
      const int e = idx / p.TL, l = idx - e * p.TL;
      V v = czero<V>();
      if (l < nl && e < p.nin) v = in[ib + (int64_t)(i0base + l) * p.is0 + (int64_t)e * p.ies];
      A[(int64_t)l * p.P + e] = v;
    }
  }
  __syncthreads();
  V* res;
  if (!p.fused) {
    res = run_stages(A, B, tw, p, p.inverse != 0);
  } else {
    res = run_stages(A, B, tw, p, false);
    // multiply by the octant of Ghat: line (x = i0, y = i1), element kz
    for (int idx = threadIdx.x; idx < p.TL * p.P; idx += blockDim.x) {
      const int l = idx / p.P, kz = idx - l * p.P;
      if (l >= nl) continue;
      const int x = i0base + l, y = i1;
      const int fx = min(x, p.Px - x), fy = min(y, p.Py - y), fz = min(kz, p.P - kz);
      res[idx] = cmul(res[idx], ghat[((int64_t)fz * p.gy + fy) * p.gx + fx]);
    }
    __syncthreads();
    V* other = (res == A) ? B : A;
    res = run_stages(res, other, tw, p, true);
  }
  // store the first nout outputs
  const int64_t ob = i1 * p.os1 + i2 * p.os2;
  if (p.oes == 1) {
    for (int idx = threadIdx.x; idx < p.TL * p.nout; idx += blockDim.x) {
      const int l = idx / p.nout, e = idx - l * p.nout;
      if (l < nl) out[ob + (int64_t)(i0base + l) * p.os0 + e] = res[(int64_t)l * p.P + e];
    }
  } else {
    for (int idx = threadIdx.x; idx < p.TL * p.nout; idx += blockDim.x) {
      const int e = idx / p.TL, l = idx - e * p.TL;
      if (l < nl) out[ob + (int64_t)(i0base + l) * p.os0 + (int64_t)e * p.oes] = res[(int64_t)l * p.P + e];
    }
  }
}

template <typename V>
static int launch_pass(const V* in, V* out, const V* tw, const V* ghat, LinePass p, int n2,
                       cudaStream_t s) {
  const size_t avail = 96 * 1024 / sizeof(V);  // complex elements of shared memory
  if (avail < 3 * (size_t)p.P) {
    set_error("FFT length %d too large for shared memory", p.P);
    return BEM_EGRID;
  }
  int TL = (int)std::min<size_t>(16, (avail - p.P) / (2 * (size_t)p.P));
  if (TL < 1) {
    set_error("FFT length %d too large for shared memory", p.P);
    return BEM_EGRID;
  }
  TL = std::min(TL, p.n0);
  p.TL = TL;
  size_t smem = ((size_t)p.P + 2 * (size_t)TL * p.P) * sizeof(V);
  dim3 grid((p.n0 + TL - 1) / TL, p.n1, n2);
  static bool attr_set[2] = {false, false};
  int which = sizeof(V) == 8 ? 0 : 1;
  if (!attr_set[which]) {
    BEM_CUDA(cudaFuncSetAttribute(k_fft_lines<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set[which] = true;
  }
  k_fft_lines<V><<<grid, 256, smem, s>>>(in, out, tw, ghat, p);
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

template <typename R>
int make_twiddles(aim_ctx* c, PrecBuf<R>& b) {
  typedef typename C2<R>::T V;
  for (int a = 0; a < 3; ++a) {
    const int P = c->gp[a];
    std::vector<V> t(P);
    for (int k = 0; k < P; ++k) {
      double ang = -2.0 * M_PI * (double)k / (double)P;
      t[k] = mk((R)std::cos(ang), (R)std::sin(ang));
    }
    BEM_TRY(upload(c, &b.tw[a], t.data(), t.size()));
  }
  return BEM_OK;
}
template int make_twiddles<float>(aim_ctx*, PrecBuf<float>&);
template int make_twiddles<double>(aim_ctx*, PrecBuf<double>&);

template <typename R>
int fft_conv(aim_ctx* c, PrecBuf<R>& b, const typename C2<R>::T* sigma, typename C2<R>::T* phi,
             int ncomp, cudaStream_t s) {
  typedef typename C2<R>::T V;
  const int nx = c->gn[0], ny = c->gn[1], nz = c->gn[2];
  const int Px = c->gp[0], Py = c->gp[1], Pz = c->gp[2];
  const int64_t P3 = (int64_t)Px * Py * Pz, ng = c->ng;
  V* ws = b.ws;
  LinePass p{};
  // X forward
  p = LinePass{};
  p.P = Px; p.nin = nx; p.nout = Px; p.ies = 1; p.oes = 1;
  p.n0 = ny; p.n1 = nz; p.is0 = nx; p.is1 = (int64_t)ny * nx; p.is2 = ng;
  p.os0 = Px; p.os1 = (int64_t)Py * Px; p.os2 = P3; p.plan = c->plan[0];
  BEM_TRY(launch_pass<V>(sigma, ws, b.tw[0], nullptr, p, ncomp, s));
  // Y forward
  p = LinePass{};
  p.P = Py; p.nin = ny; p.nout = Py; p.ies = Px; p.oes = Px;
  p.n0 = Px; p.n1 = nz; p.is0 = 1; p.is1 = (int64_t)Py * Px; p.is2 = P3;
  p.os0 = 1; p.os1 = (int64_t)Py * Px; p.os2 = P3; p.plan = c->plan[1];
  BEM_TRY(launch_pass<V>(ws, ws, b.tw[1], nullptr, p, ncomp, s));
  // Z forward * Ghat * Z inverse
  p = LinePass{};
  p.P = Pz; p.nin = nz; p.nout = nz; p.ies = (int64_t)Py * Px; p.oes = (int64_t)Py * Px;
  p.n0 = Px; p.n1 = Py; p.is0 = 1; p.is1 = Px; p.is2 = P3;
  p.os0 = 1; p.os1 = Px; p.os2 = P3; p.fused = 1; p.plan = c->plan[2];
  p.gx = Px / 2 + 1; p.gy = Py / 2 + 1; p.Px = Px; p.Py = Py;
  BEM_TRY(launch_pass<V>(ws, ws, b.tw[2], b.Ghat, p, ncomp, s));
  // Y inverse
  p = LinePass{};
  p.P = Py; p.nin = Py; p.nout = ny; p.ies = Px; p.oes = Px; p.inverse = 1;
  p.n0 = Px; p.n1 = nz; p.is0 = 1; p.is1 = (int64_t)Py * Px; p.is2 = P3;
  p.os0 = 1; p.os1 = (int64_t)Py * Px; p.os2 = P3; p.plan = c->plan[1];
  BEM_TRY(launch_pass<V>(ws, ws, b.tw[1], nullptr, p, ncomp, s));
  // X inverse
  p = LinePass{};
  p.P = Px; p.nin = Px; p.nout = nx; p.ies = 1; p.oes = 1; p.inverse = 1;
  p.n0 = ny; p.n1 = nz; p.is0 = Px; p.is1 = (int64_t)Py * Px; p.is2 = P3;
  p.os0 = nx; p.os1 = (int64_t)ny * nx; p.os2 = ng; p.plan = c->plan[0];
  BEM_TRY(launch_pass<V>(ws, phi, b.tw[0], nullptr, p, ncomp, s));
  return BEM_OK;
}
template int fft_conv<float>(aim_ctx*, PrecBuf<float>&, const float2*, float2*, int, cudaStream_t);
template int fft_conv<double>(aim_ctx*, PrecBuf<double>&, const double2*, double2*, int, cudaStream_t);

// circulant grid kernel: offset d along an axis of padded length P lives at index d mod P
__global__ void k_gcirc(double2* g, int Px, int Py, int Pz, int nx, int ny, int nz, double hx,
                        double hy, double hz, double k0) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)Px * Py * Pz) return;
  int ix = (int)(idx % Px), iy = (int)((idx / Px) % Py), iz = (int)(idx / ((int64_t)Px * Py));
  auto off = [](int i, int P, int n, bool* ok) {
    if (i < n) { *ok = true; return i; }
    if (i > P - n) { *ok = true; return i - P; }
    *ok = false;
    return 0;
  };
  bool ox, oy, oz;
  int dx = off(ix, Px, nx, &ox), dy = off(iy, Py, ny, &oy), dz = off(iz, Pz, nz, &oz);
  double2 v = make_double2(0, 0);
  if (ox && oy && oz) {
    double x = dx * hx, y = dy * hy, z = dz * hz;
    double R = sqrt(x * x + y * y + z * z);
    if (R > 0) {
      double s, co;
      sincos(k0 * R, &s, &co);
      double a = 1.0 / (4.0 * 3.14159265358979323846 * R);
      v = make_double2(co * a, -s * a);
    }
  }
  g[idx] = v;
}

__global__ void k_ghat_oct(const double2* G, int Px, int Py, int Pz, double scale, double2* o64,
                           float2* o32) {
  const int gx = Px / 2 + 1, gy = Py / 2 + 1, gz = Pz / 2 + 1;
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)gx * gy * gz) return;
  int x = (int)(idx % gx), y = (int)((idx / gx) % gy), z = (int)(idx / ((int64_t)gx * gy));
  double2 v = G[((int64_t)z * Py + y) * Px + x];
  v.x *= scale;
  v.y *= scale;
  o64[idx] = v;
  o32[idx] = make_float2((float)v.x, (float)v.y);
}

int make_ghat(aim_ctx* c) {
  const int Px = c->gp[0], Py = c->gp[1], Pz = c->gp[2];
  const int64_t P3 = (int64_t)Px * Py * Pz;
  double2* G = nullptr;
  BEM_CUDA(cudaMalloc(&G, P3 * sizeof(double2)));
  k_gcirc<<<(unsigned)((P3 + 255) / 256), 256>>>(G, Px, Py, Pz, c->gn[0], c->gn[1], c->gn[2],
                                                c->gh[0], c->gh[1], c->gh[2], c->k0);
  int rc = BEM_OK;
  LinePass p{};
  // full forward FFT along x, y, z
  p.P = Px; p.nin = Px; p.nout = Px; p.ies = 1; p.oes = 1;
  p.n0 = Py; p.n1 = Pz; p.is0 = Px; p.is1 = (int64_t)Py * Px; p.is2 = P3;
  p.os0 = Px; p.os1 = (int64_t)Py * Px; p.os2 = P3; p.plan = c->plan[0];
  rc = launch_pass<double2>(G, G, c->f64.tw[0], nullptr, p, 1, 0);
  if (rc == BEM_OK) {
    p = LinePass{};
    p.P = Py; p.nin = Py; p.nout = Py; p.ies = Px; p.oes = Px;
    p.n0 = Px; p.n1 = Pz; p.is0 = 1; p.is1 = (int64_t)Py * Px; p.is2 = P3;
    p.os0 = 1; p.os1 = (int64_t)Py * Px; p.os2 = P3; p.plan = c->plan[1];
    rc = launch_pass<double2>(G, G, c->f64.tw[1], nullptr, p, 1, 0);
  }
  if (rc == BEM_OK) {
    p = LinePass{};
    p.P = Pz; p.nin = Pz; p.nout = Pz; p.ies = (int64_t)Py * Px; p.oes = (int64_t)Py * Px;
    p.n0 = Px; p.n1 = Py; p.is0 = 1; p.is1 = Px; p.is2 = P3;
    p.os0 = 1; p.os1 = Px; p.os2 = P3; p.plan = c->plan[2];
    rc = launch_pass<double2>(G, G, c->f64.tw[2], nullptr, p, 1, 0);
  }
  const int64_t no = (int64_t)(Px / 2 + 1) * (Py / 2 + 1) * (Pz / 2 + 1);
  if (rc == BEM_OK) rc = dalloc_t(c, &c->f64.Ghat, no);
  if (rc == BEM_OK) rc = dalloc_t(c, &c->f32.Ghat, no);
  if (rc == BEM_OK) {
    k_ghat_oct<<<(unsigned)((no + 255) / 256), 256>>>(G, Px, Py, Pz, 1.0 / (double)P3, c->f64.Ghat,
                                                      c->f32.Ghat);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
      set_error("make_ghat: %s", cudaGetErrorString(e));
      rc = BEM_ECUDA;
    }
  }
  cudaFree(G);
  return rc;
}

}  // namespace bem
