// The grid step H of the adaptive integral method (Sec. III-A item 1, Eq. AIM_L): linear
// convolution of the grid sources with the grid Green's function by zero-padded FFTs.
//
// Layout: grid data [comp][nz][ny][nx] (x fastest); padded workspace [comp][Pz][Py][Px] with
// P >= 2n - 1 per axis (factors 2, 3, 5). When one padded x-y plane fits in shared memory the
// convolution is three passes that skip the zero padding:
//   plane forward : per z < nz, load the nx*ny plane, FFT the ny non-zero rows (length Px) and
//                   then all Px columns (length Py), store the Px*Py plane
//   z fused       : per (x, y), forward FFT of the nz planes (length Pz), times Ghat, inverse
//                   FFT, store the first nz outputs
//   plane inverse : per z < nz, inverse FFT of all columns, then of the ny rows that are kept,
//                   store the nx*ny plane
// Larger planes fall back to five batched 1-D passes (x, y, z-fused, y, x) with the same
// pruning. Ghat is one octant (the circulant kernel is even along every axis) with the
// 1/(Px Py Pz) normalisation folded in. Every transform is a Stockham autosort FFT in shared
// memory with radix-8/4/2/3/5 butterflies and twiddles from a per-axis table. Index divisions
// use precomputed multiply-high constants, and element e of a line is stored at e + e/16 so
// the strided stores of the early stages spread over the shared-memory banks.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace bem {

bool make_fft_plan(int P, FftPlan* plan) {
  plan->P = P;
  plan->nst = 0;
  int n = P;
  const int rads[5] = {8, 4, 2, 3, 5};
  for (int r : rads)
    while (n % r == 0) {
      if (plan->nst >= kMaxStages) return false;
      plan->rad[plan->nst++] = r;
      n /= r;
    }
  if (n != 1 || P < 1 || P >= 2048) return false;
  int Ns = 1;
  for (int s = 0; s < plan->nst; ++s) {
    plan->mag_m[s] = div_magic(P / plan->rad[s]);
    plan->mag_ns[s] = div_magic(Ns);
    Ns *= plan->rad[s];
  }
  return true;
}

// the slab passes' plans: radix-32 stages first (two stages for 1024 points), then the others
bool make_fft_plan_r32(int P, FftPlan* plan) {
  plan->P = P;
  plan->nst = 0;
  int n = P;
  const int rads[6] = {32, 8, 4, 2, 3, 5};
  for (int r : rads)
    while (n % r == 0) {
      if (plan->nst >= kMaxStages) return false;
      plan->rad[plan->nst++] = r;
      n /= r;
    }
  if (n != 1 || P < 1 || P >= 2048) return false;
  int Ns = 1;
  for (int s = 0; s < plan->nst; ++s) {
    plan->mag_m[s] = div_magic(P / plan->rad[s]);
    plan->mag_ns[s] = div_magic(Ns);
    Ns *= plan->rad[s];
  }
  return true;
}

int smooth_length(int need) {
  for (int m = std::max(need, 1);; ++m) {
    int n = m;
    for (int r : {2, 3, 5})
      while (n % r == 0) n /= r;
    if (n == 1) return m;
  }
}

// ---------------------------------------------------------------------------------------
// butterflies (forward: exp(-2 pi i / R); inverse: conjugate)
// ---------------------------------------------------------------------------------------
template <typename V> __device__ __forceinline__ V mul_mi(V a, bool inv) {  // * (-i) or * (+i)
  return inv ? mk(-a.y, a.x) : mk(a.y, -a.x);
}

template <typename V> __device__ __forceinline__ void bfly2(V* v) {
  V a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <typename V> __device__ __forceinline__ void bfly3(V* v, bool inv) {
  typedef decltype(v[0].x) R;
  const R h = (R)0.86602540378443864676;  // sin(2 pi / 3)
  V t1 = cadd(v[1], v[2]);
  V d = csub(v[1], v[2]);
  V t2 = mul_mi(mk(h * d.x, h * d.y), inv);
  V m = mk(v[0].x - (R)0.5 * t1.x, v[0].y - (R)0.5 * t1.y);
  v[0] = cadd(v[0], t1);
  v[1] = cadd(m, t2);
  v[2] = csub(m, t2);
}

template <typename V> __device__ __forceinline__ void bfly4(V* v, bool inv) {
  V y0 = cadd(v[0], v[2]), y1 = csub(v[0], v[2]), y2 = cadd(v[1], v[3]);
  V y3 = mul_mi(csub(v[1], v[3]), inv);
  v[0] = cadd(y0, y2);
  v[1] = cadd(y1, y3);
  v[2] = csub(y0, y2);
  v[3] = csub(y1, y3);
}

template <typename V> __device__ __forceinline__ void bfly5(V* v, bool inv) {
  typedef decltype(v[0].x) R;
  const R c1 = (R)0.30901699437494742410, c2 = (R)-0.80901699437494742410;  // cos 2pi/5, 4pi/5
  const R s1 = (R)0.95105651629515357212, s2 = (R)0.58778525229247312917;   // sin 2pi/5, 4pi/5
  V t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]), t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
  V a1 = mk(v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y);
  V a2 = mk(v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y);
  V b1 = mk(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y);
  V b2 = mk(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y);
  V ib1 = mul_mi(b1, inv), ib2 = mul_mi(b2, inv);  // (-i) b forward
  v[0] = cadd(v[0], cadd(t1, t2));
  v[1] = cadd(a1, ib1);
  v[4] = csub(a1, ib1);
  v[2] = cadd(a2, ib2);
  v[3] = csub(a2, ib2);
}

template <typename V> __device__ __forceinline__ void bfly8(V* v, bool inv) {
  typedef decltype(v[0].x) R;
  const R r2 = (R)0.70710678118654752440;
  V e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
  bfly4(e, inv);
  bfly4(o, inv);
  // w8^k o[k]: w8 = exp(-i pi/4) forward
  V w1 = inv ? mk(r2 * (o[1].x - o[1].y), r2 * (o[1].x + o[1].y))
             : mk(r2 * (o[1].x + o[1].y), r2 * (o[1].y - o[1].x));
  V w2 = mul_mi(o[2], inv);
  V w3 = inv ? mk(-r2 * (o[3].x + o[3].y), r2 * (o[3].x - o[3].y))
             : mk(r2 * (o[3].y - o[3].x), -r2 * (o[3].x + o[3].y));
  v[0] = cadd(e[0], o[0]);
  v[4] = csub(e[0], o[0]);
  v[1] = cadd(e[1], w1);
  v[5] = csub(e[1], w1);
  v[2] = cadd(e[2], w2);
  v[6] = csub(e[2], w2);
  v[3] = cadd(e[3], w3);
  v[7] = csub(e[3], w3);
}

__device__ __forceinline__ int sw(int e) { return e + (e >> 4); }  // shared-memory swizzle
__host__ __device__ __forceinline__ int sw_len(int n) { return n + (n >> 4) + 1; }
__device__ __forceinline__ int udiv(int n, uint32_t mag) {  // exact n / d, mag = div_magic(d)
  return mag ? (int)__umulhi((uint32_t)n, mag) : n;
}

// Line geometry in shared memory. SWL = false: element e of line l at l*ls + sw(e)*es (the
// swizzle runs along the line); SWL = true: at sw(l)*ls + e*es (columns of a plane whose rows
// are swizzled). line_fast maps consecutive threads to consecutive lines (lines adjacent in
// memory), otherwise to consecutive butterflies of one line.
struct Lines {
  int nlines, ls, es;
  uint32_t mag_nl;  // div_magic(nlines)
  bool line_fast;
};

template <typename V, int M>
__device__ __forceinline__ void dft_reg(V* v, const V* tw, int tstride, bool inv);

template <typename V, int R, bool SWL>
__device__ __forceinline__ void stage_r(const V* src, V* dst, const V* tw, int P, int Ns,
                                        uint32_t mag_m, uint32_t mag_ns, const Lines& L, bool inv) {
  const int m = P / R;
  const int stw = P / (Ns * R);
  const int total = L.nlines * m;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    int l, j;
    if (L.line_fast) { j = udiv(idx, L.mag_nl); l = idx - j * L.nlines; }
    else { l = udiv(idx, mag_m); j = idx - l * m; }
    const int k = j - udiv(j, mag_ns) * Ns;
    V v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int e = j + r * m;
      v[r] = src[SWL ? sw(l) * L.ls + e * L.es : l * L.ls + sw(e) * L.es];
    }
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        V w = tw[r * k * stw];
        if (inv) w.y = -w.y;
        v[r] = cmul(v[r], w);
      }
    }
    if constexpr (R == 32) dft_reg<V, 32>(v, tw, P / 32, inv);
    else if (R == 2) bfly2(v);
    else if (R == 3) bfly3(v, inv);
    else if (R == 4) bfly4(v, inv);
    else if (R == 5) bfly5(v, inv);
    else bfly8(v, inv);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int e = base + r * Ns;
      dst[SWL ? sw(l) * L.ls + e * L.es : l * L.ls + sw(e) * L.es] = v[r];
    }
  }
}

// all stages of plan pl; returns the buffer holding the result (a or b)
template <typename V, bool SWL>
__device__ V* fft_smem(V* a, V* b, const V* tw, const FftPlan& pl, const Lines& L, bool inv) {
  int Ns = 1;
  for (int st = 0; st < pl.nst; ++st) {
    const int R = pl.rad[st];
    const uint32_t mm = pl.mag_m[st], mn = pl.mag_ns[st];
    switch (R) {
      case 2: stage_r<V, 2, SWL>(a, b, tw, pl.P, Ns, mm, mn, L, inv); break;
      case 3: stage_r<V, 3, SWL>(a, b, tw, pl.P, Ns, mm, mn, L, inv); break;
      case 4: stage_r<V, 4, SWL>(a, b, tw, pl.P, Ns, mm, mn, L, inv); break;
      case 5: stage_r<V, 5, SWL>(a, b, tw, pl.P, Ns, mm, mn, L, inv); break;
      default: stage_r<V, 8, SWL>(a, b, tw, pl.P, Ns, mm, mn, L, inv); break;
    }
    __syncthreads();
    V* t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
}

// fft_smem with radix-32 stages as well (the slab passes only: the 32-point butterfly's
// registers would otherwise count against every kernel that uses fft_smem)
template <typename V, bool SWL>
__device__ V* fft_smem_slab(V* a, V* b, const V* tw, const FftPlan& pl, const Lines& L, bool inv) {
  int Ns = 1;
  for (int st = 0; st < pl.nst; ++st) {
    const int R = pl.rad[st];
    const uint32_t mm = pl.mag_m[st], mn = pl.mag_ns[st];
    switch (R) {
      case 2: stage_r<V, 2, SWL>(a, b, tw, pl.P, Ns, mm, mn, L, inv); break;
      case 3: stage_r<V, 3, SWL>(a, b, tw, pl.P, Ns, mm, mn, L, inv); break;
      case 4: stage_r<V, 4, SWL>(a, b, tw, pl.P, Ns, mm, mn, L, inv); break;
      case 5: stage_r<V, 5, SWL>(a, b, tw, pl.P, Ns, mm, mn, L, inv); break;
      case 32: stage_r<V, 32, SWL>(a, b, tw, pl.P, Ns, mm, mn, L, inv); break;
      default: stage_r<V, 8, SWL>(a, b, tw, pl.P, Ns, mm, mn, L, inv); break;
    }
    __syncthreads();
    V* t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
}

// ---------------------------------------------------------------------------------------
// plane passes (x and y together, one padded plane per CTA)
// ---------------------------------------------------------------------------------------
struct PlaneArgs {
  int nx, ny, nz, Px, Py, Pz;
  int64_t ng, P3;
  FftPlan px, py, pz;
  int gx, gy;        // octant dims of Ghat (Px/2+1, Py/2+1)
  int TL;            // lines per CTA in the z pass
  uint32_t mag_Px;   // div_magic(Px), div_magic(nx), div_magic(TL)
  uint32_t mag_nx;
  uint32_t mag_TL;
  uint32_t mag_Pz;
};

// plane layout in shared memory: row y at y * pitch, element x at sw(x)
template <typename V>
__global__ void __launch_bounds__(512) k_plane_fwd(const V* __restrict__ sigma, V* __restrict__ ws,
                                                   const V* __restrict__ twx, const V* __restrict__ twy,
                                                   PlaneArgs a) {
  extern __shared__ unsigned char smem_raw[];
  V* tx = reinterpret_cast<V*>(smem_raw);
  V* ty = tx + a.Px;
  const int pitch = sw_len(a.Px);
  V* A = ty + a.Py;
  V* B = A + a.Py * pitch;
  const int z = blockIdx.x, c = blockIdx.y;
  for (int i = threadIdx.x; i < a.Px; i += blockDim.x) tx[i] = twx[i];
  for (int i = threadIdx.x; i < a.Py; i += blockDim.x) ty[i] = twy[i];
  const V* src = sigma + c * a.ng + (int64_t)z * a.ny * a.nx;
  for (int i = threadIdx.x; i < a.Py * a.Px; i += blockDim.x) {
    const int y = udiv(i, a.mag_Px), x = i - y * a.Px;
    V v = czero<V>();
    if (y < a.ny && x < a.nx) v = src[y * a.nx + x];
    A[y * pitch + sw(x)] = v;
    B[y * pitch + sw(x)] = czero<V>();
  }
  __syncthreads();
  // rows (only the ny non-zero ones), then all columns
  const Lines rows{a.ny, pitch, 1, 0, false};
  V* r = fft_smem<V, false>(A, B, tx, a.px, rows, false);
  V* o = (r == A) ? B : A;
  const Lines cols{a.Px, 1, pitch, a.mag_Px, true};
  r = fft_smem<V, true>(r, o, ty, a.py, cols, false);
  V* dst = ws + c * a.P3 + (int64_t)z * a.Py * a.Px;
  for (int i = threadIdx.x; i < a.Py * a.Px; i += blockDim.x) {
    const int y = udiv(i, a.mag_Px), x = i - y * a.Px;
    dst[i] = r[y * pitch + sw(x)];
  }
}

template <typename V>
__global__ void __launch_bounds__(512) k_plane_inv(const V* __restrict__ ws, V* __restrict__ phi,
                                                   const V* __restrict__ twx, const V* __restrict__ twy,
                                                   PlaneArgs a) {
  extern __shared__ unsigned char smem_raw[];
  V* tx = reinterpret_cast<V*>(smem_raw);
  V* ty = tx + a.Px;
  const int pitch = sw_len(a.Px);
  V* A = ty + a.Py;
  V* B = A + a.Py * pitch;
  const int z = blockIdx.x, c = blockIdx.y;
  for (int i = threadIdx.x; i < a.Px; i += blockDim.x) tx[i] = twx[i];
  for (int i = threadIdx.x; i < a.Py; i += blockDim.x) ty[i] = twy[i];
  const V* src = ws + c * a.P3 + (int64_t)z * a.Py * a.Px;
  for (int i = threadIdx.x; i < a.Py * a.Px; i += blockDim.x) {
    const int y = udiv(i, a.mag_Px), x = i - y * a.Px;
    A[y * pitch + sw(x)] = src[i];
  }
  __syncthreads();
  const Lines cols{a.Px, 1, pitch, a.mag_Px, true};
  V* r = fft_smem<V, true>(A, B, ty, a.py, cols, true);
  V* o = (r == A) ? B : A;
  const Lines rows{a.ny, pitch, 1, 0, false};
  r = fft_smem<V, false>(r, o, tx, a.px, rows, true);
  V* dst = phi + c * a.ng + (int64_t)z * a.ny * a.nx;
  for (int i = threadIdx.x; i < a.ny * a.nx; i += blockDim.x) {
    const int y = udiv(i, a.mag_nx), x = i - y * a.nx;
    dst[i] = r[y * pitch + sw(x)];
  }
}

// z pass: TL consecutive x of one y; forward FFT of the nz planes, times Ghat, inverse
template <typename V>
__global__ void __launch_bounds__(256) k_zfused(V* ws, const V* __restrict__ ghat,
                                                const V* __restrict__ twz, PlaneArgs a) {
  extern __shared__ unsigned char smem_raw[];
  V* tz = reinterpret_cast<V*>(smem_raw);
  const int pitch = sw_len(a.Pz);
  V* A = tz + a.Pz;
  V* B = A + a.TL * pitch;
  const int x0 = blockIdx.x * a.TL, y = blockIdx.y, c = blockIdx.z;
  const int nl = min(a.TL, a.Px - x0);
  for (int i = threadIdx.x; i < a.Pz; i += blockDim.x) tz[i] = twz[i];
  const int64_t plane = (int64_t)a.Py * a.Px;
  V* base = ws + c * a.P3 + (int64_t)y * a.Px + x0;
  for (int i = threadIdx.x; i < a.TL * a.Pz; i += blockDim.x) {
    const int e = udiv(i, a.mag_TL), l = i - e * a.TL;
    V v = czero<V>();
    if (l < nl && e < a.nz) v = base[e * plane + l];
    A[l * pitch + sw(e)] = v;
  }
  __syncthreads();
  const Lines L{a.TL, pitch, 1, a.mag_TL, false};
  V* r = fft_smem<V, false>(A, B, tz, a.pz, L, false);
  const int fy = min(y, a.Py - y);
  for (int i = threadIdx.x; i < a.TL * a.Pz; i += blockDim.x) {
    const int l = udiv(i, a.mag_Pz), kz = i - l * a.Pz;
    if (l >= nl) continue;
    const int x = x0 + l;
    const int fx = min(x, a.Px - x), fz = min(kz, a.Pz - kz);
    const int o = l * pitch + sw(kz);
    r[o] = cmul(r[o], ghat[((int64_t)fz * a.gy + fy) * a.gx + fx]);
  }
  __syncthreads();
  V* o = (r == A) ? B : A;
  r = fft_smem<V, false>(r, o, tz, a.pz, L, true);
  for (int i = threadIdx.x; i < a.TL * a.nz; i += blockDim.x) {
    const int e = udiv(i, a.mag_TL), l = i - e * a.TL;
    if (l < nl) base[e * plane + l] = r[l * pitch + sw(e)];
  }
}

// ---------------------------------------------------------------------------------------
// transforms in registers: a line of P = L * M points held by a group of L lanes (L = 8, 16 or
// 32), element n = l + L n1 in lane l, register n1. Forward: the M-point DFT over n1 in
// registers, the twiddles W_P^(l k1), then for every k1 an L-point DFT across the lanes by
// radix-2 decimation in frequency with xor shuffles, which leaves X[k1 + M bitrev(l)] in lane l,
// register k1. The inverse undoes the steps in reverse (every shuffle butterfly inverted, the
// conjugate twiddles, the inverse M-point DFT) and takes its input in that bit-reversed order,
// so a forward and an inverse transform need no reordering and no shared memory between them.
// Both are unnormalised. The M-point DFT is one butterfly for M in {2, 3, 4, 5, 8} and two
// levels A x B (A-point DFTs of stride B, twiddles W_M^(b ka), B-point DFTs) for M in
// {6, 9, 10, 12, 15, 16}; twiddles come from the line's table W_P^j (P divisible by M).
// ---------------------------------------------------------------------------------------
template <typename V, int R>
__device__ __forceinline__ void bfly_r(V* v, bool inv) {
  if (R == 2) bfly2(v);
  else if (R == 3) bfly3(v, inv);
  else if (R == 4) bfly4(v, inv);
  else if (R == 5) bfly5(v, inv);
  else bfly8(v, inv);
}

template <int M> struct Split { static constexpr int A = 1, B = 1; };
template <> struct Split<6> { static constexpr int A = 2, B = 3; };
template <> struct Split<9> { static constexpr int A = 3, B = 3; };
template <> struct Split<10> { static constexpr int A = 2, B = 5; };
template <> struct Split<12> { static constexpr int A = 4, B = 3; };
template <> struct Split<15> { static constexpr int A = 3, B = 5; };
template <> struct Split<16> { static constexpr int A = 4, B = 4; };
template <> struct Split<32> { static constexpr int A = 4, B = 8; };

// natural-order M-point DFT of v in registers (tw: W_P^j, P = M * tstride)
template <typename V, int M>
__device__ __forceinline__ void dft_reg(V* v, const V* tw, int tstride, bool inv) {
  static_assert(M <= 16 || M == 32, "register DFT length");
  if constexpr (M == 2 || M == 3 || M == 4 || M == 5 || M == 8) {
    bfly_r<V, M>(v, inv);
  } else {
    constexpr int A = Split<M>::A, B = Split<M>::B;
    V u[B][A];
#pragma unroll
    for (int b = 0; b < B; ++b) {
#pragma unroll
      for (int a = 0; a < A; ++a) u[b][a] = v[b + B * a];
      bfly_r<V, A>(u[b], inv);
#pragma unroll
      for (int ka = 1; ka < A; ++ka)
        if (b > 0) {
          V w = tw[(b * ka) * tstride];
          if (inv) w.y = -w.y;
          u[b][ka] = cmul(u[b][ka], w);
        }
    }
#pragma unroll
    for (int ka = 0; ka < A; ++ka) {
      V t[B];
#pragma unroll
      for (int b = 0; b < B; ++b) t[b] = u[b][ka];
      bfly_r<V, B>(t, inv);
#pragma unroll
      for (int kb = 0; kb < B; ++kb) v[ka + A * kb] = t[kb];
    }
  }
}

template <typename V> __device__ __forceinline__ V shfl_x(V v, int s) {
  return mk(__shfl_xor_sync(0xffffffffu, v.x, s), __shfl_xor_sync(0xffffffffu, v.y, s));
}

template <int L> struct Log2 { static constexpr int v = L == 8 ? 3 : (L == 16 ? 4 : 5); };

// twiddles of lane lg for a line of P = L M: tk[k1] = W_P^(lg k1), ts[st] = W_(2s)^(lg mod s)
// for the shuffle stage of pair distance s = L >> (st + 1). The table holds W_P^j, so the
// indices are lg k1 (< P, no reduction needed) and (lg mod s) P / (2 s) = (lg mod s) M 2^st.
template <typename V, int L, int M>
__device__ __forceinline__ void reg_twiddles(const V* tw, int P, int lg, V* tk, V* ts) {
  (void)P;
#pragma unroll
  for (int k1 = 0; k1 < M; ++k1) tk[k1] = tw[lg * k1];
#pragma unroll
  for (int st = 0; st < Log2<L>::v; ++st) {
    const int sp = L >> (st + 1);
    ts[st] = tw[(lg & (sp - 1)) * (M << st)];
  }
}

template <typename V, int L, int M>
__device__ __forceinline__ void reg_fft_fwd(V* v, const V* tw, int P, int lg, const V* tk,
                                            const V* ts) {
  dft_reg<V, M>(v, tw, P / M, false);
#pragma unroll
  for (int k1 = 1; k1 < M; ++k1) v[k1] = cmul(v[k1], tk[k1]);
  typedef decltype(v[0].x) R;
#pragma unroll
  for (int st = 0; st < Log2<L>::v; ++st) {
    // lower lane of a pair: v + p; upper lane: (p - v) W. As one branch-free form:
    // (p + sg v) we with sg = +-1 (exact products) and we = 1 on the lower lane
    const int sp = L >> (st + 1);
    const bool top = (lg & sp) == 0;
    const R sg = top ? R(1) : R(-1);
    const V we = top ? mk(R(1), R(0)) : ts[st];
#pragma unroll
    for (int k1 = 0; k1 < M; ++k1) {
      const V p = shfl_x(v[k1], sp);
      v[k1] = cmul(mk(sg * v[k1].x + p.x, sg * v[k1].y + p.y), we);
    }
  }
}

template <typename V, int L, int M>
__device__ __forceinline__ void reg_fft_inv(V* v, const V* tw, int P, int lg, const V* tk,
                                            const V* ts) {
  typedef decltype(v[0].x) R;
#pragma unroll
  for (int st = Log2<L>::v - 1; st >= 0; --st) {
    // the upper lane first takes conj(W); then lower: own + p, upper: p - own (= p + sg own)
    const int sp = L >> (st + 1);
    const bool top = (lg & sp) == 0;
    const R sg = top ? R(1) : R(-1);
    const V we = top ? mk(R(1), R(0)) : mk(ts[st].x, -ts[st].y);
#pragma unroll
    for (int k1 = 0; k1 < M; ++k1) {
      const V own = cmul(v[k1], we);
      const V p = shfl_x(own, sp);
      v[k1] = mk(sg * own.x + p.x, sg * own.y + p.y);
    }
  }
#pragma unroll
  for (int k1 = 1; k1 < M; ++k1) v[k1] = cmul(v[k1], mk(tk[k1].x, -tk[k1].y));
  dft_reg<V, M>(v, tw, P / M, true);
}

template <int L> __device__ __forceinline__ int brev_l(int l) {
  return (int)(__brev((unsigned)l) >> (32 - Log2<L>::v));
}

// z pass: a CTA of 8 warps takes 8 * 32 / L adjacent x of one y; forward transform along z of
// the nz planes that hold data, times Ghat (in the transform's bit-reversed order), inverse,
// and the first nz outputs stored back
template <typename V, int L, int M>
__global__ void __launch_bounds__(256, M <= 6 ? 4 : 1) k_zreg(V* ws, const V* __restrict__ ghat,
                                                 const V* __restrict__ twz, PlaneArgs a) {
  constexpr int G = 32 / L;  // lines per warp
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lg = lane & (L - 1), grp = lane / L;
  const int x = blockIdx.x * (8 * G) + warp * G + grp, y = blockIdx.y, c = blockIdx.z;
  const bool live = x < a.Px;
  const int P = a.Pz;
  const int64_t plane = (int64_t)a.Py * a.Px;
  V* base = ws + c * a.P3 + (int64_t)y * a.Px + (live ? x : 0);
  V v[M];
#pragma unroll
  for (int n1 = 0; n1 < M; ++n1) {
    const int z = lg + L * n1;
    v[n1] = (live && z < a.nz) ? base[z * plane] : czero<V>();
  }
  V tk[M], ts[Log2<L>::v];
  reg_twiddles<V, L, M>(twz, P, lg, tk, ts);
  reg_fft_fwd<V, L, M>(v, twz, P, lg, tk, ts);
  const int fy = min(y, a.Py - y), fx = min(x, a.Px - x);
  const int k2 = brev_l<L>(lg);
#pragma unroll
  for (int k1 = 0; k1 < M; ++k1) {
    const int k = k1 + M * k2, fz = min(k, P - k);
    if (live) v[k1] = cmul(v[k1], ghat[((int64_t)fz * a.gy + fy) * a.gx + fx]);
  }
  reg_fft_inv<V, L, M>(v, twz, P, lg, tk, ts);
#pragma unroll
  for (int n1 = 0; n1 < M; ++n1) {
    const int z = lg + L * n1;
    if (live && z < a.nz) base[z * plane] = v[n1];
  }
}

// z pass with the CTA's lines staged through shared memory: the nz data planes of the CTA's
// 8 * 32 / L adjacent x are read and written as contiguous runs of x (one warp per line would
// touch 32 planes per load, a quarter of each sector), then each line is transformed in
// registers as in k_zreg. Ghat comes from gz, the line's values already in the lanes' order
// (lane l, register k1: frequency k1 + M brev(l)), so a warp reads it in whole sectors.
// Dynamic shared memory: NL (nz + 1) elements.
template <typename V, int L, int M>
__global__ void __launch_bounds__(256, M <= 6 ? 4 : 1) k_zreg_st(V* ws, const V* __restrict__ gz,
                                                            const V* __restrict__ twz, PlaneArgs a) {
  constexpr int G = 32 / L, NL = 8 * G;  // lines per warp, per CTA
  extern __shared__ unsigned char smem_raw[];
  const int sp = a.nz + 1;
  V* S = reinterpret_cast<V*>(smem_raw);  // [NL][sp]: the line's data along z
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lg = lane & (L - 1), xi = warp * G + lane / L;
  const int x0 = blockIdx.x * NL, y = blockIdx.y, c = blockIdx.z;
  const int P = a.Pz, nlive = min(NL, a.Px - x0);
  const int64_t plane = (int64_t)a.Py * a.Px;
  V* base = ws + c * a.P3 + (int64_t)y * a.Px + x0;
  for (int i = threadIdx.x; i < a.nz * NL; i += blockDim.x) {
    const int z = i / NL, l = i - z * NL;
    S[l * sp + z] = l < nlive ? base[z * plane + l] : czero<V>();
  }
  __syncthreads();
  V v[M];
#pragma unroll
  for (int n1 = 0; n1 < M; ++n1) {
    const int z = lg + L * n1;
    v[n1] = z < a.nz ? S[xi * sp + z] : czero<V>();
  }
  V tk[M], ts[Log2<L>::v];
  reg_twiddles<V, L, M>(twz, P, lg, tk, ts);
  reg_fft_fwd<V, L, M>(v, twz, P, lg, tk, ts);
  if (xi < nlive) {
    const V* g = gz + ((int64_t)y * a.Px + x0 + xi) * P + lg;
#pragma unroll
    for (int k1 = 0; k1 < M; ++k1) v[k1] = cmul(v[k1], g[k1 * L]);
  }
  reg_fft_inv<V, L, M>(v, twz, P, lg, tk, ts);
  // each lane rewrites only the entries it read: no barrier before the write-back
#pragma unroll
  for (int n1 = 0; n1 < M; ++n1) {
    const int z = lg + L * n1;
    if (z < a.nz) S[xi * sp + z] = v[n1];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < a.nz * NL; i += blockDim.x) {
    const int z = i / NL, l = i - z * NL;
    if (l < nlive) base[z * plane + l] = S[l * sp + z];
  }
}

// gz[(y Px + x) Pz + k1 L + l] = Ghat(fz, fy, fx) at frequency k = k1 + M brev(l) of line (x, y)
template <typename V, int L>
__global__ void k_ghat_lines(const V* __restrict__ oct, int M, int Px, int Py, int Pz, V* gz) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)Px * Py * Pz) return;
  const int r = (int)(idx % Pz);
  const int64_t line = idx / Pz;
  const int x = (int)(line % Px), y = (int)(line / Px);
  const int l = r % L, k1 = r / L;
  const int k = k1 + M * brev_l<L>(l);
  const int fz = min(k, Pz - k), fy = min(y, Py - y), fx = min(x, Px - x);
  gz[idx] = oct[((int64_t)fz * (Py / 2 + 1) + fy) * (Px / 2 + 1) + fx];
}

// plane passes in registers (one padded x-y plane per CTA of 256 threads, the x spectra of the
// rows in shared memory at pitch Px + 1 between the two directions). Forward: the ny rows that
// hold data along x (groups of LX lanes, one row each) into shared memory, then every column
// along y, stored straight to the workspace (for one register the groups of a warp write
// adjacent x of one row). Inverse: every column along y read straight from the workspace,
// keeping the ny rows that are read back, into shared memory, then those rows along x, storing
// the nx x ny window.
template <typename V, int LX, int MX, int LY, int MY>
__global__ void __launch_bounds__(384) k_plane_fwd_reg(const V* __restrict__ sigma, V* __restrict__ ws,
                                                       const V* __restrict__ twx,
                                                       const V* __restrict__ twy, PlaneArgs a) {
  extern __shared__ unsigned char smem_raw[];
  V* tx = reinterpret_cast<V*>(smem_raw);
  V* ty = tx + a.Px;
  V* S = ty + a.Py;
  const int pitch = a.Px + 1;
  const int z = blockIdx.x, c = blockIdx.y;
  for (int i = threadIdx.x; i < a.Px; i += blockDim.x) tx[i] = twx[i];
  for (int i = threadIdx.x; i < a.Py; i += blockDim.x) ty[i] = twy[i];
  __syncthreads();
  const V* src = sigma + c * a.ng + (int64_t)z * a.ny * a.nx;
  {
    const int lg = threadIdx.x & (LX - 1), grp = threadIdx.x / LX, ngrp = blockDim.x / LX;
    V tk[MX], ts[Log2<LX>::v];
    reg_twiddles<V, LX, MX>(tx, a.Px, lg, tk, ts);
    const int k2 = brev_l<LX>(lg);
    // every group runs the same number of rounds (the shuffles need whole warps)
    for (int y0 = 0; y0 < a.ny; y0 += ngrp) {
      const int y = y0 + grp;
      V v[MX];
#pragma unroll
      for (int n1 = 0; n1 < MX; ++n1) {
        const int x = lg + LX * n1;
        v[n1] = (y < a.ny && x < a.nx) ? src[y * a.nx + x] : czero<V>();
      }
      reg_fft_fwd<V, LX, MX>(v, tx, a.Px, lg, tk, ts);
      if (y < a.ny) {
#pragma unroll
        for (int k1 = 0; k1 < MX; ++k1) S[y * pitch + k1 + MX * k2] = v[k1];
      }
    }
  }
  __syncthreads();
  {
    const int lg = threadIdx.x & (LY - 1), grp = threadIdx.x / LY, ngrp = blockDim.x / LY;
    V tk[MY], ts[Log2<LY>::v];
    reg_twiddles<V, LY, MY>(ty, a.Py, lg, tk, ts);
    const int k2 = brev_l<LY>(lg);
    V* dst = ws + c * a.P3 + (int64_t)z * a.Py * a.Px;
    for (int x0 = 0; x0 < a.Px; x0 += ngrp) {
      const int kx = x0 + grp;
      V v[MY];
#pragma unroll
      for (int n1 = 0; n1 < MY; ++n1) {
        const int y = lg + LY * n1;
        v[n1] = (kx < a.Px && y < a.ny) ? S[y * pitch + kx] : czero<V>();
      }
      reg_fft_fwd<V, LY, MY>(v, ty, a.Py, lg, tk, ts);
      if (kx < a.Px) {
#pragma unroll
        for (int k1 = 0; k1 < MY; ++k1) dst[(k1 + MY * k2) * a.Px + kx] = v[k1];
      }
    }
  }
}

template <typename V, int LX, int MX, int LY, int MY>
__global__ void __launch_bounds__(384) k_plane_inv_reg(const V* __restrict__ ws, V* __restrict__ phi,
                                                       const V* __restrict__ twx,
                                                       const V* __restrict__ twy, PlaneArgs a) {
  extern __shared__ unsigned char smem_raw[];
  V* tx = reinterpret_cast<V*>(smem_raw);
  V* ty = tx + a.Px;
  V* S = ty + a.Py;
  const int pitch = a.Px + 1;
  const int z = blockIdx.x, c = blockIdx.y;
  for (int i = threadIdx.x; i < a.Px; i += blockDim.x) tx[i] = twx[i];
  for (int i = threadIdx.x; i < a.Py; i += blockDim.x) ty[i] = twy[i];
  const V* src = ws + c * a.P3 + (int64_t)z * a.Py * a.Px;
  __syncthreads();
  {
    const int lg = threadIdx.x & (LY - 1), grp = threadIdx.x / LY, ngrp = blockDim.x / LY;
    V tk[MY], ts[Log2<LY>::v];
    reg_twiddles<V, LY, MY>(ty, a.Py, lg, tk, ts);
    const int k2 = brev_l<LY>(lg);
    for (int x0 = 0; x0 < a.Px; x0 += ngrp) {
      const int kx = x0 + grp;
      V v[MY];
#pragma unroll
      for (int k1 = 0; k1 < MY; ++k1)
        v[k1] = kx < a.Px ? src[(k1 + MY * k2) * a.Px + kx] : czero<V>();
      reg_fft_inv<V, LY, MY>(v, ty, a.Py, lg, tk, ts);
      if (kx < a.Px) {
#pragma unroll
        for (int n1 = 0; n1 < MY; ++n1) {
          const int y = lg + LY * n1;
          if (y < a.ny) S[y * pitch + kx] = v[n1];
        }
      }
    }
  }
  __syncthreads();
  {
    const int lg = threadIdx.x & (LX - 1), grp = threadIdx.x / LX, ngrp = blockDim.x / LX;
    V tk[MX], ts[Log2<LX>::v];
    reg_twiddles<V, LX, MX>(tx, a.Px, lg, tk, ts);
    const int k2 = brev_l<LX>(lg);
    V* dst = phi + c * a.ng + (int64_t)z * a.ny * a.nx;
    for (int y0 = 0; y0 < a.ny; y0 += ngrp) {
      const int y = y0 + grp;
      V v[MX];
#pragma unroll
      for (int k1 = 0; k1 < MX; ++k1) v[k1] = y < a.ny ? S[y * pitch + k1 + MX * k2] : czero<V>();
      reg_fft_inv<V, LX, MX>(v, tx, a.Px, lg, tk, ts);
      if (y < a.ny) {
#pragma unroll
        for (int n1 = 0; n1 < MX; ++n1) {
          const int x = lg + LX * n1;
          if (x < a.nx) dst[y * a.nx + x] = v[n1];
        }
      }
    }
  }
}

// the register shapes (L lanes, M registers) built, one per length P = L M, the most lanes first
#define BEM_REG_SHAPES(X)                                                                         \
  X(32, 2) X(32, 3) X(32, 4) X(32, 5) X(32, 6) X(32, 8) X(32, 9) X(32, 10) X(32, 12) X(32, 15)    \
  X(32, 16) X(16, 3) X(16, 5) X(16, 9) X(16, 15) X(8, 3) X(8, 5) X(8, 9) X(8, 15)

// (L, M) of a register transform of length P, or false
static bool reg_shape(int P, int* L, int* M) {
#define BEM_S(LL, MM) \
  if (P == LL * MM) { *L = LL; *M = MM; return true; }
  BEM_REG_SHAPES(BEM_S)
#undef BEM_S
  return false;
}

template <typename V>
static void launch_zreg(int L, int M, dim3 grid, cudaStream_t s, V* ws, const V* ghat,
                        const V* gz, const V* tw, const PlaneArgs& a) {
  const int NL = 8 * (32 / L);
  const size_t smem = (size_t)NL * (a.nz + 1) * sizeof(V);
  const bool staged = gz && smem <= 48 * 1024;
#define BEM_Z(LL, MM)                                                        \
  if (L == LL && M == MM) {                                                  \
    if (staged) k_zreg_st<V, LL, MM><<<grid, 256, smem, s>>>(ws, gz, tw, a); \
    else k_zreg<V, LL, MM><<<grid, 256, 0, s>>>(ws, ghat, tw, a);            \
    return;                                                                  \
  }
  BEM_REG_SHAPES(BEM_Z)
#undef BEM_Z
}

// the plane passes in registers exist for equal x and y shapes (square padded planes)
template <typename V>
static bool launch_plane_reg(bool inverse, int L, int M, dim3 grid, size_t smem, cudaStream_t s,
                             const V* in, V* out, const V* twx, const V* twy, const PlaneArgs& a) {
  // threads: L lanes x G groups, G picked (up to 384 threads) for the fewest rounds of the
  // two directions (ny rows along x, then Px columns along y; the same counts inverted)
  int nt = 256, rounds = 1 << 30;
  for (int t = 128; t <= 384; t += 32) {
    const int G = t / L, r = (a.ny + G - 1) / G + (a.Px + G - 1) / G;
    if (r < rounds) { rounds = r; nt = t; }
  }
#define BEM_P(LL, MM)                                                                                  \
  if (L == LL && M == MM) {                                                                           \
    if (inverse) k_plane_inv_reg<V, LL, MM, LL, MM><<<grid, nt, smem, s>>>(in, out, twx, twy, a);       \
    else k_plane_fwd_reg<V, LL, MM, LL, MM><<<grid, nt, smem, s>>>(in, out, twx, twy, a);               \
    return true;                                                                                      \
  }
  BEM_REG_SHAPES(BEM_P)
#undef BEM_P
  return false;
}

// ---------------------------------------------------------------------------------------
// generic batched 1-D pass (large planes, and the set-up FFT of the grid kernel)
// ---------------------------------------------------------------------------------------
struct LinePass {
  int P, nin, nout;
  int64_t ies, oes;
  int n0, n1;
  int64_t is0, is1, is2;
  int64_t os0, os1, os2;
  int fused;    // 1: forward, multiply by Ghat, inverse (z axis: line = (x = i0, y = i1))
  int inverse;
  int TL;
  int gx, gy, Px, Py;
  uint32_t mag_P, mag_TL;
  FftPlan plan;
};

template <typename V>
__global__ void __launch_bounds__(256) k_lines(const V* in, V* out, const V* __restrict__ twg,
                                               const V* __restrict__ ghat, LinePass p) {
  extern __shared__ unsigned char smem_raw[];
  V* tw = reinterpret_cast<V*>(smem_raw);
  const int pitch = sw_len(p.P);
  V* A = tw + p.P;
  V* B = A + p.TL * pitch;
  const int i0base = blockIdx.x * p.TL;
  const int i1 = blockIdx.y, i2 = blockIdx.z;
  const int nl = min(p.TL, p.n0 - i0base);
  for (int i = threadIdx.x; i < p.P; i += blockDim.x) tw[i] = twg[i];
  const int64_t ib = i1 * p.is1 + i2 * p.is2;
  for (int idx = threadIdx.x; idx < p.TL * p.P; idx += blockDim.x) {
    int l, e;
    if (p.ies == 1) { l = udiv(idx, p.mag_P); e = idx - l * p.P; }
    else { e = udiv(idx, p.mag_TL); l = idx - e * p.TL; }
    V v = czero<V>();
    if (l < nl && e < p.nin) v = in[ib + (int64_t)(i0base + l) * p.is0 + (int64_t)e * p.ies];
    A[l * pitch + sw(e)] = v;
  }
  __syncthreads();
  const Lines L{p.TL, pitch, 1, p.mag_TL, false};
  V* res;
  if (!p.fused) {
    res = fft_smem<V, false>(A, B, tw, p.plan, L, p.inverse != 0);
  } else {
    res = fft_smem<V, false>(A, B, tw, p.plan, L, false);
    for (int idx = threadIdx.x; idx < p.TL * p.P; idx += blockDim.x) {
      const int l = udiv(idx, p.mag_P), kz = idx - l * p.P;
      if (l >= nl) continue;
      const int x = i0base + l, y = i1;
      const int fx = min(x, p.Px - x), fy = min(y, p.Py - y), fz = min(kz, p.P - kz);
      const int o = l * pitch + sw(kz);
      res[o] = cmul(res[o], ghat[((int64_t)fz * p.gy + fy) * p.gx + fx]);
    }
    __syncthreads();
    V* other = (res == A) ? B : A;
    res = fft_smem<V, false>(res, other, tw, p.plan, L, true);
  }
  const int64_t ob = i1 * p.os1 + i2 * p.os2;
  for (int idx = threadIdx.x; idx < p.TL * p.nout; idx += blockDim.x) {
    int l, e;
    if (p.oes == 1) { l = idx / p.nout; e = idx - l * p.nout; }
    else { e = udiv(idx, p.mag_TL); l = idx - e * p.TL; }
    if (l < nl) out[ob + (int64_t)(i0base + l) * p.os0 + (int64_t)e * p.oes] = res[l * pitch + sw(e)];
  }
}

static constexpr size_t kSmemBudget = 200 * 1024;

template <typename V>
static int launch_lines(const V* in, V* out, const V* tw, const V* ghat, LinePass p, int n2,
                        cudaStream_t s) {
  const size_t avail = 96 * 1024 / sizeof(V);
  const size_t pitch = sw_len(p.P);
  if (avail < p.P + 2 * pitch) {
    set_error("FFT length %d too large for shared memory", p.P);
    return BEM_EGRID;
  }
  int TL = (int)std::min<size_t>(16, (avail - p.P) / (2 * pitch));
  TL = std::max(1, std::min(TL, p.n0));
  p.TL = TL;
  p.mag_P = div_magic(p.P);
  p.mag_TL = div_magic(TL);
  size_t smem = ((size_t)p.P + 2 * (size_t)TL * pitch) * sizeof(V);
  dim3 grid((p.n0 + TL - 1) / TL, p.n1, n2);
  k_lines<V><<<grid, 256, smem, s>>>(in, out, tw, ghat, p);
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

template <typename V> static size_t plane_smem(int Px, int Py) {
  return ((size_t)Px + Py + 2 * (size_t)Py * sw_len(Px)) * sizeof(V);
}

// ---------------------------------------------------------------------------------------
// slab passes (FP32, padded x-y planes too large for shared memory; the split-ring array's
// 1024 x 1024 planes): three passes over a workspace X[c][kx][z][y] that holds, per component,
// the x-transformed data rows only (Px * nz * ny values):
//   x forward : RY rows of one data plane per CTA, zero-padded to Px, FFT along x, stored
//               kx-major so that pass two reads one contiguous nz x ny slab per kx
//   y-z fused : one kx per CTA (its Ghat slab staged in shared memory): y FFT of the nz data
//               planes (zero-padded to Py), then per ky a length-Pz DFT in registers over the
//               zero-padded z values, times Ghat, the inverse DFT, the nz kept planes back, the
//               inverse y FFT, the ny kept rows stored in place
//   x inverse : RY rows per CTA, inverse FFT along x, the nx kept values written to phi
// HBM traffic per component: ng in, 3 (Px nz ny) written and 2 read, ng out (168 MB at 512 x
// 512 x 8 against 20 ng = 336 MB for passes over the full padded grid).
// ---------------------------------------------------------------------------------------
constexpr int kSlabRY = 4;     // rows per CTA in the x passes (three CTAs per SM)
constexpr int kSlabMaxNz = 16; // data planes held per ky line in registers

struct SlabArgs {
  int nx, ny, nz, Px, Py, Pz;
  int64_t ng, P3;
  FftPlan px, py;
  int gy, gz;  // octant dims of Ghat along y and z (Py/2+1, Pz/2+1)
  uint32_t mag_Px, mag_Py, mag_ny, mag_RY;
};

__global__ void __launch_bounds__(256) k_slab_xfwd(const float2* __restrict__ sigma,
                                                   float2* __restrict__ ws,
                                                   const float2* __restrict__ twx, SlabArgs a) {
  extern __shared__ unsigned char smem_raw[];
  float2* tx = reinterpret_cast<float2*>(smem_raw);
  const int pitch = sw_len(a.Px);
  float2* A = tx + a.Px;
  float2* B = A + kSlabRY * pitch;
  const int y0 = blockIdx.x * kSlabRY, z = blockIdx.y, c = blockIdx.z;
  const int nr = min(kSlabRY, a.ny - y0);
  for (int i = threadIdx.x; i < a.Px; i += blockDim.x) tx[i] = twx[i];
  const float2* src = sigma + c * a.ng + ((int64_t)z * a.ny + y0) * a.nx;
  for (int i = threadIdx.x; i < kSlabRY * a.Px; i += blockDim.x) {
    const int r = udiv(i, a.mag_Px), x = i - r * a.Px;
    float2 v = make_float2(0.f, 0.f);
    if (r < nr && x < a.nx) v = src[(int64_t)r * a.nx + x];
    A[r * pitch + sw(x)] = v;
  }
  __syncthreads();
  const Lines rows{kSlabRY, pitch, 1, 0, false};
  const float2* res = fft_smem_slab<float2, false>(A, B, tx, a.px, rows, false);
  float2* dst = ws + c * a.P3;
  for (int i = threadIdx.x; i < kSlabRY * a.Px; i += blockDim.x) {
    const int kx = udiv(i, a.mag_RY), r = i - kx * kSlabRY;
    if (r < nr) dst[((int64_t)kx * a.nz + z) * a.ny + y0 + r] = res[r * pitch + sw(kx)];
  }
}

// M = Pz when the register DFT supports that length (natural order, dft_reg), else 0: direct
// DFTs over the nz non-zero values
template <int M>
__global__ void __launch_bounds__(256) k_slab_yz(float2* __restrict__ ws,
                                                 const float2* __restrict__ gs,
                                                 const float2* __restrict__ twy,
                                                 const float2* __restrict__ twz, SlabArgs a) {
  extern __shared__ unsigned char smem_raw[];
  float2* ty = reinterpret_cast<float2*>(smem_raw);
  float2* tz = ty + a.Py;
  float2* G = tz + a.Pz;  // this kx's Ghat slab [fz][fy]
  const int pitch = sw_len(a.Py);
  float2* A = G + a.gz * a.gy;
  float2* B = A + a.nz * pitch;
  const int kx = blockIdx.x, c = blockIdx.y;
  const int fx = min(kx, a.Px - kx);
  for (int i = threadIdx.x; i < a.Py; i += blockDim.x) ty[i] = twy[i];
  for (int i = threadIdx.x; i < a.Pz; i += blockDim.x) tz[i] = twz[i];
  const float2* g = gs + (int64_t)fx * a.gz * a.gy;
  for (int i = threadIdx.x; i < a.gz * a.gy; i += blockDim.x) G[i] = g[i];
  float2* X = ws + c * a.P3 + (int64_t)kx * a.nz * a.ny;  // [z][y]
  for (int i = threadIdx.x; i < a.nz * a.Py; i += blockDim.x) {
    const int z = udiv(i, a.mag_Py), y = i - z * a.Py;
    A[z * pitch + sw(y)] = y < a.ny ? X[(int64_t)z * a.ny + y] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const Lines L{a.nz, pitch, 1, 0, false};
  float2* r = fft_smem_slab<float2, false>(A, B, ty, a.py, L, false);
  for (int ky = threadIdx.x; ky < a.Py; ky += blockDim.x) {
    const int fy = min(ky, a.Py - ky);
    if constexpr (M > 0) {
      float2 v[M];
#pragma unroll
      for (int z = 0; z < M; ++z)
        v[z] = z < a.nz ? r[z * pitch + sw(ky)] : make_float2(0.f, 0.f);
      dft_reg<float2, M>(v, tz, 1, false);
#pragma unroll
      for (int kz = 0; kz < M; ++kz) v[kz] = cmul(v[kz], G[min(kz, M - kz) * a.gy + fy]);
      dft_reg<float2, M>(v, tz, 1, true);
#pragma unroll
      for (int z = 0; z < M; ++z)
        if (z < a.nz) r[z * pitch + sw(ky)] = v[z];
    } else {
      float2 v[kSlabMaxNz], o[kSlabMaxNz];
#pragma unroll
      for (int z = 0; z < kSlabMaxNz; ++z) {
        v[z] = z < a.nz ? r[z * pitch + sw(ky)] : make_float2(0.f, 0.f);
        o[z] = make_float2(0.f, 0.f);
      }
      for (int kz = 0; kz < a.Pz; ++kz) {
        float2 t = make_float2(0.f, 0.f);
#pragma unroll
        for (int z = 0; z < kSlabMaxNz; ++z)
          if (z < a.nz) t = cadd(t, cmul(v[z], tz[(z * kz) % a.Pz]));
        t = cmul(t, G[min(kz, a.Pz - kz) * a.gy + fy]);
#pragma unroll
        for (int z = 0; z < kSlabMaxNz; ++z)
          if (z < a.nz) o[z] = cadd(o[z], cmul(t, cconj(tz[(z * kz) % a.Pz])));
      }
#pragma unroll
      for (int z = 0; z < kSlabMaxNz; ++z)
        if (z < a.nz) r[z * pitch + sw(ky)] = o[z];
    }
  }
  __syncthreads();
  float2* o2 = (r == A) ? B : A;
  r = fft_smem_slab<float2, false>(r, o2, ty, a.py, L, true);
  for (int i = threadIdx.x; i < a.nz * a.ny; i += blockDim.x) {
    const int z = udiv(i, a.mag_ny), y = i - z * a.ny;
    X[(int64_t)z * a.ny + y] = r[z * pitch + sw(y)];
  }
}

__global__ void __launch_bounds__(256) k_slab_xinv(const float2* __restrict__ ws,
                                                   float2* __restrict__ phi,
                                                   const float2* __restrict__ twx, SlabArgs a) {
  extern __shared__ unsigned char smem_raw[];
  float2* tx = reinterpret_cast<float2*>(smem_raw);
  const int pitch = sw_len(a.Px);
  float2* A = tx + a.Px;
  float2* B = A + kSlabRY * pitch;
  const int y0 = blockIdx.x * kSlabRY, z = blockIdx.y, c = blockIdx.z;
  const int nr = min(kSlabRY, a.ny - y0);
  for (int i = threadIdx.x; i < a.Px; i += blockDim.x) tx[i] = twx[i];
  const float2* src = ws + c * a.P3;
  for (int i = threadIdx.x; i < kSlabRY * a.Px; i += blockDim.x) {
    const int kx = udiv(i, a.mag_RY), r = i - kx * kSlabRY;
    A[r * pitch + sw(kx)] = r < nr ? src[((int64_t)kx * a.nz + z) * a.ny + y0 + r]
                                   : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const Lines rows{kSlabRY, pitch, 1, 0, false};
  const float2* res = fft_smem_slab<float2, false>(A, B, tx, a.px, rows, true);
  float2* dst = phi + c * a.ng + ((int64_t)z * a.ny + y0) * a.nx;
  for (int i = threadIdx.x; i < kSlabRY * a.nx; i += blockDim.x) {
    const int r = i / a.nx, x = i - r * a.nx;
    if (r < nr) dst[(int64_t)r * a.nx + x] = res[r * pitch + sw(x)];
  }
}

// Warp-line forms of the three slab passes, for planes whose x and y lengths are 32 M points
// (M = 16 or 32): one warp holds one line, point n = lane + 32 n1 in register n1, and
// transforms it in registers (the M-point DFTs, the twiddles W_P^(lane k1) read from the table,
// five xor-shuffle stages across the lanes), leaving X[k1 + M bitrev(lane)] in register k1; the
// inverse takes that order back. No Stockham passes through shared memory: the x passes keep
// every value in registers, the y-z pass meets the nz lines of one kx in one shared buffer for
// the z transforms.
template <int M>
__device__ __forceinline__ void wline_fwd(float2* v, const float2* __restrict__ tw, int lane) {
  constexpr int P = 32 * M;
  dft_reg<float2, M>(v, tw, P / M, false);
#pragma unroll
  for (int k1 = 1; k1 < M; ++k1) v[k1] = cmul(v[k1], __ldg(&tw[lane * k1]));
#pragma unroll
  for (int st = 0; st < 5; ++st) {
    const int sp = 32 >> (st + 1);
    const bool top = (lane & sp) == 0;
    const float sg = top ? 1.f : -1.f;
    const float2 we = top ? make_float2(1.f, 0.f) : __ldg(&tw[(lane & (sp - 1)) * (M << st)]);
#pragma unroll
    for (int k1 = 0; k1 < M; ++k1) {
      const float2 p = shfl_x(v[k1], sp);
      v[k1] = cmul(make_float2(sg * v[k1].x + p.x, sg * v[k1].y + p.y), we);
    }
  }
}

template <int M>
__device__ __forceinline__ void wline_inv(float2* v, const float2* __restrict__ tw, int lane) {
  constexpr int P = 32 * M;
#pragma unroll
  for (int st = 4; st >= 0; --st) {
    const int sp = 32 >> (st + 1);
    const bool top = (lane & sp) == 0;
    const float sg = top ? 1.f : -1.f;
    float2 we = make_float2(1.f, 0.f);
    if (!top) {
      we = __ldg(&tw[(lane & (sp - 1)) * (M << st)]);
      we.y = -we.y;
    }
#pragma unroll
    for (int k1 = 0; k1 < M; ++k1) {
      const float2 own = cmul(v[k1], we);
      const float2 p = shfl_x(own, sp);
      v[k1] = make_float2(sg * own.x + p.x, sg * own.y + p.y);
    }
  }
#pragma unroll
  for (int k1 = 1; k1 < M; ++k1) {
    float2 w = __ldg(&tw[lane * k1]);
    w.y = -w.y;
    v[k1] = cmul(v[k1], w);
  }
  dft_reg<float2, M>(v, tw, P / M, true);
}

// x forward: warp w takes row y0 + w of data plane z; its Px spectrum values meet the other
// seven rows' in a shared tile [row][kx] (every 32nd entry skipped: two lanes per bank at most)
// and leave as X[c][kx][z][y0 .. y0 + 7], 64-byte runs, instead of one 8-byte value per kx
template <int M>
__global__ void __launch_bounds__(256) k_wslab_xfwd(const float2* __restrict__ sigma,
                                                    float2* __restrict__ ws,
                                                    const float2* __restrict__ twx, SlabArgs a) {
  extern __shared__ float2 tile[];  // [8 rows][TS]
  constexpr int P = 32 * M, TS = P + P / 32 + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int y0 = blockIdx.x * 8, y = y0 + warp, z = blockIdx.y, c = blockIdx.z;
  if (y < a.ny) {  // warp-uniform
    const float2* src = sigma + c * a.ng + ((int64_t)z * a.ny + y) * a.nx;
    float2 v[M];
#pragma unroll
    for (int n1 = 0; n1 < M; ++n1) {
      const int x = lane + 32 * n1;
      v[n1] = x < a.nx ? src[x] : make_float2(0.f, 0.f);
    }
    wline_fwd<M>(v, twx, lane);
    const int k2 = brev_l<32>(lane);
#pragma unroll
    for (int k1 = 0; k1 < M; ++k1) {
      const int kx = k1 + M * k2;
      tile[warp * TS + kx + (kx >> 5)] = v[k1];
    }
  }
  __syncthreads();
  const int nr = min(8, a.ny - y0);
  float2* dst = ws + c * a.P3 + (int64_t)z * a.ny + y0;
  for (int i = threadIdx.x; i < 8 * P; i += blockDim.x) {
    const int kx = i >> 3, r = i & 7;
    if (r < nr) dst[(int64_t)kx * a.nz * a.ny + r] = tile[r * TS + kx + (kx >> 5)];
  }
}

// y-z fused for one kx: warp z transforms its y line, the nz lines meet in shared memory
// (position k1 * 32 + lane) for the z DFTs and Ghat, then each warp inverts its line. Ghat is
// read where it is used (each value serves the two positions ky and P - ky of this CTA, the
// slab stays in L2 across kx and Px - kx and the components) rather than staged: without its
// 33 KB the CTA's shared memory is the 64 KB of its nz lines, three CTAs per SM instead of two.
template <int M, int MZ>
__global__ void __launch_bounds__(256) k_wslab_yz(float2* __restrict__ ws,
                                                  const float2* __restrict__ gs,
                                                  const float2* __restrict__ twy,
                                                  const float2* __restrict__ twz, SlabArgs a) {
  extern __shared__ unsigned char smem_raw[];
  float2* S = reinterpret_cast<float2*>(smem_raw);  // [z][32 M]
  constexpr int P = 32 * M;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kx = blockIdx.x, c = blockIdx.y;
  const int fx = min(kx, a.Px - kx);
  const float2* G = gs + (int64_t)fx * a.gz * a.gy;  // this kx's Ghat slab [fz][fy]
  float2* X = ws + c * a.P3 + (int64_t)kx * a.nz * a.ny;  // [z][y]
  for (int z = warp; z < a.nz; z += 8) {
    float2 v[M];
#pragma unroll
    for (int n1 = 0; n1 < M; ++n1) {
      const int y = lane + 32 * n1;
      v[n1] = y < a.ny ? X[(int64_t)z * a.ny + y] : make_float2(0.f, 0.f);
    }
    wline_fwd<M>(v, twy, lane);
#pragma unroll
    for (int k1 = 0; k1 < M; ++k1) S[z * P + k1 * 32 + lane] = v[k1];
  }
  __syncthreads();
  for (int pos = threadIdx.x; pos < P; pos += blockDim.x) {
    const int ky = (pos >> 5) + M * brev_l<32>(pos & 31);
    const int fy = min(ky, P - ky);
    float2 v[MZ];
#pragma unroll
    for (int z = 0; z < MZ; ++z) v[z] = z < a.nz ? S[z * P + pos] : make_float2(0.f, 0.f);
    dft_reg<float2, MZ>(v, twz, 1, false);
#pragma unroll
    for (int kz = 0; kz < MZ; ++kz) v[kz] = cmul(v[kz], __ldg(&G[min(kz, MZ - kz) * a.gy + fy]));
    dft_reg<float2, MZ>(v, twz, 1, true);
#pragma unroll
    for (int z = 0; z < MZ; ++z)
      if (z < a.nz) S[z * P + pos] = v[z];
  }
  __syncthreads();
  for (int z = warp; z < a.nz; z += 8) {
    float2 v[M];
#pragma unroll
    for (int k1 = 0; k1 < M; ++k1) v[k1] = S[z * P + k1 * 32 + lane];
    wline_inv<M>(v, twy, lane);
#pragma unroll
    for (int n1 = 0; n1 < M; ++n1) {
      const int y = lane + 32 * n1;
      if (y < a.ny) X[(int64_t)z * a.ny + y] = v[n1];
    }
  }
}

// x inverse: the CTA reads X[c][kx][z][y0 .. y0 + 7] as 64-byte runs into the shared tile; warp
// w takes row y0 + w from it in the transform's order, inverts it and writes the nx kept values
template <int M>
__global__ void __launch_bounds__(256) k_wslab_xinv(const float2* __restrict__ ws,
                                                    float2* __restrict__ phi,
                                                    const float2* __restrict__ twx, SlabArgs a) {
  extern __shared__ float2 tile[];  // [8 rows][TS]
  constexpr int P = 32 * M, TS = P + P / 32 + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int y0 = blockIdx.x * 8, y = y0 + warp, z = blockIdx.y, c = blockIdx.z;
  const int nr = min(8, a.ny - y0);
  const float2* src = ws + c * a.P3 + (int64_t)z * a.ny + y0;
  for (int i = threadIdx.x; i < 8 * P; i += blockDim.x) {
    const int kx = i >> 3, r = i & 7;
    if (r < nr) tile[r * TS + kx + (kx >> 5)] = src[(int64_t)kx * a.nz * a.ny + r];
  }
  __syncthreads();
  if (y >= a.ny) return;  // warp-uniform
  const int k2 = brev_l<32>(lane);
  float2 v[M];
#pragma unroll
  for (int k1 = 0; k1 < M; ++k1) {
    const int kx = k1 + M * k2;
    v[k1] = tile[warp * TS + kx + (kx >> 5)];
  }
  wline_inv<M>(v, twx, lane);
  float2* dst = phi + c * a.ng + ((int64_t)z * a.ny + y) * a.nx;
#pragma unroll
  for (int n1 = 0; n1 < M; ++n1) {
    const int x = lane + 32 * n1;
    if (x < a.nx) dst[x] = v[n1];
  }
}

// Ghat octant [fz][fy][fx] -> [fx][fz][fy] for the y-z pass (one contiguous slab per kx)
__global__ void k_ghat_slab(const float2* __restrict__ oct, int gx, int gy, int gz, float2* gs) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)gx * gy * gz) return;
  const int fy = (int)(i % gy);
  const int64_t t = i / gy;
  const int fz = (int)(t % gz), fx = (int)(t / gz);
  gs[i] = oct[((int64_t)fz * gy + fy) * gx + fx];
}

static size_t slab_x_smem(int Px) { return ((size_t)Px + 2 * (size_t)kSlabRY * sw_len(Px)) * sizeof(float2); }
static size_t slab_yz_smem(int Py, int nz, int Pz) {
  return ((size_t)Py + Pz + (size_t)(Pz / 2 + 1) * (Py / 2 + 1) + 2 * (size_t)nz * sw_len(Py)) *
         sizeof(float2);
}

typedef void (*SlabYZ)(float2*, const float2*, const float2*, const float2*, SlabArgs);
static SlabYZ slab_yz_kernel(int Pz) {
  switch (Pz) {
    case 8: return k_slab_yz<8>;
    case 9: return k_slab_yz<9>;
    case 10: return k_slab_yz<10>;
    case 12: return k_slab_yz<12>;
    case 15: return k_slab_yz<15>;
    case 16: return k_slab_yz<16>;
    default: return k_slab_yz<0>;
  }
}

// the FP32 convolution takes the slab passes when a padded plane does not fit shared memory
bool slab_path(const aim_ctx* c) {
  const int Px = c->gp[0], Py = c->gp[1], Pz = c->gp[2], nz = c->gn[2];
  return plane_smem<float2>(Px, Py) > kSmemBudget && nz <= kSlabMaxNz &&
         slab_x_smem(Px) <= kSmemBudget && slab_yz_smem(Py, nz, Pz) <= kSmemBudget;
}

static int slab_conv(aim_ctx* c, PrecBuf<float>& b, const float2* sigma, float2* phi, int ncomp,
                     float2* ws, cudaStream_t s) {
  SlabArgs a;
  a.nx = c->gn[0]; a.ny = c->gn[1]; a.nz = c->gn[2];
  a.Px = c->gp[0]; a.Py = c->gp[1]; a.Pz = c->gp[2];
  a.ng = c->ng; a.P3 = (int64_t)a.Px * a.Py * a.Pz;
  if (!make_fft_plan_r32(a.Px, &a.px) || !make_fft_plan_r32(a.Py, &a.py)) {
    set_error("slab convolution: no FFT plan for %d x %d", a.Px, a.Py);
    return BEM_EINVAL;
  }
  a.gy = a.Py / 2 + 1; a.gz = a.Pz / 2 + 1;
  a.mag_Px = div_magic(a.Px); a.mag_Py = div_magic(a.Py); a.mag_ny = div_magic(a.ny);
  a.mag_RY = div_magic(kSlabRY);
  // the warp-line forms: both in-plane lengths 1024 (or 512) and a z length the register DFT
  // takes
  if (a.Px == a.Py && (a.Px == 1024 || a.Px == 512) && a.nz <= 8 && a.Pz == 15) {
    const dim3 gw((a.ny + 7) / 8, a.nz, ncomp);
    const size_t ssm = (size_t)a.nz * a.Py * sizeof(float2);
    const size_t tsm = 8 * (size_t)(a.Px + a.Px / 32 + 1) * sizeof(float2);  // the x passes' tile
    if (a.Px == 1024) {
      k_wslab_xfwd<32><<<gw, 256, tsm, s>>>(sigma, ws, b.tw[0], a);
      k_wslab_yz<32, 15><<<dim3(a.Px, ncomp), 256, ssm, s>>>(ws, b.Gs, b.tw[1], b.tw[2], a);
      k_wslab_xinv<32><<<gw, 256, tsm, s>>>(ws, phi, b.tw[0], a);
    } else {
      k_wslab_xfwd<16><<<gw, 256, tsm, s>>>(sigma, ws, b.tw[0], a);
      k_wslab_yz<16, 15><<<dim3(a.Px, ncomp), 256, ssm, s>>>(ws, b.Gs, b.tw[1], b.tw[2], a);
      k_wslab_xinv<16><<<gw, 256, tsm, s>>>(ws, phi, b.tw[0], a);
    }
    BEM_CUDA(cudaGetLastError());
    return BEM_OK;
  }
  const dim3 gx((a.ny + kSlabRY - 1) / kSlabRY, a.nz, ncomp);
  k_slab_xfwd<<<gx, 256, slab_x_smem(a.Px), s>>>(sigma, ws, b.tw[0], a);
  slab_yz_kernel(a.Pz)<<<dim3(a.Px, ncomp), 256, slab_yz_smem(a.Py, a.nz, a.Pz), s>>>(
      ws, b.Gs, b.tw[1], b.tw[2], a);
  k_slab_xinv<<<gx, 256, slab_x_smem(a.Px), s>>>(ws, phi, b.tw[0], a);
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

int fft_init_attrs() {
  const int lim = (int)kSmemBudget;
  BEM_CUDA(cudaFuncSetAttribute(k_lines<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  BEM_CUDA(cudaFuncSetAttribute(k_lines<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  BEM_CUDA(cudaFuncSetAttribute(k_plane_fwd<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  BEM_CUDA(cudaFuncSetAttribute(k_plane_fwd<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  BEM_CUDA(cudaFuncSetAttribute(k_plane_inv<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  BEM_CUDA(cudaFuncSetAttribute(k_plane_inv<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  BEM_CUDA(cudaFuncSetAttribute(k_zfused<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  BEM_CUDA(cudaFuncSetAttribute(k_zfused<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  BEM_CUDA(cudaFuncSetAttribute(k_slab_xfwd, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  for (int pz : {8, 9, 10, 12, 15, 16, 0})
    BEM_CUDA(cudaFuncSetAttribute(slab_yz_kernel(pz), cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  BEM_CUDA(cudaFuncSetAttribute(k_wslab_yz<32, 15>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  BEM_CUDA(cudaFuncSetAttribute(k_wslab_xfwd<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  BEM_CUDA(cudaFuncSetAttribute(k_wslab_xinv<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  BEM_CUDA(cudaFuncSetAttribute(k_wslab_xfwd<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  BEM_CUDA(cudaFuncSetAttribute(k_wslab_xinv<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  BEM_CUDA(cudaFuncSetAttribute(k_wslab_yz<16, 15>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  BEM_CUDA(cudaFuncSetAttribute(k_slab_xinv, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
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
             int ncomp, typename C2<R>::T* ws, cudaStream_t s) {
  typedef typename C2<R>::T V;
  const int nx = c->gn[0], ny = c->gn[1], nz = c->gn[2];
  const int Px = c->gp[0], Py = c->gp[1], Pz = c->gp[2];
  const int64_t P3 = (int64_t)Px * Py * Pz, ng = c->ng;
  const size_t psm = plane_smem<V>(Px, Py);
  if (psm <= kSmemBudget) {
    PlaneArgs a;
    a.nx = nx; a.ny = ny; a.nz = nz; a.Px = Px; a.Py = Py; a.Pz = Pz;
    a.ng = ng; a.P3 = P3;
    a.px = c->plan[0]; a.py = c->plan[1]; a.pz = c->plan[2];
    a.gx = Px / 2 + 1; a.gy = Py / 2 + 1;
    const size_t avail = 64 * 1024 / sizeof(V);
    const size_t zp = sw_len(Pz);
    a.TL = (int)std::max<size_t>(1, std::min<size_t>(16, (avail - Pz) / (2 * zp)));
    a.mag_Px = div_magic(Px);
    a.mag_nx = div_magic(nx);
    a.mag_TL = div_magic(a.TL);
    a.mag_Pz = div_magic(Pz);
    const size_t zsm = ((size_t)Pz + 2 * (size_t)a.TL * zp) * sizeof(V);
    // the register forms for FP32 (FP64 runs at a small fraction of the FP32 rate on this GPU
    // and needs twice the registers: it keeps the shared-memory passes)
    int xl = 0, xm = 0, zl = 0, zm = 0;
    const size_t rsm = ((size_t)Px + Py + (size_t)ny * (Px + 1)) * sizeof(V);
    bool fwd_done = false, z_done = false, inv_done = false;
    if constexpr (sizeof(V) == sizeof(float2)) {
      if (Px == Py && reg_shape(Px, &xl, &xm) && rsm <= 48 * 1024) {
        fwd_done = launch_plane_reg<V>(false, xl, xm, dim3(nz, ncomp), rsm, s, sigma, ws, b.tw[0],
                                       b.tw[1], a);
        inv_done = true;  // launched below, after the z pass
      }
      if (reg_shape(Pz, &zl, &zm)) z_done = true;
    }
    if (!fwd_done) k_plane_fwd<V><<<dim3(nz, ncomp), 512, psm, s>>>(sigma, ws, b.tw[0], b.tw[1], a);
    if constexpr (sizeof(V) == sizeof(float2)) {
      if (z_done) {
        const int per = 8 * (32 / zl);  // x lines per CTA
        launch_zreg<V>(zl, zm, dim3((Px + per - 1) / per, Py, ncomp), s, ws, b.Ghat, b.Gz, b.tw[2], a);
      }
    }
    if (!z_done)
      k_zfused<V><<<dim3((Px + a.TL - 1) / a.TL, Py, ncomp), 256, zsm, s>>>(ws, b.Ghat, b.tw[2], a);
    if constexpr (sizeof(V) == sizeof(float2)) {
      if (inv_done)
        inv_done = launch_plane_reg<V>(true, xl, xm, dim3(nz, ncomp), rsm, s, ws, phi, b.tw[0],
                                       b.tw[1], a);
    }
    if (!inv_done) k_plane_inv<V><<<dim3(nz, ncomp), 512, psm, s>>>(ws, phi, b.tw[0], b.tw[1], a);
    BEM_CUDA(cudaGetLastError());
    return BEM_OK;
  }
  if constexpr (sizeof(V) == sizeof(float2)) {
    if (b.Gs) return slab_conv(c, b, sigma, phi, ncomp, ws, s);
  }
  LinePass p{};
  // X forward
  p.P = Px; p.nin = nx; p.nout = Px; p.ies = 1; p.oes = 1;
  p.n0 = ny; p.n1 = nz; p.is0 = nx; p.is1 = (int64_t)ny * nx; p.is2 = ng;
  p.os0 = Px; p.os1 = (int64_t)Py * Px; p.os2 = P3; p.plan = c->plan[0];
  BEM_TRY(launch_lines<V>(sigma, ws, b.tw[0], nullptr, p, ncomp, s));
  // Y forward
  p = LinePass{};
  p.P = Py; p.nin = ny; p.nout = Py; p.ies = Px; p.oes = Px;
  p.n0 = Px; p.n1 = nz; p.is0 = 1; p.is1 = (int64_t)Py * Px; p.is2 = P3;
  p.os0 = 1; p.os1 = (int64_t)Py * Px; p.os2 = P3; p.plan = c->plan[1];
  BEM_TRY(launch_lines<V>(ws, ws, b.tw[1], nullptr, p, ncomp, s));
  // Z forward * Ghat * Z inverse
  p = LinePass{};
  p.P = Pz; p.nin = nz; p.nout = nz; p.ies = (int64_t)Py * Px; p.oes = (int64_t)Py * Px;
  p.n0 = Px; p.n1 = Py; p.is0 = 1; p.is1 = Px; p.is2 = P3;
  p.os0 = 1; p.os1 = Px; p.os2 = P3; p.fused = 1; p.plan = c->plan[2];
  p.gx = Px / 2 + 1; p.gy = Py / 2 + 1; p.Px = Px; p.Py = Py;
  BEM_TRY(launch_lines<V>(ws, ws, b.tw[2], b.Ghat, p, ncomp, s));
  // Y inverse
  p = LinePass{};
  p.P = Py; p.nin = Py; p.nout = ny; p.ies = Px; p.oes = Px; p.inverse = 1;
  p.n0 = Px; p.n1 = nz; p.is0 = 1; p.is1 = (int64_t)Py * Px; p.is2 = P3;
  p.os0 = 1; p.os1 = (int64_t)Py * Px; p.os2 = P3; p.plan = c->plan[1];
  BEM_TRY(launch_lines<V>(ws, ws, b.tw[1], nullptr, p, ncomp, s));
  // X inverse
  p = LinePass{};
  p.P = Px; p.nin = Px; p.nout = nx; p.ies = 1; p.oes = 1; p.inverse = 1;
  p.n0 = ny; p.n1 = nz; p.is0 = Px; p.is1 = (int64_t)Py * Px; p.is2 = P3;
  p.os0 = nx; p.os1 = (int64_t)ny * nx; p.os2 = ng; p.plan = c->plan[0];
  BEM_TRY(launch_lines<V>(ws, phi, b.tw[0], nullptr, p, ncomp, s));
  return BEM_OK;
}
template int fft_conv<float>(aim_ctx*, PrecBuf<float>&, const float2*, float2*, int, float2*,
                              cudaStream_t);
template int fft_conv<double>(aim_ctx*, PrecBuf<double>&, const double2*, double2*, int, double2*,
                               cudaStream_t);

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
  rc = launch_lines<double2>(G, G, c->f64.tw[0], nullptr, p, 1, 0);
  if (rc == BEM_OK) {
    p = LinePass{};
    p.P = Py; p.nin = Py; p.nout = Py; p.ies = Px; p.oes = Px;
    p.n0 = Px; p.n1 = Pz; p.is0 = 1; p.is1 = (int64_t)Py * Px; p.is2 = P3;
    p.os0 = 1; p.os1 = (int64_t)Py * Px; p.os2 = P3; p.plan = c->plan[1];
    rc = launch_lines<double2>(G, G, c->f64.tw[1], nullptr, p, 1, 0);
  }
  if (rc == BEM_OK) {
    p = LinePass{};
    p.P = Pz; p.nin = Pz; p.nout = Pz; p.ies = (int64_t)Py * Px; p.oes = (int64_t)Py * Px;
    p.n0 = Px; p.n1 = Py; p.is0 = 1; p.is1 = Px; p.is2 = P3;
    p.os0 = 1; p.os1 = Px; p.os2 = P3; p.plan = c->plan[2];
    rc = launch_lines<double2>(G, G, c->f64.tw[2], nullptr, p, 1, 0);
  }
  const int64_t no = (int64_t)(Px / 2 + 1) * (Py / 2 + 1) * (Pz / 2 + 1);
  if (rc == BEM_OK) rc = dalloc_t(c, &c->f64.Ghat, no);
  if (rc == BEM_OK) rc = dalloc_t(c, &c->f32.Ghat, no);
  int zl = 0, zm = 0;
  if (rc == BEM_OK && reg_shape(Pz, &zl, &zm)) rc = dalloc_t(c, &c->f32.Gz, P3);
  if (rc == BEM_OK && slab_path(c)) rc = dalloc_t(c, &c->f32.Gs, no);
  if (rc == BEM_OK) {
    k_ghat_oct<<<(unsigned)((no + 255) / 256), 256>>>(G, Px, Py, Pz, 1.0 / (double)P3, c->f64.Ghat,
                                                      c->f32.Ghat);
    if (c->f32.Gz) {  // the register z pass's lane order of each line
      const unsigned nb = (unsigned)((P3 + 255) / 256);
      if (zl == 32) k_ghat_lines<float2, 32><<<nb, 256>>>(c->f32.Ghat, zm, Px, Py, Pz, c->f32.Gz);
      else if (zl == 16) k_ghat_lines<float2, 16><<<nb, 256>>>(c->f32.Ghat, zm, Px, Py, Pz, c->f32.Gz);
      else k_ghat_lines<float2, 8><<<nb, 256>>>(c->f32.Ghat, zm, Px, Py, Pz, c->f32.Gz);
    }
    if (c->f32.Gs)
      k_ghat_slab<<<(unsigned)((no + 255) / 256), 256>>>(c->f32.Ghat, Px / 2 + 1, Py / 2 + 1,
                                                          Pz / 2 + 1, c->f32.Gs);
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
