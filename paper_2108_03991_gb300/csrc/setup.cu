// Device set-up (FP64): projection stencils, the dense internal matrices Z_i and Y_i,eq, and
// the precorrected near-region matrices L^A_NR and L^Phi_NR.
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <memory>

#include "common.cuh"
#include "quad.cuh"

namespace bem {

double wall_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

void build_ix_fd(const aim_ctx* c, std::vector<int32_t>* ixcol, std::vector<double>* ixval,
                 std::vector<double>* fdE, std::vector<double>* fdT);

// ---------------------------------------------------------------------------------------
// rules (host)
// ---------------------------------------------------------------------------------------
void radon7_host(double* out) {  // (l1, l2, l3, w) x 7, weights sum to one
  const double s = std::sqrt(15.0);
  const double a1 = (6.0 - s) / 21.0, a2 = (6.0 + s) / 21.0;
  const double w1 = (155.0 - s) / 1200.0, w2 = (155.0 + s) / 1200.0;
  const double pts[7][4] = {{1.0 / 3, 1.0 / 3, 1.0 / 3, 9.0 / 40.0},
                            {a1, a1, 1 - 2 * a1, w1}, {a1, 1 - 2 * a1, a1, w1}, {1 - 2 * a1, a1, a1, w1},
                            {a2, a2, 1 - 2 * a2, w2}, {a2, 1 - 2 * a2, a2, w2}, {1 - 2 * a2, a2, a2, w2}};
  for (int i = 0; i < 7; ++i)
    for (int k = 0; k < 4; ++k) out[4 * i + k] = pts[i][k];
}

static void subdivide4_host(const double* in, int nq, double* out) {
  const double V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  double m01[3], m12[3], m20[3];
  for (int a = 0; a < 3; ++a) {
    m01[a] = 0.5 * (V[0][a] + V[1][a]);
    m12[a] = 0.5 * (V[1][a] + V[2][a]);
    m20[a] = 0.5 * (V[2][a] + V[0][a]);
  }
  const double* subs[4][3] = {{V[0], m01, m20}, {m01, V[1], m12}, {m20, m12, V[2]}, {m01, m12, m20}};
  int o = 0;
  for (int s = 0; s < 4; ++s)
    for (int q = 0; q < nq; ++q, ++o) {
      for (int a = 0; a < 3; ++a)
        out[4 * o + a] = in[4 * q] * subs[s][0][a] + in[4 * q + 1] * subs[s][1][a] + in[4 * q + 2] * subs[s][2][a];
      out[4 * o + 3] = in[4 * q + 3] / 4.0;
    }
}

// Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_n.
static void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// collapsed (Duffy) product rule with 5 x 5 points: l1 = u, l2 = v (1 - u), weight 2 wu wv (1 - u)
static void gauss_tri5_host(double* out) {
  double x[5], w[5];
  gauss_legendre(5, x, w);
  int o = 0;
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j, ++o) {
      double u = 0.5 * (x[i] + 1.0), v = 0.5 * (x[j] + 1.0);
      double wu = 0.5 * w[i], wv = 0.5 * w[j];
      out[4 * o] = u;
      out[4 * o + 1] = v * (1.0 - u);
      out[4 * o + 2] = 1.0 - out[4 * o] - out[4 * o + 1];
      out[4 * o + 3] = 2.0 * wu * wv * (1.0 - u);
    }
}

static int upload_rules() {
  double r7[28], r28[112], gl[100];
  radon7_host(r7);
  subdivide4_host(r7, 7, r28);
  gauss_tri5_host(gl);
  BEM_CUDA(cudaMemcpyToSymbol(c_r7, r7, sizeof(r7)));
  BEM_CUDA(cudaMemcpyToSymbol(c_r28, r28, sizeof(r28)));
  BEM_CUDA(cudaMemcpyToSymbol(c_gl, gl, sizeof(gl)));
  double xg[kNgl], wg[kNgl], gx[2 * kNgl];
  gauss_legendre(kNgl, xg, wg);
  for (int i = 0; i < kNgl; ++i) {
    gx[i] = 0.5 * (xg[i] + 1.0);
    gx[kNgl + i] = 0.5 * wg[i];
  }
  BEM_CUDA(cudaMemcpyToSymbol(c_glx, gx, sizeof(gx)));
  return BEM_OK;
}

// ---------------------------------------------------------------------------------------
// device geometry (FP64)
// ---------------------------------------------------------------------------------------
struct DGeo {
  const double* verts;
  const int32_t* tris;
  const double* nrm;
  const double* area;
  const double* diam;
  const double* cen;
  const int32_t* et;    // [ne][2]
  const int32_t* eopp;  // [ne][2]
  const double* elen;
  const int32_t* anc;   // [(ne+nt)][3]
  double go[3], gh[3];
};

__device__ __forceinline__ void lag3(double u, double* l) {
  l[0] = 0.5 * u * (u - 1.0);
  l[1] = 1.0 - u * u;
  l[2] = 0.5 * u * (u + 1.0);
}

// P[m][c][k] = int f_m,c(r) l_k(r) dS  (Lagrange polynomial of stencil node k of m's anchor);
// one thread per (RWG, node), exact 25-point rule.
__global__ void k_weights_e(DGeo g, int ne, double* W64, float* W32) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)ne * 27) return;
  int m = (int)(idx / 27), k = (int)(idx % 27);
  int kx = k % 3, ky = (k / 3) % 3, kz = k / 9;
  double org[3];
  for (int a = 0; a < 3; ++a) org[a] = g.go[a] + g.anc[3 * m + a] * g.gh[a];
  double acc[3] = {0, 0, 0};
  for (int side = 0; side < 2; ++side) {
    int t = g.et[2 * m + side];
    const double* v = &g.verts[3 * g.eopp[2 * m + side]];
    double cf = (side == 0 ? 1.0 : -1.0) * g.elen[m] / (2.0 * g.area[t]);
    double X[3][3];
    for (int q = 0; q < 3; ++q)
      for (int a = 0; a < 3; ++a) X[q][a] = g.verts[3 * g.tris[3 * t + q] + a];
    for (int q = 0; q < 25; ++q) {
      double r[3];
      for (int a = 0; a < 3; ++a) r[a] = c_gl[4 * q] * X[0][a] + c_gl[4 * q + 1] * X[1][a] + c_gl[4 * q + 2] * X[2][a];
      double lx[3], ly[3], lz[3];
      lag3((r[0] - org[0]) / g.gh[0], lx);
      lag3((r[1] - org[1]) / g.gh[1], ly);
      lag3((r[2] - org[2]) / g.gh[2], lz);
      double wl = c_gl[4 * q + 3] * g.area[t] * lx[kx] * ly[ky] * lz[kz] * cf;
      for (int a = 0; a < 3; ++a) acc[a] += wl * (r[a] - v[a]);
    }
  }
  for (int a = 0; a < 3; ++a) {
    W64[(int64_t)m * 81 + a * 27 + k] = acc[a];
    W32[(int64_t)m * 81 + a * 27 + k] = (float)acc[a];
  }
}

// P_Phi[t][k] = int_t l_k(r) dS
__global__ void k_weights_t(DGeo g, int ne, int nt, double* W64, float* W32) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)nt * 27) return;
  int t = (int)(idx / 27), k = (int)(idx % 27);
  int kx = k % 3, ky = (k / 3) % 3, kz = k / 9;
  double org[3];
  for (int a = 0; a < 3; ++a) org[a] = g.go[a] + g.anc[3 * (ne + t) + a] * g.gh[a];
  double X[3][3];
  for (int q = 0; q < 3; ++q)
    for (int a = 0; a < 3; ++a) X[q][a] = g.verts[3 * g.tris[3 * t + q] + a];
  double acc = 0;
  for (int q = 0; q < 25; ++q) {
    double r[3];
    for (int a = 0; a < 3; ++a) r[a] = c_gl[4 * q] * X[0][a] + c_gl[4 * q + 1] * X[1][a] + c_gl[4 * q + 2] * X[2][a];
    double lx[3], ly[3], lz[3];
    lag3((r[0] - org[0]) / g.gh[0], lx);
    lag3((r[1] - org[1]) / g.gh[1], ly);
    lag3((r[2] - org[2]) / g.gh[2], lz);
    acc += c_gl[4 * q + 3] * g.area[t] * lx[kx] * ly[ky] * lz[kz];
  }
  W64[(int64_t)t * 27 + k] = acc;
  W32[(int64_t)t * 27 + k] = (float)acc;
}

// weights in CSR order: WT[e][c] = W[src[e]][c][k[e]] (ncomp = 3 for RWG, 1 for pulses)
__global__ void k_weights_csr(const int32_t* src, const int32_t* kk, const double* W, int64_t nent,
                              int ncomp, double* T64, float* T32) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nent) return;
  const int64_t m = src[e];
  const int k = kk[e];
  for (int cc = 0; cc < ncomp; ++cc) {
    double w = W[m * 27 * ncomp + cc * 27 + k];
    T64[e * ncomp + cc] = w;
    T32[e * ncomp + cc] = (float)w;
  }
}

// ---------------------------------------------------------------------------------------
// RWG entries from triangle-pair moments
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void half_rwg(const DGeo& g, int n, int t, double* sgn, const double** v) {
  if (g.et[2 * n] == t) { *sgn = 1.0; *v = &g.verts[3 * g.eopp[2 * n]]; }
  else { *sgn = -1.0; *v = &g.verts[3 * g.eopp[2 * n + 1]]; }
}

// kind 0: int int f.f G ; kind 1: L (with -k^-2 div div) ; returns K too when wantK
// int int (r - a).(r' - b) G dS' dS from the pair moments (origin o): a = va + o, b = vb + o
// are the free vertices of the two half-RWGs; the vector-potential kernel of L before its
// l_m l_n / (4 A A') factor
__device__ __forceinline__ double2 vec_term(const Moments& M, const double* va, const double* vb) {
  double2 v = M.M2;
  for (int q = 0; q < 3; ++q) {
    v.x += -M.M1[q].x * vb[q] - va[q] * M.M1p[q].x;
    v.y += -M.M1[q].y * vb[q] - va[q] * M.M1p[q].y;
  }
  const double vv = d_dot(va, vb);
  v.x += vv * M.M0.x;
  v.y += vv * M.M0.y;
  return v;
}

__device__ void rwg_pair(const DGeo& g, int m, int n, double kr, double ki, bool isL, bool wantK,
                         double2* Lval, double2* Kval) {
  double2 L = {0, 0}, K = {0, 0};
  // 1/k^2 for the divergence term
  double den = kr * kr + ki * ki;
  double2 ik2 = make_double2((kr * kr - ki * ki) / (den * den), -2.0 * kr * ki / (den * den));
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      int t = g.et[2 * m + a], s = g.et[2 * n + b];
      Tri T, S;
      load_tri(g.verts, g.tris, g.nrm, g.area, g.diam, g.cen, t, &T);
      load_tri(g.verts, g.tris, g.nrm, g.area, g.diam, g.cen, s, &S);
      const double o[3] = {T.c[0], T.c[1], T.c[2]};
      shift_pair(&T, &S);
      Moments M;
      pair_moments(T, S, kr, ki, true, wantK, false, &M);
      double sm, sn;
      const double *pa, *pb;
      half_rwg(g, m, t, &sm, &pa);
      half_rwg(g, n, s, &sn, &pb);
      const double va[3] = {pa[0] - o[0], pa[1] - o[1], pa[2] - o[2]};
      const double vb[3] = {pb[0] - o[0], pb[1] - o[1], pb[2] - o[2]};
      double cf = sm * sn * g.elen[m] * g.elen[n] / (4.0 * g.area[t] * g.area[s]);
      const double2 v = vec_term(M, va, vb);
      L.x += cf * v.x;
      L.y += cf * v.y;
      if (isL) {
        double dv = sm * sn * g.elen[m] * g.elen[n] / (g.area[t] * g.area[s]);
        double2 t2 = cmul(M.M0, ik2);
        L.x -= dv * t2.x;
        L.y -= dv * t2.y;
      }
      if (wantK) {
        double bxa[3];
        d_cross(vb, va, bxa);
        double2 kv = {0, 0};
        for (int q = 0; q < 3; ++q) {
          kv.x += M.U[q].x * (vb[q] - va[q]) + M.Vs[q].x * bxa[q];
          kv.y += M.U[q].y * (vb[q] - va[q]) + M.Vs[q].y * bxa[q];
        }
        K.x += cf * kv.x;
        K.y += cf * kv.y;
      }
    }
  *Lval = L;
  if (Kval) *Kval = K;
}

// Dense internal matrices of one object, in three passes over its triangle pairs (m triangles
// from t0, local pair index it * m + is): the moments of every regular and small-|k| near pair
// (one thread each), the large-|k| near pairs listed for the second pass; those by one warp each
// (the edge-integral scheme of quad.cuh); then every RWG entry from the four pair moments of its
// two triangles.
__global__ void k_obj_moments(DGeo g, int t0, int m, double kr, double ki, bool wantK,
                              Moments* mom, int* hk_list, int* hk_count) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)m * m) return;
  const int it = (int)(idx / m), is = (int)(idx % m);
  Tri T, S;
  load_tri(g.verts, g.tris, g.nrm, g.area, g.diam, g.cen, t0 + it, &T);
  load_tri(g.verts, g.tris, g.nrm, g.area, g.diam, g.cen, t0 + is, &S);
  const int kind = pair_kind(T, S, kr, ki);
  if (kind >= 2) {
    const int p = atomicAdd(hk_count, 1);
    hk_list[p] = (int)idx;  // at most m * m entries: the list holds them all
    mom[idx] = Moments{};   // the point kernel adds into it
    return;
  }
  shift_pair(&T, &S);
  Moments M;
  pair_moments(T, S, kr, ki, true, wantK, false, &M, kind);
  mom[idx] = M;
}

// outer rule points per large-|k| pair (one thread per pair)
__global__ void k_hk_count(DGeo g, int t0, int m, double kr, double ki, const int* hk_list,
                           int count, int* npts) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  const int idx = hk_list[p];
  Tri T, S;
  load_tri(g.verts, g.tris, g.nrm, g.area, g.diam, g.cen, t0 + idx / m, &T);
  load_tri(g.verts, g.tris, g.nrm, g.area, g.diam, g.cen, t0 + idx % m, &S);
  shift_pair(&T, &S);
  npts[p] = hk_count_points(T, S, kr, ki);
}

// the flat point list: item = pair * 512 + finest index * 8 + rule point, pairs in list order
__global__ void k_hk_items(DGeo g, int t0, int m, double kr, double ki, const int* hk_list,
                           int count, const int64_t* off, int32_t* items) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  const int idx = hk_list[p];
  Tri T, S;
  load_tri(g.verts, g.tris, g.nrm, g.area, g.diam, g.cen, t0 + idx / m, &T);
  load_tri(g.verts, g.tris, g.nrm, g.area, g.diam, g.cen, t0 + idx % m, &S);
  shift_pair(&T, &S);
  const int D = hk_depth(sqrt(kr * kr + ki * ki), T.diam);
  const bool cop = hk_coplanar(T, S);
  int64_t o = off[p];
  Sub leaf;
  for (int f = 0; f < (1 << (2 * D)); ++f)
    if (hk_leaf(T, S, D, cop, fabs(ki), f, &leaf))
      for (int q = 0; q < 7; ++q) items[o++] = p * 512 + f * 8 + q;
}

// one outer rule point per thread: its inner integrals, added into its pair's moments (a
// segmented sum over the warp's consecutive items of one pair, then one atomic add per pair
// and warp)
__global__ void __launch_bounds__(128) k_hk_points(DGeo g, int t0, int m, double kr, double ki,
                                                   bool wantK, const int* hk_list,
                                                   const int32_t* items, int64_t nitems,
                                                   Moments* mom) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  double acc[28];
  for (int a = 0; a < 28; ++a) acc[a] = 0.0;
  int p = -1;
  if (i < nitems) {
    const int32_t code = items[i];
    p = code >> 9;
    const int f = (code >> 3) & 63, q = code & 7;
    const int idx = hk_list[p];
    Tri T, S;
    load_tri(g.verts, g.tris, g.nrm, g.area, g.diam, g.cen, t0 + idx / m, &T);
    load_tri(g.verts, g.tris, g.nrm, g.area, g.diam, g.cen, t0 + idx % m, &S);
    shift_pair(&T, &S);
    const int D = hk_depth(sqrt(kr * kr + ki * ki), T.diam);
    Sub leaf;
    hk_leaf(T, S, D, hk_coplanar(T, S), fabs(ki), f, &leaf);
    double e1[3], e2[3], cr[3];
    d_sub(leaf.v[1], leaf.v[0], e1);
    d_sub(leaf.v[2], leaf.v[0], e2);
    d_cross(e1, e2, cr);
    const double area = 0.5 * sqrt(d_dot(cr, cr));
    const double l1 = c_r7[4 * q], l2 = c_r7[4 * q + 1], l3 = c_r7[4 * q + 2];
    const double r[3] = {l1 * leaf.v[0][0] + l2 * leaf.v[1][0] + l3 * leaf.v[2][0],
                         l1 * leaf.v[0][1] + l2 * leaf.v[1][1] + l3 * leaf.v[2][1],
                         l1 * leaf.v[0][2] + l2 * leaf.v[1][2] + l3 * leaf.v[2][2]};
    hk_point(r, c_r7[4 * q + 3] * area, S, kr, ki, wantK, acc);
  }
  // suffix sums within runs of equal p (items of a pair are consecutive)
  for (int o = 1; o < 32; o <<= 1) {
    const int po = __shfl_down_sync(0xffffffffu, p, o);
    const bool take = lane + o < 32 && po == p;
    for (int a = 0; a < 28; ++a) {
      const double v = __shfl_down_sync(0xffffffffu, acc[a], o);
      if (take) acc[a] += v;
    }
  }
  const int pu = __shfl_up_sync(0xffffffffu, p, 1);
  if (p >= 0 && (lane == 0 || pu != p)) {
    double* dst = reinterpret_cast<double*>(&mom[hk_list[p]]);
    // Moments layout: M0, M2, M1[3], M1p[3], U[3], Vs[3] (double2 each)
    const int map[28] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15,
                         22, 23, 24, 25, 26, 27, 16, 17, 18, 19, 20, 21};
    for (int a = 0; a < 28; ++a) atomicAdd(dst + map[a], acc[a]);
  }
}

// Lc = L_k, Bc = K_k + I_x/2 (column-major n x n) from the pair moments
__global__ void k_obj_assemble(DGeo g, int e0, int n, int t0, int m, double kr, double ki,
                               const Moments* __restrict__ mom, const int32_t* ixcol,
                               const double* ixval, double2* Lc, double2* Bc) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  const int i = (int)(idx % n), j = (int)(idx / n);  // column-major: consecutive threads walk a column
  const int mm = e0 + i, nn = e0 + j;
  const double den = kr * kr + ki * ki;
  const double2 ik2 = make_double2((kr * kr - ki * ki) / (den * den), -2.0 * kr * ki / (den * den));
  double2 L = {0, 0}, K = {0, 0};
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      const int t = g.et[2 * mm + a], sidx = g.et[2 * nn + b];
      const Moments& M = mom[(int64_t)(t - t0) * m + (sidx - t0)];
      double sm, sn;
      const double *pa, *pb;
      half_rwg(g, mm, t, &sm, &pa);
      half_rwg(g, nn, sidx, &sn, &pb);
      const double* o = &g.cen[3 * t];  // the moments' origin: t's centroid
      const double va[3] = {pa[0] - o[0], pa[1] - o[1], pa[2] - o[2]};
      const double vb[3] = {pb[0] - o[0], pb[1] - o[1], pb[2] - o[2]};
      const double cf = sm * sn * g.elen[mm] * g.elen[nn] / (4.0 * g.area[t] * g.area[sidx]);
      const double2 v = vec_term(M, va, vb);
      L.x += cf * v.x;
      L.y += cf * v.y;
      const double dv = sm * sn * g.elen[mm] * g.elen[nn] / (g.area[t] * g.area[sidx]);
      const double2 t2 = cmul(M.M0, ik2);
      L.x -= dv * t2.x;
      L.y -= dv * t2.y;
      double bxa[3];
      d_cross(vb, va, bxa);
      double2 kv = {0, 0};
      for (int q = 0; q < 3; ++q) {
        kv.x += M.U[q].x * (vb[q] - va[q]) + M.Vs[q].x * bxa[q];
        kv.y += M.U[q].y * (vb[q] - va[q]) + M.Vs[q].y * bxa[q];
      }
      K.x += cf * kv.x;
      K.y += cf * kv.y;
    }
  for (int q = 0; q < 4; ++q)
    if (ixcol[4 * mm + q] == nn) K.x += 0.5 * ixval[4 * mm + q];
  Lc[idx] = L;
  Bc[idx] = K;
}

// L^A of object obj (column-major n x n) from its pair moments at k0: the vector-potential part
// of L alone (Eq. AIM_L's exact counterpart, used by the preconditioner blocks)
__global__ void k_obj_assemble_A(DGeo g, int e0, int n, int t0, int m,
                                 const Moments* __restrict__ mom, double2* LAc) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  const int mm = e0 + (int)(idx % n), nn = e0 + (int)(idx / n);
  double2 L = {0, 0};
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      const int t = g.et[2 * mm + a], sidx = g.et[2 * nn + b];
      const Moments& M = mom[(int64_t)(t - t0) * m + (sidx - t0)];
      double sm, sn;
      const double *pa, *pb;
      half_rwg(g, mm, t, &sm, &pa);
      half_rwg(g, nn, sidx, &sn, &pb);
      const double* o = &g.cen[3 * t];
      const double va[3] = {pa[0] - o[0], pa[1] - o[1], pa[2] - o[2]};
      const double vb[3] = {pb[0] - o[0], pb[1] - o[1], pb[2] - o[2]};
      const double cf = sm * sn * g.elen[mm] * g.elen[nn] / (4.0 * g.area[t] * g.area[sidx]);
      const double2 v = vec_term(M, va, vb);
      L.x += cf * v.x;
      L.y += cf * v.y;
    }
  LAc[idx] = L;
}

// L^Phi of the object's pulses (column-major m x m): the M0 moment of each triangle pair
__global__ void k_obj_LP(const Moments* __restrict__ mom, int m, double2* LP) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)m * m) return;
  const int i = (int)(idx % m), j = (int)(idx / m);
  LP[idx] = mom[(int64_t)i * m + j].M0;
}

// Store alpha * X (column-major) into the packed row-major block (FP64 and FP32 copies).
__global__ void k_store_block(const double2* X, int n, int ld, double2 alpha, double2* Z64,
                              float2* Z32) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * ld) return;
  int r = (int)(idx / ld), col = (int)(idx % ld);
  double2 v = make_double2(0, 0);
  if (col < n) v = cmul(alpha, X[r + (int64_t)col * n]);
  Z64[idx] = v;
  if (Z32) Z32[idx] = make_float2((float)v.x, (float)v.y);
}

__global__ void k_round32(const double2* __restrict__ a, float2* __restrict__ o, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    o[i] = make_float2((float)a[i].x, (float)a[i].y);
}

// Near region of L^A: exact entry minus the grid's own contribution
//   sum_c sum_{a,b} P_c[m,a] G_grid(anc_m + o_a - anc_n - o_b) P_c[n,b].
// gtab holds G_grid at offsets (dx, dy, dz) in [-(R+2), R+2]^3.
__global__ void k_near_LA(DGeo g, int64_t nnz, const int32_t* rows, const int32_t* cols,
                          const double* WA, const double2* gtab, int R, double k0, double2* v64,
                          float2* v32) {
  extern __shared__ double2 sg[];
  const int span = 2 * R + 5;
  for (int i = threadIdx.x; i < span * span * span; i += blockDim.x) sg[i] = gtab[i];
  __syncthreads();
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= nnz) return;
  int m = rows[idx], n = cols[idx];
  double2 L;
  rwg_pair(g, m, n, k0, 0.0, false, false, &L, nullptr);
  int D[3];
  for (int a = 0; a < 3; ++a) D[a] = g.anc[3 * m + a] - g.anc[3 * n + a];
  double2 pre = {0, 0};
  const int h = R + 2;
  for (int ka = 0; ka < 27; ++ka) {
    int ax = ka % 3 - 1, ay = (ka / 3) % 3 - 1, az = ka / 9 - 1;
    double2 acc[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int kb = 0; kb < 27; ++kb) {
      int bx = kb % 3 - 1, by = (kb / 3) % 3 - 1, bz = kb / 9 - 1;
      int dx = D[0] + ax - bx + h, dy = D[1] + ay - by + h, dz = D[2] + az - bz + h;
      double2 G = sg[(dz * span + dy) * span + dx];
      for (int c = 0; c < 3; ++c) {
        double w = WA[(int64_t)n * 81 + c * 27 + kb];
        acc[c].x += G.x * w;
        acc[c].y += G.y * w;
      }
    }
    for (int c = 0; c < 3; ++c) {
      double w = WA[(int64_t)m * 81 + c * 27 + ka];
      pre.x += w * acc[c].x;
      pre.y += w * acc[c].y;
    }
  }
  double2 v = make_double2(L.x - pre.x, L.y - pre.y);
  v64[idx] = v;
  v32[idx] = make_float2((float)v.x, (float)v.y);
}

__global__ void k_near_LP(DGeo g, int ne, int64_t nnz, const int32_t* rows, const int32_t* cols,
                          const double* WP, const double2* gtab, int R, double k0, double2* v64,
                          float2* v32) {
  extern __shared__ double2 sg[];
  const int span = 2 * R + 5;
  for (int i = threadIdx.x; i < span * span * span; i += blockDim.x) sg[i] = gtab[i];
  __syncthreads();
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= nnz) return;
  int t = rows[idx], s = cols[idx];
  Tri T, S;
  load_tri(g.verts, g.tris, g.nrm, g.area, g.diam, g.cen, t, &T);
  load_tri(g.verts, g.tris, g.nrm, g.area, g.diam, g.cen, s, &S);
  Moments M;
  pair_moments(T, S, k0, 0.0, false, false, true, &M);
  int D[3];
  for (int a = 0; a < 3; ++a) D[a] = g.anc[3 * (ne + t) + a] - g.anc[3 * (ne + s) + a];
  double2 pre = {0, 0};
  const int h = R + 2;
  for (int ka = 0; ka < 27; ++ka) {
    int ax = ka % 3 - 1, ay = (ka / 3) % 3 - 1, az = ka / 9 - 1;
    double2 acc = {0, 0};
    for (int kb = 0; kb < 27; ++kb) {
      int bx = kb % 3 - 1, by = (kb / 3) % 3 - 1, bz = kb / 9 - 1;
      int dx = D[0] + ax - bx + h, dy = D[1] + ay - by + h, dz = D[2] + az - bz + h;
      double2 G = sg[(dz * span + dy) * span + dx];
      double w = WP[(int64_t)s * 27 + kb];
      acc.x += G.x * w;
      acc.y += G.y * w;
    }
    double w = WP[(int64_t)t * 27 + ka];
    pre.x += w * acc.x;
    pre.y += w * acc.y;
  }
  double2 v = make_double2(M.M0.x - pre.x, M.M0.y - pre.y);
  v64[idx] = v;
  v32[idx] = make_float2((float)v.x, (float)v.y);
}

// ---------------------------------------------------------------------------------------
// plane-wave right-hand side: b_m = <f_m, pol exp(-j k0 khat.r)> / eta0 (7-point rule)
// ---------------------------------------------------------------------------------------
template <typename V>
__global__ void k_rhs_pw(DGeo g, int ne, int nt, double k0, double px, double py, double pz,
                         double kx, double ky, double kz, double inv_eta0, V* b) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= ne + nt) return;
  if (m >= ne) { b[m] = czero<V>(); return; }
  double2 acc = {0, 0};
  const double pol[3] = {px, py, pz}, kh[3] = {kx, ky, kz};
  for (int side = 0; side < 2; ++side) {
    int t = g.et[2 * m + side];
    Tri T;
    load_tri(g.verts, g.tris, g.nrm, g.area, g.diam, g.cen, t, &T);
    const double* v = &g.verts[3 * g.eopp[2 * m + side]];
    double cf = (side == 0 ? 1.0 : -1.0) * g.elen[m] / (2.0 * g.area[t]) * g.area[t];
    for (int q = 0; q < 7; ++q) {
      double r[3];
      rule_point(T, c_r7, q, r);
      double fp = 0;
      for (int a = 0; a < 3; ++a) fp += (r[a] - v[a]) * pol[a];
      double s, co;
      sincos(k0 * d_dot(kh, r), &s, &co);
      double w = c_r7[4 * q + 3] * cf * fp * inv_eta0;
      acc.x += w * co;
      acc.y -= w * s;
    }
  }
  b[m] = mk((decltype(b[m].x))acc.x, (decltype(b[m].x))acc.y);
}

struct TunePlan {  // a candidate plan held in temporary device memory
  GemvPlan p;
  std::vector<void*> mem;
  ~TunePlan() { for (void* q : mem) cudaFree(q); }
  template <typename T> int put(T** d, const std::vector<T>& h) {
    if (cudaMalloc((void**)d, h.size() * sizeof(T) + 16) != cudaSuccess) {
      set_error("autotune: allocation failed");
      return BEM_ENOMEM;
    }
    mem.push_back(*d);
    if (!h.empty() && cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) {
      set_error("autotune: copy failed");
      return BEM_ECUDA;
    }
    return BEM_OK;
  }
};

// GEMV autotuner: for the block layout (n, off, ld) of the FP32 matrix A, time the candidate
// launches with CUDA events on the real data and keep the fastest. Candidates: the row-plan
// kernel with (CTAs per SM, loads in flight per lane) in {(6, 4), (4, 4), (4, 8)} x {1, 2, 4}
// column parts per row; the flat kernel with (6, 4) and (4, 8); the bulk-copy-staged kernel
// with 1 CTA per SM (4 stages of 40 KB) and 2 (3 of 24 KB), when every row fits a stage.
// Every candidate's product of a fixed x is checked against the first candidate's; a launch
// that disagrees beyond FP32 rounding, or whose bounded waits timed out, is rejected and counted
// in tune_rejected. out32 receives the winner, out64 (the FP64 products) the best register-path
// candidate, alt (if not null) the best register-path and the best staged FP32 plan. tune_ms
// receives the time of 5 launches of those two.
namespace {
struct GemvCand {
  int kind;   // 0 row plan, 1 flat, 2 staged, 3 stream, 5 Part_Schedule task list,
              // 6 the same tasks taken in turn by cps persistent CTAs per SM
  int cps;    // CTAs per SM
  int split;  // column parts per row (row plan); rows per task / 8 (task list)
  int unroll; // loads in flight per lane (row plan, flat, task list)
};
}  // namespace

// Build and upload the plan of candidate g (into context memory when c_owned, else into t).
static int make_gemv_plan(aim_ctx* c, TunePlan* t, const GemvCand& g, int nsm,
                          const std::vector<int32_t>& n, const std::vector<int64_t>& off,
                          const std::vector<int32_t>& ld, int* derr, GemvPlan* out) {
  std::vector<RowInfo> rows;
  std::vector<int2> segs;
  std::vector<int32_t> cseg, cst;
  std::vector<TmaStage> st;
  std::vector<TmaDesc> dsc;
  GemvPlan p;
  if (g.kind == 5 || g.kind == 6) {
    // the paper's schedule: each block cut into the modified Part_Schedule's P_i row panels
    // (P = 4 CTA slots per SM, Alg. 2), the panels into tasks of <= 8 * split rows, one CTA each
    std::vector<int32_t> xo(n.size());
    for (size_t i = 0, acc = 0; i < n.size(); acc += n[i], ++i) xo[i] = (int32_t)acc;
    std::vector<GemvTask> tasks;
    const int form = g.kind == 5 && g.cps == 8 ? 1 : g.kind == 5 && g.cps == 16 ? 2 : 0;
    build_gemv_tasks(n, off, xo, ld, nsm, (form == 2 ? 4 : 8) * g.split, &tasks);
    if (t) BEM_TRY(t->put(&p.tasks, tasks));
    else BEM_TRY(upload(c, &p.tasks, tasks.data(), tasks.size()));
    p.ntasks = (int)tasks.size();
    p.ncta = p.ntasks;
    p.split = g.split;
    p.unroll = g.unroll;
    p.task_form = form;
    p.cps = g.cps;
    if (g.kind == 6) {
      const std::vector<int> zero(2, 0);
      if (t) BEM_TRY(t->put(&p.ctr, zero));
      else BEM_TRY(upload(c, &p.ctr, zero.data(), zero.size()));
      p.ncta = nsm * g.cps;
    }
    p.nrows = 0;
    for (int v : n) p.nrows += v;
    *out = p;
    return BEM_OK;
  }
  build_gemv_plan(n, off, ld, nsm * g.cps, &rows, &segs, &cseg, &p.cmax_over_ideal);
  const int stage_bytes = g.cps == 1 ? 40 * 1024 : 24 * 1024;
  if (g.kind == 1 || g.kind == 2) {
    const int64_t lim = g.kind == 2 ? stage_bytes / (int)sizeof(float2) : ((int64_t)1 << 40);
    if (!build_tma_stages(rows, segs, cseg, lim, &st, &cst, &dsc)) return 1;  // not applicable
  }
  std::vector<int32_t> wrow;
  int64_t nquad = 0;
  if (g.kind == 3) {
    // the storage must be gapless: row m + 1 starts where row m (length ld) ends
    int64_t end = rows.empty() ? 0 : rows[0].aoff;
    if (end != 0) return 1;
    for (const RowInfo& r : rows) {
      if (r.aoff != end) return 1;
      end += (r.n + 3) & ~3;
    }
    nquad = end / 4;
    const int64_t W = (int64_t)nsm * g.cps * (kGemvThreads / 32);
    wrow.resize(W);
    size_t m = 0;
    for (int64_t w = 0; w < W; ++w) {
      const int64_t e0 = 4 * (nquad * w / W);  // first element of warp w's share
      while (m + 1 < rows.size() && rows[m + 1].aoff <= e0) ++m;
      wrow[w] = (int32_t)m;
    }
  }
  auto put = [&](auto** d, const auto& h) -> int {
    if (t) return t->put(d, h);
    return upload(c, d, h.data(), h.size());
  };
  BEM_TRY(put(&p.rows, rows));
  BEM_TRY(put(&p.segs, segs));
  BEM_TRY(put(&p.cta_seg, cseg));
  p.ncta = nsm * g.cps;
  p.cps = g.cps;
  p.nrows = (int)rows.size();
  p.split = g.split;
  p.unroll = g.unroll;
  if (g.kind == 3) {
    BEM_TRY(put(&p.wrow, wrow));
    p.stream = 1;
    p.nquad = nquad;
  }
  if (g.kind == 1 || g.kind == 2) {
    BEM_TRY(put(&p.stages, st));
    BEM_TRY(put(&p.cta_stage, cst));
    BEM_TRY(put(&p.descs, dsc));
    p.flat = g.kind == 1;
    p.tma = g.kind == 2;
    p.nstage = g.cps == 1 ? 4 : 3;
    p.stage_bytes = stage_bytes;
    p.err = derr;
  }
  *out = p;
  return BEM_OK;
}

static int autotune_gemv(aim_ctx* c, const std::vector<int32_t>& n, const std::vector<int64_t>& off,
                         const std::vector<int32_t>& ld, const float2* A, GemvPlan* out32,
                         GemvPlan* out64, float* tune_ms, GemvPlan* alt) {
  tune_ms[0] = tune_ms[1] = 1e30f;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int64_t tot = 0;
  for (int v : n) tot += v;
  std::vector<GemvCand> cands;
  for (int cu : {0, 1, 2}) {
    const int cps = cu == 0 ? 6 : 4, u = cu == 2 ? 8 : 4;
    for (int split : {1, 2, 4}) cands.push_back({0, cps, split, u});
  }
  cands.push_back({1, 6, 1, 4});
  cands.push_back({1, 4, 1, 8});
  cands.push_back({3, 6, 1, 4});
  cands.push_back({3, 4, 1, 8});
  for (int split : {1, 2}) cands.push_back({5, 4, split, 4});
  cands.push_back({5, 8, 1, 4});
  cands.push_back({5, 16, 1, 4});
  cands.push_back({5, 16, 2, 4});
  cands.push_back({5, 4, 1, 8});
  cands.push_back({6, 5, 2, 4});
  cands.push_back({6, 4, 2, 8});
  cands.push_back({2, 1, 1, 4});
  cands.push_back({2, 2, 1, 2});
  int* derr = nullptr;
  BEM_TRY(dalloc_t(c, &derr, 1));
  BEM_CUDA(cudaMemset(derr, 0, sizeof(int)));
  TunePlan io;  // x, y of the trial launches
  std::vector<float2> xh(tot), yh(tot), yref;
  for (int64_t i = 0; i < tot; ++i) xh[i] = make_float2((float)std::sin(0.37 * i), (float)std::cos(0.11 * i));
  float2 *x = nullptr, *y = nullptr;
  BEM_TRY(io.put(&x, xh));
  BEM_TRY(io.put(&y, yh));
  // the product of candidate 0 is the reference of the others (same sums in another order)
  auto agrees = [&]() -> bool {
    if (cudaMemcpy(yh.data(), y, tot * sizeof(float2), cudaMemcpyDeviceToHost) != cudaSuccess) return false;
    if (yref.empty()) {
      yref = yh;
      return true;
    }
    double num = 0, den = 0;
    for (int64_t i = 0; i < tot; ++i) {
      num = std::max(num, (double)std::hypot(yh[i].x - yref[i].x, yh[i].y - yref[i].y));
      den = std::max(den, (double)std::hypot(yref[i].x, yref[i].y));
    }
    return num <= 1e-4 * den;
  };
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto timeit = [&](const GemvPlan& p) -> float {
    for (int w = 0; w < 2; ++w) run_gemv_plan<float>(p, A, x, y, 1, tot, nullptr, 0);
    cudaEventRecord(e0, 0);
    for (int r = 0; r < 5; ++r) run_gemv_plan<float>(p, A, x, y, 1, tot, nullptr, 0);
    cudaEventRecord(e1, 0);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms;
  };
  int best = -1, best_reg = -1, best_staged = -1;
  float tbest = 1e30f;
  int rc = BEM_OK;
  for (int i = 0; i < (int)cands.size(); ++i) {
    TunePlan t;
    GemvPlan p;
    const int r = make_gemv_plan(c, &t, cands[i], nsm, n, off, ld, derr, &p);
    float* row = nullptr;
    if (alt) {  // the context's own products: record the table
      c->tune_table.insert(c->tune_table.end(), {(float)cands[i].kind, (float)cands[i].cps,
                                                 (float)cands[i].split, (float)cands[i].unroll, -1.f});
      row = &c->tune_table.back();
    }
    if (r == 1) continue;  // rows do not fit a stage
    if (r != BEM_OK) { rc = r; break; }
    const float ms = timeit(p);
    int herr = 0;
    cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost);
    cudaMemset(derr, 0, sizeof(int));
    if (cudaGetLastError() != cudaSuccess || herr != 0 || !agrees()) {
      ++c->tune_rejected;
      continue;
    }
    if (row) *row = ms * 1e6f / 5.f;
    if (ms < tbest) { tbest = ms; best = i; }
    if (cands[i].kind == 2) {
      if (ms < tune_ms[1]) { tune_ms[1] = ms; best_staged = i; }
    } else if (ms < tune_ms[0]) {
      tune_ms[0] = ms;
      best_reg = i;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != BEM_OK) return rc;
  BEM_CUDA(cudaGetLastError());
  if (best_reg < 0) {
    set_error("GEMV autotuner: no register-path candidate gave the reference product");
    return BEM_ECUDA;
  }
  BEM_TRY(make_gemv_plan(c, nullptr, cands[best_reg], nsm, n, off, ld, derr, out64));
  GemvPlan staged;  // ncta = 0: no staged candidate ran correctly
  if (best_staged >= 0) BEM_TRY(make_gemv_plan(c, nullptr, cands[best_staged], nsm, n, off, ld, derr, &staged));
  *out32 = best == best_staged ? staged : *out64;
  if (alt) {
    alt[0] = *out64;
    alt[1] = staged;
  }
  return BEM_OK;
}

// A caller-chosen FP32 launch for the context's internal products (kind 0 row plan, 1 flat,
// 2 staged, 3 stream), checked against the autotuner's reference product before use.
static int make_pair_plan(aim_ctx* c, const GemvPlan& base, int nsm, GemvPlan* out);

int set_gemv_shape(aim_ctx* c, int kind, int cps, int split, int unroll) {
  const bool ok_shape =
      (kind == 0 && (cps == 4 || cps == 6) && (split == 1 || split == 2 || split == 4) &&
       (unroll == 4 || (unroll == 8 && cps == 4))) ||
      ((kind == 1 || kind == 3) && ((cps == 6 && unroll == 4) || (cps == 4 && unroll == 8))) ||
      (kind == 2 && (cps == 1 || cps == 2)) ||
      (kind == 5 && (split == 1 || split == 2 || split == 4) &&
       ((cps == 4 && (unroll == 4 || unroll == 8)) || ((cps == 8 || cps == 16) && unroll == 4))) ||
      (kind == 6 && (split == 1 || split == 2 || split == 4) && (unroll == 4 || unroll == 8) &&
       cps >= 1 && cps <= 8);
  if (!ok_shape) {
    set_error("aim_gemv_plan: unsupported shape (kind %d, %d CTAs/SM, split %d, unroll %d)", kind,
              cps, split, unroll);
    return BEM_EINVAL;
  }
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  std::vector<int32_t> n(c->nobj);
  for (int i = 0; i < c->nobj; ++i) n[i] = c->e1[i] - c->e0[i];
  int* derr = nullptr;
  BEM_TRY(dalloc_t(c, &derr, 1));
  BEM_CUDA(cudaMemset(derr, 0, sizeof(int)));
  GemvPlan p;
  const GemvCand g{kind, cps, kind == 0 || kind >= 5 ? split : 1,
                   kind == 2 ? (cps == 1 ? 4 : 2) : unroll};
  const int r = make_gemv_plan(c, nullptr, g, nsm, n, c->zoff, c->zld, derr, &p);
  if (r == 1) {
    set_error("aim_gemv_plan: a row does not fit a shared-memory stage");
    return BEM_EINVAL;
  }
  BEM_TRY(r);
  // the product of a fixed x must match the first autotuner candidate's (row plan, 6 CTAs/SM)
  int64_t tot = 0;
  for (int v : n) tot += v;
  std::vector<float2> xh(tot), y0(tot), y1(tot);
  for (int64_t i = 0; i < tot; ++i) xh[i] = make_float2((float)std::sin(0.37 * i), (float)std::cos(0.11 * i));
  TunePlan io;
  float2 *x = nullptr, *y = nullptr;
  BEM_TRY(io.put(&x, xh));
  BEM_TRY(io.put(&y, y0));
  BEM_TRY(run_gemv_plan<float>(c->gplan_alt[0], c->f32.Z, x, y, 1, tot, nullptr, 0));
  BEM_CUDA(cudaMemcpy(y0.data(), y, tot * sizeof(float2), cudaMemcpyDeviceToHost));
  BEM_TRY(run_gemv_plan<float>(p, c->f32.Z, x, y, 1, tot, nullptr, 0));
  BEM_CUDA(cudaMemcpy(y1.data(), y, tot * sizeof(float2), cudaMemcpyDeviceToHost));
  int herr = 0;
  BEM_CUDA(cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost));
  double num = 0, den = 0;
  for (int64_t i = 0; i < tot; ++i) {
    num = std::max(num, (double)std::hypot(y1[i].x - y0[i].x, y1[i].y - y0[i].y));
    den = std::max(den, (double)std::hypot(y0[i].x, y0[i].y));
  }
  if (herr != 0 || !(num <= 1e-4 * den)) {
    set_error("aim_gemv_plan: the launch's product differs from the reference (%g)", num / den);
    return BEM_ECUDA;
  }
  c->gplan = p;
  if (kind == 5) BEM_TRY(make_pair_plan(c, p, nsm, &c->gpair));  // the paired launch follows the shape
  return BEM_OK;
}

// The paired task list of a task-list launch shape: its tasks over C (sel 0), then over Z (sel 1)
static int make_pair_plan(aim_ctx* c, const GemvPlan& base, int nsm, GemvPlan* out) {
  std::vector<int32_t> n(c->nobj), xo(c->nobj);
  for (int i = 0, acc = 0; i < c->nobj; acc += n[i], ++i) {
    n[i] = c->e1[i] - c->e0[i];
    xo[i] = acc;
  }
  std::vector<GemvTask> t1;
  build_gemv_tasks(n, c->zoff, xo, c->zld, nsm, (base.task_form == 2 ? 4 : 8) * base.split, &t1);
  std::vector<GemvTask> t2 = t1;
  for (GemvTask& t : t2) t.sel = 1;
  t1.insert(t1.end(), t2.begin(), t2.end());
  GemvPlan p = base;
  BEM_TRY(upload(c, &p.tasks, t1.data(), t1.size()));
  p.ntasks = p.ncta = (int)t1.size();
  *out = p;
  return BEM_OK;
}

// Schedule autotuner of the system matvec: e = Z h runs beside j's GEMV or beside the AIM
// chain of j with a launch of few CTAs, after j's GEMV on the main stream with the whole GPU,
// or with j's GEMV in one paired task list. Time the captured FP32 graph for each (launch of
// e: the flat form or the dynamic task list, and its CTAs per SM; schedule 0-3) with CUDA
// events and keep the fastest, a concurrent schedule having to win by 2%; the FP64 matvec uses
// the same choice. tune_table gains rows (4, CTAs per SM or 0 for the main-stream launches,
// schedule, kind of the e launch, ns per matvec). It also times the two shapes of the
// multi-right-hand-side GEMV of the batched matvec (rows 7, 16, rows per warp, 4, ns).
int tune_matvec_schedule(aim_ctx* c) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  std::vector<int32_t> n(c->nobj);
  for (int i = 0; i < c->nobj; ++i) n[i] = c->e1[i] - c->e0[i];
  int* derr = nullptr;
  BEM_TRY(dalloc_t(c, &derr, 1));
  BEM_CUDA(cudaMemset(derr, 0, sizeof(int)));
  const int64_t N = (int64_t)c->ne + c->nt;
  std::vector<float2> xh(N);
  for (int64_t i = 0; i < N; ++i) xh[i] = make_float2((float)std::sin(0.7 * i), (float)std::cos(0.3 * i));
  BEM_CUDA(cudaMemcpy(c->f32.xin, xh.data(), N * sizeof(float2), cudaMemcpyHostToDevice));
  cudaStream_t s = nullptr;
  BEM_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  GemvCand best_g{1, 2, 1, 8};
  int best_after = 0;
  int rc = BEM_OK;
  // the paired task list (C tasks, then Z tasks) in j's launch shape when that is a task list,
  // else in the 8-row, 8-warp shape
  c->gpair = GemvPlan();
  {
    GemvPlan p;
    if (c->gplan.ntasks > 0 && !c->gplan.ctr) p = c->gplan;
    else BEM_TRY(make_gemv_plan(c, nullptr, GemvCand{5, 8, 1, 4}, nsm, n, c->zoff, c->zld, derr, &p));
    BEM_TRY(make_pair_plan(c, p, nsm, &c->gpair));
  }
  // the multi-right-hand-side launch of the batched matvec: 4 warps of 4 or of 2 rows per task,
  // the faster on 4 right-hand sides of Z (CUDA events, 5 launches each)
  {
    GemvPlan cand[2];
    BEM_TRY(make_gemv_plan(c, nullptr, GemvCand{5, 16, 4, 4}, nsm, n, c->zoff, c->zld, derr, &cand[0]));
    BEM_TRY(make_gemv_plan(c, nullptr, GemvCand{5, 16, 2, 4}, nsm, n, c->zoff, c->zld, derr, &cand[1]));
    const int64_t ne = c->ne;
    float2 *xx = nullptr, *yy = nullptr;
    BEM_CUDA(cudaMalloc(&xx, 4 * ne * sizeof(float2)));
    if (cudaMalloc(&yy, 4 * ne * sizeof(float2)) != cudaSuccess) {
      cudaFree(xx);
      set_error("schedule tuner: out of device memory");
      return BEM_ENOMEM;
    }
    cudaMemset(xx, 0, 4 * ne * sizeof(float2));
    cudaEvent_t a0, a1;
    cudaEventCreate(&a0);
    cudaEventCreate(&a1);
    float tm[2] = {0, 0};
    for (int i = 0; i < 2; ++i) {
      run_gemv_mr<float>(cand[i], c->f32.Z, xx, yy, 4, ne, nullptr, 0);
      cudaEventRecord(a0, 0);
      for (int r = 0; r < 5; ++r) run_gemv_mr<float>(cand[i], c->f32.Z, xx, yy, 4, ne, nullptr, 0);
      cudaEventRecord(a1, 0);
      cudaEventSynchronize(a1);
      cudaEventElapsedTime(&tm[i], a0, a1);
      c->tune_table.insert(c->tune_table.end(), {7.f, 16.f, (float)cand[i].split, 4.f, tm[i] * 1e6f / 5.f});
    }
    cudaEventDestroy(a0);
    cudaEventDestroy(a1);
    cudaFree(xx);
    cudaFree(yy);
    BEM_CUDA(cudaGetLastError());
    c->gmr = tm[1] < tm[0] ? cand[1] : cand[0];
  }
  // the last two entries stand for the serial schedules (e = Z h after j's GEMV with its
  // launch shape; both in one paired launch)
  const GemvCand zc[] = {{1, 1, 1, 8}, {1, 2, 1, 8}, {1, 3, 1, 8}, {6, 2, 2, 4}, {6, 3, 2, 4}, {6, 4, 2, 4},
                         {1, 2, 1, 8}, {1, 2, 1, 8}};
  const int nzc = (int)(sizeof(zc) / sizeof(zc[0]));
  for (int gi = 0; gi < nzc; ++gi) {
    const GemvCand& g = zc[gi];
    GemvPlan p;
    if ((rc = make_gemv_plan(c, nullptr, g, nsm, n, c->zoff, c->zld, derr, &p)) != BEM_OK) break;
    for (int after : {0, 1, 2, 3}) {
      const int want = gi == nzc - 1 ? 3 : gi == nzc - 2 ? 2 : -1;
      if (want >= 0 ? after != want : after >= 2) continue;
      c->gbg32 = c->gbg64 = p;
      c->z_after = after;
      for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
      c->graphs.clear();
      for (int w = 0; w < 3 && rc == BEM_OK; ++w) rc = matvec_graph<float>(c, AIM_OP_SYSTEM, c->f32.xin, c->f32.yout, s);
      if (rc != BEM_OK) break;
      cudaEventRecord(e0, s);
      for (int r = 0; r < 40 && rc == BEM_OK; ++r) rc = matvec_graph<float>(c, AIM_OP_SYSTEM, c->f32.xin, c->f32.yout, s);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      c->tune_table.insert(c->tune_table.end(), {4.f, after >= 2 ? 0.f : (float)g.cps, (float)after,
                                                 after >= 2 ? (float)(c->gplan.ctr ? 6 : c->gplan.ntasks ? 5 : 1) : (float)g.kind,
                                                 ms * 1e6f / 40.f});
      // a schedule with e beside other work must win by 2%: its time depends on how the
      // concurrent kernels interleave and varies more from run to run than the serial ones
      const float eff = after < 2 ? ms * 1.02f : ms;
      if (eff < best) { best = eff; best_g = g; best_after = after; }
    }
    if (rc != BEM_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
  c->graphs.clear();
  if (rc != BEM_OK) return rc;
  BEM_TRY(make_gemv_plan(c, nullptr, best_g, nsm, n, c->zoff, c->zld, derr, &c->gbg32));
  c->gbg64 = c->gbg32;
  c->z_after = c->z_tuned = best_after;
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

// ---------------------------------------------------------------------------------------
// orchestration
// ---------------------------------------------------------------------------------------
struct DevGeoStore {
  double *verts, *nrm, *area, *diam, *cen, *elen;
  int32_t *tris, *et, *eopp, *anc;
};

static DGeo make_dgeo(aim_ctx* c, const DevGeoStore& s) {
  DGeo g;
  g.verts = s.verts; g.tris = s.tris; g.nrm = s.nrm; g.area = s.area; g.diam = s.diam;
  g.cen = s.cen; g.et = s.et; g.eopp = s.eopp; g.elen = s.elen; g.anc = s.anc;
  for (int a = 0; a < 3; ++a) { g.go[a] = c->go[a]; g.gh[a] = c->gh[a]; }
  return g;
}

static int geo_upload(aim_ctx* c, DevGeoStore* s) {
  BEM_TRY(upload(c, &s->verts, c->verts.data(), c->verts.size()));
  BEM_TRY(upload(c, &s->nrm, c->normal.data(), c->normal.size()));
  BEM_TRY(upload(c, &s->area, c->area.data(), c->area.size()));
  BEM_TRY(upload(c, &s->diam, c->diam.data(), c->diam.size()));
  BEM_TRY(upload(c, &s->cen, c->centroid.data(), c->centroid.size()));
  BEM_TRY(upload(c, &s->elen, c->elen.data(), c->elen.size()));
  BEM_TRY(upload(c, &s->tris, c->tris.data(), c->tris.size()));
  BEM_TRY(upload(c, &s->et, c->et.data(), c->et.size()));
  BEM_TRY(upload(c, &s->eopp, c->eopp.data(), c->eopp.size()));
  BEM_TRY(upload(c, &s->anc, c->anc.data(), c->anc.size()));
  return BEM_OK;
}


static inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

struct SolverScratch {
  cusolverDnHandle_t h = nullptr;
  cusolverDnParams_t p = nullptr;
  ~SolverScratch() {
    if (p) cusolverDnDestroyParams(p);
    if (h) cusolverDnDestroy(h);
  }
};

// X <- L^{-1} B for column-major n x n matrices (in place in B), LU with partial pivoting.
static int lu_solve(SolverScratch& ss, double2* L, double2* B, int n, int64_t* ipiv, int* dinfo,
                    void** dwork, size_t* dwsize, std::vector<char>* hwork) {
  size_t dws = 0, hws = 0;
  if (cusolverDnXgetrf_bufferSize(ss.h, ss.p, n, n, CUDA_C_64F, L, n, CUDA_C_64F, &dws, &hws) !=
      CUSOLVER_STATUS_SUCCESS) {
    set_error("cusolverDnXgetrf_bufferSize failed");
    return BEM_ECUDA;
  }
  if (dws > *dwsize) {
    if (*dwork) cudaFree(*dwork);
    *dwork = nullptr;
    BEM_CUDA(cudaMalloc(dwork, dws));
    *dwsize = dws;
  }
  if (hws > hwork->size()) hwork->resize(hws);
  if (cusolverDnXgetrf(ss.h, ss.p, n, n, CUDA_C_64F, L, n, ipiv, CUDA_C_64F, *dwork, dws,
                       hwork->data(), hws, dinfo) != CUSOLVER_STATUS_SUCCESS) {
    set_error("cusolverDnXgetrf failed");
    return BEM_ECUDA;
  }
  int hinfo = 0;
  BEM_CUDA(cudaMemcpy(&hinfo, dinfo, sizeof(int), cudaMemcpyDeviceToHost));
  if (hinfo != 0) {
    set_error("singular internal matrix (getrf info %d)", hinfo);
    return BEM_ESOLVER;
  }
  if (cusolverDnXgetrs(ss.h, ss.p, CUBLAS_OP_N, n, n, CUDA_C_64F, L, n, ipiv, CUDA_C_64F, B, n,
                       dinfo) != CUSOLVER_STATUS_SUCCESS) {
    set_error("cusolverDnXgetrs failed");
    return BEM_ECUDA;
  }
  return BEM_OK;
}

// scratch of the pair-moment passes, sized for the object with the most triangles
struct MomentScratch {
  Moments* mom = nullptr;
  int* list = nullptr;
  int* count = nullptr;
  int64_t cap = 0;
  int* npts = nullptr;        // points per large-|k| pair
  int64_t* off = nullptr;     // their offsets in the point list
  int32_t* items = nullptr;   // the point list
  int64_t pcap = 0, icap = 0;
  ~MomentScratch() {
    if (mom) cudaFree(mom);
    if (list) cudaFree(list);
    if (count) cudaFree(count);
    if (npts) cudaFree(npts);
    if (off) cudaFree(off);
    if (items) cudaFree(items);
  }
  int reserve_pts(int64_t pairs, int64_t points) {
    if (pairs > pcap) {
      if (npts) cudaFree(npts);
      if (off) cudaFree(off);
      npts = nullptr;
      off = nullptr;
      BEM_CUDA(cudaMalloc(&npts, pairs * sizeof(int)));
      BEM_CUDA(cudaMalloc(&off, pairs * sizeof(int64_t)));
      pcap = pairs;
    }
    if (points > icap) {
      if (items) cudaFree(items);
      items = nullptr;
      BEM_CUDA(cudaMalloc(&items, points * sizeof(int32_t)));
      icap = points;
    }
    return BEM_OK;
  }
  int reserve(int64_t pairs) {
    if (pairs <= cap) return BEM_OK;
    if (mom) cudaFree(mom);
    if (list) cudaFree(list);
    mom = nullptr;
    list = nullptr;
    BEM_CUDA(cudaMalloc(&mom, pairs * sizeof(Moments)));
    BEM_CUDA(cudaMalloc(&list, pairs * sizeof(int)));
    if (!count) BEM_CUDA(cudaMalloc(&count, sizeof(int)));
    cap = pairs;
    return BEM_OK;
  }
};

// pair moments of every triangle pair (T, S) of object obj at wavenumber k into
// ms->mom[(T - t0) m + (S - t0)]; large-|k| near pairs through the per-point passes
static int object_moments(aim_ctx* c, const DGeo& g, int obj, std::complex<double> k, bool wantK,
                          MomentScratch* ms) {
  const int t0 = c->t0[obj], m = c->t1[obj] - c->t0[obj];
  const int64_t pairs = (int64_t)m * m;
  BEM_TRY(ms->reserve(pairs));
  BEM_CUDA(cudaMemset(ms->count, 0, sizeof(int)));
  k_obj_moments<<<nblk(pairs, 128), 128>>>(g, t0, m, k.real(), k.imag(), wantK, ms->mom, ms->list,
                                           ms->count);
  BEM_CUDA(cudaGetLastError());
  int nhk = 0;
  BEM_CUDA(cudaMemcpy(&nhk, ms->count, sizeof(int), cudaMemcpyDeviceToHost));
  if (nhk >= (1 << 22)) {
    set_error("aim_setup: object %d has %d large-|k| near pairs (at most %d)", obj, nhk, (1 << 22) - 1);
    return BEM_EINVAL;
  }
  if (nhk > 0) {
    // count the outer rule points of every large-|k| pair, lay them out, integrate per point
    BEM_TRY(ms->reserve_pts(nhk, 0));
    k_hk_count<<<nblk(nhk, 128), 128>>>(g, t0, m, k.real(), k.imag(), ms->list, nhk, ms->npts);
    BEM_CUDA(cudaGetLastError());
    std::vector<int> cnt(nhk);
    std::vector<int64_t> off(nhk);
    BEM_CUDA(cudaMemcpy(cnt.data(), ms->npts, nhk * sizeof(int), cudaMemcpyDeviceToHost));
    int64_t tot = 0;
    for (int p = 0; p < nhk; ++p) { off[p] = tot; tot += cnt[p]; }
    BEM_TRY(ms->reserve_pts(nhk, tot));
    BEM_CUDA(cudaMemcpy(ms->off, off.data(), nhk * sizeof(int64_t), cudaMemcpyHostToDevice));
    k_hk_items<<<nblk(nhk, 128), 128>>>(g, t0, m, k.real(), k.imag(), ms->list, nhk, ms->off,
                                         ms->items);
    BEM_CUDA(cudaGetLastError());
    k_hk_points<<<nblk(tot, 128), 128>>>(g, t0, m, k.real(), k.imag(), wantK, ms->list, ms->items,
                                          tot, ms->mom);
    BEM_CUDA(cudaGetLastError());
  }
  return BEM_OK;
}

// L_k (into L) and K_k + I_x/2 (into B), column-major n x n, for object obj and wavenumber k
static int object_LK(aim_ctx* c, const DGeo& g, int obj, std::complex<double> k, MomentScratch* ms,
                     double2* L, double2* B) {
  const int n = c->e1[obj] - c->e0[obj];
  const int t0 = c->t0[obj], m = c->t1[obj] - c->t0[obj];
  BEM_TRY(object_moments(c, g, obj, k, true, ms));
  k_obj_assemble<<<nblk((int64_t)n * n, 128), 128>>>(g, c->e0[obj], n, t0, m, k.real(), k.imag(),
                                                     ms->mom, c->d_ixcol, c->f64.ix, L, B);
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

static int setup_internal(aim_ctx* c, const DGeo& g, const int32_t* d_ixcol, const double* d_ixval) {
  const int nobj = c->nobj;
  c->zoff.assign(nobj, 0);
  c->zld.assign(nobj, 0);
  int64_t off = 0;
  int nmax = 0;
  for (int i = 0; i < nobj; ++i) {
    int n = c->e1[i] - c->e0[i];
    c->zld[i] = (int32_t)round_up(n, 4);
    c->zoff[i] = off;
    off += (int64_t)n * c->zld[i];
    nmax = std::max(nmax, n);
  }
  c->zelems = off;
  BEM_TRY(dalloc_t(c, &c->f64.Z, off));
  BEM_TRY(dalloc_t(c, &c->f64.Y, off));
  BEM_TRY(dalloc_t(c, &c->f64.C, off));
  BEM_TRY(dalloc_t(c, &c->f32.Z, off));
  BEM_TRY(dalloc_t(c, &c->f32.C, off));
  BEM_CUDA(cudaMemset(c->f64.C, 0, off * sizeof(double2)));
  double2 *L = nullptr, *B = nullptr;
  int64_t* ipiv = nullptr;
  int* dinfo = nullptr;
  size_t nn = (size_t)nmax * nmax;
  BEM_CUDA(cudaMalloc(&L, nn * sizeof(double2)));
  BEM_CUDA(cudaMalloc(&B, nn * sizeof(double2)));
  BEM_CUDA(cudaMalloc(&ipiv, nmax * sizeof(int64_t)));
  BEM_CUDA(cudaMalloc(&dinfo, sizeof(int)));
  SolverScratch ss;
  MomentScratch ms;
  void* dwork = nullptr;
  size_t dwsize = 0;
  std::vector<char> hwork;
  int rc = BEM_OK;
  if (cusolverDnCreate(&ss.h) != CUSOLVER_STATUS_SUCCESS || cusolverDnCreateParams(&ss.p) != CUSOLVER_STATUS_SUCCESS) {
    set_error("cusolverDnCreate failed");
    rc = BEM_ECUDA;
  }
  const double w = 2.0 * kPi * c->freq;
  {
    // pattern and ordering of the sparse internal operator (when every object qualifies)
    const double tz = wall_ms();
    if (rc == BEM_OK) rc = zsp_prepare(c, g.verts, g.tris, g.cen);
    c->setup_ms[10] += wall_ms() - tz;
  }
  for (int i = 0; i < nobj && rc == BEM_OK; ++i) {
    const int n = c->e1[i] - c->e0[i];
    const bem_material& mt = c->mat[i];
    // conductor: eps_rc = eps_r - j sigma/(w eps0); k_i = k0 sqrt(eps_rc mu_r), Im k_i <= 0
    std::complex<double> epsc(mt.eps_r, -mt.sigma / (w * kEps0));
    std::complex<double> ki = c->k0 * std::sqrt(epsc * mt.mu_r);
    if (ki.imag() > 0) ki = -ki;
    for (int pass = 0; pass < 2 && rc == BEM_OK; ++pass) {
      // pass 0: Z = -(1/(j k0 eps_rc)) L_{k_i}^{-1}(K_{k_i} + I_x/2)
      // pass 1: Y = (1/(j k0 mu_rl)) L_{k0}^{-1}(K_{k0} + I_x/2), background vacuum
      std::complex<double> k = pass == 0 ? ki : std::complex<double>(c->k0, 0.0);
      double t0 = wall_ms();
      rc = object_LK(c, g, i, k, &ms, L, B);
      if (rc == BEM_OK && pass == 0 && c->zsp) rc = zsp_gather(c, i, L, B);  // before the LU
      if (rc != BEM_OK) break;
      cudaDeviceSynchronize();
      double t1 = wall_ms();
      c->setup_ms[2 + pass] += t1 - t0;
      rc = lu_solve(ss, L, B, n, ipiv, dinfo, &dwork, &dwsize, &hwork);
      if (rc != BEM_OK) break;
      cudaDeviceSynchronize();
      c->setup_ms[4] += wall_ms() - t1;
      std::complex<double> jk0(0.0, c->k0);
      std::complex<double> alpha = pass == 0 ? -1.0 / (jk0 * epsc) : 1.0 / jk0;
      double2 al = make_double2(alpha.real(), alpha.imag());
      k_store_block<<<nblk((int64_t)n * c->zld[i], 256), 256>>>(
          B, n, c->zld[i], al, (pass == 0 ? c->f64.Z : c->f64.Y) + c->zoff[i],
          pass == 0 ? c->f32.Z + c->zoff[i] : nullptr);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) { set_error("k_store_block: %s", cudaGetErrorString(e)); rc = BEM_ECUDA; }
    }
  }
  // C_i = Y_i Z_i (row-major blocks of leading dimension ld: in cuBLAS's column-major view
  // they are the transposes, so C^T = Z^T Y^T is one plain product), in FP64, then rounded
  const double tyz = wall_ms();
  if (rc == BEM_OK) {
    cublasHandle_t bh = nullptr;
    if (cublasCreate(&bh) != CUBLAS_STATUS_SUCCESS) {
      set_error("cublasCreate failed");
      rc = BEM_ECUDA;
    }
    const cuDoubleComplex one = make_cuDoubleComplex(1, 0), zero = make_cuDoubleComplex(0, 0);
    for (int i = 0; i < nobj && rc == BEM_OK; ++i) {
      const int n = c->e1[i] - c->e0[i], ld = c->zld[i];
      const int64_t o = c->zoff[i];
      if (cublasZgemm(bh, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, &one,
                      (const cuDoubleComplex*)(c->f64.Z + o), ld, (const cuDoubleComplex*)(c->f64.Y + o),
                      ld, &zero, (cuDoubleComplex*)(c->f64.C + o), ld) != CUBLAS_STATUS_SUCCESS) {
        set_error("cublasZgemm (Y Z) failed");
        rc = BEM_ECUDA;
      }
    }
    if (bh) cublasDestroy(bh);
    if (rc == BEM_OK) {
      k_round32<<<1216, 256>>>(c->f64.C, c->f32.C, c->zelems);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) { set_error("k_round32: %s", cudaGetErrorString(e)); rc = BEM_ECUDA; }
    }
  }
  cudaDeviceSynchronize();
  c->setup_ms[5] = wall_ms() - tyz;
  if (rc == BEM_OK && c->zsp) {
    const double tz = wall_ms();
    rc = zsp_factor(c);
    c->setup_ms[10] += wall_ms() - tz;
  }
  cudaFree(L);
  cudaFree(B);
  cudaFree(ipiv);
  cudaFree(dinfo);
  if (dwork) cudaFree(dwork);
  return rc;
}

static int setup_near(aim_ctx* c, const DGeo& g) {
  const int R = c->r_near;
  const int span = 2 * R + 5;
  std::vector<double2> gt((size_t)span * span * span);
  for (int dz = -R - 2; dz <= R + 2; ++dz)
    for (int dy = -R - 2; dy <= R + 2; ++dy)
      for (int dx = -R - 2; dx <= R + 2; ++dx) {
        double x = dx * c->gh[0], y = dy * c->gh[1], z = dz * c->gh[2];
        double Rr = std::sqrt(x * x + y * y + z * z);
        double2 v = make_double2(0, 0);
        if (Rr > 0) {
          double s = std::sin(c->k0 * Rr), co = std::cos(c->k0 * Rr);
          v = make_double2(co / (4 * kPi * Rr), -s / (4 * kPi * Rr));
        }
        gt[((dz + R + 2) * span + (dy + R + 2)) * span + (dx + R + 2)] = v;
      }
  double2* d_gt = nullptr;
  BEM_TRY(upload(c, &d_gt, gt.data(), gt.size()));
  const size_t smem = gt.size() * sizeof(double2);
  // L^A_NR
  {
    int64_t nnz = c->rowA.back();
    std::vector<int32_t> rows(nnz);
    for (int m = 0; m < c->ne; ++m)
      for (int64_t i = c->rowA[m]; i < c->rowA[m + 1]; ++i) rows[i] = m;
    int32_t* d_rows = nullptr;
    BEM_TRY(upload(c, &d_rows, rows.data(), rows.size()));
    BEM_TRY(upload(c, &c->d_rowA, c->rowA.data(), c->rowA.size()));
    BEM_TRY(upload(c, &c->d_colA, c->colA.data(), c->colA.size()));
    BEM_TRY(upload(c, &c->d_lstA, c->lstA.data(), c->lstA.size()));
    if (c->clA.empty()) c->clA.push_back(0);  // no near pairs: a valid (unread) list
    BEM_TRY(upload(c, &c->d_clA, c->clA.data(), c->clA.size()));
    BEM_TRY(dalloc_t(c, &c->f64.LA, nnz));
    BEM_TRY(dalloc_t(c, &c->f32.LA, nnz));
    if (nnz)
      k_near_LA<<<nblk(nnz, 128), 128, smem>>>(g, nnz, d_rows, c->d_colA, c->f64.WA, d_gt, R, c->k0,
                                               c->f64.LA, c->f32.LA);
    BEM_CUDA(cudaGetLastError());
  }
  // L^Phi_NR
  {
    int64_t nnz = c->rowP.back();
    std::vector<int32_t> rows(nnz);
    for (int t = 0; t < c->nt; ++t)
      for (int64_t i = c->rowP[t]; i < c->rowP[t + 1]; ++i) rows[i] = t;
    int32_t* d_rows = nullptr;
    BEM_TRY(upload(c, &d_rows, rows.data(), rows.size()));
    BEM_TRY(upload(c, &c->d_rowP, c->rowP.data(), c->rowP.size()));
    BEM_TRY(upload(c, &c->d_colP, c->colP.data(), c->colP.size()));
    BEM_TRY(upload(c, &c->d_lstP, c->lstP.data(), c->lstP.size()));
    if (c->clP.empty()) c->clP.push_back(0);
    BEM_TRY(upload(c, &c->d_clP, c->clP.data(), c->clP.size()));
    BEM_TRY(dalloc_t(c, &c->f64.LP, nnz));
    BEM_TRY(dalloc_t(c, &c->f32.LP, nnz));
    if (nnz)
      k_near_LP<<<nblk(nnz, 128), 128, smem>>>(g, c->ne, nnz, d_rows, c->d_colP, c->f64.WP, d_gt, R,
                                               c->k0, c->f64.LP, c->f32.LP);
    BEM_CUDA(cudaGetLastError());
  }
  BEM_CUDA(cudaDeviceSynchronize());
  return BEM_OK;
}

int setup_device(aim_ctx* c) {
  {
    // the background-medium integrals (near region, preconditioner blocks, Y_eq) use the
    // small-|k| near rule, valid while k0 times the element size stays at or below kHighK
    double dmx = 0.0;
    for (double v : c->diam) dmx = std::max(dmx, v);
    if (c->k0 * dmx > kHighK) {
      set_error("aim_setup: k0 times the largest element (%.3g) exceeds %.2g; refine the mesh",
                c->k0 * dmx, kHighK);
      return BEM_EINVAL;
    }
  }
  double tst = wall_ms();
  BEM_TRY(upload_rules());
  DevGeoStore s;
  BEM_TRY(geo_upload(c, &s));
  DGeo g = make_dgeo(c, s);
  // projection stencils
  BEM_TRY(dalloc_t(c, &c->f64.WA, (size_t)c->ne * 81));
  BEM_TRY(dalloc_t(c, &c->f32.WA, (size_t)c->ne * 81));
  BEM_TRY(dalloc_t(c, &c->f64.WP, (size_t)c->nt * 27));
  BEM_TRY(dalloc_t(c, &c->f32.WP, (size_t)c->nt * 27));
  k_weights_e<<<nblk((int64_t)c->ne * 27, 256), 256>>>(g, c->ne, c->f64.WA, c->f32.WA);
  k_weights_t<<<nblk((int64_t)c->nt * 27, 256), 256>>>(g, c->ne, c->nt, c->f64.WP, c->f32.WP);
  BEM_CUDA(cudaGetLastError());
  // anchor node indices
  {
    std::vector<int32_t> nodeE(c->ne), nodeT(c->nt);
    for (int i = 0; i < c->ne + c->nt; ++i) {
      const int32_t* a = &c->anc[3 * (size_t)i];
      int32_t v = (int32_t)(((int64_t)a[2] * c->gn[1] + a[1]) * c->gn[0] + a[0]);
      if (i < c->ne) nodeE[i] = v; else nodeT[i - c->ne] = v;
    }
    BEM_TRY(upload(c, &c->d_nodeE, nodeE.data(), nodeE.size()));
    BEM_TRY(upload(c, &c->d_nodeT, nodeT.data(), nodeT.size()));
    // P^T in grid-node-major CSR form (counting sort by node; sources ascending per node)
    auto build = [&](const std::vector<int32_t>& node, int32_t** d_row, int32_t** d_col,
                     int32_t** d_k, int32_t** d_work, int32_t* nwork) -> int {
      const int ns = (int)node.size();
      const int nx = c->gn[0], ny = c->gn[1];
      std::vector<int32_t> row(c->ng + 1, 0), col(27 * (size_t)ns), kk(27 * (size_t)ns);
      auto nd = [&](int m, int k) {
        return node[m] + ((k / 9 - 1) * ny + ((k / 3) % 3 - 1)) * nx + (k % 3 - 1);
      };
      for (int m = 0; m < ns; ++m)
        for (int k = 0; k < 27; ++k) row[nd(m, k) + 1]++;
      for (int64_t i = 0; i < c->ng; ++i) row[i + 1] += row[i];
      std::vector<int32_t> fill(row.begin(), row.end() - 1);
      for (int m = 0; m < ns; ++m)
        for (int k = 0; k < 27; ++k) {
          int32_t p = fill[nd(m, k)]++;
          col[p] = m;
          kk[p] = k;
        }
      // node work list: nodes with entries (ascending), then the empty ones
      std::vector<int32_t> work;
      work.reserve(c->ng);
      for (int64_t i = 0; i < c->ng; ++i)
        if (row[i + 1] > row[i]) work.push_back((int32_t)i);
      *nwork = (int32_t)work.size();
      for (int64_t i = 0; i < c->ng; ++i)
        if (row[i + 1] == row[i]) work.push_back((int32_t)i);
      BEM_TRY(upload(c, d_row, row.data(), row.size()));
      BEM_TRY(upload(c, d_col, col.data(), col.size()));
      BEM_TRY(upload(c, d_k, kk.data(), kk.size()));
      BEM_TRY(upload(c, d_work, work.data(), work.size()));
      return BEM_OK;
    };
    int32_t *d_kE = nullptr, *d_kT = nullptr;
    BEM_TRY(build(nodeE, &c->d_prowE, &c->d_pcolE, &d_kE, &c->d_pnodeE, &c->nwE));
    BEM_TRY(build(nodeT, &c->d_prowT, &c->d_pcolT, &d_kT, &c->d_pnodeT, &c->nwT));
    const int64_t nE = 27 * (int64_t)c->ne, nT = 27 * (int64_t)c->nt;
    BEM_TRY(dalloc_t(c, &c->f64.WAT, 3 * nE));
    BEM_TRY(dalloc_t(c, &c->f32.WAT, 3 * nE));
    BEM_TRY(dalloc_t(c, &c->f64.WPT, nT));
    BEM_TRY(dalloc_t(c, &c->f32.WPT, nT));
    k_weights_csr<<<nblk(nE, 256), 256>>>(c->d_pcolE, d_kE, c->f64.WA, nE, 3, c->f64.WAT, c->f32.WAT);
    k_weights_csr<<<nblk(nT, 256), 256>>>(c->d_pcolT, d_kT, c->f64.WP, nT, 1, c->f64.WPT, c->f32.WPT);
    BEM_CUDA(cudaGetLastError());
  }
  // sparse tables
  std::vector<int32_t> ixcol;
  std::vector<double> ixval, fdE, fdT;
  build_ix_fd(c, &ixcol, &ixval, &fdE, &fdT);
  BEM_TRY(upload(c, &c->d_ixcol, ixcol.data(), ixcol.size()));
  BEM_TRY(upload(c, &c->f64.ix, ixval.data(), ixval.size()));
  BEM_TRY(upload(c, &c->f64.fdE, fdE.data(), fdE.size()));
  BEM_TRY(upload(c, &c->f64.fdT, fdT.data(), fdT.size()));
  {
    std::vector<float> a(ixval.begin(), ixval.end()), b(fdE.begin(), fdE.end()), d(fdT.begin(), fdT.end());
    BEM_TRY(upload(c, &c->f32.ix, a.data(), a.size()));
    BEM_TRY(upload(c, &c->f32.fdE, b.data(), b.size()));
    BEM_TRY(upload(c, &c->f32.fdT, d.data(), d.size()));
  }
  BEM_TRY(upload(c, &c->d_et, c->et.data(), c->et.size()));
  BEM_TRY(upload(c, &c->d_tedge, c->t_edges.data(), c->t_edges.size()));
  BEM_CUDA(cudaDeviceSynchronize());
  c->setup_ms[1] = wall_ms() - tst;
  // internal problem
  BEM_TRY(setup_internal(c, g, c->d_ixcol, c->f64.ix));
  // near region
  tst = wall_ms();
  BEM_TRY(setup_near(c, g));
  c->setup_ms[6] = wall_ms() - tst;
  // grid Green's function
  tst = wall_ms();
  BEM_TRY(make_twiddles<float>(c, c->f32));
  BEM_TRY(make_twiddles<double>(c, c->f64));
  BEM_TRY(fft_init_attrs());
  BEM_TRY(make_ghat(c));
  BEM_CUDA(cudaDeviceSynchronize());
  c->setup_ms[7] = wall_ms() - tst;
  tst = wall_ms();
  // GEMV work list
  {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    std::vector<int32_t> n(c->nobj);
    for (int i = 0; i < c->nobj; ++i) n[i] = c->e1[i] - c->e0[i];
    // persistent, byte-balanced plan with the autotuned launch shape
    BEM_TRY(tma_init_attrs());
    BEM_TRY(autotune_gemv(c, n, c->zoff, c->zld, c->f32.Z, &c->gplan, &c->gplan64, c->tune_ms,
                          c->gplan_alt));
    c->gplan_auto = c->gplan;
    // e = Z h runs beside the AIM chain of j in the system matvec: a launch of few CTAs (2 per
    // SM, 8 loads in flight per lane) that leaves most of every SM to the chain's kernels
    int* derr = nullptr;
    BEM_TRY(dalloc_t(c, &derr, 1));
    BEM_CUDA(cudaMemset(derr, 0, sizeof(int)));
    BEM_TRY(make_gemv_plan(c, nullptr, GemvCand{1, 2, 1, 8}, nsm, n, c->zoff, c->zld, derr, &c->gbg32));
    c->gbg64 = c->gbg32;  // a row plan holds no precision
  }
  // workspaces
  const size_t P = (size_t)c->gp[0] * c->gp[1] * c->gp[2];
  BEM_TRY(dalloc_t(c, &c->f32.sigma, 4 * (size_t)c->ng));
  BEM_TRY(dalloc_t(c, &c->f64.sigma, 4 * (size_t)c->ng));
  BEM_TRY(dalloc_t(c, &c->f32.ws, 4 * P));
  BEM_TRY(dalloc_t(c, &c->f64.ws, 4 * P));
  const size_t ntot = (size_t)c->ne + c->nt;
  BEM_TRY(dalloc_t(c, &c->f32.e, c->ne));
  BEM_TRY(dalloc_t(c, &c->f64.e, c->ne));
  BEM_TRY(dalloc_t(c, &c->f32.heq, c->ne));
  BEM_TRY(dalloc_t(c, &c->f64.heq, c->ne));
  BEM_TRY(dalloc_t(c, &c->f32.anear, c->ne));
  BEM_TRY(dalloc_t(c, &c->f64.anear, c->ne));
  BEM_TRY(dalloc_t(c, &c->f32.j, c->ne));
  BEM_TRY(dalloc_t(c, &c->f64.j, c->ne));
  BEM_TRY(dalloc_t(c, &c->f32.p, c->nt));
  BEM_TRY(dalloc_t(c, &c->f64.p, c->nt));
  BEM_TRY(dalloc_t(c, &c->f32.xin, ntot));
  BEM_TRY(dalloc_t(c, &c->f32.yout, ntot));
  BEM_TRY(dalloc_t(c, &c->f64.xin, ntot));
  BEM_TRY(dalloc_t(c, &c->f64.yout, ntot));
  BEM_TRY(init_streams(c));
  BEM_CUDA(cudaDeviceSynchronize());
  c->setup_ms[8] = wall_ms() - tst;
  c->geo_store = new DGeo(g);
  tst = wall_ms();
  BEM_TRY(zsp_check(c));
  c->setup_ms[10] += wall_ms() - tst;
  // the schedule of e = Z h is tuned for the dense form; the sparse one, when built, then
  // takes its place
  const bool zsp = c->zsp_on;
  c->zsp_on = false;
  tst = wall_ms();
  BEM_TRY(tune_matvec_schedule(c));
  c->setup_ms[9] = wall_ms() - tst;
  c->zsp_on = zsp;
  return BEM_OK;
}

// ---------------------------------------------------------------------------------------
// block-diagonal preconditioner: A_ii, the system of Eq. (AEFIEoutJ) restricted to object i's
// unknowns [h_i; q_i] with its exact dense L^A_ii and L^Phi_ii,
//   A_ii = [[j k0 L^A + (-j k0 L^A Y + I_x) Z, -(F D)^T L^Phi], [(F D)(I - Y Z), j k0 I]]
//        = [[j k0 L^A (I - C) + I_x Z,          -(F D)^T L^Phi], [(F D)(I - C),     j k0 I]]
// with C = Y Z of Eq. EFIEeqYZ (formed at set-up), inverted explicitly; the solve applies
// blockdiag(A_ii^{-1}) on the right. L^A and L^Phi come from the FP64 pair moments at k0.
// Build precision BEM_C32 (the default): each block is formed, LU-factorised and inverted in
// complex FP32, then its inverse X is checked with four pseudo-random columns V: the first
// iterative-refinement correction relative to X V, ||X (A X V - V)||_F / ||X V||_F (an estimate
// of X's forward error, from the FP32 block it inverts), above kPcCheck rebuilds that block in
// FP64. (The residual ||A X V - V|| itself is no measure here: on badly scaled blocks it is
// large for the FP64 inverse rounded to FP32 as well.) BEM_C64: every block in FP64.
// ---------------------------------------------------------------------------------------
constexpr double kPcCheck = 1e-2;
constexpr int kPcProbe = 4;

template <typename R> struct CuType;
template <> struct CuType<float> {
  static constexpr cudaDataType t = CUDA_C_32F;
  static constexpr cublasComputeType_t ct = CUBLAS_COMPUTE_32F;
};
template <> struct CuType<double> {
  static constexpr cudaDataType t = CUDA_C_64F;
  static constexpr cublasComputeType_t ct = CUBLAS_COMPUTE_64F;
};

// A_ii (column-major N x N, N = n + m) but for the -j k0 L^A C term of A11 (a GEMM adds it):
//   A11 = j k0 L^A + I_x Z,  A12 = -(F D)^T L^Phi,  A21 = F D (I - C),  A22 = j k0 I.
// Z and C: the object's packed row-major blocks (leading dimension ld); I_x and F D from their
// sparse rows (four I_x entries per edge, three F D entries per triangle).
template <typename R>
__global__ void k_pc_fill(DGeo g, int e0, int n, int t0, int m, double k0,
                          const double2* __restrict__ LA, const double2* __restrict__ LP,
                          const typename C2<R>::T* __restrict__ Z, const typename C2<R>::T* __restrict__ C,
                          int ld, const int32_t* __restrict__ ixcol, const R* __restrict__ ixval,
                          const int32_t* __restrict__ tedge, const R* __restrict__ fdT,
                          typename C2<R>::T* A) {
  typedef typename C2<R>::T V;
  const int N = n + m;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)N * N) return;
  const int r = (int)(idx % N), col = (int)(idx / N);
  R vr = 0, vi = 0;
  if (r < n && col < n) {
    const double2 a = LA[r + (int64_t)col * n];
    vr = (R)(-k0 * a.y);
    vi = (R)(k0 * a.x);
    for (int q = 0; q < 4; ++q) {
      const int k = ixcol[4 * (e0 + r) + q] - e0;
      if (k >= 0 && k < n) {
        const R w = ixval[4 * (e0 + r) + q];
        const V z = Z[(int64_t)k * ld + col];
        vr += w * z.x;
        vi += w * z.y;
      }
    }
  } else if (r < n) {
    const int e = e0 + r, cq = col - n;
    for (int a = 0; a < 2; ++a) {
      const int t = g.et[2 * e + a];
      if (t < t0 || t >= t0 + m) continue;
      for (int q = 0; q < 3; ++q)
        if (tedge[3 * t + q] == e) {
          const R f = fdT[3 * t + q];
          const double2 p = LP[(t - t0) + (int64_t)cq * m];
          vr -= f * (R)p.x;
          vi -= f * (R)p.y;
        }
    }
  } else if (col < n) {
    const int t = t0 + r - n;
    for (int q = 0; q < 3; ++q) {
      const int k = tedge[3 * t + q] - e0;
      if (k >= 0 && k < n) {
        const R f = fdT[3 * t + q];
        const V cc = C[(int64_t)k * ld + col];
        vr += f * ((k == col ? (R)1 : (R)0) - cc.x);
        vi -= f * cc.y;
      }
    }
  } else {
    vi = r == col ? (R)k0 : (R)0;
  }
  V v;
  v.x = vr;
  v.y = vi;
  A[idx] = v;
}

template <typename V>
__global__ void k_identity(V* A, int N) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)N * N) return;
  V v;
  v.x = (idx % N) == (idx / N) ? 1 : 0;
  v.y = 0;
  A[idx] = v;
}

__global__ void k_round_c32(const double2* a, float2* b, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

// probe columns: real and imaginary parts uniform in [-1, 1) from a 64-bit mix of the index
// (the finaliser of MurmurHash3)
template <typename V>
__global__ void k_pc_probe(V* P, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t h = (uint64_t)i * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
  h ^= h >> 33;
  h *= 0xff51afd7ed558ccdull;
  h ^= h >> 33;
  h *= 0xc4ceb9fe1a85ec53ull;
  h ^= h >> 33;
  V v;
  v.x = (double)(h >> 40) / 8388608.0 - 1.0;
  v.y = (double)((h >> 16) & 0xFFFFFF) / 8388608.0 - 1.0;
  P[i] = v;
}

// out = (sum |a|^2, sum |b|^2) in FP64 (one CTA of 256 threads)
template <typename V>
__global__ void k_pc_norms(const V* a, const V* b, int64_t n, double* out) {
  __shared__ double s[2][256];
  double x = 0, y = 0;
  for (int64_t i = threadIdx.x; i < n; i += 256) {
    x += (double)a[i].x * a[i].x + (double)a[i].y * a[i].y;
    y += (double)b[i].x * b[i].x + (double)b[i].y * b[i].y;
  }
  s[0][threadIdx.x] = x;
  s[1][threadIdx.x] = y;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      s[0][threadIdx.x] += s[0][threadIdx.x + w];
      s[1][threadIdx.x] += s[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = s[0][0];
    out[1] = s[1][0];
  }
}

// X (column-major N x N) into the packed row-major block of leading dimension ld, both copies
template <typename V>
__global__ void k_store_pc(const V* X, int N, int ld, double2* P64, float2* P32) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)N * ld) return;
  const int r = (int)(idx / ld), col = (int)(idx % ld);
  double2 v = make_double2(0, 0);
  if (col < N) {
    const V x = X[r + (int64_t)col * N];
    v = make_double2(x.x, x.y);
  }
  P64[idx] = v;
  P32[idx] = make_float2((float)v.x, (float)v.y);
}

static int gemm_t(cublasHandle_t h, cudaDataType t, cublasComputeType_t ct, cublasOperation_t tb,
                  int M, int N, int K, const void* alpha, const void* A, int lda, const void* B,
                  int ldb, const void* beta, void* C, int ldc) {
  if (cublasGemmEx(h, CUBLAS_OP_N, tb, M, N, K, alpha, A, t, lda, B, t, ldb, beta, C, t, ldc, ct,
                   CUBLAS_GEMM_DEFAULT) != CUBLAS_STATUS_SUCCESS) {
    set_error("cublasGemmEx (preconditioner block) failed");
    return BEM_ECUDA;
  }
  return BEM_OK;
}

// work arrays of one build precision, sized for the largest object
template <typename R> struct PcWork {
  typedef typename C2<R>::T V;
  V *LAr = nullptr, *A = nullptr, *Ac = nullptr, *X = nullptr, *P = nullptr, *W = nullptr,
    *Rr = nullptr;
  double* nrm = nullptr;
  std::vector<void*> mem;
  ~PcWork() {
    for (void* p : mem) cudaFree(p);
  }
  int alloc(int nmax, int Nmax) {
    if (A) return BEM_OK;
    const size_t NN = (size_t)Nmax * Nmax, NP = (size_t)Nmax * kPcProbe;
    V** bufs[] = {&LAr, &A, &Ac, &X, &P, &W, &Rr};
    const size_t sizes[] = {sizeof(R) == 4 ? (size_t)nmax * nmax : 0, NN, NN, NN, NP, NP, NP};
    for (int k = 0; k < 7; ++k) {
      if (!sizes[k]) continue;
      if (cudaMalloc((void**)bufs[k], sizes[k] * sizeof(V)) != cudaSuccess) {
        set_error("preconditioner scratch (%zu bytes) allocation failed", sizes[k] * sizeof(V));
        return BEM_ENOMEM;
      }
      mem.push_back(*bufs[k]);
    }
    BEM_CUDA(cudaMalloc(&nrm, 2 * sizeof(double)));
    mem.push_back(nrm);
    return BEM_OK;
  }
};

struct PcShared {
  SolverScratch ss;
  cublasHandle_t bh = nullptr;
  int64_t* ipiv = nullptr;
  int* dinfo = nullptr;
  void* dwork = nullptr;
  size_t dwsize = 0;
  std::vector<char> hwork;
  ~PcShared() {
    if (bh) cublasDestroy(bh);
    if (ipiv) cudaFree(ipiv);
    if (dinfo) cudaFree(dinfo);
    if (dwork) cudaFree(dwork);
  }
};

// X <- A^{-1} (A overwritten by its LU factors), complex type t
static int lu_inverse(PcShared& s, cudaDataType t, void* A, void* X, int n) {
  size_t dws = 0, hws = 0;
  if (cusolverDnXgetrf_bufferSize(s.ss.h, s.ss.p, n, n, t, A, n, t, &dws, &hws) !=
      CUSOLVER_STATUS_SUCCESS) {
    set_error("cusolverDnXgetrf_bufferSize failed");
    return BEM_ECUDA;
  }
  if (dws > s.dwsize) {
    if (s.dwork) cudaFree(s.dwork);
    s.dwork = nullptr;
    BEM_CUDA(cudaMalloc(&s.dwork, dws));
    s.dwsize = dws;
  }
  if (hws > s.hwork.size()) s.hwork.resize(hws);
  if (cusolverDnXgetrf(s.ss.h, s.ss.p, n, n, t, A, n, s.ipiv, t, s.dwork, dws, s.hwork.data(), hws,
                       s.dinfo) != CUSOLVER_STATUS_SUCCESS) {
    set_error("cusolverDnXgetrf failed");
    return BEM_ECUDA;
  }
  int hinfo = 0;
  BEM_CUDA(cudaMemcpy(&hinfo, s.dinfo, sizeof(int), cudaMemcpyDeviceToHost));
  if (hinfo != 0) {
    set_error("singular preconditioner block (getrf info %d)", hinfo);
    return BEM_ESOLVER;
  }
  if (cusolverDnXgetrs(s.ss.h, s.ss.p, CUBLAS_OP_N, n, n, t, A, n, s.ipiv, t, X, n, s.dinfo) !=
      CUSOLVER_STATUS_SUCCESS) {
    set_error("cusolverDnXgetrs failed");
    return BEM_ECUDA;
  }
  return BEM_OK;
}

// one block in precision R: form, invert, check (FP32), store. *resid: the check's value
// (-1 when not checked).
template <typename R>
static int pc_block(aim_ctx* c, const DGeo& g, int i, const double2* LA, const double2* LP,
                    PcWork<R>& w, PcShared& s, int ld, int64_t off, bool check, double* resid) {
  typedef typename C2<R>::T V;
  const cudaDataType t = CuType<R>::t;
  const cublasComputeType_t ct = CuType<R>::ct;
  const PrecBuf<R>& b = buf<R>(c);
  const int e0 = c->e0[i], t0 = c->t0[i];
  const int n = c->e1[i] - e0, m = c->t1[i] - t0, N = n + m;
  const double k0 = c->k0;
  k_pc_fill<R><<<nblk((int64_t)N * N, 256), 256>>>(g, e0, n, t0, m, k0, LA, LP, b.Z + c->zoff[i],
                                                    b.C + c->zoff[i], c->zld[i], c->d_ixcol, b.ix,
                                                    c->d_tedge, b.fdT, w.A);
  const V* LAr = (const V*)LA;
  if (sizeof(R) == 4) {
    k_round_c32<<<nblk((int64_t)n * n, 256), 256>>>(LA, (float2*)w.LAr, (int64_t)n * n);
    LAr = w.LAr;
  }
  BEM_CUDA(cudaGetLastError());
  // A11 -= j k0 L^A C  (C's packed row-major block is C^T in the column-major view)
  V al, one, mone, zero;
  al.x = 0;
  al.y = -k0;
  one.x = 1;
  one.y = 0;
  mone.x = -1;
  mone.y = 0;
  zero.x = 0;
  zero.y = 0;
  BEM_TRY(gemm_t(s.bh, t, ct, CUBLAS_OP_T, n, n, n, &al, LAr, n, b.C + c->zoff[i], c->zld[i], &one,
                 w.A, N));
  if (check) BEM_CUDA(cudaMemcpy(w.Ac, w.A, (size_t)N * N * sizeof(V), cudaMemcpyDeviceToDevice));
  k_identity<V><<<nblk((int64_t)N * N, 256), 256>>>(w.X, N);
  BEM_TRY(lu_inverse(s, t, w.A, w.X, N));
  *resid = -1;
  if (check) {
    const int64_t np = (int64_t)N * kPcProbe;
    k_pc_probe<V><<<nblk(np, 256), 256>>>(w.P, np);
    BEM_CUDA(cudaMemcpy(w.Rr, w.P, np * sizeof(V), cudaMemcpyDeviceToDevice));
    BEM_TRY(gemm_t(s.bh, t, ct, CUBLAS_OP_N, N, kPcProbe, N, &one, w.X, N, w.P, N, &zero, w.W, N));
    BEM_TRY(gemm_t(s.bh, t, ct, CUBLAS_OP_N, N, kPcProbe, N, &one, w.Ac, N, w.W, N, &mone, w.Rr, N));
    // the first refinement correction X (A X V - V), into P, against X V
    BEM_TRY(gemm_t(s.bh, t, ct, CUBLAS_OP_N, N, kPcProbe, N, &one, w.X, N, w.Rr, N, &zero, w.P, N));
    k_pc_norms<V><<<1, 256>>>(w.P, w.W, np, w.nrm);
    double h[2];
    BEM_CUDA(cudaMemcpy(h, w.nrm, sizeof(h), cudaMemcpyDeviceToHost));
    *resid = h[1] > 0 ? std::sqrt(h[0] / h[1]) : 0.0;
    if (!(*resid <= kPcCheck)) return BEM_OK;  // the caller rebuilds the block in FP64
  }
  k_store_pc<V><<<nblk((int64_t)N * ld, 256), 256>>>(w.X, N, ld, c->pc64 + off, c->pc32 + off);
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

int setup_precond(aim_ctx* c, int prec) {
  if (prec < 0) {
    if (c->pc_ready) return BEM_OK;
    prec = BEM_C32;
  }
  if (c->pc_ready && c->pc_prec == prec) return BEM_OK;
  if (prec != BEM_C32 && prec != BEM_C64) {
    set_error("preconditioner build precision must be BEM_C32 or BEM_C64");
    return BEM_EINVAL;
  }
  const double tst = wall_ms();
  const DGeo& g = *reinterpret_cast<const DGeo*>(c->geo_store);
  const int nobj = c->nobj;
  std::vector<int32_t> N(nobj), perm;
  std::vector<int64_t> off(nobj);
  std::vector<int32_t> ld(nobj);
  int64_t o = 0;
  int nmax = 0, mmax = 0, Nmax = 0;
  for (int i = 0; i < nobj; ++i) {
    const int n = c->e1[i] - c->e0[i], m = c->t1[i] - c->t0[i];
    N[i] = n + m;
    ld[i] = (int32_t)round_up(N[i], 4);
    off[i] = o;
    o += (int64_t)N[i] * ld[i];
    nmax = std::max(nmax, n);
    mmax = std::max(mmax, m);
    Nmax = std::max(Nmax, N[i]);
    for (int k = 0; k < n; ++k) perm.push_back(c->e0[i] + k);
    for (int k = 0; k < m; ++k) perm.push_back(c->ne + c->t0[i] + k);
  }
  if (!c->pc64) {
    BEM_TRY(dalloc_t(c, &c->pc64, o));
    BEM_TRY(dalloc_t(c, &c->pc32, o));
    BEM_TRY(upload(c, &c->d_pcperm, perm.data(), perm.size()));
    for (int k = 0; k < 2; ++k) {
      BEM_TRY(dalloc_t(c, &c->pcw32[k], perm.size()));
      BEM_TRY(dalloc_t(c, &c->pcw64[k], perm.size()));
    }
  }
  c->pc_ready = false;
  BEM_CUDA(cudaDeviceSynchronize());
  // FP64 L^A and L^Phi of one object, the pair-moment scratch and the handles
  double2 *LA = nullptr, *LP = nullptr;
  BEM_CUDA(cudaMalloc(&LA, (size_t)nmax * nmax * sizeof(double2)));
  std::unique_ptr<void, decltype(&cudaFree)> hold_la(LA, &cudaFree);
  BEM_CUDA(cudaMalloc(&LP, (size_t)mmax * mmax * sizeof(double2)));
  std::unique_ptr<void, decltype(&cudaFree)> hold_lp(LP, &cudaFree);
  MomentScratch ms;
  PcShared s;
  PcWork<float> w32;
  PcWork<double> w64;
  if (cusolverDnCreate(&s.ss.h) != CUSOLVER_STATUS_SUCCESS ||
      cusolverDnCreateParams(&s.ss.p) != CUSOLVER_STATUS_SUCCESS ||
      cublasCreate(&s.bh) != CUBLAS_STATUS_SUCCESS) {
    set_error("cuSOLVER/cuBLAS handle creation failed");
    return BEM_ECUDA;
  }
  BEM_CUDA(cudaMalloc(&s.ipiv, Nmax * sizeof(int64_t)));
  BEM_CUDA(cudaMalloc(&s.dinfo, sizeof(int)));
  BEM_TRY(prec == BEM_C32 ? w32.alloc(nmax, Nmax) : w64.alloc(nmax, Nmax));
  c->pc_nfp64 = 0;
  c->pc_resid = 0;
  for (int i = 0; i < nobj; ++i) {
    const int n = c->e1[i] - c->e0[i], m = c->t1[i] - c->t0[i];
    BEM_TRY(object_moments(c, g, i, std::complex<double>(c->k0, 0.0), false, &ms));
    k_obj_assemble_A<<<nblk((int64_t)n * n, 128), 128>>>(g, c->e0[i], n, c->t0[i], m, ms.mom, LA);
    k_obj_LP<<<nblk((int64_t)m * m, 256), 256>>>(ms.mom, m, LP);
    BEM_CUDA(cudaGetLastError());
    double r = -1;
    if (prec == BEM_C32) {
      BEM_TRY(pc_block<float>(c, g, i, LA, LP, w32, s, ld[i], off[i], true, &r));
      c->pc_resid = std::max(c->pc_resid, r);
    }
    if (prec == BEM_C64 || !(r <= kPcCheck)) {
      BEM_TRY(w64.alloc(nmax, Nmax));
      BEM_TRY(pc_block<double>(c, g, i, LA, LP, w64, s, ld[i], off[i], false, &r));
      c->pc_nfp64 += 1;
    }
  }
  BEM_CUDA(cudaDeviceSynchronize());
  // persistent GEMV plans over the object-major blocks (autotuned launch shape), made once
  if (!c->pc_planned) {
    float pc_ms[2];
    BEM_TRY(autotune_gemv(c, N, off, ld, c->pc32, &c->pcplan, &c->pcplan64, pc_ms, nullptr));
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int* derr = nullptr;
    BEM_TRY(dalloc_t(c, &derr, 1));
    BEM_TRY(make_gemv_plan(c, nullptr, GemvCand{5, 16, 4, 4}, nsm, N, off, ld, derr, &c->pcmr));
    c->pc_planned = true;
  }
  c->pc_prec = prec;
  c->pc_ms = wall_ms() - tst;
  c->pc_ready = true;
  return BEM_OK;
}

template <typename V>
__global__ void k_perm_gather(const int32_t* perm, const V* x, V* xp, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) xp[i] = x[perm[i]];
}
template <typename V>
__global__ void k_perm_scatter(const int32_t* perm, const V* yp, V* y, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[perm[i]] = yp[i];
}

// u = M_bd r (system ordering), in precision R
template <typename R>
int precond_apply(aim_ctx* c, const void* rv, void* uv, cudaStream_t s) {
  typedef typename C2<R>::T V;
  if (!c->pc_ready) {
    set_error("block-diagonal preconditioner not built");
    return BEM_EINVAL;
  }
  const int n = c->ne + c->nt;
  V* w0 = sizeof(R) == 4 ? (V*)c->pcw32[0] : (V*)c->pcw64[0];
  V* w1 = sizeof(R) == 4 ? (V*)c->pcw32[1] : (V*)c->pcw64[1];
  const V* M = sizeof(R) == 4 ? (const V*)c->pc32 : (const V*)c->pc64;
  k_perm_gather<V><<<nblk(n, 256), 256, 0, s>>>(c->d_pcperm, (const V*)rv, w0, n);
  BEM_TRY(run_gemv_plan<R>(sizeof(R) == 4 ? c->pcplan : c->pcplan64, M, w0, w1, 1, n, nullptr, s));
  k_perm_scatter<V><<<nblk(n, 256), 256, 0, s>>>(c->d_pcperm, w1, (V*)uv, n);
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}
template int precond_apply<float>(aim_ctx*, const void*, void*, cudaStream_t);
template int precond_apply<double>(aim_ctx*, const void*, void*, cudaStream_t);

__global__ void k_perm_gather32(const int32_t* perm, const double2* x, float2* xp, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const double2 v = x[perm[i]];
    xp[i] = make_float2((float)v.x, (float)v.y);
  }
}
__global__ void k_perm_scatter2(const int32_t* perm, const float2* yp, float2* y32, double2* y64,
                                int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const float2 v = yp[i];
    y32[perm[i]] = v;
    y64[perm[i]] = make_double2(v.x, v.y);
  }
}

__global__ void k_perm_gather32b(const int32_t* perm, const double2* x, int64_t xs, float2* xp,
                                 int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const double2 v = x[blockIdx.y * xs + perm[i]];
    xp[(int64_t)blockIdx.y * n + i] = make_float2((float)v.x, (float)v.y);
  }
}
__global__ void k_perm_scatter2b(const int32_t* perm, const float2* yp, float2* y32, double2* y64,
                                 int64_t ys, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const float2 v = yp[(int64_t)blockIdx.y * n + i];
    y32[blockIdx.y * ys + perm[i]] = v;
    y64[blockIdx.y * ys + perm[i]] = make_double2(v.x, v.y);
  }
}

// The FP32 preconditioner of nrhs FP64 Krylov vectors r (stride ys = N_E + N_T) at once, the
// block matrices read once for all of them: u32 (FP32, the batched product's input) and u64
// (FP64), both with stride ys.
int precond_apply_batch(aim_ctx* c, const double2* r, int nrhs, float2* u32, double2* u64,
                        cudaStream_t s) {
  if (!c->pc_ready || nrhs < 1 || nrhs > kMaxBatch) {
    set_error("batched preconditioner: not built or nrhs out of range");
    return BEM_EINVAL;
  }
  const int n = c->ne + c->nt;
  if (!c->pcb32[0])
    for (int k = 0; k < 2; ++k) BEM_TRY(dalloc_t(c, &c->pcb32[k], (size_t)kMaxBatch * n));
  const dim3 g(nblk(n, 256), nrhs);
  k_perm_gather32b<<<g, 256, 0, s>>>(c->d_pcperm, r, n, c->pcb32[0], n);
  if (c->pcmr.ntasks > 0)
    BEM_TRY(run_gemv_mr<float>(c->pcmr, (const float2*)c->pc32, c->pcb32[0], c->pcb32[1], nrhs, n,
                               nullptr, s));
  else
    BEM_TRY(run_gemv_plan<float>(c->pcplan, (const float2*)c->pc32, c->pcb32[0], c->pcb32[1], nrhs,
                                 n, nullptr, s));
  k_perm_scatter2b<<<g, 256, 0, s>>>(c->d_pcperm, c->pcb32[1], u32, u64, n, n);
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

// The FP32 preconditioner of an FP64 Krylov vector: u = M_bd (float) r, returned both in FP32
// (u32, the next FP32 product's input) and in FP64 (u64, the flexible basis); the conversions
// ride on the permutation launches.
int precond_apply_mixed(aim_ctx* c, const double2* r, float2* u32, double2* u64, cudaStream_t s) {
  if (!c->pc_ready) {
    set_error("block-diagonal preconditioner not built");
    return BEM_EINVAL;
  }
  const int n = c->ne + c->nt;
  float2* w0 = (float2*)c->pcw32[0];
  float2* w1 = (float2*)c->pcw32[1];
  k_perm_gather32<<<nblk(n, 256), 256, 0, s>>>(c->d_pcperm, r, w0, n);
  BEM_TRY(run_gemv_plan<float>(c->pcplan, (const float2*)c->pc32, w0, w1, 1, n, nullptr, s));
  k_perm_scatter2<<<nblk(n, 256), 256, 0, s>>>(c->d_pcperm, w1, u32, u64, n);
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

int rhs_plane_wave(aim_ctx* c, const double* pol, const double* kh, void* b, int prec,
                   cudaStream_t st) {
  const DGeo& g = *reinterpret_cast<const DGeo*>(c->geo_store);
  const double inv_eta0 = 1.0 / (kMu0 * kC0);
  int n = c->ne + c->nt;
  if (prec == BEM_C64)
    k_rhs_pw<double2><<<nblk(n, 128), 128, 0, st>>>(g, c->ne, c->nt, c->k0, pol[0], pol[1], pol[2],
                                                    kh[0], kh[1], kh[2], inv_eta0, (double2*)b);
  else
    k_rhs_pw<float2><<<nblk(n, 128), 128, 0, st>>>(g, c->ne, c->nt, c->k0, pol[0], pol[1], pol[2],
                                                   kh[0], kh[1], kh[2], inv_eta0, (float2*)b);
  BEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

int export_LK(aim_ctx* c, int obj, int pass, double2* L_out, double2* K_out) {
  const DGeo& g = *reinterpret_cast<const DGeo*>(c->geo_store);
  const int n = c->e1[obj] - c->e0[obj];
  const bem_material& mt = c->mat[obj];
  const double w = 2.0 * kPi * c->freq;
  std::complex<double> k(c->k0, 0.0);
  if (pass == 0) {
    std::complex<double> epsc(mt.eps_r, -mt.sigma / (w * kEps0));
    k = c->k0 * std::sqrt(epsc * mt.mu_r);
    if (k.imag() > 0) k = -k;
  }
  const size_t nn = (size_t)n * n;
  double2 *L = nullptr, *B = nullptr;
  BEM_CUDA(cudaMalloc(&L, nn * sizeof(double2)));
  cudaError_t e = cudaMalloc(&B, nn * sizeof(double2));
  if (e == cudaSuccess) {
    MomentScratch ms;
    if (object_LK(c, g, obj, k, &ms, L, B) != BEM_OK) e = cudaErrorUnknown;
    else e = cudaDeviceSynchronize();
  }
  std::vector<double2> tl, tb;
  if (e == cudaSuccess) {
    tl.resize(nn);
    tb.resize(nn);
    e = cudaMemcpy(tl.data(), L, nn * sizeof(double2), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(tb.data(), B, nn * sizeof(double2), cudaMemcpyDeviceToHost);
  }
  cudaFree(L);
  if (B) cudaFree(B);
  if (e != cudaSuccess) {
    set_error("export_LK: %s", cudaGetErrorString(e));
    return BEM_ECUDA;
  }
  // the set-up kernel writes column-major; the export is row-major
  for (int r = 0; r < n; ++r)
    for (int col = 0; col < n; ++col) {
      L_out[(size_t)r * n + col] = tl[r + (size_t)col * n];
      K_out[(size_t)r * n + col] = tb[r + (size_t)col * n];
    }
  return BEM_OK;
}

void free_geo_store(aim_ctx* c) {
  delete reinterpret_cast<DGeo*>(c->geo_store);
  c->geo_store = nullptr;
}

double k0_of(double f) { return 2.0 * kPi * f / kC0 * kEll; }

}  // namespace bem
