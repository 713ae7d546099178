// Excitation and post-processing on the device: lumped (delta-gap) ports and the radiated far
// field of the solution.
//
// Ports (Sec. II names lumped ports, after Wang 2004, without the model): a port is a closed
// ring of mesh edges around a conductor's cross-section at one axial position; a gap voltage V
// drives E_inc = V delta(s - s_p) along the axis, so <f_m, E_inc> = s_m V l_m on the ring edges
// (s_m = +1 when f_m crosses the ring along +axis), and the port current is the circulation of
// H around the ring (Ampere): I = sum_m s_m l_m h_m.
//
// Far field: only J_Delta radiates into the background in the equivalent problem (Sec. II), so
// E_far(r) = -j k0 eta0 exp(-j k0 r) / (4 pi r) (I - rhat rhat) N(rhat) with the radiation vector
// N(rhat) = int J_Delta(r') exp(j k0 rhat . r') dS', J_Delta = sum_n j_n f_n, j = h - Y_eq Z h.
#include <cmath>
#include <vector>

#include "common.cuh"

namespace bem {

// Per-triangle far-field data (host-built once per context): the 7-point rule's points and
// weights times the area, the three vertices opposite the triangle's edges, and for each edge
// its index and s l / (2 A).
struct FarGeo {
  double* pts = nullptr;   // [nt][7][3]
  double* wts = nullptr;   // [nt][7]
  double* vop = nullptr;   // [nt][3][3]
  double* cf = nullptr;    // [nt][3]
  int32_t* edge = nullptr; // [nt][3]
};

static int far_geo(aim_ctx* c, FarGeo** out) {
  if (c->far_geo) {
    *out = static_cast<FarGeo*>(c->far_geo);
    return BEM_OK;
  }
  const int nt = c->nt;
  double r7[28];
  radon7_host(r7);
  std::vector<double> pts(21 * (size_t)nt), wts(7 * (size_t)nt), vop(9 * (size_t)nt), cf(3 * (size_t)nt);
  std::vector<int32_t> edge(3 * (size_t)nt);
  for (int t = 0; t < nt; ++t) {
    const double* P[3];
    for (int i = 0; i < 3; ++i) P[i] = &c->verts[3 * c->tris[3 * t + i]];
    for (int q = 0; q < 7; ++q) {
      for (int a = 0; a < 3; ++a)
        pts[(7 * t + q) * 3 + a] =
            r7[4 * q] * P[0][a] + r7[4 * q + 1] * P[1][a] + r7[4 * q + 2] * P[2][a];
      wts[7 * t + q] = r7[4 * q + 3] * c->area[t];
    }
    for (int i = 0; i < 3; ++i) {
      const int e = c->t_edges[3 * t + i];
      edge[3 * t + i] = e;
      cf[3 * t + i] = c->t_esign[3 * t + i] * c->elen[e] / (2.0 * c->area[t]);
      const double* v = &c->verts[3 * c->t_evert[3 * t + i]];
      for (int a = 0; a < 3; ++a) vop[(3 * t + i) * 3 + a] = v[a];
    }
  }
  FarGeo* g = new FarGeo;
  int rc = BEM_OK;
  if ((rc = upload(c, &g->pts, pts.data(), pts.size())) || (rc = upload(c, &g->wts, wts.data(), wts.size())) ||
      (rc = upload(c, &g->vop, vop.data(), vop.size())) || (rc = upload(c, &g->cf, cf.data(), cf.size())) ||
      (rc = upload(c, &g->edge, edge.data(), edge.size()))) {
    delete g;
    return rc;
  }
  c->far_geo = g;
  *out = g;
  return BEM_OK;
}

void free_far_geo(aim_ctx* c) {
  delete static_cast<FarGeo*>(c->far_geo);  // device arrays are context allocations
  c->far_geo = nullptr;
}

// N[d] += sum over triangles of the 7-point rule of J_Delta(r_q) exp(j k0 rhat_d . r_q), in FP64;
// j = h - heq read in the solution's precision. One thread per triangle, block reduction, one
// set of FP64 atomics per block and direction.
template <typename V>
__global__ void __launch_bounds__(256) k_farfield(FarGeo g, int nt, const V* __restrict__ h,
                                                  const V* __restrict__ heq, double k0,
                                                  const double* __restrict__ rhat, double* N) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x, d = blockIdx.y;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  if (t < nt) {
    const double rx = rhat[3 * d], ry = rhat[3 * d + 1], rz = rhat[3 * d + 2];
    double cr[3], ci[3];
    for (int i = 0; i < 3; ++i) {
      const int e = g.edge[3 * t + i];
      const double jr = (double)h[e].x - (double)heq[e].x, ji = (double)h[e].y - (double)heq[e].y;
      cr[i] = g.cf[3 * t + i] * jr;
      ci[i] = g.cf[3 * t + i] * ji;
    }
    for (int q = 0; q < 7; ++q) {
      const double* r = &g.pts[(7 * t + q) * 3];
      double s, co;
      sincos(k0 * (rx * r[0] + ry * r[1] + rz * r[2]), &s, &co);
      const double w = g.wts[7 * t + q];
      for (int a = 0; a < 3; ++a) {
        double jr = 0, ji = 0;
        for (int i = 0; i < 3; ++i) {
          const double dv = r[a] - g.vop[(3 * t + i) * 3 + a];
          jr += cr[i] * dv;
          ji += ci[i] * dv;
        }
        acc[2 * a] += w * (jr * co - ji * s);
        acc[2 * a + 1] += w * (jr * s + ji * co);
      }
    }
  }
  __shared__ double red[8][6];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < 6; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double v = 0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) v += red[w][threadIdx.x];
    atomicAdd(&N[6 * d + threadIdx.x], v);
  }
}

template <typename V>
__global__ void k_port_rhs(const int32_t* __restrict__ edges, const double* __restrict__ val, int n,
                           V* b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[edges[i]] = mk((decltype(b[0].x))val[i], (decltype(b[0].x))0);
}

template <typename V>
__global__ void k_gather(const int32_t* __restrict__ edges, int n, const V* __restrict__ x,
                         double2* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = make_double2((double)x[edges[i]].x, (double)x[edges[i]].y);
}

static int check_edges(const aim_ctx* c, int n, const int32_t* edges, const double* signs,
                       const char* who) {
  if (n < 1 || !edges || !signs) {
    set_error("%s: empty or null port", who);
    return BEM_EINVAL;
  }
  for (int i = 0; i < n; ++i)
    if (edges[i] < 0 || edges[i] >= c->ne || !std::isfinite(signs[i])) {
      set_error("%s: edge %d out of range or bad sign", who, edges[i]);
      return BEM_EINVAL;
    }
  return BEM_OK;
}

}  // namespace bem

using namespace bem;

extern "C" {

int bem_port_ring(aim_ctx* c, int obj, int axis, double coord, double tol, int32_t* edges,
                  double* signs, int cap) {
  if (!c || obj < 0 || obj >= c->nobj || axis < 0 || axis > 2 || !(tol >= 0)) {
    set_error("bem_port_ring: bad arguments");
    return BEM_EINVAL;
  }
  int cnt = 0;
  for (int m = c->e0[obj]; m < c->e1[obj]; ++m) {
    const double za = c->verts[3 * c->ev[2 * m] + axis], zb = c->verts[3 * c->ev[2 * m + 1] + axis];
    if (std::fabs(za - coord) > tol || std::fabs(zb - coord) > tol) continue;
    // f_m points from T+ into T-: its crossing direction is that of centroid(T-) - centroid(T+)
    const double dz = c->centroid[3 * c->et[2 * m + 1] + axis] - c->centroid[3 * c->et[2 * m] + axis];
    if (cnt < cap && edges && signs) {
      edges[cnt] = m;
      signs[cnt] = dz > 0 ? 1.0 : (dz < 0 ? -1.0 : 0.0);
    }
    ++cnt;
  }
  return cnt;
}

int bem_rhs_port(aim_ctx* c, int n, const int32_t* edges, const double* signs, double v_gap,
                 void* b, int prec, void* stream) {
  if (!c || !b || (prec != BEM_C32 && prec != BEM_C64)) {
    set_error("bem_rhs_port: bad arguments");
    return BEM_EINVAL;
  }
  BEM_TRY(check_edges(c, n, edges, signs, "bem_rhs_port"));
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t N = (int64_t)c->ne + c->nt;
  const size_t es = prec == BEM_C32 ? sizeof(float2) : sizeof(double2);
  std::vector<double> val(n);
  // <f_m, E_inc> / eta0 = s_m l_m V / eta0 in SI units; the first block row of the system in
  // micrometre units is the SI row divided by ell^2, and l_m is in micrometres here
  for (int i = 0; i < n; ++i) val[i] = signs[i] * c->elen[edges[i]] * v_gap / (kEta0 * kEll);
  int32_t* de = nullptr;
  double* dv = nullptr;
  BEM_CUDA(cudaMallocAsync((void**)&de, n * sizeof(int32_t), s));
  BEM_CUDA(cudaMallocAsync((void**)&dv, n * sizeof(double), s));
  BEM_CUDA(cudaMemcpyAsync(de, edges, n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  BEM_CUDA(cudaMemcpyAsync(dv, val.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
  BEM_CUDA(cudaMemsetAsync(b, 0, N * es, s));
  if (prec == BEM_C32) k_port_rhs<<<(n + 127) / 128, 128, 0, s>>>(de, dv, n, (float2*)b);
  else k_port_rhs<<<(n + 127) / 128, 128, 0, s>>>(de, dv, n, (double2*)b);
  BEM_CUDA(cudaGetLastError());
  BEM_CUDA(cudaFreeAsync(de, s));
  BEM_CUDA(cudaFreeAsync(dv, s));
  // the host arrays must outlive the asynchronous copies
  BEM_CUDA(cudaStreamSynchronize(s));
  return BEM_OK;
}

int bem_port_current(aim_ctx* c, int n, const int32_t* edges, const double* signs, const void* x,
                     int prec, double* current, void* stream) {
  if (!c || !x || !current || (prec != BEM_C32 && prec != BEM_C64)) {
    set_error("bem_port_current: bad arguments");
    return BEM_EINVAL;
  }
  BEM_TRY(check_edges(c, n, edges, signs, "bem_port_current"));
  cudaStream_t s = (cudaStream_t)stream;
  int32_t* de = nullptr;
  double2* dh = nullptr;
  BEM_CUDA(cudaMallocAsync((void**)&de, n * sizeof(int32_t), s));
  BEM_CUDA(cudaMallocAsync((void**)&dh, n * sizeof(double2), s));
  BEM_CUDA(cudaMemcpyAsync(de, edges, n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  if (prec == BEM_C32) k_gather<<<(n + 127) / 128, 128, 0, s>>>(de, n, (const float2*)x, dh);
  else k_gather<<<(n + 127) / 128, 128, 0, s>>>(de, n, (const double2*)x, dh);
  BEM_CUDA(cudaGetLastError());
  std::vector<double2> hv(n);
  BEM_CUDA(cudaMemcpyAsync(hv.data(), dh, n * sizeof(double2), cudaMemcpyDeviceToHost, s));
  BEM_CUDA(cudaFreeAsync(de, s));
  BEM_CUDA(cudaFreeAsync(dh, s));
  BEM_CUDA(cudaStreamSynchronize(s));
  double re = 0, im = 0;
  for (int i = 0; i < n; ++i) {
    const double w = signs[i] * c->elen[edges[i]] * kEll;  // metres
    re += w * hv[i].x;
    im += w * hv[i].y;
  }
  current[0] = re;
  current[1] = im;
  return BEM_OK;
}

int bem_port_matrix(aim_ctx* c, int nport, const int32_t* ring_n, const int32_t* edges,
                    const double* signs, const bem_solve_opts* opts, double* Y,
                    bem_solve_info* infos, void* stream) {
  if (!c || nport < 1 || !ring_n || !edges || !signs || !opts || !Y) {
    set_error("bem_port_matrix: bad arguments");
    return BEM_EINVAL;
  }
  std::vector<int64_t> off(nport + 1, 0);
  for (int p = 0; p < nport; ++p) {
    if (ring_n[p] < 1) {
      set_error("bem_port_matrix: port %d has no edges", p);
      return BEM_EINVAL;
    }
    off[p + 1] = off[p] + ring_n[p];
  }
  for (int p = 0; p < nport; ++p)
    BEM_TRY(check_edges(c, ring_n[p], edges + off[p], signs + off[p], "bem_port_matrix"));
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t N = (int64_t)c->ne + c->nt;
  // ports in groups of up to kMaxBatch solved together (bem_solve_batch) when the options allow
  const int G = opts->precond <= 1 ? std::min(nport, (int)kMaxBatch) : 1;
  double2 *b = nullptr, *x = nullptr;
  BEM_CUDA(cudaMalloc((void**)&b, G * N * sizeof(double2)));
  if (cudaMalloc((void**)&x, G * N * sizeof(double2)) != cudaSuccess) {
    cudaFree(b);
    set_error("bem_port_matrix: out of device memory");
    return BEM_ENOMEM;
  }
  int worst = BEM_OK;
  std::vector<bem_solve_info> inf(G);
  for (int q0 = 0; q0 < nport && worst >= 0; q0 += G) {
    const int g = std::min(G, nport - q0);
    // unit gap voltage on port q, the others shorted; Y_pq = I_p / V_q
    int rc = BEM_OK;
    for (int i = 0; i < g && rc == BEM_OK; ++i)
      rc = bem_rhs_port(c, ring_n[q0 + i], edges + off[q0 + i], signs + off[q0 + i], 1.0, b + i * N,
                        BEM_C64, stream);
    if (rc == BEM_OK && cudaMemsetAsync(x, 0, g * N * sizeof(double2), s) != cudaSuccess) rc = BEM_ECUDA;
    if (rc == BEM_OK)
      rc = g > 1 ? bem_solve_batch(c, b, x, g, opts, inf.data(), stream)
                 : bem_solve(c, b, x, opts, inf.data(), stream);
    if (rc < 0) {
      worst = rc;
      break;
    }
    worst = std::max(worst, rc);
    for (int i = 0; i < g && worst >= 0; ++i) {
      const int q = q0 + i;
      if (infos) infos[q] = inf[i];
      for (int p = 0; p < nport; ++p) {
        double cur[2];
        const int r2 = bem_port_current(c, ring_n[p], edges + off[p], signs + off[p], x + i * N,
                                        BEM_C64, cur, stream);
        if (r2 != BEM_OK) {
          worst = r2;
          break;
        }
        Y[2 * (p * nport + q)] = cur[0];
        Y[2 * (p * nport + q) + 1] = cur[1];
      }
    }
  }
  cudaFree(b);
  cudaFree(x);
  return worst;
}

int bem_farfield(aim_ctx* c, const void* x, int prec, int ndir, const double* rhat, double* nvec,
                 void* stream) {
  if (!c || !x || !rhat || !nvec || ndir < 1 || ndir > 65535 || (prec != BEM_C32 && prec != BEM_C64)) {
    set_error("bem_farfield: bad arguments");
    return BEM_EINVAL;
  }
  for (int d = 0; d < ndir; ++d) {
    const double r2 = rhat[3 * d] * rhat[3 * d] + rhat[3 * d + 1] * rhat[3 * d + 1] + rhat[3 * d + 2] * rhat[3 * d + 2];
    if (!(std::fabs(r2 - 1.0) < 1e-6)) {
      set_error("bem_farfield: direction %d is not a unit vector", d);
      return BEM_EINVAL;
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  FarGeo* g = nullptr;
  BEM_TRY(far_geo(c, &g));
  double *dr = nullptr, *dn = nullptr;
  BEM_CUDA(cudaMallocAsync((void**)&dr, 3 * ndir * sizeof(double), s));
  BEM_CUDA(cudaMallocAsync((void**)&dn, 6 * ndir * sizeof(double), s));
  BEM_CUDA(cudaMemcpyAsync(dr, rhat, 3 * ndir * sizeof(double), cudaMemcpyHostToDevice, s));
  BEM_CUDA(cudaMemsetAsync(dn, 0, 6 * ndir * sizeof(double), s));
  const dim3 grid((c->nt + 255) / 256, ndir);
  if (prec == BEM_C32) {
    BEM_TRY(internal<float>(c, x, c->f32.e, c->f32.heq, 1, s));
    k_farfield<<<grid, 256, 0, s>>>(*g, c->nt, (const float2*)x, c->f32.heq, c->k0, dr, dn);
  } else {
    BEM_TRY(internal<double>(c, x, c->f64.e, c->f64.heq, 1, s));
    k_farfield<<<grid, 256, 0, s>>>(*g, c->nt, (const double2*)x, c->f64.heq, c->k0, dr, dn);
  }
  BEM_CUDA(cudaGetLastError());
  BEM_CUDA(cudaMemcpyAsync(nvec, dn, 6 * ndir * sizeof(double), cudaMemcpyDeviceToHost, s));
  BEM_CUDA(cudaFreeAsync(dr, s));
  BEM_CUDA(cudaFreeAsync(dn, s));
  BEM_CUDA(cudaStreamSynchronize(s));
  return BEM_OK;
}

}  // extern "C"
