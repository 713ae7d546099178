// extern "C" entry points of libbem_aim.so (declared and documented in include/bem_aim.h).
#include <cstdarg>
#include <cstring>

#include "common.cuh"

namespace bem {

static thread_local char g_err[1024] = {0};

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int dalloc(aim_ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? BEM_ENOMEM : BEM_ECUDA;
  }
  c->allocs.push_back(*p);
  return BEM_OK;
}

static int check_ctx(const aim_ctx* c, const char* who) {
  if (!c) {
    set_error("%s: null context", who);
    return BEM_EINVAL;
  }
  return BEM_OK;
}

static int check_prec(int prec, const char* who) {
  if (prec != BEM_C32 && prec != BEM_C64) {
    set_error("%s: prec must be BEM_C32 or BEM_C64", who);
    return BEM_EINVAL;
  }
  return BEM_OK;
}

}  // namespace bem

using namespace bem;

extern "C" {

const char* bem_last_error(void) { return g_err; }

int aim_setup(const bem_mesh* mesh, const aim_grid* grid, double freq_hz, aim_ctx** out) {
  g_err[0] = 0;
  if (!out) {
    set_error("aim_setup: null output pointer");
    return BEM_EINVAL;
  }
  *out = nullptr;
  if (!(freq_hz > 0) || !std::isfinite(freq_hz)) {
    set_error("aim_setup: frequency must be positive");
    return BEM_EINVAL;
  }
  aim_ctx* c = new aim_ctx();
  cudaGetDevice(&c->device);
  c->freq = freq_hz;
  c->k0 = k0_of(freq_hz);
  const double t0 = wall_ms();
  int rc = build_geometry(c, mesh, grid);
  c->setup_ms[0] = wall_ms() - t0;
  if (rc == BEM_OK) rc = setup_device(c);
  if (rc != BEM_OK) {
    aim_destroy(c);
    return rc;
  }
  *out = c;
  return BEM_OK;
}

void aim_destroy(aim_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  for (void* p : c->allocs) cudaFree(p);
  release_streams(c);
  free_net(c);
  free_geo_store(c);
  free_far_geo(c);
  free_zsp(c);
  free_tc(c);
  if (c->gm_ws) cudaFree(c->gm_ws);
  if (c->gmb_ws) cudaFree(c->gmb_ws);
  delete c;
}

int aim_info(const aim_ctx* c, int64_t* info, int n) {
  BEM_TRY(check_ctx(c, "aim_info"));
  if (!info || n < 0) {
    set_error("aim_info: bad output");
    return BEM_EINVAL;
  }
  int maxn = 0;
  for (int i = 0; i < c->nobj; ++i) maxn = std::max(maxn, c->e1[i] - c->e0[i]);
  auto ns = [](float ms5) -> int64_t { return ms5 < 1e29f ? (int64_t)(ms5 * 1e6f / 5.f) : -1; };
  const int kind = c->gplan.tma ? 2 : c->gplan.stream ? 3 : c->gplan.flat ? 1 : c->gplan.ctr ? 6 : c->gplan.ntasks ? 5 : 0;
  int64_t v[22] = {c->ne, c->nt, c->nobj, c->gn[0], c->gn[1], c->gn[2], c->gp[0], c->gp[1], c->gp[2],
                   c->rowA.empty() ? 0 : c->rowA.back(), c->rowP.empty() ? 0 : c->rowP.back(),
                   2 * c->zelems * 8, maxn, c->gplan.ncta,
                   c->gplan.tma ? -c->gplan.nstage : kind != 0 && kind < 5 ? 0 : c->gplan.split,
                   c->gplan.tma ? 0 : c->gplan.unroll, ns(c->tune_ms[0]), ns(c->tune_ms[1]),
                   c->tune_rejected, kind, c->gplan.cps, c->z_after};
  for (int i = 0; i < n && i < 22; ++i) info[i] = v[i];
  for (int i = 22; i < n && i < 32; ++i) info[i] = (int64_t)(c->setup_ms[i - 22] * 1e3);
  const bool pc = c->pc_ready;
  const int64_t w[4] = {pc ? (int64_t)(c->pc_ms * 1e3) : 0, pc ? c->pc_prec : -1,
                        pc ? c->pc_nfp64 : 0,
                        pc && c->pc_prec == BEM_C32 ? (int64_t)(c->pc_resid * 1e12) : -1};
  for (int i = 32; i < n && i < 36; ++i) info[i] = w[i - 32];
  int64_t z[6];
  zsp_stats(c, z);
  const int64_t zv[7] = {(int64_t)(c->setup_ms[10] * 1e3), z[0], z[1], z[2], z[3], z[4], z[5]};
  for (int i = 36; i < n && i < 43; ++i) info[i] = zv[i - 36];
  int64_t tv[2];
  tc_stats(c, tv);
  for (int i = 43; i < n && i < 45; ++i) info[i] = tv[i - 43];
  return BEM_OK;
}

int aim_gemv_select(aim_ctx* c, int kind) {
  BEM_TRY(check_ctx(c, "aim_gemv_select"));
  if (kind < 0 || kind > 2) {
    set_error("aim_gemv_select: kind must be 0 (autotuned), 1 (plain) or 2 (staged)");
    return BEM_EINVAL;
  }
  const bem::GemvPlan& p = kind == 0 ? c->gplan_auto : c->gplan_alt[kind - 1];
  if (p.ncta == 0) {
    set_error("aim_gemv_select: no %s plan (no candidate of that kind ran correctly at set-up)",
              kind == 2 ? "staged" : "plain");
    return BEM_EINVAL;
  }
  BEM_CUDA(cudaDeviceSynchronize());
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);  // they hold the old launches
  c->graphs.clear();
  c->gplan = p;
  // the paired launch holds the autotuned shape: another choice runs e = Z h after j's GEMV
  c->z_after = kind != 0 && c->z_tuned == 3 ? 2 : c->z_tuned;
  return BEM_OK;
}

int aim_gemv_plan(aim_ctx* c, int kind, int ctas_per_sm, int split, int unroll) {
  BEM_TRY(check_ctx(c, "aim_gemv_plan"));
  BEM_CUDA(cudaDeviceSynchronize());
  BEM_TRY(set_gemv_shape(c, kind, ctas_per_sm, split, unroll));
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);  // they hold the old launches
  c->graphs.clear();
  if (c->z_tuned == 3) c->z_after = 2;  // the paired launch holds the autotuned shape
  return BEM_OK;
}

int aim_matvec_batch(aim_ctx* c, const void* x, void* y, int nrhs, int prec, void* stream) {
  BEM_TRY(check_ctx(c, "aim_matvec_batch"));
  BEM_TRY(check_prec(prec, "aim_matvec_batch"));
  if (!x || !y || x == y || nrhs < 1 || nrhs > kMaxBatch) {
    set_error("aim_matvec_batch: distinct x and y and 1 <= nrhs <= %d required", kMaxBatch);
    return BEM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == BEM_C32) {
    BEM_TRY(batch_buffers<float>(c));
    return matvec_graph<float>(c, kBatchOp + nrhs, x, y, s);
  }
  BEM_TRY(batch_buffers<double>(c));
  return matvec_graph<double>(c, kBatchOp + nrhs, x, y, s);
}

int aim_matvec_host(aim_ctx* c, int which, const void* x, void* y, int nvec, int prec, void* stream) {
  BEM_TRY(check_ctx(c, "aim_matvec_host"));
  BEM_TRY(check_prec(prec, "aim_matvec_host"));
  if (!x || !y || x == y || nvec < 1) {
    set_error("aim_matvec_host: x and y must be distinct host pointers and nvec >= 1");
    return BEM_EINVAL;
  }
  const int64_t n = which == AIM_OP_LA ? c->ne : which == AIM_OP_LPHI ? c->nt
                    : (which == AIM_OP_SYSTEM || which == AIM_OP_EXT) ? (int64_t)c->ne + c->nt : -1;
  if (n < 0) {
    set_error("aim_matvec_host: unknown operator %d", which);
    return BEM_EINVAL;
  }
  const size_t bytes = (size_t)n * (prec == BEM_C32 ? sizeof(float2) : sizeof(double2));
  if (!c->h2d) {
    BEM_CUDA(cudaStreamCreateWithFlags(&c->h2d, cudaStreamNonBlocking));
    BEM_CUDA(cudaStreamCreateWithFlags(&c->d2h, cudaStreamNonBlocking));
    for (int b = 0; b < 2; ++b) {
      BEM_CUDA(cudaEventCreateWithFlags(&c->ev_in[b], cudaEventDisableTiming));
      BEM_CUDA(cudaEventCreateWithFlags(&c->ev_comp[b], cudaEventDisableTiming));
      BEM_CUDA(cudaEventCreateWithFlags(&c->ev_out[b], cudaEventDisableTiming));
    }
  }
  // the system operator takes the vectors kMaxBatch at a time through the batched product
  const int G = which == AIM_OP_SYSTEM ? kMaxBatch : 1;
  if (G > 1) {
    if (prec == BEM_C32) BEM_TRY(batch_buffers<float>(c));
    else BEM_TRY(batch_buffers<double>(c));
  }
  if (c->hbuf_bytes < (size_t)G * bytes) {  // kMaxBatch system vectors in FP64 serve every call
    const size_t big = (size_t)kMaxBatch * ((size_t)c->ne + c->nt) * sizeof(double2);
    BEM_CUDA(cudaDeviceSynchronize());
    for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);  // keyed by the old buffers
    c->graphs.clear();
    for (auto& pr : c->hbuf)
      for (void*& p : pr) {
        if (p) cudaFree(p);
        p = nullptr;
      }
    c->hbuf_bytes = 0;
    for (auto& pr : c->hbuf)
      for (void*& p : pr)
        if (cudaMalloc(&p, big) != cudaSuccess) {
          set_error("aim_matvec_host: out of device memory");
          return BEM_ENOMEM;
        }
    c->hbuf_bytes = big;
  }
  cudaStream_t s = (cudaStream_t)stream;
  // the copies start after the work already on the caller's stream
  BEM_CUDA(cudaEventRecord(c->ev_in[0], s));
  BEM_CUDA(cudaStreamWaitEvent(c->h2d, c->ev_in[0], 0));
  BEM_CUDA(cudaStreamWaitEvent(c->d2h, c->ev_in[0], 0));
  const char* xh = static_cast<const char*>(x);
  char* yh = static_cast<char*>(y);
  const int ngroup = (nvec + G - 1) / G;
  for (int i = 0; i < ngroup; ++i) {
    const int b = i & 1, v0 = i * G, g = std::min(G, nvec - v0);
    void* xd = c->hbuf[b][0];
    void* yd = c->hbuf[b][1];
    // group i may overwrite buffer b once product i - 2 has read it
    if (i >= 2) BEM_CUDA(cudaStreamWaitEvent(c->h2d, c->ev_comp[b], 0));
    BEM_CUDA(cudaMemcpyAsync(xd, xh + (size_t)v0 * bytes, (size_t)g * bytes, cudaMemcpyHostToDevice,
                             c->h2d));
    BEM_CUDA(cudaEventRecord(c->ev_in[b], c->h2d));
    BEM_CUDA(cudaStreamWaitEvent(s, c->ev_in[b], 0));
    // y of group i may overwrite buffer b once group i - 2 has gone to the host
    if (i >= 2) BEM_CUDA(cudaStreamWaitEvent(s, c->ev_out[b], 0));
    const int op = G > 1 ? kBatchOp + g : which;
    BEM_TRY(prec == BEM_C32 ? matvec_graph<float>(c, op, xd, yd, s) : matvec_graph<double>(c, op, xd, yd, s));
    BEM_CUDA(cudaEventRecord(c->ev_comp[b], s));
    BEM_CUDA(cudaStreamWaitEvent(c->d2h, c->ev_comp[b], 0));
    BEM_CUDA(cudaMemcpyAsync(yh + (size_t)v0 * bytes, yd, (size_t)g * bytes, cudaMemcpyDeviceToHost,
                             c->d2h));
    BEM_CUDA(cudaEventRecord(c->ev_out[b], c->d2h));
  }
  BEM_CUDA(cudaStreamWaitEvent(s, c->ev_out[(ngroup - 1) & 1], 0));
  return BEM_OK;
}

int aim_matvec_schedule(aim_ctx* c, int mode) {
  BEM_TRY(check_ctx(c, "aim_matvec_schedule"));
  if (mode < -1 || mode > 3 || (mode == 3 && c->gpair.ntasks == 0)) {
    set_error("aim_matvec_schedule: mode must be -1..3 (3 needs the paired plan of the set-up)");
    return BEM_EINVAL;
  }
  BEM_CUDA(cudaDeviceSynchronize());
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);  // they hold the old schedule
  c->graphs.clear();
  c->z_after = mode < 0 ? c->z_tuned : mode;
  return BEM_OK;
}

int aim_matvec(aim_ctx* c, int which, const void* x, void* y, int prec, void* stream) {
  BEM_TRY(check_ctx(c, "aim_matvec"));
  BEM_TRY(check_prec(prec, "aim_matvec"));
  if (!x || !y || x == y) {
    set_error("aim_matvec: x and y must be distinct device pointers");
    return BEM_EINVAL;
  }
  if (which < AIM_OP_LA || which > AIM_OP_EXT) {
    set_error("aim_matvec: unknown operator %d", which);
    return BEM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  return prec == BEM_C32 ? matvec_graph<float>(c, which, x, y, s) : matvec_graph<double>(c, which, x, y, s);
}

int internal_apply(aim_ctx* c, const void* h, void* e, void* heq, int nrhs, int prec, void* stream) {
  BEM_TRY(check_ctx(c, "internal_apply"));
  BEM_TRY(check_prec(prec, "internal_apply"));
  if (!h || (!e && !heq) || nrhs < 1 || h == e || heq == e || heq == h) {
    set_error("internal_apply: bad pointers or nrhs");
    return BEM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  return prec == BEM_C32 ? internal<float>(c, h, e, heq, nrhs, s) : internal<double>(c, h, e, heq, nrhs, s);
}

int aim_internal_tc(aim_ctx* c, const void* h, void* e, void* heq, int nrhs, void* stream) {
  BEM_TRY(check_ctx(c, "aim_internal_tc"));
  if (!h || (!e && !heq) || nrhs < 1 || h == e || heq == e || heq == h) {
    set_error("aim_internal_tc: bad pointers or nrhs");
    return BEM_EINVAL;
  }
  return internal_tc(c, (const float2*)h, (float2*)e, (float2*)heq, nrhs, (cudaStream_t)stream);
}

int aim_conv(aim_ctx* c, const void* sigma, void* phi, int ncomp, int prec, void* stream) {
  BEM_TRY(check_ctx(c, "aim_conv"));
  BEM_TRY(check_prec(prec, "aim_conv"));
  if (!sigma || !phi || ncomp < 1 || ncomp > 4) {
    set_error("aim_conv: bad pointers or ncomp");
    return BEM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  return prec == BEM_C32 ? conv<float>(c, sigma, phi, ncomp, s) : conv<double>(c, sigma, phi, ncomp, s);
}

int bem_blockdiag_gemv(int nblk, const int32_t* n, const void* A, const void* x, void* y, int nrhs,
                       int prec, void* stream) {
  BEM_TRY(check_prec(prec, "bem_blockdiag_gemv"));
  if (nblk < 1 || !n || !A || !x || !y || nrhs < 1 || x == y) {
    set_error("bem_blockdiag_gemv: bad arguments");
    return BEM_EINVAL;
  }
  std::vector<int32_t> nn(n, n + nblk), xo(nblk), ld(nblk);
  std::vector<int64_t> off(nblk);
  int64_t o = 0;
  int32_t xs = 0;
  for (int i = 0; i < nblk; ++i) {
    if (nn[i] < 1) {
      set_error("bem_blockdiag_gemv: block sizes must be positive");
      return BEM_EINVAL;
    }
    ld[i] = (int32_t)round_up(nn[i], 4);
    off[i] = o;
    xo[i] = xs;
    o += (int64_t)nn[i] * ld[i];
    xs += nn[i];
  }
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  // the persistent byte-balanced launch of the context's plain internal products (4-6 CTAs per
  // SM, rows of all blocks cut into equal-byte ranges), with the default shape (no autotuning)
  std::vector<RowInfo> rows;
  std::vector<int2> segs;
  std::vector<int32_t> cseg;
  double ratio = 0;
  const int ncta = nsm * kGemvCtasPerSm;
  build_gemv_plan(nn, off, ld, ncta, &rows, &segs, &cseg, &ratio);
  const size_t b0 = rows.size() * sizeof(RowInfo), b1 = segs.size() * sizeof(int2),
               b2 = cseg.size() * sizeof(int32_t);
  const size_t o1 = round_up(b0, 256), o2 = o1 + round_up(b1, 256);
  char* d = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  BEM_CUDA(cudaMallocAsync((void**)&d, o2 + b2, s));
  BEM_CUDA(cudaMemcpyAsync(d, rows.data(), b0, cudaMemcpyHostToDevice, s));
  BEM_CUDA(cudaMemcpyAsync(d + o1, segs.data(), b1, cudaMemcpyHostToDevice, s));
  BEM_CUDA(cudaMemcpyAsync(d + o2, cseg.data(), b2, cudaMemcpyHostToDevice, s));
  GemvPlan p;
  p.rows = (RowInfo*)d;
  p.segs = (int2*)(d + o1);
  p.cta_seg = (int32_t*)(d + o2);
  p.ncta = ncta;
  p.nrows = (int)rows.size();
  int rc = prec == BEM_C32
               ? run_gemv_plan<float>(p, (const float2*)A, (const float2*)x, (float2*)y, nrhs, xs, nullptr, s)
               : run_gemv_plan<double>(p, (const double2*)A, (const double2*)x, (double2*)y, nrhs, xs, nullptr, s);
  cudaFreeAsync(d, s);
  // the host vectors must outlive the asynchronous copies
  cudaStreamSynchronize(s);
  return rc;
}

int64_t aim_export(const aim_ctx* c, int what, int index, void* out, int64_t cap) {
  if (check_ctx(c, "aim_export") != BEM_OK) return BEM_EINVAL;
  auto copy_dev = [&](const void* src, int64_t bytes, char* dst) -> int {
    cudaError_t e = cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      set_error("aim_export: %s", cudaGetErrorString(e));
      return BEM_ECUDA;
    }
    return BEM_OK;
  };
  if (what == 0 || what == 1) {
    if (index < 0 || index >= c->nobj) {
      set_error("aim_export: object index out of range");
      return BEM_EINVAL;
    }
    const int n = c->e1[index] - c->e0[index], ld = c->zld[index];
    int64_t need = (int64_t)n * n * 16;
    if (!out) return need;
    if (cap < need) { set_error("aim_export: buffer too small"); return BEM_EINVAL; }
    std::vector<double2> tmp((size_t)n * ld);
    const double2* src = (what == 0 ? c->f64.Z : c->f64.Y) + c->zoff[index];
    if (copy_dev(src, (int64_t)tmp.size() * 16, (char*)tmp.data())) return BEM_ECUDA;
    double2* o = (double2*)out;
    for (int r = 0; r < n; ++r)
      for (int k = 0; k < n; ++k) o[(int64_t)r * n + k] = tmp[(int64_t)r * ld + k];
    return need;
  }
  if (what == 2 || what == 3) {
    const std::vector<int64_t>& row = what == 2 ? c->rowA : c->rowP;
    const std::vector<int32_t>& col = what == 2 ? c->colA : c->colP;
    const int64_t nnz = row.back(), nr = (int64_t)row.size();
    int64_t need = nr * 8 + nnz * 4 + nnz * 16;
    if (!out) return need;
    if (cap < need) { set_error("aim_export: buffer too small"); return BEM_EINVAL; }
    char* o = (char*)out;
    memcpy(o, row.data(), nr * 8);
    memcpy(o + nr * 8, col.data(), nnz * 4);
    if (copy_dev(what == 2 ? (const void*)c->f64.LA : (const void*)c->f64.LP, nnz * 16, o + nr * 8 + nnz * 4))
      return BEM_ECUDA;
    return need;
  }
  if (what == 4 || what == 5) {
    int64_t need = what == 4 ? (int64_t)c->ne * 81 * 8 : (int64_t)c->nt * 27 * 8;
    if (!out) return need;
    if (cap < need) { set_error("aim_export: buffer too small"); return BEM_EINVAL; }
    if (copy_dev(what == 4 ? (const void*)c->f64.WA : (const void*)c->f64.WP, need, (char*)out)) return BEM_ECUDA;
    return need;
  }
  if (what == 6) {
    int64_t need = (int64_t)c->anc.size() * 4;
    if (!out) return need;
    if (cap < need) { set_error("aim_export: buffer too small"); return BEM_EINVAL; }
    memcpy(out, c->anc.data(), need);
    return need;
  }
  if (what == 7) {
    int64_t need = (int64_t)c->ne * 6 * 4;
    if (!out) return need;
    if (cap < need) { set_error("aim_export: buffer too small"); return BEM_EINVAL; }
    int32_t* o = (int32_t*)out;
    for (int n = 0; n < c->ne; ++n) {
      o[6 * n] = c->ev[2 * n]; o[6 * n + 1] = c->ev[2 * n + 1];
      o[6 * n + 2] = c->et[2 * n]; o[6 * n + 3] = c->et[2 * n + 1];
      o[6 * n + 4] = c->eopp[2 * n]; o[6 * n + 5] = c->eopp[2 * n + 1];
    }
    return need;
  }
  if (what == 8) {
    int64_t need = (int64_t)c->tune_table.size() * 4;
    if (!out) return need;
    if (cap < need) { set_error("aim_export: buffer too small"); return BEM_EINVAL; }
    memcpy(out, c->tune_table.data(), need);
    return need;
  }
  if (what == 9 || what == 10) {
    const int obj = index >> 1, pass = index & 1;
    if (index < 0 || obj >= c->nobj) {
      set_error("aim_export: object index out of range");
      return BEM_EINVAL;
    }
    const int n = c->e1[obj] - c->e0[obj];
    int64_t need = (int64_t)n * n * 16;
    if (!out) return need;
    if (cap < need) { set_error("aim_export: buffer too small"); return BEM_EINVAL; }
    std::vector<double2> other((size_t)n * n);
    double2* o = (double2*)out;
    BEM_TRY(what == 9 ? export_LK(const_cast<aim_ctx*>(c), obj, pass, o, other.data())
                      : export_LK(const_cast<aim_ctx*>(c), obj, pass, other.data(), o));
    return need;
  }
  set_error("aim_export: unknown item %d", what);
  return BEM_EINVAL;
}

int bem_rhs_plane_wave(aim_ctx* c, const double* pol, const double* khat, void* b, int prec,
                       void* stream) {
  BEM_TRY(check_ctx(c, "bem_rhs_plane_wave"));
  BEM_TRY(check_prec(prec, "bem_rhs_plane_wave"));
  if (!pol || !khat || !b) {
    set_error("bem_rhs_plane_wave: null pointer");
    return BEM_EINVAL;
  }
  return rhs_plane_wave(c, pol, khat, b, prec, (cudaStream_t)stream);
}

int bem_precond_apply(aim_ctx* c, const void* r, void* u, int prec, void* stream) {
  BEM_TRY(check_ctx(c, "bem_precond_apply"));
  BEM_TRY(check_prec(prec, "bem_precond_apply"));
  if (!r || !u || r == u) {
    set_error("bem_precond_apply: r and u must be distinct device pointers");
    return BEM_EINVAL;
  }
  BEM_TRY(setup_precond(c));
  cudaStream_t s = (cudaStream_t)stream;
  return prec == BEM_C32 ? precond_apply<float>(c, r, u, s) : precond_apply<double>(c, r, u, s);
}

int aim_tc_variant(aim_ctx* c, int variant) {
  BEM_TRY(check_ctx(c, "aim_tc_variant"));
  if (variant != 0 && variant != 1) {
    set_error("aim_tc_variant: variant must be 0 or 1");
    return BEM_EINVAL;
  }
  c->tc_variant = variant;
  return BEM_OK;
}

int aim_rows_variant(aim_ctx* c, int variant) {
  BEM_TRY(check_ctx(c, "aim_rows_variant"));
  if (variant < 0 || variant > 2) {
    set_error("aim_rows_variant: variant must be 0, 1 or 2");
    return BEM_EINVAL;
  }
  BEM_CUDA(cudaDeviceSynchronize());
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);  // they hold the old launches
  c->graphs.clear();
  c->rows_variant = variant;
  return BEM_OK;
}

int aim_internal_sparse(aim_ctx* c, int on) {
  BEM_TRY(check_ctx(c, "aim_internal_sparse"));
  if (on != 0 && on != 1) {
    set_error("aim_internal_sparse: on must be 0 or 1");
    return BEM_EINVAL;
  }
  if (on && !c->zsp_ready) {
    set_error("aim_internal_sparse: no sparse internal operator was built for this structure");
    return BEM_EINVAL;
  }
  BEM_CUDA(cudaDeviceSynchronize());
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);  // they hold the old launches
  c->graphs.clear();
  c->zsp_on = on != 0;
  return BEM_OK;
}

int bem_precond_setup(aim_ctx* c, int build_prec) {
  BEM_TRY(check_ctx(c, "bem_precond_setup"));
  BEM_TRY(check_prec(build_prec, "bem_precond_setup"));
  return setup_precond(c, build_prec);
}

int bem_solve(aim_ctx* c, const void* b, void* x, const bem_solve_opts* o, bem_solve_info* info,
              void* stream) {
  BEM_TRY(check_ctx(c, "bem_solve"));
  if (!b || !x || !o || b == x) {
    set_error("bem_solve: bad pointers");
    return BEM_EINVAL;
  }
  if (!(o->tol > 0) || o->restart < 1 || o->restart > 512 || o->max_iter < 1 || o->precond < 0 ||
      o->precond > 2) {
    set_error("bem_solve: bad options");
    return BEM_EINVAL;
  }
  BEM_TRY(check_prec(o->prec_mode, "bem_solve"));
  return gmres_solve(c, b, x, o, info, (cudaStream_t)stream);
}

int bem_solve_batch(aim_ctx* c, const void* b, void* x, int nrhs, const bem_solve_opts* o,
                    bem_solve_info* infos, void* stream) {
  BEM_TRY(check_ctx(c, "bem_solve_batch"));
  if (!b || !x || !o || b == x || nrhs < 1 || nrhs > kMaxBatch) {
    set_error("bem_solve_batch: bad pointers or nrhs outside 1..%d", kMaxBatch);
    return BEM_EINVAL;
  }
  if (!(o->tol > 0) || o->restart < 1 || o->restart > 512 || o->max_iter < 1 || o->precond < 0 ||
      o->precond > 1) {
    set_error("bem_solve_batch: bad options (precond 0 or 1)");
    return BEM_EINVAL;
  }
  BEM_TRY(check_prec(o->prec_mode, "bem_solve_batch"));
  return gmres_solve_batch(c, b, x, nrhs, o, infos, (cudaStream_t)stream);
}

}  // extern "C"
