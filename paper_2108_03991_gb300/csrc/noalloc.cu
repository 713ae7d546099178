// bem_blockdiag_gemv_noalloc: the block-diagonal GEMV for callers that cannot allocate device
// memory. The paper has no counterpart; it is a service of this library.
//
// Who needs it: bem_blockdiag_gemv builds its row-panel work list in device memory that it
// allocates (cudaMallocAsync) on every call. Some callers cannot allow that: programs whose
// device memory is owned entirely by another allocator (a framework's caching allocator that
// reserved the whole GPU, so a further cudaMalloc fails or fragments it), and real-time loops
// whose rules forbid any allocation once they are running. This entry point allocates nothing:
// its work list lives in a fixed device array compiled into the library.
//
// The scratch: kNoAllocMaxTasks tasks (32 bytes each, 1 MiB) in a file-scope __device__ array.
// Every GPU that loads the library holds it until the process exits. In host code the array's
// name is only a host-side stand-in, so every call looks up its device address on the current
// device with cudaGetSymbolAddress (cheap next to the copy; nothing is cached, so a device reset
// that reloads the module leaves no stale address) and passes that address to the kernel. Every
// call overwrites the entries it uses; nothing has to start at zero. All calls share the one
// array: calls whose GPU work overlaps (different streams, or different host threads) race on it
// and must be ordered by the caller.
//
// The work list reaches the array by a copy from a static host array. A CUDA graph captured
// around the call would record that copy and read the host array again at every replay, after
// later calls may have rewritten it, and then run another call's list against this call's
// matrices. So the call refuses to run while its stream is being captured.
#include <mutex>

#include "common.cuh"

namespace bem {

constexpr int kNoAllocMaxTasks = 32768;
constexpr int kNoAllocRows = 16;  // rows per task

static __device__ __align__(256) GemvTask g_noalloc_tasks[kNoAllocMaxTasks];

static std::mutex g_noalloc_mu;
static GemvTask g_noalloc_host[kNoAllocMaxTasks];  // host staging (static storage, no heap)

// Device address of the scratch array on the current device (looked up on every call).
static int noalloc_scratch(GemvTask** out) {
  void* p = nullptr;
  BEM_CUDA(cudaGetSymbolAddress(&p, g_noalloc_tasks));
  *out = static_cast<GemvTask*>(p);
  return BEM_OK;
}

}  // namespace bem

using namespace bem;

extern "C" int bem_blockdiag_gemv_noalloc(int nblk, const int32_t* n, const void* A, const void* x,
                                          void* y, int nrhs, int prec, void* stream) {
  if (prec != BEM_C32 && prec != BEM_C64) {
    set_error("bem_blockdiag_gemv_noalloc: prec must be BEM_C32 or BEM_C64");
    return BEM_EINVAL;
  }
  if (nblk < 1 || !n || !A || !x || !y || nrhs < 1 || x == y) {
    set_error("bem_blockdiag_gemv_noalloc: bad arguments");
    return BEM_EINVAL;
  }
  int64_t ntask = 0, nsum = 0;
  for (int i = 0; i < nblk; ++i) {
    if (n[i] < 1) {
      set_error("bem_blockdiag_gemv_noalloc: block sizes must be positive");
      return BEM_EINVAL;
    }
    ntask += (n[i] + kNoAllocRows - 1) / kNoAllocRows;
    nsum += n[i];
  }
  if (ntask > kNoAllocMaxTasks || nsum > INT32_MAX) {
    set_error("bem_blockdiag_gemv_noalloc: %lld row panels of %d rows exceed the fixed scratch of "
              "%d (at most %d rows in all)", (long long)ntask, kNoAllocRows, kNoAllocMaxTasks,
              kNoAllocMaxTasks * kNoAllocRows);
    return BEM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t ce = cudaStreamIsCapturing(s, &cap);
  if (ce != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    if (ce != cudaSuccess) cudaGetLastError();
    set_error("bem_blockdiag_gemv_noalloc: the stream is being captured into a CUDA graph; this "
              "call cannot be captured (its work list is copied from a shared host array)");
    return BEM_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  GemvTask* d_tasks = nullptr;
  BEM_TRY(noalloc_scratch(&d_tasks));
  int64_t off = 0;
  int32_t xoff = 0;
  int k = 0;
  for (int i = 0; i < nblk; ++i) {
    const int32_t ld = (int32_t)round_up(n[i], 4);
    for (int r0 = 0; r0 < n[i]; r0 += kNoAllocRows) {
      GemvTask& t = g_noalloc_host[k++];
      t.aoff = off;
      t.xoff = xoff;
      t.n = n[i];
      t.ld = ld;
      t.row0 = r0;
      t.nrows = std::min(kNoAllocRows, n[i] - r0);
      t.sel = 0;
    }
    off += (int64_t)n[i] * ld;
    xoff += n[i];
  }
  // From pageable host memory the copy returns once the source has been staged, so the host
  // buffer may be reused as soon as the lock is released.
  BEM_CUDA(cudaMemcpyAsync(d_tasks, g_noalloc_host, (size_t)k * sizeof(GemvTask),
                           cudaMemcpyHostToDevice, s));
  return prec == BEM_C32
             ? run_gemv<float>(d_tasks, k, (const float2*)A, (const float2*)x, (float2*)y, nrhs,
                               xoff, nullptr, s)
             : run_gemv<double>(d_tasks, k, (const double2*)A, (const double2*)x, (double2*)y,
                                nrhs, xoff, nullptr, s);
}
