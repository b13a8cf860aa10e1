// gs_apply_TH_noalloc: the adjoint apply T^H y of gs_apply_TH without any
// device memory of its own beyond a fixed array that the library reserves at
// load time.
//
// Who needs it: callers that must not allocate device memory while they run --
// for example code that records into a CUDA graph (cudaMalloc is not a stream
// operation and cannot be captured), or a host runtime that hands out device
// memory only from an arena it set up beforehand.  The plan is built earlier,
// where allocation is allowed; this call then allocates nothing.
//
// The spread's per-work-item partial sums (the scratch of the adjoint) go to the
// file-scope array below instead of the plan's own buffer: NOALLOC_SCRATCH_BYTES
// (8 MiB), held on every device that loads the library until the process exits.
// Plans whose partials need more are rejected with GS_EINVAL.  All calls share
// the array: two calls whose GPU work overlaps (two streams, two threads, two
// plans) race on it and give wrong results, so order them on one stream.  The
// array keeps the previous call's contents; the spread kernel writes every
// entry that the reductions of the same call read, so nothing needs clearing.
//
// Set-up: the first call on a device looks up the array's device address with
// cudaGetSymbolAddress while that device is current, and caches it per device;
// make that first call before any stream capture begins.
#include <mutex>

#include "gs_internal.h"

namespace gs {
namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(8) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
void* g_scratch_ptr[MAX_DEVICES] = {};
std::mutex g_scratch_mu;

// device address of the scratch array on the current device (set up once)
gs_status scratch_address(void** out) {
  int dev = 0;
  GS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= MAX_DEVICES) {
    set_error("device ordinal %d outside 0..%d", dev, MAX_DEVICES - 1);
    return GS_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> g(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return GS_OK;
}

template <typename R>
gs_status run(Plan* P, PrecData<R>& D, const C<R>* y, C<R>* x, cudaStream_t st) {
  const size_t need = (size_t)P->nwork * (size_t)D.part_stride * sizeof(C<R>);
  if (need > NOALLOC_SCRATCH_BYTES) {
    set_error("gs_apply_TH_noalloc: this plan's spread scratch needs %zu bytes, more than the %zu-byte fixed array; "
              "use gs_apply_TH",
              need, NOALLOC_SCRATCH_BYTES);
    return GS_EINVAL;
  }
  void* s = nullptr;
  gs_status r = scratch_address(&s);
  if (r != GS_OK) return r;
  return nfft_TH_scratch<R>(P, D, y, x, P->perm, reinterpret_cast<C<R>*>(s), st);
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" gs_status gs_apply_TH_noalloc(gs_plan plan, int precision, const void* y, void* x, void* stream) {
  if (!plan || !x || !y) {
    set_error("plan, x and y must be non-NULL");
    return GS_EINVAL;
  }
  Plan* P = &plan->P;
  if (P->direct) {
    set_error("gs_apply_TH_noalloc: direct-mode plans have no spread scratch; use gs_apply_TH");
    return GS_EUNSUPPORTED;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == GS_FP64) return run<double>(P, P->d, (const double2*)y, (double2*)x, st);
  if (precision == GS_FP32) return run<float>(P, P->f, (const float2*)y, (float2*)x, st);
  set_error("unknown precision %d", precision);
  return GS_EINVAL;
}
