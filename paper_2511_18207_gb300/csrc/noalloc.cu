// hausdorff_exact_noalloc: the FP32 exact Hausdorff distance for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc or hand the library a workspace: code
// that runs while a stream is being captured into a CUDA graph by someone
// else (allocation would break or serialise the capture), plugins and
// callbacks inside a host framework that owns the device allocator, and
// real-time or safety-qualified programs that forbid allocation after
// start-up. For them this entry point computes the same result as
// hausdorff_exact(..., PROHD_FP32, ...) using a fixed scratch array that is
// part of the library image instead of a caller workspace.
//
// The scratch is a file-scope __device__ array of kNoAllocScratchBytes
// (2 MiB). Every GPU that loads the library holds one copy of it until the
// process exits. It must hold the FP32 path's buffers (one 8-byte packed
// minimum per point of A and of B, plus a few scalars), which limits
// nA + nB to about 262,000 points; larger inputs are rejected with
// PROHD_EINVAL and a message.
//
// Host code cannot use the array's name as a device address (on the host it
// is only a stand-in symbol), so the first call on each device, with that
// device current, looks the address up with cudaGetSymbolAddress and caches
// it together with the unique id of the current context. Make that first
// call before any stream capture begins. cudaDeviceReset destroys the
// context and the module that holds the array; the next call sees a new
// context id and looks the address up again (again: not under capture).
//
// All calls share the one array, and a call leaves its contents behind; the
// FP32 path resets everything it reads (status, sizes, per-point minima)
// before use. Calls whose GPU work overlaps (different streams, or
// concurrent host threads) race on the array and produce wrong results:
// serialise them.
#include <mutex>

#include "internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(2) << 20;
constexpr int kNoAllocMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};
unsigned long long g_noalloc_ctx_id[kNoAllocMaxDevices] = {};

// Unique id of the calling thread's current context (0 if none or if the
// driver lacks the calls). Ids are never reused within a process, unlike
// context handles, so a reset device is recognised.
unsigned long long current_context_id() {
  typedef CUresult (*GetCurrentFn)(CUcontext*);
  typedef CUresult (*GetIdFn)(CUcontext, unsigned long long*);
  static GetCurrentFn get_current = nullptr;
  static GetIdFn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetIdFn>(f);
    looked_up = true;
  }
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (get_current && get_id && get_current(&c) == CUDA_SUCCESS && c && get_id(c, &id) == CUDA_SUCCESS) return id;
  return 0;
}

}  // namespace

extern "C" prohd_status hausdorff_exact_noalloc(prohd_ctx* ctx, const float* A, int64_t nA, const float* B,
                                                int64_t nB, int D, prohd_hd_result* out, void* stream) {
  if (!ctx) return PROHD_EINVAL;
  if (nA < 1 || nB < 1 || D < 1 || D > 1024) {
    ctx->err = "hausdorff_exact_noalloc: set sizes must be >= 1 and D in [1, 1024]";
    return PROHD_EINVAL;
  }
  const size_t need = hausdorff_exact_workspace_size(nA, nB, D, PROHD_FP32);
  if (need == 0 || need > kNoAllocScratchBytes) {
    ctx->err = "hausdorff_exact_noalloc: nA + nB exceeds the fixed 2 MiB scratch (about 262,000 points); "
               "use hausdorff_exact with a workspace";
    return PROHD_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
    ctx->err = "hausdorff_exact_noalloc: no usable current device";
    return PROHD_ECUDA;
  }
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    const unsigned long long cid = current_context_id();
    if (!g_noalloc_ptr[dev] || cid != g_noalloc_ctx_id[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        ctx->err = std::string("hausdorff_exact_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
        return PROHD_ECUDA;
      }
      g_noalloc_ptr[dev] = p;
      // the lookup itself makes the primary context current if none was
      g_noalloc_ctx_id[dev] = current_context_id();
    }
    scratch = g_noalloc_ptr[dev];
  }
  return hausdorff_exact(ctx, A, nA, B, nB, D, PROHD_FP32, out, scratch, kNoAllocScratchBytes, stream);
}
