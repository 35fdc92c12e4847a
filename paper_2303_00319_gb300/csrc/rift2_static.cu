// rift2_detect_static: keypoint detection that allocates nothing.
//
// Some callers cannot call cudaMalloc: code that runs under a framework's caching
// allocator which owns the device memory budget, real-time loops where the implicit
// device synchronisation of cudaMalloc / cudaFree would stall other streams, and hosts
// that plan every byte of device memory up front.  This entry point serves them: its only
// scratch memory is a file-scope __device__ array of fixed size (every GPU that loads the
// library holds it until the process exits), and it creates no context, plan or table.
#include <cuda.h>

#include <cstdio>
#include <mutex>

#include "kernels.h"

namespace {

using namespace rift2;

// Scratch layout: [0, 16) min / max bits of the moment map, [16, 20) candidate count,
// [256, ...) candidate keys, room for RIFT2_STATIC_MAX_CANDIDATES of them.
constexpr size_t kCandOffset = 256;
constexpr size_t kScratchBytes =
    kCandOffset + (size_t)RIFT2_STATIC_MAX_CANDIDATES * sizeof(unsigned long long);

__device__ __align__(256) unsigned char g_detect_scratch[kScratchBytes];

// Device address of g_detect_scratch, looked up with the device current.  (In host code
// the symbol's name is only a host-side stand-in, not a device address.)  The address
// belongs to the device's primary context: it is kept together with that context's
// handle and looked up again when the current context is a different one (after a
// device reset the module is loaded anew and the old address is stale).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};
CUcontext g_ctx[kMaxDevices] = {};
using CtxGetCurrent = CUresult (*)(CUcontext*);
CtxGetCurrent g_ctx_get = nullptr;

int scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return RIFT2_E_INVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ctx_get) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault,
                                         &qr) != cudaSuccess ||
        qr != cudaDriverEntryPointSuccess || !fn) {
      fprintf(stderr, "rift2_detect_static: cuCtxGetCurrent is unavailable\n");
      return RIFT2_E_CUDA;
    }
    g_ctx_get = reinterpret_cast<CtxGetCurrent>(fn);
  }
  // Before the runtime's first context-using call on this thread no context may be
  // current yet (cur == NULL); cudaGetSymbolAddress makes the primary context current,
  // and the handle is read again after it.
  CUcontext cur = nullptr;
  if (g_ctx_get(&cur) != CUDA_SUCCESS) cur = nullptr;
  if (!g_addr[dev] || !cur || cur != g_ctx[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_detect_scratch);
    if (e != cudaSuccess || !p) {
      fprintf(stderr, "rift2_detect_static: cudaGetSymbolAddress failed: %s\n",
              cudaGetErrorString(e));
      return RIFT2_E_CUDA;
    }
    if (g_ctx_get(&cur) != CUDA_SUCCESS) cur = nullptr;
    g_addr[dev] = p;
    g_ctx[dev] = cur;
  }
  *out = g_addr[dev];
  return RIFT2_OK;
}

// True iff p is device memory (or managed memory) that device `dev` owns.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

extern "C" int rift2_detect_static(const rift2_params* params, const float* moment, int height,
                                   int width, rift2_features* out, void* stream) {
  if (!moment || !out || height < 16 || width < 16) return RIFT2_E_INVAL;
  if ((long long)((height + 1) / 2) * ((width + 1) / 2) > RIFT2_STATIC_MAX_CANDIDATES) {
    fprintf(stderr,
            "rift2_detect_static: a %d x %d map needs more than the %d candidate slots of the "
            "static scratch array\n",
            height, width, RIFT2_STATIC_MAX_CANDIDATES);
    return RIFT2_E_CAPACITY;
  }
  rift2_params p;
  rift2_default_params(&p);
  if (params) p = *params;
  if (p.n_scales != NS || p.n_orient != NO || p.patch != PATCH || p.cells != CELLS)
    return RIFT2_E_UNIMPL;
  if (p.max_keypoints < 1 || p.max_keypoints > 16384 || p.fast_arc < 1 || p.fast_arc > 16 ||
      !(p.fast_threshold >= 0))
    return RIFT2_E_INVAL;
  if (!out->kp_xy || !out->kp_score || !out->counts) return RIFT2_E_INVAL;
  if (out->cap_kp < p.max_keypoints) return RIFT2_E_CAPACITY;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RIFT2_E_CUDA;
  // every buffer must live on the current device: the kernels run there
  if (!on_device(moment, dev) || !on_device(out->kp_xy, dev) || !on_device(out->kp_score, dev) ||
      !on_device(out->counts, dev)) {
    fprintf(stderr, "rift2_detect_static: the map and the outputs must be device memory of "
                    "the current device (%d)\n", dev);
    return RIFT2_E_INVAL;
  }
  void* base = nullptr;
  int rc = scratch_address(dev, &base);
  if (rc) return rc;
  KParams kp{};
  derive_kparams(p, kp);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned* minmax = static_cast<unsigned*>(base);
  unsigned* ccount = minmax + 4;
  unsigned long long* cand =
      reinterpret_cast<unsigned long long*>(static_cast<char*>(base) + kCandOffset);
  // the array keeps the previous call's contents: reset what must start from zero
  launch_init_detect(minmax, ccount, 1, st);
  launch_minmax(moment, 1, (long long)height * width, minmax, st);
  FeatPtrs fp{};
  fp.kp_xy[0] = out->kp_xy;
  fp.kp_score[0] = out->kp_score;
  fp.counts[0] = out->counts;
  DetectWs dw{minmax, cand, ccount, RIFT2_STATIC_MAX_CANDIDATES, nullptr};
  Group gr{};
  gr.n = 1;
  gr.H[0] = height;
  gr.W[0] = width;
  if (launch_detect(moment, gr, kp, dw, fp, st) != cudaSuccess) return RIFT2_E_CUDA;
  return RIFT2_OK;
}
