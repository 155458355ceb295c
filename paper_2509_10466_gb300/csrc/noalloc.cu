// Allocation-free variant of the hole-L1 loss.
//
// inpaint_l1_hole_loss keeps its per-block partial sums in the context's workspace,
// which the library grows with cudaMalloc on demand.  Some callers cannot allow that:
// a process whose device memory is owned by another allocator (a framework's caching
// pool) where a raw cudaMalloc may fail or fragment, a per-frame real-time loop where
// cudaMalloc/cudaFree would synchronize the device and stall the other streams, or a
// deployment that forbids device allocation after start-up.  This variant needs no
// context and keeps its scratch in a fixed array that lives in the library's module,
// so it never allocates.
#include <mutex>

#include "common.cuh"

namespace inpaint {

namespace {

constexpr int MAX_PARTIALS = INPAINT_L1_NOALLOC_MAX_PIXELS / 4096;  // one partial per 4096 pixels

// Scratch shared by every call on a device: MAX_PARTIALS float sums, then MAX_PARTIALS
// unsigned hole counts (32 KiB).  Held by every device that loads the library.
static __device__ __align__(256) unsigned char g_l1_scratch[MAX_PARTIALS * (sizeof(float) + sizeof(unsigned))];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_addr[MAX_DEVICES] = {};

// Device address of g_l1_scratch in the current device's context.  It is looked up on
// every call (a runtime lookup, no allocation), so a context that was destroyed and
// created again (cudaDeviceReset) never leaves a stale address behind.  While `st` is
// capturing, the lookup is skipped and the address found by the last call on this device
// is used.
int scratch_address(cudaStream_t st, void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return record_cuda_error(e);
  if (dev < 0 || dev >= MAX_DEVICES) return INPAINT_E_INVAL;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(st, &cap);
  if (e != cudaSuccess) return record_cuda_error(e);
  std::lock_guard<std::mutex> lock(g_mu);
  if (cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_l1_scratch);
    if (e != cudaSuccess) return record_cuda_error(e);
    if (!p) return INPAINT_E_CUDA;
    g_addr[dev] = p;
  } else if (!g_addr[dev]) {
    return INPAINT_E_STATE;  // no call on this device before the capture began
  }
  *out = g_addr[dev];
  return INPAINT_OK;
}

}  // namespace

}  // namespace inpaint

using namespace inpaint;

extern "C" int inpaint_l1_hole_loss_noalloc(const float* out, const float* target, const uint8_t* hole, int B, int H,
                                            int W, float* loss, float* grad, void* stream) {
  if (!out || !target || !hole || !loss || B < 1 || H < 1 || W < 1) return INPAINT_E_INVAL;
  if ((unsigned long long)B * H * W > (unsigned long long)INPAINT_L1_NOALLOC_MAX_PIXELS) return INPAINT_E_INVAL;
  void* base = nullptr;
  const int rc = scratch_address((cudaStream_t)stream, &base);
  if (rc != INPAINT_OK) return rc;
  float* partials = static_cast<float*>(base);
  unsigned* counts = reinterpret_cast<unsigned*>(static_cast<unsigned char*>(base) + MAX_PARTIALS * sizeof(float));
  // the partial pass writes every slot it later reads, so stale contents never leak in
  return record_cuda_error(
      launch_l1_hole_loss(out, target, hole, B, H, W, partials, counts, loss, grad, (cudaStream_t)stream));
}
