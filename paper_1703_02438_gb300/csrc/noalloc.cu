// noalloc.cu — numarck_compress_noalloc: compression for callers that cannot allocate device
// memory. Some callers cannot call cudaMalloc: a simulation that has already given all of HBM
// to its own pool (in-situ checkpoint compression), code that must not take the implicit device
// synchronisation of cudaMalloc/cudaFree, or plugins whose host application forbids raw CUDA
// allocations. This entry point needs no workspace argument: its scratch memory is one
// file-scope device array of fixed size that is part of the library's device image.
//
// The array lives in this file only. Host code cannot use the array's name as a device address
// (in host code it names a host-side stand-in), so the device address is obtained once per
// device with cudaGetSymbolAddress while that device is current, and then passed on.
#include <mutex>

#include "launch.h"

static __device__ __align__(256) unsigned char g_noalloc_scratch[NUMARCK_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_ptr[kMaxDevices] = {nullptr};
bool g_dirty[kMaxDevices] = {false};

}  // namespace

extern "C" int numarck_compress_noalloc(const void* prev, const void* cur, int64_t n,
                                        const numarck_params* p, void* blob, size_t blob_cap,
                                        numarck_stream_t stream) {
  nmk::NvtxRange nvtx_("numarck_compress_noalloc");
  const size_t need = numarck_workspace_bytes(n, p);
  if (need == 0) return NUMARCK_ERR_INVALID_ARG;
  if (need > (size_t)NUMARCK_NOALLOC_SCRATCH_BYTES) return NUMARCK_ERR_CAPACITY;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return NUMARCK_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return NUMARCK_ERR_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  void* ws = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_ptr[dev] == nullptr || g_dirty[dev]) {
      void* ptr = nullptr;
      if (g_ptr[dev] == nullptr) {
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr)
          return NUMARCK_ERR_CUDA;
      } else {
        ptr = g_ptr[dev];
      }
      // The compression kernels expect a zero-filled workspace; clear all of it on first use
      // (and after a failed call, whose kernels may have left partial state behind).
      if (cudaMemsetAsync(ptr, 0, (size_t)NUMARCK_NOALLOC_SCRATCH_BYTES, s) != cudaSuccess)
        return NUMARCK_ERR_CUDA;
      g_ptr[dev] = ptr;
      g_dirty[dev] = false;
    }
    ws = g_ptr[dev];
  }
  // The 256-byte control block (bin-range keys, tile counter) must start at zero; a finished
  // call leaves it so, and clearing it here costs one small memset on the stream.
  if (cudaMemsetAsync(ws, 0, 256, s) != cudaSuccess) return NUMARCK_ERR_CUDA;
  const int rc = numarck_compress(prev, cur, n, p, blob, blob_cap, ws,
                                  (size_t)NUMARCK_NOALLOC_SCRATCH_BYTES, stream);
  if (rc == NUMARCK_ERR_CUDA) {
    std::lock_guard<std::mutex> lock(g_mu);
    g_dirty[dev] = true;
  }
  return rc;
}
