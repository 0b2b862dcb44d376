// panorama_search_noalloc: the search without any device allocation.
//
// Some callers cannot allocate device memory at search time: their device
// memory is entirely owned by another allocator (a framework's caching
// allocator or an inference server's pre-reserved pool, so cudaMalloc would
// fail or fragment it), or they run on latency-critical paths where an
// allocation -- which may synchronize the device or fail when memory is
// fragmented -- is not allowed.  For them the search workspace comes from a
// fixed array in this module's global memory instead of cudaMallocAsync.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library reserves it until the process exits.  In host code its name is
// only a host-side stand-in, so the device address is fetched with
// cudaGetSymbolAddress, once per device, with that device current, on the
// first call made on the device.  All calls share the array, and it keeps
// the last call's contents: the search clears what must start at zero on
// its stream, and calls whose work overlaps on the GPU (different streams,
// or devices sharing a context) race on the array.
#include <mutex>

#include "internal.h"
#include "search.h"

#define PANO_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)

static __device__ __align__(256) unsigned char g_pano_scratch[PANO_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};
}  // namespace

extern "C" int panorama_search_noalloc(const pano_index* idx, const float* queries, int64_t nq,
                                       const int32_t* nprobe, int32_t nprobe_scalar,
                                       const int32_t* k, int32_t k_scalar, int32_t k_max,
                                       int64_t* out_ids, float* out_dists, void* stream) {
  using namespace pano;
  clear_error();
  int dev = 0;
  PANO_CUDA(cudaGetDevice(&dev));
  PANO_CHECK(dev >= 0 && dev < kMaxDevices, PANO_EINVAL, "device ordinal out of range");
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_pano_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
      g_scratch_ptr[dev] = p;
    }
    scratch = g_scratch_ptr[dev];
  }
  return search(idx, queries, nq, nprobe, nprobe_scalar, k, k_scalar, k_max, out_ids, out_dists,
                (cudaStream_t)stream, nullptr, scratch, PANO_NOALLOC_SCRATCH_BYTES);
}
