// ht_compact_noalloc: the stable compaction of ht_compact for callers that
// must not allocate memory (see include/ht.h).  Its only scratch -- the
// identity index list the compaction reads and the word holding its length --
// lives in a fixed array in this file instead of a per-call allocation.
#include "ht_internal.h"
#include "ht_track.h"

// Scratch for up to HT_NOALLOC_MAX_PATHS indices plus one count word.  Every
// GPU that loads the library holds these 16 MiB until the process exits.
static __device__ __align__(256) int32_t ht_noalloc_scratch[HT_NOALLOC_MAX_PATHS + 1];

namespace ht {

// idx[i] = i for i < m; idx[HT_NOALLOC_MAX_PATHS] = m (the length the
// compaction reads).  Rewrites everything the compaction reads, so nothing
// from an earlier call leaks into this one.
__global__ void noalloc_iota_kernel(int32_t* idx, int32_t m) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) idx[i] = i;
  if (blockIdx.x == 0 && threadIdx.x == 0) idx[HT_NOALLOC_MAX_PATHS] = m;
}

// Device address of the scratch array in the current context.  The host-side
// symbol is not a device address; the lookup runs on every call (it allocates
// nothing), so the address stays right after cudaDeviceReset or when another
// context of the same device is made current and the module loads again.
static int noalloc_scratch(int32_t** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, ht_noalloc_scratch);
  if (e != cudaSuccess) return cuda_fail(e, "ht_compact_noalloc: cudaGetSymbolAddress");
  *out = (int32_t*)p;
  return HT_OK;
}

}  // namespace ht

using namespace ht;

extern "C" int ht_compact_noalloc(const int8_t* status, int64_t m, int32_t* path_idx, int32_t* count, void* stream) {
  clear_error();
  if (m < 0 || m > HT_NOALLOC_MAX_PATHS)
    return set_error(HT_EINVAL, "ht_compact_noalloc: m=%lld outside 0..%d (the fixed scratch size)", (long long)m,
                     HT_NOALLOC_MAX_PATHS);
  if (!count || !is_device_ptr(count) ||
      (m > 0 && (!status || !path_idx || !is_device_ptr(status) || !is_device_ptr(path_idx))))
    return set_error(HT_EINVAL, "ht_compact_noalloc: buffers must be device memory");
  int32_t* scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc != HT_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  int blocks = (int)((m + 255) / 256);
  if (blocks < 1) blocks = 1;
  if (blocks > 4096) blocks = 4096;
  noalloc_iota_kernel<<<blocks, 256, 0, st>>>(scratch, (int32_t)m);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "ht_compact_noalloc: launch");
  rc = launch_compact(scratch, scratch + HT_NOALLOC_MAX_PATHS, status, path_idx, count, st);
  if (rc != HT_OK) return rc;
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "ht_compact_noalloc");
  return HT_OK;
}
