// Host-to-device ingest of measured data with a kernel: SM loads of page-locked host
// memory through the unified address space (over the CPU-GPU link), 16-byte vectors,
// four loads in flight per thread, stored coalesced into device memory.  Loads and stores
// carry the streaming cache hint (evict first): the data are touched once here and not
// again until a later kernel, so they should not push a concurrently running kernel's
// working set out of L2.
#include <algorithm>

#include "pet_internal.cuh"

namespace petgb {

namespace {

__global__ void __launch_bounds__(512) k_copy_pinned(const uint4 *__restrict__ src, uint4 *__restrict__ dst,
                                                     size_t n) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n; i += 4 * stride) {
    const uint4 a = __ldcs(src + i), b = __ldcs(src + i + stride), c = __ldcs(src + i + 2 * stride),
                d = __ldcs(src + i + 3 * stride);
    __stcs(dst + i, a);
    __stcs(dst + i + stride, b);
    __stcs(dst + i + 2 * stride, c);
    __stcs(dst + i + 3 * stride, d);
  }
  for (; i < n; i += stride) __stcs(dst + i, __ldcs(src + i));
}

__global__ void k_copy_tail(const unsigned char *__restrict__ src, unsigned char *__restrict__ dst, int n) {
  if ((int)threadIdx.x < n) dst[threadIdx.x] = src[threadIdx.x];
}

}  // namespace

}  // namespace petgb

using namespace petgb;

extern "C" pet_status pet_copy_to_device(void *dst, const void *src, size_t bytes, int max_blocks, void *stream) {
  if (!dst || !src || max_blocks < 0) return PET_ERR_ARG;
  if (bytes == 0) return PET_OK;
  if (((uintptr_t)dst & 15) || ((uintptr_t)src & 15)) return PET_ERR_ARG;
  cudaPointerAttributes as{}, ad{};
  if (cudaPointerGetAttributes(&as, src) != cudaSuccess || cudaPointerGetAttributes(&ad, dst) != cudaSuccess) {
    cudaGetLastError();
    return PET_ERR_ARG;
  }
  if (as.type != cudaMemoryTypeHost || !as.devicePointer || ad.type != cudaMemoryTypeDevice) return PET_ERR_ARG;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PET_ERR_CUDA;
  if (ad.device != dev) return PET_ERR_ARG;  // dst on another device than the current one
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n16 = bytes / 16;
  const int tail = (int)(bytes % 16);
  const unsigned char *s = static_cast<const unsigned char *>(as.devicePointer);
  unsigned char *d = static_cast<unsigned char *>(dst);
  if (n16) {
    const size_t want = (n16 + 511) / 512;
    const size_t cap = max_blocks > 0 ? (size_t)max_blocks : (size_t)4 * nsm;
    const int grid = (int)std::min<size_t>(want, cap);
    k_copy_pinned<<<grid, 512, 0, st>>>(reinterpret_cast<const uint4 *>(s), reinterpret_cast<uint4 *>(d), n16);
    note_launch();
  }
  if (tail) {
    k_copy_tail<<<1, 32, 0, st>>>(s + n16 * 16, d + n16 * 16, tail);
    note_launch();
  }
  return cudaGetLastError() == cudaSuccess ? PET_OK : PET_ERR_CUDA;
}
