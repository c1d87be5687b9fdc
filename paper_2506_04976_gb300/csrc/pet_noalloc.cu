// Allocation-free variant of pet_rdp for callers that cannot allocate device memory.
//
// pet_rdp obtains the scratch it needs for the FP64 partial sums of the prior's value
// from the stream-ordered allocator.  Some callers may not allocate at all once they are
// running: a reconstruction service whose device memory is fully reserved at start-up,
// or a host framework that owns every device allocation and forbids others.  For them,
// pet_rdp_static keeps its partial sums in a fixed array compiled into this library.
#include <mutex>

#include "pet_internal.cuh"

using namespace petgb;

namespace {

// Scratch for the per-block FP64 partial sums of S(x): PET_RDP_STATIC_MAX_PARTIALS
// doubles (512 KiB), enough for images of up to 65536 stencil blocks of 32x8x4 voxels
// (67 million voxels).  Every GPU that loads the library holds this array until the
// process exits.
__device__ __align__(256) double g_rdp_partials[PET_RDP_STATIC_MAX_PARTIALS];

constexpr int kMaxDevices = 64;
void *g_partials_addr[kMaxDevices] = {nullptr};
std::mutex g_mu;

// Device address of g_rdp_partials on the current device.  In host code the array's
// name only stands for the symbol; its device address comes from the runtime, looked up
// with the device current.  Outside stream capture the lookup is repeated on every call,
// so an address cached before a cudaDeviceReset (which unloads the module) is never
// used again; under capture (where a lookup could trigger module loading) the address
// cached by the last call outside capture on this device is used.
pet_status partials_address(cudaStream_t st, double **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PET_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return PET_ERR_UNSUPPORTED;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return PET_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (cs == cudaStreamCaptureStatusNone) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_rdp_partials) != cudaSuccess || !p) return PET_ERR_CUDA;
    g_partials_addr[dev] = p;
  } else if (!g_partials_addr[dev]) {
    return PET_ERR_STATE;
  }
  *out = static_cast<double *>(g_partials_addr[dev]);
  return PET_OK;
}

}  // namespace

extern "C" pet_status pet_rdp_static(const pet_rdp_params *p, const float *x, float *grad, float *hdiag,
                                     double *val, int accumulate, void *stream) {
  if (!p || !x || p->nx < 1 || p->ny < 1 || p->nz < 1) return PET_ERR_ARG;
  const int nb = rdp_blocks(p->nx, p->ny, p->nz);
  cudaStream_t s = (cudaStream_t)stream;
  double *part = nullptr;
  if (val) {
    if (nb > PET_RDP_STATIC_MAX_PARTIALS) return PET_ERR_UNSUPPORTED;
    const pet_status st = partials_address(s, &part);
    if (st != PET_OK) return st;
  }
  // Every partial that the reduction reads is written by this call's stencil launch, so
  // nothing in the shared array has to be cleared first.
  const RdpArgs a = make_rdp_args(*p);
  cudaError_t e = launch_rdp(a, x, grad, hdiag, part, accumulate & PET_RDP_ACC_GRAD, nullptr, s);
  if (e == cudaSuccess && val) e = launch_reduce_sum(part, nb, val, (accumulate & PET_RDP_ACC_VAL) ? 1 : 0, s);
  return e == cudaSuccess ? PET_OK : PET_ERR_CUDA;
}
