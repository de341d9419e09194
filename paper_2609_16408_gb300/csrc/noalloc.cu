// Galerkin initial guesses without any device allocation.
//
// Some callers cannot allocate device memory from inside their own code: a host application
// that has handed all device memory to its own pool allocator, a plug-in that runs inside
// another framework's allocation policy, or a code path that must stay free of cudaMalloc /
// cudaFree because those calls synchronise the whole device.  For them this file provides
// rpa_galerkin_noalloc: the FP64 occupied-space projection of rpa_galerkin, computed with the
// caller's input and output buffers and a fixed scratch area that lives in a file-scope
// __device__ array.  Every GPU that loads this library holds that array (kScratchBytes) until
// the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "cocg.cuh"

namespace {

constexpr size_t kScratchBytes = (size_t)8 << 20;  // 8 MiB

// Scratch of rpa_galerkin_noalloc: Gram partial sums (nchunk x ns x ns doubles) followed by
// the coefficient matrix (ns x ns complex doubles).  Shared by every call on a device.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_scratch on the current device.  In host code the symbol itself is
// only a host-side stand-in and must not be passed to a kernel.  The address is looked up
// again on every call made outside a stream capture (so that a context torn down and
// re-created since the last call cannot leave a stale address behind); during a capture,
// where the lookup may not be legal, the address cached by the last uncaptured call on this
// device is used, and a capture with no cached address is refused.
cudaError_t scratch_address(cudaStream_t s, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  } else if (!g_scratch_addr[dev]) {
    return cudaErrorStreamCaptureUnsupported;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

int chunks_for(long long nd) {
  const long long c = (nd + 4095) / 4096;
  return (int)(c < 1 ? 1 : (c > 256 ? 256 : c));
}

}  // namespace

extern "C" rpa_status rpa_galerkin_noalloc(long long nd, int ns, const double* psi,
                                           const double* eps, double dV, int count,
                                           const double* omega, const double* u, double* x0,
                                           void* cuda_stream) {
  if (nd < 1 || nd >= (1LL << 31) || ns < 1 || ns > 1024 || count < 0 || !(dV > 0.0))
    return RPA_EINVAL;
  // the projection kernels take point tiles of 64 along gridDim.x (< 2^31 tiles) and state
  // tiles of 32 along gridDim.y (<= 32 here): every nd and ns accepted above fits
  const int nchunk = chunks_for(nd);
  // the coefficient matrix starts on a 256-byte boundary after the Gram partials
  const size_t gram_bytes = (((size_t)nchunk * ns * ns * sizeof(double)) + 255) & ~(size_t)255;
  const size_t coef_bytes = (size_t)ns * ns * sizeof(rpa::cpx<double>);
  if (gram_bytes + coef_bytes > kScratchBytes) return RPA_EINVAL;  // beyond the scratch size
  if (count == 0) return RPA_OK;
  if (!psi || !eps || !omega || !u || !x0) return RPA_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  void* base = nullptr;
  if (scratch_address(s, &base) != cudaSuccess) return RPA_ECUDA;
  double* gpart = static_cast<double*>(base);
  rpa::cpx<double>* cmat =
      reinterpret_cast<rpa::cpx<double>*>(static_cast<unsigned char*>(base) + gram_bytes);
  // one probe at a time: the Gram kernel writes every partial it later sums, and the
  // coefficient kernel writes the whole matrix, so nothing in the scratch needs clearing
  for (int b = 0; b < count; ++b) {
    cudaError_t e = rpa::galerkin_guess<double>(
        nd, ns, 1, psi, eps, omega + b, u + (long long)b * nd, nullptr, dV, gpart, nchunk, cmat,
        reinterpret_cast<rpa::cpx<double>*>(x0) + (long long)b * ns * nd, s);
    if (e != cudaSuccess) return RPA_ECUDA;
  }
  return RPA_OK;
}
