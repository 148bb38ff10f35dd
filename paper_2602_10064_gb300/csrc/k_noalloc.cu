// tacaw_spectrum_static: the FP32 time transform (the same kernels tacaw_spectrum runs with
// TACAW_DFT_FP32) for callers that cannot allocate device memory.  Its scratch -- the time
// twiddles, the FP64 mean and the residual -- lives in a fixed file-scope device array, so the
// call needs no context and makes no allocation; the caller passes only its input and output.
#include <cuda_runtime.h>

#include "../../include/tacaw.h"
#include "tacaw_internal.cuh"

namespace tacaw {
namespace {

// 16 MiB, held by every device that loads the library until the process exits.
constexpr size_t kStaticScratchBytes = (size_t)16 << 20;
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch in the current context.  The host-side symbol is only
// a stand-in and must never be handed to a kernel.  The address is looked up on every call
// (the lookup allocates nothing): a cached value would go stale when the context it was taken
// in is replaced (cudaDeviceReset, or another context made current on the same device).
cudaError_t scratch_address(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess) return e;
  *out = p;
  return cudaSuccess;
}

// tw[j] = exp(-2 pi i j / F), evaluated in FP64 and rounded to float.
__global__ void k_static_time_twiddles(float2* tw, int64_t F) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < F; j += (int64_t)gridDim.x * blockDim.x) {
    double s, c;
    sincospi(-2.0 * (double)j / (double)F, &s, &c);
    tw[j] = make_float2((float)c, (float)s);
  }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// True for device (or managed) memory of device `dev`, the current device: memory of another
// GPU is rejected rather than handed to the kernels as a peer address.
bool is_device(const void* p, int dev) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace
}  // namespace tacaw

extern "C" int tacaw_spectrum_static(const float* psi_k, int64_t P, int64_t F, int64_t nq, float* S_out,
                                     void* stream) {
  using namespace tacaw;
  if (!psi_k || !S_out || P < 1 || F < 1 || nq < 1) return TACAW_EINVAL;
  if (P > 65535 || F > 65535) return TACAW_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TACAW_ECUDA;
  if (!is_device(psi_k, dev) || !is_device(S_out, dev)) return TACAW_EINVAL;
  const size_t off_mean = align256((size_t)F * sizeof(float2));
  const size_t off_r = align256(off_mean + (size_t)P * nq * sizeof(double2));
  const double need = (double)off_r + (double)P * F * nq * sizeof(float2);
  if (need > (double)kStaticScratchBytes) return TACAW_ETOOBIG;
  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return TACAW_ECUDA;
  unsigned char* b = static_cast<unsigned char*>(base);
  float2* tw = reinterpret_cast<float2*>(b);
  double2* mean = reinterpret_cast<double2*>(b + off_mean);
  float2* r = reinterpret_cast<float2*>(b + off_r);
  const float2* psi = reinterpret_cast<const float2*>(psi_k);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int tb = (int)((F + 255) / 256 < 1024 ? (F + 255) / 256 : 1024);
  k_static_time_twiddles<<<tb, 256, 0, st>>>(tw, F);
  if (cudaGetLastError() != cudaSuccess) return TACAW_ECUDA;
  if (launch_mean_f64(psi, P, F, nq, nullptr, nq, mean, st) != cudaSuccess) return TACAW_ECUDA;
  if (launch_residual_f32(psi, mean, P, F, nq, nullptr, nq, r, st) != cudaSuccess) return TACAW_ECUDA;
  if (launch_dft_fp32(r, tw, P, F, nq, nq, nullptr, S_out, st) != cudaSuccess) return TACAW_ECUDA;
  return TACAW_OK;
}
