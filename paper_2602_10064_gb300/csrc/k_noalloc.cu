// tacaw_spectrum_static: the FP32 time transform (the same kernels tacaw_spectrum runs with
// TACAW_DFT_FP32) for callers that cannot allocate device memory.  Its scratch -- the time
// twiddles, the FP64 mean and the residual -- lives in a fixed file-scope device array, so the
// call needs no context and makes no allocation; the caller passes only its input and output.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/tacaw.h"
#include "tacaw_internal.cuh"

namespace tacaw {
namespace {

// 16 MiB, held by every device that loads the library until the process exits.
constexpr size_t kStaticScratchBytes = (size_t)16 << 20;
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 128;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device (looked up once per device: the
// host-side symbol is only a stand-in and must never be handed to a kernel).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
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

bool is_device(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace tacaw

extern "C" int tacaw_spectrum_static(const float* psi_k, int64_t P, int64_t F, int64_t nq, float* S_out,
                                     void* stream) {
  using namespace tacaw;
  if (!psi_k || !S_out || P < 1 || F < 1 || nq < 1) return TACAW_EINVAL;
  if (P > 65535 || F > 65535) return TACAW_EINVAL;
  if (!is_device(psi_k) || !is_device(S_out)) return TACAW_EINVAL;
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
