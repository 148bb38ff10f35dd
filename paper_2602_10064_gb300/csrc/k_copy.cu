// Device-to-host result copy by the SMs: stores into mapped page-locked host memory.
//
// Measured on GB300 with c4's 8 GiB S (2048 frames x 1024^2): right after a run, one
// copy-engine transfer into page-locked memory ran at 16-31 GB/s (a repeated copy of the same
// buffer reached 193 GB/s only from its second or third pass), while this kernel's stores from
// all SMs ran at 193 GB/s on every call.  A likely cause is the copy engine's address
// translation of the host pages after the run has displaced it; the SM stores keep many
// translations in flight.  Rows of a strided result (a coalesced serving run) are copied by
// the same kernel.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "tacaw_internal.cuh"

namespace tacaw {

namespace {

// rows of `width` elements: row r of dst (pitch dp) = row r of src (pitch sp), pitches in elements
template <class V>
__global__ void __launch_bounds__(256) k_copy_rows(const V* __restrict__ src, int64_t sp, V* __restrict__ dst,
                                                   int64_t dp, int64_t width, int64_t rows) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = blockIdx.y; r < rows; r += gridDim.y) {
    const V* s = src + r * sp;
    V* d = dst + r * dp;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < width; i += stride) d[i] = s[i];
  }
}

dim3 grid_for(int64_t width, int64_t rows) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
  const int64_t ctas = (int64_t)sms * 8;  // about 8 resident CTAs of 256 threads per SM
  const int64_t gy = std::min<int64_t>(std::max<int64_t>(rows, 1), std::min<int64_t>(ctas, 65535));
  const int64_t gx = std::max<int64_t>(1, std::min<int64_t>((width + 255) / 256, ctas / gy));
  return dim3((unsigned)gx, (unsigned)gy);
}

}  // namespace

cudaError_t launch_copy_out(const float* src, int64_t sp, float* dst_mapped, int64_t dp, int64_t width, int64_t rows,
                            cudaStream_t st) {
  if (width <= 0 || rows <= 0) return cudaSuccess;
  const bool v16 = ((uintptr_t)src % 16 == 0) && ((uintptr_t)dst_mapped % 16 == 0) && sp % 4 == 0 && dp % 4 == 0 &&
                   width % 4 == 0;
  if (v16) {
    k_copy_rows<float4><<<grid_for(width / 4, rows), 256, 0, st>>>(reinterpret_cast<const float4*>(src), sp / 4,
                                                                   reinterpret_cast<float4*>(dst_mapped), dp / 4,
                                                                   width / 4, rows);
  } else {
    k_copy_rows<float><<<grid_for(width, rows), 256, 0, st>>>(src, sp, dst_mapped, dp, width, rows);
  }
  return cudaGetLastError();
}

}  // namespace tacaw
