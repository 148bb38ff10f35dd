// TACAW accessors (Methods, "Data Structure Design": spectral diffraction, dispersion,
// spectrum image) and FP64 trajectory averaging (Supplement, "Sampling Considerations").
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "tacaw_api_internal.h"
#include "tacaw_internal.cuh"

namespace tacaw {

__global__ void k_spectral_diffraction(const float* __restrict__ S, int64_t P, int64_t F, int64_t nq, int m, int mn,
                                       int fold, float* __restrict__ out) {
  const int64_t n = P * nq;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = i / nq, q = i - p * nq;
    float v = S[((size_t)p * F + m) * nq + q];
    if (fold && mn != m) v += S[((size_t)p * F + mn) * nq + q];
    out[i] = v;
  }
}

cudaError_t launch_spectral_diffraction(const float* S, int64_t P, int64_t F, int64_t nq, int m, int fold,
                                        float* out, cudaStream_t st) {
  const int mn = (int)((F - m) % F);
  const int64_t n = P * nq;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 65535);
  k_spectral_diffraction<<<blocks, 256, 0, st>>>(S, P, F, nq, m, mn, fold, out);
  return cudaGetLastError();
}

// out[p][m][i]: bilinear interpolation at fractional grid indices (u_i, v_i) = (kx Lx, ky Ly),
// periodic wrap; index decisions and weights in FP64.
__global__ void k_dispersion(const float* __restrict__ S, int64_t P, int64_t F, int ny, int nx,
                             const double* __restrict__ u, const double* __restrict__ v, int npts,
                             float* __restrict__ out) {
  const int64_t n = P * F * npts;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pm = idx / npts;
    const int i = (int)(idx - pm * npts);
    const float* plane = S + (size_t)pm * ny * nx;
    const double uu = u[i], vv = v[i], u0 = floor(uu), v0 = floor(vv), fu = uu - u0, fv = vv - v0;
    const long long iu = (((long long)u0 % nx) + nx) % nx, iv = (((long long)v0 % ny) + ny) % ny;
    const long long iu1 = (iu + 1) % nx, iv1 = (iv + 1) % ny;
    const double s00 = plane[iv * nx + iu], s01 = plane[iv * nx + iu1];
    const double s10 = plane[iv1 * nx + iu], s11 = plane[iv1 * nx + iu1];
    out[idx] = (float)((1 - fv) * ((1 - fu) * s00 + fu * s01) + fv * ((1 - fu) * s10 + fu * s11));
  }
}

cudaError_t launch_dispersion(const float* S, int64_t P, int64_t F, int ny, int nx, const double* u,
                              const double* v, int npts, float* out, cudaStream_t st) {
  const int64_t n = P * F * npts;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 65535);
  k_dispersion<<<blocks, 256, 0, st>>>(S, P, F, ny, nx, u, v, npts, out);
  return cudaGetLastError();
}

__global__ void k_accumulate(const float* __restrict__ S, int64_t n, double w, double* __restrict__ acc) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc[i] += w * (double)S[i];
}

cudaError_t launch_accumulate(const float* S, int64_t n, double weight, double* acc, cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 65535);
  k_accumulate<<<blocks, 256, 0, st>>>(S, n, weight, acc);
  return cudaGetLastError();
}

namespace {
bool on_device(const void* p) {
  cudaPointerAttributes a{};
  if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}
}  // namespace

}  // namespace tacaw

using namespace tacaw;

extern "C" {

int tacaw_spectral_diffraction(tacaw_ctx* ctx, const float* S, int64_t P, int64_t F, int64_t nq, double dt_fs,
                               double f_thz, int32_t fold, float* out, void* stream) {
  if (!ctx) return TACAW_EINVAL;
  if (P < 1 || F < 1 || nq < 1 || !(dt_fs > 0.0)) return set_err(ctx, TACAW_EINVAL, "bad sizes or dt");
  if (!on_device(S) || !on_device(out)) return set_err(ctx, TACAW_EINVAL, "S and out must be device pointers");
  long long m = llround(f_thz * (double)F * dt_fs * 1e-3) % F;
  if (m < 0) m += F;
  const cudaError_t e = launch_spectral_diffraction(S, P, F, nq, (int)m, fold, out, (cudaStream_t)stream);
  return e == cudaSuccess ? TACAW_OK : cuda_err(ctx, e, "k_spectral_diffraction");
}

int tacaw_dispersion(tacaw_ctx* ctx, const float* S, int64_t P, int64_t F, int32_t ny, int32_t nx, double Lx,
                     double Ly, const double* kx, const double* ky, int32_t npts, float* out, void* stream) {
  if (!ctx) return TACAW_EINVAL;
  if (P < 1 || F < 1 || ny < 1 || nx < 1 || npts < 1 || !kx || !ky || !(Lx > 0) || !(Ly > 0))
    return set_err(ctx, TACAW_EINVAL, "bad dispersion arguments");
  if (!on_device(S) || !on_device(out)) return set_err(ctx, TACAW_EINVAL, "S and out must be device pointers");
  std::vector<double> uv(2 * (size_t)npts);
  for (int i = 0; i < npts; ++i) {
    uv[i] = kx[i] * Lx;
    uv[npts + i] = ky[i] * Ly;
  }
  cudaStream_t st = (cudaStream_t)stream;
  Scratch sc(st);
  double* d;
  cudaError_t e = sc.get(&d, uv.size());
  if (e == cudaSuccess) e = cudaMemcpyAsync(d, uv.data(), sizeof(double) * uv.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = launch_dispersion(S, P, F, ny, nx, d, d + npts, npts, out, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // uv is host-local
  return e == cudaSuccess ? TACAW_OK : cuda_err(ctx, e, "tacaw_dispersion");
}

int tacaw_accumulate(tacaw_ctx* ctx, const float* S, int64_t n, double weight, double* acc, void* stream) {
  if (!ctx) return TACAW_EINVAL;
  if (n < 1) return set_err(ctx, TACAW_EINVAL, "n must be >= 1");
  if (!on_device(S) || !on_device(acc)) return set_err(ctx, TACAW_EINVAL, "S and acc must be device pointers");
  const cudaError_t e = launch_accumulate(S, n, weight, acc, (cudaStream_t)stream);
  return e == cudaSuccess ? TACAW_OK : cuda_err(ctx, e, "k_accumulate");
}

}  // extern "C"
