// Time transform of one trajectory whose frames are split across processes (Supplement,
// "Sampling Considerations": frames are independent until the time transform; Methods,
// "Workflow Architecture": psi~(k, w) = F_t[psi(k, t) - <psi(k, t)>_t]).
//
// Subtracting any time-independent reference psi_ref instead of the frame mean changes psi~
// only at w = 0 (sum_n exp(-2 pi i m n / F) = F delta_m0), and the mean-subtracted psi~(0) is
// zero.  So each process transforms its own frames [f0, f0 + nf) against a reference that every
// process can form without communication (the exit wave of the trajectory's first frame):
//   psi~_part[p][m][j] = sum_{n < nf} exp(-2 pi i m (f0 + n) / F) (psi[p][n][q_j] - psi_ref[p][q_j]),
// one sum over the processes (an all-reduce) gives psi~ for w != 0, and the intensity
// S = |psi~|^2 is formed with S(w = 0) = 0.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "tacaw_api_internal.h"
#include "tacaw_internal.cuh"

namespace tacaw {

// r[p][n][j] = psi[p][n][q_j] - ref[p][q_j], the FP32 difference correctly rounded.
__global__ void k_residual_ref(const float2* __restrict__ psi, const float2* __restrict__ ref, int64_t nf,
                               int64_t nq, const int32_t* __restrict__ qsel, int64_t nsel, float2* __restrict__ r) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n = blockIdx.y, p = blockIdx.z;
  if (j >= nsel) return;
  const int64_t q = qsel ? qsel[j] : j;
  const float2 v = psi[((size_t)p * nf + n) * nq + q], m = ref[(size_t)p * nq + q];
  r[((size_t)p * nf + n) * nsel + j] = make_float2(__fsub_rn(v.x, m.x), __fsub_rn(v.y, m.y));
}

// psi~_part[p][m][j] = sum_n tw_F[(m (f0 + n)) mod F] r[p][n][j], FP32, 64 x 64 output tile per
// CTA, 4 x 4 per thread, K (local frames) in steps of 16.
constexpr int PD_BM = 64, PD_BN = 64, PD_BK = 16;

__global__ void __launch_bounds__(256) k_dft_partial(const float2* __restrict__ r, const float2* __restrict__ twF,
                                                     int64_t F, int64_t nf, int64_t f0, int64_t nsel,
                                                     float2* __restrict__ out) {
  __shared__ float2 Ws[PD_BK][PD_BM];
  __shared__ float2 Rs[PD_BK][PD_BN];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int64_t j0 = (int64_t)blockIdx.x * PD_BN, m0 = (int64_t)blockIdx.y * PD_BM, p = blockIdx.z;
  const float2* R = r + (size_t)p * nf * nsel;
  float2 acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = make_float2(0.f, 0.f);
  for (int64_t k0 = 0; k0 < nf; k0 += PD_BK) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int e = tid + 256 * i;
      const int kk = e / PD_BM, mm = e % PD_BM;
      const int64_t m = m0 + mm, n = k0 + kk;
      Ws[kk][mm] = (m < F && n < nf) ? twF[(m * ((f0 + n) % F)) % F] : make_float2(0.f, 0.f);
      const int kr = e / PD_BN, jr = e % PD_BN;
      const int64_t jj = j0 + jr, nr = k0 + kr;
      Rs[kr][jr] = (jj < nsel && nr < nf) ? R[(size_t)nr * nsel + jj] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < PD_BK; ++kk) {
      float2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = Ws[kk][ty + 16 * i];
#pragma unroll
      for (int i = 0; i < 4; ++i) b[i] = Rs[kk][tx + 16 * i];
#pragma unroll
      for (int ii = 0; ii < 4; ++ii)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          acc[ii][jj].x = fmaf(a[ii].x, b[jj].x, acc[ii][jj].x);
          acc[ii][jj].x = fmaf(-a[ii].y, b[jj].y, acc[ii][jj].x);
          acc[ii][jj].y = fmaf(a[ii].x, b[jj].y, acc[ii][jj].y);
          acc[ii][jj].y = fmaf(a[ii].y, b[jj].x, acc[ii][jj].y);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int ii = 0; ii < 4; ++ii) {
    const int64_t m = m0 + ty + 16 * ii;
    if (m >= F) continue;
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int64_t j = j0 + tx + 16 * jj;
      if (j < nsel) out[((size_t)p * F + m) * nsel + j] = acc[ii][jj];
    }
  }
}

// S[p][m][q_j] = |psi~[p][m][j]|^2, and 0 at m = 0 (full S; the caller's other q stay as set).
__global__ void k_intensity(const float2* __restrict__ pt, int64_t F, int64_t nsel, const int32_t* __restrict__ qsel,
                            int64_t nq, float* __restrict__ S) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t m = blockIdx.y, p = blockIdx.z;
  if (j >= nsel) return;
  const float2 v = pt[((size_t)p * F + m) * nsel + j];
  const int64_t q = qsel ? qsel[j] : j;
  S[((size_t)p * F + m) * nq + q] = m == 0 ? 0.f : v.x * v.x + v.y * v.y;
}

// SI[p][m] = sum_j |psi~[p][m][j]|^2 (FP64, fixed reduction tree), 0 at m = 0.
__global__ void __launch_bounds__(256) k_intensity_detector(const float2* __restrict__ pt, int64_t F, int64_t nsel,
                                                            float* __restrict__ SI) {
  __shared__ double red[256];
  const int64_t m = blockIdx.x, p = blockIdx.y;
  const float2* row = pt + ((size_t)p * F + m) * nsel;
  double acc = 0.0;
  if (m != 0)
    for (int64_t j = threadIdx.x; j < nsel; j += 256) {
      const float2 v = row[j];
      acc += (double)(v.x * v.x + v.y * v.y);
    }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) SI[(size_t)p * F + m] = (float)red[0];
}

namespace {
bool dev_ptr(const void* p) {
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

int tacaw_spectrum_partial(tacaw_ctx* ctx, const float* psi_k, int64_t P, int64_t nf, int64_t f0, int64_t F,
                           int64_t nq, const float* psi_ref, const int32_t* q_sel, int64_t n_sel, float* psi_tilde,
                           void* stream) {
  if (!ctx) return TACAW_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  NvtxRange nvtx("tacaw_spectrum_partial");
  if (P < 1 || nf < 1 || F < 1 || nq < 1 || f0 < 0 || f0 + nf > F)
    return set_err(ctx, TACAW_EINVAL, "need P, nf, F, nq >= 1 and 0 <= f0, f0 + nf <= F");
  if (P > 65535 || nf > 65535 || (F + PD_BM - 1) / PD_BM > 65535)
    return set_err(ctx, TACAW_EINVAL, "P, nf must be <= 65535");
  if (q_sel && (n_sel < 1 || n_sel > nq)) return set_err(ctx, TACAW_EINVAL, "n_sel must be in [1, nq]");
  if (!dev_ptr(psi_k) || !dev_ptr(psi_ref) || !dev_ptr(psi_tilde) || (q_sel && !dev_ptr(q_sel)))
    return set_err(ctx, TACAW_EINVAL, "psi_k, psi_ref, psi_tilde (and q_sel) must be device pointers");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaSetDevice");
  const int64_t nsel = q_sel ? n_sel : nq;
  cudaStream_t st = (cudaStream_t)stream;
  Scratch sc(st);
  float2* r;
  e = sc.get(&r, (size_t)P * nf * nsel);
  if (e != cudaSuccess) return cuda_err(ctx, e, "partial residual");
  {
    ProfScope ps(ctx, "residual_ref", st, (double)P * nf * nsel * 16 + (double)P * nsel * 8, (double)P * nf * nsel * 2);
    k_residual_ref<<<dim3((unsigned)((nsel + 255) / 256), (unsigned)nf, (unsigned)P), 256, 0, st>>>(
        reinterpret_cast<const float2*>(psi_k), reinterpret_cast<const float2*>(psi_ref), nf, nq, q_sel, nsel, r);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(ctx, e, "k_residual_ref");
  }
  float2* twF;
  int rc = get_time_tw(ctx, F, &twF);
  if (rc != TACAW_OK) return rc;
  {
    ProfScope ps(ctx, "dft_partial", st, (double)P * nf * nsel * 8 + (double)P * F * nsel * 8,
                 8.0 * F * nf * (double)P * nsel);
    const dim3 grid((unsigned)((nsel + PD_BN - 1) / PD_BN), (unsigned)((F + PD_BM - 1) / PD_BM), (unsigned)P);
    k_dft_partial<<<grid, 256, 0, st>>>(r, twF, F, nf, f0, nsel, reinterpret_cast<float2*>(psi_tilde));
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(ctx, e, "k_dft_partial");
  }
  return TACAW_OK;
}

int tacaw_intensity(tacaw_ctx* ctx, const float* psi_tilde, int64_t P, int64_t F, int64_t n_sel,
                    const int32_t* q_sel, int64_t nq, int32_t reduce, float* S_out, void* stream) {
  if (!ctx) return TACAW_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  NvtxRange nvtx("tacaw_intensity");
  if (P < 1 || F < 1 || n_sel < 1 || P > 65535 || F > 65535) return set_err(ctx, TACAW_EINVAL, "bad sizes");
  if (reduce != TACAW_REDUCE_NONE && reduce != TACAW_REDUCE_DETECTOR) return set_err(ctx, TACAW_EINVAL, "bad reduce");
  if (reduce == TACAW_REDUCE_NONE && (nq < n_sel || (!q_sel && nq != n_sel)))
    return set_err(ctx, TACAW_EINVAL, "nq must be n_sel without q_sel and >= n_sel with it");
  if (!dev_ptr(psi_tilde) || !dev_ptr(S_out) || (q_sel && !dev_ptr(q_sel)))
    return set_err(ctx, TACAW_EINVAL, "psi_tilde, S_out (and q_sel) must be device pointers");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  const float2* pt = reinterpret_cast<const float2*>(psi_tilde);
  if (reduce == TACAW_REDUCE_NONE) {
    if (q_sel && n_sel < nq) {
      e = cudaMemsetAsync(S_out, 0, sizeof(float) * P * F * nq, st);
      if (e != cudaSuccess) return cuda_err(ctx, e, "cudaMemsetAsync");
    }
    ProfScope ps(ctx, "intensity", st, (double)P * F * n_sel * 12, (double)P * F * n_sel * 3);
    k_intensity<<<dim3((unsigned)((n_sel + 255) / 256), (unsigned)F, (unsigned)P), 256, 0, st>>>(pt, F, n_sel, q_sel,
                                                                                                nq, S_out);
  } else {
    ProfScope ps(ctx, "intensity_detector", st, (double)P * F * n_sel * 8, (double)P * F * n_sel * 4);
    k_intensity_detector<<<dim3((unsigned)F, (unsigned)P), 256, 0, st>>>(pt, F, n_sel, S_out);
  }
  e = cudaGetLastError();
  return e == cudaSuccess ? TACAW_OK : cuda_err(ctx, e, "k_intensity");
}

}  // extern "C"
