// Time transform (Methods, "Workflow Architecture"):
//   psi~(k, w) = F_t[psi(k, t) - <psi(k, t)>_t],  I(k, w) = |psi~(k, w)|^2.
// The mean over frames and the residual are formed to FP64-class precision (the elastic part
// is large and the inelastic signal is a small difference), as FP32 pairs.  This file holds the plain FP32 SIMT dense DFT;
// the tensor-core variants are in k_dft_tc.cu.
#include <cuda_runtime.h>

#include "tacaw_internal.cuh"

namespace tacaw {

// mean[p][j] = (1/F) sum_n psi[p][n][q_j] to FP64-class precision.  A CTA takes 32 columns;
// 8 threads per column sum the frames n = g mod 8 (four loads in flight each) as FP32 pairs
// (pair_add), in frame order; the 8 pairs are then added in FP64 in a fixed order and divided
// by F.  Over n frames a pair loses at most about n 2^-48 of its largest partial sum (FP64
// summation: n 2^-53), far below the FP32 rounding of the residual that follows.
constexpr int MEAN_COLS = 32, MEAN_GROUPS = 8;

__global__ void __launch_bounds__(MEAN_COLS * MEAN_GROUPS)
    k_mean_f64(const float2* __restrict__ psi, int64_t F, int64_t nq, const int32_t* __restrict__ qsel,
               int64_t nsel, double2* __restrict__ mean) {
  __shared__ float4 part[MEAN_GROUPS][MEAN_COLS];  // (hi.x, lo.x, hi.y, lo.y)
  const int tx = threadIdx.x % MEAN_COLS, g = threadIdx.x / MEAN_COLS;
  const int64_t j = blockIdx.x * (int64_t)MEAN_COLS + tx;
  const int64_t p = blockIdx.y;
  float4 ps = make_float4(0.f, 0.f, 0.f, 0.f);
  if (j < nsel) {
    const int64_t q = qsel ? qsel[j] : j;
    ps = column_pair_sums<MEAN_GROUPS>(psi + (size_t)p * F * nq + q, F, nq, g);
  }
  part[g][tx] = ps;
  __syncthreads();
  if (g == 0 && j < nsel) {
    float4 col[MEAN_GROUPS];
#pragma unroll
    for (int k = 0; k < MEAN_GROUPS; ++k) col[k] = part[k][tx];
    mean[(size_t)p * nsel + j] = combine_pair_sums<MEAN_GROUPS>(col, F);
  }
}

cudaError_t launch_mean_f64(const float2* psi, int64_t P, int64_t F, int64_t nq, const int32_t* qsel, int64_t nsel,
                            double2* mean, cudaStream_t st) {
  if (P > 65535) return cudaErrorInvalidValue;
  k_mean_f64<<<dim3((unsigned)((nsel + MEAN_COLS - 1) / MEAN_COLS), (unsigned)P), MEAN_COLS * MEAN_GROUPS, 0, st>>>(
      psi, F, nq, qsel, nsel, mean);
  return cudaGetLastError();
}

// r[p][n][j] = psi[p][n][q_j] - mean[p][j]: the mean as an FP32 pair, the difference formed
// exactly (pair_sub) and rounded to float.
__global__ void k_residual_f32(const float2* __restrict__ psi, const double2* __restrict__ mean, int64_t F,
                               int64_t nq, const int32_t* __restrict__ qsel, int64_t nsel, float2* __restrict__ r) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n = blockIdx.y, p = blockIdx.z;
  if (j >= nsel) return;
  const int64_t q = qsel ? qsel[j] : j;
  const float2 v = psi[((size_t)p * F + n) * nq + q];
  const double2 m = mean[(size_t)p * nsel + j];
  float mxh, mxl, myh, myl, rx, ex, ry, ey;
  split_double(m.x, mxh, mxl);
  split_double(m.y, myh, myl);
  pair_sub(v.x, mxh, mxl, rx, ex);
  pair_sub(v.y, myh, myl, ry, ey);
  r[((size_t)p * F + n) * nsel + j] = make_float2(rx, ry);
}

cudaError_t launch_residual_f32(const float2* psi, const double2* mean, int64_t P, int64_t F, int64_t nq,
                                const int32_t* qsel, int64_t nsel, float2* r, cudaStream_t st) {
  if (P > 65535 || F > 65535) return cudaErrorInvalidValue;
  k_residual_f32<<<dim3((unsigned)((nsel + 255) / 256), (unsigned)F, (unsigned)P), 256, 0, st>>>(psi, mean, F, nq,
                                                                                                qsel, nsel, r);
  return cudaGetLastError();
}

// Plain FP32 dense DFT: S[p][m][q_j] = |sum_n W[m][n] r[p][n][j]|^2 with W[m][n] = tw_F[(m n) mod F],
// tw_F[i] = exp(-2 pi i i / F).  64 x 64 output tile per CTA, 4 x 4 per thread, K step 16.
constexpr int DFT_BM = 64, DFT_BN = 64, DFT_BK = 16;

__global__ void __launch_bounds__(256) k_dft_fp32(const float2* __restrict__ r, const float2* __restrict__ twF,
                                                  int64_t F, int64_t nsel, int64_t nq, const int32_t* __restrict__ qsel,
                                                  float* __restrict__ S) {
  __shared__ float2 Ws[DFT_BK][DFT_BM];
  __shared__ float2 Rs[DFT_BK][DFT_BN];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int64_t j0 = (int64_t)blockIdx.x * DFT_BN, m0 = (int64_t)blockIdx.y * DFT_BM, p = blockIdx.z;
  const float2* R = r + (size_t)p * F * nsel;
  float2 acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = make_float2(0.f, 0.f);
  for (int64_t k0 = 0; k0 < F; k0 += DFT_BK) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int e = tid + 256 * i;  // 0..1023
      const int kk = e / DFT_BM, mm = e % DFT_BM;
      const int64_t m = m0 + mm, n = k0 + kk;
      Ws[kk][mm] = (m < F && n < F) ? twF[(m * n) % F] : make_float2(0.f, 0.f);
      const int kr = e / DFT_BN, jr = e % DFT_BN;
      const int64_t jj = j0 + jr, nr = k0 + kr;
      Rs[kr][jr] = (jj < nsel && nr < F) ? R[(size_t)nr * nsel + jj] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < DFT_BK; ++kk) {
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
      if (j >= nsel) continue;
      const int64_t q = qsel ? qsel[j] : j;
      S[((size_t)p * F + m) * nq + q] = acc[ii][jj].x * acc[ii][jj].x + acc[ii][jj].y * acc[ii][jj].y;
    }
  }
}

cudaError_t launch_dft_fp32(const float2* r, const float2* twF, int64_t P, int64_t F, int64_t nsel, int64_t nq,
                            const int32_t* qsel, float* S, cudaStream_t st) {
  if (P > 65535 || (F + DFT_BM - 1) / DFT_BM > 65535) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)((nsel + DFT_BN - 1) / DFT_BN), (unsigned)((F + DFT_BM - 1) / DFT_BM), (unsigned)P);
  k_dft_fp32<<<grid, 256, 0, st>>>(r, twF, F, nsel, nq, qsel, S);
  return cudaGetLastError();
}

// SI[p][m] = sum_j S[p][m][q_j], FP64 accumulation with a fixed reduction tree.
__global__ void __launch_bounds__(256) k_detector_reduce(const float* __restrict__ S, int64_t F, int64_t nq,
                                                         const int32_t* __restrict__ qsel, int64_t nsel,
                                                         float* __restrict__ SI) {
  __shared__ double red[256];
  const int64_t m = blockIdx.x, p = blockIdx.y;
  const float* row = S + ((size_t)p * F + m) * nq;
  double acc = 0.0;
  for (int64_t j = threadIdx.x; j < nsel; j += 256) acc += (double)row[qsel ? qsel[j] : j];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) SI[(size_t)p * F + m] = (float)red[0];
}

cudaError_t launch_detector_reduce(const float* S, int64_t P, int64_t F, int64_t nq, const int32_t* qsel,
                                   int64_t nsel, float* SI, cudaStream_t st) {
  if (P > 65535) return cudaErrorInvalidValue;
  k_detector_reduce<<<dim3((unsigned)F, (unsigned)P), 256, 0, st>>>(S, F, nq, qsel, nsel, SI);
  return cudaGetLastError();
}

}  // namespace tacaw
