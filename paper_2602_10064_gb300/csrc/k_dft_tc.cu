// Tensor-core time transform (Methods, "Workflow Architecture": psi~(k, w) = F_t[psi - <psi>_t],
// I = |psi~|^2) as a dense real GEMM on the 5th-generation tensor cores (tcgen05).
//
// With W = exp(-2 pi i w n / F) = cos - i sin and the residual r_n = psi_n - <psi> (formed exactly
// from the FP64-class mean), the complex sum becomes the real product D = A B^T:
//   rows of D: m = 2w + c (c = 0 real, 1 imaginary part of psi~(w)),
//   K:         kappa = 2n + c' (c' = 0 real, 1 imaginary part of r_n),
//   A[2w][2n] = cos, A[2w][2n+1] = sin, A[2w+1][2n] = -sin, A[2w+1][2n+1] = cos,
//   B[j][2n + c'] = r_c'[n][q_j]   (B is K-major: each q's time series is contiguous).
// Split precision: A = A_hi + A_lo, B = B_hi + B_lo (BF16 or TF32 parts), and
// D = A_hi B_hi + A_hi B_lo + A_lo B_hi accumulated in FP32 in tensor memory.
//
// Kernel: one CTA (10 warps) per 128 x 256 tile of D.  Warp 0 lane 0 streams A and B tiles
// with TMA (128-byte swizzle) into a 4-stage shared-memory ring; warp 1 lane 0 issues
// tcgen05.mma (M 128, N 256, K 16 for BF16 / 8 for TF32) into FP32 accumulators in TMEM.
// The tensor core rounds the accumulator at every MMA with a bias, so over thousands of
// K steps (the frames of a long trajectory) the error would grow linearly; instead the MMAs
// of one chunk of TC_KC K blocks accumulate in TMEM (two 256-column buffers, alternating),
// and after every chunk warps 2..9 add the chunk's partial sums into FP32 registers on the
// CUDA cores (round to nearest).  At the end those warps form S = D[2w]^2 + D[2w+1]^2 and either
// store it (full S) or, for the detector-summed spectrum image, add it up over the tile's
// columns in FP64 and store one partial sum per (tile, w); a second kernel adds the partial sums
// of each probe in a fixed order, so S is never written and the result is deterministic.
// The columns of B are laid out per probe, cpp (a multiple of the tile width) per probe, so
// every tile belongs to one probe; columns j >= nsel of a probe are zero.
// Every wait is bounded (%globaltimer); on expiry the kernel sets the context's status word
// and leaves without hanging.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "tacaw_api_internal.h"

namespace tacaw {

constexpr int TC_BM = 128, TC_BN = 256, TC_STAGES = 4;
constexpr int TC_EPI_WARPS = 8, TC_THREADS = 64 + 32 * TC_EPI_WARPS;
constexpr int TC_KC = 16;            // K blocks (of 4 MMAs) accumulated in TMEM per chunk
constexpr int TC_EPI_COLS = TC_BN / 2;  // accumulator columns per epilogue thread
constexpr int TC_ROW_BYTES = 128;  // one swizzle span of K per tile row
constexpr int TC_A_BYTES = TC_BM * TC_ROW_BYTES, TC_B_BYTES = TC_BN * TC_ROW_BYTES;
constexpr int TC_STAGE_BYTES = TC_A_BYTES + TC_B_BYTES;
constexpr int TC_SMEM = TC_STAGES * TC_STAGE_BYTES + 1024 /*alignment*/ + 256 /*barriers*/ +
                        TC_BM * 8 /*detector partial sums of the two column halves*/;
constexpr int TC_TMEM_COLS = 2 * TC_BN;  // two accumulator buffers
constexpr unsigned long long TC_TIMEOUT_NS = 2000000000ull;  // 2 s per wait

// status word bit of a wait that ran out
constexpr int TC_ERR_TIMEOUT = TACAW_STATUS_TIMEOUT;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false (and the status word set) if the phase did not complete in time.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* status,
                                          unsigned long long timeout_ns = TC_TIMEOUT_NS) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (!mbar_try(bar, parity)) {
    if (globaltimer() - t0 > timeout_ns) {
      atomicOr(status, TC_ERR_TIMEOUT);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);        // start address
  d |= (uint64_t)1 << 16;                        // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;              // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                        // descriptor version
  d |= (uint64_t)2 << 61;                        // swizzle: 128 B
  return d;
}

// Instruction descriptor: FP32 accumulator, K-major A and B, M = 128, N = 256.
// a/b format: BF16 = 1 (kind::f16), TF32 = 2 (kind::tf32).
__host__ __device__ constexpr uint32_t tc_idesc(uint32_t ab_format) {
  return (1u << 4) | (ab_format << 7) | (ab_format << 10) | ((uint32_t)(TC_BN >> 3) << 17) |
         ((uint32_t)(TC_BM >> 4) << 24);
}

template <bool TF32>
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  if constexpr (TF32) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(tc_idesc(2)), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(tc_idesc(1)), "r"(accumulate)
        : "memory");
  }
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Persistent: CTA c takes the tiles c, c + gridDim.x, ... of D (128 x 256 each), numbered with
// the row block fastest so that the CTAs running together share their B tile through L2.  The
// shared-memory ring, the K chunks and the two TMEM accumulator buffers run on counters that
// continue across tiles, so the epilogue of one tile overlaps the first MMAs of the next.
// nphase: 1 (hi*hi) or 3 (hi*hi, hi*lo, lo*hi); nkb: K blocks of 128 bytes per phase.
template <bool TF32>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_dft_tc(const __grid_constant__ CUtensorMap mAhi, const __grid_constant__ CUtensorMap mAlo,
             const __grid_constant__ CUtensorMap mBhi, const __grid_constant__ CUtensorMap mBlo, int mtiles,
             int64_t tiles, int nphase, int nkb, int64_t F, int64_t cpp, int64_t nsel, int64_t out_nq,
             const int32_t* __restrict__ out_qsel, float* __restrict__ S, double* __restrict__ part,
             int* __restrict__ status) {
  extern __shared__ uint8_t smraw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + TC_STAGES * TC_STAGE_BYTES);
  // bars: full[S], empty[S], acc_full[2], acc_empty[2], drain; then the TMEM base address
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * TC_STAGES + 5);
  double* red = reinterpret_cast<double*>(smem + TC_STAGES * TC_STAGE_BYTES + 256);  // [2][TC_BM / 2]
  const uint32_t drain = smem_u32(bars + 2 * TC_STAGES + 4);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + TC_STAGES);
  const uint32_t accf0 = smem_u32(bars + 2 * TC_STAGES), acce0 = smem_u32(bars + 2 * TC_STAGES + 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf0 + 8 * b, 1);
      mbar_init(acce0 + 8 * b, TC_EPI_WARPS);
    }
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const int total = nphase * nkb;  // K blocks per tile; each holds 4 MMAs of 32 bytes of K
  const int nchunk = (total + TC_KC - 1) / TC_KC;

  if (warp == 0 && lane == 0) {
    // producer: K block i of the CTA's sequence (all its tiles) goes to stage i % TC_STAGES
    int64_t i = 0, issued = 0;
    bool ok = true;
    for (int64_t tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
      const int m0 = (int)(tile % mtiles) * TC_BM;
      const int n0 = (int)((tile / mtiles) * TC_BN);
      for (int kb = 0; kb < total; ++kb, ++i) {
        const int s = (int)(i % TC_STAGES);
        const uint32_t ph = (uint32_t)((i / TC_STAGES) & 1);
        if (!mbar_wait(empty0 + 8 * s, ph ^ 1u, status)) {
          ok = false;
          break;
        }
        const int phase = kb / nkb, kk = kb % nkb;
        const CUtensorMap* ma = (phase == 2) ? &mAlo : &mAhi;
        const CUtensorMap* mb = (phase == 1) ? &mBlo : &mBhi;
        const uint32_t sa = smem_u32(smem + s * TC_STAGE_BYTES), sb = sa + TC_A_BYTES;
        const int kx = kk * (TC_ROW_BYTES / (TF32 ? 4 : 2));
        mbar_expect_tx(full0 + 8 * s, TC_STAGE_BYTES);
        tma_load_2d(sa, ma, kx, m0, full0 + 8 * s);
        tma_load_2d(sb, mb, kx, n0, full0 + 8 * s);
        issued = i + 1;
      }
    }
    // leave no copy in flight: wait for the last stages this thread armed
    for (int64_t k = (issued > TC_STAGES ? issued - TC_STAGES : 0); k < issued; ++k)
      mbar_wait(full0 + 8 * (int)(k % TC_STAGES), (uint32_t)((k / TC_STAGES) & 1), status);
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: chunk g of the CTA's sequence accumulates into TMEM buffer g & 1
    int64_t i = 0, g = 0;
    bool ok = true;
    for (int64_t tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
      for (int c = 0; c < nchunk && ok; ++c, ++g) {
        const int b = (int)(g & 1);
        if (g >= 2 && !mbar_wait(acce0 + 8 * b, (uint32_t)(((g >> 1) - 1) & 1), status)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + (uint32_t)(b * TC_BN);
        const int kb1 = (c + 1) * TC_KC < total ? (c + 1) * TC_KC : total;
        for (int kb = c * TC_KC; kb < kb1; ++kb, ++i) {
          const int s = (int)(i % TC_STAGES);
          const uint32_t ph = (uint32_t)((i / TC_STAGES) & 1);
          if (!mbar_wait(full0 + 8 * s, ph, status)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t sa = smem_u32(smem + s * TC_STAGE_BYTES), sb = sa + TC_A_BYTES;
#pragma unroll
          for (int k = 0; k < TC_ROW_BYTES / 32; ++k)
            tc_mma<TF32>(d, smem_desc_sw128(sa + 32 * k), smem_desc_sw128(sb + 32 * k), (kb - c * TC_KC) | k);
          tc_commit(empty0 + 8 * s);  // frees the stage once these MMAs have read it
        }
        if (ok) tc_commit(accf0 + 8 * b);  // this chunk's MMAs complete -> buffer b readable
      }
    }
    // no MMA may be in flight when TMEM is released, also after a timeout
    tc_commit(drain);
    mbar_wait(drain, 0, status);
  } else if (warp >= 2) {
    // accumulators: warp w owns TMEM lanes 32 (w % 4) .. +31 and columns [128 h, 128 h + 128)
    const int e = warp - 2, quarter = warp & 3, half = e >> 2;
    bool ok = true;
    int64_t g = 0;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
      const int m0 = (int)(tile % mtiles) * TC_BM;
      const int64_t n0 = (tile / mtiles) * TC_BN;
      float acc[TC_EPI_COLS];
#pragma unroll
      for (int i = 0; i < TC_EPI_COLS; ++i) acc[i] = 0.f;
      for (int c = 0; c < nchunk && ok; ++c, ++g) {
        const int b = (int)(g & 1);
        ok = __all_sync(0xffffffffu, ok && mbar_wait(accf0 + 8 * b, (uint32_t)((g >> 1) & 1), status));
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t base = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(b * TC_BN + half * TC_EPI_COLS);
#pragma unroll
        for (int c0 = 0; c0 < TC_EPI_COLS; c0 += 32) {
          float v[32];
          tmem_ld32(base + (uint32_t)c0, v);
#pragma unroll
          for (int i = 0; i < 32; ++i) acc[c0 + i] += v[i];
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(acce0 + 8 * b) : "memory");
      }
      // rows m0 + 32 quarter + lane: even lanes hold Re, odd lanes Im of psi~(w); the tile's
      // columns all belong to probe p (cpp is a multiple of TC_BN)
      const int m = m0 + 32 * quarter + lane;
      const int64_t w = m >> 1;
      const bool writer = ((lane & 1) == 0) && w < F;
      const int64_t p = n0 / cpp, j0 = n0 - p * cpp + half * TC_EPI_COLS;
      if (!part) {
        if (ok) {
#pragma unroll
          for (int i = 0; i < TC_EPI_COLS; ++i) {
            const float o = __shfl_xor_sync(0xffffffffu, acc[i], 1);
            const float sv = acc[i] * acc[i] + o * o;
            const int64_t j = j0 + i;
            if (writer && j < nsel) {
              const int64_t q = out_qsel ? out_qsel[j] : j;
              S[((size_t)p * F + w) * out_nq + q] = sv;
            }
          }
        }
      } else {
        // detector sum: |psi~|^2 rounded to float as a stored S would be, summed over this
        // thread's columns as an FP32 pair (error-free two-sums: FP64-class, since GB300's FP64
        // pipe would take longer than the tile's MMAs), the pair combined in FP64, then the two
        // column halves added in FP64 in a fixed order
        float dh = 0.f, dl = 0.f;
#pragma unroll
        for (int i = 0; i < TC_EPI_COLS; ++i) {
          const float o = __shfl_xor_sync(0xffffffffu, acc[i], 1);
          const float sv = acc[i] * acc[i] + o * o;
          if (j0 + i < nsel) pair_add(dh, dl, sv);
        }
        const double dsum = (double)dh + (double)dl;
        const int r = (32 * quarter + lane) >> 1;
        if ((lane & 1) == 0) red[half * (TC_BM / 2) + r] = dsum;
        // every epilogue warp arrives here for every tile, also after a timed-out wait
        asm volatile("bar.sync 1, %0;" ::"n"(32 * TC_EPI_WARPS) : "memory");
        if (ok && half == 0 && writer) part[(size_t)(n0 / TC_BN) * F + w] = red[r] + red[TC_BM / 2 + r];
        // the next tile's partial sums reuse red
        asm volatile("bar.sync 1, %0;" ::"n"(32 * TC_EPI_WARPS) : "memory");
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
  }
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Frame mean and residual split in one pass per column block: B_hi/B_lo[J][2n + c] for
// J = p * cpp + j, from r = psi[p][n][q_j] - mean[p][j], zero for the padding columns j >= nsel
// and the K pad frames.  A CTA takes 32 columns: 8 threads per column form the frame mean to
// FP64-class precision (column_pair_sums, combine_pair_sums: the arithmetic of the mean kernel of
// the FP32 path), then the CTA walks the frames in 32 x 32 (j, n) tiles, transposed through
// shared memory; the second read of the column block comes from L2.  The difference is formed
// exactly as the FP32 pair (r, re) (pair_sub: the FP64 mean as an FP32 pair); hi = r rounded to
// the operand type, lo = (r - hi) + re, where r - hi is exact.  A tile holds RS_TN frames, so
// each thread has RS_TN / 8 loads in flight between two barriers.
constexpr int RS_GROUPS = 8, RS_TN = 64;
template <bool TF32>
__global__ void __launch_bounds__(256) k_mean_residual_split(const float2* __restrict__ psi, int64_t F, int64_t nq,
                                                             const int32_t* __restrict__ qsel, int64_t nsel,
                                                             int64_t cpp, int kpad2, void* __restrict__ Bhi,
                                                             void* __restrict__ Blo) {
  __shared__ float4 part[RS_GROUPS][32];
  __shared__ float4 msplit[32];  // mean as FP32 pairs (hi.x, lo.x, hi.y, lo.y)
  __shared__ float2 hs[RS_TN][33], ls[RS_TN][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const int64_t J0 = (int64_t)blockIdx.x * 32;
  // columns j >= nsel of a probe (padding) are zero; a block of 32 lies inside one probe
  const int64_t J = J0 + tx, p = J / cpp, j = J - p * cpp;
  const bool live = j < nsel;
  const int64_t q = live ? (qsel ? qsel[j] : j) : 0;
  const float2* col = psi + (size_t)p * F * nq + q;
  part[ty][tx] = live ? column_pair_sums<RS_GROUPS>(col, F, nq, ty) : make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
  if (ty == 0) {
    float4 c[RS_GROUPS];
#pragma unroll
    for (int k = 0; k < RS_GROUPS; ++k) c[k] = part[k][tx];
    const double2 mu = combine_pair_sums<RS_GROUPS>(c, F);
    float4 m;
    split_double(mu.x, m.x, m.y);
    split_double(mu.y, m.z, m.w);
    msplit[tx] = m;
  }
  __syncthreads();
  const float4 m = msplit[tx];
  for (int64_t n0 = 0; 2 * n0 < kpad2; n0 += RS_TN) {
    // phase 1: coalesced along j
#pragma unroll
    for (int r = ty; r < RS_TN; r += 8) {
      const int64_t n = n0 + r;
      float2 h = make_float2(0.f, 0.f), l = make_float2(0.f, 0.f);
      if (live && n < F) {
        const float2 v = col[(size_t)n * nq];
        float rx, ex, ry, ey;
        pair_sub(v.x, m.x, m.y, rx, ex);
        pair_sub(v.y, m.z, m.w, ry, ey);
        if (TF32) {
          const float ah = to_tf32(rx), bh = to_tf32(ry);
          h = make_float2(ah, bh);
          l = make_float2(to_tf32(__fadd_rn(__fsub_rn(rx, ah), ex)), to_tf32(__fadd_rn(__fsub_rn(ry, bh), ey)));
        } else {
          h = make_float2(__bfloat162float(__float2bfloat16_rn(rx)), __bfloat162float(__float2bfloat16_rn(ry)));
          l = make_float2(__fadd_rn(__fsub_rn(rx, h.x), ex), __fadd_rn(__fsub_rn(ry, h.y), ey));
        }
      }
      hs[r][tx] = h;
      ls[r][tx] = l;
    }
    __syncthreads();
    // phase 2: each warp writes rows J (contiguous along n)
    for (int cr = ty; cr < 32 * (RS_TN / 32); cr += 8) {
      const int c = cr & 31, h0 = (cr >> 5) * 32;
      const int64_t Jw = J0 + c;
      const int64_t n = n0 + h0 + tx;
      if (2 * n >= kpad2) continue;
      const float2 h = hs[h0 + tx][c], l = ls[h0 + tx][c];
      if (TF32) {
        reinterpret_cast<float2*>(Bhi)[(size_t)Jw * (kpad2 / 2) + n] = h;
        reinterpret_cast<float2*>(Blo)[(size_t)Jw * (kpad2 / 2) + n] = l;
      } else {
        __nv_bfloat162 hh, ll;
        hh.x = __float2bfloat16_rn(h.x);
        hh.y = __float2bfloat16_rn(h.y);
        ll.x = __float2bfloat16_rn(l.x);
        ll.y = __float2bfloat16_rn(l.y);
        reinterpret_cast<__nv_bfloat162*>(Bhi)[(size_t)Jw * (kpad2 / 2) + n] = hh;
        reinterpret_cast<__nv_bfloat162*>(Blo)[(size_t)Jw * (kpad2 / 2) + n] = ll;
      }
    }
    __syncthreads();  // the tile buffers are refilled for the next frames
  }
}

// Spectrum image from the detector partial sums: SI[p][w] = sum over the tpp tiles of probe p of
// part[tile][w], in FP64 and in tile order, rounded to float.
__global__ void k_detector_tiles(const double* __restrict__ part, int64_t P, int64_t F, int64_t tpp,
                                 float* __restrict__ SI) {
  const int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, p = blockIdx.y;
  if (w >= F || p >= P) return;
  const double* col = part + (size_t)p * tpp * F + w;
  double s = 0.0;
  for (int64_t t = 0; t < tpp; ++t) s += col[(size_t)t * F];
  SI[(size_t)p * F + w] = (float)s;
}

// Self-test of the bounded wait: one thread waits on an mbarrier that nothing ever arrives on,
// with a short limit, so the wait runs out, sets the status word and returns (no copy or MMA
// is in flight, no TMEM is held).
__global__ void k_wait_selftest(int* __restrict__ status, unsigned long long timeout_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  const uint32_t b = smem_u32(&bar);
  mbar_init(b, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  mbar_wait(b, 0, status, timeout_ns);
}

// ---------------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------------
namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2D row-major [rows][kpad] operand, box = 128 bytes of K by box_rows rows, 128-byte swizzle.
bool make_map(CUtensorMap* m, const void* base, bool tf32, int64_t rows, int64_t kpad, int box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  const int esz = tf32 ? 4 : 2;
  cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kpad * esz};
  cuuint32_t box[2] = {(cuuint32_t)(TC_ROW_BYTES / esz), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return enc(m, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base),
             dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

uint16_t bf16_rn(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  const uint32_t lsb = (u >> 16) & 1u;
  u += 0x7FFFu + lsb;
  return (uint16_t)(u >> 16);
}
float bf16_to_f(uint16_t h) {
  const uint32_t u = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}
// round to TF32 (10 mantissa bits), to nearest, ties away from zero
float tf32_rna(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u = (u + 0x1000u) & 0xFFFFE000u;
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

}  // namespace

// DFT operand A (hi, lo) for F frames, from FP64 cos/sin of the exactly reduced angle.
int get_dft_operands(tacaw_ctx* ctx, int64_t F, bool tf32, int64_t kpad, void** hi, void** lo) {
  const int64_t key = F * 4 + (tf32 ? 1 : 0);
  auto it = ctx->dft_ops.find(key);
  if (it != ctx->dft_ops.end()) {
    *hi = it->second.first;
    *lo = it->second.second;
    return TACAW_OK;
  }
  const int64_t M = 2 * F;
  const size_t esz = tf32 ? 4 : 2, n = (size_t)M * kpad;
  std::vector<uint8_t> h(n * esz, 0), l(n * esz, 0);
  for (int64_t w = 0; w < F; ++w)
    for (int64_t t = 0; t < F; ++t) {
      const double th = 2.0 * M_PI * (double)((w * t) % F) / (double)F;
      const double c = std::cos(th), s = std::sin(th);
      const double vals[4] = {c, s, -s, c};  // [2w][2t], [2w][2t+1], [2w+1][2t], [2w+1][2t+1]
      const int64_t idx[4] = {(2 * w) * kpad + 2 * t, (2 * w) * kpad + 2 * t + 1, (2 * w + 1) * kpad + 2 * t,
                              (2 * w + 1) * kpad + 2 * t + 1};
      for (int e = 0; e < 4; ++e) {
        if (tf32) {
          const float hv = tf32_rna((float)vals[e]);
          const float lv = tf32_rna((float)(vals[e] - (double)hv));
          std::memcpy(&h[idx[e] * 4], &hv, 4);
          std::memcpy(&l[idx[e] * 4], &lv, 4);
        } else {
          const uint16_t hv = bf16_rn((float)vals[e]);
          const uint16_t lv = bf16_rn((float)(vals[e] - (double)bf16_to_f(hv)));
          std::memcpy(&h[idx[e] * 2], &hv, 2);
          std::memcpy(&l[idx[e] * 2], &lv, 2);
        }
      }
    }
  void *dh = nullptr, *dl = nullptr;
  // stream-ordered on the legacy stream, which requests on non-blocking streams do not wait for
  cudaError_t e = cudaMallocAsync(&dh, h.size(), 0);
  if (e == cudaSuccess) e = cudaMallocAsync(&dl, l.size(), 0);
  if (e == cudaSuccess) e = cudaMemcpy(dh, h.data(), h.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dl, l.data(), l.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaStreamSynchronize(0);  // landed before any stream reads it
  if (e != cudaSuccess) {
    if (dh) cudaFree(dh);
    if (dl) cudaFree(dl);
    return cuda_err(ctx, e, "DFT operand upload");
  }
  ctx->owned.push_back(dh);
  ctx->owned.push_back(dl);
  ctx->dft_ops[key] = {dh, dl};
  *hi = dh;
  *lo = dl;
  return TACAW_OK;
}

int spectrum_tc(tacaw_ctx* ctx, const float2* psi_k, int64_t P, int64_t F, const SpecIO& io, int32_t precision,
                int32_t reduce, float* S, Scratch& sc) {
  const bool tf32 = precision == TACAW_DFT_TF32X3 || precision == TACAW_DFT_TF32;
  const int nphase = (precision == TACAW_DFT_BF16X3 || precision == TACAW_DFT_TF32X3) ? 3 : 1;
  const int esz = tf32 ? 4 : 2;
  const int kblk = TC_ROW_BYTES / esz;                 // K elements per block
  const int64_t kpad = ((2 * F + kblk - 1) / kblk) * kblk;
  const int64_t nsel = io.nsel;
  const int64_t cpp = (nsel + TC_BN - 1) / TC_BN * TC_BN;  // columns per probe, whole tiles
  const int64_t ncols = P * cpp;
  if (ncols > ((int64_t)1 << 31) - 1 || kpad > (1 << 24)) return set_err(ctx, TACAW_EINVAL, "spectrum too large");
  if (!encode_fn()) return set_err(ctx, TACAW_ECUDA, "cuTensorMapEncodeTiled is unavailable");
  void *Ahi, *Alo;
  int rc = get_dft_operands(ctx, F, tf32, kpad, &Ahi, &Alo);
  if (rc != TACAW_OK) return rc;
  uint8_t *Bhi, *Blo;
  cudaError_t e = sc.get(&Bhi, (size_t)ncols * kpad * esz);
  if (e == cudaSuccess) e = sc.get(&Blo, (size_t)ncols * kpad * esz);
  if (e != cudaSuccess) return cuda_err(ctx, e, "spectrum operand scratch");
  {
    ProfScope ps(ctx, tf32 ? "mean_residual_split_tf32" : "mean_residual_split_bf16", sc.st,
                 (double)P * F * nsel * 8 + (double)ncols * kpad * esz * 2, (double)P * F * nsel * 6);
    if (tf32)
      k_mean_residual_split<true><<<(unsigned)(ncols / 32), 256, 0, sc.st>>>(psi_k, F, io.in_nq, io.in_qsel, nsel, cpp,
                                                                            (int)kpad, Bhi, Blo);
    else
      k_mean_residual_split<false><<<(unsigned)(ncols / 32), 256, 0, sc.st>>>(psi_k, F, io.in_nq, io.in_qsel, nsel,
                                                                             cpp, (int)kpad, Bhi, Blo);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(ctx, e, "k_mean_residual_split");
  }
  CUtensorMap mAhi, mAlo, mBhi, mBlo;
  if (!make_map(&mAhi, Ahi, tf32, 2 * F, kpad, TC_BM) || !make_map(&mAlo, Alo, tf32, 2 * F, kpad, TC_BM) ||
      !make_map(&mBhi, Bhi, tf32, ncols, kpad, TC_BN) || !make_map(&mBlo, Blo, tf32, ncols, kpad, TC_BN))
    return set_err(ctx, TACAW_ECUDA, "tensor map encoding failed");
  const int mtiles = (int)((2 * F + TC_BM - 1) / TC_BM);
  const int64_t ntiles = ncols / TC_BN;
  const int64_t tiles = (int64_t)mtiles * ntiles;
  int nsm = 0;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaDeviceGetAttribute");
  const unsigned ctas = (unsigned)std::min<int64_t>(tiles, std::max(nsm, 1));  // persistent: one CTA per SM
  const int nkb = (int)(kpad / kblk);
  double* part = nullptr;
  const bool det = reduce == TACAW_REDUCE_DETECTOR;
  if (det) {
    e = sc.get(&part, (size_t)ntiles * F);
    if (e != cudaSuccess) return cuda_err(ctx, e, "detector partial sums");
  }
  e = tf32 ? cudaFuncSetAttribute(k_dft_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM)
           : cudaFuncSetAttribute(k_dft_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaFuncSetAttribute");
  {
    const double flops = 8.0 * F * F * (double)P * nsel * nphase;
    const double out_bytes = det ? (double)ntiles * F * 8 : (double)P * nsel * F * 4;
    ProfScope ps(ctx, tf32 ? "dft_tc_tf32" : "dft_tc_bf16", sc.st,
                 (double)ncols * kpad * esz * (nphase > 1 ? 2 : 1) + out_bytes, flops);
    if (tf32)
      k_dft_tc<true><<<ctas, TC_THREADS, TC_SMEM, sc.st>>>(mAhi, mAlo, mBhi, mBlo, mtiles, tiles, nphase, nkb, F,
                                                          cpp, nsel, io.out_nq, io.out_qsel, S, part, ctx->d_status);
    else
      k_dft_tc<false><<<ctas, TC_THREADS, TC_SMEM, sc.st>>>(mAhi, mAlo, mBhi, mBlo, mtiles, tiles, nphase, nkb,
                                                           F, cpp, nsel, io.out_nq, io.out_qsel, S, part,
                                                           ctx->d_status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(ctx, e, "k_dft_tc");
  }
  if (det) {
    ProfScope ps(ctx, "detector_tiles", sc.st, (double)ntiles * F * 8 + (double)P * F * 4, (double)ntiles * F);
    if (P > 65535) return set_err(ctx, TACAW_EINVAL, "too many probes");
    k_detector_tiles<<<dim3((unsigned)((F + 127) / 128), (unsigned)P), 128, 0, sc.st>>>(part, P, F, cpp / TC_BN, S);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(ctx, e, "k_detector_tiles");
  }
  return TACAW_OK;
}

}  // namespace tacaw

extern "C" int tacaw_selftest_wait(tacaw_ctx* ctx, double timeout_ms, void* stream) {
  using namespace tacaw;
  if (!ctx) return TACAW_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (!(timeout_ms > 0.0) || timeout_ms > 1000.0) return set_err(ctx, TACAW_EINVAL, "timeout_ms must be in (0, 1000]");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaSetDevice");
  k_wait_selftest<<<1, 32, 0, (cudaStream_t)stream>>>(ctx->d_status, (unsigned long long)(timeout_ms * 1e6));
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(ctx, e, "k_wait_selftest");
  return TACAW_OK;
}
