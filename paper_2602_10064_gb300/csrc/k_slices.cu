// Slice kernels: binning, projected potential, transmission, probe and the multislice step.
//
// Every 2D transform is a row pass (FFT along x inside one CTA per G rows) followed by a column
// pass (FFT along y inside one CTA per C columns); pointwise work is fused into the passes:
//   potential  (Methods, "Atomic Scattering Potentials"):
//     spread atoms -> FFT_x | FFT_y, * C M (f_A - i f_B)/Phi, IFFT_y | IFFT_x, Re -> V
//   transmission (Methods, "Multislice Propagation", t = exp(i sigma V)):
//     exp(i sigma V) -> FFT_x | FFT_y, * M / Nq, IFFT_y | IFFT_x -> t
//   slice step  (same section, psi <- IDFT(P M DFT(t psi))):
//     [IFFT_x] * t, FFT_x | FFT_y, * P M / Nq, IFFT_y    (the IFFT_x of slice s is fused into
//     the row pass of slice s+1; the last column pass writes psi(k) without the inverse)
// Between the passes only the in-band columns (|kx| <= kbl) are kept, in compact order.
#include <cuda_runtime.h>

#include "fft.cuh"
#include "tacaw_internal.cuh"

namespace tacaw {

// Per-kernel variants of the FFT pass kernels, chosen per transform length by the autotuner
// (paper_2602_10064_gb300/tune.py), which times every variant on GB300 and writes
// tuning_table.h.  Variant bits: 1 = radix-8 plans (512 and 1024 points, 16 elements per
// thread), 2 = 1.5 times as many resident threads per SM (fewer registers each), 4 = column
// passes only: twice the columns per CTA, so that each load instruction covers whole 128-byte
// lines, 8 = 32 elements per thread for the powers of two from 128 points (two-pass
// transforms, about 170 registers).  TACAW_TUNE_FORCE=v builds every kernel as variant v (the
// tuner's measurement builds).
enum KernelId {
  K_SPLAT_ROW, K_COL_POT, K_ROW_POT_OUT, K_ROW_VT, K_COL_T, K_ROW_TOUT, K_PROBE_COL, K_PROBE_ROW,
  K_SLICE_ROW, K_SLICE_COL
};
}  // namespace tacaw
#include "tuning_table.h"
namespace tacaw {
#ifndef TACAW_TUNE_FORCE
#define TACAW_TUNE_FORCE -1
#endif
template <int K, int N>
struct Tuned {
  static constexpr int V = TACAW_TUNE_FORCE >= 0 ? TACAW_TUNE_FORCE : tuned_variant(K, N);
  static constexpr bool COLUMN = K == K_COL_POT || K == K_COL_T || K == K_PROBE_COL || K == K_SLICE_COL;
  static constexpr int EV = (V & 8) ? 1 : 0;
  static constexpr int PLAN = (V & 1) && !EV;
  static constexpr int WIDE = (COLUMN && (V & 4)) ? 1 : 0;
  // resident CTAs per SM requested for a CTA of `threads`: `target` threads per SM (variant & 2:
  // 1.5 times as many)
  __host__ __device__ static constexpr int minb(int threads, int target) {
    return ((V & 2) ? target * 3 / 2 : target) / threads > 1 ? ((V & 2) ? target * 3 / 2 : target) / threads : 1;
  }
};

// Elements per thread of the row and of the column transforms (8 or 16).
#ifndef TACAW_ROW_E
#define TACAW_ROW_E 16
#endif
#ifndef TACAW_COL_E
#define TACAW_COL_E 16
#endif

// Largest power of two <= x (x >= 1).
__host__ __device__ constexpr int floor_pow2(int x) {
  int p = 1;
  while (2 * p <= x) p *= 2;
  return p;
}

// Row passes: G rows per CTA, one transform group of T threads per row.  Transforms of 24
// elements per thread need about 170 registers, so those CTAs are smaller and the SM holds
// 384 instead of 512 threads (TARGET).
// EV = 1: 32 elements per thread (two-pass transforms) for the powers of two from 128 points.
template <int N, int EV = 0>
struct RowCfg {
  static constexpr int E = (EV && fft_pow2(N) && N >= 128) ? 32 : FftPlan<N, TACAW_ROW_E>::E;
  static constexpr int T = N / E;
  static constexpr int TARGET = E >= 24 ? 384 : 512;
  static constexpr int G0 = (TARGET / 2) / T;
  static constexpr int G = G0 > 32 ? 32 : (G0 < 1 ? 1 : floor_pow2(G0));  // rows per CTA
  static constexpr int THREADS = G * T;
  static constexpr int SMEM = G * row_smem_stride<N, E>() * (int)sizeof(float2);
};

// Column passes: C columns per CTA (about 256 threads; WIDE doubles C, about 512 threads).
template <int N, int WIDE = 0, int EV = 0>
struct ColCfg {
  static constexpr int E = (EV && fft_pow2(N) && N >= 128) ? 32 : FftPlan<N, TACAW_COL_E>::E;
  static constexpr int T = N / E;
  static constexpr int TARGET = E >= 24 ? 384 : 512;
  static constexpr int C0 = ((TARGET / 2) << WIDE) / T;
  static constexpr int C = C0 > 32 ? 32 : (C0 < 4 ? 4 : floor_pow2(C0));  // columns per CTA (divides Wp)
  static constexpr int THREADS = C * T;
  // padding of the interleaved columns: measured to pay only with 32 elements per thread
  static constexpr int SH = E == 32 ? 5 : 0;
  static constexpr int SMEM = (N + (SH ? (N >> SH) : 0)) * C * (int)sizeof(float2);
};

// The configuration of each pass kernel; a kernel and its launcher name the same alias.
template <int N> using SplatCfg = RowCfg<N, Tuned<K_SPLAT_ROW, N>::EV>;
template <int N> using PotOutCfg = RowCfg<N, Tuned<K_ROW_POT_OUT, N>::EV>;
template <int N> using RowVtCfg = RowCfg<N, Tuned<K_ROW_VT, N>::EV>;
template <int N> using RowToutCfg = RowCfg<N, Tuned<K_ROW_TOUT, N>::EV>;
template <int N> using ProbeRowCfg = RowCfg<N, Tuned<K_PROBE_ROW, N>::EV>;
template <int N> using SliceRowCfg = RowCfg<N, Tuned<K_SLICE_ROW, N>::EV>;
template <int N> using ColPotCfg = ColCfg<N, Tuned<K_COL_POT, N>::WIDE, Tuned<K_COL_POT, N>::EV>;
template <int N> using ColTCfg = ColCfg<N, Tuned<K_COL_T, N>::WIDE, Tuned<K_COL_T, N>::EV>;
template <int N> using ProbeColCfg = ColCfg<N, Tuned<K_PROBE_COL, N>::WIDE, Tuned<K_PROBE_COL, N>::EV>;
template <int N> using SliceColCfg = ColCfg<N, Tuned<K_SLICE_COL, N>::WIDE, Tuned<K_SLICE_COL, N>::EV>;

// Resident CTAs per SM requested from the compiler for kernel K with configuration Cfg.
template <int K, int N, class Cfg>
__host__ __device__ constexpr int minb_of() {
  return Tuned<K, N>::minb(Cfg::THREADS, Cfg::TARGET);
}

// Barrier of one row transform: the group's own (warp, or named barrier over whole warps), or
// the CTA barrier when a group of T threads is not made of whole warps (T = 48: 1152 points).
template <int T>
__device__ __forceinline__ auto group_sync(int g) {
  if constexpr (T <= 32 || T % 32 == 0) return GroupSync<T>{1 + g};
  else return BlockSync{};
}

// CTAs of a column pass: the in-band columns c < W only, C per CTA.  The padding columns up to Wp
// are never read by a row pass (band_x_col maps no x to them), so they need no transform.
static int col_blocks(const Band& b, int C) { return (b.W + C - 1) / C; }

// Batch index over (grid.y, grid.z); batches beyond nb return before any barrier.
__device__ __forceinline__ int batch_index() { return blockIdx.y + gridDim.y * blockIdx.z; }
static dim3 batch_grid(int gx, int64_t nb) {
  unsigned y = (unsigned)(nb < 65535 ? nb : 65535);
  unsigned z = (unsigned)((nb + y - 1) / y);
  return dim3((unsigned)gx, y, z);
}

template <int N, int E>
__device__ __forceinline__ void load_row_compact(float2 (&v)[E], const float2* __restrict__ src, const Band& b,
                                                 int t) {
  constexpr int T = N / E;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int c = band_x_col(b, N, t + T * e);
    v[e] = c >= 0 ? src[c] : make_float2(0.f, 0.f);
  }
}

template <int N, int E>
__device__ __forceinline__ void store_row_compact(const float2 (&v)[E], float2* __restrict__ dst, const Band& b,
                                                  int t) {
  constexpr int T = N / E;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int c = band_x_col(b, N, t + T * e);
    if (c >= 0) dst[c] = v[e];
  }
}

// The same with the band's half-width MB known at compile time (W = 2 MB + 1): the element e of
// every thread covers positions [T e, T e + T), so whether it is in band, out of band or split
// is decided per e at compile time, and only the split elements keep a per-thread test.
template <int N, int E, int MB>
__device__ __forceinline__ void load_row_band(float2 (&v)[E], const float2* __restrict__ src, int t) {
  constexpr int T = N / E, W = 2 * MB + 1;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int x = t + T * e;
    if (T * e + T - 1 <= MB) {
      v[e] = src[x];
    } else if (T * e >= N - MB) {
      v[e] = src[x - N + W];
    } else if (T * e > MB && T * e + T - 1 < N - MB) {
      v[e] = make_float2(0.f, 0.f);
    } else {
      const int c = x <= MB ? x : (x >= N - MB ? x - N + W : -1);
      v[e] = c >= 0 ? src[c] : make_float2(0.f, 0.f);
    }
  }
}

template <int N, int E, int MB>
__device__ __forceinline__ void store_row_band(const float2 (&v)[E], float2* __restrict__ dst, int t) {
  constexpr int T = N / E, W = 2 * MB + 1;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int x = t + T * e;
    if (T * e + T - 1 <= MB) {
      dst[x] = v[e];
    } else if (T * e >= N - MB) {
      dst[x - N + W] = v[e];
    } else if (!(T * e > MB && T * e + T - 1 < N - MB)) {
      const int c = x <= MB ? x : (x >= N - MB ? x - N + W : -1);
      if (c >= 0) dst[c] = v[e];
    }
  }
}

// The compact row accessors with the band's half-width fixed at compile time (MB >= 0) or
// read from b (MB < 0).
template <int N, int MB, int E>
__device__ __forceinline__ void load_row(float2 (&v)[E], const float2* __restrict__ src, const Band& b, int t) {
  if constexpr (MB >= 0) load_row_band<N, E, MB>(v, src, t);
  else load_row_compact<N>(v, src, b, t);
}
template <int N, int MB, int E>
__device__ __forceinline__ void store_row(const float2 (&v)[E], float2* __restrict__ dst, const Band& b, int t) {
  if constexpr (MB >= 0) store_row_band<N, E, MB>(v, dst, t);
  else store_row_compact<N>(v, dst, b, t);
}

// ============================================================================================
// a1: slice binning.  One CTA per frame; stable scatter, so every slice list keeps atom order.
// ============================================================================================
constexpr int BIN_THREADS = 1024;
constexpr int BIN_MAX_S = 256;

__device__ __forceinline__ int slice_of(double z, double Lz, int S) {
  const double dz = Lz / (double)S;
  const double zw = __dsub_rn(z, __dmul_rn(Lz, floor(z / Lz)));
  int s = (int)floor(zw / dz);
  if (s >= S) s = S - 1;
  if (s < 0) s = 0;
  return s;
}

__device__ __forceinline__ void grid_coord(double x, double L, int n, int& i0, float& fr) {
  const double xw = __dsub_rn(x, __dmul_rn(L, floor(x / L)));
  const double u = __dmul_rn(xw, (double)n / L);
  double fl = floor(u);
  int i = (int)fl;
  double f = __dsub_rn(u, fl);
  if (i >= n) { i -= n; }
  if (i < 0) { i += n; }
  i0 = i;
  fr = (float)f;
}

__global__ void __launch_bounds__(BIN_THREADS) k_bin(const float* __restrict__ pos, int A, int S, double Lx,
                                                      double Ly, double Lz, int nx, int ny,
                                                      const int8_t* __restrict__ slot_of_atom,
                                                      AtomRec* __restrict__ recs, int* __restrict__ offs,
                                                      int* __restrict__ slice_out) {
  __shared__ int counts[BIN_MAX_S];
  __shared__ int cursor[BIN_MAX_S];
  __shared__ int wcount[BIN_THREADS / 32][BIN_MAX_S];
  const int f = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const float* P = pos + (size_t)f * A * 3;
  for (int s = tid; s < S; s += BIN_THREADS) counts[s] = 0;
  __syncthreads();
  for (int j = tid; j < A; j += BIN_THREADS) {
    const int s = slice_of((double)P[3 * j + 2], Lz, S);
    atomicAdd(&counts[s], 1);
    if (slice_out) slice_out[(size_t)f * A + j] = s;
  }
  __syncthreads();
  if (tid == 0) {
    int run = 0;
    for (int s = 0; s < S; ++s) {
      offs[(size_t)f * (S + 1) + s] = run;
      cursor[s] = run;
      run += counts[s];
    }
    offs[(size_t)f * (S + 1) + S] = run;
  }
  if (!recs) return;
  const unsigned lt = (1u << lane) - 1u;
  for (int base = 0; base < A; base += BIN_THREADS) {
    for (int i = tid; i < (BIN_THREADS / 32) * S; i += BIN_THREADS) wcount[i / S][i % S] = 0;
    __syncthreads();
    const int j = base + tid;
    const bool valid = j < A;
    const int s = valid ? slice_of((double)P[3 * j + 2], Lz, S) : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, s);
    const int rank = __popc(peers & lt);
    if (valid && rank == 0) wcount[w][s] = __popc(peers);
    __syncthreads();
    for (int ss = tid; ss < S; ss += BIN_THREADS) {
      int run = cursor[ss];
      for (int ww = 0; ww < BIN_THREADS / 32; ++ww) {
        const int c = wcount[ww][ss];
        wcount[ww][ss] = run;
        run += c;
      }
      cursor[ss] = run;
    }
    __syncthreads();
    if (valid) {
      const int p = wcount[w][s] + rank;
      AtomRec r;
      int ix, iy;
      grid_coord((double)P[3 * j], Lx, nx, ix, r.fx);
      grid_coord((double)P[3 * j + 1], Ly, ny, iy, r.fy);
      r.ixy = ix | (iy << 16);
      r.jslot = j | ((int)slot_of_atom[j] << 24);
      recs[(size_t)f * A + p] = r;
    }
    __syncthreads();
  }
}

__global__ void k_map_slots(const int32_t* __restrict__ Z, int64_t A, const int8_t* __restrict__ lut,
                            int8_t* __restrict__ slot, int* __restrict__ status) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < A; j += (int64_t)gridDim.x * blockDim.x) {
    const int z = Z[j];
    int s = (z >= 0 && z < 256) ? lut[z] : -1;
    if (s < 0) {
      atomicOr(status, TACAW_STATUS_SPECIES);
      s = 0;
    }
    slot[j] = (int8_t)s;
  }
}

cudaError_t launch_map_slots(const int32_t* Z, int64_t A, const int8_t* lut, int8_t* slot, int* status,
                             cudaStream_t st) {
  if (A <= 0) return cudaSuccess;
  const int64_t blocks = (A + 255) / 256;
  k_map_slots<<<(unsigned)(blocks < 1024 ? blocks : 1024), 256, 0, st>>>(Z, A, lut, slot, status);
  return cudaGetLastError();
}

// One warp per (frame, slice): stable counting sort of the slice's atom records by the grid
// row of their coordinate, and the offsets of each block of SPREAD_YB rows, so that the
// spreading pass reads only the atoms whose footprint can reach its rows.  Order within a row
// is the binning order (atom index), so the spreading sums stay deterministic.
constexpr int SORT_WARPS = 8;
__global__ void __launch_bounds__(SORT_WARPS * 32)
    k_sort_rows(const AtomRec* __restrict__ recs, const int* __restrict__ offs, int A, int S, int nseg, int ny,
                AtomRec* __restrict__ out, int* __restrict__ boffs) {
  extern __shared__ int cnt_all[];  // [SORT_WARPS][ny]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int seg = blockIdx.x * SORT_WARPS + warp;
  if (seg >= nseg) return;  // whole warps; only warp-level barriers below
  int* cnt = cnt_all + warp * ny;
  const int f = seg / S, s = seg - f * S;
  const int lo = offs[(size_t)f * (S + 1) + s], hi = offs[(size_t)f * (S + 1) + s + 1];
  const AtomRec* R = recs + (size_t)f * A;
  AtomRec* O = out + (size_t)f * A;
  const int nyb = ny / SPREAD_YB;
  int* bo = boffs + (size_t)seg * (nyb + 1);
  for (int y = lane; y < ny; y += 32) cnt[y] = 0;
  __syncwarp();
  for (int j = lo + lane; j < hi; j += 32) atomicAdd(&cnt[R[j].ixy >> 16], 1);
  __syncwarp();
  int run = lo;  // exclusive scan over rows; block offsets at multiples of SPREAD_YB
  for (int y0 = 0; y0 < ny; y0 += 32) {
    const int y = y0 + lane;
    const int c = y < ny ? cnt[y] : 0;
    int x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int n = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += n;
    }
    if (y < ny) {
      cnt[y] = run + x - c;
      if (y % SPREAD_YB == 0) bo[y / SPREAD_YB] = run + x - c;
    }
    run += __shfl_sync(0xffffffffu, x, 31);
  }
  if (lane == 0) bo[nyb] = hi;
  __syncwarp();
  const unsigned below = (1u << lane) - 1u;
  for (int base = lo; base < hi; base += 32) {  // 32 records at a time, in order: stable
    const int j = base + lane;
    const bool valid = j < hi;
    AtomRec r;
    int key = -1 - lane;  // distinct for the lanes past the end
    if (valid) {
      r = R[j];
      key = r.ixy >> 16;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int leader = __ffs(peers) - 1;
    int pos = 0;
    if (valid && lane == leader) {
      pos = cnt[key];
      cnt[key] = pos + __popc(peers);
    }
    pos = __shfl_sync(0xffffffffu, pos, leader) + __popc(peers & below);
    if (valid) O[pos] = r;
    __syncwarp();
  }
}

cudaError_t launch_sort_rows(const AtomRec* recs, const int* offs, int64_t A, int64_t nf, int S, int ny,
                             AtomRec* out, int* boffs, cudaStream_t st) {
  if (ny % SPREAD_YB != 0 || nf <= 0) return cudaErrorInvalidValue;
  const int64_t nseg = nf * S;
  const int smem = SORT_WARPS * ny * (int)sizeof(int);
  if (smem > 46 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(k_sort_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  k_sort_rows<<<(unsigned)((nseg + SORT_WARPS - 1) / SORT_WARPS), SORT_WARPS * 32, smem, st>>>(
      recs, offs, (int)A, S, (int)nseg, ny, out, boffs);
  return cudaGetLastError();
}

cudaError_t launch_bin(const float* pos, int64_t A, int64_t nf, int S, double Lx, double Ly, double Lz, int nx,
                       int ny, const int8_t* slot_of_atom, AtomRec* recs, int* offs, int* slice_out,
                       cudaStream_t st) {
  if (S > BIN_MAX_S || nf <= 0) return cudaErrorInvalidValue;
  k_bin<<<(unsigned)nf, BIN_THREADS, 0, st>>>(pos, (int)A, S, Lx, Ly, Lz, nx, ny, slot_of_atom, recs, offs,
                                             slice_out);
  return cudaGetLastError();
}

// ============================================================================================
// a2: potential.  Row pass: spread the atoms of one slice and one species pair onto G rows
// (gather per grid point, candidates in atom order, so the sum is deterministic), then FFT_x.
// ============================================================================================
// x mod n for 0 <= x < 3 n (any n, no division).
__device__ __forceinline__ int wrap3(int x, int n) {
  x -= (x >= n) ? n : 0;
  return x - ((x >= n) ? n : 0);
}
// The same for a compile-time n (a mask when n is a power of two).
template <int N>
__device__ __forceinline__ int wrap3(int x) {
  if constexpr (fft_pow2(N)) return x & (N - 1);
  else return wrap3(x, N);
}

__device__ __forceinline__ float es_kernel(float z, float beta) {
  const float a = 1.f - z * z;
  return a > 0.f ? expf(beta * (sqrtf(a) - 1.f)) : 0.f;
}

constexpr int SPREAD_MAX_W = 16;

// Shared memory of the spreading row pass: per-row accumulators (each element owned by one
// thread, so the sums are race-free and in candidate order), then the candidate tables.
template <int NX>
struct SplatSmem {
  static constexpr int NT = SplatCfg<NX>::THREADS, G = SplatCfg<NX>::G;
  static constexpr int ACC = G * NX * 8;
  static constexpr int TAB = NT * (SPREAD_MAX_W + G) * 4 + NT * 4 * 4;
  static constexpr int BYTES = (ACC + TAB) > SplatCfg<NX>::SMEM ? (ACC + TAB) : SplatCfg<NX>::SMEM;
};

template <int NX, int MB = -1>
__global__ void __launch_bounds__(SplatCfg<NX>::THREADS, minb_of<K_SPLAT_ROW, NX, SplatCfg<NX>>())
    k_splat_row(Geo geo, Band b, const AtomRec* __restrict__ recs, const int* __restrict__ boffs, int A, int S,
                int s0, int sb, int npair, int nbatch, SpreadKernel sk, float2* __restrict__ Bp) {
  constexpr int E = SplatCfg<NX>::E, T = SplatCfg<NX>::T, G = SplatCfg<NX>::G, NT = SplatCfg<NX>::THREADS;
  constexpr int PL = Tuned<K_SPLAT_ROW, NX>::PLAN;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = reinterpret_cast<float2*>(smraw);                     // FFT scratch (after spreading)
  float2* acc = reinterpret_cast<float2*>(smraw);                    // [G][NX]
  float* phx = reinterpret_cast<float*>(smraw + SplatSmem<NX>::ACC); // [NT][SPREAD_MAX_W]
  float* phy = phx + NT * SPREAD_MAX_W;                               // [NT][G]
  float* cfx = phy + NT * G;                                          // [NT] candidate records
  float* cfy = cfx + NT;
  int* cx0 = reinterpret_cast<int*>(cfy + NT);                        // first footprint column
  int* ciy = cx0 + NT;                                                // iy0 | imag << 16, -1: other pair

  const int bidx = batch_index();
  if (bidx >= nbatch) return;
  const int pair = bidx % npair, fs = bidx / npair, f = fs / sb, s = s0 + fs % sb;
  const int tid = threadIdx.x, g = tid / T, t = tid % T;
  const int ny = geo.ny, y0 = blockIdx.x * G;
  const int h = sk.half, W2 = 2 * h;
  const AtomRec* R = recs + (size_t)f * A;
  // candidates: the atoms of the row blocks covering rows [y0 - h, y0 + G - 2 + h] (their
  // footprints [iy0 + 1 - h, iy0 + h] meet rows [y0, y0 + G)), at most two contiguous ranges of
  // the row-sorted slice list (the window may wrap around y = 0)
  const int nyb = ny / SPREAD_YB;
  const int* bo = boffs + ((size_t)f * S + s) * (nyb + 1);
  const int wlo = y0 - h, whi = y0 + G - 2 + h;
  const int b_lo = wlo >= 0 ? wlo / SPREAD_YB : -((-wlo + SPREAD_YB - 1) / SPREAD_YB), b_hi = whi / SPREAD_YB;
  int s1, n1, s2 = 0, n2 = 0;
  if (b_hi - b_lo + 1 >= nyb) {
    s1 = bo[0];
    n1 = bo[nyb] - s1;
  } else if (b_lo < 0) {
    s1 = bo[b_lo + nyb];
    n1 = bo[nyb] - s1;
    s2 = bo[0];
    n2 = bo[b_hi + 1] - s2;
  } else if (b_hi >= nyb) {
    s1 = bo[b_lo];
    n1 = bo[nyb] - s1;
    s2 = bo[0];
    n2 = bo[b_hi - nyb + 1] - s2;
  } else {
    s1 = bo[b_lo];
    n1 = bo[b_hi + 1] - s1;
  }
  const int M = n1 + n2;

#pragma unroll
  for (int e = 0; e < E; ++e) acc[g * NX + t + T * e] = make_float2(0.f, 0.f);

  for (int base = 0; base < M; base += NT) {
    // 1. the batch's candidate records (atoms of other species pairs are marked and skipped)
    const int j = base + tid;
    if (j < M) {
      const AtomRec r = R[j < n1 ? s1 + j : s2 + (j - n1)];
      const int slot = r.jslot >> 24;
      cfx[tid] = r.fx;
      cfy[tid] = r.fy;
      cx0[tid] = wrap3<NX>((r.ixy & 0xffff) + 1 - h + NX);
      ciy[tid] = (slot >> 1) == pair ? ((r.ixy >> 16) | ((slot & 1) << 16)) : -1;
    }
    __syncthreads();
    const int total = M - base < NT ? M - base : NT;
    // 2. kernel tables, one entry per thread: phx[c][d] (d < 2h) and phy[c][g]
    const int per = W2 + G;
    for (int i = tid; i < total * per; i += NT) {
      const int c = i / per, k = i - c * per;
      if (k < W2) {
        phx[c * SPREAD_MAX_W + k] = es_kernel(((float)(k + 1 - h) - cfx[c]) / (float)h, sk.beta);
      } else {
        const int gg = k - W2, cy = ciy[c];
        int d = wrap3(y0 + gg - (cy & 0xffff) + ny, ny);
        if (d > ny / 2) d -= ny;
        phy[c * G + gg] = (cy >= 0 && d >= 1 - h && d <= h) ? es_kernel(((float)d - cfy[c]) / (float)h, sk.beta)
                                                           : 0.f;
      }
    }
    __syncthreads();
    // 3. taps: thread (g, t) owns columns t + T e; a footprint of 2h columns starting at x0
    //    meets them at the offsets congruent to t - x0 modulo T
    float2* arow = acc + g * NX;
    for (int c = 0; c < total; ++c) {
      const float wy = phy[c * G + g];
      if (wy == 0.f) continue;
      const int x0 = cx0[c];
      const bool im = (ciy[c] >> 16) != 0;
      const int d = wrap3<NX>(x0 - t + NX);
      for (int off = (T - d % T) % T; off < W2; off += T) {
        const int x = wrap3<NX>(x0 + off);
        const float a = wy * phx[c * SPREAD_MAX_W + off];
        if (im) arow[x].y += a;
        else arow[x].x += a;
      }
    }
    __syncthreads();
  }
  float2 v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) v[e] = acc[g * NX + t + T * e];
  __syncthreads();  // the FFT scratch of one group overlaps the accumulators of the next
  fft<NX, -1, PL>(v, sm, RowIdx<NX, E>{g * row_smem_stride<NX, E>()}, t, geo.tw + tw_offset(NX),
                  group_sync<T>(g));
  store_row<NX, MB>(v, Bp + ((size_t)bidx * ny + y0 + g) * b.Wp, b, t);
}

// Column pass of the potential: per (f, s), sum over species pairs of mtab * FFT_y, then IFFT_y.
template <int NY, bool ONE, int WPC = -1>
__global__ void __launch_bounds__(ColPotCfg<NY>::THREADS, minb_of<K_COL_POT, NY, ColPotCfg<NY>>())
    k_col_pot(Geo geo, Band b, const float2* __restrict__ Bp, const float2* __restrict__ mtab, int npair, int nbatch,
              float2* __restrict__ Ap) {
  using CC = ColPotCfg<NY>;
  constexpr int E = CC::E, T = CC::T, C = CC::C;
  constexpr int PL = Tuned<K_COL_POT, NY>::PLAN;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = reinterpret_cast<float2*>(smraw);
  const int fs = batch_index();
  if (fs >= nbatch) return;
  const int Wp = WPC > 0 ? WPC : b.Wp;
  const int c = threadIdx.x % C, t = threadIdx.x / C, cc = blockIdx.x * C + c;
  const ColIdx<C, CC::SH> idx{c};
  const BlockSync sync;
  const float2* tw = geo.tw + tw_offset(NY);
  if constexpr (ONE) {
    // one species pair: no accumulator held across the transforms
    const float2* src = Bp + (size_t)fs * NY * Wp + cc;
    float2 v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = src[(size_t)(t + T * e) * Wp];
    fft<NY, -1, PL>(v, sm, idx, t, tw, sync);
    const float2* m = mtab + cc;
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = cmul(m[(size_t)(t + T * e) * Wp], v[e]);
    fft<NY, +1, PL>(v, sm, idx, t, tw, sync);
    float2* dst = Ap + (size_t)fs * NY * Wp + cc;
#pragma unroll
    for (int e = 0; e < E; ++e) dst[(size_t)(t + T * e) * Wp] = v[e];
  } else {
    float2 acc[E];
#pragma unroll
    for (int e = 0; e < E; ++e) acc[e] = make_float2(0.f, 0.f);
    for (int pr = 0; pr < npair; ++pr) {
      const float2* src = Bp + (size_t)(fs * npair + pr) * NY * Wp + cc;
      float2 v[E];
#pragma unroll
      for (int e = 0; e < E; ++e) v[e] = src[(size_t)(t + T * e) * Wp];
      fft<NY, -1, PL>(v, sm, idx, t, tw, sync);
      const float2* m = mtab + (size_t)pr * NY * Wp + cc;
#pragma unroll
      for (int e = 0; e < E; ++e) acc[e] = acc[e] + cmul(m[(size_t)(t + T * e) * Wp], v[e]);
    }
    fft<NY, +1, PL>(acc, sm, idx, t, tw, sync);
    float2* dst = Ap + (size_t)fs * NY * Wp + cc;
#pragma unroll
    for (int e = 0; e < E; ++e) dst[(size_t)(t + T * e) * Wp] = acc[e];
  }
}

// Row pass out of the potential: IFFT_x, real part = V.  mode 0 stores V; mode 1 forms
// t = exp(i sigma V) and runs FFT_x for the transmission band limit; mode 2 stores t.
template <int NX, int MB = -1>
__global__ void __launch_bounds__(PotOutCfg<NX>::THREADS, minb_of<K_ROW_POT_OUT, NX, PotOutCfg<NX>>())
    k_row_pot_out(Geo geo, Band b, const float2* __restrict__ Ap, int nbatch, int mode, float sigma,
                  float* __restrict__ V, float2* __restrict__ out) {
  constexpr int E = PotOutCfg<NX>::E, T = PotOutCfg<NX>::T, G = PotOutCfg<NX>::G;
  constexpr int PL = Tuned<K_ROW_POT_OUT, NX>::PLAN;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = reinterpret_cast<float2*>(smraw);
  const int fs = batch_index();
  if (fs >= nbatch) return;
  const int g = threadIdx.x / T, t = threadIdx.x % T, y = blockIdx.x * G + g, ny = geo.ny;
  const RowIdx<NX, E> idx{g * row_smem_stride<NX, E>()};
  const auto sync = group_sync<T>(g);
  float2 v[E];
  load_row<NX, MB>(v, Ap + ((size_t)fs * ny + y) * b.Wp, b, t);
  fft<NX, +1, PL>(v, sm, idx, t, geo.tw + tw_offset(NX), sync);
  const size_t row = ((size_t)fs * ny + y) * NX;
  if (mode == 0) {
#pragma unroll
    for (int e = 0; e < E; ++e) V[row + t + T * e] = v[e].x;
    return;
  }
#pragma unroll
  for (int e = 0; e < E; ++e) {
    float sn, cs;
    sincosf(sigma * v[e].x, &sn, &cs);
    v[e] = make_float2(cs, sn);
  }
  if (mode == 2) {
#pragma unroll
    for (int e = 0; e < E; ++e) out[row + t + T * e] = v[e];
    return;
  }
  fft<NX, -1, PL>(v, sm, idx, t, geo.tw + tw_offset(NX), sync);
  store_row<NX, MB>(v, out + ((size_t)fs * ny + y) * b.Wp, b, t);
}

// ============================================================================================
// a3: transmission from a stored V.
// ============================================================================================
template <int NX>
__global__ void __launch_bounds__(RowVtCfg<NX>::THREADS, minb_of<K_ROW_VT, NX, RowVtCfg<NX>>())
    k_row_vt(Geo geo, Band b, const float* __restrict__ V, int nbatch, int bandlimit, float sigma,
             float2* __restrict__ out) {
  constexpr int E = RowVtCfg<NX>::E, T = RowVtCfg<NX>::T, G = RowVtCfg<NX>::G;
  constexpr int PL = Tuned<K_ROW_VT, NX>::PLAN;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = reinterpret_cast<float2*>(smraw);
  const int fs = batch_index();
  if (fs >= nbatch) return;
  const int g = threadIdx.x / T, t = threadIdx.x % T, y = blockIdx.x * G + g, ny = geo.ny;
  const size_t row = ((size_t)fs * ny + y) * NX;
  float2 v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    float sn, cs;
    sincosf(sigma * V[row + t + T * e], &sn, &cs);
    v[e] = make_float2(cs, sn);
  }
  if (!bandlimit) {
#pragma unroll
    for (int e = 0; e < E; ++e) out[row + t + T * e] = v[e];
    return;
  }
  fft<NX, -1, PL>(v, sm, RowIdx<NX, E>{g * row_smem_stride<NX, E>()}, t, geo.tw + tw_offset(NX),
                  group_sync<T>(g));
  store_row_compact<NX>(v, out + ((size_t)fs * ny + y) * b.Wp, b, t);
}

// Column pass of the band limit: FFT_y, * M * scale, IFFT_y.
template <int NY, int WPC = -1>
__global__ void __launch_bounds__(ColTCfg<NY>::THREADS, minb_of<K_COL_T, NY, ColTCfg<NY>>())
    k_col_t(Geo geo, Band b, const float2* __restrict__ Bt, int nbatch, float scale, float2* __restrict__ At) {
  using CC = ColTCfg<NY>;
  constexpr int E = CC::E, T = CC::T, C = CC::C;
  constexpr int PL = Tuned<K_COL_T, NY>::PLAN;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = reinterpret_cast<float2*>(smraw);
  const int fs = batch_index();
  if (fs >= nbatch) return;
  const int Wp = WPC > 0 ? WPC : b.Wp;
  const int c = threadIdx.x % C, t = threadIdx.x / C, cc = blockIdx.x * C + c;
  const ColIdx<C, CC::SH> idx{c};
  const BlockSync sync;
  const float2* tw = geo.tw + tw_offset(NY);
  const float2* src = Bt + (size_t)fs * NY * Wp + cc;
  float2 v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) v[e] = src[(size_t)(t + T * e) * Wp];
  fft<NY, -1, PL>(v, sm, idx, t, tw, sync);
  const int nb = cc < b.W ? b.colnb[cc] : -1;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int n = fftfreq_index(t + T * e, NY);
    v[e] = (abs(n) <= nb) ? scale * v[e] : make_float2(0.f, 0.f);
  }
  fft<NY, +1, PL>(v, sm, idx, t, tw, sync);
  float2* dst = At + (size_t)fs * NY * Wp + cc;
#pragma unroll
  for (int e = 0; e < E; ++e) dst[(size_t)(t + T * e) * Wp] = v[e];
}

// Row pass out of the band limit: IFFT_x -> t (full row).
template <int NX>
__global__ void __launch_bounds__(RowToutCfg<NX>::THREADS, minb_of<K_ROW_TOUT, NX, RowToutCfg<NX>>())
    k_row_tout(Geo geo, Band b, const float2* __restrict__ At, int nbatch, float2* __restrict__ tout) {
  constexpr int E = RowToutCfg<NX>::E, T = RowToutCfg<NX>::T, G = RowToutCfg<NX>::G;
  constexpr int PL = Tuned<K_ROW_TOUT, NX>::PLAN;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = reinterpret_cast<float2*>(smraw);
  const int fs = batch_index();
  if (fs >= nbatch) return;
  const int g = threadIdx.x / T, t = threadIdx.x % T, y = blockIdx.x * G + g, ny = geo.ny;
  float2 v[E];
  load_row_compact<NX>(v, At + ((size_t)fs * ny + y) * b.Wp, b, t);
  fft<NX, +1, PL>(v, sm, RowIdx<NX, E>{g * row_smem_stride<NX, E>()}, t, geo.tw + tw_offset(NX),
                  group_sync<T>(g));
  float2* dst = tout + ((size_t)fs * ny + y) * NX;
#pragma unroll
  for (int e = 0; e < E; ++e) dst[t + T * e] = v[e];
}

// ============================================================================================
// Probe: psi0(k) = A(k) exp(-2 pi i k.r_p) amp, then a unitary inverse transform.
// ============================================================================================
template <int NY>
__global__ void __launch_bounds__(ProbeColCfg<NY>::THREADS, minb_of<K_PROBE_COL, NY, ProbeColCfg<NY>>())
    k_probe_col(Geo geo, Band ap, const float2* __restrict__ ex, const float2* __restrict__ ey,
                const float2* __restrict__ chi, int P, float amp, float2* __restrict__ Bpr) {
  using CC = ProbeColCfg<NY>;
  constexpr int E = CC::E, T = CC::T, C = CC::C;
  constexpr int PL = Tuned<K_PROBE_COL, NY>::PLAN;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = reinterpret_cast<float2*>(smraw);
  const int p = batch_index();
  if (p >= P) return;
  const int c = threadIdx.x % C, t = threadIdx.x / C, cc = blockIdx.x * C + c;
  const int nb = cc < ap.W ? ap.colnb[cc] : -1;
  const float2 exv = cc < ap.W ? ex[(size_t)p * ap.Wp + cc] : make_float2(0.f, 0.f);
  float2 v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int row = t + T * e, n = fftfreq_index(row, NY);
    v[e] = (abs(n) <= nb) ? amp * cmul(exv, ey[(size_t)p * NY + row]) : make_float2(0.f, 0.f);
    if (chi && abs(n) <= nb) v[e] = cmul(v[e], chi[(size_t)row * ap.Wp + cc]);
  }
  fft<NY, +1, PL>(v, sm, ColIdx<C, CC::SH>{c}, t, geo.tw + tw_offset(NY), BlockSync{});
  float2* dst = Bpr + (size_t)p * NY * ap.Wp + cc;
#pragma unroll
  for (int e = 0; e < E; ++e) dst[(size_t)(t + T * e) * ap.Wp] = v[e];
}

template <int NX>
__global__ void __launch_bounds__(ProbeRowCfg<NX>::THREADS, minb_of<K_PROBE_ROW, NX, ProbeRowCfg<NX>>())
    k_probe_row(Geo geo, Band ap, const float2* __restrict__ Bpr, int P, float scale, float2* __restrict__ psi0) {
  constexpr int E = ProbeRowCfg<NX>::E, T = ProbeRowCfg<NX>::T, G = ProbeRowCfg<NX>::G;
  constexpr int PL = Tuned<K_PROBE_ROW, NX>::PLAN;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = reinterpret_cast<float2*>(smraw);
  const int p = batch_index();
  if (p >= P) return;
  const int g = threadIdx.x / T, t = threadIdx.x % T, y = blockIdx.x * G + g, ny = geo.ny;
  float2 v[E];
  load_row_compact<NX>(v, Bpr + ((size_t)p * ny + y) * ap.Wp, ap, t);
  fft<NX, +1, PL>(v, sm, RowIdx<NX, E>{g * row_smem_stride<NX, E>()}, t, geo.tw + tw_offset(NX),
                  group_sync<T>(g));
  float2* dst = psi0 + ((size_t)p * ny + y) * NX;
#pragma unroll
  for (int e = 0; e < E; ++e) dst[t + T * e] = scale * v[e];
}

// ============================================================================================
// a4/a5: the slice step.
// TF: t comes as the compact output of the band-limit column pass (At) and is inverse-
// transformed here (one wave per frame: no full-size t is written or read).
// ============================================================================================
// Shared memory of the slice row pass: the FFT scratch, plus (TF) one stashed t row per group.
template <int NX, bool TF>
struct SliceRowSmem {
  static constexpr int BYTES = SliceRowCfg<NX>::SMEM + SliceRowCfg<NX>::G * NX * (int)sizeof(float2);
};

// Asynchronous 8-byte copy global -> shared (completes at cp_async_wait_all of the same thread).
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// MB >= 0: the band's half-width, fixed at compile time (the standard 2/3 band of a square
// cell, MB = NX / 3); MB < 0: read from b.
template <int NX, bool FIRST, bool PLANE, bool TF, int MB = -1>
__global__ void __launch_bounds__(SliceRowCfg<NX>::THREADS, minb_of<K_SLICE_ROW, NX, SliceRowCfg<NX>>())
    k_slice_row(Geo geo, Band b, const float2* __restrict__ Apsi, const float2* __restrict__ psi0,
                const float2* __restrict__ ttab, int S, int s, int nfc, int nwaves, float plane_amp,
                float2* __restrict__ Bpsi) {
  constexpr int E = SliceRowCfg<NX>::E, T = SliceRowCfg<NX>::T, G = SliceRowCfg<NX>::G;
  constexpr int PL = Tuned<K_SLICE_ROW, NX>::PLAN;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = reinterpret_cast<float2*>(smraw);
  const int w = batch_index();
  if (w >= nwaves) return;
  const int g = threadIdx.x / T, t = threadIdx.x % T, y = blockIdx.x * G + g, ny = geo.ny;
  const int p = w / nfc, fl = w - p * nfc;
  const RowIdx<NX, E> idx{g * row_smem_stride<NX, E>()};
  const auto sync = group_sync<T>(g);
  float2 v[E];
  if (FIRST && PLANE && TF) {
    // constant initial wave: FFT_x(c IFFT_x(At)) = c NX At, no transform needed
    load_row_compact<NX>(v, ttab + ((size_t)(fl * S + s) * ny + y) * b.Wp, b, t);
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = (plane_amp * (float)NX) * v[e];
    store_row_compact<NX>(v, Bpsi + ((size_t)w * ny + y) * b.Wp, b, t);
    return;
  }
  // The transmission row goes to a shared-memory stash before it is used; each thread writes
  // and rereads only its own positions, so no barrier is needed.  TF: t is inverse-transformed
  // first (only one row of the wave is then live in registers).  Otherwise the full t row is
  // copied asynchronously at once, so its load overlaps the wave's load and inverse transform.
  float2* tst = reinterpret_cast<float2*>(smraw + SliceRowCfg<NX>::SMEM) + g * NX;
  if (TF) {
    load_row<NX, MB>(v, ttab + ((size_t)(fl * S + s) * ny + y) * b.Wp, b, t);
    fft<NX, +1, PL>(v, sm, idx, t, geo.tw + tw_offset(NX), sync);
#pragma unroll
    for (int e = 0; e < E; ++e) tst[t + T * e] = v[e];
  } else {
    const float2* trow = ttab + ((size_t)(fl * S + s) * ny + y) * NX;
#pragma unroll
    for (int e = 0; e < E; ++e) cp_async8(tst + t + T * e, trow + t + T * e);
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  if (FIRST) {
    if (!TF) cp_async_wait_all();
    if (PLANE) {
#pragma unroll
      for (int e = 0; e < E; ++e) v[e] = plane_amp * tst[t + T * e];
    } else {
      const float2* src = psi0 + ((size_t)p * ny + y) * NX;
#pragma unroll
      for (int e = 0; e < E; ++e) v[e] = cmul(src[t + T * e], tst[t + T * e]);
    }
  } else {
    load_row<NX, MB>(v, Apsi + ((size_t)w * ny + y) * b.Wp, b, t);
    fft<NX, +1, PL>(v, sm, idx, t, geo.tw + tw_offset(NX), sync);
    if (!TF) cp_async_wait_all();
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = cmul(v[e], tst[t + T * e]);
  }
  fft<NX, -1, PL>(v, sm, idx, t, geo.tw + tw_offset(NX), sync);
  store_row<NX, MB>(v, Bpsi + ((size_t)w * ny + y) * b.Wp, b, t);
}

// WPC > 0: the row stride of the compact columns (Wp) fixed at compile time (the standard band
// of a square grid), so the strided loads and stores take immediate offsets; else Wp.
template <int NY, bool LAST, int WPC = -1>
__global__ void __launch_bounds__(SliceColCfg<NY>::THREADS, minb_of<K_SLICE_COL, NY, SliceColCfg<NY>>())
    k_slice_col(Geo geo, Band b, const float2* __restrict__ Bpsi, const float2* __restrict__ px,
                const float2* __restrict__ py, float scale, int nfc, int nwaves, int64_t F_total, int64_t f0,
                const int2* __restrict__ disc, int64_t nsel, float2* __restrict__ Apsi, float2* __restrict__ psi_k) {
  using CC = SliceColCfg<NY>;
  constexpr int E = CC::E, T = CC::T, C = CC::C;
  constexpr int PL = Tuned<K_SLICE_COL, NY>::PLAN;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = reinterpret_cast<float2*>(smraw);
  const int w = batch_index();
  if (w >= nwaves) return;
  const int Wp = WPC > 0 ? WPC : b.Wp;
  const int c = threadIdx.x % C, t = threadIdx.x / C, cc = blockIdx.x * C + c;
  const ColIdx<C, CC::SH> idx{c};
  const BlockSync sync;
  const float2* tw = geo.tw + tw_offset(NY);
  const float2* src = Bpsi + (size_t)w * NY * Wp + cc;
  float2 v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) v[e] = src[(size_t)(t + T * e) * Wp];
  fft<NY, -1, PL>(v, sm, idx, t, tw, sync);
  const int nb = cc < b.W ? b.colnb[cc] : -1;
  const float2 pxc = cc < b.W ? px[cc] : make_float2(0.f, 0.f);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int row = t + T * e, n = fftfreq_index(row, NY);
    v[e] = (abs(n) <= nb) ? scale * cmul(cmul(v[e], pxc), py[row]) : make_float2(0.f, 0.f);
  }
  if (LAST) {
    if (cc < b.W) {
      const int p = w / nfc, fl = w - p * nfc;
      if (disc) {
        // compact exit wave: the in-band points of the disc only, in ascending q = y nx + x;
        // row y holds disc[y].y points from disc[y].x on, with x in [0, a] then [nx - a, nx)
        float2* dst = psi_k + ((size_t)p * F_total + f0 + fl) * nsel;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int row = t + T * e, n = fftfreq_index(row, NY);
          if (abs(n) <= nb) {
            const int2 d = disc[row];
            const int a = (d.y - 1) >> 1;
            const int j = d.y == geo.nx ? cc : (cc <= a ? cc : cc - b.W + 2 * a + 1);
            dst[d.x + j] = v[e];
          }
        }
      } else {
        const int x = band_col_x(b, geo.nx, cc);
        float2* dst = psi_k + (((size_t)p * F_total + f0 + fl) * NY) * geo.nx + x;
#pragma unroll
        for (int e = 0; e < E; ++e) dst[(size_t)(t + T * e) * geo.nx] = v[e];
      }
    }
    return;
  }
  fft<NY, +1, PL>(v, sm, idx, t, tw, sync);
  float2* dst = Apsi + (size_t)w * NY * Wp + cc;
#pragma unroll
  for (int e = 0; e < E; ++e) dst[(size_t)(t + T * e) * Wp] = v[e];
}

// ============================================================================================
// Potential multiplier table [pair][ny][Wp] (FP64 evaluation, float storage).
// ============================================================================================
__device__ double form_factor_f64(const double* c, double q) {
  const double q2 = q * q;
  double f = 0.0;
  for (int i = 0; i < 3; ++i) f += c[2 * i] / (q2 + c[2 * i + 1]);
  for (int i = 0; i < 3; ++i) f += c[6 + 2 * i] * exp(-c[7 + 2 * i] * q2);
  return f;
}

__global__ void k_build_mtab(int nx, int ny, Band b, int npair, int nslot, const double* __restrict__ coef,
                             const double* __restrict__ phix, const double* __restrict__ phiy, double Lx, double Ly,
                             double pref, float2* __restrict__ mtab) {
  const int64_t total = (int64_t)npair * ny * b.Wp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int cc = (int)(i % b.Wp);
    const int row = (int)((i / b.Wp) % ny);
    const int pr = (int)(i / ((int64_t)b.Wp * ny));
    float2 out = make_float2(0.f, 0.f);
    const int n = fftfreq_index(row, ny);
    if (cc < b.W && abs(n) <= b.colnb[cc]) {
      const int m = fftfreq_index(band_col_x(b, nx, cc), nx);
      const double kx = (double)m / Lx, ky = (double)n / Ly;
      const double q = sqrt(kx * kx + ky * ky);
      const double fa = form_factor_f64(coef + 12 * (2 * pr), q);
      const double fb = (2 * pr + 1 < nslot) ? form_factor_f64(coef + 12 * (2 * pr + 1), q) : 0.0;
      const double sc = pref / (phix[cc] * phiy[row]);
      out = make_float2((float)(sc * fa), (float)(-sc * fb));
    }
    mtab[i] = out;
  }
}

// ============================================================================================
// launchers
// ============================================================================================
template <class K>
static cudaError_t prep(K kernel, int smem) {
  // opt in above 46 KB: some kernels add a little static shared memory to the dynamic amount
  if (smem > 46 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return cudaSuccess;
}

// Row-pass kernels are also built for the standard 2/3 band of a square cell (half-width NX / 3
// fixed at compile time) at these lengths (the powers of two of the configurations and the
// minimal example's 1152); a launch uses that build when its band is that one
// and the context option "static_band" is on.
template <int NX>
constexpr bool std_band_built() {
  return (fft_pow2(NX) && NX >= 128 && NX <= 1024) || NX == 1152;
}
template <int NX>
bool std_band(const Band& b, int static_band) {
  return static_band && std_band_built<NX>() && b.mb == NX / 3 && b.W == 2 * (NX / 3) + 1;
}
// Padded row stride of the compact columns for that band (as make_band pads W).
constexpr int std_band_wp(int n) {
  const int w = 2 * (n / 3) + 1, up = (w + 31) / 32 * 32, wp = up < 32 ? 32 : up;
  return wp > n ? n : wp;
}

#define TACAW_DISPATCH(N, FN, ...)       \
  switch (N) {                           \
    case 32: return FN<32>(__VA_ARGS__);     \
    case 64: return FN<64>(__VA_ARGS__);     \
    case 96: return FN<96>(__VA_ARGS__);     \
    case 128: return FN<128>(__VA_ARGS__);   \
    case 192: return FN<192>(__VA_ARGS__);   \
    case 256: return FN<256>(__VA_ARGS__);   \
    case 384: return FN<384>(__VA_ARGS__);   \
    case 512: return FN<512>(__VA_ARGS__);   \
    case 768: return FN<768>(__VA_ARGS__);   \
    case 1024: return FN<1024>(__VA_ARGS__); \
    case 1152: return FN<1152>(__VA_ARGS__); \
    default: return cudaErrorInvalidValue;   \
  }

template <int NX>
static cudaError_t splat_row_n(const Geo& g, const Band& b, const AtomRec* recs, const int* boffs, int64_t A,
                               int S, int s0, int sb, int nfs, int npair, SpreadKernel sk, float2* Bp,
                               int static_band, cudaStream_t st) {
  if (s0 < 0 || sb < 1 || s0 + sb > S || nfs % sb != 0) return cudaErrorInvalidValue;
  if (2 * sk.half > SPREAD_MAX_W) return cudaErrorInvalidValue;
  const int smem = SplatSmem<NX>::BYTES;
  const int nb = nfs * npair;
  const dim3 grid = batch_grid(g.ny / SplatCfg<NX>::G, nb);
  // not at 512 points, where the fixed-band build took more registers and measured 4% slower
  if constexpr (std_band_built<NX>() && NX != 512) {
    if (std_band<NX>(b, static_band)) {
      cudaError_t e = prep(k_splat_row<NX, NX / 3>, smem);
      if (e != cudaSuccess) return e;
      k_splat_row<NX, NX / 3><<<grid, SplatCfg<NX>::THREADS, smem, st>>>(g, b, recs, boffs, (int)A, S, s0, sb,
                                                                          npair, nb, sk, Bp);
      return cudaGetLastError();
    }
  }
  cudaError_t e = prep(k_splat_row<NX>, smem);
  if (e != cudaSuccess) return e;
  k_splat_row<NX><<<grid, SplatCfg<NX>::THREADS, smem, st>>>(g, b, recs, boffs, (int)A, S, s0, sb, npair, nb, sk,
                                                             Bp);
  return cudaGetLastError();
}
cudaError_t launch_splat_row(const Geo& g, const Band& b, const AtomRec* recs, const int* boffs, int64_t A, int S,
                             int s0, int sb, int nfs, int npair, SpreadKernel sk, float2* Bp, int static_band,
                             cudaStream_t st) {
  if (g.ny % SPREAD_YB != 0) return cudaErrorInvalidValue;
  TACAW_DISPATCH(g.nx, splat_row_n, g, b, recs, boffs, A, S, s0, sb, nfs, npair, sk, Bp, static_band, st);
}

template <int NY>
static cudaError_t col_pot_n(const Geo& g, const Band& b, const float2* Bp, const float2* mtab, int npair, int nfs,
                             float2* Ap, int static_band, cudaStream_t st) {
  using CC = ColPotCfg<NY>;
  const dim3 grid = batch_grid(col_blocks(b, CC::C), nfs);
  cudaError_t e;
  if constexpr (std_band_built<NY>()) {
    constexpr int WP = std_band_wp(NY);
    if (g.nx == NY && b.Wp == WP && std_band<NY>(b, static_band)) {
      if (npair == 1) {
        if ((e = prep(k_col_pot<NY, true, WP>, CC::SMEM)) != cudaSuccess) return e;
        k_col_pot<NY, true, WP><<<grid, CC::THREADS, CC::SMEM, st>>>(g, b, Bp, mtab, npair, nfs, Ap);
      } else {
        if ((e = prep(k_col_pot<NY, false, WP>, CC::SMEM)) != cudaSuccess) return e;
        k_col_pot<NY, false, WP><<<grid, CC::THREADS, CC::SMEM, st>>>(g, b, Bp, mtab, npair, nfs, Ap);
      }
      return cudaGetLastError();
    }
  }
  if (npair == 1) {
    if ((e = prep(k_col_pot<NY, true>, CC::SMEM)) != cudaSuccess) return e;
    k_col_pot<NY, true><<<grid, CC::THREADS, CC::SMEM, st>>>(g, b, Bp, mtab, npair, nfs, Ap);
  } else {
    if ((e = prep(k_col_pot<NY, false>, CC::SMEM)) != cudaSuccess) return e;
    k_col_pot<NY, false><<<grid, CC::THREADS, CC::SMEM, st>>>(g, b, Bp, mtab, npair, nfs, Ap);
  }
  return cudaGetLastError();
}
cudaError_t launch_col_pot(const Geo& g, const Band& b, const float2* Bp, const float2* mtab, int npair, int nfs,
                           float2* Ap, int static_band, cudaStream_t st) {
  TACAW_DISPATCH(g.ny, col_pot_n, g, b, Bp, mtab, npair, nfs, Ap, static_band, st);
}

template <int NX>
static cudaError_t row_pot_out_n(const Geo& g, const Band& b, const float2* Ap, int nfs, int mode, float sigma,
                                 float* V, float2* out, int static_band, cudaStream_t st) {
  const dim3 grid = batch_grid(g.ny / PotOutCfg<NX>::G, nfs);
  if constexpr (std_band_built<NX>()) {
    if (std_band<NX>(b, static_band)) {
      k_row_pot_out<NX, NX / 3><<<grid, PotOutCfg<NX>::THREADS, PotOutCfg<NX>::SMEM, st>>>(g, b, Ap, nfs, mode,
                                                                                           sigma, V, out);
      return cudaGetLastError();
    }
  }
  k_row_pot_out<NX><<<grid, PotOutCfg<NX>::THREADS, PotOutCfg<NX>::SMEM, st>>>(g, b, Ap, nfs, mode, sigma, V, out);
  return cudaGetLastError();
}
cudaError_t launch_row_pot_out(const Geo& g, const Band& b, const float2* Ap, int nfs, int mode, float sigma,
                               float* V, float2* out, int static_band, cudaStream_t st) {
  TACAW_DISPATCH(g.nx, row_pot_out_n, g, b, Ap, nfs, mode, sigma, V, out, static_band, st);
}

template <int NX>
static cudaError_t row_vt_n(const Geo& g, const Band& b, const float* V, int nfs, int bl, float sigma, float2* out,
                            cudaStream_t st) {
  k_row_vt<NX><<<batch_grid(g.ny / RowVtCfg<NX>::G, nfs), RowVtCfg<NX>::THREADS, RowVtCfg<NX>::SMEM, st>>>(
      g, b, V, nfs, bl, sigma, out);
  return cudaGetLastError();
}
cudaError_t launch_row_vt(const Geo& g, const Band& b, const float* V, int nfs, int bandlimit, float sigma,
                          float2* out, cudaStream_t st) {
  TACAW_DISPATCH(g.nx, row_vt_n, g, b, V, nfs, bandlimit, sigma, out, st);
}

template <int NY>
static cudaError_t col_t_n(const Geo& g, const Band& b, const float2* Bt, int nfs, float scale, float2* At,
                           int static_band, cudaStream_t st) {
  using CC = ColTCfg<NY>;
  if constexpr (std_band_built<NY>()) {
    constexpr int WP = std_band_wp(NY);
    if (g.nx == NY && b.Wp == WP && std_band<NY>(b, static_band)) {
      const cudaError_t e = prep(k_col_t<NY, WP>, CC::SMEM);
      if (e != cudaSuccess) return e;
      k_col_t<NY, WP><<<batch_grid(col_blocks(b, CC::C), nfs), CC::THREADS, CC::SMEM, st>>>(g, b, Bt, nfs, scale, At);
      return cudaGetLastError();
    }
  }
  const cudaError_t e = prep(k_col_t<NY>, CC::SMEM);
  if (e != cudaSuccess) return e;
  k_col_t<NY><<<batch_grid(col_blocks(b, CC::C), nfs), CC::THREADS, CC::SMEM, st>>>(g, b, Bt, nfs,
                                                                                                   scale, At);
  return cudaGetLastError();
}
cudaError_t launch_col_t(const Geo& g, const Band& b, const float2* Bt, int nfs, float scale, float2* At,
                         int static_band, cudaStream_t st) {
  TACAW_DISPATCH(g.ny, col_t_n, g, b, Bt, nfs, scale, At, static_band, st);
}

template <int NX>
static cudaError_t row_tout_n(const Geo& g, const Band& b, const float2* At, int nfs, float2* t, cudaStream_t st) {
  using RC = RowToutCfg<NX>;
  k_row_tout<NX><<<batch_grid(g.ny / RC::G, nfs), RC::THREADS, RC::SMEM, st>>>(g, b, At, nfs, t);
  return cudaGetLastError();
}
cudaError_t launch_row_tout(const Geo& g, const Band& b, const float2* At, int nfs, float2* t, cudaStream_t st) {
  TACAW_DISPATCH(g.nx, row_tout_n, g, b, At, nfs, t, st);
}

template <int NY>
static cudaError_t probe_col_n(const Geo& g, const Band& ap, const float2* ex, const float2* ey, const float2* chi,
                               int P, float amp, float2* Bpr, cudaStream_t st) {
  using CC = ProbeColCfg<NY>;
  const cudaError_t e = prep(k_probe_col<NY>, CC::SMEM);
  if (e != cudaSuccess) return e;
  k_probe_col<NY><<<batch_grid(col_blocks(ap, CC::C), P), CC::THREADS, CC::SMEM, st>>>(
      g, ap, ex, ey, chi, P, amp, Bpr);
  return cudaGetLastError();
}
cudaError_t launch_probe_col(const Geo& g, const Band& ap, const float2* ex, const float2* ey, const float2* chi,
                             int P, float amp, float2* Bpr, cudaStream_t st) {
  TACAW_DISPATCH(g.ny, probe_col_n, g, ap, ex, ey, chi, P, amp, Bpr, st);
}

template <int NX>
static cudaError_t probe_row_n(const Geo& g, const Band& ap, const float2* Bpr, int P, float scale, float2* psi0,
                               cudaStream_t st) {
  using RC = ProbeRowCfg<NX>;
  k_probe_row<NX><<<batch_grid(g.ny / RC::G, P), RC::THREADS, RC::SMEM, st>>>(g, ap, Bpr, P, scale, psi0);
  return cudaGetLastError();
}
cudaError_t launch_probe_row(const Geo& g, const Band& ap, const float2* Bpr, int P, float scale, float2* psi0,
                             cudaStream_t st) {
  TACAW_DISPATCH(g.nx, probe_row_n, g, ap, Bpr, P, scale, psi0, st);
}

template <int NX>
static cudaError_t slice_row_n(const Geo& g, const Band& b, int first, int plane, int tfused, const float2* Apsi,
                               const float2* psi0, const float2* t, int S, int s, int P, int nfc, float plane_amp,
                               float2* Bpsi, int static_band, cudaStream_t st) {
  const int nw = P * nfc;
  const dim3 grid = batch_grid(g.ny / SliceRowCfg<NX>::G, nw);
  constexpr int TH = SliceRowCfg<NX>::THREADS;
#define TACAW_SLICE_ROW(F, PL, TFU)                                                                               \
  do {                                                                                                            \
    constexpr int SM = SliceRowSmem<NX, TFU>::BYTES;                                                              \
    cudaError_t e_ = prep(k_slice_row<NX, F, PL, TFU>, SM);                                                       \
    if (e_ != cudaSuccess) return e_;                                                                             \
    k_slice_row<NX, F, PL, TFU><<<grid, TH, SM, st>>>(g, b, Apsi, psi0, t, S, s, nfc, nw, plane_amp, Bpsi);        \
  } while (0)
  // the later slices (all but one of S) with the standard band fixed at compile time
  constexpr int MB3 = NX / 3;
  constexpr bool SPEC = std_band_built<NX>();
  const bool std_band = tacaw::std_band<NX>(b, static_band);
#define TACAW_SLICE_ROW_STD(TFU)                                                                                   \
  do {                                                                                                            \
    constexpr int SM = SliceRowSmem<NX, TFU>::BYTES;                                                              \
    cudaError_t e_ = prep(k_slice_row<NX, false, false, TFU, MB3>, SM);                                           \
    if (e_ != cudaSuccess) return e_;                                                                             \
    k_slice_row<NX, false, false, TFU, MB3><<<grid, TH, SM, st>>>(g, b, Apsi, psi0, t, S, s, nfc, nw, plane_amp,  \
                                                                  Bpsi);                                          \
  } while (0)
  if (tfused) {
    if (first && plane) TACAW_SLICE_ROW(true, true, true);
    else if (first) TACAW_SLICE_ROW(true, false, true);
    else if constexpr (SPEC) {
      if (std_band) TACAW_SLICE_ROW_STD(true);
      else TACAW_SLICE_ROW(false, false, true);
    } else TACAW_SLICE_ROW(false, false, true);
  } else {
    if (first && plane) TACAW_SLICE_ROW(true, true, false);
    else if (first) TACAW_SLICE_ROW(true, false, false);
    else if constexpr (SPEC) {
      if (std_band) TACAW_SLICE_ROW_STD(false);
      else TACAW_SLICE_ROW(false, false, false);
    } else TACAW_SLICE_ROW(false, false, false);
  }
#undef TACAW_SLICE_ROW_STD
#undef TACAW_SLICE_ROW
  return cudaGetLastError();
}
cudaError_t launch_slice_row(const Geo& g, const Band& b, int first, int plane, int tfused, const float2* Apsi,
                             const float2* psi0, const float2* t, int S, int s, int P, int nfc, float plane_amp,
                             float2* Bpsi, int static_band, cudaStream_t st) {
  TACAW_DISPATCH(g.nx, slice_row_n, g, b, first, plane, tfused, Apsi, psi0, t, S, s, P, nfc, plane_amp, Bpsi,
                 static_band, st);
}

template <int NY>
static cudaError_t slice_col_n(const Geo& g, const Band& b, int last, const float2* Bpsi, const float2* px,
                               const float2* py, float scale, int P, int nfc, int64_t F_total, int64_t f0,
                               const int2* disc, int64_t nsel, float2* Apsi, float2* psi_k, int static_band,
                               cudaStream_t st) {
  const int nw = P * nfc;
  using CC = SliceColCfg<NY>;
  const dim3 grid = batch_grid(col_blocks(b, CC::C), nw);
  constexpr int TH = CC::THREADS, SM = CC::SMEM;
  // the later slices of a square grid with the standard band: row stride fixed at compile time
  if constexpr (std_band_built<NY>()) {
    constexpr int WP = std_band_wp(NY);
    if (!last && g.nx == NY && b.Wp == WP && std_band<NY>(b, static_band)) {
      cudaError_t e = prep(k_slice_col<NY, false, WP>, SM);
      if (e != cudaSuccess) return e;
      k_slice_col<NY, false, WP><<<grid, TH, SM, st>>>(g, b, Bpsi, px, py, scale, nfc, nw, F_total, f0, disc, nsel,
                                                       Apsi, psi_k);
      return cudaGetLastError();
    }
  }
  cudaError_t e = last ? prep(k_slice_col<NY, true>, SM) : prep(k_slice_col<NY, false>, SM);
  if (e != cudaSuccess) return e;
  if (last)
    k_slice_col<NY, true><<<grid, TH, SM, st>>>(g, b, Bpsi, px, py, scale, nfc, nw, F_total, f0, disc, nsel, Apsi,
                                                psi_k);
  else
    k_slice_col<NY, false><<<grid, TH, SM, st>>>(g, b, Bpsi, px, py, scale, nfc, nw, F_total, f0, disc, nsel, Apsi,
                                                 psi_k);
  return cudaGetLastError();
}
cudaError_t launch_slice_col(const Geo& g, const Band& b, int last, const float2* Bpsi, const float2* px,
                             const float2* py, float scale, int P, int nfc, int64_t F_total, int64_t f0,
                             const int2* disc, int64_t nsel, float2* Apsi, float2* psi_k, int static_band,
                             cudaStream_t st) {
  TACAW_DISPATCH(g.ny, slice_col_n, g, b, last, Bpsi, px, py, scale, P, nfc, F_total, f0, disc, nsel, Apsi, psi_k,
                 static_band, st);
}

cudaError_t launch_build_mtab(const Geo& g, const Band& b, int npair, int nslot, const double* coef_slots,
                              const double* phix, const double* phiy, double Lx, double Ly, double pref,
                              float2* mtab, cudaStream_t st) {
  const int64_t total = (int64_t)npair * g.ny * b.Wp;
  const int blocks = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  k_build_mtab<<<blocks, 256, 0, st>>>(g.nx, g.ny, b, npair, nslot, coef_slots, phix, phiy, Lx, Ly, pref, mtab);
  return cudaGetLastError();
}

}  // namespace tacaw
