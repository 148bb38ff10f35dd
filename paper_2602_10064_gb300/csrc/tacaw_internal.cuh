// Internal declarations shared by the CUDA translation units of libtacaw.so.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace tacaw {

// Columns of an nx-point axis kept after a circular mask, stored compactly in FFT order:
// compact column c < W holds x = c for c <= mb and x = nx - (W - c) otherwise.  Wp rounds W
// up to a multiple of 32 (padding columns are zero).  colnb[c] is the largest |n| of the
// in-band rows of that column (-1 for padding), so (row n, column c) is inside the disc iff
// |n| <= colnb[c].
struct Band {
  int W, Wp, mb;
  const int* colnb;
};

// Grid shape plus the FFT twiddle tables (table for length N starts at tw + N).
struct Geo {
  int nx, ny;
  const float2* tw;  // the context's twiddle tables: length n at tw + tw_offset(n)
};

// Layout of the context's twiddle table: exp(-2 pi i j / n), j < n, at [tw_offset(n),
// tw_offset(n) + n): the powers of two 2 .. 2048 at offset n (packed into [2, 4096)), then the
// lengths with a factor 3 one after the other.
__host__ __device__ constexpr int tw_offset(int n) {
  return (n & (n - 1)) == 0 ? n
         : n == 96          ? 4096
         : n == 192         ? 4096 + 96
         : n == 384         ? 4096 + 288
         : n == 768         ? 4096 + 672
         : n == 1152        ? 4096 + 1440
                            : -1;
}
constexpr int kTwiddleEntries = 4096 + 2592;
constexpr int kTwiddleOtherLengths[5] = {96, 192, 384, 768, 1152};

// One atom after binning, in the order of its slice list.  ix0/iy0 = floor of the grid
// coordinate (x wrapped into [0, Lx), times nx / Lx, in FP64), fx/fy the remainder.
struct AtomRec {
  float fx, fy;
  int ixy;    // ix0 | iy0 << 16
  int jslot;  // atom index | species slot << 24
};

__device__ __forceinline__ int fftfreq_index(int i, int n) { return i < (n + 1) / 2 ? i : i - n; }

// Error-free FP32 sums (Knuth's two-sum): s = fl(a + b) and e with s + e = a + b exactly.
// GB300's FP64 pipe issues at 1/64 of the FP32 rate, so the elastic mean and the residual
// carry FP64-class precision as unevaluated FP32 pairs built from these, not as doubles.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// Running sum as the pair (hi, lo), |lo| <= 2^-24 |hi|: hi takes x by a two-sum, lo takes the
// exact error, then the pair is renormalised by a second two-sum (exact whichever part is
// larger).  Each step loses at most about 2^-48 |hi|.
__device__ __forceinline__ void pair_add(float& hi, float& lo, float x) {
  float s, e;
  two_sum(hi, x, s, e);
  two_sum(s, __fadd_rn(lo, e), hi, lo);
}
// Frame mean of one column to FP64-class precision, in two steps shared by the kernels that
// need it.  column_pair_sums: the thread of group g (of GROUPS) sums the frames n = g, g + GROUPS,
// ... of col[n * stride] as an FP32 pair per component, in frame order, four loads in flight;
// returns (hi.x, lo.x, hi.y, lo.y).  combine_pair_sums: the GROUPS pairs added in FP64 in group
// order and divided by F.  Over n frames a pair loses at most about n 2^-48 of its largest
// partial sum (FP64 summation: n 2^-53).
template <int GROUPS>
__device__ __forceinline__ float4 column_pair_sums(const float2* __restrict__ col, int64_t F, int64_t stride, int g) {
  float hx = 0.f, lx = 0.f, hy = 0.f, ly = 0.f;
  int64_t n = g;
  for (; n + 3 * GROUPS < F; n += 4 * GROUPS) {
    float2 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = col[(size_t)(n + u * GROUPS) * stride];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      pair_add(hx, lx, v[u].x);
      pair_add(hy, ly, v[u].y);
    }
  }
  for (; n < F; n += GROUPS) {
    const float2 v = col[(size_t)n * stride];
    pair_add(hx, lx, v.x);
    pair_add(hy, ly, v.y);
  }
  return make_float4(hx, lx, hy, ly);
}
template <int GROUPS>
__device__ __forceinline__ double2 combine_pair_sums(const float4 (&part)[GROUPS], int64_t F) {
  double sx = 0.0, sy = 0.0;
#pragma unroll
  for (int k = 0; k < GROUPS; ++k) {
    sx += (double)part[k].x + (double)part[k].y;
    sy += (double)part[k].z + (double)part[k].w;
  }
  return make_double2(sx / (double)F, sy / (double)F);
}

// The FP64 value m as an FP32 pair: hi = fl32(m), lo = fl32(m - hi) (m - hi is exact in FP64).
__device__ __forceinline__ void split_double(double m, float& hi, float& lo) {
  hi = (float)m;
  lo = (float)(m - (double)hi);
}
// x - (mh + ml) as the pair (r, re): r = fl32 of the difference, r + re the difference to
// within |ml| * 2^-24 + 2^-48 |x - mh| (x - mh is formed exactly).
__device__ __forceinline__ void pair_sub(float x, float mh, float ml, float& r, float& re) {
  float s, e;
  two_sum(x, -mh, s, e);
  two_sum(s, __fsub_rn(e, ml), r, re);
}
__device__ __forceinline__ int band_col_x(const Band& b, int nx, int c) { return c <= b.mb ? c : nx - (b.W - c); }
__device__ __forceinline__ int band_x_col(const Band& b, int nx, int x) {
  return x <= b.mb ? x : (x >= nx - b.mb ? x - nx + b.W : -1);
}

// ---- host launchers (k_slices.cu) ---------------------------------------------------------
struct SpreadKernel {
  int half;    // h = w / 2 grid points
  float beta;  // exp(beta (sqrt(1 - z^2) - 1))
};

// Bits of the context's device status word, read and cleared by tacaw_check.
constexpr int TACAW_STATUS_TIMEOUT = 1;  // a kernel's bounded wait ran out
constexpr int TACAW_STATUS_SPECIES = 2;  // an atom's Z was not in the form-factor table

// rows x width floats, row r of dst_mapped (pitch dp) = row r of src (pitch sp), pitches in
// floats, by SM stores (dst_mapped: the device address of mapped page-locked host memory, or
// any device memory).
cudaError_t launch_copy_out(const float* src, int64_t sp, float* dst_mapped, int64_t dp, int64_t width, int64_t rows,
                            cudaStream_t st);

// slot[j] = lut[Z[j]] (lut: 256 entries, -1 = not loaded); an unknown Z sets
// TACAW_STATUS_SPECIES in *status and gets slot 0.
cudaError_t launch_map_slots(const int32_t* Z, int64_t A, const int8_t* lut, int8_t* slot, int* status,
                             cudaStream_t st);
cudaError_t launch_bin(const float* pos, int64_t A, int64_t nf, int S, double Lx, double Ly, double Lz, int nx,
                       int ny, const int8_t* slot_of_atom, AtomRec* recs, int* offs, int* slice_out,
                       cudaStream_t st);
// Grid rows per block of the row-sorted atom lists of the spreading pass (divides every grid length).
constexpr int SPREAD_YB = 8;
// Row-sorted copy of the binned records: per (frame, slice) a stable sort by grid row, and the
// offsets of each block of SPREAD_YB rows, boffs [nf][S][ny / SPREAD_YB + 1] (absolute within
// the frame).
cudaError_t launch_sort_rows(const AtomRec* recs, const int* offs, int64_t A, int64_t nf, int S, int ny,
                             AtomRec* out, int* boffs, cudaStream_t st);
// Spreading row pass of slices [s0, s0 + sb) of nfs / sb frames (batch = (frame, slice, pair)),
// from the row-sorted records and their row-block offsets.
cudaError_t launch_splat_row(const Geo& g, const Band& b, const AtomRec* recs, const int* boffs, int64_t A, int S,
                             int s0, int sb, int nfs, int npair, SpreadKernel sk, float2* Bp, int static_band,
                             cudaStream_t st);
cudaError_t launch_col_pot(const Geo& g, const Band& b, const float2* Bp, const float2* mtab, int npair, int nfs,
                           float2* Ap, int static_band, cudaStream_t st);
// mode 0: store V; mode 1: t = exp(i sigma V), band-limit pass input (FFT_x, compact);
// mode 2: t = exp(i sigma V) stored directly (no transmission band limit).
cudaError_t launch_row_pot_out(const Geo& g, const Band& b, const float2* Ap, int nfs, int mode, float sigma,
                               float* V, float2* out, int static_band, cudaStream_t st);
cudaError_t launch_row_vt(const Geo& g, const Band& b, const float* V, int nfs, int bandlimit, float sigma,
                          float2* out, cudaStream_t st);
cudaError_t launch_col_t(const Geo& g, const Band& b, const float2* Bt, int nfs, float scale, float2* At,
                         int static_band, cudaStream_t st);
cudaError_t launch_row_tout(const Geo& g, const Band& b, const float2* At, int nfs, float2* t, cudaStream_t st);
// chi (nullable): exp(-i chi(k)) over [ny][ap.Wp]
cudaError_t launch_probe_col(const Geo& g, const Band& ap, const float2* ex, const float2* ey, const float2* chi,
                             int P, float amp, float2* Bpr, cudaStream_t st);
cudaError_t launch_probe_row(const Geo& g, const Band& ap, const float2* Bpr, int P, float scale, float2* psi0,
                             cudaStream_t st);
// One slice s for n_waves = P * nfc waves; wave w = p * nfc + fl uses t[(fl * S + s)], full
// rows, or with tfused the compact band-limit column-pass output, inverse-transformed in place.
// static_band: the later slices use the kernel built for the standard 2/3 band of a square cell
// (half-width NX / 3 fixed at compile time) when b is that band (likewise in the spreading and
// potential-output row passes).
cudaError_t launch_slice_row(const Geo& g, const Band& b, int first, int plane, int tfused, const float2* Apsi,
                             const float2* psi0, const float2* t, int S, int s, int P, int nfc, float plane_amp,
                             float2* Bpsi, int static_band, cudaStream_t st);
// last = 0: Apsi = IFFT_y(P M scale FFT_y(Bpsi)); last = 1: psi_k[p][f0 + fl] = P M scale FFT_y(Bpsi),
// as the full [ny][nx] grid (disc = NULL; out-of-band points are not written) or, with disc, as
// the nsel in-band points of the disc in ascending q: row y's points start at disc[y].x and
// number disc[y].y.
cudaError_t launch_slice_col(const Geo& g, const Band& b, int last, const float2* Bpsi, const float2* px,
                             const float2* py, float scale, int P, int nfc, int64_t F_total, int64_t f0,
                             const int2* disc, int64_t nsel, float2* Apsi, float2* psi_k, int static_band,
                             cudaStream_t st);
// mtab[pair][ny][Wp] = C M(k) (f_2p(|k|) - i f_2p+1(|k|)) / (Phi_x Phi_y), FP64 evaluation.
cudaError_t launch_build_mtab(const Geo& g, const Band& b, int npair, int nslot, const double* coef_slots,
                              const double* phix, const double* phiy, double Lx, double Ly, double pref,
                              float2* mtab, cudaStream_t st);

// ---- time transform (k_spectrum.cu) -----------------------------------------------------
cudaError_t launch_mean_f64(const float2* psi, int64_t P, int64_t F, int64_t nq, const int32_t* qsel,
                            int64_t nsel, double2* mean, cudaStream_t st);
// mean[p][j] = (1/F) sum_n psi[p][n][qsel[j]]: FP32 pair sums, combined and divided in FP64
// residual r[p][n][j] = psi[p][n][qsel[j]] - mean[p][j], formed exactly as an FP32 pair and
// rounded to float
cudaError_t launch_residual_f32(const float2* psi, const double2* mean, int64_t P, int64_t F, int64_t nq,
                                const int32_t* qsel, int64_t nsel, float2* r, cudaStream_t st);
// S[p][m][qsel[j]] = |sum_n W[m][n] r[p][n][j]|^2 (FP32), W from the length-F table
cudaError_t launch_dft_fp32(const float2* r, const float2* twF, int64_t P, int64_t F, int64_t nsel, int64_t nq,
                            const int32_t* qsel, float* S, cudaStream_t st);
// SI[p][m] = sum_j S[p][m][qsel[j]] (FP64 accumulation, deterministic)
cudaError_t launch_detector_reduce(const float* S, int64_t P, int64_t F, int64_t nq, const int32_t* qsel,
                                   int64_t nsel, float* SI, cudaStream_t st);

// ---- accessors (k_accessors.cu) ------------------------------------------------------------
cudaError_t launch_spectral_diffraction(const float* S, int64_t P, int64_t F, int64_t nq, int m, int fold,
                                        float* out, cudaStream_t st);
cudaError_t launch_dispersion(const float* S, int64_t P, int64_t F, int ny, int nx, const double* u,
                              const double* v, int npts, float* out, cudaStream_t st);
cudaError_t launch_accumulate(const float* S, int64_t n, double weight, double* acc, cudaStream_t st);

}  // namespace tacaw
