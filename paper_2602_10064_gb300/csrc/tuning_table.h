// Variant of each FFT pass kernel per transform length (see Tuned in k_slices.cu).
// Written by paper_2602_10064_gb300/tune.py from CUDA-event timings of every variant on GB300
// (variant & 1: radix-8 plans; variant & 2: three CTAs per SM); milliseconds per variant:
//   col_pot@1024: v0 7.54, v1 7.53, v2 8.59, v3 8.80
//   col_pot@128: v0 0.21, v1 0.21, v2 0.23, v3 0.22
//   col_pot@256: v0 1.24, v1 1.24, v2 1.25, v3 1.26
//   col_pot@512: v0 2.49, v1 2.74, v2 3.00, v3 3.22
//   col_t@1024: v0 0.71, v1 0.74, v2 0.74, v3 0.79
//   col_t@128: v0 0.01, v1 0.01, v2 0.01, v3 0.01
//   col_t@256: v0 0.07, v1 0.08, v2 0.06, v3 0.06
//   col_t@512: v0 0.13, v1 0.13, v2 0.13, v3 0.14
//   row_pot_t@1024: v0 9.86, v1 8.93, v2 10.11, v3 8.96
//   row_pot_t@128: v0 0.31, v1 0.31, v2 0.28, v3 0.29
//   row_pot_t@256: v0 1.88, v1 1.88, v2 1.64, v3 1.64
//   row_pot_t@512: v0 4.24, v1 4.21, v2 3.99, v3 4.21
//   row_tout@1024: v0 0.69, v1 0.64, v2 0.62, v3 0.56
//   row_tout@128: v0 0.01, v1 0.01, v2 0.01, v3 0.01
//   row_tout@256: v0 0.06, v1 0.06, v2 0.06, v3 0.06
//   row_tout@512: v0 0.15, v1 0.15, v2 0.13, v3 0.13
//   row_vt@1024: v0 1.62, v1 1.58, v2 1.21, v3 1.15
//   row_vt@128: v0 0.01, v1 0.01, v2 0.01, v3 0.01
//   row_vt@256: v0 0.13, v1 0.13, v2 0.13, v3 0.13
//   row_vt@512: v0 0.40, v1 0.40, v2 0.29, v3 0.29
//   slice_col@1024: v0 6.89, v1 6.94, v2 6.94, v3 7.05
//   slice_col@128: v0 0.24, v1 0.24, v2 0.25, v3 0.25
//   slice_col@256: v0 17.26, v1 17.30, v2 16.66, v3 16.63
//   slice_col@512: v0 2.30, v1 2.36, v2 2.38, v3 2.44
//   slice_row@1024: v0 13.16, v1 12.21, v2 14.77, v3 14.97
//   slice_row@128: v0 0.46, v1 0.46, v2 0.44, v3 0.44
//   slice_row@256: v0 24.09, v1 24.08, v2 21.20, v3 21.21
//   slice_row@512: v0 5.44, v1 5.42, v2 6.48, v3 6.87
//   splat_row@1024: v0 5.58, v1 4.88, v2 4.93, v3 4.51
//   splat_row@128: v0 0.27, v1 0.27, v2 0.27, v3 0.27
//   splat_row@256: v0 1.00, v1 1.00, v2 1.00, v3 1.00
//   splat_row@512: v0 4.50, v1 4.55, v2 3.64, v3 3.64
#pragma once

namespace tacaw {

// [kernel][log2(N) - 5] for N = 32 .. 1024
constexpr int kTunedVariant[10][6] = {
    {0, 0, 0, 0, 3, 3},  // splat_row
    {0, 0, 0, 0, 0, 0},  // col_pot
    {0, 0, 2, 3, 2, 1},  // row_pot_t
    {0, 0, 0, 0, 2, 3},  // row_vt
    {0, 0, 0, 2, 0, 0},  // col_t
    {0, 0, 0, 0, 3, 3},  // row_tout
    {0, 0, 0, 0, 0, 0},  // probe (not tuned)
    {0, 0, 0, 0, 0, 0},  // probe (not tuned)
    {0, 0, 2, 2, 0, 1},  // slice_row
    {0, 0, 0, 3, 0, 0},  // slice_col
};

constexpr int tuned_variant(int kernel, int n) {
  int l = 0;
  while ((32 << l) < n) ++l;
  return (kernel >= 0 && kernel < 10 && l < 6) ? kTunedVariant[kernel][l] : 0;
}

}  // namespace tacaw
