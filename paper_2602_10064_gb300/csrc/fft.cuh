// Device FFT engine for the slice kernels (lengths: powers of two 32 .. 2048, 3 * 2^k for 96 ..
// 768, and 1152).
//
// Every 2D transform of the hot path (potential, transmission band limit, the slice step of
// the multislice chain in Methods "Multislice Propagation") is split into 1D transforms along
// rows (x, contiguous) and columns (y, strided).  This header holds the 1D engine: a
// Stockham autosort FFT whose radix-R butterflies run in registers and whose data exchange
// between passes goes through shared memory.
//
// Thread ownership: a transform of length N is done by a group of T = N / E consecutive
// threads; thread t owns the E elements at positions t + T*e (e = 0..E-1) on entry and on
// exit, so global loads and stores of a row are coalesced (consecutive t, consecutive
// addresses).  A pass of radix R (R divides E) runs E/R butterflies per thread; the last pass
// lands in the owner's own registers, so an N = R1*R2*R3 transform makes two shared-memory
// exchanges (three for the four-pass plans of 384, 768 and 1152 points).  Each row group
// synchronises only itself (__syncwarp, or a named barrier when a transform spans whole
// warps), so the warps of a CTA never wait on one another; column transforms interleave
// several columns and use the CTA barrier.
//
// Twiddles come from a table tw_N[j] = exp(-2 pi i j / N) built on the host in FP64 and
// rounded to float; the inverse uses the conjugate.  Transforms are unnormalised.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tacaw {

__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 operator*(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// a * (SIGN i): forward (SIGN = -1) multiplies by -i, inverse by +i.
template <int SIGN>
__device__ __forceinline__ float2 mul_si(float2 a) {
  return SIGN < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

// exp(SIGN 2 pi i j / 16) for the small j a radix-16 butterfly needs (j compile-time after unrolling).
template <int SIGN>
__device__ __forceinline__ float2 w16(int j) {
  const float c1 = 0.92387953251128674f, s1 = 0.38268343236508978f, r2 = 0.70710678118654752f;
  float c, s;
  switch (j & 15) {
    case 0: c = 1.f; s = 0.f; break;
    case 1: c = c1; s = s1; break;
    case 2: c = r2; s = r2; break;
    case 3: c = s1; s = c1; break;
    case 4: c = 0.f; s = 1.f; break;
    case 5: c = -s1; s = c1; break;
    case 6: c = -r2; s = r2; break;
    case 7: c = -c1; s = s1; break;
    case 8: c = -1.f; s = 0.f; break;
    case 9: c = -c1; s = -s1; break;
    case 10: c = -r2; s = -r2; break;
    case 11: c = -s1; s = -c1; break;
    case 12: c = 0.f; s = -1.f; break;
    case 13: c = s1; s = -c1; break;
    case 14: c = r2; s = -r2; break;
    default: c = c1; s = -s1; break;
  }
  return make_float2(c, SIGN < 0 ? -s : s);
}

template <int SIGN>
__device__ __forceinline__ void dft2(float2* u) {
  float2 a = u[0], b = u[1];
  u[0] = a + b;
  u[1] = a - b;
}

// X[k] = sum_n u[n] exp(SIGN 2 pi i n k / 4), natural order.
template <int SIGN>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  float2 s02 = a0 + a2, d02 = a0 - a2, s13 = a1 + a3, d13 = mul_si<SIGN>(a1 - a3);
  a0 = s02 + s13;
  a2 = s02 - s13;
  a1 = d02 + d13;
  a3 = d02 - d13;
}

template <int SIGN>
__device__ __forceinline__ void dft4(float2* u) {
  dft4<SIGN>(u[0], u[1], u[2], u[3]);
}

// Radix-8 as two radix-4 transforms of the even and odd samples.
template <int SIGN>
__device__ __forceinline__ void dft8(float2* u) {
  float2 e0 = u[0], e1 = u[2], e2 = u[4], e3 = u[6];
  float2 o0 = u[1], o1 = u[3], o2 = u[5], o3 = u[7];
  dft4<SIGN>(e0, e1, e2, e3);
  dft4<SIGN>(o0, o1, o2, o3);
  const float r2 = 0.70710678118654752f;
  // w8^k = exp(SIGN 2 pi i k / 8)
  float2 t1 = cmul(o1, make_float2(r2, SIGN * r2));
  float2 t2 = mul_si<SIGN>(o2);
  float2 t3 = cmul(o3, make_float2(-r2, SIGN * r2));
  u[0] = e0 + o0;
  u[4] = e0 - o0;
  u[1] = e1 + t1;
  u[5] = e1 - t1;
  u[2] = e2 + t2;
  u[6] = e2 - t2;
  u[3] = e3 + t3;
  u[7] = e3 - t3;
}

// Radix-16 as 4 x 4: inner radix-4 over n1 (stride 4), twiddle w16^(n2 k1), outer radix-4 over n2.
template <int SIGN>
__device__ __forceinline__ void dft16(float2* u) {
  float2 y[4][4];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    y[n2][0] = u[n2];
    y[n2][1] = u[4 + n2];
    y[n2][2] = u[8 + n2];
    y[n2][3] = u[12 + n2];
    dft4<SIGN>(y[n2][0], y[n2][1], y[n2][2], y[n2][3]);
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1)
      if (n2 > 0) y[n2][k1] = cmul(y[n2][k1], w16<SIGN>(n2 * k1));
  }
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    float2 a0 = y[0][k1], a1 = y[1][k1], a2 = y[2][k1], a3 = y[3][k1];
    dft4<SIGN>(a0, a1, a2, a3);
    u[k1] = a0;
    u[k1 + 4] = a1;
    u[k1 + 8] = a2;
    u[k1 + 12] = a3;
  }
}

// X[k] = sum_n u[n] exp(SIGN 2 pi i n k / 3).
template <int SIGN>
__device__ __forceinline__ void dft3(float2& a0, float2& a1, float2& a2) {
  const float h = 0.86602540378443865f;  // sin(pi / 3)
  const float2 s = a1 + a2, d = mul_si<SIGN>(a1 - a2);
  const float2 m = a0 - 0.5f * s;
  a0 = a0 + s;
  a1 = m + h * d;
  a2 = m - h * d;
}

// exp(SIGN 2 pi i j / 24) (j compile-time after unrolling): the twiddles inside the radix-6,
// 12 and 24 butterflies.
template <int SIGN>
__device__ __forceinline__ float2 w24(int j) {
  const float c15 = 0.96592582628906829f, s15 = 0.25881904510252076f, h = 0.86602540378443865f,
              r2 = 0.70710678118654752f;
  float c, s;
  switch (j % 24) {
    case 0: c = 1.f; s = 0.f; break;
    case 1: c = c15; s = s15; break;
    case 2: c = h; s = 0.5f; break;
    case 3: c = r2; s = r2; break;
    case 4: c = 0.5f; s = h; break;
    case 5: c = s15; s = c15; break;
    case 6: c = 0.f; s = 1.f; break;
    case 7: c = -s15; s = c15; break;
    case 8: c = -0.5f; s = h; break;
    case 9: c = -r2; s = r2; break;
    case 10: c = -h; s = 0.5f; break;
    case 11: c = -c15; s = s15; break;
    case 12: c = -1.f; s = 0.f; break;
    case 13: c = -c15; s = -s15; break;
    case 14: c = -h; s = -0.5f; break;
    case 15: c = -r2; s = -r2; break;
    case 16: c = -0.5f; s = -h; break;
    case 17: c = -s15; s = -c15; break;
    case 18: c = 0.f; s = -1.f; break;
    case 19: c = s15; s = -c15; break;
    case 20: c = 0.5f; s = -h; break;
    case 21: c = r2; s = -r2; break;
    case 22: c = h; s = -0.5f; break;
    default: c = c15; s = -s15; break;
  }
  return make_float2(c, SIGN < 0 ? -s : s);
}

template <int R, int SIGN>
__device__ __forceinline__ void dft_r(float2* u);

// exp(SIGN 2 pi i j / 32) for j = n2 k1 < 32 (compile-time after unrolling).
template <int SIGN>
__device__ __forceinline__ float2 w32(int j) {
  // cos(2 pi m / 32) for m = 0 .. 8
  const float c[9] = {1.f, 0.98078528040323044f, 0.92387953251128674f, 0.83146961230254524f,
                      0.70710678118654752f, 0.55557023301960218f, 0.38268343236508978f, 0.19509032201612826f,
                      0.f};
  const int m = j & 31, q = m >> 3, r = m & 7;  // angle = q * 90 deg + r * 11.25 deg
  float cs = c[r], sn = c[8 - r];               // cos, sin of r * 11.25 deg
  float x, y;
  switch (q) {
    case 0: x = cs; y = sn; break;
    case 1: x = -sn; y = cs; break;
    case 2: x = -cs; y = -sn; break;
    default: x = sn; y = -cs; break;
  }
  return make_float2(x, SIGN < 0 ? -y : y);
}

// Radix-32 as 8 x 4: radix-8 over n1 (stride 4), twiddle w32^(n2 k1), radix-4 over n2.
template <int SIGN>
__device__ __forceinline__ void dft32(float2* u) {
  float2 y[4][8];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
#pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) y[n2][n1] = u[n2 + 4 * n1];
    dft8<SIGN>(y[n2]);
#pragma unroll
    for (int k1 = 1; k1 < 8; ++k1)
      if (n2 > 0) y[n2][k1] = cmul(y[n2][k1], w32<SIGN>(n2 * k1));
  }
#pragma unroll
  for (int k1 = 0; k1 < 8; ++k1) {
    float2 a0 = y[0][k1], a1 = y[1][k1], a2 = y[2][k1], a3 = y[3][k1];
    dft4<SIGN>(a0, a1, a2, a3);
    u[k1] = a0;
    u[k1 + 8] = a1;
    u[k1 + 16] = a2;
    u[k1 + 24] = a3;
  }
}

// Radix R1 * R2 (a divisor of 24) as R1 x R2: radix-R1 over n1 (stride R2), twiddle
// w_R^(n2 k1), radix-R2 over n2; natural order in and out.
template <int R1, int R2, int SIGN>
__device__ __forceinline__ void dft_ct(float2* u) {
  constexpr int R = R1 * R2;
  static_assert(24 % R == 0, "twiddles of dft_ct come from the 24-point table");
  float2 y[R2][R1];
#pragma unroll
  for (int n2 = 0; n2 < R2; ++n2) {
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) y[n2][n1] = u[n2 + R2 * n1];
    dft_r<R1, SIGN>(y[n2]);
#pragma unroll
    for (int k1 = 1; k1 < R1; ++k1)
      if (n2 > 0) y[n2][k1] = cmul(y[n2][k1], w24<SIGN>((24 / R) * n2 * k1));
  }
#pragma unroll
  for (int k1 = 0; k1 < R1; ++k1) {
    float2 z[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) z[n2] = y[n2][k1];
    dft_r<R2, SIGN>(z);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) u[k1 + R1 * k2] = z[k2];
  }
}

template <int R, int SIGN>
__device__ __forceinline__ void dft_r(float2* u) {
  if constexpr (R == 2) dft2<SIGN>(u);
  else if constexpr (R == 3) dft3<SIGN>(u[0], u[1], u[2]);
  else if constexpr (R == 4) dft4<SIGN>(u);
  else if constexpr (R == 6) dft_ct<2, 3, SIGN>(u);
  else if constexpr (R == 8) dft8<SIGN>(u);
  else if constexpr (R == 12) dft_ct<4, 3, SIGN>(u);
  else if constexpr (R == 24) dft_ct<8, 3, SIGN>(u);
  else if constexpr (R == 32) dft32<SIGN>(u);
  else dft16<SIGN>(u);
}

// Lengths 3 * 2^k (96 .. 768) and 9 * 2^7 (1152) besides the powers of two.
__host__ __device__ constexpr bool fft_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// Elements per thread (E) for a transform of length N: 8 or 16 for powers of two (8 for
// N <= 64), 24 for 768 and 1152 (three passes), 12 for the other lengths with a factor 3.  A
// kernel picks E per pass direction (powers of two); T = N / E threads share one transform.
template <int N, int EPREF>
struct FftPlan {
  static constexpr int E = fft_pow2(N) ? ((N <= 64) ? 8 : EPREF) : ((N == 768 || N == 1152) ? 24 : 12);
  static constexpr int T = N / E;
};

// Barrier of the whole CTA, for transforms whose threads interleave with other transforms'.
struct BlockSync {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

// Barrier of the T threads that share one transform: the warp when T <= 32, else the named
// barrier `id` (1..15) over T threads (the group's warps are consecutive and aligned).
template <int T>
struct GroupSync {
  int id;
  __device__ __forceinline__ void operator()() const {
    if constexpr (T <= 32) {
      __syncwarp();
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(T) : "memory");
    }
  }
};

// Shared-memory padding: one slot per 2^SH elements along the transform, 2^SH = E for 8, 16
// and 32 elements per thread (16 for 12 and 24).  The first pass of every plan stores each
// thread's E outputs contiguously (stride E across the threads of a warp); with one pad per E
// those 64-bit stores, and the own-position reads of every pass, stay at (or near) the minimum
// two wavefronts per warp.
template <int N, int E>
struct PadShift {
  static constexpr int SH = (E == 8 || N <= 64) ? 3 : (E == 32 ? 5 : 4);
};
template <int N, int E>
struct RowIdx {
  static constexpr int SH = PadShift<N, E>::SH;
  int base;
  __device__ __forceinline__ int operator()(int x) const { return base + x + (x >> SH); }
};
template <int N, int E>
__host__ __device__ constexpr int row_smem_stride() { return N + (N >> PadShift<N, E>::SH); }

// Column-owned transforms: C columns interleaved in shared memory, column c fastest, padded
// with one row of C slots per 2^SH rows (SH = 0: unpadded); the threads of one transform are
// spread over warps, so these transforms use BlockSync.
template <int C, int SH>
struct ColIdx {
  int c;
  __device__ __forceinline__ int operator()(int x) const { return (x + (SH ? (x >> SH) : 0)) * C + c; }
};

// One Stockham pass of radix R; NS = product of earlier radices.
template <int N, int E, int R, int NS, int SIGN, bool LAST, class Idx, class Sync>
__device__ __forceinline__ void fft_pass(float2 (&v)[E], float2* sm, const Idx& idx, int t,
                                         const float2* __restrict__ tw, const Sync& sync) {
  constexpr int T = N / E, B = E / R;
  if (!LAST) sync();  // earlier readers of the group's scratch are done
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int bi = t + T * b;
    const int k = fft_pow2(NS) ? (bi & (NS - 1)) : (int)((unsigned)bi % (unsigned)NS);
    float2 u[R];
#pragma unroll
    for (int i = 0; i < R; ++i) u[i] = v[b + B * i];
    if (NS > 1) {
#pragma unroll
      for (int i = 1; i < R; ++i) {
        float2 w = __ldg(&tw[i * k * (N / (NS * R))]);
        if (SIGN > 0) w.y = -w.y;
        u[i] = cmul(u[i], w);
      }
    }
    dft_r<R, SIGN>(u);
    if (LAST) {
#pragma unroll
      for (int i = 0; i < R; ++i) v[b + B * i] = u[i];
    } else {
      const int d = (bi - k) * R + k;
#pragma unroll
      for (int i = 0; i < R; ++i) sm[idx(d + i * NS)] = u[i];
    }
  }
  if (!LAST) {
    sync();
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = sm[idx(t + T * e)];
  }
}

// Unnormalised length-N transform of the elements owned by this thread (positions t + T e),
// SIGN = -1 forward, +1 inverse.  All T threads of the group call it together; sm (through
// idx) is the group's private scratch; sync is the barrier of the threads sharing it.  tw
// points at the table for length N.
// PLAN selects the radix schedule where there is a choice: 0 = radix-16 passes, 1 = radix-8
// passes (two butterflies per thread and pass) for 512 and 1024 points with E = 16.
template <int N, int SIGN, int PLAN = 0, int E, class Idx, class Sync>
__device__ __forceinline__ void fft(float2 (&v)[E], float2* sm, const Idx& idx, int t,
                                    const float2* __restrict__ tw, const Sync& sync) {
  if constexpr (N == 32) {
    fft_pass<32, E, 8, 1, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<32, E, 4, 8, SIGN, true>(v, sm, idx, t, tw, sync);
  } else if constexpr (N == 64) {
    fft_pass<64, E, 8, 1, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<64, E, 8, 8, SIGN, true>(v, sm, idx, t, tw, sync);
  } else if constexpr (E == 32 && N == 128) {
    fft_pass<128, E, 32, 1, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<128, E, 4, 32, SIGN, true>(v, sm, idx, t, tw, sync);
  } else if constexpr (E == 32 && N == 256) {
    fft_pass<256, E, 32, 1, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<256, E, 8, 32, SIGN, true>(v, sm, idx, t, tw, sync);
  } else if constexpr (E == 32 && N == 512) {
    fft_pass<512, E, 32, 1, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<512, E, 16, 32, SIGN, true>(v, sm, idx, t, tw, sync);
  } else if constexpr (E == 32 && N == 1024) {
    fft_pass<1024, E, 32, 1, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<1024, E, 32, 32, SIGN, true>(v, sm, idx, t, tw, sync);
  } else if constexpr (E == 8 && N == 128) {
    fft_pass<128, E, 8, 1, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<128, E, 4, 8, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<128, E, 4, 32, SIGN, true>(v, sm, idx, t, tw, sync);
  } else if constexpr (E == 8 && N == 256) {
    fft_pass<256, E, 8, 1, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<256, E, 8, 8, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<256, E, 4, 64, SIGN, true>(v, sm, idx, t, tw, sync);
  } else if constexpr (E == 8 && N == 512) {
    fft_pass<512, E, 8, 1, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<512, E, 8, 8, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<512, E, 8, 64, SIGN, true>(v, sm, idx, t, tw, sync);
  } else if constexpr (E == 8 && N == 1024) {
    fft_pass<1024, E, 8, 1, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<1024, E, 8, 8, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<1024, E, 4, 64, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<1024, E, 4, 256, SIGN, true>(v, sm, idx, t, tw, sync);
  } else if constexpr (N == 128) {
    fft_pass<128, E, 16, 1, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<128, E, 8, 16, SIGN, true>(v, sm, idx, t, tw, sync);
  } else if constexpr (N == 256) {
    fft_pass<256, E, 16, 1, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<256, E, 16, 16, SIGN, true>(v, sm, idx, t, tw, sync);
  } else if constexpr (PLAN == 1 && N == 512) {
    fft_pass<512, E, 8, 1, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<512, E, 8, 8, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<512, E, 8, 64, SIGN, true>(v, sm, idx, t, tw, sync);
  } else if constexpr (PLAN == 1 && N == 1024) {
    fft_pass<1024, E, 8, 1, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<1024, E, 8, 8, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<1024, E, 16, 64, SIGN, true>(v, sm, idx, t, tw, sync);
  } else if constexpr (N == 512) {
    fft_pass<512, E, 16, 1, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<512, E, 16, 16, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<512, E, 2, 256, SIGN, true>(v, sm, idx, t, tw, sync);
  } else if constexpr (N == 1024) {
    fft_pass<1024, E, 16, 1, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<1024, E, 16, 16, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<1024, E, 4, 256, SIGN, true>(v, sm, idx, t, tw, sync);
  } else if constexpr (N == 2048) {
    fft_pass<2048, E, 16, 1, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<2048, E, 16, 16, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<2048, E, 8, 256, SIGN, true>(v, sm, idx, t, tw, sync);
  } else if constexpr (E == 12 && N == 96) {
    fft_pass<96, E, 12, 1, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<96, E, 4, 12, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<96, E, 2, 48, SIGN, true>(v, sm, idx, t, tw, sync);
  } else if constexpr (E == 12 && N == 192) {
    fft_pass<192, E, 12, 1, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<192, E, 4, 12, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<192, E, 4, 48, SIGN, true>(v, sm, idx, t, tw, sync);
  } else if constexpr (E == 12 && N == 384) {
    fft_pass<384, E, 12, 1, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<384, E, 4, 12, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<384, E, 4, 48, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<384, E, 2, 192, SIGN, true>(v, sm, idx, t, tw, sync);
  } else if constexpr (E == 24 && N == 768) {
    fft_pass<768, E, 24, 1, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<768, E, 4, 24, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<768, E, 8, 96, SIGN, true>(v, sm, idx, t, tw, sync);
  } else if constexpr (E == 24 && N == 1152) {
    fft_pass<1152, E, 24, 1, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<1152, E, 6, 24, SIGN, false>(v, sm, idx, t, tw, sync);
    fft_pass<1152, E, 8, 144, SIGN, true>(v, sm, idx, t, tw, sync);
  } else {
    static_assert(N == 32, "unsupported FFT length");
  }
}

}  // namespace tacaw
