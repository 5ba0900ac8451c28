// Shared device helpers for the sm_103a subtraction kernels: complex
// arithmetic, compile-time twiddle factors, an in-register radix-2 FFT and
// warp reductions.  No function here comes from a vendor library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sfft.h"

namespace sfft {

// ------------------------------------------------------------------ complex types
template <typename T> struct cplx;
template <> struct cplx<float> { using t = float2; };
template <> struct cplx<double> { using t = double2; };
template <typename T> using c_t = typename cplx<T>::t;

template <typename T2> __host__ __device__ __forceinline__ T2 mk2(double x, double y) {
  T2 r; r.x = (decltype(r.x))x; r.y = (decltype(r.y))y; return r;
}
template <typename T2> __device__ __forceinline__ T2 cadd(T2 a, T2 b) { T2 r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename T2> __device__ __forceinline__ T2 csub(T2 a, T2 b) { T2 r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename T2> __device__ __forceinline__ T2 cmul(T2 a, T2 b) {
  T2 r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}

// ------------------------------------------------------------------ compile-time twiddles
// cos / sin of 2*pi*j/n evaluated in double from Taylor series on an angle
// reduced to [0, pi/4] by exact integer arithmetic on the rational j/n.  All
// arguments are compile-time constants at the call sites, so the values fold
// into immediates.
constexpr double kPi = 3.14159265358979323846264338327950288;

__host__ __device__ constexpr double ce_sin_small(double x) {
  double term = x, sum = x, x2 = x * x;
  for (int n = 1; n < 16; ++n) { term *= -x2 / double((2 * n) * (2 * n + 1)); sum += term; }
  return sum;
}
__host__ __device__ constexpr double ce_cos_small(double x) {
  double term = 1.0, sum = 1.0, x2 = x * x;
  for (int n = 1; n < 16; ++n) { term *= -x2 / double((2 * n - 1) * (2 * n)); sum += term; }
  return sum;
}
// returns cos (which=0) or sin (which=1) of 2*pi*j/n
__host__ __device__ constexpr double ce_cis(int j, int n, int which) {
  int jm = ((j % n) + n) % n;
  int quad = (4 * jm) / n;                  // quarter turn index 0..3
  int rem = 4 * jm - quad * n;              // angle within quadrant = (pi/2) * rem / n
  double c0 = 0.0, s0 = 0.0;
  if (2 * rem <= n) {                       // <= pi/4
    double phi = 0.5 * kPi * double(rem) / double(n);
    c0 = ce_cos_small(phi); s0 = ce_sin_small(phi);
  } else {                                  // use the complementary angle
    double psi = 0.5 * kPi * double(n - rem) / double(n);
    c0 = ce_sin_small(psi); s0 = ce_cos_small(psi);
  }
  double c = c0, s = s0;
  if (quad == 1) { c = -s0; s = c0; }
  if (quad == 2) { c = -c0; s = -s0; }
  if (quad == 3) { c = s0; s = -c0; }
  return which == 0 ? c : s;
}

__host__ __device__ constexpr int ce_log2(int n) { return n <= 1 ? 0 : 1 + ce_log2(n >> 1); }
__host__ __device__ constexpr int ce_bitrev(int i, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
  return r;
}

// v[k] * exp(-2 pi i k' / len) with a compile-time (k', len)
template <typename T2>
__device__ __forceinline__ T2 twiddle_mul(T2 b, int k, int len) {
  if (k == 0) return b;
  if (4 * k == len) { T2 r; r.x = b.y; r.y = -b.x; return r; }     // * (-i)
  const double c = ce_cis(k, len, 0), s = ce_cis(k, len, 1);
  using R = decltype(b.x);
  T2 r;
  r.x = b.x * (R)c + b.y * (R)s;
  r.y = b.y * (R)c - b.x * (R)s;
  return r;
}

// In-register forward DFT of length N (power of two), natural order in and out:
// X[k] = sum_n x[n] exp(-2 pi i n k / N).  Decimation in time.
template <int N, typename T2>
__device__ __forceinline__ void fft_reg(T2 (&v)[N]) {
  if constexpr (N == 1) {
    return;
  } else {
    constexpr int B = ce_log2(N);
    T2 t[N];
#pragma unroll
    for (int i = 0; i < N; ++i) t[ce_bitrev(i, B)] = v[i];
#pragma unroll
    for (int len = 2; len <= N; len <<= 1) {
#pragma unroll
      for (int i = 0; i < N; i += len) {
#pragma unroll
        for (int k = 0; k < len / 2; ++k) {
          T2 a = t[i + k];
          T2 bw = twiddle_mul(t[i + k + len / 2], k, len);
          t[i + k] = cadd(a, bw);
          t[i + k + len / 2] = csub(a, bw);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = t[i];
  }
}

// ------------------------------------------------------------------ reductions
template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------------ index helpers
// Monomials xt^a yt^b with a + b <= D ordered by degree n, then a descending:
// index(a, b) = n (n + 1) / 2 + (n - a).
__host__ __device__ constexpr int mono_index(int a, int b) {
  return (a + b) * (a + b + 1) / 2 + b;
}
__host__ __device__ constexpr int n_mono(int D) { return (D + 1) * (D + 2) / 2; }

constexpr int kMaxL = 11;
constexpr int kMaxD = 2;          // D_K, D_B <= 2
constexpr int kMaxWeightDeg = 4;  // 2 D_B

}  // namespace sfft
