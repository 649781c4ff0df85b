// Shared device/host helpers of libccsd: complex arithmetic on double2,
// antisymmetric pair indexing and CUDA error plumbing.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

namespace ccsd {

using z = double2;  // interleaved complex double, same layout as ccsd_z

__host__ __device__ __forceinline__ z zmake(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ z zadd(z a, z b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ z zsub(z a, z b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ z zmul(z a, z b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ z zconj(z a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ z zscale(double s, z a) { return make_double2(s * a.x, s * a.y); }
// a*x + b*y with complex a, real b
__host__ __device__ __forceinline__ z zaxpby(z a, z x, double b, z y) {
  return make_double2(a.x * x.x - a.y * x.y + b * y.x, a.x * x.y + a.y * x.x + b * y.y);
}

// Antisymmetric pairs x < y of an index range [0, n) are numbered row by row of
// the strict upper triangle: P(x, y) = x (2n - x - 1) / 2 + (y - x - 1).
// Consecutive y at fixed x give consecutive P.
__host__ __device__ __forceinline__ int64_t pair_count(int64_t n) { return n * (n - 1) / 2; }
__host__ __device__ __forceinline__ int64_t pair_index(int64_t x, int64_t y, int64_t n) {
  return x * (2 * n - x - 1) / 2 + (y - x - 1);
}
// Inverse of pair_index: the row x is the largest x with pair_index(x, x+1) <= P. A single-precision
// estimate from the quadratic formula (the FP64 pipe is narrow here), then exact integer
// corrections in both directions, so the result does not depend on the estimate's rounding.
__device__ __forceinline__ void pair_decode(int64_t P, int64_t n, int64_t& x, int64_t& y) {
  const float nn = (float)(2 * n - 1);
  int64_t xx = (int64_t)((nn - sqrtf(fmaxf(nn * nn - 8.0f * (float)P, 0.0f))) * 0.5f);
  if (xx < 0) xx = 0;
  if (xx > n - 2) xx = n - 2;
  while (xx > 0 && xx * (2 * n - xx - 1) / 2 > P) --xx;
  while (xx < n - 2 && (xx + 1) * (2 * n - xx - 2) / 2 <= P) ++xx;
  x = xx;
  y = P - xx * (2 * n - xx - 1) / 2 + xx + 1;
}

inline int grid_for(int64_t n, int threads, int cap = 152 * 32) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

}  // namespace ccsd
