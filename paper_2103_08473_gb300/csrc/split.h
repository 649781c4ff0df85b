// Split-precision complex GEMM (Ozaki-style digit slices on tcgen05 tensor cores).
//
//   C = alpha * op(A) * op(B) + beta * C      (complex double in and out)
//
// Each operand row (A) or column (B) is scaled by a power of two 2^e so that its
// largest real/imaginary magnitude is below 1 (below 1/2 where the digit width needs
// a bit of headroom, see split_headroom), then cut into s signed integer digits of
// b bits (round to nearest): x = sum_p d_p 2^{-b p} + r, |r| <= 2^{-b s - 1}.
// Digits are exact in the narrow type (e4m3 holds every integer up to 16, bf16 up
// to 256). The product of two digit matrices is an integer matrix; the tensor
// cores form it in FP32 with every partial sum an integer below 2^24, hence
// exactly. Products of equal weight 2^{-b(p+q)} ("levels") share one FP32
// accumulator over a K range short enough to stay exact; each level range is
// then scaled and added into C in FP64. Levels p + q <= s + 1 are kept
// (triangular scheme).
//
// Complex products use four real products per digit pair (4M) into separate
// real/imaginary TMEM accumulators; A_im * B_im enters the real part through the
// instruction descriptor's negate-B bit.
#pragma once

#include <cuda.h>

#include "common.cuh"
#include "zgemm.h"

namespace ccsd {

enum SplitKind { kSplitE4M3 = 0, kSplitBF16 = 1 };

// Digit slices of one operand, laid out for TMA: planes p*2 + part (real, imaginary) of
// rows_pad rows each (rows rounded up to 32, the padding rows zero), columns k in [0, Kp)
// (zero padded), one byte (e4m3) or two bytes (bf16) per digit.
struct SliceSet {
  void* digits = nullptr;   // device
  double* scale = nullptr;  // device, 2^e per row (rows entries)
  int64_t rows = 0, rows_pad = 0, K = 0, Kp = 0;
  int s = 0, b = 0, kind = kSplitE4M3;
  int64_t chunk = 0, nchunks = 1;  // K chunking of the slicing work (rows with K contiguous)
  int64_t row0 = 0;                // a row view: its first row within the digit set
  CUtensorMap tmap;  // 3D map (K, row, plane), box {128 bytes, 128 rows, 1 plane}, 128B swizzle
  bool have_map = false;
};

// Largest integer magnitude the digit type holds exactly: every integer up to 16 in e4m3,
// up to 256 in bf16. Digits of b bits lie in [-2^(b-1), 2^(b-1)] after the first; the first
// reaches 2^b when rows are scaled below 1. Where 2^b is beyond the exact range, rows are
// scaled below 1/2 instead (one bit of headroom), so that every digit, the first included,
// stays within 2^(b-1): e4m3 then carries b = 5. (bf16 stops at b = 8: products of 9-bit
// digits would leave no whole K block of exact FP32 accumulation.)
inline int split_exact_max(int kind) { return kind == kSplitBF16 ? 256 : 16; }
inline int split_headroom(int kind, int b) { return (1 << b) > split_exact_max(kind) ? 1 : 0; }
inline int split_max_bits(int kind) { return kind == kSplitBF16 ? 8 : 5; }

struct SplitConfig {
  int kind = kSplitE4M3;
  int b = 5;          // bits per digit
  int s = 9;          // digits per operand
  int triangular = 1; // keep pairs with p + q <= s + 1 (else all s^2 pairs)
};

// Rows [r0, r0 + n) of a slice set, as an operand of split_gemm (no copy). The tiles of a view
// also read digits of the rows after it (or the zero fill past the set); those only reach
// outputs beyond the view's extent, which the kernel does not write.
inline SliceSet slice_rows(const SliceSet& S, int64_t r0, int64_t n) {
  SliceSet V = S;
  V.rows = n;
  V.scale = S.scale + r0;
  V.row0 = S.row0 + r0;
  return V;
}

// Bytes of device memory a SliceSet of this shape needs (digits + scales).
int64_t slice_bytes(int64_t rows, int64_t K, const SplitConfig& cfg);
// Digits of op(X) viewed as rows x K (element (r,k) = trans ? X[k*ld + r] : X[r*ld + k],
// conjugated if conj), written into `out` (whose digits/scale point at device memory
// of slice_bytes). Sets out's shape fields and encodes its tensor map.
cudaError_t make_slices(const z* X, int64_t rows, int64_t K, int64_t ld, int trans, int conj,
                        const SplitConfig& cfg, SliceSet& out, void* mem, cudaStream_t s);
// Modelled seconds of one split GEMM of this shape (used to route contractions).
double split_cost_estimate(int64_t M, int64_t N, int64_t K, const SplitConfig& cfg);
// Bytes of FP64 partial products split_gemm wants when it splits K across CTAs
// (outputs with fewer tiles than SMs); 0 when it does not split.
int64_t split_part_bytes(int64_t M, int64_t N, int64_t K, const SplitConfig& cfg);
// C = alpha * A B^T + beta * C from slice sets A (M rows) and B (N rows) over the same K.
// err: device int, set nonzero by the kernel if a bounded wait gave up. part_ws: device
// memory for the K-split partials (split_part_bytes); without it K is not split.
// wait_cycles: budget of every device wait (0 = about 2 s). stall_loads (self-test of the
// failure path only): the producer issues no copies, so the MMA issuer's first wait runs out.
// conjB: C = alpha * A conj(B)^T + beta * C (the digits of B are those of the unconjugated rows).
cudaError_t split_gemm(const SliceSet& A, const SliceSet& B, z* C, int64_t ldc, z alpha, z beta,
                       int* err, void* part_ws, int64_t part_bytes, cudaStream_t s, long long wait_cycles = 0,
                       int stall_loads = 0, int conjB = 0);
// How split_gemm runs C (M x N) = A B^T over K: out[0] = 1 for the short-K kernel (0 main),
// out[1] = 1 when the operands are swapped (A's rows on the narrow side), out[2] = the tile
// width, out[3] = CTAs per cluster (1 or 2), out[4] = CTAs along K, out[5] = output tiles.
void split_describe(int64_t M, int64_t N, int64_t K, const SplitConfig& cfg, int out[6]);
// Probe: C (FP64 real, M x N) = A B^T for integer-valued A (M x K) and B (N x K) stored as
// single digits, summed in one FP32 accumulator over all of K (exactness checks of the
// tensor-core accumulation). mem: 2 slice sets of one digit each.
cudaError_t split_probe_raw(int kind, const double* Aint, const double* Bint, int64_t M, int64_t N, int64_t K,
                            double* C, void* mem, int* err, cudaStream_t s);

}  // namespace ccsd
