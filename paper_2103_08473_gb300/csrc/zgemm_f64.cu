// Complex double-precision GEMM on the FP64 tensor path (mma.sync m8n8k4.f64).
//
//   C[b] = alpha * opA(A[b]) * opB(B[b]) + beta * C[b]     (row-major, complex double)
//
// Every contraction of the CCSD residual in the FP64 mode reduces to this call
// after index permutation (transpose-transpose-GEMM-transpose). A complex
// multiply-add is four real products (4M): Re += Ar Br - Ai Bi, Im += Ar Bi + Ai Br,
// issued as four DMMAs per 8x8x4 tile pair into separate real and imaginary
// accumulators.
//
// Tiles are staged in shared memory with cp.async (16-byte copies of one complex
// element each, so any operand layout and transpose maps onto the same
// [k][m] / [k][n] shared tiles) in a two-stage pipeline. Out-of-range elements
// are zero-filled by the copy. On this chip the FP64 pipe (about 1 TFLOP/s for
// the whole GPU) is the bound: a 152-SM GPU retires one m8n8k4 DMMA per SM every
// ~150 clocks, so the kernel favours many small tiles (good load balance across
// SMs) over operand reuse.
#include "common.cuh"
#include "zgemm.h"

namespace ccsd {
namespace {

constexpr int BK = 8;  // complex elements of K per stage (2 DMMA k-steps)

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool pred) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  int n = pred ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void dmma(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

// BM x BN block tile, 4 warps arranged WM x WN, each warp (BM/WM) x (BN/WN).
template <int BM, int BN, int WM, int WN>
__global__ void __launch_bounds__(128) zgemm_dmma_kernel(ZGemmArgs g) {
  constexpr int WTM = BM / WM, WTN = BN / WN;
  constexpr int MT = WTM / 8, NT = WTN / 8;
  __shared__ __align__(16) z As[2][BK][BM];
  __shared__ __align__(16) z Bs[2][BK][BN];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm0 = (warp / WN) * WTM, wn0 = (warp % WN) * WTN;
  const int64_t bm0 = (int64_t)blockIdx.y * BM, bn0 = (int64_t)blockIdx.x * BN;
  const int64_t bz = blockIdx.z;
  const z* __restrict__ A = g.A + bz * g.sA;
  const z* __restrict__ B = g.B + bz * g.sB;
  z* __restrict__ C = g.C + bz * g.sC;

  auto load_stage = [&](int st, int64_t k0) {
    // A tile: BM x BK complex
#pragma unroll
    for (int r = 0; r < (BM * BK) / 128; ++r) {
      int e = tid + 128 * r;
      int mm, kk;
      if (g.transA) { mm = e % BM; kk = e / BM; } else { kk = e % BK; mm = e / BK; }
      int64_t m = bm0 + mm, k = k0 + kk;
      bool ok = (m < g.M) && (k < g.K);
      const z* src = ok ? (g.transA ? A + k * g.lda + m : A + m * g.lda + k) : A;
      cp_async16(&As[st][kk][mm], src, ok);
    }
#pragma unroll
    for (int r = 0; r < (BN * BK) / 128; ++r) {
      int e = tid + 128 * r;
      int nn, kk;
      if (g.transB) { kk = e % BK; nn = e / BK; } else { nn = e % BN; kk = e / BN; }
      int64_t n = bn0 + nn, k = k0 + kk;
      bool ok = (n < g.N) && (k < g.K);
      const z* src = ok ? (g.transB ? B + n * g.ldb + k : B + k * g.ldb + n) : B;
      cp_async16(&Bs[st][kk][nn], src, ok);
    }
  };

  double accr[MT][NT][2], acci[MT][NT][2];
#pragma unroll
  for (int i = 0; i < MT; ++i)
#pragma unroll
    for (int j = 0; j < NT; ++j) accr[i][j][0] = accr[i][j][1] = acci[i][j][0] = acci[i][j][1] = 0.0;

  const double sa = g.conjA ? -1.0 : 1.0, sb = g.conjB ? -1.0 : 1.0;
  const int64_t nk = (g.K + BK - 1) / BK;
  load_stage(0, 0);
  cp_async_commit();
  for (int64_t kt = 0; kt < nk; ++kt) {
    if (kt + 1 < nk) {
      load_stage((kt + 1) & 1, (kt + 1) * BK);
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const int st = kt & 1;
#pragma unroll
    for (int ks = 0; ks < BK / 4; ++ks) {
      const int kr = ks * 4 + (lane & 3);
      double ar[MT], ai[MT], br[NT], bi[NT], bin[NT];
#pragma unroll
      for (int i = 0; i < MT; ++i) {
        z a = As[st][kr][wm0 + i * 8 + (lane >> 2)];
        ar[i] = a.x;
        ai[i] = sa * a.y;
      }
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        z b = Bs[st][kr][wn0 + j * 8 + (lane >> 2)];
        br[j] = b.x;
        bi[j] = sb * b.y;
        bin[j] = -bi[j];
      }
#pragma unroll
      for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < NT; ++j) {
          dmma(accr[i][j][0], accr[i][j][1], ar[i], br[j]);
          dmma(acci[i][j][0], acci[i][j][1], ar[i], bi[j]);
          dmma(accr[i][j][0], accr[i][j][1], ai[i], bin[j]);
          dmma(acci[i][j][0], acci[i][j][1], ai[i], br[j]);
        }
    }
    __syncthreads();
  }

  // epilogue: C = alpha * acc + beta * C
#pragma unroll
  for (int i = 0; i < MT; ++i) {
    const int64_t m = bm0 + wm0 + i * 8 + (lane >> 2);
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < NT; ++j) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t n = bn0 + wn0 + j * 8 + 2 * (lane & 3) + h;
        if (n >= g.N) continue;
        z acc = make_double2(accr[i][j][h], acci[i][j][h]);
        z out = zmul(g.alpha, acc);
        z* cp = C + m * g.ldc + n;
        if (g.beta.x != 0.0 || g.beta.y != 0.0) out = zadd(out, zmul(g.beta, *cp));
        *cp = out;
      }
    }
  }
}

template <int BM, int BN, int WM, int WN>
cudaError_t launch(const ZGemmArgs& g, cudaStream_t s) {
  dim3 grid((unsigned)((g.N + BN - 1) / BN), (unsigned)((g.M + BM - 1) / BM), (unsigned)g.batch);
  zgemm_dmma_kernel<BM, BN, WM, WN><<<grid, 128, 0, s>>>(g);
  return cudaGetLastError();
}

}  // namespace

int64_t zgemm_f64_tiles(const ZGemmArgs& g, int cfg) {
  const int bm = cfg == 0 ? 64 : 32, bn = cfg == 2 ? 32 : 64;
  return ((g.M + bm - 1) / bm) * ((g.N + bn - 1) / bn) * (int64_t)g.batch;
}

cudaError_t zgemm_f64(const ZGemmArgs& g, cudaStream_t s, int cfg) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
  if (g.K <= 0) {
    // C = beta * C only
    ZGemmArgs h = g;
    return zscale_matrix(h, s);
  }
  if (g.batch > 65535 || (g.M + 31) / 32 > 65535) return cudaErrorInvalidValue;
  if (cfg < 0) {
    // Smallest tile count that still gives every SM >= 8 tiles; else the smallest tiles.
    cfg = 2;
    if (zgemm_f64_tiles(g, 0) >= 152 * 8) cfg = 0;
    else if (zgemm_f64_tiles(g, 1) >= 152 * 8) cfg = 1;
  }
  switch (cfg) {
    case 0: return launch<64, 64, 2, 2>(g, s);
    case 1: return launch<32, 64, 2, 2>(g, s);
    default: return launch<32, 32, 2, 2>(g, s);
  }
}

}  // namespace ccsd
