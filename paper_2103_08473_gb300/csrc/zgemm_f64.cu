// Complex double-precision GEMM on the FP64 tensor path (mma.sync m8n8k4.f64).
//
//   C[b] = alpha * opA(A[b]) * opB(B[b]) + beta * C[b]     (row-major, complex double)
//
// Every contraction of the CCSD residual in the FP64 mode reduces to this call
// after index permutation (transpose-transpose-GEMM-transpose). A complex
// multiply-add is either four real products (4M): Re += Ar Br - Ai Bi,
// Im += Ar Bi + Ai Br, as four DMMAs per 8x8x4 tile pair into real and imaginary
// accumulators; or three (3M, Gauss/Karatsuba): P1 += Ar Br, P2 += Ai Bi,
// P3 += (Ar + Ai)(Br + Bi) into three accumulators, then Re = P1 - P2 and
// Im = P3 - P1 - P2 once per output in the epilogue. On this chip DADD, DFMA and
// DMMA share one FP64 rate, so 3M trades one DMMA (256 multiply-adds) per tile
// pair for two fragment sums per thread: about 1.28x fewer FP64 operations, with a
// rounding error still bounded by a small multiple of eps (|Ar|+|Ai|)(|Br|+|Bi|) per
// product.
//
// Tiles are staged in shared memory with cp.async (16-byte copies of one complex
// element each, so any operand layout and transpose maps onto the same
// [k][m] / [k][n] shared tiles) in a two-stage pipeline. Out-of-range elements
// are zero-filled by the copy. On this chip the FP64 pipe (about 1 TFLOP/s for
// the whole GPU) is the bound: a 152-SM GPU retires one m8n8k4 DMMA per SM every
// ~150 clocks, so the kernel favours many small tiles (good load balance across
// SMs) over operand reuse. Blocks are rasterised so that consecutive blocks
// share a tile of the larger operand (read once from DRAM, then from L2), and
// GEMMs with few output tiles but a long K (e.g. o x o outputs summed over o v^2)
// split K across blocks; the split partials are reduced in a fixed order, so the
// result does not depend on scheduling.
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

// x or -x by the sign bit (integer pipe, keeps conjugation off the FP64 pipe)
__device__ __forceinline__ double flip(double x, unsigned long long sign) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)sign);
}

__device__ __forceinline__ void dmma(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

// BM x BN block tile, 4 warps arranged WM x WN, each warp (BM/WM) x (BN/WN).
template <int BM, int BN, int WM, int WN, bool M3>
__global__ void __launch_bounds__(128) zgemm_dmma_kernel(ZGemmArgs g, int mfast, int64_t tm, int64_t tn, int splits,
                                                         int64_t kslice) {
  constexpr int WTM = BM / WM, WTN = BN / WN;
  constexpr int MT = WTM / 8, NT = WTN / 8;
  __shared__ __align__(16) z As[2][BK][BM];
  __shared__ __align__(16) z Bs[2][BK][BN];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm0 = (warp / WN) * WTM, wn0 = (warp % WN) * WTN;
  // linear tile index over grid x; M tiles fastest when mfast, else N tiles
  const int64_t lin = blockIdx.x;
  const int64_t bm0 = (mfast ? lin % tm : lin / tn) * BM;
  const int64_t bn0 = (mfast ? lin / tm : lin % tn) * BN;
  const int64_t bz = blockIdx.z / splits, sp = blockIdx.z % splits;
  const z* __restrict__ A = g.A + bz * g.sA;
  const z* __restrict__ B = g.B + bz * g.sB;
  z* __restrict__ C = g.C + bz * g.sC;
  const int64_t kbeg = sp * kslice;
  const int64_t kend = kbeg + kslice < g.K ? kbeg + kslice : g.K;

  auto load_stage = [&](int st, int64_t k0) {
    // A tile: BM x BK complex
#pragma unroll
    for (int r = 0; r < (BM * BK + 127) / 128; ++r) {
      int e = tid + 128 * r;
      if (e >= BM * BK) break;
      int mm, kk;
      if (g.transA) { mm = e % BM; kk = e / BM; } else { kk = e % BK; mm = e / BK; }
      int64_t m = bm0 + mm, k = k0 + kk;
      bool ok = (m < g.M) && (k < kend);
      const z* src = ok ? (g.transA ? A + k * g.lda + m : A + m * g.lda + k) : A;
      cp_async16(&As[st][kk][mm], src, ok);
    }
#pragma unroll
    for (int r = 0; r < (BN * BK + 127) / 128; ++r) {
      int e = tid + 128 * r;
      if (e >= BN * BK) break;
      int nn, kk;
      if (g.transB) { kk = e % BK; nn = e / BK; } else { nn = e % BN; kk = e / BN; }
      int64_t n = bn0 + nn, k = k0 + kk;
      bool ok = (n < g.N) && (k < kend);
      const z* src = ok ? (g.transB ? B + n * g.ldb + k : B + k * g.ldb + n) : B;
      cp_async16(&Bs[st][kk][nn], src, ok);
    }
  };

  // 4M: acc0 = Re, acc1 = Im.  3M: acc0 = P1 (Ar Br), acc1 = P2 (Ai Bi), acc2 = P3 ((Ar+Ai)(Br+Bi)).
  constexpr int NACC = M3 ? 3 : 2;
  double acc[NACC][MT][NT][2];
#pragma unroll
  for (int q = 0; q < NACC; ++q)
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
      for (int j = 0; j < NT; ++j) acc[q][i][j][0] = acc[q][i][j][1] = 0.0;

  const unsigned long long sga = g.conjA ? 0x8000000000000000ull : 0ull;
  const unsigned long long sgb = g.conjB ? 0x8000000000000000ull : 0ull;
  const int64_t nk = kend > kbeg ? (kend - kbeg + BK - 1) / BK : 0;
  if (nk > 0) load_stage(0, kbeg);
  cp_async_commit();
  for (int64_t kt = 0; kt < nk; ++kt) {
    if (kt + 1 < nk) {
      load_stage((kt + 1) & 1, kbeg + (kt + 1) * BK);
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
      double ar[MT], ai[MT], br[NT], bi[NT];
#pragma unroll
      for (int i = 0; i < MT; ++i) {
        z a = As[st][kr][wm0 + i * 8 + (lane >> 2)];
        ar[i] = a.x;
        ai[i] = flip(a.y, sga);
      }
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        z b = Bs[st][kr][wn0 + j * 8 + (lane >> 2)];
        br[j] = b.x;
        bi[j] = flip(b.y, sgb);
      }
      if constexpr (M3) {
        double sa[MT], sb[NT];
#pragma unroll
        for (int i = 0; i < MT; ++i) sa[i] = ar[i] + ai[i];
#pragma unroll
        for (int j = 0; j < NT; ++j) sb[j] = br[j] + bi[j];
#pragma unroll
        for (int i = 0; i < MT; ++i)
#pragma unroll
          for (int j = 0; j < NT; ++j) {
            dmma(acc[0][i][j][0], acc[0][i][j][1], ar[i], br[j]);
            dmma(acc[1][i][j][0], acc[1][i][j][1], ai[i], bi[j]);
            dmma(acc[2][i][j][0], acc[2][i][j][1], sa[i], sb[j]);
          }
      } else {
#pragma unroll
        for (int i = 0; i < MT; ++i)
#pragma unroll
          for (int j = 0; j < NT; ++j) {
            const double bin = flip(bi[j], 0x8000000000000000ull);
            dmma(acc[0][i][j][0], acc[0][i][j][1], ar[i], br[j]);
            dmma(acc[1][i][j][0], acc[1][i][j][1], ar[i], bi[j]);
            dmma(acc[0][i][j][0], acc[0][i][j][1], ai[i], bin);
            dmma(acc[1][i][j][0], acc[1][i][j][1], ai[i], br[j]);
          }
      }
    }
    __syncthreads();
  }

  // epilogue: C = alpha * acc + beta * C, or the raw split partial into the workspace
  z* __restrict__ W = splits > 1 ? g.ws + (sp * (int64_t)g.batch + bz) * g.M * g.N : nullptr;
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
        z v;
        if constexpr (M3) {
          const double p1 = acc[0][i][j][h], p2 = acc[1][i][j][h];
          v = make_double2(p1 - p2, acc[2][i][j][h] - p1 - p2);
        } else {
          v = make_double2(acc[0][i][j][h], acc[1][i][j][h]);
        }
        if (splits > 1) {
          W[m * g.N + n] = v;
          continue;
        }
        z out = zmul(g.alpha, v);
        z* cp = C + m * g.ldc + n;
        if (g.beta.x != 0.0 || g.beta.y != 0.0) out = zadd(out, zmul(g.beta, *cp));
        *cp = out;
      }
    }
  }
}

// C[b][m][n] = alpha * sum_s ws[s][b][m][n] + beta * C[b][m][n], summed in split order.
__global__ void splitk_reduce_kernel(ZGemmArgs g, int splits) {
  const int64_t MN = g.M * g.N, total = MN * g.batch;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e / MN, r = e % MN, m = r / g.N, n = r % g.N;
    double ar = 0.0, ai = 0.0;
    for (int s = 0; s < splits; ++s) {
      const z w = g.ws[(s * (int64_t)g.batch + b) * MN + r];
      ar += w.x;
      ai += w.y;
    }
    z out = zmul(g.alpha, make_double2(ar, ai));
    z* cp = g.C + b * g.sC + m * g.ldc + n;
    if (g.beta.x != 0.0 || g.beta.y != 0.0) out = zadd(out, zmul(g.beta, *cp));
    *cp = out;
  }
}

constexpr int kSlotsPerSM = 5;  // resident 128-thread blocks per SM at <= 96 registers
constexpr int kSMs = 152;
constexpr int64_t kMaxSplitWs = int64_t(1) << 25;  // split-K partials kept under 512 MB

int splits_for(const ZGemmArgs& g, int64_t tiles) {
  const int64_t slots = (int64_t)kSMs * kSlotsPerSM;
  if (tiles >= slots) return 1;
  int64_t s = (2 * slots + tiles - 1) / tiles;
  const int64_t kmax = g.K / 64;  // at least 64 complex K per slice
  if (s > kmax) s = kmax;
  if (s > 1024) s = 1024;
  while (s > 1 && s * g.M * g.N * g.batch > kMaxSplitWs) s /= 2;
  if (s * g.batch > 65535) s = 65535 / g.batch;
  return s < 1 ? 1 : (int)s;
}

template <int BM, int BN, int WM, int WN, bool M3>
cudaError_t launch(const ZGemmArgs& g, cudaStream_t s) {
  const int64_t tm = (g.M + BM - 1) / BM, tn = (g.N + BN - 1) / BN;
  int splits = splits_for(g, tm * tn * g.batch);
  // a workspace smaller than the preferred split count takes as many partials as it holds
  if (splits > 1) {
    const int64_t fit = g.ws == nullptr ? 0 : g.ws_elems / (g.M * g.N * g.batch);
    if (fit < splits) splits = fit >= 2 ? (int)fit : 1;
  }
  const int64_t kslice = splits > 1 ? ((g.K + splits - 1) / splits + BK - 1) / BK * BK : g.K;
  if (splits > 1) splits = (int)((g.K + kslice - 1) / kslice);
  // rasterise so that consecutive blocks share a tile of the larger operand
  // (A holds M*K elements, B holds N*K): M-tiles fastest when B is the larger one
  const int mfast = g.M > g.N ? 0 : 1;
  if (tm * tn > 0x7fffffff || (int64_t)g.batch * splits > 65535) return cudaErrorInvalidValue;
  dim3 grid((unsigned)(tm * tn), 1, (unsigned)(g.batch * splits));
  zgemm_dmma_kernel<BM, BN, WM, WN, M3><<<grid, 128, 0, s>>>(g, mfast, tm, tn, splits, kslice);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || splits == 1) return e;
  splitk_reduce_kernel<<<grid_for(g.M * g.N * g.batch, 256), 256, 0, s>>>(g, splits);
  return cudaGetLastError();
}

}  // namespace

// Tile configurations: {BM, BN}. 0-2 use 2x2 warps, 3-6 use 1x4 warps (BM = 8 * MT rows).
struct Cfg {
  int bm, bn;
};
constexpr Cfg kCfgs[] = {{64, 64}, {32, 64}, {32, 32}, {16, 64}, {24, 64}, {40, 64}, {48, 64}};
constexpr int kNumCfgs = sizeof(kCfgs) / sizeof(kCfgs[0]);

int64_t zgemm_f64_tiles(const ZGemmArgs& g, int cfg) {
  const int bm = kCfgs[cfg].bm, bn = kCfgs[cfg].bn;
  return ((g.M + bm - 1) / bm) * ((g.N + bn - 1) / bn) * (int64_t)g.batch;
}

// Cost model: padded work (rows and columns rounded up to the tile) plus one tile per
// SM for the tail of the last wave; among equal costs the configuration listed first.
static int pick_cfg(const ZGemmArgs& g) {
  int best = 0;
  double best_cost = -1.0;
  for (int c = 0; c < kNumCfgs; ++c) {
    const double bm = kCfgs[c].bm, bn = kCfgs[c].bn;
    const double work = (double)((g.M + kCfgs[c].bm - 1) / kCfgs[c].bm) * bm *
                        (double)((g.N + kCfgs[c].bn - 1) / kCfgs[c].bn) * bn * g.batch;
    const double cost = work + (double)kSMs * bm * bn;
    // the 64x64 tile only when it still gives every SM >= 8 tiles
    if (c == 0 && zgemm_f64_tiles(g, 0) < kSMs * 8) continue;
    if (best_cost < 0 || cost < best_cost * 0.999) {
      best = c;
      best_cost = cost;
    }
  }
  return best;
}

int64_t zgemm_f64_workspace(const ZGemmArgs& g) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0) return 0;
  const int s = splits_for(g, zgemm_f64_tiles(g, pick_cfg(g)));
  return s > 1 ? (int64_t)s * g.M * g.N * g.batch : 0;
}

cudaError_t zgemm_f64(const ZGemmArgs& g, cudaStream_t s, int cfg) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
  if (g.K <= 0) return zscale_matrix(g, s);
  if (g.batch > 65535) return cudaErrorInvalidValue;
  if (cfg < 0 || cfg >= kNumCfgs) cfg = pick_cfg(g);
  if (g.mult4) {
    switch (cfg) {
      case 0: return launch<64, 64, 2, 2, false>(g, s);
      case 1: return launch<32, 64, 2, 2, false>(g, s);
      case 2: return launch<32, 32, 2, 2, false>(g, s);
      case 3: return launch<16, 64, 1, 4, false>(g, s);
      case 4: return launch<24, 64, 1, 4, false>(g, s);
      case 5: return launch<40, 64, 1, 4, false>(g, s);
      default: return launch<48, 64, 1, 4, false>(g, s);
    }
  }
  switch (cfg) {
    case 0: return launch<64, 64, 2, 2, true>(g, s);
    case 1: return launch<32, 64, 2, 2, true>(g, s);
    case 2: return launch<32, 32, 2, 2, true>(g, s);
    case 3: return launch<16, 64, 1, 4, true>(g, s);
    case 4: return launch<24, 64, 1, 4, true>(g, s);
    case 5: return launch<40, 64, 1, 4, true>(g, s);
    default: return launch<48, 64, 1, 4, true>(g, s);
  }
}

}  // namespace ccsd
