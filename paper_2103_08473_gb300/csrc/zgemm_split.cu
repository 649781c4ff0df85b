// Split-precision complex GEMM on tcgen05 (see split.h for the scheme).
//
// Kernel structure (one CTA per 128 x BN complex output tile, BN = 128, 96 or 64;
// 6 warps):
//   warp 0  TMA producer: per K block (128 bytes of digits per row) and slice
//           pair of the current level group, loads the A_re, A_im (128 rows) and
//           B_re, B_im (BN rows) digit tiles into a 3- or 4-stage ring of
//           128B-swizzled shared tiles. K blocks are the outer loop and the group's
//           pairs the inner one, so all CTAs walk the same narrow K front of the
//           small operand and it stays in L2.
//   warp 1  allocates the TMEM columns (512; 256 for BN = 64); one thread issues
//           the UMMAs (M = 128, N = BN, K = 32 e4m3 / 16 bf16 per instruction):
//             re += Ar Br, re += Ai (-Bi), im += Ar Bi, im += Ai Br
//           into one of two TMEM accumulator sets (re, im: BN columns each),
//           and commits each smem stage back to the producer.
//   warps 2-5  epilogue: after each level group, read the FP32 accumulator rows
//           (tcgen05.ld 32x32b), scale by 2^(e_row + e_col - b L) and add
//           alpha * value into C in FP64 by reductions in L2 (red.global.add.f64:
//           each element has one owning thread, so the order of its additions is
//           fixed), then release the TMEM set. With the operands swapped (a short M
//           on the BN side) the tile is the transpose of C's and each warp adds into
//           32 consecutive elements of a row of C.
// Where the output is two or four BN tiles wide, pairs of CTAs with the same M tile and K
// range run as clusters of two that multicast the shared 128-row tile (see CL below);
// outputs with many tiles both ways take them in bands of M tiles so that a wave shares
// a few A and B tiles in L2.
// Every mbarrier wait is bounded (clock64 budget); a wait that gives up sets the
// error word and the CTA drains its in-flight copies, frees TMEM and exits.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cudaTypedefs.h>

#include <climits>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "split.h"

namespace ccsd {
namespace {

constexpr int kMaxLevels = 16;

// Shared-memory and tensor-memory shape of the main kernel for an output tile of 128 x BN
// (BN = 128, 96 or 64 columns): a stage holds the A_re, A_im tiles (128 rows) and the B_re,
// B_im tiles (BN rows) of one K block and digit pair; the two TMEM accumulator sets hold
// BN real and BN imaginary FP32 columns each.
template <int BN>
struct MainTile {
  static constexpr uint32_t kTileA = 128 * 128;
  static constexpr uint32_t kTileB = BN * 128;
  static constexpr uint32_t kStageBytes = 2 * kTileA + 2 * kTileB;
  static constexpr int kStages = BN == 128 ? 3 : 4;
  static constexpr uint32_t kSmemBytes = kStages * kStageBytes + 1024 + 256;
  static constexpr uint32_t kTmemCols = 4 * BN <= 256 ? 256u : 512u;
  static_assert(BN == 128 || BN == 96 || BN == 64, "output tile width");
  static_assert(kSmemBytes <= 232448, "shared memory per CTA");
};

// Level groups are enumerated on the fly by every role in the same order:
// for level L = 0..lmax (weight 2^{-b(L+2)}), for K chunks of kbper[L] blocks
// (short enough that every FP32 partial sum of the level stays below 2^24),
// intersected with this CTA's K range [klo, khi); the pairs of a level are
// (p, L - p), p = max(0, L - s + 1) .. min(L, s - 1).
struct SplitArgs {
  int64_t M, N;
  int64_t a_row0, b_row0;   // first digit row of each operand (row views of a larger digit set)
  int tiles_m, tiles;       // output tiles along M, and in total
  int s, b, lmax, kblocks;  // digits, bits, last level, K blocks
  int kbper[kMaxLevels];    // K blocks per exact chunk, per level
  int ksplits, kb_split;    // CTAs along K and K blocks each
  z* C;
  int64_t ldc;
  z alpha;
  z* part;                  // ksplits > 1: FP64 partial products [ks][M][N] (pre-zeroed)
  const double* rs;
  const double* cs;
  double* probe;            // probe output (real M x N) or null
  int* err;
  long long wait_cycles;
  int stall_loads;          // self-test only: the producer issues no loads, so the first wait runs out
  int transC;               // 1: the kernel's (m, n) is the caller's C[n][m] (operands swapped)
  int conjA, conjB;         // conjugate the kernel's A / B operand (the sign of its imaginary digits)
  int a_stream;             // clusters only: A's tile is read by no other resident cluster (evict first)
  int group;                // no cluster: M tiles per band of the tile order (1: M tiles step first)
};

// ---- PTX wrappers ----------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of the given parity; gives up after `budget` clock cycles or
// when another role raised the abort flag (unless ignore_abort).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long budget, volatile int* abort_flag,
                                          bool ignore_abort = false) {
  const long long t0 = clock64();
  while (!mbar_test(bar, parity)) {
    if (!ignore_abort && *abort_flag) return false;
    if (clock64() - t0 > budget) return false;
  }
  return true;
}

// One box of digits: K offset x (a multiple of the 128-byte row segment), row y, plane z
// (digit p's real part at z = 2p, imaginary at 2p + 1). Rows past the set read as zeros.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// The same box written to every CTA of the cluster in cta_mask, at this CTA's shared offset, each
// destination's mbarrier (same offset) receiving the byte count.
__device__ __forceinline__ void tma_load_3d_mc(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar,
                                               uint16_t cta_mask) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster"
      " [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(bar), "h"(cta_mask)
      : "memory");
}
// As above, with an L2 eviction policy for the copied lines.
__device__ __forceinline__ void tma_load_3d_mc_hint(uint32_t dst, const CUtensorMap* map, int x, int y, int z,
                                                    uint32_t bar, uint16_t cta_mask, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster.L2::cache_hint"
      " [%0], [%1, {%2, %3, %4}], [%5], %6, %7;" ::"r"(dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(bar), "h"(cta_mask), "l"(policy)
      : "memory");
}
// Lines read once per pass (a digit stream with no reuse among the resident CTAs) go first.
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release;\nbarrier.cluster.wait.acquire;" ::: "memory");
}

// *p += v at L2 (no value returned, so the issuing thread does not wait for it).
__device__ __forceinline__ void red_add_f64(double* p, double v) {
  asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// d * 2^k by adding k to the exponent field (integer pipe; the FP64 pipe of this chip is the
// scarce one): exact, and the same value as the FP64 multiply, whenever both d and the result are
// normal numbers; zero, subnormal or out-of-range cases take the FP64 multiply.
__device__ __forceinline__ double scale_pow2(double d, int k) {
  const long long bits = __double_as_longlong(d);
  const int e = (int)((bits >> 52) & 0x7FF);
  if (e == 0 || e + k <= 0 || e + k >= 0x7FF) return d * ldexp(1.0, k);
  return __longlong_as_double(bits + ((long long)k << 52));
}
// An FP32 accumulator value (an integer below 2^24 in magnitude, so zero or normal) times 2^k, as
// a double, built by integer arithmetic: the sign moves to bit 63, the exponent is rebiased by
// 1023 - 127 + k and the mantissa shifted into place. The same value as (double)v * 2^k; out of
// the normal range it takes that FP64 path.
__device__ __forceinline__ double f32_times_pow2(uint32_t fbits, int k) {
  if ((fbits & 0x7FFFFFFFu) == 0u) return 0.0;
  const long long e = (long long)((fbits >> 23) & 0xFFu) - 127 + 1023 + k;
  if (e <= 0 || e >= 0x7FF) return (double)__uint_as_float(fbits) * ldexp(1.0, k);
  const unsigned long long bits = ((unsigned long long)(fbits >> 31) << 63) | ((unsigned long long)e << 52) |
                                  ((unsigned long long)(fbits & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)bits);
}
// The power of two of a positive normal double that is one (a digit row or column scale).
__device__ __forceinline__ int pow2_exponent(double s) {
  return (int)((__double_as_longlong(s) >> 52) & 0x7FF) - 1023;
}

// Shared-memory matrix descriptor: K-major operand in the canonical 128-byte
// swizzled layout written by TMA (8-row groups 1024 bytes apart).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                    // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset: 8 rows x 128 bytes
  d |= (uint64_t)1 << 46;                    // descriptor version
  d |= (uint64_t)2 << 61;                    // 128-byte swizzle
  return d;
}

// Instruction descriptor: D = F32, A/B K-major, M = 128, N = n (a multiple of 16, <= 256).
__host__ __device__ constexpr uint32_t make_idesc(int kind, int negB, uint32_t n = 128u) {
  return (1u << 4) | ((kind == kSplitBF16 ? 1u : 0u) << 7) | ((kind == kSplitBF16 ? 1u : 0u) << 10) |
         ((uint32_t)negB << 14) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

template <int KIND>
__device__ __forceinline__ void umma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (KIND == kSplitBF16) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  }
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// Arrive on the mbarrier at this shared offset in every CTA of cta_mask once the MMAs issued so
// far have completed.
__device__ __forceinline__ void umma_commit_mc(uint32_t bar, uint16_t cta_mask) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::
                   "r"(bar), "h"(cta_mask)
               : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---- the GEMM kernel ----------------------------------------------------------

// CL = 2: the two CTAs of a cluster take the two N tiles of one M tile and K range; each loads
// one part (real or imaginary) of the shared 128-row digit tile into both CTAs' shared memory
// (TMA multicast), so the long operand crosses the memory system once per cluster, and each
// releases a stage to both producers.
template <int KIND, bool PROBE, int BN, int CL>
__global__ void __launch_bounds__(192, 1)
    split_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 const __grid_constant__ SplitArgs args) {
  static_assert(CL == 1 || (CL == 2 && !PROBE), "cluster of two CTAs (both parts of A) or none");
  constexpr uint16_t kMask = (uint16_t)((1u << CL) - 1u);
  using T = MainTile<BN>;
  constexpr int kStages = T::kStages;
  constexpr uint32_t kStageBytes = T::kStageBytes, kTileA = T::kTileA, kTileB = T::kTileB;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  const uint32_t bar0 = base + kStages * kStageBytes;
  // barrier addresses (8 bytes each)
  auto full = [&](int s) { return bar0 + 8u * s; };
  auto empty = [&](int s) { return bar0 + 8u * (kStages + s); };
  auto accfull = [&](int b) { return bar0 + 8u * (2 * kStages + b); };
  auto accempty = [&](int b) { return bar0 + 8u * (2 * kStages + 2 + b); };
  const uint32_t done = bar0 + 8u * (2 * kStages + 4);
  uint8_t* gen = smem_raw + (base - raw);
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(gen + kStages * kStageBytes + 8 * (2 * kStages + 5));
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int tm, tn, ks;
  uint32_t crank = 0;
  if constexpr (CL > 1) {
    // cluster u of the grid: M tile u % tiles_m, N tiles CL (u / tiles_m) + rank, K range u / units
    crank = cluster_rank();
    const int units = args.tiles / CL, u = blockIdx.x / CL;
    ks = u / units;
    tm = (u % units) % args.tiles_m;
    tn = ((u % units) / args.tiles_m) * CL + (int)crank;
  } else {
    const int tile = blockIdx.x % args.tiles;
    ks = blockIdx.x / args.tiles;
    if (args.group > 1) {
      // bands of `group` M tiles, N tiles stepping within a band: the CTAs resident at once
      // share a few A and B tiles instead of streaming every A tile against one or two B tiles
      const int tiles_n = args.tiles / args.tiles_m, per = args.group * tiles_n;
      const int m_first = (tile / per) * args.group, rows = min(args.tiles_m - m_first, args.group);
      tm = m_first + (tile % per) % rows;
      tn = (tile % per) / rows;
    } else {
      tm = tile % args.tiles_m;
      tn = tile / args.tiles_m;
    }
  }
  const int64_t m0 = (int64_t)tm * 128, n0 = (int64_t)tn * BN;
  const int klo = ks * args.kb_split, khi = min(args.kblocks, klo + args.kb_split);
  constexpr int BKE = KIND == kSplitBF16 ? 64 : 128;  // digits per 128-byte row segment

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), CL);  // every CTA of the cluster releases the stage
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accfull(b), 1);
      mbar_init(accempty(b), 128);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                 "r"(T::kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    tc_fence_before();
  }
  __syncthreads();
  // the peer's copies and releases reach this CTA's barriers only once they are initialised
  if constexpr (CL > 1) cluster_sync_all();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;
  const long long budget = args.wait_cycles;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0 && !args.stall_loads) {
      const uint64_t a_policy = policy_evict_first();
      int it = 0;
      bool ok = true;
      for (int L = 0; L <= args.lmax && ok; ++L)
        for (int c0 = 0; c0 < args.kblocks && ok; c0 += args.kbper[L]) {
          const int gb0 = max(c0, klo), gb1 = min(c0 + args.kbper[L], khi);
          const int p0 = max(0, L - args.s + 1), p1 = min(L, args.s - 1);
          for (int kb = gb0; kb < gb1 && ok; ++kb)
            for (int p = p0; p <= p1; ++p, ++it) {
              const int q = L - p;
              const int st = it % kStages;
              const uint32_t ph = (uint32_t)(it / kStages) & 1u;
              if (!mbar_wait(empty(st), ph ^ 1u, budget, abort_flag)) {
                ok = false;
                break;
              }
              const uint32_t sa = base + st * kStageBytes;
              const int x = kb * BKE;
              mbar_expect_tx(full(st), PROBE ? kTileA + kTileB : 2 * (kTileA + kTileB));
              const int64_t ya = args.a_row0 + m0, yb = args.b_row0 + n0;
              if constexpr (CL > 1) {
                // this CTA's part of the shared A tile, into the same stage of every CTA
                if (args.a_stream)
                  tma_load_3d_mc_hint(sa + crank * kTileA, &tmA, x, (int)ya, p * 2 + (int)crank, full(st), kMask,
                                      a_policy);
                else
                  tma_load_3d_mc(sa + crank * kTileA, &tmA, x, (int)ya, p * 2 + (int)crank, full(st), kMask);
              } else {
                tma_load_3d(sa, &tmA, x, (int)ya, p * 2 + 0, full(st));
                if (!PROBE) tma_load_3d(sa + kTileA, &tmA, x, (int)ya, p * 2 + 1, full(st));
              }
              tma_load_3d(sa + 2 * kTileA, &tmB, x, (int)yb, q * 2 + 0, full(st));
              if (!PROBE) tma_load_3d(sa + 2 * kTileA + kTileB, &tmB, x, (int)yb, q * 2 + 1, full(st));
            }
        }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(args.err, 1);
      }
      // drain: every copy this thread issued must have landed before the CTA exits
      const int last = it;
      for (int j = (last > kStages ? last - kStages : 0); j < last; ++j)
        mbar_wait(full(j % kStages), (uint32_t)(j / kStages) & 1u, budget, abort_flag, true);
      // and every CTA of the cluster has released the last stages (their arrivals land here)
      if constexpr (CL > 1)
        for (int j = (last > kStages ? last - kStages : 0); j < last; ++j)
          mbar_wait(empty(j % kStages), (uint32_t)(j / kStages) & 1u, budget, abort_flag, true);
    }
  } else if (warp == 1) {
    // ---------------- UMMA issuer ----------------
    if (lane == 0) {
      const uint32_t id = make_idesc(KIND, 0, BN), idn = make_idesc(KIND, 1, BN);
      const uint32_t idRI = (args.conjA ^ args.conjB) ? id : idn, idIm1 = args.conjB ? idn : id,
                     idIm2 = args.conjA ? idn : id;
      int it = 0, g = 0;
      bool ok = true;
      for (int L = 0; L <= args.lmax && ok; ++L)
        for (int c0 = 0; c0 < args.kblocks && ok; c0 += args.kbper[L]) {
          const int gb0 = max(c0, klo), gb1 = min(c0 + args.kbper[L], khi);
          if (gb0 >= gb1) continue;
          const int p0 = max(0, L - args.s + 1), p1 = min(L, args.s - 1);
          const int buf = g & 1, use = g >> 1;
          if (!mbar_wait(accempty(buf), ((uint32_t)use & 1u) ^ 1u, budget, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t dre = tmem + (uint32_t)buf * (2u * BN), dim = dre + (uint32_t)BN;
          bool first = true;
          for (int kb = gb0; kb < gb1 && ok; ++kb)
            for (int p = p0; p <= p1; ++p, ++it) {
              const int st = it % kStages;
              const uint32_t ph = (uint32_t)(it / kStages) & 1u;
              if (!mbar_wait(full(st), ph, budget, abort_flag)) {
                ok = false;
                break;
              }
              tc_fence_after();
              const uint32_t sa = base + st * kStageBytes;
              // descriptors of the stage's four tiles; each 32-byte K step adds 2 to the start address
              // (16-byte units), the issuing thread's only per-MMA arithmetic
              const uint64_t aR0 = sw128_desc(sa), aI0 = sw128_desc(sa + kTileA);
              const uint64_t bR0 = sw128_desc(sa + 2 * kTileA), bI0 = sw128_desc(sa + 2 * kTileA + kTileB);
#pragma unroll
              for (int kk = 0; kk < 4; ++kk) {
                const uint32_t acc = (first && kk == 0) ? 0u : 1u;
                const uint64_t o = 2u * (uint64_t)kk;
                umma<KIND>(dre, aR0 + o, bR0 + o, id, acc);
                if (!PROBE) {
                  // conjugating an operand flips the sign of its imaginary digits' products
                  umma<KIND>(dre, aI0 + o, bI0 + o, idRI, 1u);
                  umma<KIND>(dim, aR0 + o, bI0 + o, idIm1, acc);
                  umma<KIND>(dim, aI0 + o, bR0 + o, idIm2, 1u);
                }
              }
              if constexpr (CL > 1)
                umma_commit_mc(empty(st), kMask);
              else
                umma_commit(empty(st));
              first = false;
            }
          if (ok) umma_commit(accfull(buf));
          ++g;
        }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(args.err, 2);
      }
      // all issued MMAs complete before TMEM is released
      umma_commit(done);
      mbar_wait(done, 0u, budget, abort_flag, true);
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: warps 2..5 ----------------
    const int q4 = warp & 3;
    const int64_t m = m0 + q4 * 32 + lane;
    const bool mrow = m < args.M;
    const double rsc = (!PROBE && mrow) ? args.rs[m] : 0.0;
    z* const out = args.ksplits > 1 ? args.part + (int64_t)ks * args.M * args.N : args.C;
    // transC: the kernel's (m, n) goes to out[n * ldo + m] (the partials likewise, in the
    // caller's orientation), so that the 32 lanes of a warp store 32 consecutive elements
    const int64_t ldo = args.ksplits > 1 ? (args.transC ? args.M : args.N) : args.ldc;
    const z alpha = args.ksplits > 1 ? make_double2(1.0, 0.0) : args.alpha;
    int g = 0;
    bool ok = true;
    for (int L = 0; L <= args.lmax && ok; ++L)
      for (int c0 = 0; c0 < args.kblocks && ok; c0 += args.kbper[L]) {
        const int gb0 = max(c0, klo), gb1 = min(c0 + args.kbper[L], khi);
        if (gb0 >= gb1) continue;
        const int buf = g & 1, use = g >> 1;
        if (!mbar_wait(accfull(buf), (uint32_t)use & 1u, budget, abort_flag)) {
          *abort_flag = 1;
          atomicOr(args.err, 4);
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t trow = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)buf * (2u * BN);
        const double gs = ldexp(1.0, -args.b * (L + 2));
        // alpha = +-1 (every K-split partial, and most calls): the accumulator values go to FP64 by
        // integer arithmetic, scaled by the row and column powers of two on the way, and are added
        // in L2, so no FP64 instruction runs on the SM; other alpha: a DMUL per part (and a complex
        // product for complex alpha)
        const bool real_alpha = alpha.y == 0.0;
        const bool unit_alpha = real_alpha && (alpha.x == 1.0 || alpha.x == -1.0);
        const uint32_t flip = (unit_alpha && alpha.x < 0.0) ? 0x80000000u : 0u;  // sign of alpha on the FP32 bits
        const int krow = (!PROBE && mrow) ? pow2_exponent(rsc) - args.b * (L + 2) : 0;
        const double rowf = rsc * gs * (real_alpha ? alpha.x : 1.0);
#pragma unroll 1
        for (int c = 0; c < BN; c += 32) {
          uint32_t re[32], im[32];
          tmem_ld32(trow + c, re);
          if (!PROBE) tmem_ld32(trow + BN + c, im);
          tmem_wait_ld();
          if (mrow && PROBE) {
            for (int j = 0; j < 32; ++j) {
              const int64_t n = n0 + c + j;
              if (n < args.N) args.probe[m * args.N + n] = (double)__uint_as_float(re[j]);
            }
          } else if (mrow) {
            // each output element belongs to this thread alone (one row of the tile, and its own
            // partial slice under a K split), so its additions land in a fixed order: fire-and-forget
            // reductions at L2 instead of a read, an add and a write-back per element
            const double* csc = args.cs + n0 + c;
            const int64_t left = args.N - (n0 + c);
            const int rem = left < 32 ? (int)left : 32;
            // transC: element (m, n) at out[n * ldo + m] (32 lanes, consecutive m); else out[m * ldo + n]
            double* o = reinterpret_cast<double*>(args.transC ? out + (n0 + c) * ldo + m : out + m * ldo + n0 + c);
            const int64_t step = 2 * (args.transC ? ldo : 1);  // doubles from column j to j + 1
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              if (j >= rem) break;
              const double sc = csc[j];
              double dx, dy;
              if (unit_alpha) {
                const int k = krow + pow2_exponent(sc);
                dx = f32_times_pow2(re[j] ^ flip, k);
                dy = f32_times_pow2(im[j] ^ flip, k);
              } else {
                const double f = rowf * sc;
                dx = (double)__uint_as_float(re[j]) * f;
                dy = (double)__uint_as_float(im[j]) * f;
                if (!real_alpha) {
                  const z w = zmul(alpha, make_double2(dx, dy));
                  dx = w.x;
                  dy = w.y;
                }
              }
              red_add_f64(o + j * step, dx);
              red_add_f64(o + j * step + 1, dy);
            }
          }
        }
        tc_fence_before();
        mbar_arrive(accempty(buf));
        ++g;
      }
  }
  __syncthreads();
  // no CTA leaves while its peer may still write to its shared memory or barriers
  if constexpr (CL > 1) cluster_sync_all();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(T::kTmemCols));
  }
}

// ---- the short-K GEMM kernel --------------------------------------------------
//
// For K of a few blocks the main kernel is bound by its FP64 flushes: every weight level is
// one group, so each output tile is read and rewritten once per level. Here every level
// keeps its own FP32 accumulator in tensor memory over the whole K (exact: K is within every
// level's bound), on 128 x 32 output tiles: level L's real and imaginary parts are TMEM
// columns 64 L .. 64 L + 31 and 64 L + 32 .. 64 L + 63 (at most 8 levels in 512 columns).
// The epilogue combines the levels in FP64 registers and writes each output once (after
// releasing tensor memory, so the next tile's products overlap the stores). With transC the
// kernel computes the transpose (its rows are the output's columns), so that the long
// dimension fills the 128-row tiles and the stores of a warp are contiguous. Persistent over
// tiles; every wait bounded, as in the main kernel.

constexpr int kSkAStages = 3;               // A tiles (one digit plane, real and imaginary)
constexpr int kSkBBufs = 2;                 // B buffers (every digit plane of one K block)
constexpr int kSkMaxLevels = 8;
constexpr uint32_t kSkTileA = 128 * 128;    // bytes of a 128-row x 128-byte digit tile
constexpr uint32_t kSkTileB = 32 * 128;     // bytes of a 32-row x 128-byte digit tile
constexpr uint32_t kSkAStage = 2 * kSkTileA;
constexpr uint32_t kSkBBuf = kSkMaxLevels * 2 * kSkTileB;
constexpr uint32_t kSkSmemBytes = kSkAStages * kSkAStage + kSkBBufs * kSkBBuf + 1024 + 256;
constexpr int kSkBN = 32;

__host__ __device__ constexpr uint32_t make_idesc_n32(int kind, int negB) {
  return (1u << 4) | ((kind == kSplitBF16 ? 1u : 0u) << 7) | ((kind == kSplitBF16 ? 1u : 0u) << 10) |
         ((uint32_t)negB << 14) | (((uint32_t)kSkBN >> 3) << 17) | ((128u >> 4) << 24);
}

// Order in which the short-K kernel takes the A digit planes: 0, s-1, 1, s-2, ... Plane p joins
// s - p products, so alternating heavy and light planes keeps each stage of the A ring busy
// long enough to cover the next plane's load. Each level's FP32 sum is exact in any order.
__device__ __forceinline__ int plane_at(int i, int s) { return (i & 1) ? s - 1 - (i >> 1) : (i >> 1); }

struct SmallKArgs {
  int64_t M, N, a_row0, b_row0;
  int tiles_m, tiles;
  int s, b, lmax, kblocks;
  z* C;
  int64_t ldc;
  z alpha, beta;
  int transC;
  const double* rs;
  const double* cs;
  int* err;
  long long wait_cycles;
  int conjA, conjB;  // conjugate the kernel's A / B operand
  int tiles_n;       // column tiles; nfast: consecutive tiles step through the columns first
  int nfast;
};

// Origin of a tile. With few column tiles (a short N), consecutive tiles, which neighbouring
// CTAs run at the same time, are the column tiles of one row tile: the A digits of that row tile
// come from DRAM once and from L2 for the others. Otherwise the row tiles step first.
__device__ __forceinline__ void sk_tile_origin(const SmallKArgs& a, int tile, int64_t& m0, int64_t& n0) {
  const int tm = a.nfast ? tile / a.tiles_n : tile % a.tiles_m;
  const int tn = a.nfast ? tile % a.tiles_n : tile / a.tiles_m;
  m0 = (int64_t)tm * 128;
  n0 = (int64_t)tn * kSkBN;
}

// Per K block: every B digit plane is loaded once into a B buffer, then each A plane p once
// into an A stage, and the products of p with every q <= s - 1 - p are issued from them.
template <int KIND>
__global__ void __launch_bounds__(192, 1)
    split_smallk_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                        SmallKArgs args) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  const uint32_t abase = base, bbase = base + kSkAStages * kSkAStage;
  const uint32_t bar0 = bbase + kSkBBufs * kSkBBuf;
  auto afull = [&](int s) { return bar0 + 8u * s; };
  auto aempty = [&](int s) { return bar0 + 8u * (kSkAStages + s); };
  auto bfull = [&](int s) { return bar0 + 8u * (2 * kSkAStages + s); };
  auto bempty = [&](int s) { return bar0 + 8u * (2 * kSkAStages + kSkBBufs + s); };
  constexpr int kBars = 2 * kSkAStages + 2 * kSkBBufs;
  const uint32_t accfull = bar0 + 8u * kBars;
  const uint32_t accempty = bar0 + 8u * (kBars + 1);
  const uint32_t done = bar0 + 8u * (kBars + 2);
  uint8_t* gen = smem_raw + (base - raw);
  uint32_t* tmem_holder =
      reinterpret_cast<uint32_t*>(gen + kSkAStages * kSkAStage + kSkBBufs * kSkBBuf + 8 * (kBars + 3));
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int BKE = KIND == kSplitBF16 ? 64 : 128;
  const int S = args.s;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kSkAStages; ++s) {
      mbar_init(afull(s), 1);
      mbar_init(aempty(s), 1);
    }
    for (int s = 0; s < kSkBBufs; ++s) {
      mbar_init(bfull(s), 1);
      mbar_init(bempty(s), 1);
    }
    mbar_init(accfull, 1);
    mbar_init(accempty, 128);
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;
  const long long budget = args.wait_cycles;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int ja = 0, jb = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < args.tiles && ok; tile += gridDim.x) {
        int64_t m0, n0;
        sk_tile_origin(args, tile, m0, n0);
        const int64_t ya = args.a_row0 + m0, yb = args.b_row0 + n0;
        for (int kb = 0; kb < args.kblocks && ok; ++kb, ++jb) {
          const int x = kb * BKE;
          {
            const int bs = jb % kSkBBufs;
            if (!mbar_wait(bempty(bs), ((uint32_t)(jb / kSkBBufs) & 1u) ^ 1u, budget, abort_flag)) {
              ok = false;
              break;
            }
            const uint32_t dst = bbase + bs * kSkBBuf;
            mbar_expect_tx(bfull(bs), (uint32_t)S * 2u * kSkTileB);
            for (int q = 0; q < S; ++q)
              for (int r = 0; r < 2; ++r)
                tma_load_3d(dst + (uint32_t)(q * 2 + r) * kSkTileB, &tmB, x, (int)yb, q * 2 + r, bfull(bs));
          }
          for (int pi = 0; pi < S; ++pi, ++ja) {
            const int p = plane_at(pi, S);
            const int as = ja % kSkAStages;
            if (!mbar_wait(aempty(as), ((uint32_t)(ja / kSkAStages) & 1u) ^ 1u, budget, abort_flag)) {
              ok = false;
              break;
            }
            const uint32_t dst = abase + as * kSkAStage;
            mbar_expect_tx(afull(as), kSkAStage);
            tma_load_3d(dst, &tmA, x, (int)ya, p * 2 + 0, afull(as));
            tma_load_3d(dst + kSkTileA, &tmA, x, (int)ya, p * 2 + 1, afull(as));
          }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(args.err, 1);
      }
      // drain: every copy issued has landed before the CTA exits
      for (int j = (ja > kSkAStages ? ja - kSkAStages : 0); j < ja; ++j)
        mbar_wait(afull(j % kSkAStages), (uint32_t)(j / kSkAStages) & 1u, budget, abort_flag, true);
      for (int j = (jb > kSkBBufs ? jb - kSkBBufs : 0); j < jb; ++j)
        mbar_wait(bfull(j % kSkBBufs), (uint32_t)(j / kSkBBufs) & 1u, budget, abort_flag, true);
    }
  } else if (warp == 1) {
    // ---------------- UMMA issuer: pair (p, q) into level p + q's accumulator ----------------
    if (lane == 0) {
      const uint32_t id = make_idesc_n32(KIND, 0), idn = make_idesc_n32(KIND, 1);
      const uint32_t idRI = (args.conjA ^ args.conjB) ? id : idn, idIm1 = args.conjB ? idn : id,
                     idIm2 = args.conjA ? idn : id;
      int ja = 0, jb = 0, t = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < args.tiles && ok; tile += gridDim.x, ++t) {
        if (!mbar_wait(accempty, ((uint32_t)t & 1u) ^ 1u, budget, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        uint32_t started = 0;  // levels whose accumulator holds this tile's partial sums
        for (int kb = 0; kb < args.kblocks && ok; ++kb, ++jb) {
          const int bs = jb % kSkBBufs;
          if (!mbar_wait(bfull(bs), (uint32_t)(jb / kSkBBufs) & 1u, budget, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sb = bbase + bs * kSkBBuf;
          for (int pi = 0; pi < S && ok; ++pi, ++ja) {
            const int p = plane_at(pi, S);
            const int as = ja % kSkAStages;
            if (!mbar_wait(afull(as), (uint32_t)(ja / kSkAStages) & 1u, budget, abort_flag)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sa = abase + as * kSkAStage;
            const uint64_t aR0 = sw128_desc(sa), aI0 = sw128_desc(sa + kSkTileA);
            for (int q = 0; q < S - p; ++q) {
              const int L = p + q;
              const uint32_t dre = tmem + (uint32_t)L * 64u, dim = dre + 32u;
              const uint32_t sbr = sb + (uint32_t)(q * 2) * kSkTileB;
              const uint64_t bR0 = sw128_desc(sbr), bI0 = sw128_desc(sbr + kSkTileB);
              const bool first = !(started & (1u << L));
#pragma unroll
              for (int kk = 0; kk < 4; ++kk) {
                const uint32_t acc = (first && kk == 0) ? 0u : 1u;
                const uint64_t o = 2u * (uint64_t)kk;  // 32 bytes of K, in the 16-byte address units
                umma<KIND>(dre, aR0 + o, bR0 + o, id, acc);
                umma<KIND>(dre, aI0 + o, bI0 + o, idRI, 1u);
                umma<KIND>(dim, aR0 + o, bI0 + o, idIm1, acc);
                umma<KIND>(dim, aI0 + o, bR0 + o, idIm2, 1u);
              }
              started |= 1u << L;
            }
            umma_commit(aempty(as));
          }
          if (ok) umma_commit(bempty(bs));
        }
        if (ok) umma_commit(accfull);
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(args.err, 2);
      }
      umma_commit(done);  // all issued MMAs complete before TMEM is released
      mbar_wait(done, 0u, budget, abort_flag, true);
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: warps 2..5, one row of the tile per thread ----------------
    const int q4 = warp & 3;
    int t = 0;
    for (int tile = blockIdx.x; tile < args.tiles; tile += gridDim.x, ++t) {
      if (!mbar_wait(accfull, (uint32_t)t & 1u, budget, abort_flag)) {
        *abort_flag = 1;
        atomicOr(args.err, 4);
        break;
      }
      tc_fence_after();
      int64_t m0, n0;
      sk_tile_origin(args, tile, m0, n0);
      const int64_t m = m0 + q4 * 32 + lane;
      // Every level's sum is an integer below 2^24 in magnitude (exact in FP32); the levels are
      // combined exactly in 64-bit integers, sum_L acc_L 2^(b (lmax - L)) < 2^62, on the integer
      // pipes, and converted to FP64 once (the FP64 pipe of this chip is the scarce one).
      long long ar[kSkBN], ai[kSkBN];
#pragma unroll
      for (int j = 0; j < kSkBN; ++j) ar[j] = ai[j] = 0;
      const uint32_t trow = tmem + ((uint32_t)(q4 * 32) << 16);
      for (int L = 0; L <= args.lmax; ++L) {
        uint32_t re[32], im[32];
        tmem_ld32(trow + (uint32_t)L * 64u, re);
        tmem_ld32(trow + (uint32_t)L * 64u + 32u, im);
        tmem_wait_ld();
        const long long w = 1LL << (args.b * (args.lmax - L));
#pragma unroll
        for (int j = 0; j < kSkBN; ++j) {
          ar[j] += (long long)__float2int_rn(__uint_as_float(re[j])) * w;
          ai[j] += (long long)__float2int_rn(__uint_as_float(im[j])) * w;
        }
      }
      tc_fence_before();
      mbar_arrive(accempty);  // tensor memory is free for the next tile
      if (m < args.M) {
        // With alpha = +-1 (the common case) the scales, all powers of two, are applied by
        // exponent arithmetic and the sign by negating the integers: the FP64 pipe only converts
        // the two integers (and adds C when beta = 1). Otherwise: FP64 products.
        const bool unit_alpha = args.alpha.y == 0.0 && (args.alpha.x == 1.0 || args.alpha.x == -1.0);
        const bool read_c = args.beta.x != 0.0 || args.beta.y != 0.0;
        const bool beta_one = args.beta.x == 1.0 && args.beta.y == 0.0;
        const int krow = pow2_exponent(args.rs[m]) - args.b * (args.lmax + 2);
        const double rsc = args.rs[m] * ldexp(1.0, -args.b * (args.lmax + 2));
        const bool neg = unit_alpha && args.alpha.x < 0.0;
#pragma unroll
        for (int j = 0; j < kSkBN; ++j) {
          const int64_t n = n0 + j;
          if (n >= args.N) break;
          z val;
          if (unit_alpha) {
            const int k = krow + pow2_exponent(args.cs[n]);
            val = make_double2(scale_pow2((double)(neg ? -ar[j] : ar[j]), k),
                               scale_pow2((double)(neg ? -ai[j] : ai[j]), k));
          } else {
            const double f = rsc * args.cs[n];
            val = zmul(args.alpha, make_double2((double)ar[j] * f, (double)ai[j] * f));
          }
          z* cp = args.transC ? args.C + n * args.ldc + m : args.C + m * args.ldc + n;
          if (read_c) val = zadd(val, beta_one ? *cp : zmul(args.beta, *cp));
          *cp = val;
        }
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// ---- digit slicing ----------------------------------------------------------


template <int KIND>
__device__ __forceinline__ void put_digit(uint8_t* out, int64_t idx, double d) {
  if constexpr (KIND == kSplitBF16) {
    reinterpret_cast<__nv_bfloat16*>(out)[idx] = __float2bfloat16_rn((float)d);
  } else {
    out[idx] = __nv_fp8_e4m3((float)d).__x;
  }
}

// Digits by integer arithmetic only (the FP64 pipe of this chip is narrow): each element x of a
// row scaled by 2^-e (|x 2^-e| < 1) becomes the 62-bit fixed-point integer V = x 2^(62 - e),
// rounded to nearest (ties to even) from the bits of x; its digits are b-bit fields of |V|
// plus a constant (digit_offset below).
__device__ __forceinline__ long long fixed62_scaled(double x, int e) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((bits >> 52) & 0x7FF);
  unsigned long long m = bits & 0xFFFFFFFFFFFFFull;
  if (E == 0 && m == 0) return 0;
  if (E != 0) m |= 1ull << 52;
  const int s = (E != 0 ? E - 1075 : -1074) + 62 - e;  // |x| 2^(62 - e) = m 2^s
  long long v;
  if (s >= 0) {
    v = s <= 10 ? (long long)(m << s) : 0x7FFFFFFFFFFFFFFFll;  // |x 2^-e| < 1 keeps s <= 9
  } else if (s < -54) {
    v = 0;  // below half a unit
  } else {
    // round to nearest, ties to even: add half a unit less one, plus the kept part's low bit
    const int r = -s;
    v = (long long)((m + (1ull << (r - 1)) - 1ull + ((m >> r) & 1ull)) >> r);
  }
  return (bits >> 63) ? -v : v;
}

// |x| as the bit pattern of a non-negative double: their integer order is the order of |x|.
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
// e with |x| = f 2^e, f in [0.5, 1), for x > 0 given by abs_bits
__device__ __forceinline__ int exponent_of(unsigned long long ab) {
  const int E = (int)(ab >> 52);
  if (E != 0) return E - 1022;
  int e = 0;
  frexp(__longlong_as_double((long long)ab), &e);  // subnormal
  return e;
}
// Balanced digits of |V| from b-bit fields: W = |V| + offset, with offset holding half a digit
// (2^(b-1)) at every digit position and half a unit at the last (rounding to nearest, ties away
// from zero); digit p is field p of W minus 2^(b-1), the first field unmasked. Every digit is in
// [-2^(b-1), 2^(b-1)] (the first up to 2^b without headroom), the remainder at most half a unit
// of the last digit, and the sign of V is applied to every digit, so that the digits of -x are
// exactly the negated digits of x (products of antisymmetric tensors stay antisymmetric).
__host__ __device__ inline unsigned long long digit_offset(int s, int b) {
  unsigned long long off = 0;
  for (int p = 0; p < s; ++p) off += (1ull << (b - 1)) << (62 - b * (p + 1));
  return off + (1ull << (62 - b * s - 1));
}
__device__ __forceinline__ int field_digit(unsigned long long W, int p, int shift, int b, bool neg) {
  const unsigned long long f = p == 0 ? (W >> shift) : ((W >> shift) & ((1ull << b) - 1ull));
  const int d = (int)f - (1 << (b - 1));
  return neg ? -d : d;
}

__device__ __forceinline__ uint32_t pack4_e4m3(int d0, int d1, int d2, int d3) {
  const __nv_fp8x2_storage_t lo = __nv_cvt_float2_to_fp8x2(make_float2((float)d0, (float)d1), __NV_SATFINITE, __NV_E4M3);
  const __nv_fp8x2_storage_t hi = __nv_cvt_float2_to_fp8x2(make_float2((float)d2, (float)d3), __NV_SATFINITE, __NV_E4M3);
  return (uint32_t)lo | ((uint32_t)hi << 16);
}
__device__ __forceinline__ uint2 pack4_bf16(int d0, int d1, int d2, int d3) {
  __nv_bfloat162 a = __floats2bfloat162_rn((float)d0, (float)d1);
  __nv_bfloat162 c = __floats2bfloat162_rn((float)d2, (float)d3);
  uint2 w;
  w.x = *reinterpret_cast<uint32_t*>(&a);
  w.y = *reinterpret_cast<uint32_t*>(&c);
  return w;
}

// The default digits (8 of 5 bits, e4m3) of four consecutive values of one part, with constant
// shifts: every 5-bit field of W lies within one of its 32-bit halves (bits 57.. of the first
// digit, then 52, 47, 42, 37, 32 in the high word and 27, 22 in the low one). A field f becomes
// the float f - 16 by adding it to the bits of 1.5 * 2^23 (exact for these small integers),
// two floats become two e4m3 bytes in one conversion, and the sign of each value is applied to
// its four bytes at once (e4m3 is sign-magnitude: the digits of -x are the negated digits of x;
// a zero digit of a negative value is -0). Plane p is written at out + o + p * plane (bytes).
__device__ __forceinline__ void cut4_e4m3_8x5(const unsigned long long (&W)[4], const bool (&neg)[4],
                                              uint8_t* __restrict__ out, int64_t o, int64_t plane) {
  const uint32_t sgn = (neg[0] ? 0x80u : 0u) | (neg[1] ? 0x8000u : 0u) | (neg[2] ? 0x800000u : 0u) |
                       (neg[3] ? 0x80000000u : 0u);
  uint32_t hi[4], lo[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    hi[u] = (uint32_t)(W[u] >> 32);
    lo[u] = (uint32_t)W[u];
  }
  constexpr int kBias = 0x4B400000 - 16;  // float bits of 1.5 * 2^23, less half a digit
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    float f[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      uint32_t fld;
      if (p == 0) fld = hi[u] >> 25;
      else if (p < 6) fld = (hi[u] >> (25 - 5 * p)) & 31u;
      else fld = (lo[u] >> (57 - 5 * p)) & 31u;
      f[u] = __int_as_float(kBias + (int)fld) - 12582912.0f;
    }
    const __nv_fp8x2_storage_t a = __nv_cvt_float2_to_fp8x2(make_float2(f[0], f[1]), __NV_SATFINITE, __NV_E4M3);
    const __nv_fp8x2_storage_t c = __nv_cvt_float2_to_fp8x2(make_float2(f[2], f[3]), __NV_SATFINITE, __NV_E4M3);
    *reinterpret_cast<uint32_t*>(out + o + p * plane) = ((uint32_t)a | ((uint32_t)c << 16)) ^ sgn;
  }
}

// Rows with K contiguous, in two passes over (row, K chunk) work items, one warp each, so
// that both many short rows and few long rows keep the GPU busy: pass 1 takes each
// chunk's largest |re|, |im| and folds its exponent into the row's with an integer
// atomicMax (deterministic); after the scales are set, pass 2 cuts 4 consecutive k per
// lane, so loads are coalesced and every digit plane is stored 128 bytes per warp.
__global__ void rowexp_n_kernel(const z* __restrict__ X, int64_t rows, int64_t K, int64_t ld, int64_t chunk,
                                int64_t nchunks, int* __restrict__ ex) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = warp; w < rows * nchunks; w += nwarps) {
    const int64_t r = w / nchunks, c = w % nchunks;
    const int64_t k1 = min(K, (c + 1) * chunk);
    const z* row = X + r * ld;
    unsigned long long mx = 0;
    for (int64_t k = c * chunk + lane; k < k1; k += 32) {
      const z v = row[k];
      mx = max(mx, max(abs_bits(v.x), abs_bits(v.y)));
    }
    for (int off = 16; off > 0; off >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if (lane == 0 && mx > 0) atomicMax(ex + r, exponent_of(mx));
  }
}

template <int KIND>
__global__ void __launch_bounds__(256, 4) slice_kernel(const z* __restrict__ X, int64_t rows, int64_t K, int64_t ld, int conj, int s, int b,
                             uint8_t* __restrict__ out, int64_t rows_pad, int64_t Kp, int64_t chunk, int64_t nchunks,
                             const int* __restrict__ ex, unsigned long long doff) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = warp; w < rows_pad * nchunks; w += nwarps) {
    const int64_t r = w / nchunks, c = w % nchunks;
    const bool live = r < rows;
    const z* row = X + r * ld;
    const int er = live ? ex[r] : 0;
    const int64_t k1 = min(Kp, (c + 1) * chunk);
    for (int64_t k0 = c * chunk + 4 * (int64_t)lane; k0 < k1; k0 += 128) {
      unsigned long long Wr[4], Wi[4];
      bool nr[4], ni[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t k = k0 + u;
        long long vr = 0, vi = 0;
        if (live && k < K) {
          const z v = row[k];
          vr = fixed62_scaled(v.x, er);
          vi = fixed62_scaled(v.y, er);
          if (conj) vi = -vi;
        }
        nr[u] = vr < 0;
        ni[u] = vi < 0;
        Wr[u] = (unsigned long long)(nr[u] ? -vr : vr) + doff;
        Wi[u] = (unsigned long long)(ni[u] ? -vi : vi) + doff;
      }
      if (KIND == kSplitE4M3 && s == 8 && b == 5) {
        const int64_t plane = 2 * rows_pad * Kp;  // from digit p of a part to digit p + 1
        cut4_e4m3_8x5(Wr, nr, out, r * Kp + k0, plane);
        cut4_e4m3_8x5(Wi, ni, out, (rows_pad + r) * Kp + k0, plane);
        continue;
      }
      int shift = 62;
      for (int p = 0; p < s; ++p) {
        shift -= b;
        int dr[4], di[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          dr[u] = field_digit(Wr[u], p, shift, b, nr[u]);
          di[u] = field_digit(Wi[u], p, shift, b, ni[u]);
        }
        const int64_t o0 = ((int64_t)(p * 2 + 0) * rows_pad + r) * Kp + k0;
        const int64_t o1 = ((int64_t)(p * 2 + 1) * rows_pad + r) * Kp + k0;
        if constexpr (KIND == kSplitBF16) {
          *reinterpret_cast<uint2*>(out + 2 * o0) = pack4_bf16(dr[0], dr[1], dr[2], dr[3]);
          *reinterpret_cast<uint2*>(out + 2 * o1) = pack4_bf16(di[0], di[1], di[2], di[3]);
        } else {
          *reinterpret_cast<uint32_t*>(out + o0) = pack4_e4m3(dr[0], dr[1], dr[2], dr[3]);
          *reinterpret_cast<uint32_t*>(out + o1) = pack4_e4m3(di[0], di[1], di[2], di[3]);
        }
      }
    }
  }
}

// Operands whose rows are strided (element (r, k) at X[k*ld + r]): pass 1 finds each row's
// power-of-two scale with one thread per row (reads coalesced across rows); pass 2 moves
// 32-row x 64-k tiles through shared memory so both the reads (along r) and the digit
// stores (along k) are coalesced.
// Exponent of each row's largest |re|, |im| as an integer max (deterministic): 32 rows x 8
// K-strides per block, the K range split across blockIdx.y. ex[] starts at INT_MIN.
__global__ void rowexp_t_kernel(const z* __restrict__ X, int64_t rows, int64_t K, int64_t ld, int* __restrict__ ex) {
  __shared__ unsigned long long sh[8][33];
  const int64_t r = (int64_t)blockIdx.x * 32 + threadIdx.x;
  unsigned long long mx = 0;
  if (r < rows)
    for (int64_t k = (int64_t)blockIdx.y * 8 + threadIdx.y; k < K; k += (int64_t)gridDim.y * 8) {
      const z v = X[k * ld + r];
      mx = max(mx, max(abs_bits(v.x), abs_bits(v.y)));
    }
  sh[threadIdx.y][threadIdx.x] = mx;
  __syncthreads();
  if (threadIdx.y == 0 && r < rows) {
    for (int y = 1; y < 8; ++y) mx = max(mx, sh[y][threadIdx.x]);
    if (mx > 0) atomicMax(ex + r, exponent_of(mx));
  }
}

__global__ void rowexp_finalize_kernel(int* __restrict__ ex, int64_t rows, double* __restrict__ scale,
                                       double* __restrict__ inv, int headroom) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
    // untouched (all-zero row): memset pattern 0x80808080
    const int e = (ex[r] < -2000 ? 0 : ex[r]) + headroom;
    scale[r] = ldexp(1.0, e);
    inv[r] = ldexp(1.0, -e);
    ex[r] = e;  // the digit passes scale by 2^-e with integer operations
  }
}

template <int KIND>
__global__ void __launch_bounds__(256, 4) slice_t_kernel(const z* __restrict__ X, int64_t rows, int64_t K, int64_t ld, int conj, int s, int b,
                               uint8_t* __restrict__ out, int64_t rows_pad, int64_t Kp, const int* __restrict__ ex,
                               unsigned long long doff) {
  __shared__ z tile[64][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32, k0 = (int64_t)blockIdx.y * 64;
  for (int idx = threadIdx.x; idx < 64 * 32; idx += blockDim.x) {
    const int kk = idx / 32, rr = idx % 32;
    const int64_t r = r0 + rr, k = k0 + kk;
    tile[kk][rr] = (r < rows && k < K) ? X[k * ld + r] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  for (int item = threadIdx.x; item < 32 * 16; item += blockDim.x) {
    const int rr = item / 16, kg = item % 16;
    const int64_t r = r0 + rr, k = k0 + 4 * kg;
    const int er = r < rows ? ex[r] : 0;
    unsigned long long Wr[4], Wi[4];
    bool nr[4], ni[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const z v = tile[4 * kg + u][rr];
      long long vr = fixed62_scaled(v.x, er), vi = fixed62_scaled(v.y, er);
      if (conj) vi = -vi;
      nr[u] = vr < 0;
      ni[u] = vi < 0;
      Wr[u] = (unsigned long long)(nr[u] ? -vr : vr) + doff;
      Wi[u] = (unsigned long long)(ni[u] ? -vi : vi) + doff;
    }
    if (KIND == kSplitE4M3 && s == 8 && b == 5) {
      const int64_t plane = 2 * rows_pad * Kp;
      cut4_e4m3_8x5(Wr, nr, out, r * Kp + k, plane);
      cut4_e4m3_8x5(Wi, ni, out, (rows_pad + r) * Kp + k, plane);
      continue;
    }
    int shift = 62;
    for (int p = 0; p < s; ++p) {
      shift -= b;
      int dr[4], di[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        dr[u] = field_digit(Wr[u], p, shift, b, nr[u]);
        di[u] = field_digit(Wi[u], p, shift, b, ni[u]);
      }
      const int64_t o0 = ((int64_t)(p * 2 + 0) * rows_pad + r) * Kp + k;
      const int64_t o1 = ((int64_t)(p * 2 + 1) * rows_pad + r) * Kp + k;
      if constexpr (KIND == kSplitBF16) {
        *reinterpret_cast<uint2*>(out + 2 * o0) = pack4_bf16(dr[0], dr[1], dr[2], dr[3]);
        *reinterpret_cast<uint2*>(out + 2 * o1) = pack4_bf16(di[0], di[1], di[2], di[3]);
      } else {
        *reinterpret_cast<uint32_t*>(out + o0) = pack4_e4m3(dr[0], dr[1], dr[2], dr[3]);
        *reinterpret_cast<uint32_t*>(out + o1) = pack4_e4m3(di[0], di[1], di[2], di[3]);
      }
    }
  }
}

// Integer-valued doubles to digits (probe input), real part only, slice 0.
template <int KIND>
__global__ void raw_digits_kernel(const double* __restrict__ X, int64_t rows, int64_t K, uint8_t* __restrict__ out,
                                  int64_t rows_pad, int64_t Kp) {
  const int64_t total = rows_pad * Kp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / Kp, k = e % Kp;
    put_digit<KIND>(out, e, (r < rows && k < K) ? X[r * K + k] : 0.0);
  }
}

// ---- host helpers -----------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

int esize(int kind) { return kind == kSplitBF16 ? 2 : 1; }
int bke(int kind) { return kind == kSplitBF16 ? 64 : 128; }
int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
// Rows of each digit plane are padded to whole 32-row blocks of the transposing slicer (tiles
// past them are zero filled by the tensor map).
constexpr int64_t kRowPad = 32;

// 3-D map over the digit array: K (128-byte segments of the box), rows, planes. A box of
// box_rows rows that runs past the rows of a plane is zero filled without reading memory, so a
// short operand (e.g. 20 occupied rows under a 128-row tile) costs only its own rows.
cudaError_t encode_map_rows(const SliceSet& S, uint32_t box_rows, CUtensorMap* out) {
  auto enc = get_encode();
  if (!enc) return cudaErrorNotSupported;
  const int es = esize(S.kind);
  cuuint64_t dims[3] = {(cuuint64_t)S.Kp, (cuuint64_t)S.rows_pad, (cuuint64_t)(S.s * 2)};
  cuuint64_t strides[2] = {(cuuint64_t)(S.Kp * es), (cuuint64_t)(S.rows_pad * S.Kp * es)};
  cuuint32_t box[3] = {(cuuint32_t)(128 / es), box_rows, 1u};
  cuuint32_t estr[3] = {1u, 1u, 1u};
  CUresult r = enc(out, S.kind == kSplitBF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 3,
                   S.digits, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// The set's own map, box {128 bytes, 128 rows, 1 plane}.
cudaError_t encode_map(SliceSet& S) {
  S.have_map = encode_map_rows(S, 128u, &S.tmap) == cudaSuccess;
  return S.have_map ? cudaSuccess : cudaErrorInvalidValue;
}

int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      n = 148;
    }
  }
  return n;
}

double maxdigit(int p, int b, int headroom) { return p == 0 && !headroom ? std::ldexp(1.0, b) : std::ldexp(1.0, b - 1); }

// K blocks per exact chunk of each level: the pairs (p, L - p) of level L share one
// FP32 accumulator, so a chunk may add at most (2^24 - 1) / (products_per_k * sum |d_p d_q|)
// values of k before every partial sum could exceed 2^24.
bool fill_levels(SplitArgs& a, int s, int b, int kblocks, int kind) {
  if (s < 1 || s > kMaxLevels) return false;
  a.s = s;
  a.b = b;
  a.lmax = s - 1;
  a.kblocks = kblocks;
  const int hb = split_headroom(kind, b);
  for (int L = 0; L <= a.lmax; ++L) {
    double sum = 0.0;
    for (int p = std::max(0, L - s + 1); p <= std::min(L, s - 1); ++p)
      sum += maxdigit(p, b, hb) * maxdigit(L - p, b, hb);
    const double klen = std::floor((16777216.0 - 1.0) / (2.0 * sum));  // complex: 2 products per k
    const int kb = (int)std::floor(klen / bke(kind));
    if (kb < 1) return false;
    a.kbper[L] = kb;
  }
  return true;
}

// The short-K kernel takes a launch when every level fits its tensor memory (at most 8
// levels) and one accumulator per level stays exact over the whole K, and K is short
// enough (a few blocks) that the main kernel would be bound by its per-level flushes.
constexpr int kSmallKMaxBlocks = 4;
bool smallk_eligible(const SplitArgs& a) {
  if (a.lmax + 1 > 8 || a.kblocks > kSmallKMaxBlocks) return false;
  for (int L = 0; L <= a.lmax; ++L)
    if (a.kbper[L] < a.kblocks) return false;
  return true;
}

// K split across CTAs when the output has too few tiles to fill the GPU, or a few waves of
// tiles that leave the last wave partly idle. With fewer tiles than SMs the split starts at
// about two CTAs per SM (a 20 x 20 output with a long K runs on every SM, not on a few);
// from there, or from no split with one to four waves of tiles, the factor that best fills
// whole waves (CTAs / (waves x SMs)) is taken where it beats the smaller factors by more
// than 5%. Each split keeps >= kMinKbPerSplit K blocks (half that for outputs of fewer than 16
// tiles, whose long K is the whole of their work: the skinny products over o^2 v or o v^2)
// so that a level group's MMA work stays above its FP64 flush in the epilogue.
#ifndef SPLIT_MIN_KB_PER_SPLIT
#define SPLIT_MIN_KB_PER_SPLIT 12
#endif
constexpr int kMinKbPerSplit = SPLIT_MIN_KB_PER_SPLIT;
void plan_ksplit(int64_t tiles, int kblocks, int& ksplits, int& kb_split, int64_t slots) {
  ksplits = 1;
  const int64_t sms = slots;
  const int kb_min = tiles < 16 ? std::max(1, kMinKbPerSplit / 2) : kMinKbPerSplit;
  const int64_t kmax = std::max(1, kblocks / kb_min);
  auto fill = [&](int64_t ctas) { return (double)ctas / (double)(((ctas + sms - 1) / sms) * sms); };
  if (tiles > 0 && tiles < 4 * sms) {
    const int64_t lo = tiles < sms ? std::min<int64_t>((2 * sms + tiles - 1) / tiles, kmax) : 1;
    const int64_t hi = std::min<int64_t>(kmax, std::max<int64_t>(2 * lo, 32));
    ksplits = (int)lo;
    double best = fill(tiles * lo);
    for (int64_t ks = lo + 1; ks <= hi; ++ks) {
      const double f = fill(tiles * ks);
      if (f > best + 0.05) {
        best = f;
        ksplits = (int)ks;
      }
    }
  }
  kb_split = (kblocks + ksplits - 1) / ksplits;
  ksplits = (kblocks + kb_split - 1) / kb_split;
}

// Orientation and tile width of the main kernel for C (M x N): the operand whose rows go to
// the 128-row side, and BN. The least padded tile area wins, each width weighted by an
// efficiency factor. Alone, a narrower tile runs slower (a 4096 x 4096 x 8192 product: 96-wide
// tiles at 0.77 and 64-wide at 0.61 of the 128-wide rate), but on a short operand it also
// halves the reads of the long one: the o20/v120 ladder (190 x 7140 x 7140) is fastest on
// swapped 96-wide tiles, 0.70 of the time of 128-wide ones; the factors keep that choice;
// a change from 128-wide tiles without swap must gain more than 3%. A short M (few pair
// rows, e.g. the occupied pairs of the ladder) then swaps to the BN side.
struct MainTiling {
  bool swap = false;
  int bn = 128;
  int64_t tiles_m = 0, tiles = 0;
  double area = 0.0;  // padded tile area over the tensor-pipe efficiency
};
MainTiling choose_tiling(int64_t M, int64_t N) {
  static const int widths[3] = {128, 96, 64};
  static const double eff[3] = {1.0, 0.97, 0.85};
  MainTiling t;
  t.area = (double)round_up(M, 128) * (double)round_up(N, 128);
  for (int sw = 0; sw < 2; ++sw)
    for (int w = 0; w < 3; ++w) {
      const int64_t rows = sw ? N : M, cols = sw ? M : N;
      const double area = (double)round_up(rows, 128) * (double)round_up(cols, widths[w]) / eff[w];
      if (area < t.area * 0.97) {
        t.area = area;
        t.swap = sw != 0;
        t.bn = widths[w];
      }
    }
  const int64_t rows = t.swap ? N : M, cols = t.swap ? M : N;
  t.tiles_m = (rows + 127) / 128;
  t.tiles = t.tiles_m * ((cols + t.bn - 1) / t.bn);
  return t;
}

// C = alpha * sum_ks part[ks] + beta * C, summed in split order.
__global__ void part_reduce_kernel(const z* __restrict__ part, int ks, int64_t M, int64_t N, z* __restrict__ C,
                                   int64_t ldc, z alpha, z beta) {
  const int64_t MN = M * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < MN; e += (int64_t)gridDim.x * blockDim.x) {
    double ar = 0.0, ai = 0.0;
    for (int k = 0; k < ks; ++k) {
      const z w = part[k * MN + e];
      ar += w.x;
      ai += w.y;
    }
    z* cp = C + (e / N) * ldc + (e % N);
    z out = zmul(alpha, make_double2(ar, ai));
    if (beta.x != 0.0 || beta.y != 0.0) out = zadd(out, zmul(beta, *cp));
    *cp = out;
  }
}

template <int KIND, bool PROBE, int BN, int CL>
cudaError_t launch_split(const CUtensorMap& mapA, const CUtensorMap& mapB, const SplitArgs& a, cudaStream_t s) {
  auto kern = split_kernel<KIND, PROBE, BN, CL>;
  constexpr uint32_t smem = MainTile<BN>::kSmemBytes;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [&]() {
    attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (attr_err != cudaSuccess) return attr_err;
  const int64_t grid = (int64_t)a.tiles * a.ksplits;
  if (grid <= 0) return cudaSuccess;
  if (grid > 0x7fffffff || grid % CL != 0) return cudaErrorInvalidValue;
  if constexpr (CL == 1) {
    kern<<<(unsigned)grid, 192, smem, s>>>(mapA, mapB, a);
  } else {
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3(192, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, mapA, mapB, a);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

// CTAs of the main kernel resident at once: one per SM, or, in clusters of two, twice the
// clusters the GPU can hold (a GPC with an odd number of free SMs leaves one idle).
template <int KIND, int BN>
int64_t main_slots(int cl) {
  if (cl == 1) return num_sms();
  static int64_t slots = 0;
  static std::once_flag once;
  std::call_once(once, [&]() {
    auto kern = split_kernel<KIND, false, BN, 2>;
    constexpr uint32_t smem = MainTile<BN>::kSmemBytes;
    int n = 0;
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(2 * (unsigned)num_sms(), 1, 1);
    cfg.blockDim = dim3(192, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess &&
        cudaOccupancyMaxActiveClusters(&n, kern, &cfg) == cudaSuccess && n > 0)
      slots = 2 * (int64_t)n;
    else
      cudaGetLastError();
  });
  return slots;  // 0: clusters unavailable
}

template <int KIND>
int64_t main_slots_bn(int bn, int cl) {
  switch (bn) {
    case 96: return main_slots<KIND, 96>(cl);
    case 64: return main_slots<KIND, 64>(cl);
    default: return main_slots<KIND, 128>(cl);
  }
}

template <int KIND>
cudaError_t launch_main(const CUtensorMap& mapA, const CUtensorMap& mapB, const SplitArgs& a, int bn, int cl,
                        cudaStream_t s) {
  if (cl == 2) {
    switch (bn) {
      case 96: return launch_split<KIND, false, 96, 2>(mapA, mapB, a, s);
      case 64: return launch_split<KIND, false, 64, 2>(mapA, mapB, a, s);
      default: return launch_split<KIND, false, 128, 2>(mapA, mapB, a, s);
    }
  }
  switch (bn) {
    case 96: return launch_split<KIND, false, 96, 1>(mapA, mapB, a, s);
    case 64: return launch_split<KIND, false, 64, 1>(mapA, mapB, a, s);
    default: return launch_split<KIND, false, 128, 1>(mapA, mapB, a, s);
  }
}

template <int KIND>
cudaError_t launch_smallk(const CUtensorMap& mapA, const CUtensorMap& mapB, const SmallKArgs& a, cudaStream_t s) {
  auto kern = split_smallk_kernel<KIND>;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [&]() {
    attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSkSmemBytes);
  });
  if (attr_err != cudaSuccess) return attr_err;
  if (a.tiles <= 0) return cudaSuccess;
  const int grid = std::min(a.tiles, num_sms());
  kern<<<grid, 192, kSkSmemBytes, s>>>(mapA, mapB, a);
  return cudaGetLastError();
}

// C = alpha A B^T + beta C on the short-K kernel. B's rows (the caller's N, C's contiguous
// dimension) go to the 128-row side, the output transposed, so that the lanes of a warp store
// consecutive elements of a row of C; unless that pads much more than the other orientation
// (a short N on the 128-row side).
cudaError_t split_gemm_smallk(const SliceSet& A, const SliceSet& B, const SplitArgs& lv, z* C, int64_t ldc, z alpha,
                              z beta, int* err, long long wait_cycles, cudaStream_t s, int conjB) {
  const double area_keep = (double)round_up(A.rows, 128) * (double)round_up(B.rows, kSkBN);
  const double area_swap = (double)round_up(B.rows, 128) * (double)round_up(A.rows, kSkBN);
  const bool swap = area_swap <= 1.05 * area_keep;
  const SliceSet& KA = swap ? B : A;
  const SliceSet& KB = swap ? A : B;
  SmallKArgs k;
  std::memset(&k, 0, sizeof(k));
  k.conjA = swap ? conjB : 0;  // the caller's B is the kernel's A when swapped
  k.conjB = swap ? 0 : conjB;
  k.M = KA.rows;
  k.N = KB.rows;
  k.a_row0 = KA.row0;
  k.b_row0 = KB.row0;
  const int64_t tm = (k.M + 127) / 128, tn = (k.N + kSkBN - 1) / kSkBN;
  if (tm * tn > 0x7fffffff) return cudaErrorInvalidValue;
  k.tiles_m = (int)tm;
  k.tiles_n = (int)tn;
  k.nfast = tn <= tm ? 1 : 0;
  k.tiles = (int)(tm * tn);
  k.s = lv.s;
  k.b = lv.b;
  k.lmax = lv.lmax;
  k.kblocks = lv.kblocks;
  k.C = C;
  k.ldc = ldc;
  k.alpha = alpha;
  k.beta = beta;
  k.transC = swap ? 1 : 0;
  k.rs = KA.scale;
  k.cs = KB.scale;
  k.err = err;
  k.wait_cycles = wait_cycles > 0 ? wait_cycles : 4000000000LL;
  CUtensorMap mapB;
  cudaError_t e = encode_map_rows(KB, (uint32_t)kSkBN, &mapB);
  if (e != cudaSuccess) return e;
  return KA.kind == kSplitBF16 ? launch_smallk<kSplitBF16>(KA.tmap, mapB, k, s)
                               : launch_smallk<kSplitE4M3>(KA.tmap, mapB, k, s);
}

// Tiling, cluster and K split of a main-kernel launch. An output two N tiles wide (the ladder's
// occupied pairs on the narrow side, or a long operand against up to 256 rows) runs in clusters
// of two CTAs that share the 128-row operand's tile (read once per pair of N tiles); also with
// four N tiles, where each pair shares it.
#ifndef SPLIT_CLUSTER
#define SPLIT_CLUSTER 1
#endif
#ifndef SPLIT_STREAM_HINT
#define SPLIT_STREAM_HINT 1
#endif
#ifndef SPLIT_GROUP
#define SPLIT_GROUP 8
#endif
struct MainPlan {
  MainTiling tl;
  int cl = 1;
  int ksplits = 1, kb_split = 1;
};
MainPlan plan_main(int64_t M, int64_t N, int kblocks, int kind) {
  MainPlan P;
  P.tl = choose_tiling(M, N);
  int64_t slots = num_sms();
  const int64_t tiles_n = P.tl.tiles_m > 0 ? P.tl.tiles / P.tl.tiles_m : 0;
  if (SPLIT_CLUSTER && (tiles_n == 2 || tiles_n == 4)) {
    const int64_t sl = kind == kSplitBF16 ? main_slots_bn<kSplitBF16>(P.tl.bn, 2) : main_slots_bn<kSplitE4M3>(P.tl.bn, 2);
    if (sl > 0) {
      P.cl = 2;
      slots = sl;
    }
  }
  plan_ksplit(P.tl.tiles, kblocks, P.ksplits, P.kb_split, slots);
  return P;
}

}  // namespace

int64_t slice_bytes(int64_t rows, int64_t K, const SplitConfig& cfg) {
  const int64_t rows_pad = round_up(std::max<int64_t>(rows, 1), kRowPad);
  const int64_t Kp = round_up(std::max<int64_t>(K, 1), bke(cfg.kind));
  // digits, then per-row scale and inverse scale (doubles) and exponent (int)
  return round_up((int64_t)cfg.s * 2 * rows_pad * Kp * esize(cfg.kind), 1024) + 3 * round_up(rows_pad * 8, 1024);
}

cudaError_t make_slices(const z* X, int64_t rows, int64_t K, int64_t ld, int trans, int conj, const SplitConfig& cfg,
                        SliceSet& out, void* mem, cudaStream_t s) {
  if (cfg.s < 1 || cfg.s > 14 || cfg.b < 1 || cfg.b > split_max_bits(cfg.kind) || cfg.b * cfg.s > 56)
    return cudaErrorInvalidValue;
  out.rows = rows;
  out.rows_pad = round_up(std::max<int64_t>(rows, 1), kRowPad);
  out.K = K;
  out.Kp = round_up(std::max<int64_t>(K, 1), bke(cfg.kind));
  out.s = cfg.s;
  out.b = cfg.b;
  out.kind = cfg.kind;
  out.digits = mem;
  out.scale = reinterpret_cast<double*>(static_cast<uint8_t*>(mem) +
                                        round_up((int64_t)cfg.s * 2 * out.rows_pad * out.Kp * esize(cfg.kind), 1024));
  cudaError_t e = encode_map(out);
  if (e != cudaSuccess) return e;
  double* inv = out.scale + round_up(out.rows_pad * 8, 1024) / 8;
  int* ex = reinterpret_cast<int*>(inv + round_up(out.rows_pad * 8, 1024) / 8);
  e = cudaMemsetAsync(ex, 0x80, (size_t)rows * sizeof(int), s);  // 0x80808080 < every exponent
  if (e != cudaSuccess) return e;
  constexpr int64_t kWarps = 152 * 64;  // work items wanted in flight
  if (trans) {
    const int64_t rb = (rows + 31) / 32;
    const int64_t ky = std::max<int64_t>(1, std::min<int64_t>((K + 63) / 64, (152 * 64 + rb - 1) / rb));
    rowexp_t_kernel<<<dim3((unsigned)rb, (unsigned)std::min<int64_t>(ky, 65535)), dim3(32, 8), 0, s>>>(X, rows, K, ld, ex);
  } else {
    // K chunks of whole 128-element blocks, enough of them that rows x chunks covers the GPU
    int64_t nch = std::min<int64_t>((kWarps + rows - 1) / rows, (out.Kp + 127) / 128);
    nch = std::max<int64_t>(nch, 1);
    const int64_t chunk = round_up((out.Kp + nch - 1) / nch, 128);
    nch = (out.Kp + chunk - 1) / chunk;
    out.chunk = chunk;
    out.nchunks = nch;
    const int blocks = (int)std::min<int64_t>((rows * nch * 32 + 255) / 256, 152 * 64);
    rowexp_n_kernel<<<std::max(blocks, 1), 256, 0, s>>>(X, rows, K, ld, chunk, nch, ex);
  }
  rowexp_finalize_kernel<<<grid_for(rows, 256), 256, 0, s>>>(ex, rows, out.scale, inv, split_headroom(cfg.kind, cfg.b));
  if (trans) {
    const dim3 grid((unsigned)(out.rows_pad / 32), (unsigned)(out.Kp / 64));
    if (grid.y > 65535) return cudaErrorInvalidValue;
    if (cfg.kind == kSplitBF16)
      slice_t_kernel<kSplitBF16><<<grid, 256, 0, s>>>(X, rows, K, ld, conj, cfg.s, cfg.b, (uint8_t*)out.digits,
                                                      out.rows_pad, out.Kp, ex, digit_offset(cfg.s, cfg.b));
    else
      slice_t_kernel<kSplitE4M3><<<grid, 256, 0, s>>>(X, rows, K, ld, conj, cfg.s, cfg.b, (uint8_t*)out.digits,
                                                      out.rows_pad, out.Kp, ex, digit_offset(cfg.s, cfg.b));
    return cudaGetLastError();
  }
  const int blocks = (int)std::min<int64_t>((out.rows_pad * out.nchunks * 32 + 255) / 256, 152 * 64);
  if (cfg.kind == kSplitBF16)
    slice_kernel<kSplitBF16><<<blocks, 256, 0, s>>>(X, rows, K, ld, conj, cfg.s, cfg.b, (uint8_t*)out.digits,
                                                    out.rows_pad, out.Kp, out.chunk, out.nchunks, ex,
                                                    digit_offset(cfg.s, cfg.b));
  else
    slice_kernel<kSplitE4M3><<<blocks, 256, 0, s>>>(X, rows, K, ld, conj, cfg.s, cfg.b, (uint8_t*)out.digits,
                                                    out.rows_pad, out.Kp, out.chunk, out.nchunks, ex,
                                                    digit_offset(cfg.s, cfg.b));
  return cudaGetLastError();
}

double split_cost_estimate(int64_t M, int64_t N, int64_t K, const SplitConfig& cfg) {
  // Model of one split GEMM on this GPU: the tensor-core digit products at ~2.8 PFLOP/s
  // (e4m3; half for bf16), each level group's FP64 flush (~6 FP64 operations per complex
  // output element of every 128x128 tile, with its read and write of the output) at ~3.8e11
  // operations/s (fitted to short-K launches, where the flushes dominate), and slicing both operands
  // (read twice, digits written once) at ~5 TB/s. Padding to whole tiles and K blocks counted.
  const int bk = bke(cfg.kind);
  const MainTiling tl = choose_tiling(M, N);  // padded area (over the width's efficiency) of the main kernel
  const double Kp = (double)round_up(K, bk);
  const double pairs = 0.5 * cfg.s * (cfg.s + 1);
  const double mma = pairs * 8.0 * tl.area * Kp / (cfg.kind == kSplitBF16 ? 1.4e15 : 2.8e15);
  SplitArgs a;
  std::memset(&a, 0, sizeof(a));
  const int kblocks = (int)(Kp / bk);
  double groups = 0.0;
  if (!fill_levels(a, cfg.s, cfg.b, kblocks, cfg.kind)) return 1e30;
  for (int L = 0; L <= a.lmax; ++L) groups += std::ceil((double)kblocks / a.kbper[L]);
  const double slicing0 = ((double)(M + N) * K * 32.0 + (double)(M + N) * Kp * 2.0 * cfg.s * esize(cfg.kind)) / 5e12;
  if (smallk_eligible(a)) {
    // short K: 128 x 32 tiles with the long side as rows, products at ~40% of the tensor rate
    // (N = 32 instructions), every output written once
    const double lo = (double)std::min(M, N), hi = (double)std::max(M, N);
    const double sk_mma = pairs * 8.0 * (double)round_up((int64_t)hi, 128) * (double)round_up((int64_t)lo, 32) * Kp /
                          (0.4 * (cfg.kind == kSplitBF16 ? 1.4e15 : 2.8e15));
    const double store = (double)M * N * 32.0 / 5e12;
    return std::max(sk_mma, store) + slicing0;
  }
  const double flush = (double)tl.tiles * groups * 128.0 * tl.bn * 6.0 / 3.8e11;
  const double slicing = ((double)(M + N) * K * 32.0 + (double)(M + N) * Kp * 2.0 * cfg.s * esize(cfg.kind)) / 5e12;
  return std::max(mma, flush) + slicing;
}

int64_t split_part_bytes(int64_t M, int64_t N, int64_t K, const SplitConfig& cfg) {
  const int kblocks = (int)((std::max<int64_t>(K, 1) + bke(cfg.kind) - 1) / bke(cfg.kind));
  const MainPlan P = plan_main(M, N, kblocks, cfg.kind);
  return P.ksplits > 1 ? (int64_t)P.ksplits * M * N * (int64_t)sizeof(z) : 0;
}

void split_describe(int64_t M, int64_t N, int64_t K, const SplitConfig& cfg, int out[6]) {
  const int kblocks = (int)(round_up(std::max<int64_t>(K, 1), bke(cfg.kind)) / bke(cfg.kind));
  SplitArgs a;
  std::memset(&a, 0, sizeof(a));
  for (int i = 0; i < 6; ++i) out[i] = 0;
  if (!fill_levels(a, cfg.s, cfg.b, kblocks, cfg.kind)) return;
  if (smallk_eligible(a)) {
    out[0] = 1;
    return;
  }
  const MainPlan P = plan_main(M, N, kblocks, cfg.kind);
  out[1] = P.tl.swap ? 1 : 0;
  out[2] = P.tl.bn;
  out[3] = P.cl;
  out[4] = P.ksplits;
  out[5] = (int)P.tl.tiles;
}

cudaError_t split_gemm(const SliceSet& A, const SliceSet& B, z* C, int64_t ldc, z alpha, z beta, int* err,
                       void* part_ws, int64_t part_bytes, cudaStream_t s, long long wait_cycles, int stall_loads,
                       int conjB) {
  if (A.kind != B.kind || A.Kp != B.Kp || A.s != B.s || A.b != B.b || !A.have_map || !B.have_map)
    return cudaErrorInvalidValue;
  SplitArgs a;
  std::memset(&a, 0, sizeof(a));
  // the failure-path self-test keeps the plain orientation, 128-wide tiles and no cluster
  const int kblocks = (int)(A.Kp / bke(A.kind));
  MainPlan mp;
  if (!stall_loads) mp = plan_main(A.rows, B.rows, kblocks, A.kind);
  MainTiling& tl = mp.tl;
  if (stall_loads) {
    tl.tiles_m = (A.rows + 127) / 128;
    tl.tiles = tl.tiles_m * ((B.rows + 127) / 128);
  }
  const SliceSet& KA = tl.swap ? B : A;  // the kernel's 128-row operand
  const SliceSet& KB = tl.swap ? A : B;  // its BN-row operand
  if (tl.tiles > 0x7fffffff) return cudaErrorInvalidValue;
  a.M = KA.rows;
  a.N = KB.rows;
  a.a_row0 = KA.row0;
  a.b_row0 = KB.row0;
  a.tiles_m = (int)tl.tiles_m;
  a.tiles = (int)tl.tiles;
  a.transC = tl.swap ? 1 : 0;
  a.conjA = tl.swap ? conjB : 0;  // the caller's B is the kernel's A when swapped
  a.conjB = tl.swap ? 0 : conjB;
  a.C = C;
  a.ldc = ldc;
  a.alpha = alpha;
  a.rs = KA.scale;
  a.cs = KB.scale;
  a.err = err;
  a.wait_cycles = wait_cycles > 0 ? wait_cycles : 4000000000LL;  // default ~2 s at 2 GHz
  a.stall_loads = stall_loads;
  if (!fill_levels(a, A.s, A.b, kblocks, A.kind)) return cudaErrorInvalidValue;
  if (!stall_loads && smallk_eligible(a))
    return split_gemm_smallk(A, B, a, C, ldc, alpha, beta, err, wait_cycles, s, conjB);
  a.ksplits = mp.ksplits;
  a.kb_split = mp.kb_split;
  // one cluster covers every N tile: no other CTA reads this A tile, so under L2 pressure its
  // lines go before the partial sums and the narrow operand, which are read again
  a.a_stream = (SPLIT_STREAM_HINT && mp.cl == 2 && tl.tiles == 2 * tl.tiles_m) ? 1 : 0;
  // many tiles both ways (e.g. the (ov)^3 products): bands of SPLIT_GROUP M tiles
  {
    const int64_t tiles_n = tl.tiles_m > 0 ? tl.tiles / tl.tiles_m : 0;
    a.group = (mp.cl == 1 && SPLIT_GROUP > 1 && tl.tiles_m >= 2 * SPLIT_GROUP && tiles_n >= 2 * SPLIT_GROUP)
                  ? SPLIT_GROUP
                  : 1;
  }
  if (stall_loads) {
    a.ksplits = 1;
    a.kb_split = kblocks;
  }
  const int64_t part1 = a.M * a.N * (int64_t)sizeof(z);  // one split partial
  if (a.ksplits > 1 && (part_ws == nullptr || part_bytes < (int64_t)a.ksplits * part1)) {
    // a smaller workspace: as many partials as it holds (at least two), else no split
    const int64_t fit = part_ws == nullptr || part1 == 0 ? 0 : part_bytes / part1;
    a.ksplits = (int)std::max<int64_t>(1, std::min<int64_t>(fit, a.ksplits));
    a.kb_split = (kblocks + a.ksplits - 1) / a.ksplits;
    a.ksplits = (kblocks + a.kb_split - 1) / a.kb_split;
  }
  const int64_t need = a.ksplits > 1 ? (int64_t)a.ksplits * part1 : 0;
  cudaError_t e = cudaSuccess;
  if (a.ksplits > 1) {
    a.part = static_cast<z*>(part_ws);
    e = cudaMemsetAsync(part_ws, 0, need, s);
  } else if (beta.x != 1.0 || beta.y != 0.0) {
    ZGemmArgs g;
    g.M = A.rows;
    g.N = B.rows;
    g.C = C;
    g.ldc = ldc;
    g.beta = beta;
    e = zscale_matrix(g, s);
  }
  if (e != cudaSuccess) return e;
  CUtensorMap mapB = KB.tmap;
  if (tl.bn != 128) {
    e = encode_map_rows(KB, (uint32_t)tl.bn, &mapB);
    if (e != cudaSuccess) return e;
  }
  e = A.kind == kSplitBF16 ? launch_main<kSplitBF16>(KA.tmap, mapB, a, tl.bn, mp.cl, s)
                           : launch_main<kSplitE4M3>(KA.tmap, mapB, a, tl.bn, mp.cl, s);
  if (e != cudaSuccess || a.ksplits == 1) return e;
  // the partials are in C's orientation (A.rows x B.rows) whichever operand took the 128-row side
  part_reduce_kernel<<<grid_for(A.rows * B.rows, 256), 256, 0, s>>>(a.part, a.ksplits, A.rows, B.rows, C, ldc, alpha,
                                                                      beta);
  return cudaGetLastError();
}

cudaError_t split_probe_raw(int kind, const double* Aint, const double* Bint, int64_t M, int64_t N, int64_t K,
                            double* C, void* mem, int* err, cudaStream_t s) {
  SplitConfig cfg;
  cfg.kind = kind;
  cfg.s = 1;
  cfg.b = kind == kSplitBF16 ? 8 : 4;
  SliceSet A, B;
  const int64_t ba = slice_bytes(M, K, cfg);
  uint8_t* m8 = static_cast<uint8_t*>(mem);
  for (SliceSet* S : {&A, &B}) {
    const int64_t rows = S == &A ? M : N;
    S->rows = rows;
    S->rows_pad = round_up(std::max<int64_t>(rows, 1), kRowPad);
    S->K = K;
    S->Kp = round_up(std::max<int64_t>(K, 1), bke(kind));
    S->s = 1;
    S->b = cfg.b;
    S->kind = kind;
    S->digits = S == &A ? (void*)m8 : (void*)(m8 + ba);
    S->scale = nullptr;
    cudaError_t e = encode_map(*S);
    if (e != cudaSuccess) return e;
    const double* src = S == &A ? Aint : Bint;
    const int64_t tot = S->rows_pad * S->Kp;
    if (kind == kSplitBF16)
      raw_digits_kernel<kSplitBF16><<<grid_for(tot, 256), 256, 0, s>>>(src, rows, K, (uint8_t*)S->digits, S->rows_pad,
                                                                       S->Kp);
    else
      raw_digits_kernel<kSplitE4M3><<<grid_for(tot, 256), 256, 0, s>>>(src, rows, K, (uint8_t*)S->digits, S->rows_pad,
                                                                       S->Kp);
  }
  SplitArgs a;
  std::memset(&a, 0, sizeof(a));
  a.M = M;
  a.N = N;
  a.tiles_m = (int)((M + 127) / 128);
  a.tiles = a.tiles_m * (int)((N + 127) / 128);
  a.probe = C;
  a.err = err;
  a.wait_cycles = 4000000000LL;
  // one group: the single pair (0, 0) over the whole K in one accumulator
  a.s = 1;
  a.b = cfg.b;
  a.lmax = 0;
  a.kblocks = (int)(A.Kp / bke(kind));
  a.kbper[0] = a.kblocks;
  a.ksplits = 1;
  a.kb_split = a.kblocks;
  return kind == kSplitBF16 ? launch_split<kSplitBF16, true, 128, 1>(A.tmap, B.tmap, a, s)
                            : launch_split<kSplitE4M3, true, 128, 1>(A.tmap, B.tmap, a, s);
}

}  // namespace ccsd
