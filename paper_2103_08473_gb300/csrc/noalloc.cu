// ccsd_zgemm_noalloc: the engine's complex GEMM for callers that cannot allocate
// device memory.
//
// Some callers must not call cudaMalloc: code that runs inside another
// framework's memory budget (a caching allocator such as PyTorch's owns the
// device memory, and memory taken behind its back can make its own allocations
// fail), code in a latency-critical loop (cudaMalloc and cudaFree can
// synchronise the device), and code that has to keep the device footprint it
// fixed at start-up. ccsd_zgemm needs such a caller to pass a split-K
// workspace. This variant keeps the split-K partials in a fixed array that
// lives in the library's own device memory instead, so it allocates nothing.
//
// The array is a file-scope __device__ variable of kStaticSplitElems complex
// doubles (4 MiB). Every GPU that loads the library holds it until the process
// exits. In host code its name is only a host-side stand-in, so each call looks
// up the array's device address with cudaGetSymbolAddress while the caller's
// device is current. The lookup allocates nothing and is redone on every call,
// so the address stays right after a device reset reloads the module.
#include <string>

#include "ccsd.h"
#include "errors.h"
#include "zgemm.h"

namespace {

using ccsd::z;

constexpr long long kStaticSplitElems = 1LL << 18;  // complex doubles: 4 MiB
static __device__ __align__(256) z g_splitk_scratch[kStaticSplitElems];

// The message is read back with ccsd_last_error(NULL).
ccsd_status fail(ccsd_status st, const std::string& msg) {
  ccsd::set_context_free_error(msg);
  return st;
}

}  // namespace

extern "C" ccsd_status ccsd_zgemm_noalloc(int precision, int transA, int conjA, int transB, int conjB, long long M,
                                          long long N, long long K, ccsd_z alpha, const ccsd_z* A, long long lda,
                                          const ccsd_z* B, long long ldb, ccsd_z beta, ccsd_z* C, long long ldc,
                                          int cfg, void* stream) {
  if (M < 0 || N < 0 || K < 0 || !A || !B || !C) return fail(CCSD_ERR_ARG, "ccsd_zgemm_noalloc: bad sizes or NULL");
  if (cfg > 6) return fail(CCSD_ERR_ARG, "ccsd_zgemm_noalloc: cfg must be < 7");
  if (precision != CCSD_PREC_FP64) return fail(CCSD_ERR_UNSUPPORTED, "ccsd_zgemm_noalloc: precision not built");
  // The static scratch must hold at least two split partials of the output.
  if (2 * M * N > kStaticSplitElems)
    return fail(CCSD_ERR_ARG, "ccsd_zgemm_noalloc: output of " + std::to_string(M * N) +
                                  " complex elements exceeds the limit of " + std::to_string(kStaticSplitElems / 2) +
                                  " (M*N) for the static split-K scratch; use ccsd_zgemm with a workspace");
  // the array's address on the current device (the lookup allocates nothing)
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_splitk_scratch);
  if (e != cudaSuccess) return fail(CCSD_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  z* scratch = static_cast<z*>(p);
  ccsd::ZGemmArgs g;
  g.M = M;
  g.N = N;
  g.K = K;
  g.A = (const z*)A;
  g.lda = lda;
  g.B = (const z*)B;
  g.ldb = ldb;
  g.C = (z*)C;
  g.ldc = ldc;
  g.alpha = ccsd::zmake(alpha.re, alpha.im);
  g.beta = ccsd::zmake(beta.re, beta.im);
  g.transA = transA != 0;
  g.transB = transB != 0;
  g.conjA = conjA != 0;
  g.conjB = conjB != 0;
  // Every partial the reduction reads is written earlier in the same call, so no
  // part of the array has to start at zero.
  g.ws = scratch;
  g.ws_elems = kStaticSplitElems;
  cudaStream_t st = (cudaStream_t)stream;
  e = ccsd::zgemm_f64(g, st, cfg);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(CCSD_ERR_CUDA, std::string("ccsd_zgemm_noalloc: ") + cudaGetErrorString(e));
  return CCSD_OK;
}
