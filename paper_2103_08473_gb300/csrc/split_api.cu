// C ABI of the split-precision complex GEMM and of its accumulation probe.
#include <string>

#include "ccsd.h"
#include "errors.h"
#include "split.h"

using namespace ccsd;

namespace {
ccsd_status fail(ccsd_status st, const std::string& msg) {
  set_context_free_error(msg);
  return st;
}
SplitConfig config(int kind, int bits, int slices) {
  SplitConfig c;
  c.kind = kind;
  c.b = bits;
  c.s = slices;
  return c;
}
bool config_ok(int kind, int bits, int slices) {
  return (kind == kSplitE4M3 || kind == kSplitBF16) && slices >= 1 && slices <= 32 && bits >= 1 &&
         bits <= split_max_bits(kind);
}
constexpr size_t kErrBytes = 256;
}  // namespace

extern "C" {

size_t ccsd_split_workspace(int kind, int bits, int slices, long long M, long long N, long long K) {
  if (!config_ok(kind, bits, slices) || M < 0 || N < 0 || K < 0) return 0;
  const SplitConfig c = config(kind, bits, slices);
  return (size_t)(slice_bytes(M, K, c) + slice_bytes(N, K, c) + split_part_bytes(M, N, K, c)) + kErrBytes;
}

ccsd_status ccsd_split_zgemm(int kind, int bits, int slices, int transA, int conjA, int transB, int conjB, long long M,
                             long long N, long long K, ccsd_z alpha, const ccsd_z* A, long long lda, const ccsd_z* B,
                             long long ldb, ccsd_z beta, ccsd_z* C, long long ldc, void* workspace, size_t ws_bytes,
                             void* stream) {
  if (!config_ok(kind, bits, slices)) return fail(CCSD_ERR_ARG, "ccsd_split_zgemm: bad kind/bits/slices");
  if (M < 0 || N < 0 || K < 1 || !A || !B || !C || !workspace)
    return fail(CCSD_ERR_ARG, "ccsd_split_zgemm: bad sizes or NULL");
  const size_t need = ccsd_split_workspace(kind, bits, slices, M, N, K);
  if (ws_bytes < need)
    return fail(CCSD_ERR_ARG, "ccsd_split_zgemm: workspace needs " + std::to_string(need) + " bytes");
  if (M == 0 || N == 0) return CCSD_OK;
  const SplitConfig c = config(kind, bits, slices);
  cudaStream_t st = (cudaStream_t)stream;
  uint8_t* w = static_cast<uint8_t*>(workspace);
  int* err = reinterpret_cast<int*>(w);
  SliceSet SA, SB;
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
  if (e == cudaSuccess) e = make_slices((const z*)A, M, K, lda, transA, conjA, c, SA, w + kErrBytes, st);
  // op(B) is K x N: its columns are the rows of the B digit set
  if (e == cudaSuccess)
    e = make_slices((const z*)B, N, K, ldb, transB ? 0 : 1, conjB, c, SB, w + kErrBytes + slice_bytes(M, K, c), st);
  uint8_t* part = w + kErrBytes + slice_bytes(M, K, c) + slice_bytes(N, K, c);
  if (e == cudaSuccess)
    e = split_gemm(SA, SB, (z*)C, ldc, zmake(alpha.re, alpha.im), zmake(beta.re, beta.im), err, part,
                   split_part_bytes(M, N, K, c), st);
  int h_err = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(CCSD_ERR_CUDA, std::string("ccsd_split_zgemm: ") + cudaGetErrorString(e));
  if (h_err) return fail(CCSD_ERR_TIMEOUT, "ccsd_split_zgemm: a bounded device wait gave up (code " +
                                               std::to_string(h_err) + ")");
  return CCSD_OK;
}

ccsd_status ccsd_split_describe(int kind, int bits, int slices, long long M, long long N, long long K, int* out) {
  if (!config_ok(kind, bits, slices) || M < 0 || N < 0 || K < 0 || !out)
    return fail(CCSD_ERR_ARG, "ccsd_split_describe: bad kind/bits/slices, sizes or NULL");
  split_describe(M, N, K, config(kind, bits, slices), out);
  return CCSD_OK;
}

ccsd_status ccsd_split_probe(int kind, long long M, long long N, long long K, const double* A, const double* B,
                             double* C, void* workspace, size_t ws_bytes, void* stream) {
  if (kind != kSplitE4M3 && kind != kSplitBF16) return fail(CCSD_ERR_ARG, "ccsd_split_probe: bad kind");
  if (M < 1 || N < 1 || K < 1 || !A || !B || !C || !workspace) return fail(CCSD_ERR_ARG, "ccsd_split_probe: bad args");
  const size_t need = ccsd_split_workspace(kind, kind == kSplitBF16 ? 8 : 4, 1, M, N, K);
  if (ws_bytes < need) return fail(CCSD_ERR_ARG, "ccsd_split_probe: workspace needs " + std::to_string(need) + " bytes");
  cudaStream_t st = (cudaStream_t)stream;
  uint8_t* w = static_cast<uint8_t*>(workspace);
  int* err = reinterpret_cast<int*>(w);
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
  if (e == cudaSuccess) e = split_probe_raw(kind, A, B, M, N, K, C, w + kErrBytes, err, st);
  int h_err = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(CCSD_ERR_CUDA, std::string("ccsd_split_probe: ") + cudaGetErrorString(e));
  if (h_err) return fail(CCSD_ERR_TIMEOUT, "ccsd_split_probe: a bounded device wait gave up");
  return CCSD_OK;
}

ccsd_status ccsd_split_wait_selftest(void* stream) {
  // One 128 x 128 x 128 split GEMM whose producer warp issues no copies: the MMA issuer's
  // wait on the first stage must give up after ~2 ms, raise the abort flag (the epilogue
  // warps stop waiting too), free TMEM and return with the error word set.
  const SplitConfig c = config(kSplitE4M3, 5, 2);
  const int64_t n = 128, sb = slice_bytes(n, n, c);
  cudaStream_t st = (cudaStream_t)stream;
  void* mem = nullptr;
  const size_t bytes = kErrBytes + 2 * (size_t)sb + 3 * (size_t)n * n * sizeof(z);
  if (cudaMalloc(&mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(CCSD_ERR_OOM, "ccsd_split_wait_selftest: device memory");
  }
  uint8_t* w = static_cast<uint8_t*>(mem);
  int* err = reinterpret_cast<int*>(w);
  z* X = reinterpret_cast<z*>(w + kErrBytes + 2 * sb);  // A, B, C: n x n each
  SliceSet SA, SB;
  cudaError_t e = cudaMemsetAsync(mem, 0, bytes, st);
  if (e == cudaSuccess) e = make_slices(X, n, n, n, 0, 0, c, SA, w + kErrBytes, st);
  if (e == cudaSuccess) e = make_slices(X + n * n, n, n, n, 0, 0, c, SB, w + kErrBytes + sb, st);
  if (e == cudaSuccess)
    e = split_gemm(SA, SB, X + 2 * n * n, n, zmake(1, 0), zmake(0, 0), err, nullptr, 0, st, 4000000LL, 1);
  int h_err = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(mem);
  if (e != cudaSuccess) return fail(CCSD_ERR_CUDA, std::string("ccsd_split_wait_selftest: ") + cudaGetErrorString(e));
  if (h_err == 0) return fail(CCSD_ERR_CUDA, "ccsd_split_wait_selftest: the stalled wait did not give up");
  return fail(CCSD_ERR_TIMEOUT, "ccsd_split_wait_selftest: bounded wait gave up as intended (code " +
                                    std::to_string(h_err) + ")");
}

}  // extern "C"
