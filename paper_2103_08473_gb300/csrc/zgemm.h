// Complex GEMM interfaces of libccsd (host side).
#pragma once

#include "common.cuh"

namespace ccsd {

// C[b] = alpha * opA(A[b]) * opB(B[b]) + beta * C[b], row-major complex double.
//   opA element (m,k) = transA ? A[k*lda + m] : A[m*lda + k]   (conjugated if conjA)
//   opB element (k,n) = transB ? B[n*ldb + k] : B[k*ldb + n]   (conjugated if conjB)
//   C element (m,n)   = C[m*ldc + n]
// Batch b offsets the three pointers by b*sA, b*sB, b*sC elements.
struct ZGemmArgs {
  int64_t M = 0, N = 0, K = 0;
  int batch = 1;
  const z* A = nullptr;
  int64_t lda = 0, sA = 0;
  const z* B = nullptr;
  int64_t ldb = 0, sB = 0;
  z* C = nullptr;
  int64_t ldc = 0, sC = 0;
  z alpha{1.0, 0.0}, beta{0.0, 0.0};
  int transA = 0, transB = 0, conjA = 0, conjB = 0;
  // Split-K workspace (complex elements). GEMMs with too few output tiles to fill the GPU
  // split K into S slices whose partial products go to ws and are summed in a fixed order.
  z* ws = nullptr;
  int64_t ws_elems = 0;
  int cfg = -1;  // FP64 tile configuration (0..6), -1 = cost model
  int mult4 = 0; // 1: four real products per complex product (4M); 0: three (3M)
};

// FP64 tensor-core (DMMA) path. cfg < 0 picks the tile shape from the tile count.
cudaError_t zgemm_f64(const ZGemmArgs& g, cudaStream_t s, int cfg = -1);
int64_t zgemm_f64_tiles(const ZGemmArgs& g, int cfg);
// Workspace (complex elements) zgemm_f64 wants for this shape to split K (0 if it does not split).
int64_t zgemm_f64_workspace(const ZGemmArgs& g);
// C[b] = beta * C[b] over the M x N (ldc) matrices (the K = 0 case).
cudaError_t zscale_matrix(const ZGemmArgs& g, cudaStream_t s);

}  // namespace ccsd
