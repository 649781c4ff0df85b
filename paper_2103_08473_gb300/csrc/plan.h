// Contraction planner of libccsd (host C++).
//
// Every line of the Appendix A working equations is a binary tensor contraction
//   C(lc) = beta * C(lc) + alpha * A(la) * B(lb)      (labels as in the paper)
// in the style of the symbolic contraction strings of the paper's tensor runtime
// ("S(a,b,i,j) += V(a,b,c,d) * T(c,d,i,j)", "+" = complex conjugate). The planner
// turns each one, once at context creation, into a short list of device
// operations: index permutations that bring the operands to [free][contracted]
// form (skipped where a transposed GEMM operand does the job), one complex GEMM
// (or GEMV when a side has no free index), and a permutation of the result when
// the output labels interleave the two free sets. Permutations of constant
// operands (integral blocks) are done once at plan time and cached.
//
// The op list is executed in order on one stream, so it can be captured in a
// CUDA graph. Temporaries live in a scratch region whose base is allocated after
// planning (its size is the high-water mark of the plan).
#pragma once

#include <algorithm>
#include <cstdint>
#include <functional>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "common.cuh"
#include "zgemm.h"

namespace ccsd {

// A device pointer that may be resolved late (scratch base + offset).
struct Ptr {
  z* direct = nullptr;
  z* const* base = nullptr;
  int64_t off = 0;
  z* get() const { return direct ? direct : (*base) + off; }
};

// Dense row-major tensor view: dims[k] belongs to label lab[k].
struct T {
  Ptr p;
  std::string lab;
  std::vector<int64_t> dims;
  bool cnst = false;
  int64_t size() const {
    int64_t s = 1;
    for (auto d : dims) s *= d;
    return s;
  }
};

// Complex GEMM back end used by a plan (FP64 DMMA, or split precision), and the
// workspace (complex elements) it wants for a shape.
using GemmFn = std::function<cudaError_t(const ZGemmArgs&, cudaStream_t)>;
using WsFn = std::function<int64_t(const ZGemmArgs&)>;

struct Op {
  std::string name;
  std::function<cudaError_t(cudaStream_t)> run;
  double flops = 0.0;  // algorithmic real flops (8 per complex multiply-add)
  // GEMM ops: the arguments (pointers resolved at run time) and the tile configuration the
  // autotuner may set (-1 = cost model).
  std::shared_ptr<int> cfg;
  std::shared_ptr<ZGemmArgs> args;
};

class Plan {
 public:
  Plan(int o, int v, z* const* scratch_base, cudaStream_t setup_stream)
      : o_(o), v_(v), scratch_base_(scratch_base), setup_(setup_stream) {}

  // Dims from label letters: i..n occupied (o), a..h virtual (v).
  T view(z* p, const std::string& lab, bool cnst = false) const;
  T view(Ptr p, const std::string& lab, bool cnst = false) const;

  // C = beta C + alpha op(A) with A relabelled to C's index order.
  void add(const std::string& name, const T& C, z alpha, const T& A, bool conjA, double beta);
  // C = beta C + alpha opA(A) opB(B), contracted over the labels A and B share.
  void contract(const std::string& name, const T& C, z alpha, const T& A, bool conjA, const T& B, bool conjB,
                double beta);
  // Raw op (custom kernels, packed GEMMs).
  void custom(const std::string& name, std::function<cudaError_t(cudaStream_t)> fn, double flops = 0.0);
  // GEMM op on raw pointers through the plan's GEMM back end.
  void gemm(const std::string& name, const ZGemmArgs& g);

  // ws: split-K workspace (complex elements); aux: other per-call workspace (bytes),
  // e.g. the digit slices of a split-precision GEMM. Both are sized by their peaks.
  void set_gemm(GemmFn fn, WsFn ws, WsFn aux = nullptr) {
    gemm_ = std::move(fn);
    wsfn_ = std::move(ws);
    auxfn_ = std::move(aux);
  }
  void note_aux_bytes(int64_t b) { aux_peak_ = std::max(aux_peak_, b); }
  // Size the workspaces for a GEMM that a custom op will run through gemm_fn().
  void note_gemm(const ZGemmArgs& g) {
    if (wsfn_) ws_peak_ = std::max(ws_peak_, wsfn_(g));
    if (auxfn_) aux_peak_ = std::max(aux_peak_, auxfn_(g));
  }
  int64_t aux_bytes() const { return aux_peak_; }
  const GemmFn& gemm_fn() const { return gemm_; }
  // Largest GEMM workspace any op of the plan wants (complex elements).
  int64_t gemm_workspace_elems() const { return ws_peak_; }

  std::vector<Op>& ops() { return ops_; }
  int64_t scratch_elems() const { return scratch_peak_; }
  // A custom op that keeps its own temporaries at the start of the scratch region (none of the
  // plan's temporaries is live while a custom op runs) makes the region at least this large.
  void reserve_scratch(int64_t elems) { scratch_peak_ = std::max(scratch_peak_, elems); }
  // Persistent buffers created by the planner (cached permutations of constants), and their bytes.
  std::vector<void*>& owned() { return owned_; }
  int64_t owned_bytes() const { return owned_bytes_; }
  // Constant operands larger than this (bytes) are not cached in their permuted layout: each use
  // permutes them into the scratch region instead (default: no limit). Large problems trade one
  // extra pass over such an integral block per use for its permuted copy's memory.
  void set_cache_limit(int64_t bytes) { cache_limit_ = bytes; }
  cudaError_t status() const { return status_; }
  const std::string& error() const { return error_; }

 private:
  Ptr temp(int64_t elems);
  T permuted(const T& src, const std::string& lab, bool conj, const std::string& name);
  void fail(const std::string& msg, cudaError_t e = cudaErrorInvalidValue);
  int64_t dim_of(char c) const;

  int o_, v_;
  z* const* scratch_base_;
  cudaStream_t setup_;
  GemmFn gemm_;
  WsFn wsfn_, auxfn_;
  int64_t ws_peak_ = 0, aux_peak_ = 0;
  std::vector<Op> ops_;
  int64_t scratch_off_ = 0, scratch_peak_ = 0;
  std::map<std::string, T> const_cache_;
  std::vector<void*> owned_;
  int64_t owned_bytes_ = 0;
  int64_t cache_limit_ = INT64_MAX;
  cudaError_t status_ = cudaSuccess;
  std::string error_;
};

// y = alpha * op(M) x + beta y (complex), M(r, k) = rowmajor ? M[r*ld + k] : M[k*ld + r].
cudaError_t zgemv(int64_t R, int64_t K, z alpha, const z* M, int64_t ld, int rowmajor, int conjM, const z* x,
                  int conjx, double beta, z* y, cudaStream_t s);

}  // namespace ccsd
