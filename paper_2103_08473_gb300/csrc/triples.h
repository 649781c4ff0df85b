// Perturbative triples corrections at converged CCSD amplitudes (host side).
#pragma once

#include <vector>

#include "common.cuh"
#include "split.h"

namespace ccsd {

// Optional timing: four events per batch (before the e-term GEMMs, before the m-term GEMMs,
// before the energy kernel, after its accumulation), recorded on the evaluation's stream.
struct TriplesTimer {
  std::vector<cudaEvent_t> ev;
  cudaError_t mark(cudaStream_t s) {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    ev.push_back(e);
    return cudaEventRecord(e, s);
  }
  // After the stream is synchronised: ms[0..2] = time of the e-term GEMMs, the m-term GEMMs and
  // the energy kernels, summed over the batches.
  cudaError_t sums(double ms[3]) const {
    ms[0] = ms[1] = ms[2] = 0.0;
    for (size_t b = 0; b + 3 < ev.size(); b += 4)
      for (int g = 0; g < 3; ++g) {
        float t = 0.f;
        cudaError_t r = cudaEventElapsedTime(&t, ev[b + g], ev[b + g + 1]);
        if (r != cudaSuccess) return r;
        ms[g] += t;
      }
    return cudaSuccess;
  }
  ~TriplesTimer() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
};

// Device pointers of the context's constant blocks and amplitudes, and the call's workspace.
struct TriplesArgs {
  int o = 0, v = 0;
  const z* t1 = nullptr;       // [i][a]
  const z* t2 = nullptr;       // [i][j][a][b]
  const z* oovv = nullptr;     // <ij||ab> [i][j][a][b]
  const z* ooov = nullptr;     // <kl||ic> [k][l][i][c]
  const z* vovv_pk = nullptr;  // <ak||cd> [(a,k)][P(c,d)]
  const z* fov = nullptr;      // f_ia [i][a]
  const double* d = nullptr;   // real diagonal of the Fock matrix (o + v)
  z* t2pk = nullptr;           // o*o*P(v): t2 packed over its virtual pair
  z* work = nullptr;           // max_batch * triples_batch_elems(v)
  int max_batch = 1;           // triples (i, j, k) per batch, k consecutive
  float4* dsf = nullptr;       // triples_dsf_elems(o, v): double-single copies of t1, f_ov, t2 and
                               // <ij||ab> for the energy kernel's fifth-order terms
  double* partials = nullptr;  // triples_partials() doubles
  double* pair_acc = nullptr;  // o*o*3 doubles, zeroed by the caller; [(i*o + j)*3 + m] += the
                               // pair's sums of |X|^2/D (m=0), Re(X Z)/D (1), Re(X conj Y) (2)
  // Split precision (null: FP64). The e-terms: digits of conj(<eL||ab>) over K = e for every L
  // (rows L*P(v) + P(a,b)) and of t2 over K = e (rows (p*o + q)*v + c). The m-terms: digits of
  // conj(<pq||ma>) over K = m (rows (p*o + q)*v + a) and of the pair-packed t2 over K = m (rows
  // L*P(v) + P(b,c)). Each term is then ONE split GEMM per batch of k, of row views whose rows
  // run over the batch's k (the antisymmetry of t2 and of <pq||ma> in their occupied pair turns
  // the (k,i) rows into the contiguous (i,k) ones); two of the six products come out in a
  // second layout, E2[P(a,b)][t][c] and M2[a][t][P(b,c)].
  const SliceSet* sa = nullptr;
  const SliceSet* sb = nullptr;
  const SliceSet* sm = nullptr;
  const SliceSet* st = nullptr;
  int* split_err = nullptr;
  TriplesTimer* timer = nullptr;  // optional
  int64_t batches = 0;            // out: batches run
  int64_t launches = 0;           // out: kernels launched
};

// Complex elements of workspace per triple of a batch (the packed parts of W: two in FP64, four
// in split precision).
int64_t triples_batch_elems(int v, bool split);
// float4 elements of the double-single copies (t1, f_ov: o v each; t2, <ij||ab>: o^2 v^2 each).
int64_t triples_dsf_elems(int o, int v);
// Doubles of block partials the energy kernel writes per batch.
int64_t triples_partials(const TriplesArgs& a);
// Enqueue the whole evaluation on s (no synchronisation). o < 3 or v < 3: nothing to do.
cudaError_t triples_eval(TriplesArgs& a, cudaStream_t s);

}  // namespace ccsd
