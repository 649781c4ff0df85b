// C ABI of libccsd (include/ccsd.h): context creation, the Appendix A residual
// plan, the denominator update + DIIS iteration (CUDA-graph replayed), energy,
// amplitude checkpointing and inspection.
#include <cmath>
#include <algorithm>
#include <array>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ccsd.h"
#include "errors.h"
#include "ops.h"
#include "plan.h"
#include "split.h"
#include "triples.h"
#include "zgemm.h"

using namespace ccsd;

namespace {
thread_local std::string g_create_error;
}  // namespace

namespace ccsd {
void set_context_free_error(const std::string& msg) { g_create_error = msg; }
}  // namespace ccsd

struct ccsd_ctx {
  int o = 0, v = 0, n = 0, naux = 0;
  int64_t Po = 0, Pv = 0;
  ccsd_opts opts{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  std::vector<void*> allocs;

  // constants
  double* dvec = nullptr;  // real diagonal of the Fock matrix (n)
  z *foo = nullptr, *fov = nullptr, *fvv = nullptr;
  z *oooo = nullptr, *ooov = nullptr, *oovv = nullptr;
  z *Wpk = nullptr, *vovv_pk = nullptr, *oovv_pk = nullptr, *J = nullptr;
  // amplitudes and residual
  z *t1 = nullptr, *t2 = nullptr, *S1 = nullptr, *S2 = nullptr;
  z *t1_prev = nullptr, *t2_prev = nullptr, *t1_save = nullptr, *t2_save = nullptr;
  // intermediates
  z *tau = nullptr, *tau_pk = nullptr;
  z* vblk = nullptr;  // rows of <ak||cd> over all (c, d), unpacked block by block from vovv_pk
  int64_t vblk_rows = 0;
  z *Hvv = nullptr, *Gvv = nullptr, *Hoo = nullptr, *Goo = nullptr, *Hov = nullptr, *Yov = nullptr, *Zoo = nullptr;
  z *Hr = nullptr, *R = nullptr;
  z *C = nullptr, *Yovoo = nullptr, *Ypk = nullptr, *Yfull = nullptr;
  z *Afull = nullptr, *Yoooo = nullptr, *Apk = nullptr, *Lpk = nullptr, *Hpk = nullptr;
  z* scratch = nullptr;
  z* gemm_ws = nullptr;  // split-K partials of the plan's GEMMs
  int64_t gemm_ws_elems = 0;
  // split precision: digit slices on the tensor cores for the large contractions
  bool use_split = false;
  SplitConfig split;
  double split_min_flops = 2e10;
  void* split_ws = nullptr;  // per-call digit slices of both operands
  int64_t split_ws_bytes = 0;
  int64_t plan_cached_bytes = 0;  // permuted copies of constant operands the residual plan keeps
  int64_t split_budget = int64_t(4) << 30;  // digit bytes of both operands per split call
  int* split_err = nullptr;  // set by the tensor-core kernel if a bounded wait gave up
  SliceSet Wsl, tausl;       // <ab||cd> digits (built once) and tau digits (per evaluation)
  // split mode, when they fit: digits of the unpacked <ak||cd> rows (a,k,c) over K = d, one set
  // per block of a, cut once; the H^{ak}_{ci} t1 term then slices only t1 per evaluation
  std::vector<SliceSet> vovv_sl;
  uint8_t* t1sl_mem = nullptr;
  void* tausl_mem = nullptr; // tau digits of the on-the-fly ladder (kept across its blocks)
  // store_w = 0: B^Q over virtuals, and per-block (ac|bd) and packed <ab||cd> rows
  z *Bvv = nullptr, *Dblk = nullptr, *Wblk = nullptr;
  int64_t df_w_off = -1;  // store_w = 0: offset of the packed rows after D in the plan's scratch
  SliceSet Bsl;  // split mode: digits of B^Q_vv as rows (a, c) over Q, cut once (both operands of the rebuild)
  // CC2: the DF factor blocks B^Q_vo, B^Q_oo, B^Q_ov (B^Q_vv is Bvv) and the per-evaluation dressed
  // factors Bt[Q][a][i] = ((1 - t1) B^Q (1 + t1))_ai and Dt[Q][j][i] = (B^Q (1 + t1))_ji
  z *c2_Bvo = nullptr, *c2_Boo = nullptr, *c2_Bov = nullptr, *c2_Bt = nullptr, *c2_Dt = nullptr;
  int df_block = 0;
  std::function<bool(const ZGemmArgs&)> routes_split;
  // iteration state
  double* upd_partials = nullptr;
  double* stats = nullptr;
  double* stats_host = nullptr;  // pinned
  int* err_host = nullptr;        // pinned copy of split_err
  z* e_partials = nullptr;
  z* e_dev = nullptr;
  z* e_host = nullptr;  // pinned
  DiisArgs diis;
  Plan* plan = nullptr;
  cudaGraphExec_t graph = nullptr;
  // profiling: one event per op boundary, recorded inside the iteration graph
  std::vector<std::string> tnames;
  std::vector<cudaEvent_t> tev;
  std::vector<double> tsum;
  int tcount = 0;
  int kernels_per_iter = 0;
  int64_t device_bytes = 0;
  int64_t iterations_run = 0;
  // growth record of the update norm (ccsd_divergence_index's rule, kept across ccsd_iterate calls)
  struct Growth {
    int up = 0;
    double base = 0.0, last = 0.0;
    bool started = false;
    void reset() { *this = Growth(); }
    // true when norm ends a run of >= iters consecutive increases with norm > factor * base
    bool push(double norm, int iters, double factor) {
      if (!started || !(norm > last)) {
        up = 0;
        base = norm;
      } else {
        up += 1;
      }
      started = true;
      last = norm;
      return iters > 0 && up >= iters && norm > factor * base;
    }
  } growth, lgrowth;
  // Lambda equations (built on first use): multipliers, the plan of their residual (the adjoint of
  // the residual plan), its buffers and DIIS subspace; the density plan
  z *l1 = nullptr, *l2 = nullptr;
  Plan *lplan = nullptr, *dplan = nullptr;
  z *lscratch = nullptr, *dscratch = nullptr;
  DiisArgs ldiis;
  z *lG = nullptr, *ltaub = nullptr, *lHrb = nullptr, *lXb = nullptr, *lzb = nullptr, *lCb = nullptr,
    *lCanti = nullptr, *lCp = nullptr, *lAb = nullptr, *lAanti = nullptr, *lpk = nullptr,
    *lpk2 = nullptr, *lout = nullptr, *lout2 = nullptr, *lout3 = nullptr, *lApk = nullptr;
  z *lGvvb = nullptr, *lHvvb = nullptr, *lGoob = nullptr, *lHoob = nullptr, *lHovb = nullptr;
  z *dgoo = nullptr, *dgvo = nullptr, *dgvv = nullptr, *dq1 = nullptr, *dq2 = nullptr, *dq3 = nullptr, *dgam = nullptr,
    *dgam2 = nullptr;
  int64_t lambda_iterations = 0;
  // profile = 1: one event per Lambda-plan op boundary, and the summed device time per op
  std::vector<cudaEvent_t> lev;
  cudaGraphExec_t lgraph = nullptr;  // one Lambda iteration (plan, update, norms, DIIS), captured once
  int lkernels_per_iter = 0;
  std::vector<double> ltsum;
  int64_t ltcount = 0;
  // the last ccsd_triples call: batch size, batches, kernel launches and (profile = 1) device time of
  // its e-term GEMMs, m-term GEMMs and energy kernels
  int64_t tri_batch = 0, tri_batches = 0, tri_launches = 0;
  double tri_ms[3] = {0.0, 0.0, 0.0};
};

namespace {

ccsd_status set_err(ccsd_ctx* c, ccsd_status st, const std::string& msg) {
  if (c) c->err = msg;
  else g_create_error = msg;
  return st;
}

#define CK(call)                                                                                     \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess)                                                                           \
      return set_err(ctx, e_ == cudaErrorMemoryAllocation ? CCSD_ERR_OOM : CCSD_ERR_CUDA,            \
                     std::string(#call) + ": " + cudaGetErrorString(e_));                            \
  } while (0)

template <typename Tp>
ccsd_status dalloc(ccsd_ctx* ctx, Tp** p, int64_t count) {
  void* m = nullptr;
  size_t bytes = (size_t)std::max<int64_t>(count, 1) * sizeof(Tp);
  cudaError_t e = cudaMalloc(&m, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, CCSD_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  ctx->allocs.push_back(m);
  ctx->device_bytes += (int64_t)bytes;
  *p = (Tp*)m;
  return CCSD_OK;
}

#define CS(call)                        \
  do {                                  \
    ccsd_status s_ = (call);            \
    if (s_ != CCSD_OK) return s_;       \
  } while (0)

// out[d0][d1][d2][d3] (+)= alpha * in[...] where output dim d is input dim perm[d].
cudaError_t permute4(const z* in, const int64_t idims[4], const int perm[4], z* out, z alpha, double beta, int conj,
                     cudaStream_t s) {
  PermuteArgs a;
  a.rank = 4;
  int64_t ist[4];
  ist[3] = 1;
  for (int k = 2; k >= 0; --k) ist[k] = ist[k + 1] * idims[k + 1];
  int64_t od[4];
  for (int d = 0; d < 4; ++d) od[d] = idims[perm[d]];
  int64_t ost[4];
  ost[3] = 1;
  for (int k = 2; k >= 0; --k) ost[k] = ost[k + 1] * od[k + 1];
  for (int d = 0; d < 4; ++d) {
    a.dims[d] = od[d];
    a.istr[d] = ist[perm[d]];
    a.ostr[d] = ost[d];
  }
  a.in = in;
  a.out = out;
  a.alpha = alpha;
  a.beta = beta;
  a.conj = conj;
  return permute_add(a, s);
}

// Space ranges: 'o' = [0, o), 'v' = [o, n).
void space(const ccsd_ctx* c, char s, int64_t& off, int64_t& len) {
  off = s == 'o' ? 0 : c->o;
  len = s == 'o' ? c->o : c->v;
}

// Extract B[Q][P-range][R-range] into a contiguous [naux][np][nr] buffer.
cudaError_t extract_B(const ccsd_ctx* c, const z* B, char P, char Rs, z* out, cudaStream_t s) {
  int64_t p0, np, r0, nr;
  space(c, P, p0, np);
  space(c, Rs, r0, nr);
  PermuteArgs a;
  a.rank = 3;
  a.dims[0] = c->naux;
  a.dims[1] = np;
  a.dims[2] = nr;
  a.istr[0] = (int64_t)c->n * c->n;
  a.istr[1] = c->n;
  a.istr[2] = 1;
  a.ostr[0] = np * nr;
  a.ostr[1] = nr;
  a.ostr[2] = 1;
  a.in = B + p0 * c->n + r0;
  a.out = out;
  return permute_add(a, s);
}

// One GEMM of an integral build (a Coulomb block over Q): FP64, or in split mode on the
// tensor cores with at least 44-bit digits (the integrals are built once).
ccsd_status coulomb_gemm(ccsd_ctx* ctx, ZGemmArgs g) {
  g.mult4 = ctx->opts.complex_4m;
  if (!ctx->use_split) {
    CK(zgemm_f64(g, ctx->stream));
    return CCSD_OK;
  }
  SplitConfig c = ctx->split;
  c.s = std::max(c.s, (44 + c.b) / c.b);
  const int64_t sa = slice_bytes(g.M, g.K, c), sb = slice_bytes(g.N, g.K, c), sp = split_part_bytes(g.M, g.N, g.K, c);
  void* mem = nullptr;
  if (cudaMalloc(&mem, sa + sb + sp) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, CCSD_ERR_OOM, "slices of the Coulomb build");
  }
  uint8_t* w = static_cast<uint8_t*>(mem);
  SliceSet SA, SB;
  cudaError_t e = make_slices(g.A, g.M, g.K, g.lda, g.transA, 0, c, SA, w, ctx->stream);
  if (e == cudaSuccess) e = make_slices(g.B, g.N, g.K, g.ldb, g.transB ? 0 : 1, 0, c, SB, w + sa, ctx->stream);
  if (e == cudaSuccess)
    e = split_gemm(SA, SB, g.C, g.ldc, zmake(1, 0), zmake(0, 0), ctx->split_err, w + sa + sb, sp, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(mem);
  if (e != cudaSuccess) return set_err(ctx, CCSD_ERR_CUDA, std::string("split Coulomb build: ") + cudaGetErrorString(e));
  return CCSD_OK;
}

// Coulomb block D[(p,r)][(q,s)] = sum_Q B^Q_pr B^Q_qs for spaces (P,R) x (Q,S).
ccsd_status coulomb_df(ccsd_ctx* ctx, const z* B, char P, char Rr, char Q, char S, z* D, z* tmp1, z* tmp2) {
  int64_t po, np, ro, nr, qo, nq, so, ns;
  space(ctx, P, po, np);
  space(ctx, Rr, ro, nr);
  space(ctx, Q, qo, nq);
  space(ctx, S, so, ns);
  CK(extract_B(ctx, B, P, Rr, tmp1, ctx->stream));
  CK(extract_B(ctx, B, Q, S, tmp2, ctx->stream));
  ZGemmArgs g;
  g.M = np * nr;
  g.N = nq * ns;
  g.K = ctx->naux;
  g.A = tmp1;
  g.lda = g.M;
  g.transA = 1;
  g.B = tmp2;
  g.ldb = g.N;
  g.C = D;
  g.ldc = g.N;
  return coulomb_gemm(ctx, g);
}

// <pq||rs> block for spaces "PQRS" from the DF factors, written as out[p][q][r][s].
ccsd_status build_block_df(ccsd_ctx* ctx, const z* B, const char* sp, z* out) {
  int64_t o_, np, nq, nr, ns;
  space(ctx, sp[0], o_, np);
  space(ctx, sp[1], o_, nq);
  space(ctx, sp[2], o_, nr);
  space(ctx, sp[3], o_, ns);
  const int64_t nb = (int64_t)ctx->naux * ctx->n * ctx->n;
  z *t1 = nullptr, *t2 = nullptr, *D = nullptr;
  std::vector<void*> mine;
  auto cleanup = [&]() {
    for (void* p : mine) cudaFree(p);
  };
  auto get = [&](z** p, int64_t cnt) -> bool {
    void* m = nullptr;
    if (cudaMalloc(&m, (size_t)std::max<int64_t>(cnt, 1) * sizeof(z)) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    mine.push_back(m);
    *p = (z*)m;
    return true;
  };
  if (!get(&t1, nb) || !get(&t2, nb) || !get(&D, np * nr * nq * ns)) {
    cleanup();
    return set_err(ctx, CCSD_ERR_OOM, "integral build temporaries");
  }
  ccsd_status st = coulomb_df(ctx, B, sp[0], sp[2], sp[1], sp[3], D, t1, t2);
  if (st != CCSD_OK) { cleanup(); return st; }
  // direct part: out[p][q][r][s] = D[p][r][q][s]
  {
    const int64_t idims[4] = {np, nr, nq, ns};
    const int perm[4] = {0, 2, 1, 3};
    cudaError_t e = permute4(D, idims, perm, out, zmake(1, 0), 0.0, 0, ctx->stream);
    if (e != cudaSuccess) { cleanup(); return set_err(ctx, CCSD_ERR_CUDA, cudaGetErrorString(e)); }
  }
  // exchange part: out[p][q][r][s] -= X[p][s][q][r], X = (ps|qr)
  if (sp[2] != sp[3]) {
    st = coulomb_df(ctx, B, sp[0], sp[3], sp[1], sp[2], D, t1, t2);
    if (st != CCSD_OK) { cleanup(); return st; }
  }
  {
    const int64_t idims[4] = {np, ns, nq, nr};  // X[p][s][q][r]
    const int perm[4] = {0, 2, 3, 1};           // out dims (p, q, r, s) <- X dims (0, 2, 3, 1)
    cudaError_t e = permute4(D, idims, perm, out, zmake(-1, 0), 1.0, 0, ctx->stream);
    if (e != cudaSuccess) { cleanup(); return set_err(ctx, CCSD_ERR_CUDA, cudaGetErrorString(e)); }
  }
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  cleanup();
  if (e != cudaSuccess) return set_err(ctx, CCSD_ERR_CUDA, cudaGetErrorString(e));
  return CCSD_OK;
}

// <ak||cd> packed over c < d (vovv_pk[(a,k)][P(c,d)]) from the DF factors, in blocks of a so
// that the dense vovv block is never formed: D[(a,c)][(k,d)] = (ac|kd) = sum_Q B^Q_ac B^Q_kd for
// the block (one GEMM over Q), then <ak||cd> = (ac|kd) - (ad|kc) = D[a][c][k][d] - D[a][d][k][c].
ccsd_status build_vovv_pk_df(ccsd_ctx* ctx, const z* B) {
  const int64_t o = ctx->o, v = ctx->v, naux = ctx->naux, Pv = ctx->Pv;
  const int64_t per_a = v * o * v;  // D elements per a
  const int64_t blk = std::max<int64_t>(1, std::min<int64_t>(v, (int64_t)(1.0e9 / (16.0 * (double)per_a))));
  void *mvv = nullptr, *mov = nullptr, *mD = nullptr;
  if (cudaMalloc(&mvv, naux * v * v * sizeof(z)) != cudaSuccess ||
      cudaMalloc(&mov, naux * o * v * sizeof(z)) != cudaSuccess ||
      cudaMalloc(&mD, blk * per_a * sizeof(z)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(mvv);
    cudaFree(mov);
    cudaFree(mD);
    return set_err(ctx, CCSD_ERR_OOM, "vovv build temporaries");
  }
  z *bvv = (z*)mvv, *bov = (z*)mov, *D = (z*)mD;
  ccsd_status st = CCSD_OK;
  cudaError_t e = extract_B(ctx, B, 'v', 'v', bvv, ctx->stream);
  if (e == cudaSuccess) e = extract_B(ctx, B, 'o', 'v', bov, ctx->stream);
  if (e != cudaSuccess) st = set_err(ctx, CCSD_ERR_CUDA, cudaGetErrorString(e));
  for (int64_t a0 = 0; a0 < v && st == CCSD_OK; a0 += blk) {
    const int64_t na = std::min(blk, v - a0);
    ZGemmArgs g;  // D[(a,c)][(k,d)], a in [a0, a0 + na)
    g.M = na * v;
    g.N = o * v;
    g.K = naux;
    g.A = bvv + a0 * v;
    g.lda = v * v;
    g.transA = 1;
    g.B = bov;
    g.ldb = o * v;
    g.C = D;
    g.ldc = o * v;
    st = coulomb_gemm(ctx, g);
    if (st != CCSD_OK) break;
    e = pack_vovv_rows(D, ctx->vovv_pk + a0 * o * Pv, na, o, v, ctx->stream);
    if (e != cudaSuccess) st = set_err(ctx, CCSD_ERR_CUDA, cudaGetErrorString(e));
  }
  e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess && st == CCSD_OK) st = set_err(ctx, CCSD_ERR_CUDA, cudaGetErrorString(e));
  cudaFree(mvv);
  cudaFree(mov);
  cudaFree(mD);
  return st;
}

ccsd_status build_block_full(ccsd_ctx* ctx, const z* V, const char* sp, z* out);

// The same from the full integral tensor (tiny n only): the dense block as a temporary.
ccsd_status build_vovv_pk_full(ccsd_ctx* ctx, const z* V) {
  const int64_t ov = (int64_t)ctx->o * ctx->v, vv = (int64_t)ctx->v * ctx->v;
  void* m = nullptr;
  if (cudaMalloc(&m, ov * vv * sizeof(z)) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, CCSD_ERR_OOM, "vovv temporary");
  }
  ccsd_status st = build_block_full(ctx, V, "vovv", (z*)m);
  if (st == CCSD_OK) {
    cudaError_t e = pack_pairs((z*)m, ctx->vovv_pk, ov, ctx->v, 0, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) st = set_err(ctx, CCSD_ERR_CUDA, cudaGetErrorString(e));
  }
  cudaFree(m);
  return st;
}

// W[P(a,b)][P(c,d)] = <ab||cd> packed, from the DF factors (dense (ac|bd) as a temporary).
ccsd_status build_w_df(ccsd_ctx* ctx, const z* B) {
  const int64_t v = ctx->v;
  const int64_t nb = (int64_t)ctx->naux * v * v;
  void *m1 = nullptr, *m2 = nullptr, *mD = nullptr;
  if (cudaMalloc(&m1, nb * sizeof(z)) != cudaSuccess || cudaMalloc(&m2, nb * sizeof(z)) != cudaSuccess ||
      cudaMalloc(&mD, v * v * v * v * sizeof(z)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(m1);
    cudaFree(m2);
    cudaFree(mD);
    return set_err(ctx, CCSD_ERR_OOM, "vvvv build temporaries");
  }
  ccsd_status st = coulomb_df(ctx, B, 'v', 'v', 'v', 'v', (z*)mD, (z*)m1, (z*)m2);
  if (st == CCSD_OK) {
    cudaError_t e = pack_vvvv((z*)mD, ctx->Wpk, v, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) st = set_err(ctx, CCSD_ERR_CUDA, cudaGetErrorString(e));
  }
  cudaFree(m1);
  cudaFree(m2);
  cudaFree(mD);
  return st;
}

// Block of the full integral tensor V[n][n][n][n] for spaces "PQRS".
ccsd_status build_block_full(ccsd_ctx* ctx, const z* V, const char* sp, z* out) {
  const int64_t n = ctx->n;
  int64_t off[4], len[4];
  for (int k = 0; k < 4; ++k) space(ctx, sp[k], off[k], len[k]);
  PermuteArgs a;
  a.rank = 4;
  const int64_t st[4] = {n * n * n, n * n, n, 1};
  int64_t ost = 1;
  for (int k = 3; k >= 0; --k) {
    a.dims[k] = len[k];
    a.istr[k] = st[k];
    a.ostr[k] = ost;
    ost *= len[k];
  }
  a.in = V + off[0] * st[0] + off[1] * st[1] + off[2] * st[2] + off[3];
  a.out = out;
  CK(permute_add(a, ctx->stream));
  return CCSD_OK;
}

// ---------------------------------------------------------------------------
// Particle-particle ladder with <ab||cd> never stored: for blocks of a, rebuild
// D[(a,c)][(b,d)] = (ac|bd) = sum_Q B^Q_ac B^Q_bd for b > a (one GEMM over Q), pack the rows
// <ab||cd> = (ac|bd) - (ad|bc) for a < b, c < d, and contract them at once against tau:
// Lpk[P(ij)][P(ab)] = sum_{c<d} tau^{cd}_{ij} <ab||cd> for those a b columns.
// ---------------------------------------------------------------------------
struct DfBlock {
  int64_t a0, a1, AB0, AB1;
};

std::vector<DfBlock> df_blocks(int64_t v, int64_t blk) {
  std::vector<DfBlock> out;
  for (int64_t a0 = 0; a0 < v - 1; a0 += blk) {
    DfBlock b;
    b.a0 = a0;
    b.a1 = std::min(v - 1, a0 + blk);
    b.AB0 = pair_index(a0, a0 + 1, v);
    b.AB1 = b.a1 >= v - 1 ? pair_count(v) : pair_index(b.a1, b.a1 + 1, v);
    out.push_back(b);
  }
  return out;
}

ccsd_status plan_df_ladder(ccsd_ctx* ctx, Plan* P) {
  const int64_t v = ctx->v, naux = ctx->naux, Po = ctx->Po, Pv = ctx->Pv;
  int64_t blk = ctx->opts.df_block;
  if (blk <= 0) blk = std::max<int64_t>(1, (int64_t)(6e9 / (16.0 * (double)v * v * v)));
  blk = std::min<int64_t>(blk, std::max<int64_t>(v - 1, 1));
  ctx->df_block = (int)blk;
  const auto blocks = df_blocks(v, blk);
  int64_t dmax = 0, wmax = 0;
  for (const auto& b : blocks) {
    dmax = std::max(dmax, (b.a1 - b.a0) * v * (v - b.a0 - 1) * v);
    wmax = std::max(wmax, b.AB1 - b.AB0);
  }
  // D and the packed rows live at the start of the plan's scratch region (set once it exists):
  // no temporary of the plan is live while the ladder op runs
  ctx->df_w_off = (dmax + 15) / 16 * 16;
  P->reserve_scratch(ctx->df_w_off + wmax * Pv);
  if (ctx->use_split) {
    // B^Q_vv is constant: its digits (rows (a, c), K = Q) are cut once; every block's rebuild
    // reads row ranges of them
    uint8_t* m = nullptr;
    CS(dalloc(ctx, &m, slice_bytes(v * v, naux, ctx->split)));
    CK(make_slices(ctx->Bvv, v * v, naux, v * v, 1, 0, ctx->split, ctx->Bsl, m, ctx->stream));
  }
  // GEMM shapes of the blocks, for the workspace peaks
  for (const auto& b : blocks) {
    ZGemmArgs gd;
    gd.M = (b.a1 - b.a0) * v;
    gd.N = (v - b.a0 - 1) * v;
    gd.K = naux;
    if (ctx->use_split) P->note_aux_bytes(split_part_bytes(gd.M, gd.N, gd.K, ctx->split));
    else P->note_gemm(gd);
    ZGemmArgs gl;
    gl.M = Po;
    gl.N = b.AB1 - b.AB0;
    gl.K = Pv;
    gl.transB = 1;
    if (ctx->use_split)
      P->note_aux_bytes(slice_bytes(gl.N, Pv, ctx->split) + split_part_bytes(Po, gl.N, Pv, ctx->split));
    else
      P->note_gemm(gl);
  }
  if (ctx->use_split) {
    uint8_t* m = nullptr;
    CS(dalloc(ctx, &m, slice_bytes(Po, Pv, ctx->split)));
    ctx->tausl_mem = m;
  }
  const double fl = 8.0 * (double)Po * (double)Pv * (double)Pv;
  P->custom("ladder:gemm", [ctx, blocks, v, naux, Po, Pv](cudaStream_t s) {
    const GemmFn& gemm = ctx->plan->gemm_fn();
    cudaError_t e = cudaSuccess;
    if (ctx->use_split)
      e = make_slices(ctx->tau_pk, Po, Pv, Pv, 0, 0, ctx->split, ctx->tausl, ctx->tausl_mem, s);
    for (const auto& b : blocks) {
      if (e != cudaSuccess) break;
      ZGemmArgs gd;  // D[(a,c)][(b,d)] = sum_Q B^Q_{ac} B^Q_{bd}, a in [a0, a1), b > a0
      gd.M = (b.a1 - b.a0) * v;
      gd.N = (v - b.a0 - 1) * v;
      gd.K = naux;
      gd.A = ctx->Bvv + b.a0 * v;
      gd.lda = v * v;
      gd.transA = 1;
      gd.B = ctx->Bvv + (b.a0 + 1) * v;
      gd.ldb = v * v;
      gd.C = ctx->Dblk;
      gd.ldc = gd.N;
      if (ctx->use_split)
        e = split_gemm(slice_rows(ctx->Bsl, b.a0 * v, gd.M), slice_rows(ctx->Bsl, (b.a0 + 1) * v, gd.N), gd.C,
                       gd.ldc, zmake(1, 0), zmake(0, 0), ctx->split_err, ctx->split_ws,
                       split_part_bytes(gd.M, gd.N, gd.K, ctx->split), s);
      else
        e = gemm(gd, s);
      if (e == cudaSuccess) e = pack_vvvv_rows(ctx->Dblk, ctx->Wblk, v, b.a0, b.a1, s);
      const int64_t nb = b.AB1 - b.AB0;
      if (e != cudaSuccess || nb <= 0) continue;
      if (ctx->use_split) {
        SliceSet SW;
        uint8_t* w = static_cast<uint8_t*>(ctx->split_ws);
        e = make_slices(ctx->Wblk, nb, Pv, Pv, 0, 0, ctx->split, SW, w, s);
        if (e == cudaSuccess)
          e = split_gemm(ctx->tausl, SW, ctx->Lpk + b.AB0, Pv, zmake(1, 0), zmake(0, 0), ctx->split_err,
                         w + slice_bytes(nb, Pv, ctx->split), split_part_bytes(Po, nb, Pv, ctx->split), s);
      } else {
        ZGemmArgs gl;  // Lpk[:, AB0:AB1] = tau_pk W_blk^T
        gl.M = Po;
        gl.N = nb;
        gl.K = Pv;
        gl.A = ctx->tau_pk;
        gl.lda = Pv;
        gl.B = ctx->Wblk;
        gl.ldb = Pv;
        gl.transB = 1;
        gl.C = ctx->Lpk + b.AB0;
        gl.ldc = Pv;
        e = gemm(gl, s);
      }
    }
    return e;
  }, fl);
  return CCSD_OK;
}

// ---------------------------------------------------------------------------
// Split GEMMs of the plan in chunks: the digits of both operands of one call are held to a
// budget (a quarter of the device memory free when the plan is made, 4 to 8 GB) by cutting
// M, N (whole 128-row tiles) and, where a single row tile is still too long, K (each K chunk
// is a GEMM of its own, with its own scales, accumulated in FP64).
// ---------------------------------------------------------------------------
int64_t split_call_budget() {
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    free_b = 0;
  }
  const int64_t lo = int64_t(4) << 30, hi = int64_t(8) << 30;
  return std::min(hi, std::max(lo, (int64_t)(free_b / 4)));
}

struct SplitChunks {
  int64_t mc, nc, kc;
};

SplitChunks split_chunks(int64_t M, int64_t N, int64_t K, const SplitConfig& c, int64_t budget) {
  SplitChunks ch{std::max<int64_t>(M, 1), std::max<int64_t>(N, 1), std::max<int64_t>(K, 1)};
  auto half = [](int64_t x) { return std::max<int64_t>(128, (x / 2 + 127) / 128 * 128); };
  for (int guard = 0; guard < 200; ++guard) {
    const int64_t ba = slice_bytes(ch.mc, ch.kc, c), bb = slice_bytes(ch.nc, ch.kc, c);
    if (ba + bb <= budget) break;
    if (ba >= bb && ch.mc > 128) ch.mc = half(ch.mc);
    else if (ch.nc > 128) ch.nc = half(ch.nc);
    else if (ch.mc > 128) ch.mc = half(ch.mc);
    else if (ch.kc > 128) ch.kc = half(ch.kc);
    else break;
  }
  return ch;
}

// Largest K-split partial buffer over the chunk shapes (full and tail chunks).
int64_t split_chunk_part_bytes(int64_t M, int64_t N, int64_t K, const SplitChunks& ch, const SplitConfig& c) {
  int64_t best = 0;
  for (int64_t m : {ch.mc, M % ch.mc})
    for (int64_t n : {ch.nc, N % ch.nc})
      for (int64_t k : {ch.kc, K % ch.kc})
        if (m > 0 && n > 0 && k > 0) best = std::max(best, split_part_bytes(m, n, k, c));
  return best;
}

int64_t split_chunked_bytes(int64_t M, int64_t N, int64_t K, const SplitConfig& c, int64_t budget) {
  const SplitChunks ch = split_chunks(M, N, K, c, budget);
  return slice_bytes(ch.mc, ch.kc, c) + slice_bytes(ch.nc, ch.kc, c) + split_chunk_part_bytes(M, N, K, ch, c);
}

cudaError_t split_gemm_chunked(ccsd_ctx* ctx, const ZGemmArgs& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  if (g.K <= 0) return zscale_matrix(g, s);
  const SplitConfig& c = ctx->split;
  const SplitChunks ch = split_chunks(g.M, g.N, g.K, c, ctx->split_budget);
  uint8_t* w = static_cast<uint8_t*>(ctx->split_ws);
  uint8_t* wb = w + slice_bytes(ch.mc, ch.kc, c);
  uint8_t* part = wb + slice_bytes(ch.nc, ch.kc, c);
  const int64_t part_bytes = split_chunk_part_bytes(g.M, g.N, g.K, ch, c);
  const int64_t nm = (g.M + ch.mc - 1) / ch.mc, nn = (g.N + ch.nc - 1) / ch.nc;
  // slice the operand with fewer chunks in the outer loop: the inner one is re-cut per outer chunk
  const bool m_outer = nm <= nn;
  cudaError_t e = cudaSuccess;
  for (int64_t k0 = 0; k0 < g.K && e == cudaSuccess; k0 += ch.kc) {
    const int64_t kn = std::min(ch.kc, g.K - k0);
    const z beta = k0 == 0 ? g.beta : zmake(1, 0);
    auto slice_a = [&](int64_t m0, int64_t mn, SliceSet& SA) {
      const z* A = g.transA ? g.A + k0 * g.lda + m0 : g.A + m0 * g.lda + k0;
      return make_slices(A, mn, kn, g.lda, g.transA, g.conjA, c, SA, w, s);
    };
    auto slice_b = [&](int64_t n0, int64_t nnn, SliceSet& SB) {
      const z* B = g.transB ? g.B + n0 * g.ldb + k0 : g.B + k0 * g.ldb + n0;
      return make_slices(B, nnn, kn, g.ldb, g.transB ? 0 : 1, g.conjB, c, SB, wb, s);
    };
    const int64_t outer_n = m_outer ? nm : nn, inner_n = m_outer ? nn : nm;
    for (int64_t oi = 0; oi < outer_n && e == cudaSuccess; ++oi) {
      SliceSet SA, SB;
      const int64_t m0o = oi * ch.mc, n0o = oi * ch.nc;
      e = m_outer ? slice_a(m0o, std::min(ch.mc, g.M - m0o), SA) : slice_b(n0o, std::min(ch.nc, g.N - n0o), SB);
      for (int64_t ii = 0; ii < inner_n && e == cudaSuccess; ++ii) {
        const int64_t m0 = m_outer ? m0o : ii * ch.mc, n0 = m_outer ? ii * ch.nc : n0o;
        e = m_outer ? slice_b(n0, std::min(ch.nc, g.N - n0), SB) : slice_a(m0, std::min(ch.mc, g.M - m0), SA);
        if (e == cudaSuccess)
          e = split_gemm(SA, SB, g.C + m0 * g.ldc + n0, g.ldc, g.alpha, beta, ctx->split_err, part, part_bytes, s);
      }
    }
  }
  return e;
}

// ---------------------------------------------------------------------------
// The residual plan: Appendix A, one contraction per printed term.
// Labels i,j,k,l run over occupied and a,b,c,d over virtual spinors.
// ---------------------------------------------------------------------------
// Constant operands (integral blocks) of up to this size keep a permuted copy for the plan
// (opts.permute_cache_limit, default 2 GiB); larger ones (oovv from o60/v400 on: 9.2 GB) are
// permuted into the plan's scratch at each use, one more HBM pass per use instead of a resident copy.
int64_t cache_limit_bytes(const ccsd_opts& o) {
  if (o.permute_cache_limit < 0.0) return -1;
  return o.permute_cache_limit > 0.0 ? (int64_t)o.permute_cache_limit : int64_t(2) << 30;
}

// The GEMM back end of a plan: split precision where ctx->routes_split says so, else the FP64 DMMA
// kernel with the context's split-K workspace.
void set_plan_gemm(ccsd_ctx* ctx, Plan* P) {
  const std::function<bool(const ZGemmArgs&)> to_split = ctx->routes_split;
  P->set_gemm(
      [ctx, to_split](const ZGemmArgs& g, cudaStream_t s) {
        if (to_split(g)) return split_gemm_chunked(ctx, g, s);
        ZGemmArgs h = g;
        h.ws = ctx->gemm_ws;
        h.ws_elems = ctx->gemm_ws_elems;
        h.mult4 = ctx->opts.complex_4m;
        return zgemm_f64(h, s, h.cfg);
      },
      [to_split](const ZGemmArgs& g) { return to_split(g) ? (int64_t)0 : zgemm_f64_workspace(g); },
      [ctx, to_split](const ZGemmArgs& g) {
        return to_split(g) ? split_chunked_bytes(g.M, g.N, g.K, ctx->split, ctx->split_budget) : 0;
      });
}

ccsd_status build_residual_plan(ccsd_ctx* ctx) {
  const int o = ctx->o, v = ctx->v;
  // CC2: the singles of Appendix A with their intermediates tau, H^a_c, H^k_i, H^k_c, and the CC2
  // doubles; the CCSD-only intermediates and doubles terms are not planned
  const bool cc2 = ctx->opts.method == CCSD_METHOD_CC2;
  // CCD: the doubles equations at T1 = 0. Every term with a t1 factor vanishes, and so does every
  // term that only feeds one (C^{kb}_{ij} enters S2 only through C t1; S1 is not solved): the
  // plan leaves them out and writes S1 = 0, whatever t1 holds
  const bool ccd = ctx->opts.method == CCSD_METHOD_CCD;
  const double t1f = ccd ? 0.0 : 1.0;  // weight of the t1 t1 products in tau and X
  const int64_t Po = ctx->Po, Pv = ctx->Pv;
  // rows a of <ak||cd> unpacked at a time for the H^{ak}_{ci} term (at most about 1 GB)
  ctx->vblk_rows = ctx->opts.vovv_block > 0
                       ? std::min<int64_t>(v, ctx->opts.vovv_block)
                       : std::max<int64_t>(1, std::min<int64_t>(v, (int64_t)(1.0e9 / (16.0 * o * (double)v * v))));
  if (!cc2) CS(dalloc(ctx, &ctx->vblk, ctx->vblk_rows * o * (int64_t)v * v));
  Plan* P = new Plan(o, v, &ctx->scratch, ctx->stream);
  P->set_cache_limit(cache_limit_bytes(ctx->opts));
  ctx->plan = P;
  // In split mode a single GEMM of at least split_min_flops goes to the tensor-core digit
  // path when its modelled time beats the FP64 path (measured on this chip: 1.3e12 of the
  // conventional 8 flops per complex multiply-add per second with 3M products, 0.95e12 with
  // 4M); with split_min_flops <= 0 every GEMM goes there.
  const double fp64_rate = ctx->opts.complex_4m ? 0.95e12 : 1.3e12;
  auto to_split = [ctx, fp64_rate](const ZGemmArgs& g) {
    if (!ctx->use_split || g.batch != 1) return false;
    const double fl = 8.0 * (double)g.M * (double)g.N * (double)g.K;
    if (ctx->split_min_flops <= 0.0) return true;
    return fl >= ctx->split_min_flops && split_cost_estimate(g.M, g.N, g.K, ctx->split) < fl / fp64_rate;
  };
  ctx->routes_split = to_split;
  if (ctx->use_split)
    ctx->split_budget = ctx->opts.split_budget > 0.0 ? (int64_t)ctx->opts.split_budget : split_call_budget();
  set_plan_gemm(ctx, P);
  const z one = zmake(1, 0), mone = zmake(-1, 0), half = zmake(0.5, 0);
  auto V = [&](z* p, const char* lab) { return P->view(p, lab, true); };
  auto W = [&](z* p, const char* lab) { return P->view(p, lab, false); };

  // tau^{ab}_{ij} = t^{ab}_{ij} + P^-_ij (t^a_i t^b_j), and its (i<j, c<d) packed copy
  // R (o^2 v^2) hosts, in turn: X of the H^{ak}_{ci} term, the ring product, the products of the
  // goo, vt1 (packed), gvv and ct1 terms before their antisymmetrisation, and tau packed over
  // (c<d) for S1 (their lifetimes do not overlap)
  z *t1 = ctx->t1, *t2 = ctx->t2, *tau = ctx->tau, *taupk = ctx->tau_pk, *X = ctx->R;
  P->custom("tau", [=](cudaStream_t s) {
    cudaError_t e = tau_build(t1, t2, tau, o, v, 1.0, t1f, 1, s);
    if (e != cudaSuccess) return e;
    return pack_pairs(tau, taupk, o, v, 1, s);
  });
  if (!cc2) {
    // X^{ad}_{li} = 1/2 t^{ad}_{li} + t^a_l t^d_i (the pair amplitude of the H^{ak}_{ci} term), stored
    // X[i][a][l][d]: the [free][summed] layout its GEMM reads without a permutation
    P->custom("Hvoov", [=](cudaStream_t s) { return tau_build(t1, t2, X, o, v, 0.5, t1f, 0, s, 1); });
  }

  // H^a_c = F^a_c + 1/2 sum_kld V^{kl}_{cd} tau^{da}_{kl}
  P->add("Hvv", W(ctx->Hvv, "ac"), one, V(ctx->fvv, "ac"), false, 0.0);
  P->contract("Hvv", W(ctx->Hvv, "ac"), half, V(ctx->oovv, "klcd"), false, W(tau, "klda"), false, 1.0);
  if (!cc2 && !ccd) {
    // T[i][a][k][c] = sum_d V^{ak}_{cd} t^d_i (the second term of H^{ak}_{ci}) first, into Hr: the rows of
    // <ak||cd> are unpacked from vovv_pk block by block of a (the dense vovv is never stored) and each
    // block is one GEMM writing the columns (a, k, c) of its a range in every row i.
    {
      const int64_t vb = ctx->vblk_rows, Pv_ = Pv;
      for (int64_t a0 = 0; a0 < v; a0 += vb) {
        ZGemmArgs g;
        g.M = o;
        g.N = std::min<int64_t>(vb, v - a0) * o * v;
        g.K = v;
        g.transB = 1;
        P->note_gemm(g);
      }
      z *vpk = ctx->vovv_pk, *vblk = ctx->vblk, *hr = ctx->Hr;
      const int64_t nblk = (v + vb - 1) / vb;
      bool cached = false;
      if (ctx->use_split) {
        // <ak||cd> is constant: cut the digits of its unpacked rows once, block by block, when
        // they take at most a tenth of the free device memory (and 16 GB)
        int64_t total = slice_bytes(o, v, ctx->split);
        for (int64_t a0 = 0; a0 < v; a0 += vb) total += slice_bytes(std::min<int64_t>(vb, v - a0) * o * v, v, ctx->split);
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
          cudaGetLastError();
          fr = 0;
        }
        if (total <= std::min<int64_t>(int64_t(16) << 30, (int64_t)(fr / 10))) {
          ctx->vovv_sl.resize(nblk);
          for (int64_t b = 0; b < nblk; ++b) {
            const int64_t a0 = b * vb, na = std::min<int64_t>(vb, v - a0);
            uint8_t* m = nullptr;
            CS(dalloc(ctx, &m, slice_bytes(na * o * v, v, ctx->split)));
            UnpackArgs u;  // vblk[(a - a0, k)][c][d] = <ak||cd>
            u.in = vpk + a0 * o * Pv_;
            u.out = vblk;
            u.n1 = na * o;
            u.n2 = v;
            u.beta = 0.0;
            CK(unpack_pairs(u, ctx->stream));
            CK(make_slices(vblk, na * o * v, v, v, 0, 0, ctx->split, ctx->vovv_sl[b], m, ctx->stream));
          }
          CS(dalloc(ctx, &ctx->t1sl_mem, slice_bytes(o, v, ctx->split)));
          cached = true;
        }
      }
      if (cached) {
        P->custom("Hvoov:gemm", [ctx, o, v, vb, nblk, hr, t1](cudaStream_t s) {
          SliceSet ST;  // Hr[i][(a,k,c)] = sum_d t1[i][d] <ak||cd>, block by block of a
          cudaError_t e = make_slices(t1, o, v, v, 0, 0, ctx->split, ST, ctx->t1sl_mem, s);
          for (int64_t b = 0; b < nblk && e == cudaSuccess; ++b)
            e = split_gemm(ST, ctx->vovv_sl[b], hr + b * vb * o * v, (int64_t)v * o * v, zmake(1, 0), zmake(0, 0),
                           ctx->split_err, nullptr, 0, s);
          return e;
        }, 8.0 * o * (double)v * o * v * v);
      } else {
      P->custom("Hvoov:gemm", [ctx, o, v, vb, Pv_, vpk, vblk, hr, t1](cudaStream_t s) {
        const GemmFn& gemm = ctx->plan->gemm_fn();
        cudaError_t e = cudaSuccess;
        for (int64_t a0 = 0; a0 < v && e == cudaSuccess; a0 += vb) {
          const int64_t na = std::min<int64_t>(vb, v - a0);
          UnpackArgs u;  // vblk[(a - a0, k)][c][d] = <ak||cd>
          u.in = vpk + a0 * o * Pv_;
          u.out = vblk;
          u.n1 = na * o;
          u.n2 = v;
          u.beta = 0.0;
          e = unpack_pairs(u, s);
          if (e != cudaSuccess) break;
          ZGemmArgs g;  // Hr[i][(a,k,c)] = sum_d t1[i][d] vblk[(a,k,c)][d]
          g.M = o;
          g.N = na * o * v;
          g.K = v;
          g.A = t1;
          g.lda = v;
          g.B = vblk;
          g.ldb = v;
          g.transB = 1;
          g.C = hr + a0 * o * v;
          g.ldc = (int64_t)v * o * v;
          e = gemm(g, s);
        }
        return e;
      }, 8.0 * o * (double)v * o * v * v);
      }
    }
    // G^a_c = H^a_c + sum_kd V^{ak}_{cd} t^d_k - sum_k F^k_c t^a_k; the middle term is the trace
    // sum_k T[k][a][k][c] of the product above
    P->add("Gvv", W(ctx->Gvv, "ac"), one, W(ctx->Hvv, "ac"), false, 0.0);
    {
      z *hr = ctx->Hr, *gvv = ctx->Gvv;
      P->custom("Gvv", [=](cudaStream_t s) { return trace_ik(hr, o, v, gvv, 1.0, 1.0, s); });
    }
    P->contract("Gvv", W(ctx->Gvv, "ac"), mone, V(ctx->fov, "kc"), false, W(t1, "ka"), false, 1.0);
  } else if (ccd) {
    P->add("Gvv", W(ctx->Gvv, "ac"), one, W(ctx->Hvv, "ac"), false, 0.0);  // G^a_c = H^a_c at T1 = 0
  }
  // H^k_i = -F^k_i + 1/2 sum_lcd V^{kl}_{cd} tau^{cd}_{li}
  P->add("Hoo", W(ctx->Hoo, "ki"), mone, V(ctx->foo, "ki"), false, 0.0);
  P->contract("Hoo", W(ctx->Hoo, "ki"), half, V(ctx->oovv, "klcd"), false, W(tau, "licd"), false, 1.0);
  if (!cc2) {
    // G^k_i = H^k_i - sum_lc V^{kl}_{ic} t^c_l - sum_c F^k_c t^c_i
    P->add("Goo", W(ctx->Goo, "ki"), one, W(ctx->Hoo, "ki"), false, 0.0);
    if (!ccd) {
      P->contract("Goo", W(ctx->Goo, "ki"), mone, V(ctx->ooov, "klic"), false, W(t1, "lc"), false, 1.0);
      P->contract("Goo", W(ctx->Goo, "ki"), mone, V(ctx->fov, "kc"), false, W(t1, "ic"), false, 1.0);
    }
  }
  // H^k_c = F^k_c + sum_ld V^{kl}_{cd} t^d_l (it feeds S1 only: not needed in CCD)
  if (!ccd) {
    P->add("Hov", W(ctx->Hov, "kc"), one, V(ctx->fov, "kc"), false, 0.0);
    P->contract("Hov", W(ctx->Hov, "kc"), one, V(ctx->oovv, "klcd"), false, W(t1, "ld"), false, 1.0);
  }
  if (!cc2) {
    // H^{ak}_{ci} (stored [i][a][k][c]) = V^{ak}_{ci} + sum_d V^{ak}_{cd} t^d_i - sum_l V^{kl}_{ic} t^a_l
    //                                   + sum_ld V^{kl}_{cd} (1/2 t^{ad}_{li} + t^a_l t^d_i)
    // (in CCD the t1 terms are absent and V^{ak}_{ci} starts Hr)
    P->add("Hvoov", W(ctx->Hr, "iakc"), one, V(ctx->J, "iakc"), false, ccd ? 0.0 : 1.0);
    if (!ccd)
      P->contract("Hvoov", W(ctx->Hr, "iakc"), mone, V(ctx->ooov, "klic"), false, W(t1, "la"), false, 1.0);
    P->contract("Hvoov", W(ctx->Hr, "iakc"), one, W(X, "iald"), false, V(ctx->oovv, "klcd"), false, 1.0);
  }
  if (!cc2 && !ccd) {
    // C^{kb}_{ij} = V^{ij+}_{kb} + P^-_ij sum_c V^{bk}_{ci} t^c_j - 1/2 sum_cd V^{bk}_{cd} tau^{cd}_{ij}
    // V^{ij+}_{kb} = conj(<ij||kb>), read from ooov[i][j][k][b] with the permutation of the add
    P->add("C", W(ctx->C, "kbij"), one, V(ctx->ooov, "ijkb"), true, 0.0);
    // Yovoo[i][b][k][j] = sum_c V^{bk}_{ci} t^c_j = sum_c J[i][b][k][c] t^c_j
    P->contract("C", W(ctx->Yovoo, "ibkj"), one, V(ctx->J, "ibkc"), false, W(t1, "jc"), false, 0.0);
    P->add("C", W(ctx->C, "kbij"), one, W(ctx->Yovoo, "ibkj"), false, 1.0);
    P->add("C", W(ctx->C, "kbij"), mone, W(ctx->Yovoo, "jbki"), false, 1.0);
    {
      ZGemmArgs g;  // Ypk[(b,k)][P(ij)] = sum_{c<d} V^{bk}_{cd} tau^{cd}_{ij}
      g.M = (int64_t)v * o;
      g.N = Po;
      g.K = Pv;
      g.A = ctx->vovv_pk;
      g.lda = Pv;
      g.B = taupk;
      g.ldb = Pv;
      g.transB = 1;
      g.C = ctx->Ypk;
      g.ldc = Po;
      P->gemm("C:gemm", g);
      z *ypk = ctx->Ypk, *yf = ctx->Yfull;
      P->custom("C:unpack", [=](cudaStream_t s) {
        UnpackArgs u;
        u.in = ypk;
        u.out = yf;
        u.n1 = (int64_t)v * o;
        u.n2 = o;
        u.alpha = mone;
        u.beta = 0.0;
        return unpack_pairs(u, s);
      });
      P->add("C", W(ctx->C, "kbij"), one, W(ctx->Yfull, "bkij"), false, 1.0);
    }
  }
  if (!cc2) {
    // A^{kl}_{ij} = V^{kl}_{ij} + P^-_ij sum_c V^{kl}_{ic} t^c_j + 1/2 sum_cd V^{kl}_{cd} tau^{cd}_{ij}
    P->add("A", W(ctx->Afull, "klij"), one, V(ctx->oooo, "klij"), false, 0.0);
    if (!ccd) {
      P->contract("A", W(ctx->Yoooo, "klij"), one, V(ctx->ooov, "klic"), false, W(t1, "jc"), false, 0.0);
      P->add("A", W(ctx->Afull, "klij"), one, W(ctx->Yoooo, "klij"), false, 1.0);
      P->add("A", W(ctx->Afull, "klij"), mone, W(ctx->Yoooo, "klji"), false, 1.0);
    }
    {
      z *af = ctx->Afull, *apk = ctx->Apk;
      P->custom("A:pack", [=](cudaStream_t s) { return pack_pairs(af, apk, o, o, 1, s); });
      ZGemmArgs g;  // Apk[P(kl)][P(ij)] += sum_{c<d} V^{kl}_{cd} tau^{cd}_{ij}
      g.M = Po;
      g.N = Po;
      g.K = Pv;
      g.A = ctx->oovv_pk;
      g.lda = Pv;
      g.B = taupk;
      g.ldb = Pv;
      g.transB = 1;
      g.C = ctx->Apk;
      g.ldc = Po;
      g.beta = one;
      P->gemm("A:gemm", g);
    }

    // S^{ab}_{ij}: driver V^{ij+}_{ab}
    P->add("driver", W(ctx->S2, "ijab"), one, V(ctx->oovv, "ijab"), true, 0.0);
    // ring: sum_kc P^-_ij P^-_ab (H^{ak}_{ci} t^{cb}_{jk}),  R[i][a][j][b] = sum_kc H^{ak}_{ci} t^{cb}_{jk}
    P->contract("ring", W(ctx->R, "iajb"), one, W(ctx->Hr, "iakc"), false, W(t2, "jkcb"), false, 0.0);
    P->add("ring", W(ctx->S2, "ijab"), one, W(ctx->R, "iajb"), false, 1.0);
    P->add("ring", W(ctx->S2, "ijab"), mone, W(ctx->R, "jaib"), false, 1.0);
    P->add("ring", W(ctx->S2, "ijab"), mone, W(ctx->R, "ibja"), false, 1.0);
    P->add("ring", W(ctx->S2, "ijab"), one, W(ctx->R, "jbia"), false, 1.0);
    // sum_k P^-_ji G^k_j t^{ab}_{ik}:  W1[j][i][a][b] = sum_k G^k_j t^{ab}_{ik}
    P->contract("goo", W(ctx->R, "jiab"), one, W(ctx->Goo, "kj"), false, W(t2, "ikab"), false, 0.0);
    P->add("goo", W(ctx->S2, "ijab"), one, W(ctx->R, "jiab"), false, 1.0);
    P->add("goo", W(ctx->S2, "ijab"), mone, W(ctx->R, "ijab"), false, 1.0);
    // sum_c P^-_ij (V^{cj+}_{ab} t^c_i):  W1[i][j][a][b] = sum_c t^c_i conj(V^{cj}_{ab}); (a, b) is the
    // antisymmetric pair of both, so the product is formed packed, straight from vovv_pk
    // (W1pk[i][(j, P(a,b))] in R) and added to S2 with (i, j) antisymmetrised in one pass
    if (!ccd) {
      ZGemmArgs g;
      g.M = o;
      g.N = (int64_t)o * Pv;
      g.K = v;
      g.A = t1;
      g.lda = v;
      g.B = ctx->vovv_pk;
      g.ldb = (int64_t)o * Pv;
      g.conjB = 1;
      g.C = ctx->R;
      g.ldc = (int64_t)o * Pv;
      P->gemm("vt1:gemm", g);
      z *w1pk = ctx->R, *s2 = ctx->S2;
      P->custom("vt1", [=](cudaStream_t s) {
        UnpackArgs u;  // S2[i][j][a][b] += W1[i][j][a][b] - W1[j][i][a][b]
        u.in = w1pk;
        u.out = s2;
        u.n1 = (int64_t)o * o;
        u.n2 = v;
        u.anti_rows = o;
        u.beta = 1.0;
        return unpack_pairs(u, s);
      });
    }
    // sum_c P^-_ab G^a_c t^{cb}_{ij}:  W1[a][i][j][b] = sum_c G^a_c t^{cb}_{ij}
    P->contract("gvv", W(ctx->R, "aijb"), one, W(ctx->Gvv, "ac"), false, W(t2, "ijcb"), false, 0.0);
    P->add("gvv", W(ctx->S2, "ijab"), one, W(ctx->R, "aijb"), false, 1.0);
    P->add("gvv", W(ctx->S2, "ijab"), mone, W(ctx->R, "bija"), false, 1.0);
    // sum_k P^-_ab (C^{ka}_{ij} t^b_k):  W1[a][i][j][b] = sum_k C^{ka}_{ij} t^b_k
    if (!ccd) {
      P->contract("ct1", W(ctx->R, "aijb"), one, W(ctx->C, "kaij"), false, W(t1, "kb"), false, 0.0);
      P->add("ct1", W(ctx->S2, "ijab"), one, W(ctx->R, "aijb"), false, 1.0);
      P->add("ct1", W(ctx->S2, "ijab"), mone, W(ctx->R, "bija"), false, 1.0);
    }
    // 1/2 sum_kl A^{kl}_{ij} tau^{ab}_{kl}  (packed: sum_{k<l})
    {
      ZGemmArgs g;  // Hpk[P(ij)][P(ab)] = sum_{k<l} A^{kl}_{ij} tau^{ab}_{kl}
      g.M = Po;
      g.N = Pv;
      g.K = Po;
      g.A = ctx->Apk;
      g.lda = Po;
      g.transA = 1;
      g.B = taupk;
      g.ldb = Pv;
      g.C = ctx->Hpk;
      g.ldc = Pv;
      P->gemm("hole:gemm", g);
      z *hpk = ctx->Hpk, *s2 = ctx->S2;
      P->custom("hole:unpack", [=](cudaStream_t s) {
        UnpackArgs u;
        u.in = hpk;
        u.out = s2;
        u.n1 = o;
        u.n2 = v;
        u.unpack_rows = 1;
        return unpack_pairs(u, s);
      });
    }
    // particle-particle ladder 1/2 sum_cd V^{ab}_{cd} tau^{cd}_{ij}  (packed: sum_{c<d})
    {
      ZGemmArgs g;  // Lpk[P(ij)][P(ab)] = sum_{c<d} tau^{cd}_{ij} <ab||cd>
      g.M = Po;
      g.N = Pv;
      g.K = Pv;
      g.A = taupk;
      g.lda = Pv;
      g.B = ctx->Wpk;
      g.ldb = Pv;
      g.transB = 1;
      g.C = ctx->Lpk;
      g.ldc = Pv;
      if (!ctx->opts.store_w) {
        CS(plan_df_ladder(ctx, P));
      } else if (ctx->use_split) {
        // W digits were cut once at creation; only tau is sliced per evaluation
        P->note_aux_bytes(slice_bytes(Po, Pv, ctx->split) + split_part_bytes(Po, Pv, Pv, ctx->split));
        z* lpk = ctx->Lpk;
        P->custom("ladder:gemm", [ctx, taupk, lpk, Po, Pv](cudaStream_t s) {
          cudaError_t e = make_slices(taupk, Po, Pv, Pv, 0, 0, ctx->split, ctx->tausl, ctx->split_ws, s);
          uint8_t* part = static_cast<uint8_t*>(ctx->split_ws) + slice_bytes(Po, Pv, ctx->split);
          if (e == cudaSuccess)
            e = split_gemm(ctx->tausl, ctx->Wsl, lpk, Pv, zmake(1, 0), zmake(0, 0), ctx->split_err, part,
                           split_part_bytes(Po, Pv, Pv, ctx->split), s);
          return e;
        }, 8.0 * (double)Po * (double)Pv * (double)Pv);
      } else {
        P->gemm("ladder:gemm", g);
      }
      z *lpk = ctx->Lpk, *s2 = ctx->S2;
      P->custom("ladder:unpack", [=](cudaStream_t s) {
        UnpackArgs u;
        u.in = lpk;
        u.out = s2;
        u.n1 = o;
        u.n2 = v;
        u.unpack_rows = 1;
        return unpack_pairs(u, s);
      });
    }
  } else {
    // CC2 doubles: S^{ab}_{ij} = <ab||ij>~ + P^-_ab sum_e f_be t^{ae}_{ij} - P^-_ij sum_m f_mj t^{ab}_{im},
    // <ab||ij>~ = (ai|bj)~ - (aj|bi)~ over the T1-dressed factors Bt^Q = ((1 - t1) B^Q (1 + t1))_vo:
    //   Bt[Q] = B_vo + B_vv t1^T - t1^T (B_oo + B_ov t1^T)
    // (one batched GEMM over Q per product; the appendix's W intermediates expanded in t1 are the
    // same integral)
    const int64_t nq = ctx->naux;
    z *bvo = ctx->c2_Bvo, *bvv = ctx->Bvv, *boo = ctx->c2_Boo, *bov = ctx->c2_Bov, *bt = ctx->c2_Bt,
      *dt = ctx->c2_Dt;
    const int m4 = ctx->opts.complex_4m;
    P->custom("cc2:dress", [=](cudaStream_t s) {
      cudaError_t e = cudaMemcpyAsync(bt, bvo, sizeof(z) * nq * v * o, cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(dt, boo, sizeof(z) * nq * o * o, cudaMemcpyDeviceToDevice, s);
      ZGemmArgs g;  // Bt[Q][a][i] += sum_b B_vv[Q][a][b] t^b_i
      g.M = v;
      g.N = o;
      g.K = v;
      g.batch = (int)nq;
      g.A = bvv;
      g.lda = v;
      g.sA = (int64_t)v * v;
      g.B = t1;
      g.ldb = v;
      g.transB = 1;
      g.C = bt;
      g.ldc = o;
      g.sC = (int64_t)v * o;
      g.beta = one;
      g.mult4 = m4;
      if (e == cudaSuccess) e = zgemm_f64(g, s);
      ZGemmArgs h;  // Dt[Q][j][i] += sum_b B_ov[Q][j][b] t^b_i
      h.M = o;
      h.N = o;
      h.K = v;
      h.batch = (int)nq;
      h.A = bov;
      h.lda = v;
      h.sA = (int64_t)o * v;
      h.B = t1;
      h.ldb = v;
      h.transB = 1;
      h.C = dt;
      h.ldc = o;
      h.sC = (int64_t)o * o;
      h.beta = one;
      h.mult4 = m4;
      if (e == cudaSuccess) e = zgemm_f64(h, s);
      ZGemmArgs u;  // Bt[Q][a][i] -= sum_j t^a_j Dt[Q][j][i]
      u.M = v;
      u.N = o;
      u.K = o;
      u.batch = (int)nq;
      u.A = t1;
      u.lda = v;
      u.transA = 1;
      u.B = dt;
      u.ldb = o;
      u.sB = (int64_t)o * o;
      u.C = bt;
      u.ldc = o;
      u.sC = (int64_t)v * o;
      u.alpha = mone;
      u.beta = one;
      u.mult4 = m4;
      if (e == cudaSuccess) e = zgemm_f64(u, s);
      return e;
    }, 8.0 * (double)nq * ((double)v * o * v + (double)o * o * v + (double)v * o * o));
    {
      ZGemmArgs g;  // R[a][i][b][j] = (ai|bj)~ = sum_Q Bt[Q][a][i] Bt[Q][b][j]
      g.M = (int64_t)v * o;
      g.N = (int64_t)v * o;
      g.K = nq;
      g.A = bt;
      g.lda = (int64_t)v * o;
      g.transA = 1;
      g.B = bt;
      g.ldb = (int64_t)v * o;
      g.C = ctx->R;
      g.ldc = (int64_t)v * o;
      P->gemm("cc2:J", g);
    }
    P->add("cc2:driver", W(ctx->S2, "ijab"), one, W(ctx->R, "aibj"), false, 0.0);
    P->add("cc2:driver", W(ctx->S2, "ijab"), mone, W(ctx->R, "ajbi"), false, 1.0);
    // sum_e P^-_ab f_be t^{ae}_{ij}
    P->contract("cc2:fvv", W(ctx->R, "ijab"), one, W(t2, "ijae"), false, V(ctx->fvv, "be"), false, 0.0);
    P->add("cc2:fvv", W(ctx->S2, "ijab"), one, W(ctx->R, "ijab"), false, 1.0);
    P->add("cc2:fvv", W(ctx->S2, "ijab"), mone, W(ctx->R, "ijba"), false, 1.0);
    // - sum_m P^-_ij f_mj t^{ab}_{im}
    P->contract("cc2:foo", W(ctx->R, "ijab"), one, W(t2, "imab"), false, V(ctx->foo, "mj"), false, 0.0);
    P->add("cc2:foo", W(ctx->S2, "ijab"), mone, W(ctx->R, "ijab"), false, 1.0);
    P->add("cc2:foo", W(ctx->S2, "ijab"), one, W(ctx->R, "jiab"), false, 1.0);
  }

  // S^a_i (CCD: zero)
  if (ccd) {
    z* s1 = ctx->S1;
    P->custom("S1", [=](cudaStream_t s) { return cudaMemsetAsync(s1, 0, sizeof(z) * (size_t)o * v, s); });
  } else {
    P->add("S1", W(ctx->S1, "ia"), one, V(ctx->fov, "ia"), true, 0.0);                                   // F^{i+}_a
    P->contract("S1", W(ctx->S1, "ia"), one, W(ctx->Hvv, "ac"), false, W(t1, "ic"), false, 1.0);          // H^a_c t^c_i
    P->contract("S1", W(ctx->S1, "ia"), one, W(ctx->Hoo, "ki"), false, W(t1, "ka"), false, 1.0);          // H^k_i t^a_k
    P->contract("S1", W(ctx->S1, "ia"), one, W(ctx->Hov, "kc"), false, W(t2, "ikac"), false, 1.0);        // H^k_c t^{ac}_{ik}
    P->add("S1", W(ctx->Yov, "kc"), one, W(ctx->Hov, "kc"), false, 0.0);                                   // H^k_c - 2 F^k_c
    P->add("S1", W(ctx->Yov, "kc"), zmake(-2, 0), V(ctx->fov, "kc"), false, 1.0);
    P->contract("S1", W(ctx->Zoo, "ik"), one, W(ctx->Yov, "kc"), false, W(t1, "ic"), false, 0.0);
    P->contract("S1", W(ctx->S1, "ia"), one, W(ctx->Zoo, "ik"), false, W(t1, "ka"), false, 1.0);
    {
      // 1/2 sum_kcd V^{ak}_{cd} tau^{cd}_{ik} = sum_k sum_{c<d}: tau packed over (c<d) into R, one GEMM
      // against vovv_pk
      z *taur = ctx->R;
      P->custom("S1", [=](cudaStream_t s) { return pack_pairs(tau, taur, (int64_t)o * o, v, 0, s); });
      ZGemmArgs g;
      g.M = o;
      g.N = v;
      g.K = (int64_t)o * Pv;
      g.A = ctx->R;
      g.lda = (int64_t)o * Pv;
      g.B = ctx->vovv_pk;
      g.ldb = (int64_t)o * Pv;
      g.transB = 1;
      g.C = ctx->S1;
      g.ldc = v;
      g.beta = one;
      P->gemm("S1:gemm", g);
    }
    P->contract("S1", W(ctx->S1, "ia"), half, V(ctx->ooov, "klic"), false, W(tau, "klca"), false, 1.0);    // 1/2 V^{kl}_{ic} tau^{ca}_{kl}
    P->contract("S1", W(ctx->S1, "ia"), mone, V(ctx->J, "iakc"), false, W(t1, "kc"), false, 1.0);         // - V^{ak}_{ci} t^c_k
  }

  if (P->status() != cudaSuccess) return set_err(ctx, CCSD_ERR_CUDA, "residual plan: " + P->error());
  for (void* m : P->owned()) ctx->allocs.push_back(m);
  ctx->device_bytes += P->owned_bytes();
  ctx->plan_cached_bytes = P->owned_bytes();
  P->owned().clear();
  CS(dalloc(ctx, &ctx->scratch, P->scratch_elems()));
  if (ctx->df_w_off >= 0) {
    ctx->Dblk = ctx->scratch;
    ctx->Wblk = ctx->scratch + ctx->df_w_off;
  }
  ctx->gemm_ws_elems = P->gemm_workspace_elems();
  CS(dalloc(ctx, &ctx->gemm_ws, ctx->gemm_ws_elems));
  if (ctx->use_split) {
    ctx->split_ws_bytes = P->aux_bytes();
    uint8_t* w = nullptr;
    CS(dalloc(ctx, &w, ctx->split_ws_bytes));
    ctx->split_ws = w;
  }
  return CCSD_OK;
}

// Names of the timed segments: the plan's ops, then the iteration tail.
void init_timers(ccsd_ctx* ctx) {
  if (!ctx->tnames.empty()) return;
  for (auto& op : ctx->plan->ops()) ctx->tnames.push_back(op.name);
  for (const char* nm : {"update", "norm", "diis"}) ctx->tnames.push_back(nm);
  ctx->tev.resize(ctx->tnames.size() + 1);
  for (auto& e : ctx->tev) cudaEventCreate(&e);
  ctx->tsum.assign(ctx->tnames.size(), 0.0);
  ctx->tcount = 0;
}

cudaError_t mark(ccsd_ctx* ctx, bool timed, size_t k) {
  if (!timed) return cudaSuccess;
  return cudaEventRecordWithFlags(ctx->tev[k], ctx->stream, cudaEventRecordExternal);
}

// Runs the plan in order; each op sits in an NVTX range named after it (':' -> '_'),
// so a profiler can select one op's launches in an eager evaluation.
cudaError_t run_ops(ccsd_ctx* ctx, bool timed) {
  auto& ops = ctx->plan->ops();
  cudaError_t e = mark(ctx, timed, 0);
  for (size_t k = 0; k < ops.size() && e == cudaSuccess; ++k) {
    std::string nm = ops[k].name;
    std::replace(nm.begin(), nm.end(), ':', '_');
    nvtxRangePushA(nm.c_str());
    e = ops[k].run(ctx->stream);
    nvtxRangePop();
    if (e == cudaSuccess) e = mark(ctx, timed, k + 1);
  }
  return e;
}

// Add the elapsed time of every completed segment [first, last) to the sums.
void collect_timers(ccsd_ctx* ctx, size_t last) {
  for (size_t k = 0; k < last; ++k) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->tev[k], ctx->tev[k + 1]) == cudaSuccess) ctx->tsum[k] += ms;
  }
  cudaGetLastError();
  ctx->tcount += 1;
}

// The amplitude backup (before an iteration, or around ccsd_residual with the caller's amplitudes)
// keeps t1 and the unique doubles (i<j, a<b): t2 is antisymmetric in both pairs, and the restore
// rebuilds it from them (its diagonal pairs are zero), exactly for antisymmetric amplitudes, in a
// quarter of the memory of a full copy.
cudaError_t backup_amplitudes(ccsd_ctx* ctx, z* t1_to, z* t2pk_to) {
  const int64_t n1 = (int64_t)ctx->o * ctx->v;
  cudaError_t e = cudaMemcpyAsync(t1_to, ctx->t1, n1 * sizeof(z), cudaMemcpyDeviceToDevice, ctx->stream);
  if (e == cudaSuccess) e = pack_pairs(ctx->t2, t2pk_to, ctx->o, ctx->v, 1, ctx->stream);
  return e;
}

cudaError_t restore_amplitudes(ccsd_ctx* ctx, const z* t1_from, const z* t2pk_from) {
  const int64_t n1 = (int64_t)ctx->o * ctx->v;
  cudaError_t e = cudaMemcpyAsync(ctx->t1, t1_from, n1 * sizeof(z), cudaMemcpyDeviceToDevice, ctx->stream);
  if (e != cudaSuccess) return e;
  UnpackArgs u;
  u.in = t2pk_from;
  u.out = ctx->t2;
  u.n1 = ctx->o;
  u.n2 = ctx->v;
  u.unpack_rows = 1;
  u.beta = 0.0;
  return unpack_pairs(u, ctx->stream);
}

// One iteration: backup, residual, t <- t + S/D (S <- S/D), norms, DIIS.
cudaError_t iteration_ops(ccsd_ctx* ctx, bool timed) {
  const int64_t n1 = (int64_t)ctx->o * ctx->v;
  const size_t nops = ctx->plan->ops().size();
  cudaError_t e = backup_amplitudes(ctx, ctx->t1_prev, ctx->t2_prev);
  if (e == cudaSuccess) e = run_ops(ctx, timed);
  // CCD: the singles equations are not solved, t1 stays zero (its update is zeroed)
  if (e == cudaSuccess && ctx->opts.method == CCSD_METHOD_CCD)
    e = cudaMemsetAsync(ctx->S1, 0, (size_t)n1 * sizeof(z), ctx->stream);
  if (e == cudaSuccess)
    e = denom_update(ctx->t1, ctx->t2, ctx->S1, ctx->S2, ctx->dvec, ctx->o, ctx->v, ctx->opts.level_shift,
                     ctx->upd_partials, ctx->stream);
  if (e == cudaSuccess) e = mark(ctx, timed, nops + 1);
  if (e == cudaSuccess) e = norm_finalize(ctx->upd_partials, update_blocks(), ctx->stats, ctx->stream);
  if (e == cudaSuccess) e = mark(ctx, timed, nops + 2);
  if (e == cudaSuccess && ctx->opts.diis_dim > 0) e = diis_step(ctx->diis, ctx->t1, ctx->t2, ctx->S1, ctx->S2, ctx->stream);
  if (e == cudaSuccess) e = mark(ctx, timed, nops + 3);
  return e;
}

ccsd_status copy_in(ccsd_ctx* ctx, z* dst, const void* src, int64_t count, int on_device) {
  CK(cudaMemcpyAsync(dst, src, count * sizeof(z), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     ctx->stream));
  return CCSD_OK;
}
ccsd_status copy_out(ccsd_ctx* ctx, void* dst, const z* src, int64_t count, int on_device) {
  CK(cudaMemcpyAsync(dst, src, count * sizeof(z), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     ctx->stream));
  return CCSD_OK;
}

bool hermitian(const ccsd_z* m, int64_t n, int64_t count) {
  for (int64_t q = 0; q < count; ++q) {
    const ccsd_z* a = m + q * n * n;
    double mx = 0.0, dev = 0.0;
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < n; ++j) {
        const ccsd_z x = a[i * n + j], y = a[j * n + i];
        mx = std::max(mx, std::hypot(x.re, x.im));
        dev = std::max(dev, std::hypot(x.re - y.re, x.im + y.im));
      }
    if (!(dev <= 1e-12 * std::max(mx, 1e-300)) && dev > 0.0) return false;
  }
  return true;
}

// Measured tile choice for every FP64 GEMM op of the plan: after one warm-up launch each of
// the 7 tile configurations runs twice between CUDA events and the fastest is kept. Shapes
// already in `cache` reuse their result. GEMMs routed to the split path are left alone.
// Outputs of the timed launches are garbage; the plan is run afresh afterwards.
using TuneCache = std::map<std::array<int64_t, 5>, int>;
ccsd_status autotune_plan(ccsd_ctx* ctx, TuneCache& cache) {
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  ccsd_status st = CCSD_OK;
  for (auto& op : ctx->plan->ops()) {
    if (!op.cfg || !op.args) continue;
    const ZGemmArgs& g = *op.args;
    if (ctx->routes_split && ctx->routes_split(g)) continue;
    const std::array<int64_t, 5> key = {g.M, g.N, g.K, g.transA, g.transB};
    auto it = cache.find(key);
    if (it != cache.end()) {
      *op.cfg = it->second;
      continue;
    }
    int best = -1;
    float bt = 0.f;
    for (int c = 0; c < 7 && st == CCSD_OK; ++c) {
      *op.cfg = c;
      cudaError_t e = op.run(ctx->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->stream);
      for (int r = 0; r < 2 && e == cudaSuccess; ++r) e = op.run(ctx->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) st = set_err(ctx, CCSD_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
      else if (best < 0 || ms < bt) {
        best = c;
        bt = ms;
      }
    }
    *op.cfg = best;
    cache[key] = best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

thread_local TuneCache* g_tune_cache = nullptr;  // shared by the systems of one batch while it is created

ccsd_status create_impl(int o, int v, const double* eps, const ccsd_z* fock, ccsd_int_kind kind, const ccsd_z* ints,
                        int naux, const ccsd_opts* opts, ccsd_ctx* ctx) {
  if (o < 1 || v < 1) return set_err(ctx, CCSD_ERR_ARG, "o and v must be >= 1");
  if (!eps || !ints) return set_err(ctx, CCSD_ERR_ARG, "eps and ints must not be NULL");
  if (kind == CCSD_INT_DF && naux < 1) return set_err(ctx, CCSD_ERR_ARG, "naux must be >= 1 for DF integrals");
  if (kind != CCSD_INT_DF && kind != CCSD_INT_FULL) return set_err(ctx, CCSD_ERR_ARG, "unknown integral kind");
  ctx->o = o;
  ctx->v = v;
  ctx->n = o + v;
  ctx->naux = kind == CCSD_INT_DF ? naux : 0;
  ctx->Po = pair_count(o);
  ctx->Pv = pair_count(v);
  if (opts) ctx->opts = *opts;
  else ccsd_default_opts(&ctx->opts);
  if (ctx->opts.diis_dim < 0 || ctx->opts.diis_dim > 16) return set_err(ctx, CCSD_ERR_ARG, "diis_dim must be in [0, 16]");
  if (ctx->opts.accelerator != CCSD_ACCEL_DIIS && ctx->opts.accelerator != CCSD_ACCEL_CROP)
    return set_err(ctx, CCSD_ERR_ARG, "accelerator must be CCSD_ACCEL_DIIS or CCSD_ACCEL_CROP");
  if (ctx->opts.diverge_iters < 0 || !(ctx->opts.diverge_factor >= 1.0))
    return set_err(ctx, CCSD_ERR_ARG, "diverge_iters must be >= 0 and diverge_factor >= 1");
  if (ctx->opts.vovv_block < 0) return set_err(ctx, CCSD_ERR_ARG, "vovv_block must be >= 0");
  if (ctx->opts.method != CCSD_METHOD_CCSD && ctx->opts.method != CCSD_METHOD_CCD &&
      ctx->opts.method != CCSD_METHOD_CC2)
    return set_err(ctx, CCSD_ERR_ARG, "unknown method");
  if (ctx->opts.method == CCSD_METHOD_CC2) {
    if (kind != CCSD_INT_DF)
      return set_err(ctx, CCSD_ERR_UNSUPPORTED, "CC2 is built on the T1-dressed DF factors: DF integrals needed");
    ctx->opts.store_w = 0;  // CC2 never uses <ab||cd>: keep only B^Q_vv
  }
  if (ctx->opts.precision != CCSD_PREC_FP64 && ctx->opts.precision != CCSD_PREC_SPLIT)
    return set_err(ctx, CCSD_ERR_ARG, "unknown precision mode");
  if (ctx->opts.precision == CCSD_PREC_SPLIT) {
    ctx->use_split = true;
    ctx->split.kind = kSplitE4M3;
    if (ctx->opts.digit_bits < 0 || ctx->opts.digit_bits > 5)
      return set_err(ctx, CCSD_ERR_ARG, "digit_bits must be in [1, 5] (e4m3 digits), 0 = 5");
    ctx->split.b = ctx->opts.digit_bits > 0 ? ctx->opts.digit_bits : 5;
    // default: about 39 bits of every row's scale (8 digits of 5 bits, 10 of 4)
    ctx->split.s = ctx->opts.slices > 0 ? ctx->opts.slices : (39 + ctx->split.b) / ctx->split.b;
    ctx->split_min_flops = ctx->opts.split_min_flops;
    if (ctx->split.s > 14 || ctx->split.b * ctx->split.s > 56)
      return set_err(ctx, CCSD_ERR_ARG, "slices must be <= 14 with digit_bits * slices <= 56");
  }
  if (!ctx->opts.store_w && kind != CCSD_INT_DF)
    return set_err(ctx, CCSD_ERR_UNSUPPORTED, "store_w = 0 needs DF factors (CCSD_INT_DF)");
  const int n = ctx->n;
  if (fock && !hermitian(fock, n, 1)) return set_err(ctx, CCSD_ERR_ARG, "Fock matrix is not Hermitian");
  if (kind == CCSD_INT_DF && !hermitian(ints, n, naux)) return set_err(ctx, CCSD_ERR_ARG, "B^Q is not Hermitian in (p,r)");
  if (ctx->opts.stream) {
    ctx->stream = (cudaStream_t)ctx->opts.stream;
  } else {
    CK(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
    ctx->own_stream = true;
  }

  // Fock blocks and the denominator diagonal
  std::vector<ccsd_z> F((size_t)n * n, ccsd_z{0.0, 0.0});
  if (fock) std::memcpy(F.data(), fock, sizeof(ccsd_z) * n * n);
  else
    for (int p = 0; p < n; ++p) F[(size_t)p * n + p].re = eps[p];
  std::vector<double> dv(n);
  for (int p = 0; p < n; ++p) dv[p] = F[(size_t)p * n + p].re;
  std::vector<ccsd_z> foo((size_t)o * o), fov((size_t)o * v), fvv((size_t)v * v);
  for (int i = 0; i < o; ++i)
    for (int j = 0; j < o; ++j) foo[(size_t)i * o + j] = F[(size_t)i * n + j];
  for (int i = 0; i < o; ++i)
    for (int a = 0; a < v; ++a) fov[(size_t)i * v + a] = F[(size_t)i * n + o + a];
  for (int a = 0; a < v; ++a)
    for (int b = 0; b < v; ++b) fvv[(size_t)a * v + b] = F[(size_t)(o + a) * n + o + b];
  CS(dalloc(ctx, &ctx->dvec, n));
  CS(dalloc(ctx, &ctx->foo, (int64_t)o * o));
  CS(dalloc(ctx, &ctx->fov, (int64_t)o * v));
  CS(dalloc(ctx, &ctx->fvv, (int64_t)v * v));
  CK(cudaMemcpyAsync(ctx->dvec, dv.data(), sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->foo, foo.data(), sizeof(z) * o * o, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->fov, fov.data(), sizeof(z) * o * v, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->fvv, fvv.data(), sizeof(z) * v * v, cudaMemcpyHostToDevice, ctx->stream));

  CS(dalloc(ctx, &ctx->split_err, 1));
  CK(cudaMemsetAsync(ctx->split_err, 0, sizeof(int), ctx->stream));
  // integral blocks
  const int64_t oo = (int64_t)o * o, vv = (int64_t)v * v, ov = (int64_t)o * v;
  CS(dalloc(ctx, &ctx->oooo, oo * oo));
  CS(dalloc(ctx, &ctx->ooov, oo * ov));
  CS(dalloc(ctx, &ctx->oovv, oo * vv));
  CS(dalloc(ctx, &ctx->vovv_pk, ov * ctx->Pv));
  CS(dalloc(ctx, &ctx->J, ov * ov));
  if (ctx->opts.store_w) CS(dalloc(ctx, &ctx->Wpk, ctx->Pv * ctx->Pv));
  else CS(dalloc(ctx, &ctx->Bvv, (int64_t)naux * v * v));
  if (ctx->opts.method == CCSD_METHOD_CC2) {
    CS(dalloc(ctx, &ctx->c2_Bvo, (int64_t)naux * v * o));
    CS(dalloc(ctx, &ctx->c2_Boo, (int64_t)naux * o * o));
    CS(dalloc(ctx, &ctx->c2_Bov, (int64_t)naux * o * v));
    CS(dalloc(ctx, &ctx->c2_Bt, (int64_t)naux * v * o));
    CS(dalloc(ctx, &ctx->c2_Dt, (int64_t)naux * o * o));
  }
  {
    void* dints = nullptr;
    const int64_t cnt = kind == CCSD_INT_DF ? (int64_t)naux * n * n : (int64_t)n * n * n * n;
    if (cudaMalloc(&dints, cnt * sizeof(z)) != cudaSuccess) {
      cudaGetLastError();
      return set_err(ctx, CCSD_ERR_OOM, "device copy of the integrals");
    }
    ccsd_status st = CCSD_OK;
    cudaError_t e = cudaMemcpyAsync(dints, ints, cnt * sizeof(z), cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) st = set_err(ctx, CCSD_ERR_CUDA, cudaGetErrorString(e));
    // vovo is needed only as J[i][a][k][c] = <ak||ci>: built into a temporary
    void* mvovo = nullptr;
    if (st == CCSD_OK && cudaMalloc(&mvovo, ov * ov * sizeof(z)) != cudaSuccess) {
      cudaGetLastError();
      st = set_err(ctx, CCSD_ERR_OOM, "vovo temporary");
    }
    const char* names[4] = {"oooo", "ooov", "oovv", "vovo"};
    z* outs[4] = {ctx->oooo, ctx->ooov, ctx->oovv, (z*)mvovo};
    for (int b = 0; b < 4 && st == CCSD_OK; ++b)
      st = kind == CCSD_INT_DF ? build_block_df(ctx, (const z*)dints, names[b], outs[b])
                               : build_block_full(ctx, (const z*)dints, names[b], outs[b]);
    if (st == CCSD_OK) {
      const int64_t d_vovo[4] = {v, o, v, o};  // [a][k][c][i] -> J[i][a][k][c]
      const int pJ[4] = {3, 0, 1, 2};
      e = permute4((z*)mvovo, d_vovo, pJ, ctx->J, zmake(1, 0), 0.0, 0, ctx->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
      if (e != cudaSuccess) st = set_err(ctx, CCSD_ERR_CUDA, cudaGetErrorString(e));
    }
    cudaFree(mvovo);
    if (st == CCSD_OK)
      st = kind == CCSD_INT_DF ? build_vovv_pk_df(ctx, (const z*)dints) : build_vovv_pk_full(ctx, (const z*)dints);
    if (st == CCSD_OK) {
      if (kind == CCSD_INT_DF && !ctx->opts.store_w) {
        e = extract_B(ctx, (const z*)dints, 'v', 'v', ctx->Bvv, ctx->stream);
        if (e == cudaSuccess && ctx->opts.method == CCSD_METHOD_CC2) {
          e = extract_B(ctx, (const z*)dints, 'v', 'o', ctx->c2_Bvo, ctx->stream);
          if (e == cudaSuccess) e = extract_B(ctx, (const z*)dints, 'o', 'o', ctx->c2_Boo, ctx->stream);
          if (e == cudaSuccess) e = extract_B(ctx, (const z*)dints, 'o', 'v', ctx->c2_Bov, ctx->stream);
        }
        if (e != cudaSuccess) st = set_err(ctx, CCSD_ERR_CUDA, cudaGetErrorString(e));
      } else if (kind == CCSD_INT_DF) {
        st = build_w_df(ctx, (const z*)dints);
      } else {
        z* vvvv = nullptr;
        if (cudaMalloc(&vvvv, vv * vv * sizeof(z)) != cudaSuccess) {
          cudaGetLastError();
          st = set_err(ctx, CCSD_ERR_OOM, "vvvv temporary");
        } else {
          st = build_block_full(ctx, (const z*)dints, "vvvv", vvvv);
          if (st == CCSD_OK) {
            e = pack_pairs(vvvv, ctx->Wpk, v, v, 1, ctx->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
            if (e != cudaSuccess) st = set_err(ctx, CCSD_ERR_CUDA, cudaGetErrorString(e));
          }
          cudaFree(vvvv);
        }
      }
    }
    cudaStreamSynchronize(ctx->stream);
    cudaFree(dints);
    if (st != CCSD_OK) return st;
  }
  if (ctx->use_split && ctx->opts.store_w) {
    // <ab||cd> is constant: cut its digits once
    uint8_t* mem = nullptr;
    CS(dalloc(ctx, &mem, slice_bytes(ctx->Pv, ctx->Pv, ctx->split)));
    CK(make_slices(ctx->Wpk, ctx->Pv, ctx->Pv, ctx->Pv, 0, 0, ctx->split, ctx->Wsl, mem, ctx->stream));
  }
  // derived constant layouts
  CS(dalloc(ctx, &ctx->oovv_pk, ctx->Po * ctx->Pv));
  CK(pack_pairs(ctx->oovv, ctx->oovv_pk, o, v, 1, ctx->stream));

  // amplitudes, residuals and intermediates
  const int64_t n2 = oo * vv;
  CS(dalloc(ctx, &ctx->t1, ov));
  CS(dalloc(ctx, &ctx->t2, n2));
  CS(dalloc(ctx, &ctx->S1, ov));
  CS(dalloc(ctx, &ctx->S2, n2));
  CS(dalloc(ctx, &ctx->t1_prev, ov));
  CS(dalloc(ctx, &ctx->t2_prev, ctx->Po * ctx->Pv));  // the backup: unique doubles only
  // the backup of ccsd_residual (amplitudes given by the caller) and the one an iteration keeps
  // for a non-finite update are never live at the same time: one buffer serves both
  ctx->t1_save = ctx->t1_prev;
  ctx->t2_save = ctx->t2_prev;
  CS(dalloc(ctx, &ctx->tau, n2));
  CS(dalloc(ctx, &ctx->tau_pk, ctx->Po * ctx->Pv));
  CS(dalloc(ctx, &ctx->Hvv, vv));
  CS(dalloc(ctx, &ctx->Gvv, vv));
  CS(dalloc(ctx, &ctx->Hoo, oo));
  CS(dalloc(ctx, &ctx->Goo, oo));
  CS(dalloc(ctx, &ctx->Hov, ov));
  CS(dalloc(ctx, &ctx->Yov, ov));
  CS(dalloc(ctx, &ctx->Zoo, oo));
  CS(dalloc(ctx, &ctx->Hr, n2));
  CS(dalloc(ctx, &ctx->R, n2));
  CS(dalloc(ctx, &ctx->C, ov * oo));
  {
    // Yovoo, Yfull and Ypk are temporaries of the C^{kb}_{ij} block only, which runs while R is
    // free (after the H^{ak}_{ci} term has read X from it, before the ring product): they live
    // in R when they fit
    auto r16 = [](int64_t x) { return (x + 15) / 16 * 16; };
    const int64_t y1 = r16(ov * oo), yp = ov * ctx->Po;
    if (2 * y1 + yp <= n2) {
      ctx->Yovoo = ctx->R;
      ctx->Yfull = ctx->R + y1;
      ctx->Ypk = ctx->R + 2 * y1;
    } else {
      CS(dalloc(ctx, &ctx->Yovoo, ov * oo));
      CS(dalloc(ctx, &ctx->Ypk, ov * ctx->Po));
      CS(dalloc(ctx, &ctx->Yfull, ov * oo));
    }
  }
  CS(dalloc(ctx, &ctx->Afull, oo * oo));
  CS(dalloc(ctx, &ctx->Yoooo, oo * oo));
  CS(dalloc(ctx, &ctx->Apk, ctx->Po * ctx->Po));
  // the hole-ladder product (Hpk) is unpacked into S2 before the particle ladder writes Lpk
  CS(dalloc(ctx, &ctx->Lpk, ctx->Po * ctx->Pv));
  ctx->Hpk = ctx->Lpk;
  CS(dalloc(ctx, &ctx->upd_partials, 2 * update_blocks()));
  CS(dalloc(ctx, &ctx->stats, 4));
  CS(dalloc(ctx, &ctx->e_partials, energy_blocks()));
  CS(dalloc(ctx, &ctx->e_dev, 1));
  CK(cudaMallocHost(&ctx->stats_host, 4 * sizeof(double)));
  CK(cudaMallocHost(&ctx->e_host, sizeof(z)));
  CK(cudaMallocHost(&ctx->err_host, sizeof(int)));
  *ctx->err_host = 0;
  CK(cudaMemsetAsync(ctx->t1, 0, ov * sizeof(z), ctx->stream));
  CK(cudaMemsetAsync(ctx->t2, 0, n2 * sizeof(z), ctx->stream));

  // DIIS subspace
  if (ctx->opts.diis_dim > 0) {
    DiisArgs& d = ctx->diis;
    d.o = o;
    d.v = v;
    d.m = ctx->opts.diis_dim;
    d.start = ctx->opts.diis_start;
    d.crop = ctx->opts.accelerator == CCSD_ACCEL_CROP ? 1 : 0;
    d.L = ov + ctx->Po * ctx->Pv;
    CS(dalloc(ctx, &d.hist_t, d.m * d.L));
    CS(dalloc(ctx, &d.hist_e, d.m * d.L));
    CS(dalloc(ctx, &d.Bmat, (int64_t)d.m * d.m));
    CS(dalloc(ctx, &d.coef, d.m));
    CS(dalloc(ctx, &d.partials, (int64_t)d.m * diis_blocks()));
    CS(dalloc(ctx, &d.state, 1));
    CK(diis_reset(d, ctx->stream));
  }

  CS(build_residual_plan(ctx));
  init_timers(ctx);
  if (ctx->opts.autotune) {
    TuneCache local;
    CS(autotune_plan(ctx, g_tune_cache ? *g_tune_cache : local));
  }

  // MP2 guess: one denominator update from t = 0 (CCD: the singles stay zero)
  CK(run_ops(ctx, false));
  if (ctx->opts.method == CCSD_METHOD_CCD) CK(cudaMemsetAsync(ctx->S1, 0, (size_t)ov * sizeof(z), ctx->stream));
  CK(denom_update(ctx->t1, ctx->t2, ctx->S1, ctx->S2, ctx->dvec, o, v, ctx->opts.level_shift, ctx->upd_partials,
                  ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return CCSD_OK;
}

void free_ctx(ccsd_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
  if (ctx->lgraph) cudaGraphExecDestroy(ctx->lgraph);
  for (auto e : ctx->tev) cudaEventDestroy(e);
  for (void* p : ctx->allocs) cudaFree(p);
  for (Plan* P : {ctx->plan, ctx->lplan, ctx->dplan})
    if (P) {
      for (void* p : P->owned()) cudaFree(p);
      delete P;
    }
  if (ctx->stats_host) cudaFreeHost(ctx->stats_host);
  if (ctx->e_host) cudaFreeHost(ctx->e_host);
  if (ctx->err_host) cudaFreeHost(ctx->err_host);
  for (auto ev : ctx->lev) cudaEventDestroy(ev);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

// ---------------------------------------------------------------------------
// Lambda equations. R = dL/dt of L = E(t) + sum_mu lambda_mu S_mu(t), the stationarity conditions
// that the appendix "Working equations for CCSD lambda equations" writes with Hbar intermediates.
// The plan is the adjoint of the residual plan, term by term in reverse order (one op per line of
// the CPU oracle's explicit adjoint). It reads the intermediates that the residual plan leaves at
// the current amplitudes: tau, H^a_c, G^a_c, H^k_i, G^k_i, H^k_c, Yov = H^k_c - 2 F^k_c, Zoo,
// H^{ak}_{ci} in Hr, C, and A from its packed copy. It writes R1 into S1 and R2 into S2.
// ---------------------------------------------------------------------------
// Frees a plan that never reached the context, with the cached permutations it still owns.
struct PlanDeleter {
  void operator()(Plan* p) const {
    for (void* m : p->owned()) cudaFree(m);
    delete p;
  }
};

ccsd_status build_lambda_plan(ccsd_ctx* ctx) {
  const int o = ctx->o, v = ctx->v;
  const int64_t Po = ctx->Po, Pv = ctx->Pv, ov = (int64_t)o * v, n2 = ov * ov, o4 = (int64_t)o * o * o * o;
  // buffers an earlier build that failed (out of memory further on) already allocated are reused
  auto once = [ctx](auto** p, int64_t count) { return *p ? CCSD_OK : dalloc(ctx, p, count); };
  CS(once(&ctx->l1, ov));
  CS(once(&ctx->l2, n2));
  for (z** p : {&ctx->lG, &ctx->ltaub, &ctx->lHrb, &ctx->lXb, &ctx->lzb}) CS(once(p, n2));
  for (z** p : {&ctx->lCb, &ctx->lCanti, &ctx->lCp}) CS(once(p, ov * o * o));
  for (z** p : {&ctx->lAb, &ctx->lAanti}) CS(once(p, o4));
  CS(once(&ctx->lApk, Po * Po));
  CS(once(&ctx->lpk, (int64_t)o * o * Pv));
  CS(once(&ctx->lpk2, Po * Pv));
  CS(once(&ctx->lout, Po * Pv));
  CS(once(&ctx->lout2, (int64_t)o * o * Pv));
  CS(once(&ctx->lout3, std::max<int64_t>((int64_t)o * o * Pv, ov * Po)));  // also C-bar packed over (i<j)
  CS(once(&ctx->lGvvb, (int64_t)v * v));
  CS(once(&ctx->lHvvb, (int64_t)v * v));
  CS(once(&ctx->lGoob, (int64_t)o * o));
  CS(once(&ctx->lHoob, (int64_t)o * o));
  CS(once(&ctx->lHovb, ov));
  CK(cudaMemsetAsync(ctx->l1, 0, ov * sizeof(z), ctx->stream));
  CK(cudaMemsetAsync(ctx->l2, 0, n2 * sizeof(z), ctx->stream));
  if (ctx->opts.diis_dim > 0) {
    DiisArgs& d = ctx->ldiis;
    const DiisArgs earlier = d;
    d = ctx->diis;  // same shape and options; its own history
    d.hist_t = earlier.hist_t;
    d.hist_e = earlier.hist_e;
    d.Bmat = earlier.Bmat;
    d.coef = earlier.coef;
    d.partials = earlier.partials;
    d.state = earlier.state;
    CS(once(&d.hist_t, d.m * d.L));
    CS(once(&d.hist_e, d.m * d.L));
    CS(once(&d.Bmat, (int64_t)d.m * d.m));
    CS(once(&d.coef, d.m));
    CS(once(&d.partials, (int64_t)d.m * diis_blocks()));
    CS(once(&d.state, 1));
    CK(diis_reset(d, ctx->stream));
  }
  // the context takes the plan only once it is complete (a failed build leaves no plan behind)
  std::unique_ptr<Plan, PlanDeleter> holder(new Plan(o, v, &ctx->lscratch, ctx->stream));
  holder->set_cache_limit(cache_limit_bytes(ctx->opts));
  Plan* P = holder.get();
  set_plan_gemm(ctx, P);
  const z one = zmake(1, 0), mone = zmake(-1, 0), half = zmake(0.5, 0), quarter = zmake(0.25, 0),
          eighth = zmake(0.125, 0);
  auto V = [&](z* p, const char* lab) { return P->view(p, lab, true); };
  auto W = [&](z* p, const char* lab) { return P->view(p, lab, false); };
  z *t1 = ctx->t1, *t2 = ctx->t2, *l1 = ctx->l1, *l2 = ctx->l2, *r1 = ctx->S1, *G = ctx->lG, *taub = ctx->ltaub;
  z *Hrb = ctx->lHrb, *Xb = ctx->lXb, *zb = ctx->lzb;

  // energy: dE/dt1 = f_ia, dE/dtau = 1/4 <ij||ab>
  P->add("L:E", W(r1, "ia"), one, V(ctx->fov, "ia"), false, 0.0);
  P->add("L:E", W(taub, "ijab"), quarter, V(ctx->oovv, "ijab"), false, 0.0);
  // S2 terms, weighted by 1/4 l2 (unique doubles); each antisymmetriser's adjoint on l2 gives 2
  P->contract("L:ring", W(Hrb, "iakc"), one, W(l2, "ijab"), false, W(t2, "jkcb"), false, 0.0);
  P->contract("L:ring", W(G, "jkcb"), one, W(l2, "ijab"), false, W(ctx->Hr, "iakc"), false, 0.0);
  P->contract("L:goo", W(ctx->lGoob, "kj"), half, W(l2, "ijab"), false, W(t2, "ikab"), false, 0.0);
  P->contract("L:goo", W(G, "ikab"), half, W(l2, "ijab"), false, W(ctx->Goo, "kj"), false, 1.0);
  {
    // sum_c P^-_ij conj(V^{cj}_{ab}) t^c_i:  R1[i][c] += sum_{j, a<b} l2[i][j][P(a,b)] conj(<cj||ab>)
    z* lpk = ctx->lpk;
    P->custom("L:vt1", [=](cudaStream_t s) { return pack_pairs(l2, lpk, (int64_t)o * o, v, 0, s); });
    ZGemmArgs g;
    g.M = o;
    g.N = v;
    g.K = (int64_t)o * Pv;
    g.A = lpk;
    g.lda = (int64_t)o * Pv;
    g.B = ctx->vovv_pk;
    g.ldb = (int64_t)o * Pv;
    g.transB = 1;
    g.conjB = 1;
    g.C = r1;
    g.ldc = v;
    g.beta = one;
    P->gemm("L:vt1:gemm", g);
  }
  P->contract("L:gvv", W(ctx->lGvvb, "ac"), half, W(l2, "ijab"), false, W(t2, "ijcb"), false, 0.0);
  P->contract("L:gvv", W(G, "ijcb"), half, W(l2, "ijab"), false, W(ctx->Gvv, "ac"), false, 1.0);
  P->contract("L:ct1", W(ctx->lCb, "kaij"), half, W(l2, "ijab"), false, W(t1, "kb"), false, 0.0);
  P->contract("L:ct1", W(r1, "kb"), half, W(l2, "ijab"), false, W(ctx->C, "kaij"), false, 1.0);
  {
    // hole ladder 1/2 sum_kl A^{kl}_{ij} tau^{ab}_{kl}, all three labels pairs antisymmetric: over
    // packed pairs, as in the residual. A-bar[kl][ij] = 1/8 sum_ab l2[ijab] tau[klab]
    //   -> lApk[P(kl)][P(ij)] = 1/4 sum_{a<b} tau_pk[P(kl)][P(ab)] l2_pk[P(ij)][P(ab)];
    // tau-bar[klab] += 1/8 sum_ij l2[ijab] A[klij] -> 1/4 sum_{i<j} Apk[P(kl)][P(ij)] l2_pk[P(ij)][P(ab)]
    z *lpk2 = ctx->lpk2, *lout = ctx->lout, *lapk = ctx->lApk, *lab = ctx->lAb;
    P->custom("L:hole", [=](cudaStream_t s) { return pack_pairs(l2, lpk2, o, v, 1, s); });
    ZGemmArgs g;
    g.M = Po;
    g.N = Po;
    g.K = Pv;
    g.A = ctx->tau_pk;
    g.lda = Pv;
    g.B = lpk2;
    g.ldb = Pv;
    g.transB = 1;
    g.C = lapk;
    g.ldc = Po;
    g.alpha = quarter;
    P->gemm("L:hole:gemm", g);
    P->custom("L:hole", [=](cudaStream_t s) {
      UnpackArgs u;  // A-bar in full, for the terms that read it unpacked
      u.in = lapk;
      u.out = lab;
      u.n1 = o;
      u.n2 = o;
      u.unpack_rows = 1;
      u.beta = 0.0;
      return unpack_pairs(u, s);
    });
    ZGemmArgs h;
    h.M = Po;
    h.N = Pv;
    h.K = Po;
    h.A = ctx->Apk;
    h.lda = Po;
    h.B = lpk2;
    h.ldb = Pv;
    h.C = lout;
    h.ldc = Pv;
    h.alpha = quarter;
    P->gemm("L:hole:gemm", h);
    P->custom("L:hole", [=](cudaStream_t s) {
      UnpackArgs u;
      u.in = lout;
      u.out = taub;
      u.n1 = o;
      u.n2 = v;
      u.unpack_rows = 1;
      u.beta = 1.0;
      return unpack_pairs(u, s);
    });
  }
  {
    // ladder: 1/8 sum_ab l2[ijab] <ab||cd> = 1/4 sum_{a<b}, one packed GEMM against <ab||cd>
    // (l2 packed over both pairs by the hole term above)
    z *lpk2 = ctx->lpk2, *lout = ctx->lout;
    if (ctx->use_split) {
      // against the digits of <ab||cd> cut at creation (rows (a<b) over K = (c<d)): the GEMM wants
      // rows (c<d) over K = (a<b), i.e. <ab||cd> = conj(<cd||ab>), the cached rows conjugated
      P->note_aux_bytes(slice_bytes(Po, Pv, ctx->split) + split_part_bytes(Po, Pv, Pv, ctx->split));
      P->custom("L:ladder:gemm", [ctx, lpk2, lout, Po, Pv](cudaStream_t s) {
        SliceSet SA;
        uint8_t* w = static_cast<uint8_t*>(ctx->split_ws);
        cudaError_t e = make_slices(lpk2, Po, Pv, Pv, 0, 0, ctx->split, SA, w, s);
        if (e == cudaSuccess)
          e = split_gemm(SA, ctx->Wsl, lout, Pv, zmake(1, 0), zmake(0, 0), ctx->split_err,
                         w + slice_bytes(Po, Pv, ctx->split), split_part_bytes(Po, Pv, Pv, ctx->split), s, 0, 0, 1);
        return e;
      }, 8.0 * (double)Po * (double)Pv * (double)Pv);
    } else {
      ZGemmArgs g;
      g.M = Po;
      g.N = Pv;
      g.K = Pv;
      g.A = lpk2;
      g.lda = Pv;
      g.B = ctx->Wpk;
      g.ldb = Pv;
      g.C = lout;
      g.ldc = Pv;
      P->gemm("L:ladder:gemm", g);
    }
    P->custom("L:ladder", [=](cudaStream_t s) {
      UnpackArgs u;
      u.in = lout;
      u.out = taub;
      u.n1 = o;
      u.n2 = v;
      u.unpack_rows = 1;
      u.alpha = quarter;
      u.beta = 1.0;
      return unpack_pairs(u, s);
    });
  }
  // S1 terms, weighted by l1
  P->contract("L:hvv", W(ctx->lHvvb, "ac"), one, W(l1, "ia"), false, W(t1, "ic"), false, 0.0);
  P->contract("L:hvv", W(r1, "ic"), one, W(l1, "ia"), false, W(ctx->Hvv, "ac"), false, 1.0);
  P->contract("L:hoo", W(ctx->lHoob, "ki"), one, W(l1, "ia"), false, W(t1, "ka"), false, 0.0);
  P->contract("L:hoo", W(r1, "ka"), one, W(l1, "ia"), false, W(ctx->Hoo, "ki"), false, 1.0);
  P->contract("L:hov", W(ctx->lHovb, "kc"), one, W(l1, "ia"), false, W(t2, "ikac"), false, 0.0);
  {
    // the t2 adjoint of sum_kc H^k_c t^{ac}_{ik} is the outer product l1[i][a] H[k][c]: a K = 1 GEMM
    ZGemmArgs g;
    g.M = ov;
    g.N = ov;
    g.K = 1;
    g.A = l1;
    g.lda = 1;
    g.B = ctx->Hov;
    g.ldb = ov;
    g.C = zb;
    g.ldc = ov;
    P->gemm("L:hov:outer", g);
    P->add("L:hov", W(G, "ikac"), one, W(zb, "iakc"), false, 1.0);
  }
  // hf: sum_k (sum_c (H^k_c - 2F^k_c) t^c_i) t^a_k, with Q[k][i] = sum_a l1[i][a] t1[k][a] (lHoob above)
  P->contract("L:hf", W(ctx->lHovb, "kc"), one, W(ctx->lHoob, "ki"), false, W(t1, "ic"), false, 1.0);
  P->contract("L:hf", W(r1, "ic"), one, W(ctx->lHoob, "ki"), false, W(ctx->Yov, "kc"), false, 1.0);
  P->contract("L:hf", W(r1, "ka"), one, W(ctx->Zoo, "ik"), false, W(l1, "ia"), false, 1.0);
  {
    // 1/2 sum_kcd V^{ak}_{cd} tau^{cd}_{ik}:  tau-bar[i][k][c][d] += 1/2 sum_a l1[i][a] <ak||cd>, packed
    z* o2 = ctx->lout2;
    ZGemmArgs g;
    g.M = o;
    g.N = (int64_t)o * Pv;
    g.K = v;
    g.A = l1;
    g.lda = v;
    g.B = ctx->vovv_pk;
    g.ldb = (int64_t)o * Pv;
    g.C = o2;
    g.ldc = (int64_t)o * Pv;
    P->gemm("L:vovv:gemm", g);
    P->custom("L:vovv", [=](cudaStream_t s) {
      UnpackArgs u;
      u.in = o2;
      u.out = taub;
      u.n1 = (int64_t)o * o;
      u.n2 = v;
      u.alpha = half;
      u.beta = 1.0;
      return unpack_pairs(u, s);
    });
  }
  P->contract("L:ooov", W(taub, "klca"), half, W(l1, "ia"), false, V(ctx->ooov, "klic"), false, 1.0);
  P->contract("L:vovo", W(r1, "kc"), mone, W(l1, "ia"), false, V(ctx->J, "iakc"), false, 1.0);
  // A^{kl}_{ij}
  {
    // tau-bar[ijcd] += 1/2 sum_kl A-bar[klij] <kl||cd> = sum_{k<l}, packed over (i<j) and (c<d)
    z *lout = ctx->lout;
    ZGemmArgs g;
    g.M = Po;
    g.N = Pv;
    g.K = Po;
    g.A = ctx->lApk;
    g.lda = Po;
    g.transA = 1;
    g.B = ctx->oovv_pk;
    g.ldb = Pv;
    g.C = lout;
    g.ldc = Pv;
    P->gemm("L:A:gemm", g);
    P->custom("L:A", [=](cudaStream_t s) {
      UnpackArgs u;
      u.in = lout;
      u.out = taub;
      u.n1 = o;
      u.n2 = v;
      u.unpack_rows = 1;
      u.beta = 1.0;
      return unpack_pairs(u, s);
    });
  }
  P->add("L:A", W(ctx->lAanti, "klij"), one, W(ctx->lAb, "klij"), false, 0.0);
  P->add("L:A", W(ctx->lAanti, "klij"), mone, W(ctx->lAb, "klji"), false, 1.0);
  P->contract("L:A", W(r1, "jc"), one, W(ctx->lAanti, "klij"), false, V(ctx->ooov, "klic"), false, 1.0);
  // C^{kb}_{ij}: -1/2 sum_kb C-bar[k][b][i][j] <bk||cd> into tau-bar, packed over c<d and (C-bar
  // is antisymmetric in i, j) over i<j: C-bar as [(b,k)][P(i,j)], one GEMM with the (b,k) rows summed
  {
    z *cp = ctx->lCp, *o3 = ctx->lout3;
    P->add("L:C", W(cp, "bkij"), one, W(ctx->lCb, "kbij"), false, 0.0);
    P->custom("L:C", [=](cudaStream_t s) { return pack_pairs(cp, o3, (int64_t)v * o, o, 0, s); });
    z* out = ctx->lout;
    ZGemmArgs g;
    g.M = Po;
    g.N = Pv;
    g.K = (int64_t)v * o;
    g.A = o3;
    g.lda = Po;
    g.transA = 1;
    g.B = ctx->vovv_pk;
    g.ldb = Pv;
    g.C = out;
    g.ldc = Pv;
    P->gemm("L:C:gemm", g);
    P->custom("L:C", [=](cudaStream_t s) {
      UnpackArgs u;
      u.in = out;
      u.out = taub;
      u.n1 = o;
      u.n2 = v;
      u.unpack_rows = 1;
      u.alpha = zmake(-0.5, 0);
      u.beta = 1.0;
      return unpack_pairs(u, s);
    });
  }
  P->add("L:C", W(ctx->lCanti, "kbij"), one, W(ctx->lCb, "kbij"), false, 0.0);
  P->add("L:C", W(ctx->lCanti, "kbij"), mone, W(ctx->lCb, "kbji"), false, 1.0);
  P->contract("L:C", W(r1, "jc"), one, W(ctx->lCanti, "kbij"), false, V(ctx->J, "ibkc"), false, 1.0);
  // H^{ak}_{ci}: the ooov and X terms read H-bar before G-bar's diagonal is added to it
  P->contract("L:Hvoov", W(r1, "la"), mone, W(Hrb, "iakc"), false, V(ctx->ooov, "klic"), false, 1.0);
  P->contract("L:Hvoov", W(Xb, "liad"), one, W(Hrb, "iakc"), false, V(ctx->oovv, "klcd"), false, 0.0);
  // G^a_c = H^a_c + sum_kd V^{ak}_{cd} t^d_k - sum_k F^k_c t^a_k: the fov term here; the vovv term
  // rides on the diagonal k = i of H-bar (the adjoint of the trace the residual plan takes)
  P->contract("L:Gvv", W(r1, "ka"), mone, W(ctx->lGvvb, "ac"), false, V(ctx->fov, "kc"), false, 1.0);
  {
    z *hrb = Hrb, *gvb = ctx->lGvvb;
    P->custom("L:Gvv", [=](cudaStream_t s) { return diag_add_ik(hrb, o, v, gvb, 1.0, s); });
  }
  {
    // R1[i][d] += sum_{akc} H-bar[i][a][k][c] <ak||cd>, over blocks of a of <ak||cd> unpacked from vovv_pk
    const int64_t vb = ctx->vblk_rows, Pv_ = Pv;
    for (int64_t a0 = 0; a0 < v; a0 += vb) {
      ZGemmArgs g;
      g.M = o;
      g.N = v;
      g.K = std::min<int64_t>(vb, v - a0) * o * v;
      P->note_gemm(g);
    }
    z *vpk = ctx->vovv_pk, *vblk = ctx->vblk, *hrb = Hrb;
    P->custom("L:Hvoov:gemm", [ctx, o, v, vb, Pv_, vpk, vblk, hrb, r1](cudaStream_t s) {
      const GemmFn& gemm = ctx->lplan->gemm_fn();
      cudaError_t e = cudaSuccess;
      for (int64_t a0 = 0; a0 < v && e == cudaSuccess; a0 += vb) {
        const int64_t na = std::min<int64_t>(vb, v - a0);
        UnpackArgs u;  // vblk[(a - a0, k)][c][d] = <ak||cd>
        u.in = vpk + a0 * o * Pv_;
        u.out = vblk;
        u.n1 = na * o;
        u.n2 = v;
        u.beta = 0.0;
        e = unpack_pairs(u, s);
        if (e != cudaSuccess) break;
        ZGemmArgs g;  // R1[i][d] += sum_{(a,k,c)} H-bar[i][(a,k,c)] vblk[(a,k,c)][d]
        g.M = o;
        g.N = v;
        g.K = na * o * v;
        g.A = hrb + a0 * o * v;
        g.lda = (int64_t)v * o * v;
        g.B = vblk;
        g.ldb = v;
        g.C = r1;
        g.ldc = v;
        g.beta = zmake(1, 0);
        e = gemm(g, s);
      }
      return e;
    }, 8.0 * o * (double)v * o * v * v);
  }
  // X = 1/2 t2 + t1 t1
  P->add("L:X", W(G, "liad"), half, W(Xb, "liad"), false, 1.0);
  P->contract("L:X", W(r1, "la"), one, W(Xb, "liad"), false, W(t1, "id"), false, 1.0);
  P->contract("L:X", W(r1, "id"), one, W(Xb, "liad"), false, W(t1, "la"), false, 1.0);
  // H^k_c, G^k_i, H^k_i, G^a_c -> H^a_c
  P->contract("L:Hov", W(r1, "ld"), one, W(ctx->lHovb, "kc"), false, V(ctx->oovv, "klcd"), false, 1.0);
  P->add("L:Goo", W(ctx->lHoob, "ki"), one, W(ctx->lGoob, "ki"), false, 1.0);
  P->contract("L:Goo", W(r1, "lc"), mone, W(ctx->lGoob, "ki"), false, V(ctx->ooov, "klic"), false, 1.0);
  P->contract("L:Goo", W(r1, "ic"), mone, W(ctx->lGoob, "ki"), false, V(ctx->fov, "kc"), false, 1.0);
  P->contract("L:Hoo", W(taub, "licd"), half, W(ctx->lHoob, "ki"), false, V(ctx->oovv, "klcd"), false, 1.0);
  P->add("L:Gvv", W(ctx->lHvvb, "ac"), one, W(ctx->lGvvb, "ac"), false, 1.0);
  P->contract("L:Hvv", W(taub, "klda"), half, W(ctx->lHvvb, "ac"), false, V(ctx->oovv, "klcd"), false, 1.0);
  // tau = t2 + P^-_ij t1 t1
  P->add("L:tau", W(G, "ijab"), one, W(taub, "ijab"), false, 1.0);
  P->add("L:tau", W(zb, "ijab"), one, W(taub, "ijab"), false, 0.0);
  P->add("L:tau", W(zb, "ijab"), mone, W(taub, "jiab"), false, 1.0);
  P->contract("L:tau", W(r1, "ia"), one, W(zb, "ijab"), false, W(t1, "jb"), false, 1.0);
  P->contract("L:tau", W(r1, "jb"), one, W(zb, "ijab"), false, W(t1, "ia"), false, 1.0);
  // R2: the derivative with respect to each unique t^{ab}_{ij}, extended antisymmetrically
  P->add("L:R2", W(ctx->S2, "ijab"), one, W(G, "ijab"), false, 0.0);
  P->add("L:R2", W(ctx->S2, "ijab"), mone, W(G, "jiab"), false, 1.0);
  P->add("L:R2", W(ctx->S2, "ijab"), mone, W(G, "ijba"), false, 1.0);
  P->add("L:R2", W(ctx->S2, "ijab"), one, W(G, "jiba"), false, 1.0);

  if (P->status() != cudaSuccess) return set_err(ctx, CCSD_ERR_CUDA, "lambda plan: " + P->error());
  for (void* m : P->owned()) ctx->allocs.push_back(m);
  ctx->device_bytes += P->owned_bytes();
  P->owned().clear();
  CS(once(&ctx->lscratch, P->scratch_elems()));
  if (P->gemm_workspace_elems() > ctx->gemm_ws_elems) {
    CS(dalloc(ctx, &ctx->gemm_ws, P->gemm_workspace_elems()));
    ctx->gemm_ws_elems = P->gemm_workspace_elems();
  }
  if (ctx->use_split && P->aux_bytes() > ctx->split_ws_bytes) {
    uint8_t* w = nullptr;
    CS(dalloc(ctx, &w, P->aux_bytes()));
    ctx->split_ws = w;
    ctx->split_ws_bytes = P->aux_bytes();
  }
  ctx->lplan = holder.release();
  return CCSD_OK;
}

// The Lagrange one-body density (appendix "Working equations for Lagrange 1-body density matrix"),
// block by block; the occupied block is written transposed (the convention of the other three).
ccsd_status build_density_plan(ccsd_ctx* ctx) {
  const int o = ctx->o, v = ctx->v, n = ctx->n;
  CS(dalloc(ctx, &ctx->dgoo, (int64_t)o * o));
  CS(dalloc(ctx, &ctx->dgvo, (int64_t)v * o));
  CS(dalloc(ctx, &ctx->dgvv, (int64_t)v * v));
  CS(dalloc(ctx, &ctx->dq1, (int64_t)o * o));
  CS(dalloc(ctx, &ctx->dq2, (int64_t)o * o));
  CS(dalloc(ctx, &ctx->dq3, (int64_t)v * v));
  CS(dalloc(ctx, &ctx->dgam, (int64_t)n * n));
  CS(dalloc(ctx, &ctx->dgam2, (int64_t)n * n));
  std::unique_ptr<Plan, PlanDeleter> holder(new Plan(o, v, &ctx->dscratch, ctx->stream));
  Plan* D = holder.get();
  set_plan_gemm(ctx, D);
  const z one = zmake(1, 0), mone = zmake(-1, 0), half = zmake(0.5, 0), mhalf = zmake(-0.5, 0);
  auto W = [&](z* p, const char* lab) { return D->view(p, lab, false); };
  z *t1 = ctx->t1, *t2 = ctx->t2, *l1 = ctx->l1, *l2 = ctx->l2;
  // gamma_ij = 1/2 sum_mef t^{ef}_{im} lambda^{mj}_{ef} - sum_e t^e_i lambda^j_e, stored at [j][i]
  D->contract("D:oo", W(ctx->dgoo, "ji"), half, W(t2, "imef"), false, W(l2, "mjef"), false, 0.0);
  D->contract("D:oo", W(ctx->dgoo, "ji"), mone, W(t1, "ie"), false, W(l1, "je"), false, 1.0);
  // gamma_ai = t^a_i + sum_me lambda^m_e (t^{ae}_{im} - t^e_i t^a_m)
  //            - 1/2 sum_mnef lambda^{mn}_{ef} (t^{ef}_{in} t^a_m + t^e_i t^{af}_{mn})
  D->add("D:vo", W(ctx->dgvo, "ai"), one, W(t1, "ia"), false, 0.0);
  D->contract("D:vo", W(ctx->dgvo, "ai"), one, W(l1, "me"), false, W(t2, "imae"), false, 1.0);
  D->contract("D:vo", W(ctx->dq1, "mi"), one, W(l1, "me"), false, W(t1, "ie"), false, 0.0);
  D->contract("D:vo", W(ctx->dgvo, "ai"), mone, W(ctx->dq1, "mi"), false, W(t1, "ma"), false, 1.0);
  D->contract("D:vo", W(ctx->dq2, "mi"), one, W(l2, "mnef"), false, W(t2, "inef"), false, 0.0);
  D->contract("D:vo", W(ctx->dgvo, "ai"), mhalf, W(ctx->dq2, "mi"), false, W(t1, "ma"), false, 1.0);
  D->contract("D:vo", W(ctx->dq3, "ea"), one, W(l2, "mnef"), false, W(t2, "mnaf"), false, 0.0);
  D->contract("D:vo", W(ctx->dgvo, "ai"), mhalf, W(t1, "ie"), false, W(ctx->dq3, "ea"), false, 1.0);
  // gamma_ab = 1/2 sum_mne t^{ae}_{mn} lambda^{mn}_{be} + sum_m t^a_m lambda^m_b
  D->contract("D:vv", W(ctx->dgvv, "ab"), half, W(t2, "mnae"), false, W(l2, "mnbe"), false, 0.0);
  D->contract("D:vv", W(ctx->dgvv, "ab"), one, W(t1, "ma"), false, W(l1, "mb"), false, 1.0);
  if (D->status() != cudaSuccess) return set_err(ctx, CCSD_ERR_CUDA, "density plan: " + D->error());
  for (void* m : D->owned()) ctx->allocs.push_back(m);
  ctx->device_bytes += D->owned_bytes();
  D->owned().clear();
  CS(dalloc(ctx, &ctx->dscratch, D->scratch_elems()));
  if (D->gemm_workspace_elems() > ctx->gemm_ws_elems) {
    CS(dalloc(ctx, &ctx->gemm_ws, D->gemm_workspace_elems()));
    ctx->gemm_ws_elems = D->gemm_workspace_elems();
  }
  if (ctx->use_split && D->aux_bytes() > ctx->split_ws_bytes) {
    uint8_t* w = nullptr;
    CS(dalloc(ctx, &w, D->aux_bytes()));
    ctx->split_ws = w;
    ctx->split_ws_bytes = D->aux_bytes();
  }
  (void)n;
  ctx->dplan = holder.release();
  return CCSD_OK;
}

ccsd_status lambda_ready(ccsd_ctx* ctx) {
  if (ctx->opts.method != CCSD_METHOD_CCSD)
    return set_err(ctx, CCSD_ERR_UNSUPPORTED, "the Lambda equations are built for CCSD (method = CCSD)");
  if (!ctx->opts.store_w)
    return set_err(ctx, CCSD_ERR_UNSUPPORTED, "the Lambda equations need the stored <ab||cd> (store_w = 1)");
  if (!ctx->lplan) CS(build_lambda_plan(ctx));
  return CCSD_OK;
}

cudaError_t run_plan(Plan* P, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  for (auto& op : P->ops())
    if ((e = op.run(s)) != cudaSuccess) break;
  return e;
}

// The Lambda plan with an event at every op boundary (profile = 1); lambda_collect adds the
// elapsed times once the stream is synchronised.
void lambda_timers_init(ccsd_ctx* ctx) {
  if (!ctx->lev.empty()) return;
  const size_t n = ctx->lplan->ops().size();
  ctx->lev.resize(n + 1);
  for (auto& ev : ctx->lev) cudaEventCreate(&ev);
  ctx->ltsum.assign(n, 0.0);
}

cudaError_t run_lambda_timed(ccsd_ctx* ctx) {
  auto& ops = ctx->lplan->ops();
  lambda_timers_init(ctx);
  cudaError_t e = cudaEventRecordWithFlags(ctx->lev[0], ctx->stream, cudaEventRecordExternal);
  for (size_t k = 0; k < ops.size() && e == cudaSuccess; ++k) {
    e = ops[k].run(ctx->stream);
    if (e == cudaSuccess) e = cudaEventRecordWithFlags(ctx->lev[k + 1], ctx->stream, cudaEventRecordExternal);
  }
  return e;
}

// One Lambda iteration: the plan (timed or not), t <- t + R/D on the multipliers, norms, DIIS.
cudaError_t lambda_iteration_ops(ccsd_ctx* ctx, bool timed) {
  cudaError_t e = timed ? run_lambda_timed(ctx) : run_plan(ctx->lplan, ctx->stream);
  if (e == cudaSuccess)
    e = denom_update(ctx->l1, ctx->l2, ctx->S1, ctx->S2, ctx->dvec, ctx->o, ctx->v, ctx->opts.level_shift,
                     ctx->upd_partials, ctx->stream);
  if (e == cudaSuccess) e = norm_finalize(ctx->upd_partials, update_blocks(), ctx->stats, ctx->stream);
  if (e == cudaSuccess && ctx->opts.diis_dim > 0) e = diis_step(ctx->ldiis, ctx->l1, ctx->l2, ctx->S1, ctx->S2, ctx->stream);
  return e;
}

void lambda_collect(ccsd_ctx* ctx) {
  for (size_t k = 0; k + 1 < ctx->lev.size(); ++k) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->lev[k], ctx->lev[k + 1]) == cudaSuccess) ctx->ltsum[k] += ms;
  }
  cudaGetLastError();
  ctx->ltcount += 1;
}

// A block of an n x n matrix: out[(r0 + r) * n + c0 + c] = in[r * cols + c].
cudaError_t put_block(const z* in, int64_t rows, int64_t cols, z* out, int64_t n, int64_t r0, int64_t c0,
                      cudaStream_t s) {
  PermuteArgs a;
  a.rank = 2;
  a.dims[0] = rows;
  a.dims[1] = cols;
  a.istr[0] = cols;
  a.istr[1] = 1;
  a.ostr[0] = n;
  a.ostr[1] = 1;
  a.in = in;
  a.out = out + r0 * n + c0;
  return permute_add(a, s);
}

}  // namespace

extern "C" {

void ccsd_default_opts(ccsd_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->max_iter = 50;
  o->tol = 1e-10;
  o->norm = 0;
  o->diis_dim = 8;
  o->diis_start = 2;
  o->level_shift = 0.0;
  o->precision = CCSD_PREC_FP64;
  o->slices = 0;
  o->store_w = 1;
  o->profile = 0;
  o->stream = nullptr;
  o->split_min_flops = 1e8;
  o->df_block = 0;
  o->autotune = 0;
  o->digit_bits = 0;
  o->complex_4m = 0;
  o->split_budget = 0.0;
  o->method = CCSD_METHOD_CCSD;
  o->accelerator = CCSD_ACCEL_DIIS;
  o->diverge_iters = 8;
  o->diverge_factor = 1e3;
  o->vovv_block = 0;
  o->permute_cache_limit = 0.0;
}

int ccsd_divergence_index(const double* norms, int count, int iters, double factor) {
  if (count < 0 || (count > 0 && !norms)) return -1;
  ccsd_ctx::Growth g;
  for (int k = 0; k < count; ++k) {
    if (!std::isfinite(norms[k])) return 0;
    if (g.push(norms[k], iters, factor)) return k + 1;
  }
  return 0;
}

ccsd_status ccsd_create(int o, int v, const double* eps, const ccsd_z* fock, ccsd_int_kind kind, const ccsd_z* ints,
                        int naux, const ccsd_opts* opts, ccsd_ctx** out) {
  if (!out) return set_err(nullptr, CCSD_ERR_ARG, "out must not be NULL");
  *out = nullptr;
  ccsd_ctx* ctx = new ccsd_ctx();
  ccsd_status st = create_impl(o, v, eps, fock, kind, ints, naux, opts, ctx);
  if (st != CCSD_OK) {
    g_create_error = ctx->err;
    free_ctx(ctx);
    return st;
  }
  *out = ctx;
  return CCSD_OK;
}

ccsd_status ccsd_residual(ccsd_ctx* ctx, const ccsd_z* t1, const ccsd_z* t2, ccsd_z* r1, ccsd_z* r2, int on_device) {
  if (!ctx) return CCSD_ERR_ARG;
  if ((t1 == nullptr) != (t2 == nullptr)) return set_err(ctx, CCSD_ERR_ARG, "t1 and t2 must both be given or both NULL");
  const int64_t n1 = (int64_t)ctx->o * ctx->v, n2 = n1 * ctx->o * ctx->v;
  if (t1) {
    CK(backup_amplitudes(ctx, ctx->t1_save, ctx->t2_save));
    CS(copy_in(ctx, ctx->t1, t1, n1, on_device));
    CS(copy_in(ctx, ctx->t2, t2, n2, on_device));
  }
  const bool timed = ctx->opts.profile != 0;
  CK(run_ops(ctx, timed));
  if (ctx->use_split) CK(cudaMemcpyAsync(ctx->err_host, ctx->split_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  if (r1) CS(copy_out(ctx, r1, ctx->S1, n1, on_device));
  if (r2) CS(copy_out(ctx, r2, ctx->S2, n2, on_device));
  if (t1) {
    CK(restore_amplitudes(ctx, ctx->t1_save, ctx->t2_save));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  if (timed) collect_timers(ctx, ctx->plan->ops().size());
  if (ctx->use_split && *ctx->err_host)
    return set_err(ctx, CCSD_ERR_TIMEOUT, "a bounded wait in the tensor-core GEMM gave up");
  return CCSD_OK;
}

ccsd_status ccsd_iterate(ccsd_ctx* ctx, int max_iter, int* iters_done, double* res_norm) {
  if (!ctx) return CCSD_ERR_ARG;
  if (max_iter <= 0) max_iter = ctx->opts.max_iter;
  const bool timed = ctx->opts.profile != 0;
  if (!ctx->graph) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = iteration_ops(ctx, timed);
    cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return set_err(ctx, CCSD_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(g, nodes.data(), &nn);
    int kern = 0;
    for (auto nd : nodes) {
      cudaGraphNodeType ty;
      if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++kern;
    }
    ctx->kernels_per_iter = kern;
    e = cudaGraphInstantiate(&ctx->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return set_err(ctx, CCSD_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  int it = 0;
  double nrm = INFINITY;
  ccsd_status st = CCSD_ERR_NOT_CONVERGED;
  for (it = 1; it <= max_iter; ++it) {
    CK(cudaGraphLaunch(ctx->graph, ctx->stream));
    CK(cudaMemcpyAsync(ctx->stats_host, ctx->stats, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (ctx->use_split) CK(cudaMemcpyAsync(ctx->err_host, ctx->split_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->use_split && *ctx->err_host) {
      st = set_err(ctx, CCSD_ERR_TIMEOUT, "a bounded wait in the tensor-core GEMM gave up (code " +
                                               std::to_string(*ctx->err_host) + ")");
      break;
    }
    ctx->iterations_run += 1;
    if (timed) collect_timers(ctx, ctx->tnames.size());
    nrm = ctx->opts.norm == 1 ? ctx->stats_host[1] : ctx->stats_host[0];
    if (!std::isfinite(ctx->stats_host[0]) || !std::isfinite(ctx->stats_host[1])) {
      CK(restore_amplitudes(ctx, ctx->t1_prev, ctx->t2_prev));
      CK(cudaStreamSynchronize(ctx->stream));
      st = set_err(ctx, CCSD_ERR_DIVERGED, "non-finite amplitude update at iteration " + std::to_string(it));
      break;
    }
    if (nrm <= ctx->opts.tol) {
      st = CCSD_OK;
      break;
    }
    if (ctx->growth.push(nrm, ctx->opts.diverge_iters, ctx->opts.diverge_factor)) {
      st = set_err(ctx, CCSD_ERR_DIVERGED, "update norm rose in " + std::to_string(ctx->growth.up) +
                                               " consecutive iterations to " + std::to_string(nrm) + " (from " +
                                               std::to_string(ctx->growth.base) + ") at iteration " +
                                               std::to_string(it));
      break;
    }
  }
  if (it > max_iter) it = max_iter;
  if (iters_done) *iters_done = it;
  if (res_norm) *res_norm = nrm;
  if (st == CCSD_ERR_NOT_CONVERGED) set_err(ctx, st, "not converged in " + std::to_string(max_iter) + " iterations");
  return st;
}

ccsd_status ccsd_energy(ccsd_ctx* ctx, ccsd_z* e) {
  if (!ctx || !e) return ctx ? set_err(ctx, CCSD_ERR_ARG, "e must not be NULL") : CCSD_ERR_ARG;
  CK(energy_eval(ctx->fov, ctx->oovv, ctx->t1, ctx->t2, ctx->o, ctx->v, ctx->e_partials, ctx->e_dev, ctx->stream));
  CK(cudaMemcpyAsync(ctx->e_host, ctx->e_dev, sizeof(z), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  e->re = ctx->e_host->x;
  e->im = ctx->e_host->y;
  return CCSD_OK;
}

ccsd_status ccsd_triples(ccsd_ctx* ctx, int max_batch, double* out, double* pair_terms) {
  if (!ctx) return CCSD_ERR_ARG;
  if (!out) return set_err(ctx, CCSD_ERR_ARG, "out must not be NULL");
  if (max_batch < 0) return set_err(ctx, CCSD_ERR_ARG, "max_batch must be >= 0");
  const int o = ctx->o, v = ctx->v;
  std::vector<double> acc((size_t)o * o * 3, 0.0);
  if (o >= 3 && v >= 3) {
    const int64_t per = triples_batch_elems(v, ctx->use_split) * (int64_t)sizeof(z);
    int nb = max_batch;
    if (nb == 0) {
      size_t fr = 0, tot = 0;
      CK(cudaMemGetInfo(&fr, &tot));
      const int64_t budget = std::min<int64_t>((int64_t)(fr / 4), int64_t(8) << 30);
      nb = (int)std::max<int64_t>(1, std::min<int64_t>(o - 2, budget / per));
    }
    nb = std::min(nb, o - 2);
    // workspace of this call only, freed on every return path
    struct Scratch {
      std::vector<void*> p;
      ~Scratch() {
        for (void* q : p) cudaFree(q);
      }
      bool get(void** out, size_t bytes) {
        if (cudaMalloc(out, bytes) != cudaSuccess) {
          cudaGetLastError();
          return false;
        }
        p.push_back(*out);
        return true;
      }
    } mem;
    TriplesArgs a;
    a.o = o;
    a.v = v;
    a.t1 = ctx->t1;
    a.t2 = ctx->t2;
    a.oovv = ctx->oovv;
    a.ooov = ctx->ooov;
    a.vovv_pk = ctx->vovv_pk;
    a.fov = ctx->fov;
    a.d = ctx->dvec;
    a.max_batch = nb;
    void *t2pk = nullptr, *work = nullptr, *partials = nullptr, *pacc = nullptr, *dsf = nullptr;
    if (!mem.get(&t2pk, sizeof(z) * (size_t)o * o * ctx->Pv) || !mem.get(&work, (size_t)per * nb) ||
        !mem.get(&dsf, sizeof(float4) * (size_t)triples_dsf_elems(o, v)) ||
        !mem.get(&partials, sizeof(double) * (size_t)triples_partials(a)) ||
        !mem.get(&pacc, sizeof(double) * acc.size()))
      return set_err(ctx, CCSD_ERR_OOM, "triples workspace");
    a.t2pk = (z*)t2pk;
    a.work = (z*)work;
    a.dsf = (float4*)dsf;
    a.partials = (double*)partials;
    a.pair_acc = (double*)pacc;
    SliceSet SA, SB, SM, ST;
    int64_t setup_launches = 0;
    if (ctx->use_split) {
      // e-terms: digits of <ab||Le> for every L (rows L*P(v) + P over K = e, straight from vovv_pk)
      // and of t2 with its virtual labels swapped (rows (p*o + q)*v + c over K = e).
      // m-terms: digits of conj(<pq||ma>) (ooov with its last two labels swapped, rows
      // (p*o + q)*v + a over K = m) and of the pair-packed t2 with m last (rows L*P(v) + P(b,c)).
      void *t2T = nullptr, *sam = nullptr, *sbm = nullptr, *oT = nullptr, *tpT = nullptr, *smm = nullptr,
           *stm = nullptr;
      const int64_t ra = (int64_t)o * ctx->Pv, rb = (int64_t)o * o * v;
      if (!mem.get(&t2T, sizeof(z) * (size_t)rb * v) || !mem.get(&sam, (size_t)slice_bytes(ra, v, ctx->split)) ||
          !mem.get(&sbm, (size_t)slice_bytes(rb, v, ctx->split)) || !mem.get(&oT, sizeof(z) * (size_t)rb * o) ||
          !mem.get(&tpT, sizeof(z) * (size_t)ra * o) || !mem.get(&smm, (size_t)slice_bytes(rb, o, ctx->split)) ||
          !mem.get(&stm, (size_t)slice_bytes(ra, o, ctx->split)))
        return set_err(ctx, CCSD_ERR_OOM, "triples digit sets");
      const int64_t d_t2[4] = {o, o, v, v};
      const int pT[4] = {0, 1, 3, 2};
      CK(permute4(ctx->t2, d_t2, pT, (z*)t2T, zmake(1, 0), 0.0, 0, ctx->stream));
      CK(make_slices(ctx->vovv_pk, ra, v, ra, 1, 1, ctx->split, SA, sam, ctx->stream));
      CK(make_slices((const z*)t2T, rb, v, v, 0, 0, ctx->split, SB, sbm, ctx->stream));
      const int64_t d_ooov[4] = {o, o, o, v};
      CK(permute4(ctx->ooov, d_ooov, pT, (z*)oT, zmake(1, 0), 0.0, 0, ctx->stream));
      CK(make_slices((const z*)oT, rb, o, o, 0, 1, ctx->split, SM, smm, ctx->stream));
      // the packed t2 goes through the triples' own buffer first
      CK(pack_pairs(ctx->t2, (z*)t2pk, (int64_t)o * o, v, 0, ctx->stream));
      const int64_t d_pk[4] = {o, o, ctx->Pv, 1};
      const int pP[4] = {0, 2, 1, 3};
      CK(permute4((const z*)t2pk, d_pk, pP, (z*)tpT, zmake(1, 0), 0.0, 0, ctx->stream));
      CK(make_slices((const z*)tpT, ra, o, o, 0, 0, ctx->split, ST, stm, ctx->stream));
      a.sa = &SA;
      a.sb = &SB;
      a.sm = &SM;
      a.st = &ST;
      a.split_err = ctx->split_err;
      setup_launches = 1 + 3 + 3 + 1 + 3 + 1 + 1 + 3;
    }
    TriplesTimer timer;
    if (ctx->opts.profile) a.timer = &timer;
    CK(cudaMemsetAsync(pacc, 0, sizeof(double) * acc.size(), ctx->stream));
    CK(triples_eval(a, ctx->stream));
    CK(cudaMemcpyAsync(acc.data(), pacc, sizeof(double) * acc.size(), cudaMemcpyDeviceToHost, ctx->stream));
    if (ctx->use_split) CK(cudaMemcpyAsync(ctx->err_host, ctx->split_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->use_split && *ctx->err_host)
      return set_err(ctx, CCSD_ERR_TIMEOUT, "a bounded wait in the tensor-core GEMM gave up (code " +
                                                std::to_string(*ctx->err_host) + ")");
    ctx->tri_batch = nb;
    ctx->tri_batches = a.batches;
    ctx->tri_launches = setup_launches + a.launches;
    ctx->tri_ms[0] = ctx->tri_ms[1] = ctx->tri_ms[2] = 0.0;
    if (a.timer) CK(timer.sums(ctx->tri_ms));
  } else {
    ctx->tri_batch = ctx->tri_batches = ctx->tri_launches = 0;
    ctx->tri_ms[0] = ctx->tri_ms[1] = ctx->tri_ms[2] = 0.0;
  }
  // per-pair contributions to the three energies, and their sums in pair order
  out[0] = out[1] = out[2] = 0.0;
  for (int i = 0; i < o; ++i)
    for (int j = 0; j < o; ++j) {
      const double* s = &acc[((size_t)i * o + j) * 3];
      const double c[3] = {-s[0], -s[0] - s[1], -s[0] + s[2]};
      for (int m = 0; m < 3; ++m) {
        out[m] += c[m];
        if (pair_terms) pair_terms[((size_t)i * o + j) * 3 + m] = c[m];
      }
    }
  return CCSD_OK;
}

ccsd_status ccsd_lambda_residual(ccsd_ctx* ctx, const ccsd_z* l1, const ccsd_z* l2, ccsd_z* r1, ccsd_z* r2,
                                 int on_device) {
  if (!ctx) return CCSD_ERR_ARG;
  if ((l1 == nullptr) != (l2 == nullptr)) return set_err(ctx, CCSD_ERR_ARG, "l1 and l2 must both be given or both NULL");
  CS(lambda_ready(ctx));
  const int64_t n1 = (int64_t)ctx->o * ctx->v, n2 = n1 * ctx->o * ctx->v;
  if (l1) {
    CS(copy_in(ctx, ctx->l1, l1, n1, on_device));
    CS(copy_in(ctx, ctx->l2, l2, n2, on_device));
  }
  CK(run_ops(ctx, false));  // the residual plan's intermediates at the current amplitudes
  CK(run_plan(ctx->lplan, ctx->stream));
  if (ctx->use_split) CK(cudaMemcpyAsync(ctx->err_host, ctx->split_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  if (r1) CS(copy_out(ctx, r1, ctx->S1, n1, on_device));
  if (r2) CS(copy_out(ctx, r2, ctx->S2, n2, on_device));
  CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->use_split && *ctx->err_host)
    return set_err(ctx, CCSD_ERR_TIMEOUT, "a bounded wait in the tensor-core GEMM gave up");
  return CCSD_OK;
}

ccsd_status ccsd_lambda_iterate(ccsd_ctx* ctx, int max_iter, int* iters_done, double* res_norm) {
  if (!ctx) return CCSD_ERR_ARG;
  CS(lambda_ready(ctx));
  if (max_iter <= 0) max_iter = ctx->opts.max_iter;
  CK(run_ops(ctx, false));  // the intermediates stay fixed: the amplitudes do not change
  int it = 0;
  double nrm = INFINITY;
  ccsd_status st = CCSD_ERR_NOT_CONVERGED;
  const bool timed = ctx->opts.profile != 0;
  ctx->lgrowth.reset();
  if (!ctx->lgraph) {
    // the iteration is captured once and replayed (its buffers never move)
    if (timed) lambda_timers_init(ctx);
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = lambda_iteration_ops(ctx, timed);
    cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return set_err(ctx, CCSD_ERR_CUDA,
                     std::string("Lambda graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(g, nodes.data(), &nn);
    ctx->lkernels_per_iter = 0;
    for (auto nd : nodes) {
      cudaGraphNodeType ty;
      if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++ctx->lkernels_per_iter;
    }
    e = cudaGraphInstantiate(&ctx->lgraph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess)
      return set_err(ctx, CCSD_ERR_CUDA, std::string("Lambda graph instantiate: ") + cudaGetErrorString(e));
  }
  for (it = 1; it <= max_iter; ++it) {
    CK(cudaGraphLaunch(ctx->lgraph, ctx->stream));
    CK(cudaMemcpyAsync(ctx->stats_host, ctx->stats, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (ctx->use_split) CK(cudaMemcpyAsync(ctx->err_host, ctx->split_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->use_split && *ctx->err_host) {
      st = set_err(ctx, CCSD_ERR_TIMEOUT, "a bounded wait in the tensor-core GEMM gave up");
      break;
    }
    ctx->lambda_iterations += 1;
    if (timed) lambda_collect(ctx);
    nrm = ctx->opts.norm == 1 ? ctx->stats_host[1] : ctx->stats_host[0];
    if (!std::isfinite(ctx->stats_host[0]) || !std::isfinite(ctx->stats_host[1])) {
      st = set_err(ctx, CCSD_ERR_DIVERGED, "non-finite multiplier update at iteration " + std::to_string(it));
      break;
    }
    if (nrm <= ctx->opts.tol) {
      st = CCSD_OK;
      break;
    }
    if (ctx->lgrowth.push(nrm, ctx->opts.diverge_iters, ctx->opts.diverge_factor)) {
      st = set_err(ctx, CCSD_ERR_DIVERGED, "multiplier update norm rose in " + std::to_string(ctx->lgrowth.up) +
                                               " consecutive iterations at iteration " + std::to_string(it));
      break;
    }
  }
  if (it > max_iter) it = max_iter;
  if (iters_done) *iters_done = it;
  if (res_norm) *res_norm = nrm;
  if (st == CCSD_ERR_NOT_CONVERGED) set_err(ctx, st, "not converged in " + std::to_string(max_iter) + " iterations");
  return st;
}

ccsd_status ccsd_get_lambda(ccsd_ctx* ctx, ccsd_z* l1, ccsd_z* l2, int on_device) {
  if (!ctx) return CCSD_ERR_ARG;
  CS(lambda_ready(ctx));
  const int64_t n1 = (int64_t)ctx->o * ctx->v, n2 = n1 * ctx->o * ctx->v;
  if (l1) CS(copy_out(ctx, l1, ctx->l1, n1, on_device));
  if (l2) CS(copy_out(ctx, l2, ctx->l2, n2, on_device));
  CK(cudaStreamSynchronize(ctx->stream));
  return CCSD_OK;
}

ccsd_status ccsd_density(ccsd_ctx* ctx, ccsd_z* gamma, int symmetrize) {
  if (!ctx) return CCSD_ERR_ARG;
  if (!gamma) return set_err(ctx, CCSD_ERR_ARG, "gamma must not be NULL");
  CS(lambda_ready(ctx));
  if (!ctx->dplan) CS(build_density_plan(ctx));
  const int o = ctx->o, v = ctx->v, n = ctx->n;
  CK(run_plan(ctx->dplan, ctx->stream));
  CK(put_block(ctx->dgoo, o, o, ctx->dgam, n, 0, 0, ctx->stream));
  CK(put_block(ctx->l1, o, v, ctx->dgam, n, 0, o, ctx->stream));
  CK(put_block(ctx->dgvo, v, o, ctx->dgam, n, o, 0, ctx->stream));
  CK(put_block(ctx->dgvv, v, v, ctx->dgam, n, o, o, ctx->stream));
  const z* out = ctx->dgam;
  if (symmetrize) {
    // the Hermitian part: 1/2 gamma + 1/2 gamma^+
    PermuteArgs a;
    a.rank = 2;
    a.dims[0] = n;
    a.dims[1] = n;
    a.istr[0] = n;
    a.istr[1] = 1;
    a.ostr[0] = n;
    a.ostr[1] = 1;
    a.in = ctx->dgam;
    a.out = ctx->dgam2;
    a.alpha = zmake(0.5, 0);
    CK(permute_add(a, ctx->stream));
    a.istr[0] = 1;
    a.istr[1] = n;
    a.conj = 1;
    a.beta = 1.0;
    CK(permute_add(a, ctx->stream));
    out = ctx->dgam2;
  }
  CK(cudaMemcpyAsync(gamma, out, sizeof(z) * (size_t)n * n, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return CCSD_OK;
}

ccsd_status ccsd_get_amplitudes(ccsd_ctx* ctx, ccsd_z* t1, ccsd_z* t2, int on_device) {
  if (!ctx) return CCSD_ERR_ARG;
  const int64_t n1 = (int64_t)ctx->o * ctx->v, n2 = n1 * ctx->o * ctx->v;
  if (t1) CS(copy_out(ctx, t1, ctx->t1, n1, on_device));
  if (t2) CS(copy_out(ctx, t2, ctx->t2, n2, on_device));
  CK(cudaStreamSynchronize(ctx->stream));
  return CCSD_OK;
}

ccsd_status ccsd_set_amplitudes(ccsd_ctx* ctx, const ccsd_z* t1, const ccsd_z* t2, int on_device) {
  if (!ctx) return CCSD_ERR_ARG;
  if (!t1 || !t2) return set_err(ctx, CCSD_ERR_ARG, "t1 and t2 must not be NULL");
  const int64_t n1 = (int64_t)ctx->o * ctx->v, n2 = n1 * ctx->o * ctx->v;
  CS(copy_in(ctx, ctx->t1, t1, n1, on_device));
  CS(copy_in(ctx, ctx->t2, t2, n2, on_device));
  if (ctx->opts.diis_dim > 0) CK(diis_reset(ctx->diis, ctx->stream));
  ctx->growth.reset();
  CK(cudaStreamSynchronize(ctx->stream));
  return CCSD_OK;
}

ccsd_status ccsd_get_tensor(ccsd_ctx* ctx, const char* name, ccsd_z* out, size_t count, int on_device) {
  if (!ctx || !name || !out) return ctx ? set_err(ctx, CCSD_ERR_ARG, "NULL argument") : CCSD_ERR_ARG;
  const int64_t o = ctx->o, v = ctx->v, oo = o * o, vv = v * v, ov = o * v;
  const z* src = nullptr;
  int64_t cnt = 0;
  std::string nm(name);
  if (nm == "tau") { src = ctx->tau; cnt = oo * vv; }
  else if (nm == "Hvv") { src = ctx->Hvv; cnt = vv; }
  else if (nm == "Gvv") { src = ctx->Gvv; cnt = vv; }
  else if (nm == "Hoo") { src = ctx->Hoo; cnt = oo; }
  else if (nm == "Goo") { src = ctx->Goo; cnt = oo; }
  else if (nm == "Hov") { src = ctx->Hov; cnt = ov; }
  else if (nm == "Hvoov") { src = ctx->Hr; cnt = oo * vv; }
  else if (nm == "C") { src = ctx->C; cnt = ov * oo; }
  else if (nm == "A") {
    UnpackArgs u;
    u.in = ctx->Apk;
    u.out = ctx->Yoooo;
    u.n1 = o;
    u.n2 = o;
    u.unpack_rows = 1;
    u.beta = 0.0;
    CK(unpack_pairs(u, ctx->stream));
    src = ctx->Yoooo;
    cnt = oo * oo;
  } else if (nm == "ladder") {
    UnpackArgs u;
    u.in = ctx->Lpk;
    u.out = ctx->R;
    u.n1 = o;
    u.n2 = v;
    u.unpack_rows = 1;
    u.beta = 0.0;
    CK(unpack_pairs(u, ctx->stream));
    src = ctx->R;
    cnt = oo * vv;
  } else {
    return set_err(ctx, CCSD_ERR_ARG, "unknown tensor name '" + nm + "'");
  }
  if ((int64_t)count != cnt) return set_err(ctx, CCSD_ERR_ARG, "count must be " + std::to_string(cnt) + " for " + nm);
  CS(copy_out(ctx, out, src, cnt, on_device));
  CK(cudaStreamSynchronize(ctx->stream));
  return CCSD_OK;
}

ccsd_status ccsd_timings(ccsd_ctx* ctx, const char** names, double* ms, int cap, int* n) {
  if (!ctx) return CCSD_ERR_ARG;
  const int cnt = ctx->tcount > 0 ? (int)ctx->tnames.size() : 0;
  const int lcnt = (ctx->lplan && ctx->ltcount > 0) ? (int)ctx->ltsum.size() : 0;
  if (n) *n = cnt + lcnt;
  if (cap <= 0) return CCSD_OK;
  for (int k = 0; k < cnt && k < cap; ++k) {
    if (names) names[k] = ctx->tnames[k].c_str();
    if (ms) ms[k] = ctx->tsum[k] / ctx->tcount;
  }
  // then the Lambda plan's ops, per timed Lambda iteration
  for (int k = 0; k < lcnt && cnt + k < cap; ++k) {
    if (names) names[cnt + k] = ctx->lplan->ops()[k].name.c_str();
    if (ms) ms[cnt + k] = ctx->ltsum[k] / ctx->ltcount;
  }
  std::fill(ctx->tsum.begin(), ctx->tsum.end(), 0.0);
  ctx->tcount = 0;
  std::fill(ctx->ltsum.begin(), ctx->ltsum.end(), 0.0);
  ctx->ltcount = 0;
  return CCSD_OK;
}

ccsd_status ccsd_query(const ccsd_ctx* ctx, const char* key, double* value) {
  if (!ctx || !key || !value) return CCSD_ERR_ARG;
  const std::string k(key);
  if (k == "kernels_per_iteration") *value = ctx->kernels_per_iter;
  else if (k == "device_bytes") *value = (double)ctx->device_bytes;
  else if (k == "plan_scratch_bytes") *value = 16.0 * (double)ctx->plan->scratch_elems();
  else if (k == "plan_cached_bytes") *value = (double)ctx->plan_cached_bytes;
  else if (k == "gemm_workspace_bytes") *value = 16.0 * (double)ctx->gemm_ws_elems;
  else if (k == "split_workspace_bytes") *value = (double)ctx->split_ws_bytes;
  else if (k == "diis_bytes") *value = 2.0 * 16.0 * (double)ctx->diis.m * (double)ctx->diis.L;
  else if (k == "iterations_run") *value = (double)ctx->iterations_run;
  else if (k == "plan_ops") *value = (double)ctx->plan->ops().size();
  else if (k == "lambda_iterations") *value = (double)ctx->lambda_iterations;
  else if (k == "lambda_kernels_per_iteration") *value = (double)ctx->lkernels_per_iter;
  else if (k.rfind("lambda_op_ms:", 0) == 0) {
    // average device time per timed Lambda iteration of the ops with that name (profile = 1)
    const std::string nm = k.substr(13);
    double sum = 0.0;
    if (ctx->lplan && ctx->ltcount > 0)
      for (size_t i = 0; i < ctx->lplan->ops().size() && i < ctx->ltsum.size(); ++i)
        if (ctx->lplan->ops()[i].name == nm) sum += ctx->ltsum[i];
    *value = ctx->ltcount > 0 ? sum / (double)ctx->ltcount : 0.0;
  }
  else if (k == "triples_batch") *value = (double)ctx->tri_batch;
  else if (k == "triples_batches") *value = (double)ctx->tri_batches;
  else if (k == "triples_launches") *value = (double)ctx->tri_launches;
  else if (k == "triples_egemm_ms") *value = ctx->tri_ms[0];
  else if (k == "triples_mgemm_ms") *value = ctx->tri_ms[1];
  else if (k == "triples_energy_ms") *value = ctx->tri_ms[2];
  else if (k == "o") *value = ctx->o;
  else if (k == "v") *value = ctx->v;
  else return CCSD_ERR_ARG;
  return CCSD_OK;
}

ccsd_status ccsd_zgemm(int precision, int transA, int conjA, int transB, int conjB, long long M, long long N,
                       long long K, ccsd_z alpha, const ccsd_z* A, long long lda, const ccsd_z* B, long long ldb,
                       ccsd_z beta, ccsd_z* C, long long ldc, ccsd_z* workspace, size_t ws_elems, int cfg,
                       void* stream) {
  ccsd_ctx* ctx = nullptr;
  if (M < 0 || N < 0 || K < 0 || !A || !B || !C) return set_err(ctx, CCSD_ERR_ARG, "ccsd_zgemm: bad sizes or NULL");
  if (cfg > 6) return set_err(ctx, CCSD_ERR_ARG, "ccsd_zgemm: cfg must be < 7");
  if (precision != CCSD_PREC_FP64) return set_err(ctx, CCSD_ERR_UNSUPPORTED, "ccsd_zgemm: precision not built");
  ZGemmArgs g;
  g.M = M;
  g.N = N;
  g.K = K;
  g.A = (const z*)A;
  g.lda = lda;
  g.B = (const z*)B;
  g.ldb = ldb;
  g.C = (z*)C;
  g.ldc = ldc;
  g.alpha = zmake(alpha.re, alpha.im);
  g.beta = zmake(beta.re, beta.im);
  g.transA = transA != 0;
  g.transB = transB != 0;
  g.conjA = conjA != 0;
  g.conjB = conjB != 0;
  g.ws = (z*)workspace;
  g.ws_elems = workspace ? (int64_t)ws_elems : 0;
  cudaStream_t st = (cudaStream_t)stream;
  CK(zgemm_f64(g, st, cfg));
  CK(cudaStreamSynchronize(st));
  return CCSD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched systems: one context per system, one fork/join CUDA graph per batch
// iteration over the still-active systems.
// ---------------------------------------------------------------------------
struct ccsd_batch {
  std::vector<ccsd_ctx*> sys;
  cudaStream_t main = nullptr;
  bool own_main = false;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraphExec_t graph = nullptr;
  std::vector<int> active, in_graph, iters, status;
  std::vector<double> norms;
  double* stats_host = nullptr;  // pinned, 2 per system
  int* err_host = nullptr;       // pinned, 1 per system
  std::string err;
};

namespace {

ccsd_status batch_err(ccsd_batch* b, ccsd_status st, const std::string& msg) {
  b->err = msg;
  return st;
}

void batch_free(ccsd_batch* b) {
  if (!b) return;
  if (b->main) cudaStreamSynchronize(b->main);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (ccsd_ctx* c : b->sys) free_ctx(c);
  for (auto e : b->join) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->stats_host) cudaFreeHost(b->stats_host);
  if (b->err_host) cudaFreeHost(b->err_host);
  if (b->own_main && b->main) cudaStreamDestroy(b->main);
  delete b;
}

// Capture: fork from the batch stream to every active system's stream, run its iteration
// (residual, update, norms, DIIS) and copy its norms to pinned memory, join back.
ccsd_status batch_build_graph(ccsd_batch* b) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  b->in_graph = b->active;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->main, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) e = cudaEventRecord(b->fork, b->main);
  for (int k : b->in_graph) {
    ccsd_ctx* c = b->sys[k];
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, b->fork, 0);
    if (e == cudaSuccess) e = iteration_ops(c, false);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->stats_host + 2 * k, c->stats, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && c->use_split)
      e = cudaMemcpyAsync(b->err_host + k, c->split_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->join[k], c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->main, b->join[k], 0);
  }
  cudaError_t e2 = cudaStreamEndCapture(b->main, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return batch_err(b, CCSD_ERR_CUDA, std::string("batch graph capture: ") +
                                            cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return batch_err(b, CCSD_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
  return CCSD_OK;
}

}  // namespace

extern "C" {

ccsd_status ccsd_batch_create(int nsys, const int* o, const int* v, const double* const* eps,
                              const ccsd_z* const* B, const int* naux, const ccsd_opts* opts, ccsd_batch** out) {
  if (!out) return set_err(nullptr, CCSD_ERR_ARG, "out must not be NULL");
  *out = nullptr;
  if (nsys < 1 || !o || !v || !eps || !B || !naux) return set_err(nullptr, CCSD_ERR_ARG, "bad batch arguments");
  ccsd_opts base;
  if (opts) base = *opts;
  else ccsd_default_opts(&base);
  ccsd_batch* b = new ccsd_batch();
  if (base.stream) {
    b->main = (cudaStream_t)base.stream;
  } else if (cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking) == cudaSuccess) {
    b->own_main = true;
  } else {
    batch_free(b);
    return set_err(nullptr, CCSD_ERR_CUDA, "batch stream");
  }
  TuneCache cache;  // shared tile choices across systems of equal GEMM shapes
  g_tune_cache = &cache;
  for (int k = 0; k < nsys; ++k) {
    ccsd_opts ok = base;
    ok.stream = nullptr;  // every system on its own stream
    ok.profile = 0;
    ccsd_ctx* c = nullptr;
    ccsd_status st = ccsd_create(o[k], v[k], eps[k], nullptr, CCSD_INT_DF, B[k], naux[k], &ok, &c);
    if (st != CCSD_OK) {
      g_tune_cache = nullptr;
      const std::string msg = "system " + std::to_string(k) + ": " + g_create_error;
      batch_free(b);
      return set_err(nullptr, st, msg);
    }
    b->sys.push_back(c);
  }
  g_tune_cache = nullptr;
  b->join.resize(nsys);
  bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  for (auto& e : b->join) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaMallocHost(&b->stats_host, 2 * nsys * sizeof(double)) == cudaSuccess;
  ok = ok && cudaMallocHost(&b->err_host, nsys * sizeof(int)) == cudaSuccess;
  if (!ok) {
    batch_free(b);
    return set_err(nullptr, CCSD_ERR_CUDA, "batch events / pinned memory");
  }
  for (int k = 0; k < nsys; ++k) b->err_host[k] = 0;
  b->active.resize(nsys);
  for (int k = 0; k < nsys; ++k) b->active[k] = k;
  b->iters.assign(nsys, 0);
  b->status.assign(nsys, CCSD_ERR_NOT_CONVERGED);
  b->norms.assign(nsys, INFINITY);
  *out = b;
  return CCSD_OK;
}

ccsd_status ccsd_batch_iterate(ccsd_batch* b, int max_iter, int* iters_done, double* res_norm, int* status) {
  if (!b) return CCSD_ERR_ARG;
  const int nsys = (int)b->sys.size();
  if (max_iter <= 0) max_iter = b->sys[0]->opts.max_iter;
  for (int it = 0; it < max_iter && !b->active.empty(); ++it) {
    if (!b->graph || b->in_graph != b->active) {
      ccsd_status st = batch_build_graph(b);
      if (st != CCSD_OK) return st;
    }
    cudaError_t e = cudaGraphLaunch(b->graph, b->main);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->main);
    if (e != cudaSuccess) return batch_err(b, CCSD_ERR_CUDA, std::string("batch iteration: ") + cudaGetErrorString(e));
    std::vector<int> still;
    for (int k : b->active) {
      ccsd_ctx* c = b->sys[k];
      b->iters[k] += 1;
      c->iterations_run += 1;
      const double mx = b->stats_host[2 * k], l2 = b->stats_host[2 * k + 1];
      const double nrm = c->opts.norm == 1 ? l2 : mx;
      b->norms[k] = nrm;
      if (c->use_split && b->err_host[k]) {
        b->status[k] = CCSD_ERR_TIMEOUT;
      } else if (!std::isfinite(mx) || !std::isfinite(l2)) {
        restore_amplitudes(c, c->t1_prev, c->t2_prev);
        cudaStreamSynchronize(c->stream);
        b->status[k] = CCSD_ERR_DIVERGED;
      } else if (nrm <= c->opts.tol) {
        b->status[k] = CCSD_OK;
      } else if (c->growth.push(nrm, c->opts.diverge_iters, c->opts.diverge_factor)) {
        b->status[k] = CCSD_ERR_DIVERGED;
      } else {
        still.push_back(k);
      }
    }
    b->active = still;
  }
  bool all_ok = true;
  for (int k = 0; k < nsys; ++k) {
    if (iters_done) iters_done[k] = b->iters[k];
    if (res_norm) res_norm[k] = b->norms[k];
    if (status) status[k] = b->status[k];
    all_ok = all_ok && b->status[k] == CCSD_OK;
  }
  if (!all_ok) return batch_err(b, CCSD_ERR_NOT_CONVERGED, "not every system converged");
  return CCSD_OK;
}

ccsd_status ccsd_batch_energy(ccsd_batch* b, ccsd_z* e) {
  if (!b || !e) return CCSD_ERR_ARG;
  for (size_t k = 0; k < b->sys.size(); ++k) {
    ccsd_status st = ccsd_energy(b->sys[k], e + k);
    if (st != CCSD_OK) return batch_err(b, st, "system " + std::to_string(k) + ": " + b->sys[k]->err);
  }
  return CCSD_OK;
}

ccsd_status ccsd_batch_get_amplitudes(ccsd_batch* b, int k, ccsd_z* t1, ccsd_z* t2, int on_device) {
  if (!b || k < 0 || k >= (int)b->sys.size()) return CCSD_ERR_ARG;
  return ccsd_get_amplitudes(b->sys[k], t1, t2, on_device);
}

const char* ccsd_batch_last_error(const ccsd_batch* b) { return b ? b->err.c_str() : g_create_error.c_str(); }

void ccsd_batch_destroy(ccsd_batch* b) { batch_free(b); }

const char* ccsd_last_error(const ccsd_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

void ccsd_destroy(ccsd_ctx* ctx) { free_ctx(ctx); }

}  // extern "C"
