// Contraction planner (see plan.h) and the GEMV used when one side of a
// contraction has no free index.
#include <algorithm>
#include <sstream>

#include "ops.h"
#include "plan.h"

namespace ccsd {
namespace {

__global__ void zgemv_rowmajor_kernel(int64_t R, int64_t K, z alpha, const z* __restrict__ M, int64_t ld, int conjM,
                                      const z* __restrict__ x, int conjx, double beta, z* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); r < R; r += warps) {
    double ar = 0.0, ai = 0.0;
    const z* row = M + r * ld;
    for (int64_t k = lane; k < K; k += 32) {
      z m = row[k], xv = x[k];
      if (conjM) m.y = -m.y;
      if (conjx) xv.y = -xv.y;
      ar += m.x * xv.x - m.y * xv.y;
      ai += m.x * xv.y + m.y * xv.x;
    }
    for (int off = 16; off > 0; off >>= 1) {
      ar += __shfl_down_sync(0xffffffffu, ar, off);
      ai += __shfl_down_sync(0xffffffffu, ai, off);
    }
    if (lane == 0) {
      z acc = zmul(alpha, make_double2(ar, ai));
      y[r] = beta != 0.0 ? make_double2(acc.x + beta * y[r].x, acc.y + beta * y[r].y) : acc;
    }
  }
}

// Column-major matrix: 32 consecutive outputs per block (one per lane, coalesced loads along a
// row of M), the K range shared by the block's 32 warps (warp w takes k = w, w + 32, ...); the
// warps' partial sums are added in shared memory in warp order, so the result is reproducible.
constexpr int kColWarps = 32;
__global__ void __launch_bounds__(32 * kColWarps) zgemv_colmajor_kernel(int64_t R, int64_t K, z alpha,
                                                                       const z* __restrict__ M, int64_t ld, int conjM,
                                                                       const z* __restrict__ x, int conjx, double beta,
                                                                       z* __restrict__ y) {
  __shared__ double part[kColWarps][32][2];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t r0 = (int64_t)blockIdx.x * 32; r0 < R; r0 += (int64_t)gridDim.x * 32) {
    const int64_t r = r0 + lane;
    double ar = 0.0, ai = 0.0;
    if (r < R) {
#pragma unroll 4
      for (int64_t k = w; k < K; k += kColWarps) {
        z m = M[k * ld + r], xv = x[k];
        if (conjM) m.y = -m.y;
        if (conjx) xv.y = -xv.y;
        ar += m.x * xv.x - m.y * xv.y;
        ai += m.x * xv.y + m.y * xv.x;
      }
    }
    part[w][lane][0] = ar;
    part[w][lane][1] = ai;
    __syncthreads();
    if (w == 0 && r < R) {
      double sr = 0.0, si = 0.0;
      for (int q = 0; q < kColWarps; ++q) {
        sr += part[q][lane][0];
        si += part[q][lane][1];
      }
      z acc = zmul(alpha, make_double2(sr, si));
      y[r] = beta != 0.0 ? make_double2(acc.x + beta * y[r].x, acc.y + beta * y[r].y) : acc;
    }
    __syncthreads();
  }
}

bool has(const std::string& s, char c) { return s.find(c) != std::string::npos; }

std::vector<int64_t> rowmajor_strides(const std::vector<int64_t>& dims) {
  std::vector<int64_t> st(dims.size());
  int64_t s = 1;
  for (int k = (int)dims.size() - 1; k >= 0; --k) {
    st[k] = s;
    s *= dims[k];
  }
  return st;
}

}  // namespace

cudaError_t zgemv(int64_t R, int64_t K, z alpha, const z* M, int64_t ld, int rowmajor, int conjM, const z* x,
                  int conjx, double beta, z* y, cudaStream_t s) {
  if (R <= 0) return cudaSuccess;
  if (rowmajor) {
    zgemv_rowmajor_kernel<<<grid_for(R * 32, 256), 256, 0, s>>>(R, K, alpha, M, ld, conjM, x, conjx, beta, y);
  } else {
    zgemv_colmajor_kernel<<<grid_for(R, 32), 32 * kColWarps, 0, s>>>(R, K, alpha, M, ld, conjM, x, conjx, beta, y);
  }
  return cudaGetLastError();
}

int64_t Plan::dim_of(char c) const {
  if (c >= 'i' && c <= 'n') return o_;
  if (c >= 'a' && c <= 'h') return v_;
  return -1;
}

T Plan::view(z* p, const std::string& lab, bool cnst) const {
  Ptr q;
  q.direct = p;
  return view(q, lab, cnst);
}

T Plan::view(Ptr p, const std::string& lab, bool cnst) const {
  T t;
  t.p = p;
  t.lab = lab;
  t.cnst = cnst;
  for (char c : lab) t.dims.push_back(dim_of(c));
  return t;
}

void Plan::fail(const std::string& msg, cudaError_t e) {
  if (status_ == cudaSuccess) {
    status_ = e;
    error_ = msg;
  }
}

Ptr Plan::temp(int64_t elems) {
  Ptr p;
  p.base = scratch_base_;
  p.off = scratch_off_;
  scratch_off_ += (elems + 15) / 16 * 16;  // keep 256-byte alignment
  scratch_peak_ = std::max(scratch_peak_, scratch_off_);
  return p;
}

void Plan::custom(const std::string& name, std::function<cudaError_t(cudaStream_t)> fn, double flops) {
  ops_.push_back(Op{name, std::move(fn), flops});
}

void Plan::gemm(const std::string& name, const ZGemmArgs& g) {
  if (wsfn_) ws_peak_ = std::max(ws_peak_, wsfn_(g));
  if (auxfn_) aux_peak_ = std::max(aux_peak_, auxfn_(g));
  GemmFn fn = gemm_;
  auto cfg = std::make_shared<int>(-1);
  auto args = std::make_shared<ZGemmArgs>(g);
  ops_.push_back(Op{name, [fn, args, cfg](cudaStream_t s) {
                      ZGemmArgs h = *args;
                      h.cfg = *cfg;
                      return fn(h, s);
                    }, 8.0 * g.M * g.N * g.K * g.batch, cfg, args});
}

void Plan::add(const std::string& name, const T& C, z alpha, const T& A, bool conjA, double beta) {
  if (C.lab.size() != A.lab.size()) return fail(name + ": add rank mismatch " + C.lab + " <- " + A.lab);
  PermuteArgs a;
  a.rank = (int)C.lab.size();
  auto ast = rowmajor_strides(A.dims), cst = rowmajor_strides(C.dims);
  for (int d = 0; d < a.rank; ++d) {
    size_t pos = A.lab.find(C.lab[d]);
    if (pos == std::string::npos) return fail(name + ": label missing in add");
    if (A.dims[pos] != C.dims[d]) return fail(name + ": dim mismatch in add");
    a.dims[d] = C.dims[d];
    a.istr[d] = ast[pos];
    a.ostr[d] = cst[d];
  }
  a.alpha = alpha;
  a.beta = beta;
  a.conj = conjA ? 1 : 0;
  Ptr pin = A.p, pout = C.p;
  ops_.push_back(Op{name, [a, pin, pout](cudaStream_t s) {
                      PermuteArgs b = a;
                      b.in = pin.get();
                      b.out = pout.get();
                      return permute_add(b, s);
                    }});
}

T Plan::permuted(const T& src, const std::string& lab, bool conj, const std::string& name) {
  T out;
  out.lab = lab;
  for (char c : lab) out.dims.push_back(src.dims[src.lab.find(c)]);
  if (src.cnst && src.p.direct && src.size() * (int64_t)sizeof(z) <= cache_limit_) {
    std::ostringstream key;
    key << (const void*)src.p.direct << ":" << src.lab << ">" << lab << (conj ? "*" : "");
    auto it = const_cache_.find(key.str());
    if (it != const_cache_.end()) return it->second;
    void* mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, std::max<int64_t>(src.size(), 1) * sizeof(z));
    if (e != cudaSuccess) {
      fail(name + ": cudaMalloc for cached permutation", e);
      return out;
    }
    owned_.push_back(mem);
    owned_bytes_ += std::max<int64_t>(src.size(), 1) * (int64_t)sizeof(z);
    out.p.direct = (z*)mem;
    out.cnst = true;
    // run the permutation once, now
    Plan tmp(o_, v_, scratch_base_, setup_);
    tmp.add(name + ":cache", out, zmake(1.0, 0.0), src, conj, 0.0);
    e = tmp.ops()[0].run(setup_);
    if (e != cudaSuccess) fail(name + ": cached permutation launch", e);
    const_cache_[key.str()] = out;
    return out;
  }
  out.p = temp(src.size());
  add(name + ":perm", out, zmake(1.0, 0.0), src, conj, 0.0);
  return out;
}

void Plan::contract(const std::string& name, const T& C, z alpha, const T& A0, bool cA0, const T& B0, bool cB0,
                    double beta) {
  const int64_t mark = scratch_off_;
  std::string FA, FB, K;
  for (char c : C.lab) {
    if (has(A0.lab, c) && !has(B0.lab, c)) FA += c;
    else if (has(B0.lab, c) && !has(A0.lab, c)) FB += c;
    else return fail(name + ": output label '" + std::string(1, c) + "' must be in exactly one operand");
  }
  for (char c : A0.lab)
    if (!has(C.lab, c)) {
      if (!has(B0.lab, c)) return fail(name + ": summed label only in A");
      K += c;
    }
  for (char c : B0.lab)
    if (!has(C.lab, c) && !has(A0.lab, c)) return fail(name + ": summed label only in B");
  if (K.empty()) return fail(name + ": outer products are not planned");

  bool direct = false, swap = false;
  if (C.lab == FA + FB) direct = true;
  else if (C.lab == FB + FA) { direct = true; swap = true; }
  const T& A = swap ? B0 : A0;
  const T& B = swap ? A0 : B0;
  bool cA = swap ? cB0 : cA0, cB = swap ? cA0 : cB0;
  const std::string fa = swap ? FB : FA, fb = swap ? FA : FB;

  auto others = [](const std::string& s, const std::string& free) {
    std::string r;
    for (char c : s)
      if (!has(free, c)) r += c;
    return r;
  };
  const std::string cands[2] = {others(A.lab, fa), others(B.lab, fb)};
  int best = -1;
  int64_t best_cost = -1;
  bool bestAt = false, bestBt = false, bestAok = false, bestBok = false;
  for (int ci = 0; ci < 2; ++ci) {
    const std::string& kx = cands[ci];
    bool Aok = false, At = false, Bok = false, Bt = false;
    if (A.lab == fa + kx) Aok = true;
    else if (A.lab == kx + fa) { Aok = true; At = true; }
    if (B.lab == kx + fb) Bok = true;
    else if (B.lab == fb + kx) { Bok = true; Bt = true; }
    int64_t cost = (Aok ? 0 : (A.cnst ? 1 : A.size())) + (Bok ? 0 : (B.cnst ? 1 : B.size()));
    if (best < 0 || cost < best_cost) {
      best = ci;
      best_cost = cost;
      bestAt = At;
      bestBt = Bt;
      bestAok = Aok;
      bestBok = Bok;
    }
  }
  const std::string kx = cands[best];
  T Ap = A, Bp = B;
  bool tA = bestAt, tB = bestBt;
  if (!bestAok) {
    Ap = permuted(A, fa + kx, cA, name);
    cA = false;
    tA = false;
  }
  if (!bestBok) {
    // [free][summed] (K contiguous): the layout the digit slicer of the split path reads fastest
    Bp = permuted(B, fb + kx, cB, name);
    cB = false;
    tB = true;
  }
  int64_t M = 1, N = 1, KK = 1;
  for (char c : fa) M *= A.dims[A.lab.find(c)];
  for (char c : fb) N *= B.dims[B.lab.find(c)];
  for (char c : kx) KK *= A.dims[A.lab.find(c)];

  T Cp = C;
  const bool need_out_perm = !direct;
  if (need_out_perm) {
    Cp.lab = fa + fb;
    Cp.dims.clear();
    for (char c : Cp.lab) Cp.dims.push_back(C.dims[C.lab.find(c)]);
    Cp.p = temp(C.size());
  }
  const z galpha = need_out_perm ? zmake(1.0, 0.0) : alpha;
  const double gbeta = need_out_perm ? 0.0 : beta;
  if (status_ != cudaSuccess) return;

  const Ptr pa = Ap.p, pb = Bp.p, pc = Cp.p;
  const double flops = 8.0 * (double)M * N * KK;
  if (N == 1 || M == 1) {
    // GEMV: the side with a single free element is the vector.
    if (N == 1) {
      const int rowmajor = tA ? 0 : 1;
      const int64_t ld = tA ? M : KK;
      const int cm = cA, cx = cB;
      ops_.push_back(Op{name + ":gemv", [=](cudaStream_t s) {
                          return zgemv(M, KK, galpha, pa.get(), ld, rowmajor, cm, pb.get(), cx, gbeta, pc.get(), s);
                        }, flops});
    } else {
      const int rowmajor = tB ? 1 : 0;
      const int64_t ld = tB ? KK : N;
      const int cm = cB, cx = cA;
      ops_.push_back(Op{name + ":gemv", [=](cudaStream_t s) {
                          return zgemv(N, KK, galpha, pb.get(), ld, rowmajor, cm, pa.get(), cx, gbeta, pc.get(), s);
                        }, flops});
    }
  } else {
    ZGemmArgs g;
    g.M = M;
    g.N = N;
    g.K = KK;
    g.lda = tA ? M : KK;
    g.ldb = tB ? KK : N;
    g.ldc = N;
    g.transA = tA;
    g.transB = tB;
    g.conjA = cA;
    g.conjB = cB;
    g.alpha = galpha;
    g.beta = zmake(gbeta, 0.0);
    if (wsfn_) ws_peak_ = std::max(ws_peak_, wsfn_(g));
    if (auxfn_) aux_peak_ = std::max(aux_peak_, auxfn_(g));
    GemmFn fn = gemm_;
    auto cfg = std::make_shared<int>(-1);
    auto args = std::make_shared<ZGemmArgs>(g);
    ops_.push_back(Op{name + ":gemm", [=](cudaStream_t s) {
                        ZGemmArgs h = *args;
                        h.A = pa.get();
                        h.B = pb.get();
                        h.C = pc.get();
                        h.cfg = *cfg;
                        return fn(h, s);
                      }, flops, cfg, args});
  }
  if (need_out_perm) add(name + ":out", C, alpha, Cp, false, beta);
  scratch_off_ = mark;
}

}  // namespace ccsd
