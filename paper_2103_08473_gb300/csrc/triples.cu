// Perturbative triples corrections E(+T), E((T)), E(-T) at converged CCSD amplitudes
// (appendix "Working equations for perturbative Triples", Eqs. W-term, Z-term, Y-term,
// 4order-term and 5order-term).
//
// Readings (the same as the CPU oracle's): the integrals of W are the Hermitian partners
// <ab||ie> and <am||jk> of the printed <ie||ab> and <jk||am>; D = e_a + e_b + e_c - e_i - e_j - e_k
// over the real diagonal of f; E(+T) = -sum |X|^2 / D; the (T) term is -sum Re(X Z) / D with
// Z = conj(<Phi_3| V T1 + F T2 |Phi_0>); the -T term is +sum Re(X conj(Y)). X is the cyclic sum of
// W over the virtual labels. Sums run over unique i<j<k, a<b<c (the appendix's full sums / 36).
//
// Work plan. For every occupied pair i<j the triples (i, j, k), k > j, are taken in batches of
// consecutive k. For a batch, six batched FP64 GEMMs form W in two antisymmetry-packed parts:
//   E[t][P(a,b)][c] = sum_{(L;pq) in (i;jk),(j;ki),(k;ij)} sum_e <ab||Le> t^{ec}_{pq}
//                    (rows of the packed <eL||ab>, conjugated, times t2[p][q] as [e][c]),
//   M[t][a][P(b,c)] = sum_{(pq;L) in (ij;k),(jk;i),(ki;j)} sum_m <am||pq> t^{bc}_{Lm}
//                    (<pq||ma> conjugated, times the pair-packed t2[L] as [m][P(b,c)]).
// The e-terms are antisymmetric in (a,b) and the m-terms in (b,c), so each part is stored packed
// and the GEMMs do half the work of the full contractions. One fused kernel then reads the six
// elements that make X at each unique (a<b<c), builds Z, Y and D on the fly from t1, t2, <ij||ab>,
// f_ov and the orbital energies, and reduces the three energy terms. Per-block partial sums go to a
// fixed slot and are added to the pair's accumulator in a fixed order, so the result is
// reproducible run to run.

#include "triples.h"

#include <nvtx3/nvToolsExt.h>

#include "ops.h"
#include "zgemm.h"

namespace ccsd {

namespace {

constexpr int kTriplesThreads = 256;

struct EnergyArgs {
  int o = 0, v = 0;
  int64_t Pv = 0;
  int i = 0, j = 0, k0 = 0, nk = 0;
  const z *E = nullptr, *M = nullptr;
  // split precision: the products of the second layout, E2[P(a,b)][t][c] and M2[a][t][P(b,c)]
  const z *E2 = nullptr, *M2 = nullptr;
  const z *t1 = nullptr, *t2 = nullptr, *oovv = nullptr, *fov = nullptr;
  // the same four in double-single form (float4 per complex: re hi, re lo, im hi, im lo)
  const float4 *t1f = nullptr, *t2f = nullptr, *oovvf = nullptr, *fovf = nullptr;
  const double* d = nullptr;
  double* partials = nullptr;  // gridDim.x * 3
};

// ---- double-single arithmetic --------------------------------------------------------
// A value is the unevaluated sum hi + lo of two floats (|lo| <= ulp(hi) / 2), about 48 bits.
// Knuth's two-sum and the fused-multiply-add form of Dekker's two-product make each step's
// rounding error exact, so sums and products carry ~2^-47 relative error. The fifth-order
// terms Z and Y (and t1's determinant) are formed this way on the FP32 pipe, which this chip
// has ~64x more of than FP64; X, D and the energy sums stay in FP64.
struct dsf {
  float h, l;
};
struct dsc {
  dsf r, i;
};
__device__ __forceinline__ dsf ds_quick(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dsf ds_add(dsf x, dsf y) {
  const float s = __fadd_rn(x.h, y.h);
  const float bb = __fsub_rn(s, x.h);
  const float e = __fadd_rn(__fsub_rn(x.h, __fsub_rn(s, bb)), __fsub_rn(y.h, bb));
  return ds_quick(s, __fadd_rn(e, __fadd_rn(x.l, y.l)));
}
__device__ __forceinline__ dsf ds_neg(dsf x) { return {-x.h, -x.l}; }
__device__ __forceinline__ dsf ds_mul(dsf x, dsf y) {
  const float p = __fmul_rn(x.h, y.h);
  float e = __fmaf_rn(x.h, y.h, -p);
  e = __fmaf_rn(x.h, y.l, e);
  e = __fmaf_rn(x.l, y.h, e);
  return ds_quick(p, e);
}
__device__ __forceinline__ dsc dsc_load(const float4* p) {
  const float4 q = *p;
  return {{q.x, q.y}, {q.z, q.w}};
}
__device__ __forceinline__ dsc dsc_add(dsc a, dsc b) { return {ds_add(a.r, b.r), ds_add(a.i, b.i)}; }
__device__ __forceinline__ dsc dsc_sub(dsc a, dsc b) { return {ds_add(a.r, ds_neg(b.r)), ds_add(a.i, ds_neg(b.i))}; }
__device__ __forceinline__ dsc dsc_mul(dsc a, dsc b) {
  return {ds_add(ds_mul(a.r, b.r), ds_neg(ds_mul(a.i, b.i))), ds_add(ds_mul(a.r, b.i), ds_mul(a.i, b.r))};
}
__device__ __forceinline__ dsc dsc_conj_mul(dsc a, dsc b) {  // conj(a) * b
  return {ds_add(ds_mul(a.r, b.r), ds_mul(a.i, b.i)), ds_add(ds_mul(a.r, b.i), ds_neg(ds_mul(a.i, b.r)))};
}
__device__ __forceinline__ z dsc_to_z(dsc a) {
  return make_double2((double)a.r.h + (double)a.r.l, (double)a.i.h + (double)a.i.l);
}

// float4 (re hi, re lo, im hi, im lo) of every complex element: the double-single copies the
// energy kernel reads.
__global__ void to_double_single_kernel(const z* __restrict__ in, float4* __restrict__ out, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const z x = in[e];
    const float rh = __double2float_rn(x.x), ih = __double2float_rn(x.y);
    out[e] = make_float4(rh, __double2float_rn(x.x - (double)rh), ih, __double2float_rn(x.y - (double)ih));
  }
}

__global__ void __launch_bounds__(kTriplesThreads) triples_energy_kernel(EnergyArgs g) {
  const int64_t v = g.v, o = g.o, Pv = g.Pv, nk = g.nk;
  // one warp per row (t, P(a,b)), decoded once; its lanes walk c = b+1 .. v-1, the unique
  // triples a<b<c of the row
  const int lane = threadIdx.x & 31;
  const int64_t rows = nk * Pv;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double s4 = 0.0, s5 = 0.0, s5m = 0.0;
  for (int64_t row = w0; row < rows; row += nw) {
    const int64_t pab = row % Pv;
    const int t = (int)(row / Pv);
    int64_t a, b;
    pair_decode(pab, v, a, b);
    for (int64_t c = b + 1 + lane; c < v; c += 32) {
      const int k = g.k0 + t;
      const z* E = g.E + (int64_t)t * Pv * v;
      const z* M = g.M + (int64_t)t * v * Pv;
      const int64_t pbc = pair_index(b, c, v), pac = pair_index(a, c, v);
      // X = W^{abc} + W^{bca} + W^{cab}, W = E (antisymmetric in its first two virtual labels)
      //                                  + M (antisymmetric in its last two)
      z X = E[pab * v + c];
      X = zadd(X, E[pbc * v + a]);
      X = zsub(X, E[pac * v + b]);
      X = zadd(X, M[a * Pv + pbc]);
      X = zsub(X, M[b * Pv + pac]);
      X = zadd(X, M[c * Pv + pab]);
      if (g.E2) {
        const z* E2 = g.E2 + (int64_t)t * v;  // [P][t][c]: row stride nk * v
        const z* M2 = g.M2 + (int64_t)t * Pv;  // [a][t][P]: row stride nk * Pv
        X = zadd(X, E2[pab * nk * v + c]);
        X = zadd(X, E2[pbc * nk * v + a]);
        X = zsub(X, E2[pac * nk * v + b]);
        X = zadd(X, M2[a * nk * Pv + pbc]);
        X = zsub(X, M2[b * nk * Pv + pac]);
        X = zadd(X, M2[c * nk * Pv + pab]);
      }
      const double D = g.d[o + a] + g.d[o + b] + g.d[o + c] - g.d[g.i] - g.d[g.j] - g.d[k];
      // Z and Y summed over the cyclic orders of the occupied and of the virtual labels
      const int occ[3] = {g.i, g.j, k};
      const int vir[3] = {a, b, c};
      dsc Zd = {{0.f, 0.f}, {0.f, 0.f}}, Yd = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
      for (int s = 0; s < 3; ++s) {
        const int64_t p = occ[s], q = occ[(s + 1) % 3], rr = occ[(s + 2) % 3];
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          const int64_t x = vir[u], y = vir[(u + 1) % 3], zz = vir[(u + 2) % 3];
          const int64_t idx = ((p * o + q) * v + x) * v + y;
          const dsc w = dsc_load(g.oovvf + idx), tt = dsc_load(g.t2f + idx);
          const dsc a1 = dsc_load(g.t1f + rr * v + zz), f = dsc_load(g.fovf + rr * v + zz);
          // <pq||xy> conj(t^z_r) + conj(t^{xy}_{pq}) f_rz
          Zd = dsc_add(Zd, dsc_add(dsc_conj_mul(a1, w), dsc_conj_mul(tt, f)));
          // t^{xy}_{pq} t^z_r
          Yd = dsc_add(Yd, dsc_mul(tt, a1));
        }
      }
      // the determinant of t1 over rows (i, j, k) and columns (a, b, c)
      dsc m[3][3];
#pragma unroll
      for (int rr = 0; rr < 3; ++rr)
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) m[rr][cc] = dsc_load(g.t1f + (int64_t)occ[rr] * v + vir[cc]);
      const dsc c0 = dsc_sub(dsc_mul(m[1][1], m[2][2]), dsc_mul(m[1][2], m[2][1]));
      const dsc c1 = dsc_sub(dsc_mul(m[1][0], m[2][2]), dsc_mul(m[1][2], m[2][0]));
      const dsc c2 = dsc_sub(dsc_mul(m[1][0], m[2][1]), dsc_mul(m[1][1], m[2][0]));
      Yd = dsc_add(Yd, dsc_add(dsc_sub(dsc_mul(m[0][0], c0), dsc_mul(m[0][1], c1)), dsc_mul(m[0][2], c2)));
      const z Zs = dsc_to_z(Zd), Ys = dsc_to_z(Yd);
      const double inv = 1.0 / D;
      s4 += (X.x * X.x + X.y * X.y) * inv;
      s5 += (X.x * Zs.x - X.y * Zs.y) * inv;
      s5m += X.x * Ys.x + X.y * Ys.y;
    }
  }
  // fixed-shape block reduction
  __shared__ double red[3][kTriplesThreads / 32];
  const int warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    s4 += __shfl_down_sync(0xffffffffu, s4, off);
    s5 += __shfl_down_sync(0xffffffffu, s5, off);
    s5m += __shfl_down_sync(0xffffffffu, s5m, off);
  }
  if (lane == 0) {
    red[0][warp] = s4;
    red[1][warp] = s5;
    red[2][warp] = s5m;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double acc = 0.0;
    for (int w = 0; w < kTriplesThreads / 32; ++w) acc += red[threadIdx.x][w];
    g.partials[(int64_t)blockIdx.x * 3 + threadIdx.x] = acc;
  }
}

// pair_acc[0..2] += the block partials, summed in block order by one thread per term.
__global__ void triples_accumulate_kernel(const double* __restrict__ partials, int nblocks,
                                          double* __restrict__ pair_acc) {
  const int m = threadIdx.x;
  if (m >= 3) return;
  double acc = 0.0;
  for (int b = 0; b < nblocks; ++b) acc += partials[(int64_t)b * 3 + m];
  pair_acc[m] += acc;
}

int energy_grid(int64_t work) {
  int64_t g = (work + kTriplesThreads - 1) / kTriplesThreads;
  const int64_t cap = 152 * 8;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

int64_t triples_partials(const TriplesArgs& a) {
  (void)a;
  return 152 * 8 * 3;
}

int64_t triples_dsf_elems(int o, int v) {
  const int64_t ov = (int64_t)o * v;
  return 2 * ov + 2 * ov * ov;
}

int64_t triples_batch_elems(int v, bool split) { return (split ? 4 : 2) * pair_count(v) * (int64_t)v; }

cudaError_t triples_eval(TriplesArgs& a, cudaStream_t s) {
  const int o = a.o, v = a.v;
  if (o < 3 || v < 3) return cudaSuccess;
  const int64_t Pv = pair_count(v), v2 = (int64_t)v * v;
  const int64_t part = Pv * v;  // elements of E (and of M) per triple
  z* Ebuf = a.work;
  z* Mbuf = a.work + part * a.max_batch;
  z* E2buf = a.sa ? a.work + 2 * part * a.max_batch : nullptr;
  z* M2buf = a.sa ? a.work + 3 * part * a.max_batch : nullptr;
  cudaError_t e = pack_pairs(a.t2, a.t2pk, (int64_t)o * o, v, 0, s);
  if (e != cudaSuccess) return e;
  a.launches += 1;
  // double-single copies for the energy kernel: t1, f_ov, t2, <ij||ab>
  const int64_t ov = (int64_t)o * v, o2v2 = ov * ov;
  float4 *t1f = a.dsf, *fovf = a.dsf + ov, *t2f = a.dsf + 2 * ov, *oovvf = a.dsf + 2 * ov + o2v2;
  to_double_single_kernel<<<grid_for(ov, kTriplesThreads), kTriplesThreads, 0, s>>>(a.t1, t1f, ov);
  to_double_single_kernel<<<grid_for(ov, kTriplesThreads), kTriplesThreads, 0, s>>>(a.fov, fovf, ov);
  to_double_single_kernel<<<grid_for(o2v2, kTriplesThreads), kTriplesThreads, 0, s>>>(a.t2, t2f, o2v2);
  to_double_single_kernel<<<grid_for(o2v2, kTriplesThreads), kTriplesThreads, 0, s>>>(a.oovv, oovvf, o2v2);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  a.launches += 4;
  const z minus1 = make_double2(-1.0, 0.0), one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
  for (int i = 0; i < o - 2; ++i) {
    for (int j = i + 1; j < o - 1; ++j) {
      for (int k0 = j + 1; k0 < o; k0 += a.max_batch) {
        const int nk = (o - k0) < a.max_batch ? (o - k0) : a.max_batch;
        ++a.batches;
        if (a.timer && (e = a.timer->mark(s)) != cudaSuccess) return e;
        // ---- e-terms: E[t][P(a,b)][c] over k = k0 + t
        if (a.sa) {
          nvtxRangePushA("triples_eterms");  // a profiler selects these launches by this range
          // one split GEMM per term over the whole batch, C = -A_L B_pq^T over K = e:
          //   (k; ij): rows L = k of <eL||ab> for every k of the batch against t2[i][j]
          //            -> E[t][P(a,b)][c];
          //   (i; jk) and (j; ki) = -(j; ik): rows L = i (L = j) against t2[j][k] (t2[i][k]) for
          //            every k of the batch -> E2[P(a,b)][t][c]
          const int64_t ij = (int64_t)i * o + j;
          e = split_gemm(slice_rows(*a.sa, (int64_t)k0 * Pv, (int64_t)nk * Pv), slice_rows(*a.sb, ij * v, v), Ebuf,
                         v, minus1, zero, a.split_err, nullptr, 0, s);
          if (e == cudaSuccess)
            e = split_gemm(slice_rows(*a.sa, (int64_t)i * Pv, Pv),
                           slice_rows(*a.sb, ((int64_t)j * o + k0) * v, (int64_t)nk * v), E2buf, (int64_t)nk * v,
                           minus1, zero, a.split_err, nullptr, 0, s);
          if (e == cudaSuccess)
            e = split_gemm(slice_rows(*a.sa, (int64_t)j * Pv, Pv),
                           slice_rows(*a.sb, ((int64_t)i * o + k0) * v, (int64_t)nk * v), E2buf, (int64_t)nk * v,
                           one, one, a.split_err, nullptr, 0, s);
          nvtxRangePop();
          if (e != cudaSuccess) return e;
          a.launches += 3;
        } else {
          ZGemmArgs g;
          g.M = Pv;
          g.N = v;
          g.K = v;
          g.batch = nk;
          g.transA = 1;
          g.conjA = 1;
          g.lda = (int64_t)o * Pv;
          g.ldb = v;
          g.C = Ebuf;
          g.ldc = v;
          g.sC = part;
          g.alpha = minus1;  // <ab||Le> = -conj(<eL||ab>)
          // (i; jk): A = rows L = i, B = t2[j][k]
          g.A = a.vovv_pk + (int64_t)i * Pv;
          g.sA = 0;
          g.B = a.t2 + ((int64_t)j * o + k0) * v2;
          g.sB = v2;
          g.beta = zero;
          if ((e = zgemm_f64(g, s)) != cudaSuccess) return e;
          // (j; ki): A = rows L = j, B = t2[k][i]
          g.A = a.vovv_pk + (int64_t)j * Pv;
          g.B = a.t2 + ((int64_t)k0 * o + i) * v2;
          g.sB = (int64_t)o * v2;
          g.beta = one;
          if ((e = zgemm_f64(g, s)) != cudaSuccess) return e;
          // (k; ij): A = rows L = k, B = t2[i][j]
          g.A = a.vovv_pk + (int64_t)k0 * Pv;
          g.sA = Pv;
          g.B = a.t2 + ((int64_t)i * o + j) * v2;
          g.sB = 0;
          if ((e = zgemm_f64(g, s)) != cudaSuccess) return e;
          a.launches += 3;
        }
        if (a.timer && (e = a.timer->mark(s)) != cudaSuccess) return e;
        // ---- m-terms: M[t][a][P(b,c)]
        if (a.sm) {
          // one split GEMM per term over the batch, C = -A_pq B_L^T over K = m:
          //   (jk; i) and (ki; j) = -(ik; j): rows (j,k) ((i,k)) of conj(<pq||ma>) for every k of
          //            the batch against the packed t2[i] (t2[j]) -> M[t][a][P(b,c)];
          //   (ij; k): rows (i,j) against the packed t2[k] of every k -> M2[a][t][P(b,c)]
          const int64_t ij = (int64_t)i * o + j;
          e = split_gemm(slice_rows(*a.sm, ((int64_t)j * o + k0) * v, (int64_t)nk * v),
                         slice_rows(*a.st, (int64_t)i * Pv, Pv), Mbuf, Pv, minus1, zero, a.split_err, nullptr, 0, s);
          if (e == cudaSuccess)
            e = split_gemm(slice_rows(*a.sm, ((int64_t)i * o + k0) * v, (int64_t)nk * v),
                           slice_rows(*a.st, (int64_t)j * Pv, Pv), Mbuf, Pv, one, one, a.split_err, nullptr, 0, s);
          if (e == cudaSuccess)
            e = split_gemm(slice_rows(*a.sm, ij * v, v), slice_rows(*a.st, (int64_t)k0 * Pv, (int64_t)nk * Pv),
                           M2buf, (int64_t)nk * Pv, minus1, zero, a.split_err, nullptr, 0, s);
          if (e != cudaSuccess) return e;
        } else {
        ZGemmArgs h;
        h.M = v;
        h.N = Pv;
        h.K = o;
        h.batch = nk;
        h.transA = 1;
        h.conjA = 1;
        h.lda = v;
        h.ldb = Pv;
        h.C = Mbuf;
        h.ldc = Pv;
        h.sC = part;
        h.alpha = minus1;  // <am||pq> = -conj(<pq||ma>)
        const int64_t ov = (int64_t)o * v;
        // (ij; k): A = ooov[i][j], B = t2pk[k]
        h.A = a.ooov + ((int64_t)i * o + j) * ov;
        h.sA = 0;
        h.B = a.t2pk + (int64_t)k0 * o * Pv;
        h.sB = (int64_t)o * Pv;
        h.beta = zero;
        if ((e = zgemm_f64(h, s)) != cudaSuccess) return e;
        // (jk; i): A = ooov[j][k], B = t2pk[i]
        h.A = a.ooov + ((int64_t)j * o + k0) * ov;
        h.sA = ov;
        h.B = a.t2pk + (int64_t)i * o * Pv;
        h.sB = 0;
        h.beta = one;
        if ((e = zgemm_f64(h, s)) != cudaSuccess) return e;
        // (ki; j): A = ooov[k][i], B = t2pk[j]
        h.A = a.ooov + ((int64_t)k0 * o + i) * ov;
        h.sA = (int64_t)o * ov;
        h.B = a.t2pk + (int64_t)j * o * Pv;
        if ((e = zgemm_f64(h, s)) != cudaSuccess) return e;
        }
        if (a.timer && (e = a.timer->mark(s)) != cudaSuccess) return e;
        // ---- energies of the batch
        EnergyArgs q;
        q.o = o;
        q.v = v;
        q.Pv = Pv;
        q.i = i;
        q.j = j;
        q.k0 = k0;
        q.nk = nk;
        q.E = Ebuf;
        q.M = Mbuf;
        q.E2 = E2buf;
        q.M2 = M2buf;
        q.t1 = a.t1;
        q.t2 = a.t2;
        q.oovv = a.oovv;
        q.fov = a.fov;
        q.t1f = t1f;
        q.fovf = fovf;
        q.t2f = t2f;
        q.oovvf = oovvf;
        q.d = a.d;
        q.partials = a.partials;
        const int grid = energy_grid((int64_t)nk * Pv * 32);
        triples_energy_kernel<<<grid, kTriplesThreads, 0, s>>>(q);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        triples_accumulate_kernel<<<1, 32, 0, s>>>(a.partials, grid, a.pair_acc + ((int64_t)i * o + j) * 3);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        a.launches += 3 + 2;  // the m-term GEMMs, the energy kernel and its accumulation
        if (a.timer && (e = a.timer->mark(s)) != cudaSuccess) return e;
      }
    }
  }
  return cudaSuccess;
}

}  // namespace ccsd
