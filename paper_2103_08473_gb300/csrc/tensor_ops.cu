// HBM-bound kernels of libccsd: index permutations (the P^-_pq antisymmetrisers
// and the reorders of the transpose-transpose-GEMM-transpose contractions),
// antisymmetric pair packing, tau, the denominator ("Jacobi") update with its
// norms, the energy, and DIIS. All reductions are two-stage with a fixed order,
// so every result is bit-reproducible run to run.
#include "ops.h"
#include "zgemm.h"

namespace ccsd {
namespace {

constexpr int kThreads = 256;
constexpr int kUpdateBlocks = 152 * 4;
constexpr int kEnergyBlocks = 152 * 2;
constexpr int kDiisBlocks = 152 * 2;


// ---- permutations ----------------------------------------------------------

// out = alpha op(v) + beta out for one element. The common cases (alpha = +-1 with beta 0 or 1)
// flip sign bits with integer operations and add at most once per part: the FP64 pipe of this
// chip is narrow, and the general complex form costs eight FP64 operations per element.
__device__ __forceinline__ double flip_sign(double x, unsigned long long m) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)m);
}
__device__ __forceinline__ void perm_put(z* o, z v, int mode, unsigned long long sx, unsigned long long sy, z alpha,
                                         double beta, int conj) {
  if (mode == 1) {
    *o = make_double2(flip_sign(v.x, sx), flip_sign(v.y, sy));
  } else if (mode == 2) {
    const z w = *o;
    *o = make_double2(w.x + flip_sign(v.x, sx), w.y + flip_sign(v.y, sy));
  } else {
    if (conj) v.y = -v.y;
    *o = beta != 0.0 ? zaxpby(alpha, v, beta, *o) : zmul(alpha, v);
  }
}

// Output-ordered elementwise copy: coalesced when the innermost output dim is also
// innermost in the input.
__global__ void permute_direct_kernel(PermuteArgs g, int64_t total) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = e, io = 0, oo = 0;
    for (int d = g.rank - 1; d >= 0; --d) {
      int64_t c = r % g.dims[d];
      r /= g.dims[d];
      io += c * g.istr[d];
      oo += c * g.ostr[d];
    }
    perm_put(g.out + oo, g.in[io], g.mode, g.sx, g.sy, g.alpha, g.beta, g.conj);
  }
}

// Division by a divisor fixed at launch, as a multiply and a shift (Granlund and Montgomery,
// "Division by invariant integers using multiplication", 1994): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, n / d = (umulhi(m, n) + n) >> l for every n < 2^31.
struct FastDiv {
  uint32_t d = 1, m = 1, l = 0;
};
FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  while ((1ull << f.l) < d) ++f.l;
  f.m = (uint32_t)(((1ull << 32) * ((1ull << f.l) - d)) / d + 1);
  return f;
}
__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) { return (__umulhi(f.m, n) + n) >> f.l; }

// The direct permutation with every element offset below 2^31: 32-bit index arithmetic, each
// division by a dimension a multiply and a shift, and each warp over 128 consecutive output
// elements (four coalesced 512-byte accesses, all loads issued before the stores).
struct PermuteFast {
  const z* in;
  z* out;
  int rank;
  FastDiv dims[kMaxRank];
  uint32_t istr[kMaxRank], ostr[kMaxRank];
  z alpha;
  double beta;
  int conj, mode;
  unsigned long long sx, sy;
};
__global__ void __launch_bounds__(256) permute_fast_kernel(PermuteFast g, uint32_t total) {
  constexpr int U = 4;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < (total + 127u) / 128u; w += nwarps) {
    uint32_t io[U], oo[U];
    bool live[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t e = w * 128u + (uint32_t)u * 32u + lane;
      live[u] = e < total;
      uint32_t r = live[u] ? e : 0u, i = 0, o = 0;
#pragma unroll
      for (int d = kMaxRank - 1; d >= 0; --d) {
        if (d >= g.rank) continue;
        const uint32_t q = fdiv(r, g.dims[d]);
        const uint32_t c = r - q * g.dims[d].d;
        i += c * g.istr[d];
        o += c * g.ostr[d];
        r = q;
      }
      io[u] = i;
      oo[u] = o;
    }
    z v[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (live[u]) v[u] = g.in[io[u]];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (live[u]) perm_put(g.out + oo[u], v[u], g.mode, g.sx, g.sy, g.alpha, g.beta, g.conj);
  }
}

// 32 x 32 shared-memory transpose over output dims (p, q): q is innermost in the
// output, p is innermost (stride 1) in the input, so both the loads and the
// stores are coalesced. The remaining dims are walked by blockIdx.y.
__global__ void permute_tiled_kernel(PermuteArgs g, int p, int64_t nrest, int64_t tiles_p, int64_t tiles_q) {
  __shared__ z tile[32][33];
  const int q = g.rank - 1;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int64_t r = blockIdx.y; r < nrest; r += gridDim.y) {
    int64_t rr = r, ib = 0, ob = 0;
    for (int d = g.rank - 1; d >= 0; --d) {
      if (d == p || d == q) continue;
      int64_t c = rr % g.dims[d];
      rr /= g.dims[d];
      ib += c * g.istr[d];
      ob += c * g.ostr[d];
    }
    for (int64_t t = blockIdx.x; t < tiles_p * tiles_q; t += gridDim.x) {
      const int64_t p0 = (t / tiles_q) * 32, q0 = (t % tiles_q) * 32;
      for (int yy = ty; yy < 32; yy += 8) {
        int64_t pp = p0 + tx, qq = q0 + yy;
        if (pp < g.dims[p] && qq < g.dims[q]) tile[yy][tx] = g.in[ib + pp * g.istr[p] + qq * g.istr[q]];
      }
      __syncthreads();
      for (int yy = ty; yy < 32; yy += 8) {
        int64_t qq = q0 + tx, pp = p0 + yy;
        if (pp < g.dims[p] && qq < g.dims[q]) {
          perm_put(g.out + ob + pp * g.ostr[p] + qq * g.ostr[q], tile[tx][yy], g.mode, g.sx, g.sy, g.alpha, g.beta,
                   g.conj);
        }
      }
      __syncthreads();
    }
  }
}

__global__ void zscale_kernel(z* C, int64_t M, int64_t N, int64_t ldc, int64_t sC, int batch, z beta) {
  const int64_t total = M * N * batch;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t n = e % N, m = (e / N) % M, b = e / (M * N);
    z* p = C + b * sC + m * ldc + n;
    *p = (beta.x == 0.0 && beta.y == 0.0) ? make_double2(0.0, 0.0) : zmul(beta, *p);
  }
}

// ---- amplitudes ------------------------------------------------------------

// out = c2 t2 + c11 (t1 t1 products) at (x, y, a, b), stored [x][y][a][b] (yaxb = 0) or
// [y][a][x][b] (yaxb = 1); b is innermost in both, so reads and writes stay coalesced.
__global__ void tau_kernel(const z* __restrict__ t1, const z* __restrict__ t2, z* __restrict__ out, int o, int v,
                           double c2, double c11, int anti, int yaxb) {
  const int64_t total = (int64_t)o * o * v * v;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int b, a, x, y;
    int64_t q = e;
    if (yaxb) {
      b = (int)(e % v);
      x = (int)((e / v) % o);
      a = (int)((e / ((int64_t)v * o)) % v);
      y = (int)(e / ((int64_t)v * o * v));
      q = (((int64_t)x * o + y) * v + a) * v + b;
    } else {
      b = (int)(e % v);
      a = (int)((e / v) % v);
      y = (int)((e / ((int64_t)v * v)) % o);
      x = (int)(e / ((int64_t)v * v * o));
    }
    z r = zmul(t1[(int64_t)x * v + a], t1[(int64_t)y * v + b]);
    if (anti) r = zsub(r, zmul(t1[(int64_t)y * v + a], t1[(int64_t)x * v + b]));
    z t = t2 ? t2[q] : make_double2(0.0, 0.0);
    out[e] = make_double2(c2 * t.x + c11 * r.x, c2 * t.y + c11 * r.y);
  }
}

__global__ void pack_pairs_kernel(const z* __restrict__ in, z* __restrict__ out, int64_t n1, int64_t n2,
                                  int pack_rows) {
  const int64_t P2 = pair_count(n2);
  const int64_t R = pack_rows ? pair_count(n1) : n1;
  const int64_t total = R * P2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col = e % P2, row = e / P2;
    int64_t a, b;
    pair_decode(col, n2, a, b);
    int64_t rin = row;
    if (pack_rows) {
      int64_t x, y;
      pair_decode(row, n1, x, y);
      rin = x * n1 + y;
    }
    out[e] = in[(rin * n2 + a) * n2 + b];
  }
}

// IT: the index type, 32-bit when every index is below 2^31 (the divisions by n1 and n2 are the
// kernel's main cost otherwise). With real alpha = +-1 and beta 0 or 1 the value is moved by sign
// flips and at most one add per part (no FP64 products on this chip's narrow FP64 pipe).
template <typename IT>
__global__ void unpack_pairs_kernel(UnpackArgs g, int unit) {
  const IT n1 = (IT)g.n1, n2 = (IT)g.n2, anti = (IT)g.anti_rows;
  const IT P2 = (IT)pair_count(g.n2);
  const IT R = g.unpack_rows ? n1 * n1 : n1;
  const IT total = R * n2 * n2;
  for (IT e = (IT)blockIdx.x * (IT)blockDim.x + (IT)threadIdx.x; e < total; e += (IT)gridDim.x * (IT)blockDim.x) {
    const IT ab = e % (n2 * n2), r = e / (n2 * n2);
    const IT b = ab % n2, a = ab / n2;
    bool neg = false;
    IT prow = r;
    bool zero = (a == b);
    if (g.unpack_rows) {
      const IT x = r / n1, y = r % n1;
      if (x == y) zero = true;
      else if (x < y) prow = (IT)pair_index(x, y, g.n1);
      else { prow = (IT)pair_index(y, x, g.n1); neg = !neg; }
    }
    z val = make_double2(0.0, 0.0);
    if (!zero) {
      IT pc;
      if (a < b) pc = (IT)pair_index(a, b, g.n2);
      else { pc = (IT)pair_index(b, a, g.n2); neg = !neg; }
      z x = g.in[prow * P2 + pc];
      if (anti > 0) {  // rows r = (x, y): in[(x, y)] - in[(y, x)]
        const IT rx = r / anti, ry = r % anti;
        x = zsub(x, g.in[(ry * anti + rx) * P2 + pc]);
      }
      if (unit) {
        const long long m = (neg != (g.alpha.x < 0.0)) ? (long long)0x8000000000000000ull : 0ll;
        val = make_double2(__longlong_as_double(__double_as_longlong(x.x) ^ m),
                           __longlong_as_double(__double_as_longlong(x.y) ^ m));
      } else {
        val = zscale(neg ? -1.0 : 1.0, zmul(g.alpha, x));
      }
    }
    z* op = g.out + e;
    if (g.beta == 0.0) *op = val;
    else if (unit && g.beta == 1.0) *op = make_double2(op->x + val.x, op->y + val.y);
    else *op = make_double2(g.beta * op->x + val.x, g.beta * op->y + val.y);
  }
}

__global__ void pack_vvvv_kernel(const z* __restrict__ D, z* __restrict__ W, int64_t v) {
  const int64_t P = pair_count(v);
  const int64_t total = P * P;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t a, b, c, d;
    pair_decode(e / P, v, a, b);
    pair_decode(e % P, v, c, d);
    // <ab||cd> = (ac|bd) - (ad|bc), D[a][c][b][d] = (ac|bd)
    z x = D[((a * v + c) * v + b) * v + d];
    z y = D[((a * v + d) * v + b) * v + c];
    W[e] = zsub(x, y);
  }
}

__global__ void pack_vvvv_rows_kernel(const z* __restrict__ D, z* __restrict__ W, int64_t v, int64_t a0, int64_t AB0,
                                      int64_t rows) {
  const int64_t P = pair_count(v), Nd = (v - a0 - 1) * v;
  const int64_t total = rows * P;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t a, b, c, d;
    pair_decode(AB0 + e / P, v, a, b);
    pair_decode(e % P, v, c, d);
    const z* Da = D + (a - a0) * v * Nd;
    // <ab||cd> = (ac|bd) - (ad|bc)
    W[e] = zsub(Da[c * Nd + (b - a0 - 1) * v + d], Da[d * Nd + (b - a0 - 1) * v + c]);
  }
}

// <ak||cd> packed over c < d for a block of na rows a, from the Coulomb block
// D[(a,x)][(k,y)] = (ax|ky):  W[(a,k)][P(c,d)] = D[a][c][k][d] - D[a][d][k][c].
__global__ void pack_vovv_rows_kernel(const z* __restrict__ D, z* __restrict__ W, int64_t na, int64_t o,
                                      int64_t v) {
  const int64_t P = pair_count(v), total = na * o * P;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / P, a = r / o, k = r % o;
    int64_t c, d;
    pair_decode(e % P, v, c, d);
    const z* Da = D + a * v * o * v;
    W[e] = zsub(Da[(c * o + k) * v + d], Da[(d * o + k) * v + c]);
  }
}

// out[a][c] = alpha * sum_k H[k][a][k][c] + beta * out[a][c] for H stored [i][a][k][c] (o v o v).
__global__ void trace_ik_kernel(const z* __restrict__ H, int64_t o, int64_t v, z* __restrict__ out, double alpha,
                                double beta) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < v * v;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = e / v, c = e % v;
    double sr = 0.0, si = 0.0;
    for (int64_t k = 0; k < o; ++k) {
      const z h = H[((k * v + a) * o + k) * v + c];
      sr += h.x;
      si += h.y;
    }
    const z prev = beta != 0.0 ? out[e] : make_double2(0.0, 0.0);
    out[e] = make_double2(alpha * sr + beta * prev.x, alpha * si + beta * prev.y);
  }
}

// The adjoint of trace_ik: H[k][a][k][c] += alpha * G[a][c] for every k.
__global__ void diag_add_ik_kernel(z* __restrict__ H, int64_t o, int64_t v, const z* __restrict__ G, double alpha) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < o * v * v;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = e / (v * v), a = (e / v) % v, c = e % v;
    z* h = H + ((k * v + a) * o + k) * v + c;
    const z g = G[a * v + c];
    *h = make_double2(h->x + alpha * g.x, h->y + alpha * g.y);
  }
}

// ---- update and norms ------------------------------------------------------

template <typename T>
__device__ T block_reduce_sum(T x, T* sh) {
  for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = x;
  __syncthreads();
  T r = 0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
  __syncthreads();
  return r;
}
__device__ double block_reduce_max(double x, double* sh) {
  for (int off = 16; off > 0; off >>= 1) {
    double y = __shfl_down_sync(0xffffffffu, x, off);
    x = (y > x || y != y) ? y : x;  // NaN wins
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = x;
  __syncthreads();
  double r = 0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r = (sh[i] > r || sh[i] != sh[i]) ? sh[i] : r;
  __syncthreads();
  return r;
}

// 1/D by Newton's iteration for the reciprocal, r <- r + r (1 - D r), from the correctly rounded
// FP32 reciprocal: each step squares the relative error (2^-24 -> ~2^-48 -> within an ulp of
// FP64), for four FMAs on this chip's narrow FP64 pipe. Outside FP32's range (and for zero,
// infinite or NaN D) the IEEE quotient.
__device__ __forceinline__ double recip_newton(double D) {
  const float f = __frcp_rn((float)D);
  if (!(fabsf(f) > 0.0f && fabsf(f) < INFINITY)) return 1.0 / D;
  double r = (double)f;
  r = fma(r, fma(-D, r, 1.0), r);
  r = fma(r, fma(-D, r, 1.0), r);
  return r;
}

// One update element: d = S/D (one reciprocal for both parts), t += d, S = d; returns |d|^2.
// The max-abs norm is taken on |d|^2 (one square root per block, not per element).
__device__ __forceinline__ double update_one(z* __restrict__ t, z* __restrict__ S, double D) {
  const double inv = recip_newton(D);
  z d = *S;
  d.x *= inv;
  d.y *= inv;
  *t = zadd(*t, d);
  *S = d;
  return d.x * d.x + d.y * d.y;
}

// The largest |d|^2 as an integer max over the bit patterns (|d|^2 >= 0, and a NaN, sign
// cleared, orders above infinity), off the FP64 pipe.
__device__ __forceinline__ void max_bits(unsigned long long& mx, double m2) {
  mx = max(mx, (unsigned long long)__double_as_longlong(m2) & 0x7FFFFFFFFFFFFFFFull);
}

// Work items are (row, chunk): rows 0..o-1 are t1's rows i (v elements, D = e_i - e_a - shift),
// rows o.. are t2's pair rows ij (v^2 elements, D = e_i + e_j - e_a - e_b - 2 shift), each cut
// into nc chunks. A row's e_i + e_j is formed once; the shifted virtual energies sit in shared
// memory (SH) or are formed per element.
template <bool SH>
__global__ void denom_update_kernel(z* __restrict__ t1, z* __restrict__ t2, z* __restrict__ S1,
                                    z* __restrict__ S2, const double* __restrict__ e, int o, int v, double shift,
                                    int nc, double* partials) {
  extern __shared__ double es_sh[];
  __shared__ double sh[32];
  if (SH) {
    for (int a = threadIdx.x; a < v; a += blockDim.x) es_sh[a] = e[o + a] + shift;
    __syncthreads();
  }
  auto es = [&](int a) { return SH ? es_sh[a] : e[o + a] + shift; };
  const int vv = v * v;
  const int64_t items = (int64_t)(o + o * o) * nc;
  double s2 = 0.0;
  unsigned long long mx = 0;
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const int row = (int)(it / nc), c = (int)(it % nc);
    if (row < o) {
      const int chunk = (v + nc - 1) / nc, lo = c * chunk, hi = min(v, lo + chunk);
      const double ei = e[row];
      z* tr = t1 + (int64_t)row * v;
      z* sr = S1 + (int64_t)row * v;
      for (int a = lo + threadIdx.x; a < hi; a += blockDim.x) {
        const double m2 = update_one(tr + a, sr + a, ei - es(a));
        s2 += m2;
        max_bits(mx, m2);
      }
    } else {
      const int ij = row - o, i = ij / o, j = ij - i * o;
      const int chunk = (vv + nc - 1) / nc, lo = c * chunk, hi = min(vv, lo + chunk);
      const double eij = e[i] + e[j];
      z* tr = t2 + (int64_t)ij * vv;
      z* sr = S2 + (int64_t)ij * vv;
      for (int ab = lo + threadIdx.x; ab < hi; ab += blockDim.x) {
        const int a = ab / v, b = ab - a * v;
        const double m2 = update_one(tr + ab, sr + ab, eij - (es(a) + es(b)));
        if (i < j && a < b) s2 += m2;
        max_bits(mx, m2);
      }
    }
  }
  const double bm = block_reduce_max(__longlong_as_double((long long)mx), sh);
  const double bs = block_reduce_sum(s2, sh);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = sqrt(bm);  // max |d| of the block
    partials[2 * blockIdx.x + 1] = bs;
  }
}

__global__ void norm_finalize_kernel(const double* partials, int nb, double* stats) {
  __shared__ double sh[32];
  double mx = 0.0, s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    const double m = partials[2 * i];
    mx = (m > mx || m != m) ? m : mx;
    s += partials[2 * i + 1];
  }
  const double bm = block_reduce_max(mx, sh);
  const double bs = block_reduce_sum(s, sh);
  if (threadIdx.x == 0) {
    stats[0] = bm;
    stats[1] = sqrt(bs);
  }
}

// ---- energy ----------------------------------------------------------------

// E = sum f_ia t_ia + 1/4 sum <ij||ab> tau_ij^ab. Both factors of the second sum are
// antisymmetric in (i, j) and in (a, b), so each unique term i < j, a < b appears four times
// with the same product: the kernel sums the unique terms once (a quarter of the FP64 work,
// this chip's narrow pipe), over 32-bit indices (IT) where they fit.
template <typename IT>
__global__ void energy_kernel(const z* __restrict__ fov, const z* __restrict__ oovv, const z* __restrict__ t1,
                              const z* __restrict__ t2, int o, int v, z* partials) {
  __shared__ double sh[32];
  const IT n1 = (IT)o * v, vv = (IT)v * v, n2 = (IT)o * o * vv;
  double er = 0.0, ei = 0.0;
  for (IT k = (IT)blockIdx.x * blockDim.x + threadIdx.x; k < n1 + n2; k += (IT)gridDim.x * blockDim.x) {
    z p;
    if (k < n1) {
      p = zmul(fov[k], t1[k]);
    } else {
      const IT q = k - n1, ab = q % vv, ij = q / vv;
      const IT b = ab % (IT)v, a = ab / (IT)v, j = ij % (IT)o, i = ij / (IT)o;
      if (i >= j || a >= b) continue;
      const z tau = zadd(t2[q], zsub(zmul(t1[i * v + a], t1[j * v + b]), zmul(t1[j * v + a], t1[i * v + b])));
      p = zmul(oovv[q], tau);
    }
    er += p.x;
    ei += p.y;
  }
  er = block_reduce_sum(er, sh);
  ei = block_reduce_sum(ei, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = make_double2(er, ei);
}

__global__ void energy_finalize_kernel(const z* partials, int nb, z* out) {
  __shared__ double sh[32];
  double er = 0.0, ei = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    er += partials[i].x;
    ei += partials[i].y;
  }
  er = block_reduce_sum(er, sh);
  ei = block_reduce_sum(ei, sh);
  if (threadIdx.x == 0) *out = make_double2(er, ei);
}

// ---- DIIS ------------------------------------------------------------------

// Unique-element index k in [0, L) -> position in the full t1 / t2 arrays.
__device__ __forceinline__ int64_t unique_to_full(int64_t k, int o, int v) {
  const int64_t n1 = (int64_t)o * v;
  if (k < n1) return k;
  const int64_t q = k - n1, Pv = pair_count(v);
  int64_t i, j, a, b;
  pair_decode(q / Pv, o, i, j);
  pair_decode(q % Pv, v, a, b);
  return n1 + ((i * o + j) * v + a) * v + b;
}

__global__ void diis_push_kernel(DiisArgs d, const z* __restrict__ t1, const z* __restrict__ t2,
                                 const z* __restrict__ e1, const z* __restrict__ e2) {
  const int slot = d.state->head;
  const int64_t n1 = (int64_t)d.o * d.v;
  z* ht = d.hist_t + slot * d.L;
  z* he = d.hist_e + slot * d.L;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < d.L;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = unique_to_full(k, d.o, d.v);
    ht[k] = f < n1 ? t1[f] : t2[f - n1];
    he[k] = f < n1 ? e1[f] : e2[f - n1];
  }
}

// Re <e_new, e_slot> for every stored slot; per-block partials [slot][block].
__global__ void diis_dots_kernel(DiisArgs d) {
  __shared__ double sh[32];
  const int newslot = d.state->head;
  const int count = d.state->count + 1 > d.m ? d.m : d.state->count + 1;
  const z* en = d.hist_e + newslot * d.L;
  for (int s = 0; s < count; ++s) {
    const z* es = d.hist_e + s * d.L;
    double acc = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < d.L;
         k += (int64_t)gridDim.x * blockDim.x) {
      const z x = en[k], y = es[k];
      acc += x.x * y.x + x.y * y.y;
    }
    acc = block_reduce_sum(acc, sh);
    if (threadIdx.x == 0) d.partials[s * gridDim.x + blockIdx.x] = acc;
  }
}

// One block: finish the dots, advance the ring buffer, and (if due) solve
// [[B, 1], [1^T, 0]] [c; lam] = [0; 1] by LU with partial pivoting in age order.
__global__ void diis_solve_kernel(DiisArgs d, int nb) {
  __shared__ double sh[32];
  __shared__ double M[17][18];
  DiisState* st = d.state;
  const int newslot = st->head;
  const int count = st->count + 1 > d.m ? d.m : st->count + 1;
  for (int s = 0; s < count; ++s) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += d.partials[s * nb + i];
    acc = block_reduce_sum(acc, sh);
    if (threadIdx.x == 0) {
      d.Bmat[newslot * d.m + s] = acc;
      d.Bmat[s * d.m + newslot] = acc;
    }
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  st->count = count;
  st->head = (newslot + 1) % d.m;
  st->iter += 1;
  st->used = 0;
  if (st->iter < d.start || count < 2) return;
  // age order: oldest slot first
  const int oldest = (st->head - count + d.m) % d.m;
  const int n = count + 1;
  for (int r = 0; r < count; ++r) {
    const int sr = (oldest + r) % d.m;
    for (int c = 0; c < count; ++c) M[r][c] = d.Bmat[sr * d.m + (oldest + c) % d.m];
    M[r][count] = 1.0;
    M[r][n] = 0.0;
  }
  for (int c = 0; c < count; ++c) M[count][c] = 1.0;
  M[count][count] = 0.0;
  M[count][n] = 1.0;
  for (int k = 0; k < n; ++k) {
    int piv = k;
    double best = fabs(M[k][k]);
    for (int r = k + 1; r < n; ++r)
      if (fabs(M[r][k]) > best) { best = fabs(M[r][k]); piv = r; }
    if (piv != k)
      for (int c = 0; c <= n; ++c) { double tmp = M[k][c]; M[k][c] = M[piv][c]; M[piv][c] = tmp; }
    const double dkk = M[k][k];
    if (dkk == 0.0) return;  // singular subspace: keep the plain update
    for (int r = k + 1; r < n; ++r) {
      const double f = M[r][k] / dkk;
      for (int c = k; c <= n; ++c) M[r][c] -= f * M[k][c];
    }
  }
  double x[17];
  for (int r = n - 1; r >= 0; --r) {
    double s = M[r][n];
    for (int c = r + 1; c < n; ++c) s -= M[r][c] * x[c];
    x[r] = s / M[r][r];
  }
  for (int r = 0; r < count; ++r) d.coef[r] = x[r];
  st->used = 1;
  if (!d.crop) return;
  // CROP: the newest slot will hold the optimal pair (sum_r c_r t_r, sum_r c_r e_r). Its inner
  // products follow from the old ones: Re<e~, e_s> = sum_r c_r B[r][s], Re<e~, e~> = sum_r c_r
  // Re<e~, e_r>, all taken from B before it is overwritten.
  double rowc[16];
  for (int q = 0; q < count; ++q) {
    const int sq = (oldest + q) % d.m;
    double acc = 0.0;
    for (int r = 0; r < count; ++r) acc += x[r] * d.Bmat[((oldest + r) % d.m) * d.m + sq];
    rowc[q] = acc;
  }
  double bnn = 0.0;
  for (int r = 0; r < count; ++r) bnn += x[r] * rowc[r];
  for (int q = 0; q < count; ++q) {
    const int sq = (oldest + q) % d.m;
    if (sq == newslot) continue;
    d.Bmat[newslot * d.m + sq] = rowc[q];
    d.Bmat[sq * d.m + newslot] = rowc[q];
  }
  d.Bmat[newslot * d.m + newslot] = bnn;
}

// CROP: replace the newest subspace pair by the optimal combination (unique-element layout).
// Every thread reads all slots at its own elements before writing the newest slot there.
__global__ void crop_writeback_kernel(DiisArgs d) {
  const DiisState st = *d.state;
  if (!st.used) return;
  const int oldest = (st.head - st.count + d.m) % d.m;
  const int newest = (st.head - 1 + d.m) % d.m;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < d.L;
       k += (int64_t)gridDim.x * blockDim.x) {
    z at = make_double2(0.0, 0.0), ae = make_double2(0.0, 0.0);
    for (int r = 0; r < st.count; ++r) {
      const double c = d.coef[r];
      const int64_t off = (int64_t)((oldest + r) % d.m) * d.L + k;
      const z ht = d.hist_t[off], he = d.hist_e[off];
      at.x += c * ht.x;
      at.y += c * ht.y;
      ae.x += c * he.x;
      ae.y += c * he.y;
    }
    d.hist_t[(int64_t)newest * d.L + k] = at;
    d.hist_e[(int64_t)newest * d.L + k] = ae;
  }
}

// t = sum_r coef[r] * hist_t[slot(r)], written to the full t1 / t2 (antisymmetric fill).
__global__ void diis_combine_kernel(DiisArgs d, z* __restrict__ t1, z* __restrict__ t2) {
  const DiisState st = *d.state;
  if (!st.used) return;
  const int oldest = (st.head - st.count + d.m) % d.m;
  const int64_t n1 = (int64_t)d.o * d.v, n2 = (int64_t)d.o * d.o * d.v * d.v;
  const int64_t Pv = pair_count(d.v);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n1 + n2;
       k += (int64_t)gridDim.x * blockDim.x) {
    int64_t u;
    double sgn = 1.0;
    bool zero = false;
    if (k < n1) {
      u = k;
    } else {
      const int64_t q = k - n1;
      const int64_t b = q % d.v, a = (q / d.v) % d.v;
      const int64_t j = (q / ((int64_t)d.v * d.v)) % d.o, i = q / ((int64_t)d.v * d.v * d.o);
      if (i == j || a == b) zero = true;
      int64_t pij = 0, pab = 0;
      if (!zero) {
        if (i < j) pij = pair_index(i, j, d.o); else { pij = pair_index(j, i, d.o); sgn = -sgn; }
        if (a < b) pab = pair_index(a, b, d.v); else { pab = pair_index(b, a, d.v); sgn = -sgn; }
      }
      u = n1 + pij * Pv + pab;
    }
    z acc = make_double2(0.0, 0.0);
    if (!zero)
      for (int r = 0; r < st.count; ++r) {
        const double c = d.coef[r];
        const z h = d.hist_t[((oldest + r) % d.m) * d.L + u];
        acc.x += c * h.x;
        acc.y += c * h.y;
      }
    acc = zscale(sgn, acc);
    if (k < n1) t1[k] = acc; else t2[k - n1] = acc;
  }
}

__global__ void diis_reset_kernel(DiisState* st) {
  st->count = 0;
  st->head = 0;
  st->iter = 0;
  st->used = 0;
}

}  // namespace

// ---- launchers -----------------------------------------------------------------

cudaError_t zscale_matrix(const ZGemmArgs& g, cudaStream_t s) {
  zscale_kernel<<<grid_for(g.M * g.N * g.batch, kThreads), kThreads, 0, s>>>(g.C, g.M, g.N, g.ldc, g.sC, g.batch,
                                                                                g.beta);
  return cudaGetLastError();
}

#ifndef PERMUTE_FAST
#define PERMUTE_FAST 1
#endif
cudaError_t permute_add(const PermuteArgs& a0, cudaStream_t s) {
  if (a0.rank < 1 || a0.rank > kMaxRank) return cudaErrorInvalidValue;
  // the same permutation with dims of extent 1 dropped and neighbours that are contiguous in
  // both the input and the output merged into one
  PermuteArgs a = a0;
  a.rank = 0;
  for (int d = 0; d < a0.rank; ++d) {
    if (a0.dims[d] == 0) return cudaSuccess;
    if (a0.dims[d] == 1) continue;
    if (a.rank > 0) {
      const int t = a.rank - 1;
      if (a.istr[t] == a0.dims[d] * a0.istr[d] && a.ostr[t] == a0.dims[d] * a0.ostr[d]) {
        a.dims[t] *= a0.dims[d];
        a.istr[t] = a0.istr[d];
        a.ostr[t] = a0.ostr[d];
        continue;
      }
    }
    a.dims[a.rank] = a0.dims[d];
    a.istr[a.rank] = a0.istr[d];
    a.ostr[a.rank] = a0.ostr[d];
    ++a.rank;
  }
  if (a.rank == 0) {  // a single element
    a.rank = 1;
    a.dims[0] = 1;
    a.istr[0] = a.ostr[0] = 1;
  }
  {
    constexpr unsigned long long kSign = 0x8000000000000000ull;
    const bool unit = a.alpha.y == 0.0 && (a.alpha.x == 1.0 || a.alpha.x == -1.0);
    a.mode = unit && a.beta == 0.0 ? 1 : unit && a.beta == 1.0 ? 2 : 0;
    a.sx = a.alpha.x < 0.0 ? kSign : 0ull;
    a.sy = a.sx ^ (a.conj ? kSign : 0ull);
  }
  int64_t total = 1, imax = 0, omax = 0;
  for (int d = 0; d < a.rank; ++d) {
    total *= a.dims[d];
    imax += (a.dims[d] - 1) * a.istr[d];
    omax += (a.dims[d] - 1) * a.ostr[d];
  }
  const int q = a.rank - 1;
  int p = -1;
  if (a.istr[q] != 1 && a.dims[q] > 1)
    for (int d = 0; d < q; ++d)
      if (a.istr[d] == 1 && a.dims[d] > 1) p = d;
  if (p < 0) {
    constexpr int64_t kLim = (int64_t)1 << 31;
    if (PERMUTE_FAST && total < kLim && imax < kLim && omax < kLim) {
      PermuteFast f;
      f.in = a.in;
      f.out = a.out;
      f.rank = a.rank;
      for (int d = 0; d < a.rank; ++d) {
        f.dims[d] = make_fastdiv((uint32_t)a.dims[d]);
        f.istr[d] = (uint32_t)a.istr[d];
        f.ostr[d] = (uint32_t)a.ostr[d];
      }
      f.alpha = a.alpha;
      f.beta = a.beta;
      f.conj = a.conj;
      f.mode = a.mode;
      f.sx = a.sx;
      f.sy = a.sy;
      permute_fast_kernel<<<grid_for((total + 127) / 128 * 32, kThreads), kThreads, 0, s>>>(f, (uint32_t)total);
    } else {
      permute_direct_kernel<<<grid_for(total, kThreads), kThreads, 0, s>>>(a, total);
    }
  } else {
    const int64_t tp = (a.dims[p] + 31) / 32, tq = (a.dims[q] + 31) / 32;
    const int64_t nrest = total / (a.dims[p] * a.dims[q]);
    int64_t gx = tp * tq;
    if (gx > 4096) gx = 4096;
    int64_t gy = nrest;
    if (gy > 65535) gy = 65535;
    permute_tiled_kernel<<<dim3((unsigned)gx, (unsigned)gy), dim3(32, 8), 0, s>>>(a, p, nrest, tp, tq);
  }
  return cudaGetLastError();
}

cudaError_t tau_build(const z* t1, const z* t2, z* out, int o, int v, double c2, double c11, int anti,
                      cudaStream_t s, int yaxb) {
  const int64_t total = (int64_t)o * o * v * v;
  tau_kernel<<<grid_for(total, kThreads), kThreads, 0, s>>>(t1, t2, out, o, v, c2, c11, anti, yaxb);
  return cudaGetLastError();
}

cudaError_t pack_pairs(const z* in, z* out, int64_t n1, int64_t n2, int pack_rows, cudaStream_t s) {
  const int64_t total = (pack_rows ? pair_count(n1) : n1) * pair_count(n2);
  if (total == 0) return cudaSuccess;
  pack_pairs_kernel<<<grid_for(total, kThreads), kThreads, 0, s>>>(in, out, n1, n2, pack_rows);
  return cudaGetLastError();
}

cudaError_t unpack_pairs(const UnpackArgs& a, cudaStream_t s) {
  const int64_t total = (a.unpack_rows ? a.n1 * a.n1 : a.n1) * a.n2 * a.n2;
  if (total == 0) return cudaSuccess;
  const int unit = a.alpha.y == 0.0 && (a.alpha.x == 1.0 || a.alpha.x == -1.0);
  if (total < ((int64_t)1 << 31) && a.n1 * a.n1 < ((int64_t)1 << 31))
    unpack_pairs_kernel<uint32_t><<<grid_for(total, kThreads), kThreads, 0, s>>>(a, unit);
  else
    unpack_pairs_kernel<int64_t><<<grid_for(total, kThreads), kThreads, 0, s>>>(a, unit);
  return cudaGetLastError();
}

cudaError_t pack_vvvv(const z* D, z* W, int64_t v, cudaStream_t s) {
  const int64_t P = pair_count(v);
  if (P == 0) return cudaSuccess;
  pack_vvvv_kernel<<<grid_for(P * P, kThreads), kThreads, 0, s>>>(D, W, v);
  return cudaGetLastError();
}

cudaError_t pack_vvvv_rows(const z* D, z* W, int64_t v, int64_t a0, int64_t a1, cudaStream_t s) {
  const int64_t AB0 = pair_index(a0, a0 + 1, v);
  const int64_t AB1 = a1 >= v - 1 ? pair_count(v) : pair_index(a1, a1 + 1, v);
  const int64_t rows = AB1 - AB0;
  if (rows <= 0) return cudaSuccess;
  pack_vvvv_rows_kernel<<<grid_for(rows * pair_count(v), kThreads), kThreads, 0, s>>>(D, W, v, a0, AB0, rows);
  return cudaGetLastError();
}

cudaError_t pack_vovv_rows(const z* D, z* W, int64_t na, int64_t o, int64_t v, cudaStream_t s) {
  const int64_t total = na * o * pair_count(v);
  if (total <= 0) return cudaSuccess;
  pack_vovv_rows_kernel<<<grid_for(total, kThreads), kThreads, 0, s>>>(D, W, na, o, v);
  return cudaGetLastError();
}

cudaError_t diag_add_ik(z* H, int64_t o, int64_t v, const z* G, double alpha, cudaStream_t s) {
  diag_add_ik_kernel<<<grid_for(o * v * v, kThreads), kThreads, 0, s>>>(H, o, v, G, alpha);
  return cudaGetLastError();
}

cudaError_t trace_ik(const z* H, int64_t o, int64_t v, z* out, double alpha, double beta, cudaStream_t s) {
  if (v <= 0) return cudaSuccess;
  trace_ik_kernel<<<grid_for(v * v, kThreads), kThreads, 0, s>>>(H, o, v, out, alpha, beta);
  return cudaGetLastError();
}

int update_blocks() { return kUpdateBlocks; }

cudaError_t denom_update(z* t1, z* t2, z* S1, z* S2, const double* e, int o, int v, double shift,
                         double* partials, cudaStream_t s) {
  if (o < 0 || v < 0 || (int64_t)v * v > 0x7fffffff || (int64_t)o * o > 0x7fffffff) return cudaErrorInvalidValue;
  // chunks per row: enough items for two per block, each at least one pass of the block
  const int64_t rows = (int64_t)o + (int64_t)o * o, vv = (int64_t)v * v;
  const int nc =
      rows > 0 ? (int)std::max<int64_t>(1, std::min<int64_t>((2 * kUpdateBlocks + rows - 1) / rows, vv / kThreads)) : 1;
  const size_t smem = (size_t)v * sizeof(double);
  if (smem <= 32768)
    denom_update_kernel<true><<<kUpdateBlocks, kThreads, smem, s>>>(t1, t2, S1, S2, e, o, v, shift, nc, partials);
  else
    denom_update_kernel<false><<<kUpdateBlocks, kThreads, 0, s>>>(t1, t2, S1, S2, e, o, v, shift, nc, partials);
  return cudaGetLastError();
}

cudaError_t norm_finalize(const double* partials, int nblocks, double* stats, cudaStream_t s) {
  norm_finalize_kernel<<<1, 1024, 0, s>>>(partials, nblocks, stats);
  return cudaGetLastError();
}

int energy_blocks() { return kEnergyBlocks; }

cudaError_t energy_eval(const z* fov, const z* oovv, const z* t1, const z* t2, int o, int v, z* partials,
                        z* e_out, cudaStream_t s) {
  const int64_t n = (int64_t)o * v + (int64_t)o * o * v * v;
  if (n < ((int64_t)1 << 31))
    energy_kernel<uint32_t><<<kEnergyBlocks, kThreads, 0, s>>>(fov, oovv, t1, t2, o, v, partials);
  else
    energy_kernel<int64_t><<<kEnergyBlocks, kThreads, 0, s>>>(fov, oovv, t1, t2, o, v, partials);
  energy_finalize_kernel<<<1, 1024, 0, s>>>(partials, kEnergyBlocks, e_out);
  return cudaGetLastError();
}

int diis_blocks() { return kDiisBlocks; }

cudaError_t diis_reset(const DiisArgs& d, cudaStream_t s) {
  diis_reset_kernel<<<1, 1, 0, s>>>(d.state);
  return cudaGetLastError();
}

cudaError_t diis_step(const DiisArgs& d, z* t1, z* t2, const z* e1, const z* e2, cudaStream_t s) {
  if (d.m < 1 || d.m > 16) return cudaErrorInvalidValue;
  diis_push_kernel<<<grid_for(d.L, kThreads), kThreads, 0, s>>>(d, t1, t2, e1, e2);
  diis_dots_kernel<<<kDiisBlocks, kThreads, 0, s>>>(d);
  diis_solve_kernel<<<1, 1024, 0, s>>>(d, kDiisBlocks);
  const int64_t n = (int64_t)d.o * d.v + (int64_t)d.o * d.o * d.v * d.v;
  diis_combine_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(d, t1, t2);
  if (d.crop) crop_writeback_kernel<<<grid_for(d.L, kThreads), kThreads, 0, s>>>(d);
  return cudaGetLastError();
}

}  // namespace ccsd
