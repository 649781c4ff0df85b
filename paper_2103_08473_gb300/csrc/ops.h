// Host launchers for the HBM-bound kernels of libccsd: index permutations,
// antisymmetric pair packing, tau, the denominator update, reductions and DIIS.
#pragma once

#include "common.cuh"

namespace ccsd {

constexpr int kMaxRank = 8;

// out[x] = alpha * op(in[perm(x)]) + beta * out[x] over the output index space
// dims[0..rank) (row-major enumeration). istr/ostr give, for every output
// dimension, its stride (in complex elements) in the input and in the output.
// op conjugates when conj != 0. beta == 0 never reads out.
struct PermuteArgs {
  const z* in = nullptr;
  z* out = nullptr;
  int rank = 0;
  int64_t dims[kMaxRank] = {};
  int64_t istr[kMaxRank] = {};
  int64_t ostr[kMaxRank] = {};
  z alpha{1.0, 0.0};
  double beta = 0.0;
  int conj = 0;
  // set by permute_add: 1 when alpha = +-1 and beta = 0 (a copy with sign flips), 2 when
  // alpha = +-1 and beta = 1 (one add per part); sx, sy: sign bits to flip on re, im
  int mode = 0;
  unsigned long long sx = 0, sy = 0;
};
cudaError_t permute_add(const PermuteArgs& a, cudaStream_t s);

// out[x][y][a][b] = c2 * t2[x][y][a][b] + c11 * (t1[x][a] t1[y][b] - anti * t1[y][a] t1[x][b]);
// with yaxb = 1 the same values are stored as out[y][a][x][b].
cudaError_t tau_build(const z* t1, const z* t2, z* out, int o, int v, double c2, double c11, int anti,
                      cudaStream_t s, int yaxb = 0);

// Pack the antisymmetric trailing pair: out[r][P(a,b)] = in[r][a][b] for a < b, r over R rows.
// With pack_rows, r itself runs over the pairs x < y of an n1 x n1 leading pair (R = n1*n1 in
// the input, pair_count(n1) in the output).
cudaError_t pack_pairs(const z* in, z* out, int64_t n1, int64_t n2, int pack_rows, cudaStream_t s);

// Unpack-accumulate: out[r][a][b] = beta * out + alpha * sgn(a,b) * in[r][P(min,max)] (zero on
// a == b). With unpack_rows the leading pair is packed too (sgn over both pairs). With
// anti_rows = m (unpack_rows == 0, n1 = m * m rows r = (x, y)), the rows are antisymmetrised on
// the way: out[(x,y)][a][b] = beta * out + alpha * sgn(a,b) * (in[(x,y)][P] - in[(y,x)][P]).
struct UnpackArgs {
  const z* in = nullptr;
  z* out = nullptr;
  int64_t n1 = 0;   // leading pair extent (unpack_rows) or number of rows R
  int64_t n2 = 0;   // trailing pair extent
  int unpack_rows = 0;
  int64_t anti_rows = 0;
  z alpha{1.0, 0.0};
  double beta = 1.0;  // out = beta * out + ...
};
cudaError_t unpack_pairs(const UnpackArgs& a, cudaStream_t s);

// W[P(a,b)][P(c,d)] = D[a][c][b][d] - D[a][d][b][c]  (D dense v^4 Coulomb block (ac|bd))
cudaError_t pack_vvvv(const z* D, z* W, int64_t v, cudaStream_t s);
// Rows of the same packed W for a in [a0, a1), b in (a, v), from the block
// D[(a - a0) v + c][(b - a0 - 1) v + d] = (ac|bd) (b > a0 only): W[P(a,b) - P(a0,a0+1)][P(c,d)].
cudaError_t pack_vvvv_rows(const z* D, z* W, int64_t v, int64_t a0, int64_t a1, cudaStream_t s);

// <ak||cd> packed over c < d for na rows a from the Coulomb block D[(a,x)][(k,y)] = (ax|ky):
// W[(a,k)][P(c,d)] = D[a][c][k][d] - D[a][d][k][c].
cudaError_t pack_vovv_rows(const z* D, z* W, int64_t na, int64_t o, int64_t v, cudaStream_t s);
// out[a][c] = alpha * sum_k H[k][a][k][c] + beta * out[a][c] for H stored [i][a][k][c] (o, v, o, v).
cudaError_t trace_ik(const z* H, int64_t o, int64_t v, z* out, double alpha, double beta, cudaStream_t s);
// The adjoint of trace_ik: H[k][a][k][c] += alpha * G[a][c] for every k (H stored [i][a][k][c]).
cudaError_t diag_add_ik(z* H, int64_t o, int64_t v, const z* G, double alpha, cudaStream_t s);

// Denominator update over t1 (o*v) and full t2 (o*o*v*v):
//   d = S / D, t += d, S <- d.   D^a_i = e_i - e_a - shift, D^{ab}_{ij} = e_i + e_j - e_a - e_b - 2 shift
// (e = the real diagonal of the Fock matrix). Writes per-block partial max|d| and
// sum |d|^2 (unique amplitudes) to `partials` (2 * nblocks doubles); norm_finalize
// reduces them into stats[0] = max |d|, stats[1] = ||d||_2 in a fixed order.
int update_blocks();
cudaError_t denom_update(z* t1, z* t2, z* S1, z* S2, const double* e, int o, int v, double shift,
                         double* partials, cudaStream_t s);
cudaError_t norm_finalize(const double* partials, int nblocks, double* stats, cudaStream_t s);

// E = sum_ia fov[i][a] t1[i][a] + 1/4 sum_ijab oovv[i][j][a][b] tau[i][j][a][b] (tau on the fly).
// Two-stage deterministic reduction: block partials then one block; result in e_out (device).
int energy_blocks();
cudaError_t energy_eval(const z* fov, const z* oovv, const z* t1, const z* t2, int o, int v, z* partials,
                        z* e_out, cudaStream_t s);

// DIIS on the stacked unique amplitudes x = [t1 (o*v) | t2 packed (i<j, a<b)], length L.
struct DiisState {
  int count;  // vectors stored
  int head;   // next slot
  int iter;   // iterations pushed so far
  int used;   // 1 if the last push extrapolated
};
struct DiisArgs {
  int o = 0, v = 0, m = 0, start = 2;
  int crop = 0;  // 1: CROP, the newest slot is replaced by the optimal combination after each solve
  int64_t L = 0;
  z* hist_t = nullptr;   // m * L
  z* hist_e = nullptr;   // m * L
  double* Bmat = nullptr;  // m * m, indexed by slot
  double* coef = nullptr;  // m, in age order (oldest first)
  double* partials = nullptr;  // m * nblocks
  DiisState* state = nullptr;
};
int diis_blocks();
cudaError_t diis_reset(const DiisArgs& d, cudaStream_t s);
// Push (t, e) (full t1/t2 layout), update the subspace matrix, and if the iteration number is
// >= start with >= 2 vectors, overwrite t1/t2 with the extrapolated amplitudes. With crop = 1
// the pushed pair is then replaced in the subspace by the combination itself (sum c t, sum c e)
// and its rows of the subspace matrix by the matching combinations of the old rows.
cudaError_t diis_step(const DiisArgs& d, z* t1, z* t2, const z* e1, const z* e2, cudaStream_t s);

}  // namespace ccsd
