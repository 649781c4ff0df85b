/*
 * ccsd.h - C ABI of libccsd, a single-GPU (sm_103a) engine for the per-iteration
 * amplitude residual of Kramers-unrestricted complex CCSD.
 *
 * The problem statement follows the paper (arXiv:2103.08473):
 *   - Hamiltonian with complex one-body part and antisymmetrised two-electron
 *     integrals V^{pq}_{rs} = <pq||rs> (Eq. Hamiltonian, Eq. two_electron);
 *   - CCSD amplitude equations <Phi_l| exp(-T) H exp(T) |Phi_0> = 0 (Eq. CCSD)
 *     evaluated with the working equations of Appendix A;
 *   - MP2 initial guess, denominator ("Jacobi") update and DIIS
 *     (Sec. "Coupled cluster implementation");
 *   - all tensors are created before iterating (same section).
 *
 * Conventions shared by every call
 *   - Complex numbers are interleaved (re, im) doubles: ccsd_z is layout-
 *     compatible with C99 double _Complex, std::complex<double>,
 *     cuDoubleComplex and numpy complex128.
 *   - Spinors are ordered occupied first: p in [0, o) occupied, [o, o+v) virtual.
 *   - t1 / r1:  [i][a], row-major, o*v elements, t1[i*v + a] = t^a_i.
 *   - t2 / r2:  [i][j][a][b], row-major, o*o*v*v elements, full storage of
 *               t^{ab}_{ij}, antisymmetric in (i,j) and in (a,b). Packing by
 *               antisymmetry is internal.
 *   - Density-fitting factors B: [Q][p][r], naux*n*n elements, Hermitian in
 *     (p, r); (pr|qs) = sum_Q B^Q_pr B^Q_qs and <pq||rs> = (pr|qs) - (ps|qr).
 *   - Full integrals V: [p][q][r][s], n^4 elements, V[p][q][r][s] = <pq||rs>.
 *   - Fock: n*n Hermitian, [p][q] = f_pq; NULL means diag(eps).
 *
 * Ownership: ccsd_create copies every input; the caller keeps its buffers.
 * Output buffers belong to the caller. With on_device != 0, pointers are device
 * pointers on the context's device; otherwise host pointers (pageable or
 * pinned). The context owns all device memory it allocates and frees it in
 * ccsd_destroy.
 *
 * Errors: every call returns a ccsd_status; nothing throws across the ABI, and
 * nothing calls exit/abort or traps on the device. ccsd_last_error() returns a
 * human-readable message for the last failing call on that context. A context
 * is not thread-safe: use one host thread per context at a time.
 *
 * Streams: all device work of a context is issued on opts.stream (a
 * cudaStream_t; NULL = the legacy default stream). Calls that return host
 * values synchronise that stream.
 */
#ifndef CCSD_H
#define CCSD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ccsd_ctx ccsd_ctx;

/* Interleaved complex double. */
typedef struct {
  double re, im;
} ccsd_z;

typedef enum {
  CCSD_OK = 0,
  CCSD_ERR_ARG = 1,           /* invalid argument (sizes, NULL pointers, non-Hermitian input) */
  CCSD_ERR_OOM = 2,           /* device allocation failed */
  CCSD_ERR_CUDA = 3,          /* a CUDA runtime call or kernel launch failed */
  CCSD_ERR_NOT_CONVERGED = 4, /* iteration cap reached before the tolerance */
  CCSD_ERR_DIVERGED = 5,      /* NaN/Inf in the update, or sustained growth of its norm; amplitudes
                                 left at the last finite iterate */
  CCSD_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up */
  CCSD_ERR_UNSUPPORTED = 7    /* option combination not built */
} ccsd_status;

typedef enum {
  CCSD_INT_DF = 0,  /* ints = B[naux][n][n] */
  CCSD_INT_FULL = 1 /* ints = V[n][n][n][n] = <pq||rs> (small n only); naux ignored */
} ccsd_int_kind;

typedef enum {
  CCSD_PREC_FP64 = 0, /* every contraction in complex FP64 */
  CCSD_PREC_SPLIT = 1 /* large contractions as split-precision tensor-core GEMMs, FP64 recombination */
} ccsd_precision;

typedef enum {
  CCSD_METHOD_CCSD = 0, /* singles and doubles (Appendix A) */
  CCSD_METHOD_CCD = 1,  /* doubles only: the doubles equations of Appendix A at T1 = 0, the
                           variant the paper also times. The residual plan leaves out every term
                           with a t1 factor and the intermediates that only feed them (C^{kb}_{ij},
                           H^k_c, the singles): ccsd_residual returns S1 = 0 and the CCD S2
                           whatever t1 it is given, and the iterations keep t1 at zero */
  CCSD_METHOD_CC2 = 2   /* CC2 (appendix "Working equations for CC2 amplitude equations"): the
                           singles equations of Appendix A unchanged, the doubles equation
                           S^{ab}_{ij} = <ab||ij>~ + P^-_ab sum_e f_be t^{ae}_{ij}
                           - P^-_ij sum_m f_mj t^{ab}_{im}, where <ab||ij>~ is the integral of
                           exp(-T1) H exp(T1). It is evaluated from the T1-dressed DF factors
                           (1 - t1) B^Q (1 + t1), which reproduce the appendix's W terms exactly.
                           Needs DF integrals (CCSD_ERR_UNSUPPORTED otherwise); <ab||cd> is
                           never built. ccsd_get_tensor then has only "tau", "Hvv", "Hoo" and
                           "Hov". */
} ccsd_method;

typedef enum {
  CCSD_ACCEL_DIIS = 0, /* Pulay DIIS (Sec. "Coupled cluster implementation"): diis_dim amplitude and
                          error vectors, t <- sum_i c_i t_i with sum_i c_i = 1 minimising
                          |sum_i c_i e_i|, e = S/D; the oldest vector is dropped */
  CCSD_ACCEL_CROP = 1  /* CROP (Ziolkowski et al. 2008; the lighter-memory alternative the same
                          section names): the same solve, but the subspace keeps the optimal
                          combinations (sum c t, sum c e) in place of the newest raw pair, so
                          that few vectors suffice (diis_dim = 3 is the usual choice) */
} ccsd_accelerator;

typedef struct {
  int max_iter;       /* iteration cap for ccsd_iterate (default 50) */
  double tol;         /* convergence threshold on the update norm (default 1e-10) */
  int norm;           /* 0: max |S/D| (default), 1: 2-norm of S/D over unique amplitudes */
  int diis_dim;       /* DIIS subspace size, 0 = off (default 8) */
  int diis_start;     /* first iteration that extrapolates (default 2) */
  double level_shift; /* added to virtual orbital energies in the denominators only (default 0) */
  int precision;      /* ccsd_precision (default CCSD_PREC_FP64) */
  int slices;         /* split precision: e4m3 digits per operand, 1..14 with digit_bits * slices <= 56
                         (default 0 = about 39 bits: 8 digits of 5 bits, 10 of 4) */
  int store_w;        /* 1: store <ab||cd> (packed); 0: never store it, rebuild it in blocks of rows
                         from the DF factors inside each ladder evaluation (DF input only) (default 1) */
  int profile;        /* 1: record per-term CUDA-event timings (default 0) */
  void* stream;       /* cudaStream_t, NULL = legacy default stream */
  double split_min_flops; /* split precision: contractions of at least this many flops (8 per complex
                             multiply-add) run on the tensor cores when a cost model of this GPU says
                             that is faster than FP64; the ladder always does; <= 0 sends every GEMM
                             there (default 1e8) */
  int df_block;       /* store_w = 0: virtual indices a per rebuilt block of <ab||cd> rows
                         (default 0 = as many as fit about 6 GB of (ac|bd), held in the residual plan's
                         scratch region) */
  int autotune;       /* 1: at creation, time every FP64 GEMM of the plan in each tile shape and keep
                         the fastest (default 0: a cost model picks the shape) */
  int digit_bits;     /* split precision: bits per digit, 1..5 (default 0 = 5). Digits are integers
                         e4m3 holds exactly (|d| <= 16); at 5 bits every row is scaled below 1/2
                         so that its first digit stays within 16 too */
  int complex_4m;     /* FP64 GEMMs: 1 = four real products per complex product (4M); 0 = three
                         (3M: Ar Br, Ai Bi, (Ar + Ai)(Br + Bi), combined once per output), about
                         1.28x fewer FP64 operations (default 0) */
  double split_budget; /* split precision: bytes of digits (both operands) one tensor-core GEMM call
                          may hold; larger GEMMs run in chunks of M, N and then K (default 0 = a
                          quarter of the free device memory at creation, 4 to 8 GB) */
  int method;          /* ccsd_method (default CCSD_METHOD_CCSD) */
  int accelerator;     /* ccsd_accelerator: the subspace method of ccsd_iterate and ccsd_lambda_iterate
                          when diis_dim > 0 (default CCSD_ACCEL_DIIS) */
  int diverge_iters;   /* growth check of ccsd_iterate / ccsd_lambda_iterate / ccsd_batch_iterate: the
                          update norm rising in this many consecutive iterations, by more than
                          diverge_factor overall, is CCSD_ERR_DIVERGED (default 8; 0 = off). The rule is
                          ccsd_divergence_index */
  double diverge_factor; /* growth check factor (default 1e3) */
  int vovv_block;      /* rows a of <ak||cd> unpacked at a time for the H^{ak}_{ci} term and its Lambda
                          adjoint (default 0 = as many as fit about 1 GB) */
  double permute_cache_limit; /* integral blocks of up to this many bytes keep a copy in each other
                                 layout a contraction reads; larger ones are permuted at each use
                                 (default 0 = 2 GiB; < 0: none is kept) */
} ccsd_opts;

/* Fill opts with the defaults listed above. */
void ccsd_default_opts(ccsd_opts* opts);

/*
 * Create a context: copy eps (n doubles, host), the optional Fock matrix
 * (n*n, host) and the integrals (host) to the device, build the integral
 * blocks (oooo, ooov, oovv, vovo, vovv, and <ab||cd> packed over a<b, c<d),
 * allocate every tensor of the iteration up front and set the amplitudes to the
 * MP2 guess (one denominator update from t = 0).
 * Errors: CCSD_ERR_ARG for o < 1, v < 1, naux < 1 (DF), NULL pointers, a Fock
 * matrix or DF factor that is not Hermitian to 1e-12 relative; CCSD_ERR_OOM.
 * On error *out is set to NULL.
 */
ccsd_status ccsd_create(int o, int v, const double* eps, const ccsd_z* fock, ccsd_int_kind kind,
                        const ccsd_z* ints, int naux, const ccsd_opts* opts, ccsd_ctx** out);

/*
 * Residuals S^a_i, S^{ab}_{ij} of Appendix A at the given amplitudes
 * (t1: o*v, t2: o*o*v*v; outputs r1, r2 of the same sizes). Does not change the
 * context's current amplitudes: they are restored afterwards from a copy of t1 and of the
 * unique doubles (i<j, a<b), which rebuilds t2 exactly when it is antisymmetric in both
 * pairs (as every t2 of the iterations is, to rounding). t1/t2 may be NULL to use the
 * current ones.
 */
ccsd_status ccsd_residual(ccsd_ctx* ctx, const ccsd_z* t1, const ccsd_z* t2, ccsd_z* r1, ccsd_z* r2,
                          int on_device);

/*
 * Run up to max_iter iterations from the current amplitudes (max_iter <= 0:
 * opts.max_iter): residual, denominator update t <- t + S/D, DIIS, norm.
 * Returns CCSD_OK on convergence (norm <= opts.tol), CCSD_ERR_NOT_CONVERGED at
 * the cap, CCSD_ERR_DIVERGED on NaN/Inf (amplitudes restored to the last finite
 * iterate: t1 and the unique doubles, t2 rebuilt from them) or on sustained growth of the norm (opts.diverge_iters, diverge_factor;
 * the amplitudes are those of the last, finite, iteration). The growth record runs
 * across calls and restarts at ccsd_set_amplitudes. iters_done / res_norm may be NULL.
 */
ccsd_status ccsd_iterate(ccsd_ctx* ctx, int max_iter, int* iters_done, double* res_norm);

/*
 * The growth rule of the iterations (the paper has no counterpart; a safeguard of the
 * library), applied to a host sequence of update norms: the 1-based index of the first
 * norm norms[k] that ends a run of `iters` or more consecutive increases
 * (norms[k-r] < ... < norms[k], r >= iters) with norms[k] > factor * norms[k-r], the norm
 * where the run began; 0 if there is none, or if iters <= 0. A non-finite norm ends the
 * sequence (the iterations report it as divergence on their own). count < 0 or a NULL
 * norms with count > 0 returns -1.
 */
int ccsd_divergence_index(const double* norms, int count, int iters, double factor);

/* Energy of the current amplitudes: sum_ia f_ia t^a_i + 1/4 sum <ij||ab> tau^{ab}_{ij}, the second
 * sum taken once over the unique i < j, a < b (t2 is antisymmetric in (i,j) and in (a,b)). */
ccsd_status ccsd_energy(ccsd_ctx* ctx, ccsd_z* e);

/*
 * Perturbative triples corrections at the current amplitudes (normally converged),
 * following the appendix "Working equations for perturbative Triples" (Eqs. W-term,
 * Z-term, Y-term, 4order-term, 5order-term). The outputs are real and in Hartree, and each
 * is a correction to add to the CCSD energy:
 *   out[0] = E(+T)  = -sum |X|^2 / D                        (fourth order)
 *   out[1] = E((T)) = E(+T) - sum Re(X Z) / D               (fifth order)
 *   out[2] = E(-T)  = E(+T) + sum Re(X conj(Y))             (alternative fifth order)
 * The sums run over i<j<k and a<b<c, which equals the appendix's full sums divided by 36.
 *   - X is W^{abc} + W^{bca} + W^{cab}, the connected triples <Phi^{abc}_{ijk}| V T2 |Phi_0>.
 *     The integrals of W are read as <ab||ie> and <am||jk>, the Hermitian partners of the
 *     printed <ie||ab> and <jk||am>.
 *   - Z is the conjugate of <Phi^{abc}_{ijk}| V T1 + F T2 |Phi_0>.
 *   - Y is the triples part of exp(T1 + T2)|Phi_0>.
 *   - D = e_a + e_b + e_c - e_i - e_j - e_k, over the real diagonal of the Fock matrix
 *     (no level shift).
 * W comes from complex GEMMs, one occupied pair i<j at a time, with up to max_batch
 * consecutive k > j per batch. In an FP64 context every step is FP64: batched GEMMs on the
 * FP64 tensor path. In a split-precision context (opts.precision) the e-terms of W, three
 * P(v) x v x v products per triple, are split GEMMs on the tensor cores. Their digits are cut
 * once per call; their error is that of the split GEMM, 2^(1 - bits*slices) relative to each
 * row's scale. Everything else stays FP64.
 *   max_batch <= 0 sizes the batch to a quarter of the free device memory, at most 8 GB.
 *   Each triple of a batch needs 2 * v * v(v-1)/2 complex elements of workspace.
 * out: host, 3 doubles.
 * pair_terms: NULL, or host with o*o*3 doubles. pair_terms[(i*o + j)*3 + m] receives the
 * contribution of the triples (i, j, k > j) to out[m]; it is zero unless i < j. out[m] is
 * the sum of these contributions in pair order.
 * The workspace is allocated by this call and freed before it returns. Synchronises the
 * stream. The result is reproducible run to run.
 * Errors: CCSD_ERR_ARG for a NULL out or a negative max_batch; CCSD_ERR_OOM when the
 * workspace for one triple (and, split, the digit sets) does not fit; CCSD_ERR_TIMEOUT if a
 * bounded wait of the split GEMM gave up.
 */
ccsd_status ccsd_triples(ccsd_ctx* ctx, int max_batch, double* out, double* pair_terms);

/*
 * Lambda equations and the one-body density at the current amplitudes (normally converged),
 * appendices "Working equations for CCSD lambda equations" and "... Lagrange 1-body density
 * matrix". The appendix prints the Lambda equations with intermediates it leaves to its
 * reference. They are the stationarity conditions of the coupled-cluster Lagrangian
 * L = E(t) + sum_mu lambda_mu S_mu(t) with respect to t, and this is how the library evaluates
 * them: R = dL/dt, the adjoint of the residual, term by term. The multipliers are
 * l1[i*v + a] = lambda^i_a and l2 [i][j][a][b] = lambda^{ij}_{ab}, antisymmetric like t2.
 * Available for method = CCSD with store_w = 1 (CCSD_ERR_UNSUPPORTED otherwise). The
 * multipliers and their DIIS history are created, at zero, by the first call that needs them.
 *
 * ccsd_lambda_residual: R1 (o*v) and R2 (o*o*v*v; the derivative with respect to each unique
 *   t^{ab}_{ij}, extended antisymmetrically) at the given multipliers. With l1 and l2 given
 *   they become the context's multipliers; with both NULL the context's own are used.
 * ccsd_lambda_iterate: up to max_iter updates lambda <- lambda + R/D, with the amplitudes'
 *   denominators, level shift, subspace accelerator (DIIS or CROP) and norm. Returns CCSD_OK
 *   on convergence (norm <= tol), CCSD_ERR_NOT_CONVERGED at the cap, CCSD_ERR_DIVERGED on
 *   NaN/Inf or sustained growth (as ccsd_iterate; the record restarts with each call).
 * ccsd_get_lambda: copy the multipliers out.
 * ccsd_density: gamma (host, n*n, occupied first) =
 *   <0| (1 + Lambda) exp(-T) a+_q a_p exp(T) |0>, less the reference occupation delta_ij, at
 *   the current amplitudes and multipliers. The printed blocks are used, with the occupied
 *   block transposed into the convention of the other three. With symmetrize != 0, the
 *   Hermitian part (gamma + gamma^+)/2 is returned.
 */
ccsd_status ccsd_lambda_residual(ccsd_ctx* ctx, const ccsd_z* l1, const ccsd_z* l2, ccsd_z* r1, ccsd_z* r2,
                                 int on_device);
ccsd_status ccsd_lambda_iterate(ccsd_ctx* ctx, int max_iter, int* iters_done, double* res_norm);
ccsd_status ccsd_get_lambda(ccsd_ctx* ctx, ccsd_z* l1, ccsd_z* l2, int on_device);
ccsd_status ccsd_density(ccsd_ctx* ctx, ccsd_z* gamma, int symmetrize);

/* Copy the current amplitudes out / in (checkpoint and resume). Setting resets DIIS. t2 must be
 * antisymmetric in (i,j) and in (a,b): the packed contractions and the energy read its unique
 * elements. */
ccsd_status ccsd_get_amplitudes(ccsd_ctx* ctx, ccsd_z* t1, ccsd_z* t2, int on_device);
ccsd_status ccsd_set_amplitudes(ccsd_ctx* ctx, const ccsd_z* t1, const ccsd_z* t2, int on_device);

/*
 * Copy an intermediate of the last residual evaluation to `out` (count complex
 * elements expected). Names and layouts: "tau" [i][j][a][b], "Hvv" [a][c],
 * "Gvv" [a][c], "Hoo" [k][i], "Goo" [k][i], "Hov" [k][c], "Hvoov" [i][a][k][c]
 * (= H^{ak}_{ci}), "C" [k][b][i][j], "A" [k][l][i][j], "ladder" [i][j][a][b]
 * (= 1/2 sum_cd <ab||cd> tau^{cd}_{ij}). CCSD_ERR_ARG for an unknown name or a
 * wrong count.
 */
ccsd_status ccsd_get_tensor(ccsd_ctx* ctx, const char* name, ccsd_z* out, size_t count, int on_device);

/*
 * Per-op device timings (opts.profile = 1): CUDA events recorded between the
 * ops of the residual plan and the update / norm / DIIS steps, inside the
 * iteration's CUDA graph, followed by the ops of the Lambda plan (names "L:...",
 * per Lambda iteration) when Lambda iterations were timed. Writes up to `cap`
 * (name, average milliseconds per evaluation) pairs, averaged over the evaluations
 * since the previous call, and resets the averages (cap <= 0 only queries *n). *n
 * receives the number of timed segments (0 if nothing was timed). Names are owned by
 * the context.
 */
ccsd_status ccsd_timings(ccsd_ctx* ctx, const char** names, double* ms, int cap, int* n);

/*
 * Scalar facts about a context: "kernels_per_iteration" (kernel nodes of the
 * iteration graph), "device_bytes" (device memory the context allocated, the cached
 * operand permutations of its plans included), and parts of it: "plan_scratch_bytes" (the
 * residual plan's temporaries), "plan_cached_bytes" (its permuted copies of integral blocks),
 * "gemm_workspace_bytes", "split_workspace_bytes", "diis_bytes" (the subspace history);
 * "iterations_run", "plan_ops", "o", "v",
 * "lambda_iterations", "lambda_kernels_per_iteration" (kernel nodes of the Lambda iteration
 * graph, captured at the first ccsd_lambda_iterate), and with opts.profile = 1
 * "lambda_op_ms:<op>" (average device ms per Lambda iteration of the Lambda-plan ops named <op>,
 * e.g. "L:ladder:gemm"). Of the last ccsd_triples call: "triples_batch" (triples per
 * batch), "triples_batches", "triples_launches" (kernels launched), and with
 * opts.profile = 1 the device time in ms of its e-term GEMMs ("triples_egemm_ms"),
 * m-term GEMMs ("triples_mgemm_ms") and energy kernels ("triples_energy_ms"), summed
 * over the batches (0 without profiling). CCSD_ERR_ARG for an unknown key.
 */
ccsd_status ccsd_query(const ccsd_ctx* ctx, const char* key, double* value);

/*
 * The engine's complex GEMM on device pointers (row-major, complex double):
 *   C = alpha * opA(A) * opB(B) + beta * C
 * opA(A)(m,k) = transA ? A[k*lda + m] : A[m*lda + k], conjugated if conjA; likewise B
 * with (k,n) = transB ? B[n*ldb + k] : B[k*ldb + n]. precision: CCSD_PREC_FP64 (FP64
 * tensor-core path). cfg < 0 picks the tile shape, cfg >= 0 forces one (0..6). The
 * optional workspace (ws_elems complex elements, device) enables split-K for small
 * outputs; without it the GEMM does not split, and a workspace smaller than the
 * preferred split count takes as many partials (M*N each) as it holds, when that is
 * at least two. Synchronous on `stream`.
 * CCSD_ERR_ARG for negative sizes, NULL pointers or a bad cfg.
 */
ccsd_status ccsd_zgemm(int precision, int transA, int conjA, int transB, int conjB, long long M, long long N,
                       long long K, ccsd_z alpha, const ccsd_z* A, long long lda, const ccsd_z* B, long long ldb,
                       ccsd_z beta, ccsd_z* C, long long ldc, ccsd_z* workspace, size_t ws_elems, int cfg,
                       void* stream);

/*
 * Split-precision complex GEMM (Ozaki-style digit slices on the tcgen05 tensor
 * cores), same operation and layouts as ccsd_zgemm:
 *   C = alpha * opA(A) * opB(B) + beta * C   (complex double in and out, device pointers)
 * kind 0: e4m3 digits (kind::f8f6f4), bits <= 5; kind 1: bf16 digits (kind::f16), bits <= 8.
 * Each row of opA(A) and each column of opB(B) is scaled by a power of two and cut into
 * `slices` integer digits of `bits` bits (at 5 bits in e4m3 the scale leaves one bit of
 * headroom so that every digit is an integer the type holds exactly); the digits of -x are
 * exactly the negated digits of x. Digit products of equal weight are summed exactly in
 * FP32 tensor-memory accumulators over K ranges short enough to stay exact, and combined
 * in FP64. A K of at most 4 blocks (512 e4m3, 256 bf16 elements) with at most 8 digits
 * runs on a second kernel that keeps every weight in tensor memory and writes each output
 * once. Error ~ 2^(-bits*slices) relative to the row/column scales (2^(1-bits*slices)
 * with headroom). Results are bit-reproducible run to run (every output element has one
 * owning thread; K-split partials are summed in a fixed order). ccsd_split_describe
 * reports how a shape is scheduled.
 * workspace: device memory of at least ccsd_split_workspace(...) bytes. Synchronous on
 * `stream`. CCSD_ERR_TIMEOUT if a bounded device wait gave up.
 */
size_t ccsd_split_workspace(int kind, int bits, int slices, long long M, long long N, long long K);
ccsd_status ccsd_split_zgemm(int kind, int bits, int slices, int transA, int conjA, int transB, int conjB,
                             long long M, long long N, long long K, ccsd_z alpha, const ccsd_z* A, long long lda,
                             const ccsd_z* B, long long ldb, ccsd_z beta, ccsd_z* C, long long ldc,
                             void* workspace, size_t ws_bytes, void* stream);

/*
 * How ccsd_split_zgemm runs an M x N x K product (a scheduling record, the paper has no
 * counterpart): out[6] (host) receives 1 for the short-K kernel (else 0), 1 when the
 * operands are swapped (M on the narrow tile side), the tile width, the CTAs per cluster
 * (2: two CTAs share the long operand's tile by TMA multicast), the CTAs along K and the
 * output tiles (the last four 0 for the short-K kernel). Queries the current device's
 * cluster occupancy; launches nothing. CCSD_ERR_ARG on a bad configuration or NULL.
 */
ccsd_status ccsd_split_describe(int kind, int bits, int slices, long long M, long long N, long long K, int* out);

/*
 * Accumulation probe of the split GEMM's tensor-core path: C[m][n] = sum_k A[m][k] B[n][k]
 * (real, row-major, device) for integer-valued A, B that fit the digit type of `kind`
 * (|x| <= 16 for e4m3, <= 256 for bf16), accumulated in one FP32 TMEM accumulator over
 * the whole K. Used to test that integer sums below 2^24 come out exact.
 */
ccsd_status ccsd_split_probe(int kind, long long M, long long N, long long K, const double* A, const double* B,
                             double* C, void* workspace, size_t ws_bytes, void* stream);

/*
 * Self-test of the failure path of the split GEMM's device waits (the paper has no
 * counterpart). Every wait of the kernel is bounded; this runs one small split GEMM
 * (its own ~1 MB of device memory, allocated and freed here) whose TMA producer issues
 * no copies, with a ~2 ms wait budget, so that the MMA issuer's first wait gives up.
 * The kernel then raises its abort flag, frees its tensor memory and returns.
 * Returns CCSD_ERR_TIMEOUT when that happened as intended (the device stays usable),
 * CCSD_ERR_CUDA if the wait did not give up or a CUDA call failed. Synchronous on stream.
 */
ccsd_status ccsd_split_wait_selftest(void* stream);

/*
 * ccsd_zgemm for callers that cannot allocate device memory. The paper has no
 * counterpart: this is a service of the library, not a step of the method.
 *
 * Who needs it: callers that run inside another framework's memory budget (a
 * caching allocator such as PyTorch's owns the device memory, and memory taken
 * behind its back can make its own allocations fail), callers in a
 * latency-critical loop (cudaMalloc / cudaFree can synchronise the device), and
 * callers that must keep the device footprint they fixed at start-up. Such a
 * caller cannot hand ccsd_zgemm a split-K workspace.
 *
 * Same arguments and result as ccsd_zgemm without the workspace: the split-K
 * partials go to a fixed array of 2^18 complex doubles (4 MiB) that the library
 * keeps in device memory; every GPU that loads the library holds it until the
 * process exits. The call allocates nothing (no cudaMalloc, cudaFree or any
 * allocating library routine). Each call looks up the array's address on the
 * current device (cudaGetSymbolAddress, which allocates nothing), so the
 * address stays valid after a device reset. Limit: M*N <= 2^17 complex
 * elements (at least two split partials must fit, and up to
 * 2^18 / (M*N) of them are used); larger outputs return
 * CCSD_ERR_ARG with a message naming the limit (use ccsd_zgemm with a
 * workspace for those). All calls share the one array and it keeps the last
 * call's contents; nothing in it has to start at zero, because every partial a
 * call reads it wrote itself earlier in that call. Calls that overlap on the
 * GPU (different streams or host threads at the same time) race on the array:
 * serialise them. Synchronous on `stream`; errors via ccsd_last_error(NULL).
 */
ccsd_status ccsd_zgemm_noalloc(int precision, int transA, int conjA, int transB, int conjB, long long M,
                               long long N, long long K, ccsd_z alpha, const ccsd_z* A, long long lda,
                               const ccsd_z* B, long long ldb, ccsd_z beta, ccsd_z* C, long long ldc, int cfg,
                               void* stream);

/*
 * Batched solve of many independent systems (the paper's calculations are one
 * system at a time; this is a throughput mode of the library). Each system k has
 * o[k], v[k], eps[k] (n_k doubles), DF factors B[k] ([naux[k]][n_k][n_k]) and the
 * Fock matrix diag(eps[k]). All systems share opts (opts->stream is the stream the
 * batch launches on). One batch iteration is one CUDA graph launch in which every
 * still-active system runs its own iteration on its own stream (fork/join), so the
 * small systems fill the GPU together; systems drop out as they converge
 * (norm <= opts->tol) or diverge. Amplitudes start at each system's MP2 guess.
 */
typedef struct ccsd_batch ccsd_batch;
ccsd_status ccsd_batch_create(int nsys, const int* o, const int* v, const double* const* eps,
                              const ccsd_z* const* B, const int* naux, const ccsd_opts* opts, ccsd_batch** out);
/* Up to max_iter batch iterations (<= 0: opts.max_iter). Per system (arrays of nsys, may be
 * NULL): iterations run, last norm, and status (CCSD_OK converged, CCSD_ERR_NOT_CONVERGED,
 * CCSD_ERR_DIVERGED on NaN/Inf or sustained growth, as ccsd_iterate). Returns CCSD_OK if every system converged, else CCSD_ERR_NOT_CONVERGED
 * (or the first CUDA error). */
ccsd_status ccsd_batch_iterate(ccsd_batch* b, int max_iter, int* iters_done, double* res_norm, int* status);
/* Energies of the current amplitudes of every system (nsys values). */
ccsd_status ccsd_batch_energy(ccsd_batch* b, ccsd_z* e);
/* Amplitudes of system k (as ccsd_get_amplitudes). */
ccsd_status ccsd_batch_get_amplitudes(ccsd_batch* b, int k, ccsd_z* t1, ccsd_z* t2, int on_device);
const char* ccsd_batch_last_error(const ccsd_batch* b);
void ccsd_batch_destroy(ccsd_batch* b);

/* Message for the last failing call on ctx; with ctx NULL, of the last failed call made without a
 * context (ccsd_create, ccsd_zgemm, ccsd_zgemm_noalloc) on this host thread. */
const char* ccsd_last_error(const ccsd_ctx* ctx);

/* Free every device buffer of the context. NULL is a no-op. */
void ccsd_destroy(ccsd_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* CCSD_H */
