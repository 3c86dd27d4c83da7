/*
 * sylv.h -- C ABI of the GB300 (sm_103a) factorized Krylov solver for the
 * Sylvester equation
 *
 *        A X + X B = C1 C2^T,   A: n x n, B: m x m sparse, C1: n x s, C2: m x s,
 *
 * (Satake, Fukaya, Sogabe, Zhang, "Factorized Krylov subspace methods for
 * solving large Sylvester equations", eq. 1.1) and its Lyapunov case
 * B = A^T, C2 = C1 (Sec. 4.3).  The solution is returned in factored form
 * X = V X^ W^T with V (n x r), W (m x r) column-orthonormal block Krylov
 * bases and X^ (r x r) small (Corollary 3.2).
 *
 * Conventions for every entry point:
 *  - Host pointers unless stated otherwise.  Dense matrices are column-major
 *    with leading dimension = number of rows.  CSR is 0-based with int32
 *    indices and float64 values; column indices inside a row may come in any
 *    order, duplicates are summed.
 *  - Return value: 0 (SYLV_OK) or one of the sylv_status codes below.  No
 *    entry point aborts or exits; after SYLV_ECUDA the handle should be
 *    destroyed.  sylv_strerror() gives a message; sylv_last_error() gives the
 *    detail of the last failure on the calling thread.
 *  - A handle is not thread safe: one thread at a time per handle.
 */
#ifndef SYLV_H_
#define SYLV_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SYLV_OK = 0,         /* converged: ||R^_k|| <= tol ||R^_0|| (Algorithms 4.1/4.2 test) and, with the
                          true-residual certificate on (the default), true_rel_bound <= tol */
  SYLV_EINVAL = 1,     /* bad argument: shape, NULL, malformed CSR, s < 1, tol < 0 ... */
  SYLV_ENOMEM = 2,     /* device allocation failed */
  SYLV_ENOTCONV = 3,   /* maxit reached; the factors hold the last iterate */
  SYLV_EBREAKDOWN = 4, /* zero denominator (CG: <P^,Q^> <= 0; BiCGSTAB: <R~0,Q^(1:s,1:s)> = 0,
                          omega = 0, rho = 0) or a rank-deficient C1 or C2; a later basis block
                          that loses part of its rank is deflated (its dependent columns become
                          zero basis columns), not a breakdown */
  SYLV_ENONFINITE = 5, /* NaN/Inf in the iteration (e.g. from non-finite inputs) */
  SYLV_ETIMEOUT = 6,   /* the host gave up waiting for the device (sylv_options.timeout_s) */
  SYLV_ECUDA = 7,      /* a CUDA runtime call failed */
  SYLV_ESTATE = 8      /* call out of order (e.g. factors requested before any solve) */
} sylv_status;

typedef enum {
  SYLV_FP64 = 0, /* factors, sparse products and Gram products in float64 */
  SYLV_MIXED = 1 /* factors, SpMM and Gram in float32 (FP32 accumulation inside a CTA),
                    small coefficient recurrences, residual checks and an outer
                    iterative refinement on the true residual in float64 */
} sylv_precision;

/* Sparse matrix in CSR form (host memory, read during sylv_create only). */
typedef struct {
  int64_t nrows, ncols, nnz;
  const int32_t* row_ptr; /* nrows + 1 entries, row_ptr[0] = 0, nondecreasing, row_ptr[nrows] = nnz */
  const int32_t* col_idx; /* nnz entries in [0, ncols) */
  const double* val;      /* nnz entries */
} sylv_csr;

typedef struct {
  int32_t precision;   /* sylv_precision */
  int32_t lyapunov;    /* 1: B = A^T and C2 = C1 (Sec. 4.3); pass B = NULL, C2 = NULL */
  int32_t poll_every;  /* iterations enqueued between host polls of the device status (0: 8) */
  int32_t refine_max;  /* SYLV_MIXED: maximum outer refinement rounds (0: 12) */
  double deflate_tol;  /* block Krylov exhaustion threshold delta (0: 1e-12 FP64, 1e-6 mixed) */
  double timeout_s;    /* host wait limit per solve (0: 3600 s) */
  void* cuda_stream;   /* cudaStream_t to run on, or NULL for a stream owned by the handle */
  int32_t profile;     /* 1: time every kernel launch with CUDA events (see sylv_get_profile) */
  int32_t no_true_residual; /* SYLV_FP64 only: 1 skips the float64 true-residual certificate after the
                               solve; the stop is then the test of Algorithms 4.1/4.2 alone */
  int32_t stream_mode; /* 0: auto (SYLV_MIXED and SYLV_FP64 block Arnoldi bases on the tensor cores run the
                          two bases on their own streams, ahead of the small side; the CUDA-core SYLV_FP64
                          kernels use one stream, where FP64-bound kernels gain nothing from overlap);
                          1: everything on one stream (clean per-kernel profiles); 2: concurrent */
  int32_t small_gemm;  /* products of the small Sylvester operator, eq. 3.7, in BiCGSTAB: 0 auto (tensor
                          cores from order r = 448 on), 1 CUDA cores only (float64, or double-float in
                          SYLV_MIXED), 2 tensor cores at every order; the tensor-core form splits both
                          factors into BF16 digits (Ozaki scheme) and keeps float64 accuracy */
  int32_t basis_gemm;  /* SYLV_FP64 block Arnoldi bases (BiCGSTAB, CGS, GPBiCG): the Gram products and block
                          updates of eq. 3.4, 0 auto (tensor cores; CUDA cores if their digit planes do not
                          fit in device memory), 1 CUDA cores (float64 FMAs), 2 tensor cores (SYLV_ENOMEM if
                          they do not fit).  The tensor-core form holds each basis block, once it is built,
                          as five FP16 planes of 11-bit digits in two layouts (20 bytes per basis element
                          besides the 8 of float64) and splits the other operand into eight planes of 7-bit
                          digits; the products are exact sums of digit products, rounded once to float64
                          (Ozaki scheme) */
  double stop_margin;  /* with the true-residual certificate on (SYLV_FP64 by default): the recurrence test of
                          Algorithms 4.1/4.2 stops at ||R^_k|| <= stop_margin * tol * ||R^_0|| (0: 0.4), so
                          that the certificate (sylv_info.true_rel_bound <= tol) holds at the first check.
                          1.0 gives the printed test.  SYLV_MIXED inner solves are not affected */
  int32_t cert_gemm;   /* where the certificate's tall-skinny products with the bases run: 0 auto (on the
                          tensor cores, on digit planes of the bases -- the float64 Arnoldi bases' own, or
                          split once after the solve from bases of 2^25 elements or more when they take at
                          most 30% of the free device memory; otherwise double-float kernels on the FP32
                          pipes), 1 always the double-float kernels, 2 digit planes at every size (within
                          the same memory rule).  Both are accurate far below the certified bound's
                          resolution; the choice changes the time only */
} sylv_options;

typedef struct {
  int32_t status;       /* sylv_status of the solve */
  int32_t iters;        /* completed iterations k (sum over refinement rounds in SYLV_MIXED) */
  int64_t matvecs;      /* sparse block products A*V_j (equal count for B^T*W_j), all rounds */
  int64_t width;        /* r: columns of V and W returned; X^ is r x r */
  double rel_res;       /* ||R^_k|| / ||R^_0||, the monitored residual of Algorithms 4.1/4.2 */
  double true_rel_res;  /* estimate of ||C1 C2^T - A X - X B||_F / ||C1 C2^T||_F in float64 (unbiased in
                           its square, from Gaussian probes of the residual), or -1 if not computed */
  double solve_ms;      /* wall time of the solve call on the host */
  int32_t refinements;  /* SYLV_MIXED: outer refinement rounds used */
  int32_t reserved;
  int64_t kernel_launches; /* CUDA kernels this call enqueued (no-ops after a stop included) */
  double true_rel_bound;   /* upper bound on the true relative residual that holds with probability
                              >= 1 - 1e-4 over the probes, whatever the residual (or -1 if not computed).
                              With the certificate on, SYLV_OK means true_rel_bound <= tol; a solve whose
                              recurrence met its test but whose bound did not returns SYLV_ENOTCONV
                              (SYLV_MIXED first runs more refinement rounds) */
} sylv_info;

/* Per-kernel-class totals of the last solve (sylv_options.profile = 1).
 * bytes / flops are the algorithmic amounts (each operand read once, each
 * result written once), so bytes / (ms 1e-3) is the achieved bandwidth. */
typedef struct {
  char name[24];      /* "spmm", "gram", "update", "cholqr_scale", "reduce", "small_gemm", ... */
  int64_t launches;
  double ms;          /* summed kernel time (CUDA events on the solve stream) */
  double bytes;       /* summed algorithmic DRAM bytes */
  double flops;       /* summed algorithmic floating-point operations */
} sylv_kernel_stat;

typedef struct sylv_handle sylv_handle;

/* Default options (FP64, Sylvester, poll every 8 iterations). */
void sylv_default_options(sylv_options* opt);

/*
 * Problem statement, eq. 1.1 (Sec. 1).  Checks the input and copies A, B^T
 * (built from B on the host), C1 and C2 to device memory; the caller keeps
 * ownership of its buffers.  The thin QR factorisations C1 = V_1 R_L,
 * C2 = W_1 R_R (CholQR2, diag(R) > 0) that start Algorithms 4.1/4.2 run at the
 * start of each solve.
 *   A        n x n CSR;   B  m x m CSR (NULL when opt->lyapunov)
 *   C1       n x s column-major;  C2 m x s column-major (NULL when opt->lyapunov)
 *   s        number of columns of C1, C2 (1 <= s <= 8)
 *   opt      NULL for defaults
 *   out      receives the handle (NULL on failure)
 * Errors: SYLV_EINVAL (shapes, CSR), SYLV_ENOMEM, SYLV_ECUDA (also: no device),
 *         SYLV_ENONFINITE (NaN/Inf in A, B, C1 or C2).
 */
int sylv_create(const sylv_csr* A, const sylv_csr* B, const double* C1, const double* C2, int64_t s,
                const sylv_options* opt, sylv_handle** out);

/*
 * Batched Lyapunov equations A_i X_i + X_i A_i^T = C_i C_i^T, i = 0..count-1, of
 * uneven sizes n_i and block widths s_i (1..8), solved together by factorized CG
 * (Algorithm 4.1 in the one-basis form of Sec. 4.3): every phase of an iteration
 * is one persistent launch over all running instances, and one iteration is a
 * CUDA graph replayed until every instance has converged.  Row-chunk size and
 * grid size of the streaming phases are picked by a built-in autotuner on the
 * first solve.
 *   A[i]   n_i x n_i CSR (host);  C1[i]  n_i x s[i] column-major (host)
 *   B, C2  must be NULL;  opt->lyapunov must be 1; float64 only (SYLV_FP64)
 * sylv_cg(h, ...) then solves all instances (sylv_bicgstab is EINVAL); its info
 * aggregates: status OK only if every instance converged (else the first failing
 * status), iters = max, matvecs / width = sums, rel_res / true_rel_res = max.
 * Per-instance results: sylv_batch_instance + the single-instance calls.
 */
int sylv_create_batch(int32_t count, const sylv_csr* A, const sylv_csr* B, const double* const* C1,
                      const double* const* C2, const int64_t* s, const sylv_options* opt, sylv_handle** out);

/*
 * The internal handle of instance `inst` of a batched handle (owned by the batch:
 * do not destroy it).  sylv_get_factors / sylv_get_history / sylv_get_hessenberg
 * on it return that instance's results of the last batched solve.
 */
int sylv_batch_instance(sylv_handle* h, int32_t inst, sylv_handle** out);

/*
 * Factorized CG, Algorithm 4.1 (A, B symmetric positive definite; block
 * Lanczos bases).  Runs at most maxit iterations from X_0 = 0 and stops at the
 * first k with ||R^_{k+1}|| <= tol ||R^_0||.  The factors V_{k+1}, X^_{k+1},
 * W_{k+1} (r = (k+1)s) stay on the device for sylv_get_factors.
 * Device memory for maxit iterations is (re)allocated here.  A rank-deficient
 * C1 or C2 (including C = 0) returns SYLV_EBREAKDOWN.
 * Returns the status also stored in info->status (info may be NULL).
 */
int sylv_cg(sylv_handle* h, double tol, int32_t maxit, sylv_info* info);

/*
 * Factorized BiCGSTAB, Algorithm 4.2 (general A, B; block Arnoldi bases with
 * block classical Gram-Schmidt applied twice).  Returns V_{2k+2}, X^_{k+1},
 * W_{2k+2} (r = (2k+2)s).  Otherwise as sylv_cg.
 */
int sylv_bicgstab(sylv_handle* h, double tol, int32_t maxit, sylv_info* info);

/*
 * Factorized CGS (conjugate gradient squared, Sonneveld 1989), which Sec. 4 names
 * among the methods the factorized approach carries over to; the paper prints no
 * listing, so the recurrence is CGS on the Kronecker system (eq. 1.2) written with
 * the matrix operations of Sec. 2 and factorized as Algorithm 4.2 is: the same block
 * Arnoldi bases (two steps per iteration), additions of padded small matrices
 * (eq. 3.5), inner products with R~_0 = R_0 on the leading s x s block (eq. 3.6),
 * and two applications of the small operator of eq. 3.7 per iteration.  General A,
 * B; returns V_{2k+2}, X^_{k+1}, W_{2k+2} as sylv_bicgstab.  Batched handles:
 * SYLV_EINVAL.  Otherwise as sylv_cg.
 */
int sylv_cgs(sylv_handle* h, double tol, int32_t maxit, sylv_info* info);

/*
 * Factorized CR (conjugate residual, Stiefel 1955), the other method Sec. 4 names for
 * symmetric problems; no listing in the paper, so the recurrence is CR on the Kronecker
 * system (eq. 1.2) in the matrix operations of Sec. 2, factorized as Algorithm 4.1 is:
 * block Lanczos bases (A, B symmetric; not checked), one step per iteration plus one
 * before the first, the small operator of eq. 3.7 applied to R^ (one per iteration),
 * L(P) by its recurrence.  Lyapunov handles use the one-basis form of Sec. 4.3.
 * Returns V_{k+1}, X^_{k+1}, W_{k+1} as sylv_cg; matvecs = iters + 1.  Batched handles:
 * SYLV_EINVAL.  Otherwise as sylv_cg.
 */
int sylv_cr(sylv_handle* h, double tol, int32_t maxit, sylv_info* info);

/*
 * Factorized GPBiCG (generalized product-type BiCG, Zhang 1997), the third method Sec. 4
 * names; no listing in the paper, so the recurrence is GPBiCG on the Kronecker system
 * (eq. 1.2) in the matrix operations of Sec. 2 (R~_0 = R_0; zeta, eta minimising
 * ||T - zeta L(T) - eta Y|| with eta = 0 in the first step), factorized as Algorithm 4.2
 * is: the same block Arnoldi bases (two steps per iteration), additions of padded small
 * matrices (eq. 3.5), inner products of small matrices (eq. 3.6), two applications of the
 * small operator of eq. 3.7 per iteration.  General A, B; returns V_{2k+2}, X^_{k+1},
 * W_{2k+2} as sylv_bicgstab.  Batched handles: SYLV_EINVAL.  Otherwise as sylv_cg.
 */
int sylv_gpbicg(sylv_handle* h, double tol, int32_t maxit, sylv_info* info);

/*
 * Copies the factors of the last solve: V (n x r), X^ (r x r), W (m x r),
 * column-major, float64.  Any of V, Xhat, W may be NULL to skip it; *r
 * receives r (the call with all three NULL only queries r).  In the Lyapunov
 * case W equals V.  Errors: SYLV_ESTATE (no solve yet), SYLV_ECUDA.
 */
int sylv_get_factors(sylv_handle* h, double* V, double* Xhat, double* W, int64_t* r);

/*
 * Final low-rank compression of the last solve's X = V X^ W^T (float64 BiCGSTAB, CGS or
 * GPBiCG, whose block Arnoldi bases are orthonormal; deflated zero columns allowed).  The
 * paper has no counterpart (its methods return the factors as built).  Computes the
 * SVD X^ = U S Z^T on the device (one-sided Jacobi) and keeps the smallest rank q whose
 * discarded singular values have norm <= tol * ||X||_F -- the best rank-q approximation,
 * ||X - X_q||_F = that norm.  Afterwards sylv_get_factors returns V U_q (n x q), diag(s_q)
 * and W Z_q (m x q) until the next solve; *q receives q.
 * Errors: SYLV_EINVAL (mixed or Lanczos solves, refinement rounds, batched handles, tol < 0),
 * SYLV_ESTATE (no solve yet, or already compressed), SYLV_ENOMEM, SYLV_ENOTCONV (the Jacobi
 * iteration did not converge in 100 sweeps), SYLV_ECUDA.
 */
int sylv_compress(sylv_handle* h, double tol, int64_t* q);

/*
 * Residual history of the last solve: hist[0] = 1, hist[k] = ||R^_k||/||R^_0||.
 * Writes min(cap, len) values; *len receives the full length (hist may be NULL).
 */
int sylv_get_history(sylv_handle* h, double* hist, int64_t cap, int64_t* len);

/*
 * Block Hessenberg matrix of one basis from the last solve (eq. 3.4,
 * A V_k = V_{k+1} H_{k+1,k}): side 0 -> H of (A, C1), side 1 -> G of (B^T, C2).
 * Copies the leading rows x cols part (column-major, leading dimension rows)
 * with rows = (nblocks) s and cols = (nblocks - 1) s; *nblocks receives the
 * number of basis blocks built.  H may be NULL to query nblocks.
 */
int sylv_get_hessenberg(sylv_handle* h, int32_t side, double* H, int64_t cap, int32_t* nblocks);

/*
 * Sparse block product through the solver's SpMM kernel (the sparse apply of
 * eq. 3.4): Y = Op X with Op = A (side 0) or B^T (side 1), X and Y column-major
 * (rows x k), 1 <= k <= 8, host memory.  Runs in the handle's precision.
 */
int sylv_apply(sylv_handle* h, int32_t side, const double* X, double* Y, int64_t k);

/*
 * The factored Sylvester operator of eq. 3.7 on the bases of the last solve:
 *   out = [H Z, 0] + [Z G^T; 0]
 * with H = H_{k+1,k}, G = G_{k+1,k} ((r + s) x r leading parts of the Hessenberg matrices of
 * eq. 3.4, G = H for the Lyapunov case) and Z r x r; the same device path the solver uses (the
 * BiCGSTAB-type methods' dense operator: tensor cores from order 448 on unless
 * sylv_options.small_gemm says otherwise; double-float products in SYLV_MIXED).
 *   r    a positive multiple of s, at most (nblocks - 1) s of the last solve
 *   Z    r x r column-major (host);  out  (r + s) x (r + s) column-major (host)
 * The call uses the handle's small-matrix work space (the factors of the last solve are kept).
 * Errors: SYLV_EINVAL (r, NULL pointers, batched handle), SYLV_ESTATE (no solve yet),
 * SYLV_ENONFINITE, SYLV_ETIMEOUT, SYLV_ECUDA.
 */
int sylv_small_operator(sylv_handle* h, int64_t r, const double* Z, double* out);

/*
 * Sets the host wait limit of the handle's later solves (sylv_options.timeout_s;
 * 0: 3600 s).  A solve that runs past it returns SYLV_ETIMEOUT without waiting
 * for the kernels it enqueued; they finish on the device, and every later call
 * on the handle is ordered after them, so the handle stays usable.
 * Errors: SYLV_EINVAL (NULL handle, negative or NaN limit).  Not in the paper.
 */
int sylv_set_timeout(sylv_handle* h, double timeout_s);

/*
 * Kernel timing of the last solve, one entry per kernel class (only with
 * sylv_options.profile = 1; otherwise *count = 0).  Writes min(cap, count)
 * entries to out (may be NULL to query count).
 */
int sylv_get_profile(sylv_handle* h, sylv_kernel_stat* out, int32_t cap, int32_t* count);

/* Largest n * k accepted by sylv_spmm_noalloc: the size, in doubles, of its
 * fixed staging area for X (the same again is reserved for Y, 16 MiB in all). */
#define SYLV_NOALLOC_MAX_ELEMS (1 << 20)

/*
 * Y = A X without allocating device memory: the sparse block product of
 * sylv_apply for callers that cannot call cudaMalloc -- processes whose device
 * memory is owned by another allocator (for example a framework's caching pool
 * holding the device memory budget) and latency-bound loops that cannot afford
 * the device-wide synchronisation cudaMalloc/cudaFree may cause.  The paper has
 * no counterpart; this is a library facility.
 *   n, nnz, row_ptr, col_idx, val   A (n x n) in CSR form, all DEVICE pointers
 *   X, Y                            DEVICE pointers, n x k column-major; 1 <= k <= 8
 * Every pointer must be device (or managed) memory of the CURRENT device; a host
 * pointer or another device's memory returns SYLV_EINVAL (checked with
 * cudaPointerGetAttributes, which allocates nothing).
 *   cuda_stream                     cudaStream_t (NULL: the legacy default stream)
 * Float64.  Asynchronous: returns once the kernels are enqueued on cuda_stream;
 * launch errors are returned, errors inside the kernels surface at the caller's
 * next synchronisation.  The inputs and outputs stay owned by the caller.
 * Staging uses one fixed device array compiled into the library (every GPU that
 * loads it holds 16 MiB until the process exits).  Limits and rules:
 *  - n * k > SYLV_NOALLOC_MAX_ELEMS returns SYLV_EINVAL (use sylv_apply);
 *  - the first call on each device looks up the array's device address with
 *    cudaGetSymbolAddress (with that device current); make that first call
 *    before any stream capture;
 *  - that address belongs to the device's primary context: after
 *    cudaDeviceReset do not call this entry point again in the same process;
 *  - every call, on every stream, shares the one array: calls that can overlap
 *    on the GPU (different streams without ordering) race and corrupt each
 *    other's results; order them on one stream or with events.
 * Errors: SYLV_EINVAL (arguments, size limit, pointer not on the current
 * device), SYLV_ECUDA (a launch failed, or a CUDA error left pending by earlier
 * work, which is reported and left set rather than cleared).
 */
int sylv_spmm_noalloc(int64_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx, const double* val,
                      const double* X, double* Y, int64_t k, void* cuda_stream);

const char* sylv_strerror(int status);
const char* sylv_last_error(void);
void sylv_destroy(sylv_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* SYLV_H_ */
