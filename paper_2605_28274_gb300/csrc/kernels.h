// Host-side launchers of the solver kernels (internal to libsylv).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "common.cuh"

namespace sylv {

// Kernels enqueued by the calling host thread.  Every launch passes its grid through
// counted(), so sylv_info.kernel_launches is a count of actual launches.
int64_t& launch_counter();
template <typename G>
inline G counted(G grid) {
  ++launch_counter();
  return grid;
}

// ---------------------------------------------------------------- float64 basis products on the tensor cores
// (kernels_obasis.cu) The Arnoldi basis of one side as five FP16 planes of 11-bit digits, in a
// Gram layout and an update layout, plus the digits of the block being orthogonalised (Y) and
// of the coefficient block, and the column exponents.  One allocation of ob_side_bytes().
struct ObSide {
  uint16_t* G = nullptr;   // basis digit planes, Gram layout
  uint16_t* U = nullptr;   // basis digit planes, update layout
  uint16_t* YB = nullptr;  // digits of Y
  uint16_t* HB = nullptr;  // digits of the coefficient block
  int* vexp = nullptr;     // exponents of the basis columns
  int* ey = nullptr;       // exponents of the columns of Y
  int* eh = nullptr;       // exponents of the columns of the coefficient block
  // column maxima of |x| as IEEE bits, [0, 8) the new basis block (from the last CholQR scale),
  // [8, 16) Y (from the SpMM and the first update); the coefficient-block split zeroes both
  unsigned long long* mx = nullptr;
  int64_t np = 0;          // basis rows padded to 128
  int rp = 0;              // basis columns padded to 128
  int64_t plane = 0;       // elements per digit plane
};
size_t ob_side_bytes(int64_t n, int R, int s);
void ob_carve(void* mem, int64_t n, int R, int s, ObSide& o);
bool ob_setup();
// Digits of the new basis block Vb (n x s row-major; basis columns col0 .. col0 + s - 1), whose
// column maxima the last CholQR scale left in mx[0, 8).
void launch_ob_split_basis(cudaStream_t, const DevState*, int64_t n, int s, const double* Vb, int col0, const ObSide&);
// Per-split partial Gram products V^T Y over the first js basis columns (the partial layout of
// launch_gram), Y's column maxima in mx[8, 16); returns the number of splits.
int launch_ob_gram(cudaStream_t, DevState*, int64_t n, int s, int js, const double* Y, const ObSide&, double* partial);
// Y -= V Hc over the first js basis columns (Hc: js x s, the layout launch_reduce_H writes),
// with the optional per-CTA partial Y^T Y of the result and, with ymax, the column maxima of
// the result into mx[8, 16); V enters through its leading `planes` digit planes (5: all).
// Returns the number of CTAs.
int launch_ob_update(cudaStream_t, DevState*, int64_t n, int s, int js, const double* Hc, double* Y, const ObSide&,
                     double* self_partial, bool ymax, int planes, bool split_done = false);
// H_{1:j,j} (+)= the sum of the ncta Gram partials (the partial layout of launch_ob_gram), also
// into Hc, and the digits of Hc for the next launch_ob_update (split_done = true) in the last CTA
// of the same launch.  side: 0 or 1 (each side's launches count on their own ticket).
void launch_ob_reduce_H(cudaStream_t, DevState*, int side, const double* partial, int ncta, int nb, int s, double* H,
                        int64_t ldh, int64_t row0, int64_t col0, double* Hc, bool add, const ObSide&);

// Products of the float64 true-residual certificate on a side's digit planes (float64-accurate
// like the basis kernels).  o: the side's ObSide with YB, HB, ey, eh, mx replaced by scratch of
// ob_cols_scratch_bytes(rows, basis columns, s) bytes carved by ob_cols_carve (the operands here
// have s columns, not the basis block width).
size_t ob_cols_scratch_bytes(int64_t n_max, int R_max, int s);
void ob_cols_carve(void* mem, int64_t n_max, int R_max, int s, ObSide& o);
// P[m ldp + col0 + t] = (V^T Y)(m, t) over the first js basis columns; Y n x s with row stride ldy.
// partial: scratch of (number of SMs) x js x s doubles.  Returns the number of k splits.
int launch_ob_gram_cols(cudaStream_t, DevState*, int64_t n, int s, int js, const double* Y, int64_t ldy,
                        const ObSide&, double* partial, double* P, int64_t ldp, int col0);
// Z (n x s, row stride ldz) += V Hc over the first js basis columns (Hc js x s row-major).
void launch_ob_update_cols(cudaStream_t, DevState*, int64_t n, int s, int js, const double* Hc, double* Z, int64_t ldz,
                           const ObSide&);

// out[0, count) ~ N(0, 1): SplitMix64 from seed and Box-Muller (counter-based, one thread per pair).
void launch_gauss_probes(cudaStream_t, double* out, size_t count, uint64_t seed);
// Digit planes (both layouts) and column exponents of all nb blocks of a basis already built
// (float32 or float64 elements), for the true-residual certificate's products; mx_all: scratch
// of nb * s column maxima.  o: carved by ob_carve for at least nb * s columns.
void launch_ob_split_bases(cudaStream_t, int64_t n, int s, int nb, const void* V, bool is_float, int64_t bstride,
                           unsigned long long* mx_all, const ObSide& o);

// Sets the message returned by sylv_last_error() on the calling thread.
void set_last_error(const std::string& msg);

// ---------------------------------------------------------------- basis side
// All factor blocks are stored block-row-major: block b is an n x s row-major
// array at V + b * bstride (bstride = n * s elements).

// Y = Op X (- Xprev M): CSR SpMM over an s-wide block; the optional term is the
// three-term recurrence of block Lanczos (M = H_{j-1,j}, s x s, column-major ld ldm).
template <typename T>
void launch_spmm(cudaStream_t, const DevState*, int64_t n, int s, const int32_t* rp, const int32_t* ci,
                 const T* val, const T* X, T* Y, const T* Xprev, const double* M, int64_t ldm,
                 unsigned long long* colmax = nullptr);

// Per-CTA partial Gram products  P_c = sum over the CTA's rows of V_b^T Y  for
// blocks b = 0..nb-1 (V points at the first block), written in the factor precision T
// into the (double-sized) partial buffer.  Returns the number of CTAs.
template <typename T>
int launch_gram(cudaStream_t, const DevState*, int64_t n, int s, const T* V, int64_t bstride, int nb,
                const T* Y, double* partial);

// Sum the partials in a fixed order: Hc[e] = sum_c partial[c][e], e < nb*s*s, and
// store (add) the nb*s x s result into H at (row0, col0) (column-major, ld ldh).
void launch_reduce_H(cudaStream_t, const DevState*, const double* partial, int ncta, int nb, int s, double* H,
                     int64_t ldh, int64_t row0, int64_t col0, double* Hc, bool add, bool float_partials);

// Y -= [V_0 .. V_{nb-1}] Hc  (Hc: nb*s x s row-major).  With self_partial != NULL also
// writes per-CTA partials of Y^T Y.  Returns the number of CTAs.
template <typename T>
int launch_update(cudaStream_t, const DevState*, int64_t n, int s, const T* V, int64_t bstride, int nb,
                  const double* Hc, T* Y, double* self_partial);

// Per-CTA partials of Y^T Y.  Returns the number of CTAs.
template <typename T>
int launch_selfgram(cudaStream_t, const DevState*, int64_t n, int s, const T* Y, double* self_partial);

// Arguments of one Cholesky pass of CholQR2 on the s x s Gram reduced from the partials.
struct CholArgs {
  int side;           // 0: A basis, 1: B^T basis (exhaustion flag slot)
  int pass;           // 1 or 2
  int s;
  double delta;       // exhaustion / rank-loss threshold
  const double* Hcol; // pass 1: projection coefficients of this step (column block), or NULL
  int64_t ldh, hrows; // rows of Hcol to include in nu
  double* R1;         // pass 1 writes R1 here; pass 2 reads it
  double* Rinv;       // s x s inverse of this pass's R (float64)
  void* RinvT;        // same in the factor precision
  int factor_is_float;
  double* Hsub;       // pass 2: H_{j+1,j} = R2 R1 stored here (ld ldh), or NULL
  double* Hsup;       // pass 2, Lanczos: H_{j,j+1} = (R2 R1)^T stored here, or NULL
  double* Rout;       // pass 2: R2 R1 also stored here (s x s, ld s), or NULL
  int setup;          // QR of C1/C2: any loss of rank is a breakdown
};
// One CholQR pass in one launch: Cholesky of the s x s Gram summed from partial_in (ncta_in
// Gram partials) in every CTA, then Y <- Y R^{-1} over the n x s block, with the
// optional per-CTA partial Y^T Y of the result into partial_out (a different buffer from
// partial_in, at least 2 x SMs x s^2 doubles) and column maxima into colmax.  The factors are
// stored by CTA 0 as the fields of CholArgs say.  Returns the number of CTAs (the partial_out count).
template <typename T>
int launch_cholscale(cudaStream_t, DevState*, const double* partial_in, int ncta_in, const CholArgs&, int64_t n, T* Y,
                     double* partial_out, unsigned long long* colmax);

// Copy a column-major n x s float64 matrix into block-row-major factor storage.
template <typename T>
void launch_pack(cudaStream_t, int64_t n, int s, const double* Ccol, T* Vblk);
// Block-row-major factors (nb blocks) -> column-major n x (nb s) float64.
template <typename T>
void launch_unpack(cudaStream_t, int64_t n, int s, int nb, const T* Vblk, int64_t bstride, double* Vcol);
// Element-wise float64 -> T conversion.
template <typename T>
void launch_convert(cudaStream_t, int64_t count, const double* src, T* dst);

// ---------------------------------------------------------------- small side (float64)
// Small matrices are column-major with a fixed leading dimension lds, zero outside
// their extent, so the zero padding of Algorithms 4.1/4.2 costs nothing.
struct SmallCtx {
  DevState* st;
  double* hist;  // residual history
  int s;
  int64_t lds;
  double *Xh, *Rh, *Ph, *Qh, *Sh, *Th, *Rt;  // Rt: shadow residual R~_0 (s x s, ld s)
  double* Uh;                                // CGS, GPBiCG: U^
  double *gW, *gZ, *gTp, *gY;                // GPBiCG only: W^, Z^, T_prev^, Y^
  double* gPart;                             // GPBiCG: 5 x GP_ZETA_CTAS partials of the zeta/eta step
  const double* H;  // A-side block Hessenberg (ld ldh)
  const double* G;  // B^T-side (== H in the Lyapunov case)
  int64_t ldh;
  double* partials;  // per-CTA scratch for the fused reductions
  int lyapunov;
  int df_small;      // 1: the dense factored operator runs in double-float on the FP32 pipes
  // df_small only: hi/lo float pairs of H, G (ld ldh; Gs == Hs in the Lyapunov case) and of
  // the operand Z (ld lds); *split_cols = columns of H and G already split in this solve
  void *Hs, *Gs, *Zs;
  int* split_cols;
  // tensor-core products (Ozaki splitting) for operand orders r >= oz_min_r; oz_scratch holds
  // ozaki_scratch_bytes(ldh) bytes (null: never)
  void* oz_scratch;
  int oz_min_r;
};

// R^_0 = R_L R_R^T, P^_0 = R^_0, R~_0 = R^_0, rho_0, ||R^_0||, history[0] = 1.
void launch_init_small(cudaStream_t, const SmallCtx&, const double* RL, const double* RR, double tol, bool cgs);

// Algorithm 4.1 pieces.  cg_q: mode 0 Q^ = [H P^, 0] + [P^ G^T; 0]; mode 1 M = [H P^, 0]
// (Lyapunov, into the T^ buffer); mode 2 Q^ = M + M^T.  Modes 0/2 also set alpha.
void launch_cg_q(cudaStream_t, const SmallCtx&, int mode, int r);
// X^ += alpha P^, R^ -= alpha Q^, residual test, rho, beta (extent r -> r+s).
void launch_cg_update(cudaStream_t, const SmallCtx&, int k, int r, bool cr = false);
// P^ = R^ + beta P^ over extent rp.
void launch_cg_p(cudaStream_t, const SmallCtx&, int rp);

// Algorithm 4.2 pieces.  Out = [H Z, 0] + [Z G^T; 0] with Z of extent r (block upper
// Hessenberg H, G); with omega also reduces <Out(1:r,1:r), Z>, <Out, Out> and sets omega.
// Returns the number of kernels launched.
int launch_sylv_gemm(cudaStream_t, const SmallCtx&, int r, const double* Z, double* Out, bool omega);
// Final low-rank compression (compress.cu): one-sided Jacobi SVD of the r x r core and the
// products of the block-stored bases with the kept singular vectors.
void jacobi_schedule(int r, std::vector<int>& pairs);  // (r2 - 1) rounds x r2 entries, r2 = r + r % 2
int launch_jacobi_round(cudaStream_t, int r, double* G, double* Z, int64_t ld, const int* pairs_round, double eps,
                        double tau, int* rotated);
void launch_column_norms(cudaStream_t, int r, const double* G, int64_t ld, double* s);
void launch_apply_blocks(cudaStream_t, int64_t rows, int su, int r, const double* V, int64_t bstride,
                         const double* M, int64_t ldm, const int* cols, const double* scale, int q, double* Out);

// The same operator in float64 accuracy on the tcgen05 tensor cores (kernels_ozaki.cu).
size_t ozaki_scratch_bytes(int rmax);
bool ozaki_setup();  // once per device: opt-in to the kernel's shared-memory size
int launch_sylv_gemm_ozaki(cudaStream_t, DevState* st, int r, int s, const double* H, const double* G, int64_t ldh,
                           const double* Z, double* Out, int64_t lds, bool omega, void* scratch);
double sylv_gemm_flops(int r, int s);
void launch_bicg_alpha(cudaStream_t, const SmallCtx&);
// Factorized CGS (Sec. 4 names it; same bases and operator as Algorithm 4.2): with V^ = L(P^)
// in Qh and alpha from launch_bicg_alpha, cgs_q forms Q^ (in Qh), W^ = U^ + Q^ (in Th) and
// X^ += alpha W^ (extent rp); with T^ = L(W^) in Sh, cgs_update forms R^ -= alpha T^, the
// test and beta (extent rpp); cgs_p forms U^ and P^.
void launch_cgs_q(cudaStream_t, const SmallCtx&, int rp);
// Factorized CR (Sec. 4 names it; block Lanczos bases as Algorithm 4.1): cr_op applies the
// operator to R^ (extent r -> r+s) into the S^ buffer and sets rho = <R^, L(R)^> (first) or
// beta and rho; cr_p forms P^ and L(P)^ (in the Q^ buffer, extent rpp) and alpha.  The update
// of X^, R^ and the test is launch_cg_update(.., cr = true) with L(P)^ in place of Q^.
void launch_cr_op(cudaStream_t, const SmallCtx&, int mode, int r, bool first);
// Factorized GPBiCG (Sec. 4 names it; same bases and operator as Algorithm 4.2).  With
// e1 = (2k+1)s, e2 = e1 + s: gp_p forms P^ (e1); the operator gives L(P)^ in Qh and
// launch_bicg_alpha alpha; gp_ty forms Y^ (gY) and T^ (Th) (e2); the operator gives L(T)^ in
// Sh; gp_zeta the five inner products, zeta and eta; gp_update U^, Z^, X^, R^, the test and
// beta; gp_w W^ and T_prev^ (e3).
constexpr int GP_ZETA_CTAS = 1024;
void launch_gp_p(cudaStream_t, const SmallCtx&, int e1);
void launch_gp_ty(cudaStream_t, const SmallCtx&, int e2);
void launch_gp_zeta(cudaStream_t, const SmallCtx&, int k, int e2);
void launch_gp_update(cudaStream_t, const SmallCtx&, int k, int e2);
void launch_gp_w(cudaStream_t, const SmallCtx&, int e3);
void launch_cr_p(cudaStream_t, const SmallCtx&, int rpp);
void launch_cgs_update(cudaStream_t, const SmallCtx&, int k, int rpp);
void launch_cgs_p(cudaStream_t, const SmallCtx&, int rpp);
void launch_bicg_s(cudaStream_t, const SmallCtx&, int rp);
void launch_bicg_update(cudaStream_t, const SmallCtx&, int k, int rp, int rpp);
void launch_bicg_p(cudaStream_t, const SmallCtx&, int rpp);

// ---------------------------------------------------------------- true residual (float64 accumulation)
// P (nb*su x k, row-major) = U^T Y with U in block-row-major storage (nb blocks of width su,
// element TU) and Y n x k row-major float64, k <= 16.  partial: scratch of at least
// tsg_partial_elems(nb*su, k) doubles (max_rc > 0 caps the row chunks).
int64_t tsg_partial_elems(int64_t ncol, int k);
template <typename TU>
void launch_tsg(cudaStream_t, int64_t n, const TU* U, int64_t bstride, int su, int nb, const double* Y, int k,
                double* partial, int max_rc, double* P);
// Z = beta Z + alpha U M  (U as above, M nb*su x k row-major, Z n x k row-major).
template <typename TU>
void launch_tsu(cudaStream_t, int64_t n, const TU* U, int64_t bstride, int su, int nb, const double* M, int k,
                double alpha, double beta, double* Z);
// out (r x k row-major) = op(Xh) in, op = Xh or Xh^T (Xh column-major, ld lds).
void launch_small_apply(cudaStream_t, int r, int k, const double* Xh, int64_t lds, bool trans, const double* in,
                        double* out);
// Y = alpha Y + C G (C n x s row-major, G s x k row-major, Y n x k row-major).
void launch_lowrank_axpy(cudaStream_t, int64_t n, int s, int k, const double* C, const double* G, double alpha,
                         double* Y);
// out (rows x 16) = [a | b], and back (a, b rows x 8; all row-major).
void launch_interleave(cudaStream_t, int64_t rows, const double* a, const double* b, double* out);
void launch_deinterleave(cudaStream_t, int64_t rows, const double* in, double* a, double* b);
// y += a x element-wise.
void launch_axpy(cudaStream_t, int64_t count, double a, const double* x, double* y);
// out = -(X1 + X2) element-wise.
void launch_neg_sum(cudaStream_t, int64_t count, const double* X1, const double* X2, double* out);
// out[0] = sum of squares of x (deterministic; ticket must be zero).
void launch_sumsq(cudaStream_t, int64_t count, const double* x, double* partials, unsigned int* ticket, double* out);
// out[0] = trace(G1 G2) for s x s matrices.
void launch_trace_prod(cudaStream_t, int s, const double* G1, const double* G2, double* out);

// ---------------------------------------------------------------- batched Lyapunov CG
// One entry per instance (device array).  All buffers belong to the instance's own
// handle; the batched phase kernels below walk every active instance in one launch
// and read the iteration index k from here, so one CUDA graph serves every iteration.
struct BatchInst {
  int64_t n;
  int s, k;             // block width; current iteration (advanced on the device)
  const int32_t* rp;
  const int32_t* ci;
  const double* val;    // CSR of A (float64)
  double* V;            // basis blocks (n x s row-major each)
  double* H;            // block tridiagonal Lanczos matrix, dense column-major (ld ldh)
  int64_t ldh;
  double *X, *R, *P, *Q, *M;  // small matrices (ld lds); M = [H P^, 0]
  int64_t lds;
  DevState* st;
  double* hist;
  double *R1, *Rinv;    // CholQR scratch (s x s)
  double* psm;          // per-tile partial sums of the small phases
  int item_begin, item_end;  // this instance's (row chunk) work items
};

struct BatchCtx {
  BatchInst* insts;     // device array
  int count;
  const int2* items;    // (instance, first row) per row-chunk work item
  int nitems;
  int chunk;            // rows per work item (autotuned)
  int grid;             // CTAs of the persistent row phases (autotuned)
  double* gpart;        // [nitems][64] Gram partials
  double* spart;        // [nitems][64] self-Gram partials
  double delta;
  int* running;         // device counter of instances still running
  int sgrid;            // CTAs of the persistent small-matrix phases
};

// The 15 phases of one factorized-CG (Lyapunov) iteration over all instances.
void launch_batch_iteration(cudaStream_t, const BatchCtx&);
// Only the sparse-apply and Gram phases (for the autotuner).
void launch_batch_spmm_gram(cudaStream_t, const BatchCtx&);

}  // namespace sylv
